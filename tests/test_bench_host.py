"""bench.py's host-side bookkeeping on CPU: the committed per-launch DRAM
traffic is used only while the kernel's sources hash as they did when it was
captured, and the nvidia-smi clock log is parsed into the median SM clock and
the throttle reasons seen."""
import json
import os
import shutil
import subprocess
import sys
import tempfile
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _copy_tree(tmp_path):
    """A throwaway copy of what the traffic lookup reads."""
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "profiles"), root / "profiles")
    shutil.copytree(os.path.join(ROOT, "paper_1711_03888_gb300", "csrc"), root / "paper_1711_03888_gb300" / "csrc",
                    ignore=shutil.ignore_patterns("*.o", "*.so"))
    return root


def test_traffic_entries_follow_the_committed_sources():
    """An entry gives its captured traffic exactly while its kernel's sources
    hash as recorded, and nothing once they have changed."""
    import hashlib
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    kernels = [k for k in d if not k.startswith("_")]
    assert kernels
    for k in kernels:
        h = hashlib.sha256()
        for f in d[k]["sources"]:
            h.update(open(os.path.join(ROOT, "paper_1711_03888_gb300", "csrc", f), "rb").read())
        t = bench._traffic(k)
        if h.hexdigest()[:16] == d[k]["sources_sha256_16"]:
            assert t == pytest.approx(d[k]["dram_read"] + d[k]["dram_write"])
        else:
            assert t is None, f"{k}: traffic used after its sources changed"
    assert bench._traffic("no_such_kernel") is None


def test_traffic_is_dropped_once_a_source_changes(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    import hashlib
    d = json.load(open(root / "profiles" / "traffic.json"))
    k = next(k for k in d if not k.startswith("_"))
    # pin the entry to the copy's current sources, so it is in use to begin with
    h = hashlib.sha256()
    for f in d[k]["sources"]:
        h.update((root / "paper_1711_03888_gb300" / "csrc" / f).read_bytes())
    d[k]["sources_sha256_16"] = h.hexdigest()[:16]
    (root / "profiles" / "traffic.json").write_text(json.dumps(d))
    assert bench._traffic(k) is not None
    src = root / "paper_1711_03888_gb300" / "csrc" / d[k]["sources"][-1]
    src.write_bytes(src.read_bytes() + b"\n// edited\n")
    assert bench._traffic(k) is None
    # a missing or unreadable table gives no traffic either
    (root / "profiles" / "traffic.json").write_text("{")
    assert bench._traffic(k) is None
    os.unlink(root / "profiles" / "traffic.json")
    assert bench._traffic(k) is None


_NCU_CSV_HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
                   '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')


def _ncu_row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python","h","{kernel}","1","7","(256, 1, 1)","(456, 6, 1)","0","10.3",'
            f'"Command line profiler metrics","{metric}","{unit}","{value}"')


def test_write_traffic_from_an_ncu_log(tmp_path, monkeypatch):
    """--write-traffic averages each kernel's launches, converts ncu's units,
    pins the current source hashes, and an "a + b" name sums both kernels."""
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    sizes = "void szg::(anonymous namespace)::encode_sizes_multi_kernel<4096>(szg::MultiArgs)"
    pack = "void szg::(anonymous namespace)::encode_pack_multi_kernel<4096>(szg::MultiArgs)"
    rows = [_NCU_CSV_HEADER]
    for i, (k, rd, wr, us) in enumerate([(sizes, "1,600,000,000", "0.001", 430.0),
                                         (pack, "1,500,000,000", "1.0", 1400.0),
                                         (pack, "1,700,000,000", "1.2", 1600.0)]):
        rows += [_ncu_row(i, k, "dram__bytes_read.sum", "byte", rd),
                 _ncu_row(i, k, "dram__bytes_write.sum", "Gbyte", wr),
                 _ncu_row(i, k, "gpu__time_duration.sum", "usecond", us)]
    log = tmp_path / "launches.csv"
    log.write_text("==PROF== a line before the table\n" + "\n".join(rows) + "\n")
    out = bench.write_traffic(str(log), "ncu --metrics ...")
    assert set(k for k in out if not k.startswith("_")) == {"encode_sizes_multi_kernel", "encode_pack_multi_kernel"}
    p = out["encode_pack_multi_kernel"]
    assert p["launches_captured"] == 2
    assert p["dram_read"] == pytest.approx(1.6e9) and p["dram_write"] == pytest.approx(1.1e9)
    assert p["ncu_duration_ns"] == pytest.approx(1.5e6)
    assert bench._traffic("encode_pack_multi_kernel") == pytest.approx(2.7e9)
    assert bench._traffic("encode_sizes_multi_kernel + encode_pack_multi_kernel") == pytest.approx(2.7e9 + 1.601e9)
    r = bench.ncu_dram_rate("encode_sizes_multi_kernel + encode_pack_multi_kernel", 1000.0)
    assert r["duration_ms"] == pytest.approx(1.93)
    # a part that is missing leaves the sum unknown
    assert bench._traffic("encode_pack_multi_kernel + decode_multi_kernel") is None


def _fake_log(lines):
    """A ClockSampler on its nvidia-smi path, fed by a process that prints
    `lines` in nvidia-smi's CSV form and then waits to be terminated."""
    s = bench.ClockSampler(0)
    s.f = tempfile.NamedTemporaryFile("w", prefix="sz_clocks_", suffix=".csv", delete=False)
    s.path = s.f.name
    script = "".join(f"echo '{ln}'; " for ln in lines) + "sleep 30"
    s.proc = subprocess.Popen(["bash", "-c", script], stdout=s.f)
    deadline = time.time() + 10
    while os.path.getsize(s.path) < sum(len(ln) + 1 for ln in lines) and time.time() < deadline:
        time.sleep(0.02)
    return s


def test_clock_log_median_and_reasons():
    lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _fake_log(lines)
    path = s.path
    r = s.stop()
    assert r["source"] == "nvidia-smi"
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(path)


def test_clock_log_reports_every_slowdown_reason():
    lines = ["0, 1200, 2070, 500, 0x68, Active, Active, Active, Not Active"]
    r = _fake_log(lines).stop()
    assert r["sm_mhz"] == 1200.0
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_unsampled_clocks_say_so():
    s = bench.ClockSampler(0)
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_ncu_dram_rate_from_the_committed_capture(tmp_path, monkeypatch):
    import hashlib
    root0 = _copy_tree(tmp_path / "pinned")
    monkeypatch.setattr(bench, "ROOT", str(root0))
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for k in (k for k in d if not k.startswith("_")):      # entries pinned to the copy's sources
        h = hashlib.sha256()
        for f in d[k]["sources"]:
            h.update((root0 / "paper_1711_03888_gb300" / "csrc" / f).read_bytes())
        d[k]["sources_sha256_16"] = h.hexdigest()[:16]
    (root0 / "profiles" / "traffic.json").write_text(json.dumps(d))
    for k in (k for k in d if not k.startswith("_")):
        r = bench.ncu_dram_rate(k, 1000.0)
        b = d[k]["dram_read"] + d[k]["dram_write"]
        assert r["dram_bytes"] == pytest.approx(b)
        assert r["dram_gbs"] == pytest.approx(b / d[k]["ncu_duration_ns"])
        assert r["dram_frac"] == pytest.approx(r["dram_gbs"] / 1000.0)
        assert r["duration_ms"] == pytest.approx(d[k]["ncu_duration_ns"] / 1e6)
    k = next(k for k in d if not k.startswith("_"))
    src = root0 / "paper_1711_03888_gb300" / "csrc" / d[k]["sources"][0]
    src.write_bytes(b"// edited\n" + src.read_bytes())
    assert bench.ncu_dram_rate(k, 1000.0) is None
