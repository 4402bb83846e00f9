"""Benchmark of the SZ-LV hot path on GB300.

Workload (default): the large cosmology snapshot -- 2^27 particles, six
float32 fields (3.2 GB), relative error bound 1e-4, 4096 halos.  One step is
the whole hot path: compress the six arrays (range, quantize + histogram,
codebook, encode) and decompress the six streams (decoder setup, decode), all
on device-resident data.  Inputs (3.2 GB) exceed the 129 MB L2, so no flush is
needed between steps.

value       = uncompressed bytes / step time (compress + decompress), all ranks.
e2e         = the same round trip through the C ABI's host-memory calls
              (sz_compress_host, sz_decompress_host) on pinned host buffers:
              H2D inputs, compress, D2H streams, H2D streams, decompress,
              D2H outputs, all inside the timed region (the library overlaps
              the copies of one group of arrays with the kernels of another).
roofline    = the dominant kernel's algorithmic bytes per launch over its
              average launch time (CUDA events on its stream, inside the
              timed region), against the measured HBM copy bandwidth.
cpu_baseline= the CPU oracle on a bounded sample of the same arrays.

Multi-GPU: one process per GPU (torchrun); each rank compresses its own
snapshot (independent seeds, no collective on the data path; weak scaling).
`--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FIELDS = ("xx", "yy", "zz", "vx", "vy", "vz")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """SM clock and clock-event reasons during a region, read (never set)
    through NVML by a sampling thread every 5 ms; nvidia-smi if NVML cannot be
    loaded."""

    # nvmlClocksEventReasons bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self.stop_flag = threading.Event()
        self.thread = None
        self.proc = None

    def _nvml(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit")
        h = C.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(self.index, C.byref(h)) != 0:
            raise OSError("nvml handle")
        mx = C.c_uint(0)
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx)) == 0:     # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        return lib, h, get_reasons

    def _loop(self, lib, h, get_reasons):
        import ctypes as C
        clk, rs = C.c_uint(0), C.c_ulonglong(0)
        while not self.stop_flag.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0:
                self.samples.append(float(clk.value))
            if get_reasons(h, C.byref(rs)) == 0:
                for bit, name in self.REASONS.items():
                    if rs.value & bit:
                        self.reasons.add(name)
            time.sleep(0.005)

    def start(self):
        try:
            lib, h, get_reasons = self._nvml()
            self.thread = threading.Thread(target=self._loop, args=(lib, h, get_reasons), daemon=True)
            self.thread.start()
            return
        except Exception:
            self.thread = None
        try:
            self.f = tempfile.NamedTemporaryFile("w", prefix="sz_clocks_", suffix=".csv", delete=False)
            self.path = self.f.name
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            sm = sorted(self.samples)
            return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": self.max_mhz,
                    "reasons": sorted(self.reasons), "samples": len(sm), "source": "nvml"}
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "source": "nvidia-smi"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_over_ranks(v: float, ws: int, op: str) -> float:
    """All-reduce of one host scalar (timing bookkeeping only; the data path
    has no collective).  NCCL reduces a CUDA tensor, gloo a CPU one."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _max_over_ranks(v: float, ws: int) -> float:
    return _reduce_over_ranks(v, ws, "max")


def _sum_over_ranks(v: float, ws: int) -> float:
    return _reduce_over_ranks(v, ws, "sum")


def rank_snapshot_seed(rank: int) -> int:
    """Weak scaling: rank r compresses its own snapshot, generated with seed
    3 + r (independent data, the same size on every rank)."""
    return 3 + rank


def weak_scaling_value(bytes_per_rank: float, seconds_per_step: float, ws: int):
    """Whole-job throughput: all ranks' bytes over the slowest rank's step
    time.  Returns (GB/s, max step seconds, total bytes)."""
    t = _max_over_ranks(seconds_per_step, ws)
    b = _sum_over_ranks(bytes_per_rank, ws)
    return b / t / 1e9, t, b


RD_EBS = (1e-2, 1e-3, 1e-4, 1e-5, 1e-6)


def rd_points(sz, ctx, xs, ebs=RD_EBS, params=None, md_mode=None):
    """Rate-distortion points (Fig. 9) of one snapshot's fields xs (float32
    CUDA tensors) at value-range-relative bounds `ebs`: bits per value (all
    fields' stream bits over all values) and PSNR (mean over fields of
    20 log10(R / RMSE), R = the field's value range; None when lossless).
    md_mode = SZ_MODE_LV_PRX compresses xs (xx, yy, zz) as one reordered MD
    snapshot and compares each decoded field with the reordered original.
    Also the closed form -20 log10(eb / sqrt 3) of uniform quantization noise
    and the worst |x - x'| / (eb R) over the fields.  The streams use the
    fixed chunk-size rule (the batched form's autotuner is switched off on
    ctx), so a point's rate does not depend on run-time measurements."""
    import torch
    sz.sz_ctx_set_autotune(ctx, False)
    pts = []
    n_tot = sum(x.numel() for x in xs)
    for eb in ebs:
        if md_mode is None:
            outs, nb = sz.sz_compress_batch(ctx, xs, [eb] * len(xs), sz.SZ_EB_REL, params=params)
            refs = xs
        else:
            n = xs[0].numel()
            perm = torch.empty(n, dtype=torch.int32, device=xs[0].device)
            outs, nb = sz.sz_compress_snapshot(ctx, [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ], xs, n,
                                               [eb] * 3, sz.SZ_EB_REL, md_mode, params, perm=perm)
        sz.sz_sync(ctx)
        sizes = [int(nb[i]) for i in range(len(xs))]
        if md_mode is not None:
            refs = [x[perm.long()] for x in xs]
        ys = [torch.empty_like(x) for x in xs]
        sz.sz_decompress_batch(ctx, outs, sizes, ys)
        sz.sz_sync(ctx)
        psnr, worst, lossless = [], 0.0, True
        for x, y in zip(refs, ys):
            fin = torch.isfinite(x)
            R = (x[fin].max().double() - x[fin].min().double()).item()
            e = x[fin].double() - y[fin].double()
            mse = e.square().mean().item()
            if mse > 0:
                lossless = False
                psnr.append(20 * math.log10(R / math.sqrt(mse)))
            if R > 0:
                worst = max(worst, e.abs().max().item() / (eb * R))
        pts.append({"eb": eb, "bits_per_value": 8 * sum(sizes) / n_tot,
                    "psnr_db": None if lossless else sum(psnr) / len(psnr),
                    "psnr_closed_form_db": -20 * math.log10(eb / math.sqrt(3)), "max_err_over_eb": worst})
    return pts


def rkeys_bench(sz, device, steps):
    """Table 6: the plain cosmology snapshot (2^20 particles, 64 halos, six
    fields) in stored order (SZ-LV) and reordered by the R-index built from
    the coordinates, the velocities or all six fields (segments of 4096, no
    ignored digits), rel eb 1e-4: per-field ratios, the overall ratio and the
    compression rate of the six fields (reordering included)."""
    import torch
    import synth
    snap = synth.cosmology(1 << 20, 64, 1, device="cuda")
    xs = [snap[f] for f in FIELDS]
    n = xs[0].numel()
    raw = 4 * n
    ctx = sz.Context(device)
    stream = torch.cuda.current_stream()
    tags = [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ, sz.SZ_FIELD_VX, sz.SZ_FIELD_VY, sz.SZ_FIELD_VZ]
    out = {"workload": "plain cosmology snapshot, 2^20 particles x 6 fields, rel eb 1e-4, segment 4096, p = 0",
           "keys": {}}
    for name, mode, key in (("stored order (SZ-LV)", sz.SZ_MODE_LV, 0), ("coordinates", sz.SZ_MODE_LV_PRX, 0),
                            ("velocities", sz.SZ_MODE_LV_PRX, 1), ("coordinates + velocities", sz.SZ_MODE_LV_PRX, 2)):
        prm = sz._params(0, 0, 4096, 0, 0, key) if mode == sz.SZ_MODE_LV_PRX else None

        def run():
            return sz.sz_compress_snapshot(ctx, tags, xs, n, [1e-4] * 6, sz.SZ_EB_REL, mode, prm)

        for _ in range(2):
            outs, nb = run()
            sz.sz_sync(ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            a.record(stream)
            outs, nb = run()
            b.record(stream)
        sz.sz_sync(ctx)
        torch.cuda.synchronize()
        t = sum(a.elapsed_time(b) for a, b in ev) / steps / 1e3
        sizes = [int(nb[i]) for i in range(6)]
        out["keys"][name] = {"ratio": 6 * raw / sum(sizes), "compress_gbs": 6 * raw / t / 1e9,
                             "per_field": {f: raw / b for f, b in zip(FIELDS, sizes)}}
    ctx.close()
    return out


def rd_bench(sz, device, xs):
    """Fig. 9 sweep: the large cosmology snapshot under LV and LCF, and the
    MD snapshot under best_speed (LV) and best_tradeoff (LV-PRX, p = 6)."""
    import synth
    ctx = sz.Context(device)
    out = {"ebs": list(RD_EBS),
           "cosmology_lv": rd_points(sz, ctx, xs),
           "cosmology_lcf": rd_points(sz, ctx, xs, params=sz._params(predictor=sz.SZ_PRED_LCF))}
    md = synth.md_fcc(device="cuda")
    ms = [md[f] for f in ("xx", "yy", "zz")]
    out["md_lv"] = rd_points(sz, ctx, ms)
    out["md_lv_prx"] = rd_points(sz, ctx, ms, params=sz._params(0, 0, 16384, 6), md_mode=sz.SZ_MODE_LV_PRX)
    out["note"] = ("bits/value = 8 x stream bytes / values; PSNR averaged over fields; None = lossless "
                   "(the raw fallback)")
    ctx.close()
    return out


def lcf_bench(sz, ctx, stream, step, xs, ys, outs, args, raw_bytes, ratio_lv, with_cpu=True):
    """The per-array path with the LCF predictor on the benchmark arrays:
    compress / decompress GB/s from CUDA events, the ratio against LV's, and
    each kernel phase's device time.  Checks the error bound first."""
    import torch
    holders = step(plain=True, lcf=True)
    sz.sz_sync(ctx)
    sizes = [h.value for h in holders]
    for x, y in zip(xs, ys):
        fin = torch.isfinite(x)
        R = (x[fin].max().double() - x[fin].min().double()).item()
        assert (x.double() - y.double()).abs().max().item() <= args.eb * R * (1 + 1e-12)
    step(plain=True, lcf=True)
    sz.sz_sync(ctx)
    k = max(1, min(args.steps, 3))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    torch.cuda.synchronize()
    sz.sz_profile_enable(ctx, True)
    for i in range(k):
        ev[i][0].record(stream)
        step(ev[i][1], plain=True, lcf=True)
        ev[i][2].record(stream)
    sz.sz_sync(ctx)
    torch.cuda.synchronize()
    prof = sz.sz_profile_read(ctx)
    sz.sz_profile_enable(ctx, False)
    tc = sum(e[0].elapsed_time(e[1]) for e in ev) / 1e3 / k
    td = sum(e[1].elapsed_time(e[2]) for e in ev) / 1e3 / k
    ms = {ph: ms / k for ph, (c, ms) in prof.items() if c}
    # the dominant LCF kernel by device time: decode, whose algorithmic bytes
    # are the streams read plus the floats written
    peak, peak_kind = _peaks()
    dec_bytes = sum(sizes) + raw_bytes
    dec_gbs = dec_bytes / (ms["decode"] / 1e3) / 1e9
    # the oracle beside it (CPU-baseline leg: rank 0 at N = 1 only): LCF round
    # trips of the first 2^22 elements of each field, one thread per field
    cpu = None
    if with_cpu:
        import oracle
        oracle.build()
        from concurrent.futures import ThreadPoolExecutor
        samp = [x[: 1 << 22].cpu().numpy() for x in xs]

        def one(a):
            oracle.decompress(oracle.compress(a, args.eb, 1, 4096, 64, pred=oracle.PRED_LCF))

        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=len(samp)) as ex:
            list(ex.map(one, samp))
        t_or = time.perf_counter() - t0
        cpu = {"value": 4 * sum(a.size for a in samp) / t_or / 1e9, "unit": "GB/s", "cores": len(samp),
               "kind": "oracle",
               "sample": "first 2^22 elements of each field, LCF compress + decompress, one thread per field"}
    return {"compress_gbs": raw_bytes / tc / 1e9, "decompress_gbs": raw_bytes / td / 1e9,
            "round_trip_gbs": raw_bytes / (tc + td) / 1e9, "ratio": raw_bytes / sum(sizes), "ratio_lv": ratio_lv,
            "ms_per_step": {ph: round(v, 4) for ph, v in ms.items()},
            "roofline": {"kernel": "decode_kernel (LCF team loops)", "bound": "hbm", "achieved": dec_gbs,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": dec_gbs / peak,
                         "algorithmic_bytes_per_step": dec_bytes},
            "cpu_oracle": cpu,
            "note": "per field: sz_compress / sz_decompress with predictor SZ_PRED_LCF (second differences)"}


def link_rates(hx, hy):
    """Host<->device copy rates of the pinned buffers the end-to-end leg uses
    (plain copies, one direction at a time and both at once): the ceiling of
    that leg.  GB/s."""
    import torch
    d = [torch.empty_like(x, device="cuda") for x in hx]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nb = sum(4 * x.numel() for x in hx)

    def h2d():
        with torch.cuda.stream(s1):
            for a, b in zip(hx, d):
                b.copy_(a, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            for a, b in zip(d, hy):
                b.copy_(a, non_blocking=True)

    def timed(f, reps=3):
        # best and median of a few copies: one slow host-side step (they occur
        # on shared hosts) must not stand for the link
        f()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            f()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        ts.sort()
        return ts[0], ts[len(ts) // 2]

    (t_in, m_in), (t_out, m_out) = timed(h2d), timed(d2h)
    t_both, m_both = timed(lambda: (h2d(), d2h()))
    del d
    return {"h2d_gbs": nb / t_in / 1e9, "d2h_gbs": nb / t_out / 1e9, "both_gbs": 2 * nb / t_both / 1e9,
            "h2d_gbs_median": nb / m_in / 1e9, "d2h_gbs_median": nb / m_out / 1e9,
            "both_gbs_median": 2 * nb / m_both / 1e9, "stat": "best and median of 3 copies after one"}


def _ncu_entry(kernel: str):
    """The committed ncu record of `kernel` (per-launch DRAM bytes and device
    time on the full workload), if the kernel's sources are unchanged since
    the capture; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(kernel)
        if not e:
            return None
        h = hashlib.sha256()
        for f in e["sources"]:
            h.update(open(os.path.join(ROOT, "paper_1711_03888_gb300", "csrc", f), "rb").read())
        if h.hexdigest()[:16] != e["sources_sha256_16"]:
            return None
        return e
    except Exception:
        return None


def _ncu_sum(kernel: str):
    """(DRAM bytes, device ns) per launch of `kernel` -- or of every kernel of
    "a + b", summed -- from the committed ncu summary; None if any part is
    missing or stale."""
    b = ns = 0.0
    for k in kernel.split(" + "):
        e = _ncu_entry(k.strip())
        try:
            b += float(e["bytes_per_launch_full"])
            ns += float(e["ncu_duration_ns"])
        except (KeyError, TypeError, ValueError):
            return None
    return b, ns


def _traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if the
    kernel source is unchanged since the capture; else None."""
    r = _ncu_sum(kernel)
    return None if r is None else r[0]


def ncu_dram_rate(kernel: str, peak: float):
    """The DRAM rate ncu measured for one launch of `kernel` (bytes read and
    written over its serialised device time), and its fraction of `peak`."""
    r = _ncu_sum(kernel)
    if r is None or r[1] <= 0:
        return None
    b, ns = r
    gbs = b / ns
    return {"dram_bytes": b, "duration_ms": ns / 1e6, "dram_gbs": gbs, "dram_frac": gbs / peak}


# The batched step's kernels whose DRAM traffic bench.py reports, and the
# sources each is built from (an entry counts only while these hash alike).
NCU_KERNELS = {
    "range_multi_kernel": ["k_multi.cu", "sz_range.cuh", "sz_device.cuh", "sz_internal.h"],
    "quant_multi_kernel": ["k_multi.cu", "sz_quant.cuh", "sz_device.cuh", "sz_internal.h"],
    "encode_sizes_multi_kernel": ["k_multi.cu", "sz_encode.cuh", "sz_device.cuh", "sz_internal.h"],
    "encode_pack_multi_kernel": ["k_multi.cu", "sz_encode.cuh", "sz_device.cuh", "sz_internal.h"],
    "decode_multi_kernel": ["k_decode.cu", "sz_blocksort.cuh", "sz_device.cuh", "sz_internal.h"],
}
_UNIT = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12,
         "b": 1.0, "kb": 1e3, "mb": 1e6, "gb": 1e9, "tb": 1e12,
         "nsecond": 1.0, "usecond": 1e3, "msecond": 1e6, "second": 1e9,
         "ns": 1.0, "us": 1e3, "ms": 1e6, "s": 1e9}


def write_traffic(csv_path: str, command: str) -> dict:
    """profiles/traffic.json from an ncu CSV log (--metrics gpu__time_duration.sum,
    dram__bytes_read.sum,dram__bytes_write.sum --csv): per kernel of
    NCU_KERNELS, the mean over its captured launches, with the hash of its
    sources.  Host only."""
    import csv
    rows = [r for r in csv.reader(open(csv_path)) if r]
    hdr_i = next(i for i, r in enumerate(rows) if "Metric Name" in r and "Kernel Name" in r)
    hdr = rows[hdr_i]
    col = {h: hdr.index(h) for h in ("ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value")}
    launches = {}
    for r in rows[hdr_i + 1:]:
        if len(r) < len(hdr):
            continue
        unit = r[col["Metric Unit"]].strip().lower()
        v = float(r[col["Metric Value"]].replace(",", "")) * _UNIT.get(unit, 1.0)
        d = launches.setdefault(r[col["ID"]], {"name": r[col["Kernel Name"]]})
        d[r[col["Metric Name"]]] = v
    out = {"_about": ("Per-launch DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass) "
                      "of the batched step's kernels on the large cosmology snapshot: 6 arrays of 2^27 float32 "
                      "per launch, rel eb 1e-4. Command: " + command + ". Written by bench.py --write-traffic; "
                      "bench.py uses an entry only while the listed sources hash to sources_sha256_16.")}
    csrc = os.path.join(ROOT, "paper_1711_03888_gb300", "csrc")
    for k, srcs in NCU_KERNELS.items():
        ls = [d for d in launches.values() if re.search(r"\b" + k + r"\b", d["name"])]
        ls = [d for d in ls if "dram__bytes_read.sum" in d and "dram__bytes_write.sum" in d]
        if not ls:
            continue
        h = hashlib.sha256()
        for f in srcs:
            h.update(open(os.path.join(csrc, f), "rb").read())
        rd = sum(d["dram__bytes_read.sum"] for d in ls) / len(ls)
        wr = sum(d["dram__bytes_write.sum"] for d in ls) / len(ls)
        ns = sum(d.get("gpu__time_duration.sum", 0.0) for d in ls) / len(ls)
        out[k] = {"sources": srcs, "sources_sha256_16": h.hexdigest()[:16], "bytes_per_launch_full": rd + wr,
                  "dram_read": rd, "dram_write": wr, "ncu_duration_ns": ns, "launches_captured": len(ls)}
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return out


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg / reference arm)
# ---------------------------------------------------------------------------

def oracle_round_trip(arrays, eb):
    """Round trip of each array through the oracle, one thread per array (the
    paper's one-process-per-array model); returns (seconds, bytes)."""
    import oracle
    oracle.build()
    from concurrent.futures import ThreadPoolExecutor

    def one(x):
        s = oracle.compress(x, eb, 1, 4096, 64)
        oracle.decompress(s)
        return len(s)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=len(arrays)) as ex:
        list(ex.map(one, arrays))
    return time.perf_counter() - t0, sum(4 * a.size for a in arrays)


class _Holder:
    """View of one entry of a batch's size array (valid after sz_sync)."""

    def __init__(self, arr, i):
        self.arr, self.i = arr, i

    @property
    def value(self):
        return int(self.arr[self.i])


def _stats_ms(seconds):
    """best / median / mean of per-step times (seconds in, ms out)."""
    import numpy as np
    v = 1e3 * np.asarray(seconds, dtype=np.float64)
    return {"best": float(v.min()), "median": float(np.median(v)), "mean": float(v.mean())}


def cpu_sample(snap, n_sample):
    import numpy as np
    return [np.ascontiguousarray(snap[f][:n_sample].cpu().numpy()) for f in FIELDS]


# ---------------------------------------------------------------------------

def _round_trip_timed(sz, ctx, stream, xs, ebs, outs, ys, steps, traced=False):
    """steps x (sz_compress_batch + sz_decompress_batch) with CUDA events around
    each half; returns (compress seconds per step, decompress seconds per step,
    stream sizes, per-phase trace or None)."""
    import torch
    if traced:
        sz.sz_profile_enable(ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b, c in ev:
        a.record(stream)
        _, nb = sz.sz_compress_batch(ctx, xs, ebs, sz.SZ_EB_REL, outs=outs)
        b.record(stream)
        sz.sz_decompress_batch(ctx, outs, [o.numel() for o in outs], ys)
        c.record(stream)
    sz.sz_sync(ctx)
    torch.cuda.synchronize()
    prof = None
    if traced:
        prof = sz.sz_profile_read(ctx)
        sz.sz_profile_enable(ctx, False)
    tc = sum(a.elapsed_time(b) for a, b, _ in ev) / steps / 1e3
    td = sum(b.elapsed_time(c) for _, b, c in ev) / steps / 1e3
    return tc, td, [int(nb[i]) for i in range(len(xs))], prof


def bounds_bench(sz, ctx, stream, xs, ys, outs, raw_bytes, steps, peak):
    """The large snapshot at its other relative bounds (1e-3 and 1e-5), through
    the same batched calls: round-trip rates, ratio, and the traced decoder's
    rate of its algorithmic bytes against the HBM peak."""
    res = {}
    for eb in (1e-3, 1e-5):
        ebs = [eb] * len(xs)
        for _ in range(2):
            _round_trip_timed(sz, ctx, stream, xs, ebs, outs, ys, 1)
        tc, td, sizes, _ = _round_trip_timed(sz, ctx, stream, xs, ebs, outs, ys, steps)
        _, _, _, prof = _round_trip_timed(sz, ctx, stream, xs, ebs, outs, ys, steps, traced=True)
        sb = sum(sizes)
        if prof.get("encode_sizes", (0, 0.0))[0]:       # two-pass encode: both kernels count
            prof = dict(prof)
            prof["encode"] = (prof["encode"][0], prof["encode"][1] + prof["encode_sizes"][1])
        rec = {"compress_gbs": raw_bytes / tc / 1e9, "decompress_gbs": raw_bytes / td / 1e9,
               "round_trip_gbs": raw_bytes / (tc + td) / 1e9, "ratio": raw_bytes / sb,
               "compress_frac_hbm": raw_bytes / tc / 1e9 / peak, "decompress_frac_hbm": raw_bytes / td / 1e9 / peak}
        for ph, algo in (("decode", sb + raw_bytes), ("encode", raw_bytes // 2 + sb), ("quant", raw_bytes * 3 // 2)):
            cnt, ms = prof.get(ph, (0, 0.0))
            if cnt:
                avg = ms / cnt / 1e3
                per_launch = algo * steps / cnt
                rec[ph] = {"avg_ms": 1e3 * avg, "achieved_gbs": per_launch / avg / 1e9,
                           "frac": per_launch / avg / 1e9 / peak}
        res[f"{eb:g}"] = rec
    return res


def small_bench(sz, device, eb, steps, peak):
    """The plain cosmology snapshot of 2^20 particles x 6 fields (4 MiB arrays,
    64 halos) through the batched calls: round-trip rates and ratio."""
    import torch
    import synth
    snap = synth.cosmology(1 << 20, 64, 1, device="cuda")
    xs = [snap[f] for f in FIELDS]
    raw = 4 * sum(x.numel() for x in xs)
    ctx = sz.Context(device)
    outs = [torch.empty(sz.sz_max_compressed_bytes(x.numel()), dtype=torch.uint8, device="cuda") for x in xs]
    ys = [torch.empty(x.numel(), dtype=torch.float32, device="cuda") for x in xs]
    stream = torch.cuda.current_stream()
    ebs = [eb] * len(xs)
    for _ in range(3):
        _round_trip_timed(sz, ctx, stream, xs, ebs, outs, ys, 1)
    tc, td, sizes, _ = _round_trip_timed(sz, ctx, stream, xs, ebs, outs, ys, steps)
    res = {"workload": f"plain cosmology snapshot: 2^20 particles x 6 float32 fields, 64 halos, rel eb {eb:g}",
           "compress_gbs": raw / tc / 1e9, "decompress_gbs": raw / td / 1e9, "round_trip_gbs": raw / (tc + td) / 1e9,
           "compress_ms": 1e3 * tc, "decompress_ms": 1e3 * td, "ratio": raw / sum(sizes),
           "compress_frac_hbm": raw / tc / 1e9 / peak, "decompress_frac_hbm": raw / td / 1e9 / peak,
           "tuned_chunk": sz.sz_batch_tuning(ctx, 1 << 20)["chunk_elems"]}
    ctx.close()
    return res


# ---------------------------------------------------------------------------
# Batched form: 128 simulated ranks x 6 fields of uneven sizes
# ---------------------------------------------------------------------------

def batched_bench(sz, device, steps):
    """768 arrays of 2^U[14,24] float32 (128 ranks x 6 fields, per-array rel eb
    from {1e-3, 1e-4}): one sz_compress_batch call (one CUDA graph) against
    768 sz_compress calls on the same stream; then the batched decompression.
    Device-resident inputs; CUDA events around each variant."""
    import torch
    import synth
    arrays = synth.batch_ranks(device="cuda")
    xs = [t for _, _, t, _ in arrays]
    ebs = [e for _, _, _, e in arrays]
    nbytes = sum(4 * x.numel() for x in xs)
    ctx = sz.Context(device)
    outs = [torch.empty(sz.sz_max_compressed_bytes(x.numel()), dtype=torch.uint8, device="cuda") for x in xs]
    ys = [torch.empty(max(x.numel(), 1), dtype=torch.float32, device="cuda") for x in xs]
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        sz.sz_sync(ctx)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / k / 1e3

    def batch():
        return sz.sz_compress_batch(ctx, xs, ebs, sz.SZ_EB_REL, outs=outs)[1]

    def plain():
        for x, e, o in zip(xs, ebs, outs):
            sz.sz_compress(ctx, x, e, sz.SZ_EB_REL, None, o)

    for _ in range(3):
        nb = batch()
        sz.sz_sync(ctx)
    sizes = [int(nb[i]) for i in range(len(xs))]
    t_batch = timed(batch, steps)
    plain()
    sz.sz_sync(ctx)
    t_plain = timed(plain, max(1, min(steps, 2)))

    def decomp():
        sz.sz_decompress_batch(ctx, outs, [o.numel() for o in outs], ys)

    decomp()
    sz.sz_sync(ctx)
    t_dec = timed(decomp, steps)
    # what the autotuner chose (one entry per size class present) ...
    classes = {}
    for x in xs:
        t = sz.sz_batch_tuning(ctx, x.numel())
        key = f"{t['class'][0]}..{t['class'][1]}"
        if key not in classes:
            classes[key] = {"chunk": t["chunk_elems"], "fixed_rule_chunk": t["fixed_chunk_elems"],
                            "trial_ms": t["trial_ms"], "arrays": 0}
        classes[key]["arrays"] += 1
    t0 = sz.sz_batch_tuning(ctx, xs[0].numel())
    tuned = {"classes": classes, "range_tile": t0["range_tile"], "quant_group": t0["quant_group"],
             "tile_trial_ms": t0["tile_trial_ms"],
             "note": "chosen by timing compress + decompress of the batch on the device for each candidate "
                     "chunk size (first sight of a size class), then the persistent kernel's item sizes"}
    # ... against the fixed rule (2048 up to 2^16 elements, else 4096; default item sizes)
    sz.sz_ctx_set_autotune(ctx, False)
    for _ in range(2):
        nbf = batch()
        sz.sz_sync(ctx)
    sizes_f = [int(nbf[i]) for i in range(len(xs))]
    t_batch_f = timed(batch, steps)
    decomp()
    sz.sz_sync(ctx)
    t_dec_f = timed(decomp, steps)
    tuned["fixed_rule"] = {"compress_ms": 1e3 * t_batch_f, "decompress_ms": 1e3 * t_dec_f,
                           "round_trip_ms": 1e3 * (t_batch_f + t_dec_f), "ratio": nbytes / sum(sizes_f)}
    tuned["tuned_round_trip_ms"] = 1e3 * (t_batch + t_dec)
    res = {"workload": "768 float32 arrays (128 ranks x 6 fields), 2^U[14,24] elements each, per-array rel eb "
                       "from {1e-3, 1e-4}; cosmology generator per rank sub-box",
           "arrays": len(xs), "gbytes": nbytes / 1e9, "ratio": nbytes / sum(sizes),
           "batched_compress_gbs": nbytes / t_batch / 1e9, "batched_compress_ms": 1e3 * t_batch,
           "plain_compress_gbs": nbytes / t_plain / 1e9, "plain_compress_ms": 1e3 * t_plain,
           "speedup": t_plain / t_batch,
           "decompress_gbs": nbytes / t_dec / 1e9, "decompress_ms": 1e3 * t_dec, "autotuner": tuned}
    ctx.close()
    return res


# ---------------------------------------------------------------------------
# Molecular-dynamics snapshot: the three position arrays, with and without the
# R-index reordering (Sec. IV-B; Tables 4-5)
# ---------------------------------------------------------------------------

def md_bench(sz, device, steps, with_cpu=True):
    """FCC crystal of 100^3 cells (3.92 M atoms after 2 % vacancies, 10 %
    swapped), xx/yy/zz: best_speed (SZ-LV in stored order) against best_tradeoff
    (SZ-LV-PRX: segment 16384, p = 6 ignored digits, and p = 0 = full radix
    sort within segments) and best_compression (SZ-CPC2000: full R-index sort,
    Rice-coded key differences; also its decoding rate), at rel eb 1e-4 and
    1e-3.  Compression GB/s of the three arrays (reordering included) and the
    ratio; CUDA events on the stream."""
    import torch
    import synth
    md = synth.md_fcc(device="cuda")
    xs = [md[f] for f in ("xx", "yy", "zz")]
    n = xs[0].numel()
    nbytes = 4 * n * len(xs)
    ctx = sz.Context(device)
    fields = [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ]
    stream = torch.cuda.current_stream()
    out = {"workload": f"MD snapshot: FCC crystal 100^3 cells, {n} atoms, 3 float32 position arrays",
           "atoms": n, "modes": {}}
    cpc_outs = [torch.empty(sz.sz_cpc_max_bytes(n), dtype=torch.uint8, device="cuda")] + \
        [torch.empty(16, dtype=torch.uint8, device="cuda") for _ in range(2)]
    for eb in (1e-4, 1e-3):
        for name, mode, p in (("best_speed LV", sz.SZ_MODE_LV, None), ("best_tradeoff LV-PRX p=6", sz.SZ_MODE_LV_PRX, 6),
                              ("LV-RX (p=0)", sz.SZ_MODE_LV_PRX, 0),
                              ("best_compression SZ-CPC2000", sz.SZ_MODE_CPC2000, None)):
            params = sz._params(0, 0, 16384, p) if p is not None else None
            outs_m = cpc_outs if mode == sz.SZ_MODE_CPC2000 else None

            def run():
                return sz.sz_compress_snapshot(ctx, fields, xs, n, [eb] * 3, sz.SZ_EB_REL, mode, params, outs=outs_m)

            for _ in range(2):
                outs, nb = run()
                sz.sz_sync(ctx)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                a.record(stream)
                outs, nb = run()
                b.record(stream)
            sz.sz_sync(ctx)
            torch.cuda.synchronize()
            t = sum(a.elapsed_time(b) for a, b in ev) / steps / 1e3
            rec = {"compress_gbs": nbytes / t / 1e9, "ms": 1e3 * t,
                   "ratio": nbytes / sum(int(nb[i]) for i in range(3))}
            if mode == sz.SZ_MODE_CPC2000:
                # decoding the coordinate stream (all three arrays)
                ys = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
                size = int(nb[0])
                for _ in range(2):
                    sz.sz_decompress_cpc(ctx, outs[0], size, ys)
                    sz.sz_sync(ctx)
                evd = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(steps)]
                for a, b in evd:
                    a.record(stream)
                    sz.sz_decompress_cpc(ctx, outs[0], size, ys)
                    b.record(stream)
                sz.sz_sync(ctx)
                torch.cuda.synchronize()
                td = sum(a.elapsed_time(b) for a, b in evd) / steps / 1e3
                rec["decompress_gbs"] = nbytes / td / 1e9
                # decoding reads the stream and writes three float arrays; the oracle beside it
                peak, _ = _peaks()
                rec["decode_roofline_frac"] = (size + nbytes) / td / 1e9 / peak
                if eb == 1e-4 and with_cpu:      # CPU-baseline leg: rank 0 at N = 1 only
                    import oracle
                    oracle.build()
                    hx = [x.cpu().numpy() for x in xs]
                    t0 = time.perf_counter()
                    s_or, _ = oracle.compress_cpc(*hx, eb, 1)
                    oracle.decompress_cpc(s_or)
                    rec["cpu_oracle_gbs"] = nbytes / (time.perf_counter() - t0) / 1e9
                    rec["cpu_oracle_note"] = "compress + decompress of the same crystal by the oracle, one thread"
            out["modes"][f"{name} @ {eb:g}"] = rec
    ctx.close()
    return out


# ---------------------------------------------------------------------------
# Served form: Poisson arrivals of compress / decompress requests
# ---------------------------------------------------------------------------

def _percentile(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def make_requests(rng, rate, seconds, pools, streams, log2_lo=18.0, log2_hi=27.0):
    """Open-loop request list: (arrival_s, op, tensor, n, in_bytes).  Sizes are
    2^U[log2_lo, log2_hi] floats sliced (16-byte aligned) from the device
    pools; decompress requests take one of the pre-compressed streams."""
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            return out
        if rng.random() < 0.5:
            n = int(round(2.0 ** rng.uniform(log2_lo, log2_hi)))
            fits = [p for p in pools if p.numel() >= n]
            src = fits[int(rng.integers(len(fits)))]
            off = int(rng.integers(0, (src.numel() - n) // 4 + 1)) * 4
            out.append((t, "c", src[off: off + n], n, 0))
        else:
            st, n, nb = streams[int(rng.integers(len(streams)))]
            out.append((t, "d", st, n, nb))


def run_served(sz, ctx, reqs, eb):
    """Submit at the arrival times (producer), wait and release in ticket order
    (consumer thread).  Returns per-request latencies and the makespan."""
    import ctypes as C
    tickets = [None] * len(reqs)
    lat = [0.0] * len(reqs)
    bad = []
    ready = threading.Semaphore(0)

    def consumer():
        for i in range(len(reqs)):
            ready.acquire()
            r = sz.sz_serve_wait(ctx, tickets[i], 600.0)
            if r.status != sz.SZ_OK:
                bad.append((i, r.status))
            lat[i] = r.latency_s
            if r.out:
                sz.sz_serve_release(ctx, r.out)

    th = threading.Thread(target=consumer)
    # the producer sleeps between arrivals (releasing the GIL) and spins only
    # for the last 0.2 ms, so the consumer releases outputs promptly
    old_sw = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)
    th.start()
    t0 = time.perf_counter()
    for i, (ta, op, x, n, nb) in enumerate(reqs):
        while True:
            d = ta - (time.perf_counter() - t0)
            if d <= 0:
                break
            if d > 3e-4:
                time.sleep(d - 2e-4)
        if op == "c":
            req = sz.request(sz.SZ_OP_COMPRESS, x, n, eb=eb, kind=sz.SZ_EB_REL)
        else:
            req = sz.request(sz.SZ_OP_DECOMPRESS, x, n, in_bytes=nb)
        tickets[i] = sz.sz_serve_submit(ctx, req)
        ready.release()
    th.join()
    span = time.perf_counter() - t0
    sys.setswitchinterval(old_sw)
    if bad:
        raise RuntimeError(f"served requests failed: {bad[:5]}")
    return lat, span


def run_serial_plain(sz, ctx, reqs, eb, out_c, out_d):
    """The same requests issued at their arrival times, one after another,
    through the plain calls: each sz_compress / sz_decompress is followed by
    sz_sync, so a request that arrives while the previous one runs waits for
    it.  Latency = completion - arrival (host clock); the device time of each
    call from CUDA events."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in reqs]
    torch.cuda.synchronize()
    lat = []
    t0 = time.perf_counter()
    for e, (ta, op, x, n, nb) in zip(ev, reqs):
        while True:
            d = ta - (time.perf_counter() - t0)
            if d <= 0:
                break
            if d > 3e-4:
                time.sleep(d - 2e-4)
        e[0].record(stream)
        if op == "c":
            sz.sz_compress(ctx, x, eb, sz.SZ_EB_REL, None, out_c)
        else:
            sz.sz_decompress(ctx, x, nb, out_d, n)
        e[1].record(stream)
        sz.sz_sync(ctx)
        lat.append(time.perf_counter() - t0 - ta)
    torch.cuda.synchronize()
    span = time.perf_counter() - t0
    svc = [a.elapsed_time(b) / 1e3 for a, b in ev]
    return lat, sum(svc), span


def served_bench(sz, snap, eb, rate, seconds, stress, stress_seconds, slots, budget_gb, device):
    """Config-4 style serving run; returns the "served" object of the JSON line."""
    import numpy as np
    import torch
    import synth
    rng = np.random.default_rng(5)
    md = synth.md_fcc(device="cuda")
    pools = [snap[f] for f in FIELDS] + [md[f] for f in ("xx", "yy", "zz")]
    plain = sz.Context(device)
    # pre-compressed streams for the decompress requests
    streams = []
    for i in range(32):
        n = int(round(2.0 ** rng.uniform(18.0, 27.0)))
        fits = [p for p in pools if p.numel() >= n]
        src = fits[int(rng.integers(len(fits)))]
        off = int(rng.integers(0, (src.numel() - n) // 4 + 1)) * 4
        out, nb = sz.sz_compress(plain, src[off: off + n], eb, sz.SZ_EB_REL)
        sz.sz_sync(plain)
        streams.append((out[: nb.value].clone(), n, nb.value))
        del out
    nmax = max(p.numel() for p in pools)
    out_c = torch.empty(sz.sz_max_compressed_bytes(nmax), dtype=torch.uint8, device="cuda")
    out_d = torch.empty(nmax, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    ctx = sz.Context(device, budget=int(budget_gb * (1 << 30)))
    sz.sz_serve_start(ctx, slots)
    # warm-up: every slot's workspace grows to the largest request size once
    big = pools[0][: nmax // 4 * 4]
    warm = [(0.0, "c", big, big.numel(), 0)] * slots + [(0.0, "d", st, n, nb) for st, n, nb in streams[:slots]]
    run_served(sz, ctx, warm, eb)

    res = {"workload": f"Poisson arrivals, {rate:g} req/s for {seconds:g} s; compress or decompress (p=1/2); "
                       f"2^U[18,27] float32 per request sliced from the cosmology snapshot and the MD crystal; "
                       f"rel eb {eb:g}",
           "slots": slots, "budget_gb": budget_gb}
    for tag, lam, secs in (("nominal", rate, seconds), ("stress", rate * stress, stress_seconds)):
        reqs = make_requests(rng, lam, secs, pools, streams)
        nbytes = sum(4 * r[3] for r in reqs)
        lat, span = run_served(sz, ctx, reqs, eb)
        lat_p, busy_p, span_p = run_serial_plain(sz, plain, reqs, eb, out_c, out_d)
        res[tag] = {
            "rate_per_s": lam, "requests": len(reqs), "gbytes": nbytes / 1e9,
            "p50_ms": 1e3 * _percentile(lat, 50), "p99_ms": 1e3 * _percentile(lat, 99),
            "gbs": nbytes / span / 1e9,
            "serial_plain": {"p50_ms": 1e3 * _percentile(lat_p, 50), "p99_ms": 1e3 * _percentile(lat_p, 99),
                             "gbs_device_busy": nbytes / busy_p / 1e9, "gbs_wall": nbytes / span_p / 1e9},
        }
    res["counters"] = sz.sz_serve_stats(ctx)
    sz.sz_serve_stop(ctx)
    ctx.close()
    # the stress arrivals under a budget below what they keep in flight, so
    # that admission waits for budget (a 2^27-element compress holds ~1.3 GB)
    small_gb = 3.0
    ctx = sz.Context(device, budget=int(small_gb * (1 << 30)))
    sz.sz_serve_start(ctx, slots)
    run_served(sz, ctx, [(0.0, "c", big[: 1 << 27], 1 << 27, 0)] + [(0.0, "d", st, n, nb) for st, n, nb in streams[:2]],
               eb)
    reqs = make_requests(rng, rate * stress, stress_seconds, pools, streams)
    lat, span = run_served(sz, ctx, reqs, eb)
    nbytes = sum(4 * r[3] for r in reqs)
    res["stress_small_budget"] = {"budget_gb": small_gb, "rate_per_s": rate * stress, "requests": len(reqs),
                                  "p50_ms": 1e3 * _percentile(lat, 50), "p99_ms": 1e3 * _percentile(lat, 99),
                                  "gbs": nbytes / span / 1e9, "counters": sz.sz_serve_stats(ctx)}
    sz.sz_serve_stop(ctx)
    ctx.close()
    plain.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log2n", type=int, default=27)
    ap.add_argument("--eb", type=float, default=1e-4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-lcf", action="store_true")
    ap.add_argument("--no-rd", action="store_true")
    ap.add_argument("--no-rkeys", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-log2n", type=int, default=26)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-md", action="store_true")
    ap.add_argument("--no-bounds", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-stress", type=float, default=10.0)
    ap.add_argument("--serve-stress-seconds", type=float, default=0.25)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=48.0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="headline batch at the fixed chunk-size rule (for runs under a profiler)")
    ap.add_argument("--write-traffic", metavar="NCU_CSV",
                    help="host only: write profiles/traffic.json from an ncu CSV log and exit")
    ap.add_argument("--traffic-command", default="", help="the ncu command line recorded with --write-traffic")
    args = ap.parse_args()
    if args.write_traffic:
        print(json.dumps(write_traffic(args.write_traffic, args.traffic_command), indent=1))
        return

    ws, rank, local = _dist()
    n = 1 << args.log2n
    halos = 4096 if args.log2n == 27 else max(1, int(round(64 * n / (1 << 20))))
    workload = f"large cosmology snapshot: 2^{args.log2n} particles x 6 float32 fields, {halos} halos, rel eb {args.eb:g}"
    config = {"workload": workload, "particles": n, "fields": 6, "eb_rel": args.eb, "eb_kind": "relative",
              "step": "compress 6 arrays + decompress 6 streams", "l2": "inputs (3.2 GB) larger than L2",
              "parallelism": f"replicas x{ws} (independent snapshots, no data-path collective)"}

    if args.impl == "reference":
        if rank != 0:
            return
        import synth
        import torch
        snap = synth.cosmology(n, halos, 3, device="cuda" if torch.cuda.is_available() else "cpu")
        arrays = cpu_sample(snap, 1 << args.cpu_log2n)
        del snap
        for _ in range(args.warmup):
            oracle_round_trip(arrays, args.eb)
        tt, b = 0.0, 0
        for _ in range(args.steps):
            t, b = oracle_round_trip(arrays, args.eb)
            tt += t
        v = b * args.steps / tt / 1e9
        sample = f"first 2^{args.cpu_log2n} elements of each of the 6 fields, one thread per field"
        print(json.dumps({"impl": "reference", "metric": "round-trip (compress+decompress) throughput, uncompressed float32",
                          "value": v, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * tt / args.steps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
                          "cpu_baseline": {"value": v, "unit": "GB/s", "cores": len(arrays), "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import synth
    import paper_1711_03888_gb300 as sz

    snap = synth.cosmology(n, halos, rank_snapshot_seed(rank), device="cuda")
    xs = [snap[f] for f in FIELDS]
    raw_bytes = 4 * n * len(xs)
    ctx = sz.Context(local)
    if args.no_autotune:
        # the fixed chunk-size rule; the autotuner's own trials are timings,
        # which a profiler that serialises launches would distort
        sz.sz_ctx_set_autotune(ctx, False)
    outs = [torch.empty(sz.sz_max_compressed_bytes(n), dtype=torch.uint8, device="cuda") for _ in xs]
    ys = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in xs]
    stream = torch.cuda.current_stream()

    lcf_params = sz._params(predictor=sz.SZ_PRED_LCF)

    def step(ev_mid=None, plain=False, lcf=False):
        # fully asynchronous: the decoder reads each stream's size from its
        # header, so in_bytes is the buffer capacity and no host sync is needed.
        # The snapshot's six fields go through the batched form (one persistent
        # launch replayed as a CUDA graph); plain=True uses one sz_compress per
        # field; lcf=True the same with the LCF predictor.
        if plain:
            prm = lcf_params if lcf else None
            holders = [sz.sz_compress(ctx, x, args.eb, sz.SZ_EB_REL, prm, o)[1] for x, o in zip(xs, outs)]
        else:
            _, nb = sz.sz_compress_batch(ctx, xs, [args.eb] * len(xs), sz.SZ_EB_REL, outs=outs)
            holders = [_Holder(nb, i) for i in range(len(xs))]
        if ev_mid is not None:
            ev_mid.record(stream)
        if plain:
            for o, y in zip(outs, ys):
                sz.sz_decompress(ctx, o, o.numel(), y)
        else:
            sz.sz_decompress_batch(ctx, outs, [o.numel() for o in outs], ys)
        return holders

    # correctness guard on the benchmarked configuration: max error <= eb_abs
    holders = step()
    sz.sz_sync(ctx)
    sizes = [h.value for h in holders]
    for x, y in zip(xs, ys):
        fin = torch.isfinite(x)
        R = (x[fin].max().double() - x[fin].min().double()).item()
        err = (x.double() - y.double()).abs().max().item()
        assert err <= args.eb * R * (1 + 1e-12), f"error bound violated: {err} > {args.eb * R}"
    ratio = raw_bytes / sum(sizes)

    tuning = sz.sz_batch_tuning(ctx, n)     # the autotuner ran on the guard call (first sight)

    clocks = ClockSampler(local)
    clocks.start()            # sampling from the warm-up through the timed regions
    for _ in range(args.warmup):
        step()
        sz.sz_sync(ctx)
    torch.cuda.synchronize()
    # ---- headline: the product's calls as a user makes them -- the batch's CUDA
    # graph replay and the batched decoder -- with no tracing; CUDA events on
    # the stream around the compress half and the decompress half of each step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    _barrier(ws)
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        holders = step(ev[i][1])
        ev[i][2].record(stream)
    sz.sz_sync(ctx)
    sizes = [h.value for h in holders]
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    _barrier(ws)
    tc_steps = [e[0].elapsed_time(e[1]) / 1e3 for e in ev]
    td_steps = [e[1].elapsed_time(e[2]) / 1e3 for e in ev]
    t_c = sum(tc_steps)
    t_d = sum(td_steps)
    t_step = (t_c + t_d) / args.steps
    value, t_step_max, total_bytes = weak_scaling_value(raw_bytes, t_step, ws)
    comp_gbs = raw_bytes / (t_c / args.steps) / 1e9
    decomp_gbs = raw_bytes / (t_d / args.steps) / 1e9
    stats = {"timing": "CUDA events on the stream, graph replay (no tracing), per step",
             "compress_ms": _stats_ms(tc_steps), "decompress_ms": _stats_ms(td_steps),
             "step_ms": _stats_ms([a + b for a, b in zip(tc_steps, td_steps)])}
    stats["compress_gbs_best"] = raw_bytes / (stats["compress_ms"]["best"] / 1e3) / 1e9
    stats["decompress_gbs_best"] = raw_bytes / (stats["decompress_ms"]["best"] / 1e3) / 1e9
    stats["round_trip_gbs_median"] = raw_bytes / (stats["step_ms"]["median"] / 1e3) / 1e9

    # ---- breakdown: the same steps traced, each kernel between two events on
    # the step's stream (the batch's graph work then runs as direct launches
    # of the same kernels in the same order)
    sz.sz_profile_enable(ctx, True)
    evt = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        evt[i][0].record(stream)
        step()
        evt[i][1].record(stream)
    sz.sz_sync(ctx)
    torch.cuda.synchronize()
    prof = sz.sz_profile_read(ctx)
    sz.sz_profile_enable(ctx, False)
    clk = clocks.stop()
    traced_step_ms = _stats_ms([a.elapsed_time(b) for a, b in evt])

    # ---- the per-array (plain) path on the same arrays, for comparison ------------
    for _ in range(2):
        step(plain=True)
        sz.sz_sync(ctx)
    evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    sz.sz_profile_enable(ctx, True)     # per-kernel times of the stand-alone launches
    for i in range(args.steps):
        evp[i][0].record(stream)
        step(evp[i][1], plain=True)
        evp[i][2].record(stream)
    sz.sz_sync(ctx)
    torch.cuda.synchronize()
    prof_plain = sz.sz_profile_read(ctx)
    sz.sz_profile_enable(ctx, False)
    tp_c = sum(e[0].elapsed_time(e[1]) for e in evp) / 1e3 / args.steps
    tp_d = sum(e[1].elapsed_time(e[2]) for e in evp) / 1e3 / args.steps
    plain = {"compress_gbs": raw_bytes / tp_c / 1e9, "decompress_gbs": raw_bytes / tp_d / 1e9,
             "round_trip_gbs": raw_bytes / (tp_c + tp_d) / 1e9,
             "note": "per field: sz_compress (4 launches) and sz_decompress (2 launches), instead of the "
                     "batched graph and the batched decoder"}

    # ---- the LCF predictor (Sec. IV-A, original SZ) on the same arrays ---------
    lcf = None
    if not args.no_lcf:
        lcf = lcf_bench(sz, ctx, stream, step, xs, ys, outs, args, raw_bytes, ratio,
                        with_cpu=not args.no_cpu and rank == 0 and ws == 1)

    # ---- roofline of the dominant kernel -----------------------------------
    peak, peak_kind = _peaks()
    stream_bytes = sum(sizes)
    # algorithmic bytes per launch: what each launch must move given the pass
    # structure.  Per array of n elements: range reads 4n; quantize reads 4n and
    # writes 2n codes; encode reads the 2n codes and writes the stream; decode
    # reads the stream and writes 4n.  The batch graph covers all six arrays.
    per_stream = stream_bytes / len(xs)
    # Per step: the plain path runs one launch per array and phase; the batched
    # step's per-phase kernels (range_multi, quant_multi, encode_multi,
    # decode_multi) run one launch over all six arrays.
    k6 = len(xs)
    algo_plain = {"range": 4 * n * k6, "quant": 6 * n * k6, "encode": 2 * n * k6 + stream_bytes,
                  "decode": stream_bytes + 4 * n * k6}
    algo_batched = dict(algo_plain)
    kernel_multi = {"range": "range_multi_kernel", "quant": "quant_multi_kernel", "encode": "encode_multi_kernel",
                    "decode": "decode_multi_kernel"}
    kernel_of = {"encode": "encode_kernel", "decode": "decode_kernel", "quant": "quant_kernel",
                 "range": "range_kernel", "codebook": "codebook_kernel", "decode_setup": "decode_setup_kernel"}

    def kernel_table(pr, steps, algo_step):
        """Per phase: launches, average launch time, time per step and the
        achieved rate of its algorithmic bytes (algo_step: bytes per step,
        spread evenly over the phase's launches in a step)."""
        tot = sum(v[1] for v in pr.values()) or 1.0
        out = {}
        for ph, (cnt, ms) in pr.items():
            if cnt == 0:
                continue
            avg = ms / cnt / 1e3
            e = {"launches": cnt, "avg_ms": 1e3 * avg, "ms_per_step": ms / steps, "share": ms / tot}
            if ph in algo_step:
                per_launch = algo_step[ph] * steps / cnt
                e["algorithmic_bytes_per_launch"] = per_launch
                e["achieved_gbs"] = per_launch / avg / 1e9
                e["frac"] = e["achieved_gbs"] / peak
            out[ph] = e
        return out

    # The encode step may run as two kernels (chunk sizes, then packing): its
    # row times both against the step's algorithmic bytes (codes read once,
    # stream written); the passes are also listed apart.
    prof_raw = prof
    two_pass = prof.get("encode_sizes", (0, 0.0))[0] > 0
    encode_passes = None
    if two_pass:
        encode_passes = {"sizes_ms_per_step": prof["encode_sizes"][1] / args.steps,
                         "pack_ms_per_step": prof["encode"][1] / args.steps}
        prof = dict(prof)
        prof["encode"] = (prof["encode"][0], prof["encode"][1] + prof["encode_sizes"][1])
        prof["encode_sizes"] = (0, 0.0)
        kernel_multi["encode"] = "encode_sizes_multi_kernel + encode_pack_multi_kernel"
    kernels = kernel_table(prof, args.steps, algo_batched)
    if encode_passes:
        kernels["encode"]["passes"] = encode_passes
    pp = dict(prof_plain)
    if pp.get("encode_sizes", (0, 0.0))[0]:
        pp["encode"] = (pp["encode"][0], pp["encode"][1] + pp["encode_sizes"][1])
        pp["encode_sizes"] = (0, 0.0)
    kernels_plain = kernel_table(pp, args.steps, algo_plain)
    for ph, kname in kernel_multi.items():
        if ph in kernels:
            kernels[ph]["ncu"] = ncu_dram_rate(kname, peak)
    # The bytes the pass structure forces, per step: with a relative bound the
    # range and quantize passes each read the input, the u16 codes go out and
    # back, and the stream is written; decompression reads the stream and
    # writes the floats.
    dep_c, dep_d = 12 * n * k6 + stream_bytes, stream_bytes + 4 * n * k6
    dependency = {"compress_bytes_per_step": dep_c, "decompress_bytes_per_step": dep_d,
                  "compress_gbs": dep_c / (t_c / args.steps) / 1e9,
                  "decompress_gbs": dep_d / (t_d / args.steps) / 1e9}
    dependency["compress_frac"] = dependency["compress_gbs"] / peak
    dependency["decompress_frac"] = dependency["decompress_gbs"] / peak
    # The dominant single kernel of the batched step by device time per step.
    # While tracing is on, the batch's graph work runs as direct launches of the
    # same per-phase kernels, each between two events on the step's stream.
    # (The codebook kernel works on the 2^16-entry histogram whatever n is: a
    # fixed latency, not a bandwidth-bound pass, so it is not a candidate.)
    # The two-pass encoder is two kernels: each is a candidate of its own, the
    # sizes pass with the codes it reads, the packing pass with the codes it
    # reads and the stream it writes.
    single = {}   # phase -> (kernel, avg ms per launch, ms per step, algorithmic bytes per launch)
    for ph in ("range", "quant", "encode", "decode"):
        if ph in kernels:
            single[ph] = (kernel_multi[ph], kernels[ph]["avg_ms"], kernels[ph]["ms_per_step"],
                          kernels[ph]["algorithmic_bytes_per_launch"])
    if two_pass and "encode" in single:
        del single["encode"]
        (cs, ms_s), (cp, ms_p) = prof_raw["encode_sizes"], prof_raw["encode"]
        single["encode_sizes"] = ("encode_sizes_multi_kernel", ms_s / cs, ms_s / args.steps,
                                  2 * n * k6 * args.steps / cs)
        single["encode_pack"] = ("encode_pack_multi_kernel", ms_p / cp, ms_p / args.steps,
                                 algo_batched["encode"] * args.steps / cp)
    dom = max(single, key=lambda ph: single[ph][2])
    kname, avg_ms, _, abytes = single[dom]
    achieved = abytes / (avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": _traffic(kname),
                "algorithmic_bytes_per_launch": abytes,
                "avg_launch_ms": avg_ms,
                "timing": "CUDA events around each launch on its stream, inside the timed region"}
    # kernels launched in the timed region: one per traced launch, plus the
    # batched decoder's unit scan, which shares the setup phase's event pair
    launches = sum(c for c, _ in prof_raw.values()) + prof_raw.get("decode_setup", (0, 0.0))[0]

    # ---- end to end through host buffers ------------------------------------
    e2e = None
    if not args.no_e2e:
        hx = [x.cpu().pin_memory() for x in xs]
        hs = [torch.empty(sz.sz_max_compressed_bytes(n), dtype=torch.uint8).pin_memory() for _ in xs]
        hy = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in xs]
        h2d = d2h = 0

        def e2e_step():
            nonlocal h2d, d2h
            _, _, nb = sz.sz_compress_host(ctx, hx, [args.eb] * len(hx), sz.SZ_EB_REL, outs=hs)
            _, n_out = sz.sz_decompress_host(ctx, hs, nb, hy)
            h2d = 4 * sum(x.numel() for x in hx) + sum(nb)
            d2h = sum(nb) + 4 * sum(n_out)

        for _ in range(max(3, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        _barrier(ws)
        # every call is synchronous, so each step's wall time is its own; the
        # value is the mean over the steps (the list shows host-side outliers)
        k2 = max(1, min(args.steps, 10))
        step_ms = []
        t0 = time.perf_counter()
        for _ in range(k2):
            ts = time.perf_counter()
            e2e_step()
            step_ms.append(1e3 * (time.perf_counter() - ts))
        torch.cuda.synchronize()
        te = _max_over_ranks((time.perf_counter() - t0) / k2, ws)
        assert np.array_equal(hy[0][: 1 << 16].numpy().view(np.uint32), ys[0][: 1 << 16].cpu().numpy().view(np.uint32))
        e2e = {"value": total_bytes / te / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * te, "step_ms": [round(v, 2) for v in step_ms],
               "stats_ms": _stats_ms([v / 1e3 for v in step_ms]),
               "gbs_median_step": raw_bytes / (float(np.median(step_ms)) / 1e3) / 1e9,
               "link": link_rates(hx, hy)}
        del hx, hs, hy

    # ---- the workload's other bounds (1e-3, 1e-5) on the same arrays ------------
    bounds = None
    if not args.no_bounds:
        bounds = bounds_bench(sz, ctx, stream, xs, ys, outs, raw_bytes, max(3, min(args.steps, 5)), peak)

    # ---- the small plain snapshot (2^20 x 6) -------------------------------------
    small = None
    if rank == 0 and not args.no_small:
        small = small_bench(sz, local, args.eb, args.steps, peak)

    # ---- batched form (rank 0): 768 uneven arrays, one graph vs 768 calls --------
    batched = None
    if rank == 0 and not args.no_batched:
        batched = batched_bench(sz, local, args.steps)

    # ---- MD snapshot (rank 0): reordering modes ---------------------------------
    md = None
    if rank == 0 and not args.no_md:
        md = md_bench(sz, local, args.steps, with_cpu=not args.no_cpu and ws == 1)

    # ---- R-index keys from coordinates / velocities (rank 0; Table 6) -------------
    rkeys = None
    if rank == 0 and not args.no_rkeys:
        rkeys = rkeys_bench(sz, local, args.steps)

    # ---- rate-distortion sweep (rank 0; Fig. 9) ----------------------------------
    rd = None
    if rank == 0 and not args.no_rd:
        rd = rd_bench(sz, local, xs)

    # ---- served form (rank 0): Poisson arrivals vs the same requests serially --
    served = None
    if rank == 0 and not args.no_serve:
        served = served_bench(sz, snap, args.eb, args.serve_rate, args.serve_seconds, args.serve_stress,
                              args.serve_stress_seconds, args.serve_slots, args.serve_budget_gb, local)

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only) -----------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        arrays = cpu_sample(snap, 1 << args.cpu_log2n)
        t, b = oracle_round_trip(arrays, args.eb)
        cpu = {"value": b / t / 1e9, "unit": "GB/s", "cores": len(arrays), "kind": "oracle",
               "sample": f"first 2^{args.cpu_log2n} elements of each of the 6 fields, compress + decompress, "
                         f"one thread per field",
               "wall_s": t, "cpu_seconds_approx": t * len(arrays)}

    if rank == 0:
        line = {
            "metric": "round-trip (compress+decompress) throughput, uncompressed float32",
            "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
            "compress_gbs": comp_gbs, "decompress_gbs": decomp_gbs,
            "compress_frac_hbm": comp_gbs / peak, "decompress_frac_hbm": decomp_gbs / peak,
            "dependency_bytes": dependency,
            "ratio": ratio, "stats": stats, "traced_step_ms": traced_step_ms, "tuning": tuning,
            "roofline": roofline, "kernels": kernels, "kernels_plain_path": kernels_plain,
            "gpu_launches": launches, "other_bounds": bounds, "small_snapshot": small,
            "plain_path": plain, "lcf": lcf, "batched": batched, "md": md, "rkeys": rkeys, "rd": rd,
            "served": served,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "wall_s_timed": t_wall,
        }
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
