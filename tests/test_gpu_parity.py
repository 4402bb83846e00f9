"""GPU parity: the CUDA path, called through the C ABI, against the CPU
oracle on the same seeded inputs.  Integer/byte work must be bit-exact: the
compressed stream must equal the oracle's byte for byte, and the
reconstruction must equal the oracle's bit for bit (which implies the error
bound |x - x'| <= eb_abs the oracle pins establish)."""
import heapq

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sz():
    import __graft_entry__ as g
    g.build()
    import paper_1711_03888_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(sz):
    c = sz.Context(0)
    yield c
    c.close()


def _gpu_stream(sz, ctx, x_cpu, eb, kind, chunk):
    x = x_cpu.cuda()
    out, nb = sz.sz_compress(ctx, x, eb, kind, sz._params(chunk))
    sz.sz_sync(ctx)
    return out[: nb.value].cpu().numpy().tobytes()


def _gpu_decode(sz, ctx, stream_bytes, n):
    buf = torch.frombuffer(bytearray(stream_bytes), dtype=torch.uint8).cuda()
    out = torch.full((max(n, 1),), float("nan"), dtype=torch.float32, device="cuda")
    no = sz.sz_decompress(ctx, buf, len(stream_bytes), out, n)
    sz.sz_sync(ctx)
    assert no.value == n
    return out[:n].cpu().numpy()


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _check(sz, ctx, oracle, x_cpu, eb, kind, chunk):
    x_cpu = x_cpu.contiguous()
    ref = oracle.compress(x_cpu.numpy(), eb, kind, chunk, chunk // 64)
    got = _gpu_stream(sz, ctx, x_cpu, eb, kind, chunk)
    if got != ref:
        h1, h2 = oracle.parse_header(got) if len(got) >= 160 else {}, oracle.parse_header(ref)
        diff = next((i for i in range(min(len(got), len(ref))) if got[i] != ref[i]), None)
        raise AssertionError(f"stream mismatch: len {len(got)} vs {len(ref)}, first diff at byte {diff}, "
                             f"gpu header {h1}, oracle header {h2}")
    yr = oracle.decompress(ref)
    yg = _gpu_decode(sz, ctx, ref, x_cpu.numel())
    assert np.array_equal(_bits(yg), _bits(yr))
    return ref


CASES = [
    ("walk", 1, 2048), ("walk", 3, 2048), ("walk", 100, 2048), ("walk", 2047, 2048), ("walk", 2048, 2048),
    ("walk", 2049, 2048), ("walk", 3 * 4096 + 17, 4096), ("walk", 70001, 8192), ("walk", 16384 * 5 + 1, 16384),
    ("uniform", 50000, 4096), ("cosmo_xx", 1 << 16, 4096), ("cosmo_vy", 1 << 16, 8192),
    ("md_zz", 60000, 8192), ("wild", 30000, 2048), ("spiky", 40000, 4096), ("const", 5000, 2048),
]


def _make(kind, n):
    if kind == "walk":
        return synth.random_walk_f32(n, 21)
    if kind == "uniform":
        return synth.uniform_f32(n, 6, -3.0, 5.0)
    if kind.startswith("cosmo"):
        return synth.cosmology(n, 8, 1)[kind.split("_")[1]]
    if kind.startswith("md"):
        return synth.md_fcc(cells=25, seed=2)[kind.split("_")[1]][:n].clone()
    if kind == "wild":
        w = synth.uniform_f32(n, 7, -1e30, 1e30).numpy().copy()
        w[::97] = np.nan
        w[5::211] = np.inf
        w[7::223] = -np.inf
        w[9::50] = np.float32(1e-42)
        w[11::50] = -0.0
        return torch.from_numpy(w)
    if kind == "spiky":
        x = synth.random_walk_f32(n, 8, 1e-3).numpy().copy()
        x[::777] = 1e6
        return torch.from_numpy(x)
    if kind == "const":
        return torch.full((n,), 2.5, dtype=torch.float32)
    raise ValueError(kind)


@pytest.mark.parametrize("kind,n,chunk", CASES)
@pytest.mark.parametrize("eb", [1e-3, 1e-5])
def test_stream_parity_relative(sz, ctx, oracle, kind, n, chunk, eb):
    _check(sz, ctx, oracle, _make(kind, n), eb, 1, chunk)


@pytest.mark.parametrize("eb_abs", [0.0, 1e-7, 0.05, 3.0])
def test_stream_parity_absolute(sz, ctx, oracle, eb_abs):
    _check(sz, ctx, oracle, _make("walk", 30000), eb_abs, 0, 4096)
    _check(sz, ctx, oracle, _make("spiky", 30000), eb_abs, 0, 2048)


def _degenerate(kind, n):
    i = np.arange(n)
    if kind == "all_nan":
        return np.full(n, np.nan, np.float32)
    if kind == "all_inf":
        return np.where(i % 2 == 0, np.inf, -np.inf).astype(np.float32)
    if kind == "nan_payloads":      # quiet and signalling NaNs of both signs, distinct payloads
        bits = np.where(i % 2 == 0, 0x7FC00000, 0xFF800000).astype(np.uint32) | ((i % 4093) + 1).astype(np.uint32)
        return bits.view(np.float32)
    if kind == "two_values":
        return np.where(i % 3 == 0, 1.0, -1.0).astype(np.float32)
    if kind == "one_finite":        # the value range is one point among non-finite values
        x = np.full(n, np.nan, np.float32)
        x[n // 2] = 7.25
        return x
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["all_nan", "all_inf", "nan_payloads", "two_values", "one_finite"])
@pytest.mark.parametrize("n", [1, 7, 2049, 9000])
@pytest.mark.parametrize("eb,ek", [(1e-4, 1), (1e-3, 0)])
def test_degenerate_arrays(sz, ctx, oracle, kind, n, eb, ek):
    """Arrays without a finite value range (every value NaN or infinite, or one
    finite value among them), NaN payloads, and a two-symbol codebook: the
    stream equals the oracle's and the decode is bit-exact, NaN payloads included."""
    x = torch.from_numpy(_degenerate(kind, n))
    ref = _check(sz, ctx, oracle, x, eb, ek, 2048)
    if kind != "two_values":
        # stored raw: the decode reproduces every input bit, NaN payloads included
        assert oracle.parse_header(ref)["flags"] == 1
        assert np.array_equal(_bits(oracle.decompress(ref)), _bits(x.numpy()))


def test_empty_array(sz, ctx, oracle):
    x = torch.zeros(0, dtype=torch.float32)
    ref = oracle.compress(x.numpy(), 1e-4, 1, 2048, 32)
    got = _gpu_stream(sz, ctx, x, 1e-4, 1, 2048)
    assert got == ref and len(got) == 160
    assert _gpu_decode(sz, ctx, ref, 0).size == 0


def test_near_ties_and_large_lattice(sz, ctx, oracle):
    """Values on and next to lattice half-points exercise the binary64 slow
    path; values with |q| > 2^22 exercise the out-of-range candidate path."""
    D = 2.0 ** -8
    k = np.arange(-20000, 20000)
    halves = ((k + 0.5) * D).astype(np.float32)
    nxt = np.nextafter(halves, np.float32(np.inf))
    prv = np.nextafter(halves, np.float32(-np.inf))
    x = np.stack([halves, nxt, prv], 1).ravel()
    _check(sz, ctx, oracle, torch.from_numpy(x), D / 2, 0, 4096)
    big = (1000.0 + np.cumsum(np.random.default_rng(8).normal(0, 1e-4, 20000))).astype(np.float32)
    _check(sz, ctx, oracle, torch.from_numpy(big), 1e-6, 0, 4096)
    _check(sz, ctx, oracle, torch.from_numpy(big), 1e-9, 0, 4096)


def test_unaligned_input(sz, ctx, oracle):
    base = _make("walk", 20001)
    for off in (1, 2, 3):
        x = base.cuda()[off:]
        ref = oracle.compress(base[off:].numpy(), 1e-4, 1, 2048, 32)
        out, nb = sz.sz_compress(ctx, x, 1e-4, 1, sz._params(2048))
        sz.sz_sync(ctx)
        assert out[: nb.value].cpu().numpy().tobytes() == ref
    # the batched kernels take the unaligned views through their global-memory loop
    offs = (1, 2, 3)
    outs, nb = sz.sz_compress_batch(ctx, [base.cuda()[off:] for off in offs], [1e-4] * 3, 1)
    sz.sz_sync(ctx)
    for i, off in enumerate(offs):
        got = outs[i][: nb[i]].cpu().numpy().tobytes()
        h = oracle.parse_header(got)
        assert got == oracle.compress(base[off:].numpy(), 1e-4, 1, h["chunk"], h["sub"])


def test_decoder_reads_oracle_streams_and_reuse(sz, ctx, oracle):
    """Several calls back to back on one context reuse the workspace."""
    for seed in range(4):
        x = synth.random_walk_f32(10000 + 999 * seed, seed)
        _check(sz, ctx, oracle, x, 10.0 ** -(2 + seed), 1, 2048)


def test_capacity_error_reports_size(sz, ctx, oracle):
    x_cpu = _make("walk", 50000)
    ref = oracle.compress(x_cpu.numpy(), 1e-4, 1, 4096, 64)
    x = x_cpu.cuda()
    for cap in (100, 1000, len(ref) - 16):
        out = torch.full((len(ref) + 4096,), 0xAB, dtype=torch.uint8, device="cuda")
        _, nb = sz.sz_compress(ctx, x, 1e-4, 1, sz._params(4096), out=out, out_cap=cap)
        st = sz.sz_sync(ctx, check=False)
        assert st == sz.SZ_ERR_CAPACITY
        assert nb.value == len(ref)
        assert (out[cap:].cpu().numpy() == 0xAB).all()       # nothing written past the cap
    out = torch.empty(len(ref), dtype=torch.uint8, device="cuda")
    _, nb = sz.sz_compress(ctx, x, 1e-4, 1, sz._params(4096), out=out)
    sz.sz_sync(ctx)
    assert out.cpu().numpy().tobytes() == ref
    small = torch.empty(10, dtype=torch.float32, device="cuda")
    buf = torch.frombuffer(bytearray(ref), dtype=torch.uint8).cuda()
    no = sz.sz_decompress(ctx, buf, len(ref), small, 10)
    assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_CAPACITY and no.value == 50000


def test_corrupt_streams_are_rejected(sz, ctx, oracle):
    x_cpu = _make("cosmo_vx", 1 << 15)
    ref = bytearray(oracle.compress(x_cpu.numpy(), 1e-4, 1, 2048, 32))
    h = oracle.parse_header(bytes(ref))
    out = torch.empty(1 << 15, dtype=torch.float32, device="cuda")

    def run(buf, nbytes=None):
        t = torch.frombuffer(bytearray(buf), dtype=torch.uint8).cuda()
        sz.sz_decompress(ctx, t, len(buf) if nbytes is None else nbytes, out, out.numel())
        return sz.sz_sync(ctx, check=False)

    assert run(ref) == sz.SZ_OK
    assert run(ref, 100) == sz.SZ_ERR_CORRUPT                  # truncated below the header
    assert run(ref, len(ref) - 16) == sz.SZ_ERR_CORRUPT        # truncated payload
    bad = bytearray(ref); bad[0] ^= 1
    assert run(bad) == sz.SZ_ERR_CORRUPT                       # magic
    bad = bytearray(ref); bad[h["off_lens"]] = 30
    assert run(bad) == sz.SZ_ERR_CORRUPT                       # code length > 24
    bad = bytearray(ref); bad[h["off_chunk_word"] + 8 * 3: h["off_chunk_word"] + 8 * 4] = (1 << 50).to_bytes(8, "little")
    assert run(bad) == sz.SZ_ERR_CORRUPT                       # chunk offset out of range
    bad = bytearray(ref); bad[h["off_sublen"]: h["off_sublen"] + 2] = (60000).to_bytes(2, "little")
    assert run(bad) == sz.SZ_ERR_CORRUPT                       # sub-stream length inconsistent
    for E in ((1 << 60) + 5, (1 << 64) - 1, (1 << 15) + 1):
        # an escape count whose record size would wrap, or beyond the element count:
        # rejected by the header check before any chunk is decoded
        bad = bytearray(ref); bad[64:72] = E.to_bytes(8, "little")
        assert run(bad) == sz.SZ_ERR_CORRUPT
    rng = np.random.default_rng(1)
    for trial in range(8):                                      # random payload damage: no fault, no hang
        bad = bytearray(ref)
        pos = rng.integers(h["off_payload"], len(ref), 64)
        for p in pos:
            bad[p] = rng.integers(0, 256)
        assert run(bad) in (sz.SZ_OK, sz.SZ_ERR_CORRUPT)
    assert run(ref) == sz.SZ_OK


def test_batch_equals_plain(sz, ctx, oracle):
    xs = [synth.random_walk_f32(n, i) for i, n in enumerate([1, 5000, 2048, 123457, 0, 70000])]
    ebs = [1e-3, 1e-4, 1e-2, 1e-5, 1e-4, 1e-3]
    outs, nb = sz.sz_compress_batch(ctx, [x.cuda() for x in xs], ebs, 1)
    sz.sz_sync(ctx)
    for i, x in enumerate(xs):
        got = outs[i][: nb[i]].cpu().numpy().tobytes()
        h = oracle.parse_header(got)
        ref = oracle.compress(x.numpy(), ebs[i], 1, h["chunk"], h["sub"])
        assert got == ref
    bufs = [outs[i][: nb[i]] for i in range(len(xs))]
    ys = [torch.empty(max(x.numel(), 1), dtype=torch.float32, device="cuda") for x in xs]
    no = sz.sz_decompress_batch(ctx, bufs, [nb[i] for i in range(len(xs))], ys)
    sz.sz_sync(ctx)
    for i, x in enumerate(xs):
        assert no[i] == x.numel()
        yr = oracle.decompress(outs[i][: nb[i]].cpu().numpy().tobytes())
        assert np.array_equal(_bits(ys[i][: x.numel()].cpu().numpy()), _bits(yr))


def _rebuilds_needed(freq, limit=24):
    """How many times the (w >> 1) | 1 rescaling must run before the prefix
    tree of `freq` is at most `limit` deep (tree built by always merging the
    two lightest nodes, leaves before internal nodes on equal weight)."""
    f = sorted(int(v) for v in freq)
    k = 0
    while True:
        heap = [(w, 0, i, 0) for i, w in enumerate(f)]
        heapq.heapify(heap)
        made = 0
        while len(heap) > 1:
            a, b = heapq.heappop(heap), heapq.heappop(heap)
            heapq.heappush(heap, (a[0] + b[0], 1, made, max(a[3], b[3]) + 1))
            made += 1
        if heap[0][3] <= limit:
            return k
        f = sorted((w >> 1) | 1 for w in f)
        k += 1


@pytest.mark.parametrize("scale,rebuilds", [(1, 1), (3, 3), (6, 4), (12, 5), (48, 7)])
def test_length_limit_rebuilds(sz, ctx, oracle, scale, rebuilds):
    """Step histograms that grow like Fibonacci numbers force the 24-bit code
    length limit to rescale the counts several times (the Huffman stage,
    Sec. II / IV-B): one to seven rebuilds.  Plain and batched compression must give
    the oracle's stream byte for byte."""
    x = synth.skewed_steps_f32(26, scale)
    _, cnt = np.unique(np.diff(x.numpy()), return_counts=True)
    assert _rebuilds_needed(cnt) == rebuilds
    ref = _check(sz, ctx, oracle, x, 0.5, 0, 4096)
    syms, lens = oracle.stream_codebook(ref)
    assert lens.max() <= 24 and syms.size == 26
    outs, nb = sz.sz_compress_batch(ctx, [x.cuda(), synth.random_walk_f32(9000, 3).cuda()], [0.5, 1e-3], 0)
    sz.sz_sync(ctx)
    got = outs[0][: nb[0]].cpu().numpy().tobytes()
    hg = oracle.parse_header(got)
    assert got == oracle.compress(x.numpy(), 0.5, 0, hg["chunk"], hg["sub"])


@pytest.mark.parametrize("field", ["xx", "vz"])
def test_full_size_large_cosmology_array(sz, ctx, oracle, field):
    """One array of the large cosmology snapshot (2^27 particles, 4096 halos)
    at the size and launch configuration the benchmark uses."""
    snap = synth.cosmology(1 << 27, 4096, 3, device="cuda")
    x = snap[field]
    del snap
    out, nb = sz.sz_compress(ctx, x, 1e-4, 1)
    sz.sz_sync(ctx)
    got = out[: nb.value].cpu().numpy().tobytes()
    x_cpu = x.cpu()
    h = oracle.parse_header(got)
    ref = oracle.compress(x_cpu.numpy(), 1e-4, 1, h["chunk"], h["sub"])
    assert got == ref
    y = torch.empty_like(x)
    sz.sz_decompress(ctx, out[: nb.value], nb.value, y)
    sz.sz_sync(ctx)
    yr = oracle.decompress(ref)
    assert np.array_equal(_bits(y.cpu().numpy()), _bits(yr))
