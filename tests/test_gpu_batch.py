"""GPU parity of the batched form (one persistent launch over many arrays):
every array's stream must be byte-identical to sz_compress on that array
(and to the oracle), whatever the mix of sizes, bounds and degenerate cases."""
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


def _plain(sz, ctx, x, eb, kind, chunk=0):
    out, nb = sz.sz_compress(ctx, x, eb, kind, sz._params(chunk))
    sz.sz_sync(ctx)
    return out[: nb.value].cpu().numpy().tobytes()


def _chunk_of(stream):
    # the chunk size a stream was made with (the batched form's autotuner picks it)
    import struct
    return struct.unpack_from("<I", stream, 32)[0] if len(stream) >= 160 else 0


def _batch(sz, ctx, xs, ebs, kind):
    outs, nb = sz.sz_compress_batch(ctx, xs, ebs, kind)
    sz.sz_sync(ctx)
    return [outs[i][: nb[i]].cpu().numpy().tobytes() for i in range(len(xs))]


def _edge_arrays():
    rng = np.random.default_rng(3)
    xs = []
    for n in [0, 1, 5, 2047, 2049, 70001, 200000, 65536, 65537]:
        xs.append(synth.random_walk_f32(n, int(rng.integers(1 << 20))))
    xs.append(torch.full((9000,), 7.0, dtype=torch.float32))           # R = 0: raw
    w = synth.uniform_f32(30000, 7, -1e30, 1e30).numpy().copy()
    w[::97] = np.nan
    w[5::211] = np.inf
    xs.append(torch.from_numpy(w))                                    # NaN / Inf
    s = synth.random_walk_f32(40000, 8, 1e-3).numpy().copy()
    s[::777] = 1e6
    xs.append(torch.from_numpy(s))                                    # escapes
    xs.append(synth.uniform_f32(1 << 15, 9, -1.0, 1.0))               # raw by the size rule at tiny eb
    return xs


def test_batch_edge_mix_matches_oracle(sz, ctx, oracle):
    xs = _edge_arrays()
    ebs = [1e-3, 1e-4, 1e-2, 1e-5, 1e-4, 1e-3, 1e-4, 1e-3, 1e-4, 1e-4, 1e-4, 1e-6, 1e-9]
    for kind in (sz.SZ_EB_REL, sz.SZ_EB_ABS):
        got = _batch(sz, ctx, [x.cuda() for x in xs], ebs, kind)
        for x, e, g in zip(xs, ebs, got):
            h = oracle.parse_header(g)
            assert g == oracle.compress(x.numpy(), e, kind, h["chunk"], h["sub"])


def test_batch_repeated_calls_and_shapes(sz, ctx):
    """The pool is reused across calls and re-laid out for new shapes."""
    a = [synth.random_walk_f32(n, n).cuda() for n in (3000, 500000, 12345)]
    b = [synth.random_walk_f32(n, n + 1).cuda() for n in (70000, 10, 999999, 4096, 1)]
    for xs in (a, a, b, a, b):
        ebs = [1e-4] * len(xs)
        got = _batch(sz, ctx, xs, ebs, sz.SZ_EB_REL)
        assert got == [_plain(sz, ctx, x, 1e-4, sz.SZ_EB_REL, _chunk_of(g)) for x, g in zip(xs, got)]


def test_batch_full_config_many_ranks(sz, ctx, oracle):
    """The batched workload: 128 simulated ranks x 6 fields, sizes 2^14..2^24,
    relative bounds from {1e-3, 1e-4}.  Every stream equals the plain path's;
    a sample is checked against the oracle."""
    arrays = synth.batch_ranks(device="cuda")
    xs = [t for _, _, t, _ in arrays]
    ebs = [e for _, _, _, e in arrays]
    assert len(xs) == 768
    got = _batch(sz, ctx, xs, ebs, sz.SZ_EB_REL)
    for x, e, g in zip(xs, ebs, got):
        assert g == _plain(sz, ctx, x, e, sz.SZ_EB_REL, _chunk_of(g))
    rng = np.random.default_rng(0)
    for i in rng.choice(768, 6, replace=False):
        h = oracle.parse_header(got[i])
        assert got[i] == oracle.compress(xs[i].cpu().numpy(), ebs[i], 1, h["chunk"], h["sub"])
    # batched decompression of all 768 streams equals the per-stream decoder
    bufs = [torch.frombuffer(bytearray(g), dtype=torch.uint8).cuda() for g in got]
    ys = [torch.empty(max(x.numel(), 1), dtype=torch.float32, device="cuda") for x in xs]
    no = sz.sz_decompress_batch(ctx, bufs, [len(g) for g in got], ys)
    assert sz.sz_sync(ctx) == sz.SZ_OK
    for i, x in enumerate(xs):
        assert no[i] == x.numel()
        assert ys[i][: x.numel()].cpu().numpy().tobytes() == _plain_decode(sz, ctx, bufs[i], x.numel())


def _plain_p(sz, ctx, x, eb, kind, chunk):
    out, nb = sz.sz_compress(ctx, x, eb, kind, sz._params(chunk))
    sz.sz_sync(ctx)
    return out[: nb.value].cpu().numpy().tobytes()


@pytest.mark.parametrize("chunk", [0, 2048, 4096])
def test_batch_large_arrays_per_phase_path(sz, ctx, chunk):
    """Arrays of 2^22 elements and more take one launch per phase over all of
    them, beside the persistent kernel of the small ones; streams still equal
    the plain path's, including a raw (constant) and a NaN-laden large array."""
    L = 1 << 22
    snap = synth.cosmology(L + 777, 64, 21, device="cuda")
    xs = [snap["xx"][:L], snap["vy"], synth.random_walk_f32(5000, 3).cuda(), snap["zz"][: L + 4],
          torch.full((L + 1,), -3.5, dtype=torch.float32, device="cuda"), synth.random_walk_f32(70001, 4).cuda()]
    w = snap["vx"].clone()
    w[::1001] = float("nan")
    w[7::5003] = float("inf")
    xs.append(w)
    ebs = [1e-4, 1e-3, 1e-4, 1e-5, 1e-4, 1e-3, 1e-4]
    outs, nb = sz.sz_compress_batch(ctx, xs, ebs, sz.SZ_EB_REL, sz._params(chunk))
    sz.sz_sync(ctx)
    got = [outs[i][: nb[i]].cpu().numpy().tobytes() for i in range(len(xs))]
    for x, e, g in zip(xs, ebs, got):
        assert g == _plain_p(sz, ctx, x, e, sz.SZ_EB_REL, _chunk_of(g))
    # again, replaying the cached graph on new data in the same buffers
    for x in xs:
        x.copy_(x.flip(0) * 0.5)
    outs, nb = sz.sz_compress_batch(ctx, xs, ebs, sz.SZ_EB_REL, sz._params(chunk), outs=outs)
    sz.sz_sync(ctx)
    for i, (x, e) in enumerate(zip(xs, ebs)):
        g = outs[i][: nb[i]].cpu().numpy().tobytes()
        assert g == _plain_p(sz, ctx, x, e, sz.SZ_EB_REL, _chunk_of(g))


def _plain_decode(sz, ctx, buf, n):
    y = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    no = sz.sz_decompress(ctx, buf, buf.numel(), y, n)
    sz.sz_sync(ctx)
    return y[: no.value].cpu().numpy().tobytes()


def test_batch_decompress_mixed_streams(sz, ctx, oracle):
    """One batched decompression over streams of every chunk size, raw, empty,
    NaN-laden and escape-heavy streams equals the per-stream decoder, and a
    corrupt stream among them fails alone (its neighbours still decode)."""
    snap = synth.cosmology(300000, 32, 5, device="cuda")
    xs, chunks = [], []
    for i, C in enumerate([2048, 4096, 8192, 16384, 0, 0]):
        xs.append(snap[["xx", "yy", "zz", "vx", "vy", "vz"][i]][: 250000 - 7 * i].contiguous())
        chunks.append(C)
    xs.append(torch.full((70001,), 2.5, dtype=torch.float32, device="cuda"))        # raw
    xs.append(torch.empty(0, dtype=torch.float32, device="cuda"))                   # empty
    w = synth.uniform_f32(40000, 7, -1e30, 1e30).numpy().copy()
    w[::97] = np.nan
    xs.append(torch.from_numpy(w).cuda())                                             # NaN / huge range
    s = synth.random_walk_f32(60000, 8, 1e-3).numpy().copy()
    s[::301] = 1e6
    xs.append(torch.from_numpy(s).cuda())                                             # escapes
    chunks += [0, 0, 0, 0]
    streams = []
    for x, C in zip(xs, chunks):
        out, nb = sz.sz_compress(ctx, x, 1e-4, sz.SZ_EB_REL, sz._params(C))
        sz.sz_sync(ctx)
        streams.append(out[: nb.value].clone())
    expect = [_plain_decode(sz, ctx, st, x.numel()) for st, x in zip(streams, xs)]
    ys = [torch.empty(max(x.numel(), 1), dtype=torch.float32, device="cuda") for x in xs]
    no = sz.sz_decompress_batch(ctx, streams, [st.numel() for st in streams], ys)
    assert sz.sz_sync(ctx) == sz.SZ_OK
    for i, x in enumerate(xs):
        assert no[i] == x.numel()
        assert ys[i][: x.numel()].cpu().numpy().tobytes() == expect[i], i
    # sample against the oracle
    for i in (0, 3, 6, 9):
        yr = oracle.decompress(streams[i].cpu().numpy().tobytes())
        assert ys[i][: xs[i].numel()].cpu().numpy().tobytes() == yr.tobytes()
    # a corrupt stream in the middle
    bad = streams[2].clone()
    bad[0] ^= 1
    s2 = streams[:2] + [bad] + streams[3:]
    ys2 = [torch.zeros_like(y) for y in ys]
    no2 = sz.sz_decompress_batch(ctx, s2, [st.numel() for st in s2], ys2)
    assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_CORRUPT
    for i, x in enumerate(xs):
        if i == 2:
            continue
        assert no2[i] == x.numel()
        assert ys2[i][: x.numel()].cpu().numpy().tobytes() == expect[i], i


def test_batch_traced_direct_launches_equal_graph(sz, ctx):
    """With tracing on, the batched form launches its graph's kernels directly
    (for per-kernel timing); streams and results equal the graph replay's."""
    snap = synth.cosmology((1 << 22) + 3, 64, 31, device="cuda")
    xs = [snap["xx"], snap["vy"], synth.random_walk_f32(5000, 3).cuda(), snap["zz"][: 1 << 20].contiguous()]
    ebs = [1e-4, 1e-3, 1e-4, 1e-4]
    outs, nb = sz.sz_compress_batch(ctx, xs, ebs, sz.SZ_EB_REL)
    sz.sz_sync(ctx)
    ref = [outs[i][: nb[i]].cpu().numpy().tobytes() for i in range(len(xs))]
    sz.sz_profile_enable(ctx, True)
    try:
        outs2, nb2 = sz.sz_compress_batch(ctx, xs, ebs, sz.SZ_EB_REL)
        sz.sz_sync(ctx)
        prof = sz.sz_profile_read(ctx)
    finally:
        sz.sz_profile_enable(ctx, False)
    got = [outs2[i][: nb2[i]].cpu().numpy().tobytes() for i in range(len(xs))]
    assert got == ref
    assert prof["range"][0] >= 1 and prof["encode"][0] >= 1      # per-phase launches were timed
    assert ref[2] == _plain(sz, ctx, xs[2], ebs[2], sz.SZ_EB_REL, _chunk_of(ref[2]))


def test_batch_autotuner_picks_measured_chunk_sizes(sz, oracle):
    """Default parameters: the first batch of a size class times every
    candidate chunk size (compress + decompress on the device) and keeps the
    fastest; the streams carry that chunk size and equal the oracle's at it.
    Later calls reuse the cached choice.  With the tuner off the fixed rule
    applies."""
    ctx = sz.Context(0)
    try:
        snap = synth.cosmology((1 << 22) + 5, 64, 41, device="cuda")
        xs = [snap["xx"], snap["vy"][: 1 << 20].contiguous(), snap["zz"][: 30000].contiguous(),
              snap["vx"][: (1 << 21) + 3].contiguous()]
        ebs = [1e-4, 1e-3, 1e-4, 1e-4]
        got = _batch(sz, ctx, xs, ebs, sz.SZ_EB_REL)
        for x, e, g in zip(xs, ebs, got):
            t = sz.sz_batch_tuning(ctx, x.numel())
            assert t["chunk_elems"] in (2048, 4096, 8192, 16384)
            assert t["class"][0] <= x.numel() <= t["class"][1]
            ran = {c: ms for c, ms in t["trial_ms"].items() if ms > 0}
            assert ran and min(ran, key=ran.get) == t["chunk_elems"]     # the fastest trial wins
            assert _chunk_of(g) == t["chunk_elems"]
            C = t["chunk_elems"]
            assert g == oracle.compress(x.cpu().numpy(), e, 1, C, C // 64)
        before = {x.numel(): sz.sz_batch_tuning(ctx, x.numel())["trial_ms"] for x in xs}
        again = _batch(sz, ctx, xs, ebs, sz.SZ_EB_REL)
        assert again == got
        assert before == {x.numel(): sz.sz_batch_tuning(ctx, x.numel())["trial_ms"] for x in xs}
        sz.sz_ctx_set_autotune(ctx, False)
        fixed = _batch(sz, ctx, xs, ebs, sz.SZ_EB_REL)
        for x, g in zip(xs, fixed):
            assert _chunk_of(g) == sz.sz_batch_tuning(ctx, x.numel())["fixed_chunk_elems"]
            assert _chunk_of(g) == (2048 if x.numel() <= 65536 else 4096)
    finally:
        ctx.close()


def test_batch_autotuner_tiles_of_the_persistent_kernel(sz, oracle):
    """Many small arrays run in the persistent kernel: its range-tile and
    quantize-group sizes are tuned too (they change no byte of any stream)."""
    ctx = sz.Context(0)
    try:
        arrays = synth.batch_ranks(device="cuda")[:600]
        xs = [t for _, _, t, _ in arrays]
        ebs = [e for _, _, _, e in arrays]
        got = _batch(sz, ctx, xs, ebs, sz.SZ_EB_REL)
        t = sz.sz_batch_tuning(ctx, xs[0].numel())
        assert (t["range_tile"], t["quant_group"]) in ((1 << 16, 8), (1 << 15, 4), (1 << 17, 8), (1 << 16, 4))
        assert sum(1 for v in t["tile_trial_ms"] if v > 0) >= 2
        rng = np.random.default_rng(1)
        for i in rng.choice(len(xs), 5, replace=False):
            C = _chunk_of(got[i])
            assert got[i] == oracle.compress(xs[i].cpu().numpy(), ebs[i], 1, C, C // 64)
    finally:
        ctx.close()
