"""GPU parity of the LCF predictor (Sec. IV-A, the original SZ's linear curve
fitting on the lattice): streams byte-identical to the oracle's, decoded
arrays bit-identical to the oracle's decoder, through the single and the
batched decoders, the batch and host entry points, and the MD reordering."""
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


def _lcf(sz, chunk=0):
    return sz._params(chunk, predictor=sz.SZ_PRED_LCF)


def _compress(sz, ctx, x, eb, kind, params):
    out, nb = sz.sz_compress(ctx, x.cuda(), eb, kind, params)
    sz.sz_sync(ctx)
    return out[: nb.value].cpu().numpy().tobytes()


def _decompress(sz, ctx, s, n):
    d = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
    y = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    no = sz.sz_decompress(ctx, d, len(s), y)
    sz.sz_sync(ctx)
    assert no.value == n
    return y[:n].cpu().numpy()


def _edge_arrays():
    rng = np.random.default_rng(21)
    xs = [synth.random_walk_f32(n, int(rng.integers(1 << 20)), 0.2) for n in (0, 1, 2, 3, 5, 2047, 2049, 70001)]
    xs.append(torch.full((9000,), 7.0, dtype=torch.float32))          # R = 0: raw
    w = synth.uniform_f32(30000, 7, -1e30, 1e30).numpy().copy()
    w[::97] = np.nan
    w[5::211] = np.inf
    xs.append(torch.from_numpy(w))                                   # NaN / Inf (raw by the size rule)
    s = synth.random_walk_f32(40000, 8, 1e-3).numpy().copy()
    s[::777] = 1e6                                                   # spikes: +J, -2J, +J escapes
    s[100::1001] = np.nan
    xs.append(torch.from_numpy(s))
    t = np.cumsum(np.cumsum(synth.uniform_f32(50000, 9, -1.0, 1.0).numpy().astype(np.float64)))
    xs.append(torch.from_numpy(t.astype(np.float32)))                # smooth: LCF's favourable case
    return xs


@pytest.mark.parametrize("chunk", [0, 2048, 8192, 16384])
def test_lcf_edge_mix_matches_oracle(sz, ctx, oracle, chunk):
    xs = _edge_arrays()
    ebs = [1e-3, 1e-4, 1e-2, 1e-4, 1e-5, 1e-4, 1e-3, 1e-4, 1e-4, 1e-4, 1e-6, 1e-5]
    for kind in (sz.SZ_EB_REL, sz.SZ_EB_ABS):
        for x, e in zip(xs, ebs):
            g = _compress(sz, ctx, x, e, kind, _lcf(sz, chunk))
            h = oracle.parse_header(g)
            assert h["predictor"] == 2
            assert g == oracle.compress(x.numpy(), e, kind, h["chunk"], h["sub"], pred=oracle.PRED_LCF)
            y = _decompress(sz, ctx, g, x.numel())
            assert np.array_equal(y.view(np.uint32), oracle.decompress(g).view(np.uint32))


def test_lcf_full_field_matches_oracle(sz, ctx, oracle):
    """A 2^24-element cosmology field (thousands of chunks, the fast 32-bit
    quantizer path and its carries across warps and chunks)."""
    snap = synth.cosmology(1 << 24, 256, 5)
    for f in ("xx", "vz"):
        x = snap[f]
        g = _compress(sz, ctx, x, 1e-4, sz.SZ_EB_REL, _lcf(sz))
        h = oracle.parse_header(g)
        assert g == oracle.compress(x.numpy(), 1e-4, 1, h["chunk"], h["sub"], pred=oracle.PRED_LCF)
        y = _decompress(sz, ctx, g, x.numel())
        lv = _compress(sz, ctx, x, 1e-4, sz.SZ_EB_REL, None)
        # both predictors code the same lattice: identical reconstructions
        assert np.array_equal(y.view(np.uint32), _decompress(sz, ctx, lv, x.numel()).view(np.uint32))


def test_lcf_batched_decoder_mixed_with_lv(sz, ctx):
    """sz_decompress_batch over LV and LCF streams together (the batched
    decoder picks the reconstruction per stream)."""
    xs = [synth.random_walk_f32(n, n, 0.1).cuda() for n in (100000, 4096, 777, 300000, 1)]
    streams, sizes = [], []
    for i, x in enumerate(xs):
        out, nb = sz.sz_compress(ctx, x, 1e-4, sz.SZ_EB_REL, _lcf(sz) if i % 2 == 0 else None)
        sz.sz_sync(ctx)
        streams.append(out)
        sizes.append(nb.value)
    ys = [torch.empty(x.numel(), dtype=torch.float32, device="cuda") for x in xs]
    no = sz.sz_decompress_batch(ctx, streams, sizes, ys)
    sz.sz_sync(ctx)
    for x, s, n, y in zip(xs, streams, sizes, ys):
        ref = _decompress(sz, ctx, s[:n].cpu().numpy().tobytes(), x.numel())
        assert np.array_equal(y.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_lcf_batch_and_host_entry_points(sz, ctx):
    xs = [synth.random_walk_f32(n, n + 3, 0.5) for n in (5000, 123457, 2, 65536)]
    ebs = [1e-4, 1e-3, 1e-4, 1e-5]
    want = [_compress(sz, ctx, x, e, sz.SZ_EB_REL, _lcf(sz)) for x, e in zip(xs, ebs)]
    outs, nb = sz.sz_compress_batch(ctx, [x.cuda() for x in xs], ebs, sz.SZ_EB_REL, params=_lcf(sz))
    sz.sz_sync(ctx)
    assert [outs[i][: nb[i]].cpu().numpy().tobytes() for i in range(len(xs))] == want
    st, houts, hnb = sz.sz_compress_host(ctx, [x.pin_memory() for x in xs], ebs, sz.SZ_EB_REL, params=_lcf(sz))
    assert [houts[i][: hnb[i]].numpy().tobytes() for i in range(len(xs))] == want


def test_lcf_md_reordering(sz, ctx):
    """best_tradeoff reordering with the LCF predictor: the streams decode to
    the same (reordered) floats as the LV streams of the same snapshot."""
    md = synth.md_fcc(cells=20, seed=4)
    xs = [md[k].cuda() for k in ("xx", "yy", "zz")]
    n = xs[0].numel()
    fields = [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ]
    got = {}
    for pred in (sz.SZ_PRED_LV, sz.SZ_PRED_LCF):
        prm = sz._params(0, 0, 16384, 6, pred)
        outs, nb = sz.sz_compress_snapshot(ctx, fields, xs, n, [1e-4] * 3, sz.SZ_EB_REL, sz.SZ_MODE_LV_PRX, prm)
        sz.sz_sync(ctx)
        got[pred] = [_decompress(sz, ctx, outs[i][: nb[i]].cpu().numpy().tobytes(), n) for i in range(3)]
    for a, b in zip(got[sz.SZ_PRED_LV], got[sz.SZ_PRED_LCF]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_lcf_bad_predictor_byte_and_bad_param(sz, ctx):
    x = synth.random_walk_f32(20000, 1)
    g = bytearray(_compress(sz, ctx, x, 1e-4, sz.SZ_EB_REL, _lcf(sz)))
    g[43] = 3
    d = torch.frombuffer(g, dtype=torch.uint8).cuda()
    y = torch.empty(20000, dtype=torch.float32, device="cuda")
    sz.sz_decompress(ctx, d, len(g), y)
    assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_CORRUPT
    with pytest.raises(sz.SzError):
        sz.sz_compress(ctx, x.cuda(), 1e-4, sz.SZ_EB_REL, sz._params(predictor=3))
