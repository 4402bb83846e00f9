"""GPU parity of best_compression (SZ-CPC2000, Sec. II CPC2000 steps 1-4 and
Sec. IV-B): the coordinate stream is byte-identical to the oracle's, its
decode bit-exact with the oracle's decoder, the permutation the oracle's, and
the further fields' SZ-LV streams identical to the oracle's streams of the
reordered fields; edge sizes, non-finite coordinates, a too-fine bound, a
short buffer and a cut stream."""
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


def _gpu_cpc(sz, ctx, fields, eb, kind=1, extra=()):
    xs = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in list(fields) + list(extra)]
    n = xs[0].numel()
    tags = [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ] + [sz.SZ_FIELD_VX, sz.SZ_FIELD_VY, sz.SZ_FIELD_VZ][:len(extra)]
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    ebs = eb if isinstance(eb, (list, tuple)) else [eb] * len(xs)
    outs, nb = sz.sz_compress_snapshot(ctx, tags, xs, n, ebs, kind, sz.SZ_MODE_CPC2000, None, perm=perm)
    st = sz.sz_sync(ctx, check=False)
    return st, outs, [int(nb[i]) for i in range(len(xs))], perm[:n].cpu().numpy().view(np.uint32)


def _gpu_decode(sz, ctx, s, n):
    d = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
    ys = [torch.empty(max(n, 1), dtype=torch.float32, device="cuda") for _ in range(3)]
    no = sz.sz_decompress_cpc(ctx, d, len(s), ys)
    st = sz.sz_sync(ctx, check=False)
    return st, no.value, [y[:n].cpu().numpy() for y in ys]


def _check(sz, ctx, oracle, f, eb, kind=1):
    st, outs, nb, perm = _gpu_cpc(sz, ctx, f, eb, kind)
    assert st == sz.SZ_OK
    g = outs[0][: nb[0]].cpu().numpy().tobytes()
    want, operm = oracle.compress_cpc(*f, eb, kind)
    assert nb[1] == nb[2] == 0
    assert (perm == operm).all()
    assert g == want
    st, no, ys = _gpu_decode(sz, ctx, g, f[0].size)
    assert st == sz.SZ_OK and no == f[0].size
    for y, o in zip(ys, oracle.decompress_cpc(g)):
        assert np.array_equal(y.view(np.uint32), o.view(np.uint32))


@pytest.mark.parametrize("eb,kind", [(1e-3, 1), (1e-4, 1), (0.02, 0)])
def test_cpc_md_matches_oracle(sz, ctx, oracle, eb, kind):
    md = synth.md_fcc(cells=12, seed=3)
    f = [md[k].numpy().copy() for k in ("xx", "yy", "zz")]
    f[0][::997] = np.nan
    f[2][5::1301] = -np.inf
    _check(sz, ctx, oracle, f, eb, kind)


@pytest.mark.parametrize("n", [0, 1, 2, 4095, 4096, 4097, 12289, 70001])
def test_cpc_edge_sizes(sz, ctx, oracle, n):
    f = [synth.uniform_f32(n, 40 + a, -50.0, 50.0).numpy() for a in range(3)]
    _check(sz, ctx, oracle, f, 1e-3)


def test_cpc_full_md_snapshot_with_velocities(sz, ctx, oracle):
    """The 3.92 M-atom crystal (100^3 cells) with three velocity fields: the
    coordinate stream equals the oracle's and the velocity streams equal the
    oracle's SZ-LV streams of the velocities in the sorted order."""
    md = synth.md_fcc(device="cpu")
    f = [md[k].numpy() for k in ("xx", "yy", "zz")]
    n = f[0].size
    vel = [synth.normal(9, 60 + a, n).numpy().astype(np.float32) for a in range(3)]
    st, outs, nb, perm = _gpu_cpc(sz, ctx, f, 1e-4, 1, extra=vel)
    assert st == sz.SZ_OK
    g = outs[0][: nb[0]].cpu().numpy().tobytes()
    want, operm = oracle.compress_cpc(*f, 1e-4, 1)
    assert (perm == operm).all() and g == want
    for i, v in enumerate(vel):
        s = outs[3 + i][: nb[3 + i]].cpu().numpy().tobytes()
        h = oracle.parse_header(s)
        assert s == oracle.compress(v[perm], 1e-4, 1, h["chunk"], h["sub"], reordered=True)
    st, no, ys = _gpu_decode(sz, ctx, g, n)
    assert st == sz.SZ_OK
    for y, o in zip(ys, oracle.decompress_cpc(g)):
        assert np.array_equal(y.view(np.uint32), o.view(np.uint32))


def test_cpc_errors(sz, ctx):
    md = synth.md_fcc(cells=6, seed=1)
    f = [md[k].numpy() for k in ("xx", "yy", "zz")]
    n = f[0].size
    # lattice coordinates wider than 21 bits: the key would not be lossless
    st, _, _, _ = _gpu_cpc(sz, ctx, f, 1e-8)
    assert st == sz.SZ_ERR_UNSUPPORTED
    # a short output buffer reports the size it needs
    xs = [torch.from_numpy(a).cuda() for a in f]
    tags = [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ]
    small = torch.empty(512, dtype=torch.uint8, device="cuda")
    outs, nb = sz.sz_compress_snapshot(ctx, tags, xs, n, [1e-3] * 3, 1, sz.SZ_MODE_CPC2000, None,
                                       outs=[small, small, small])
    assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_CAPACITY
    assert int(nb[0]) > 512
    # a cut stream and a foreign stream
    st, outs, nb, _ = _gpu_cpc(sz, ctx, f, 1e-3)
    g = outs[0][: nb[0]].cpu().numpy().tobytes()
    assert _gpu_decode(sz, ctx, g[:-64], n)[0] == sz.SZ_ERR_CORRUPT
    assert _gpu_decode(sz, ctx, bytes(4096), n)[0] == sz.SZ_ERR_CORRUPT
    # the context still works
    assert _gpu_decode(sz, ctx, g, n)[0] == sz.SZ_OK


def test_cpc_decoder_capacity_and_foreign_formats(sz, ctx):
    """A coordinate stream decoded into too small an array reports capacity
    with the particle count; each decoder rejects the other format's stream
    (SZ-LV vs SZ-CPC2000 magic) and the context keeps working."""
    md = synth.md_fcc(cells=6, seed=5)
    f = [md[k].numpy() for k in ("xx", "yy", "zz")]
    n = f[0].size
    st, outs, nb, _ = _gpu_cpc(sz, ctx, f, 1e-3)
    assert st == sz.SZ_OK
    g = outs[0][: nb[0]]
    small = [torch.empty(n - 1, dtype=torch.float32, device="cuda") for _ in range(3)]
    no = sz.sz_decompress_cpc(ctx, g, nb[0], small)
    assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_CAPACITY
    assert no.value == n
    # an SZ-LV stream into the coordinate decoder, and the coordinate stream into the SZ-LV decoder
    lv, lnb = sz.sz_compress(ctx, torch.from_numpy(f[0]).cuda(), 1e-3, sz.SZ_EB_REL)
    sz.sz_sync(ctx)
    ys = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    sz.sz_decompress_cpc(ctx, lv, lnb.value, ys)
    assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_CORRUPT
    sz.sz_decompress(ctx, g, nb[0], ys[0])
    assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_CORRUPT
    st, no2, back = _gpu_decode(sz, ctx, g.cpu().numpy().tobytes(), n)
    assert st == sz.SZ_OK and no2 == n
