"""GPU parity of the molecular-dynamics modes (Sec. IV-B / V): best_tradeoff
(SZ-LV-PRX: R-index keys, segment-wise partial radix sort, one permutation
for every field) and best_speed (SZ-LV in stored order).  The permutation
must equal the oracle's exactly and every stream must be byte-identical."""
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


def _snapshot_gpu(sz, ctx, fields, eb, kind, segment, p, mode=None):
    mode = sz.SZ_MODE_LV_PRX if mode is None else mode
    n = fields[0].numel()
    xs = [f.cuda() for f in fields]
    perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda") if mode == sz.SZ_MODE_LV_PRX else None
    ids = [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ, sz.SZ_FIELD_VX, sz.SZ_FIELD_VY, sz.SZ_FIELD_VZ][:len(xs)]
    outs, nb = sz.sz_compress_snapshot(ctx, ids, xs, n, [eb] * len(xs), kind, mode,
                                       sz._params(0, 0, segment, p), perm=perm)
    sz.sz_sync(ctx)
    streams = [outs[i][: nb[i]].cpu().numpy().tobytes() for i in range(len(xs))]
    return streams, (perm[:n].cpu().numpy().view(np.uint32) if perm is not None else None)


@pytest.mark.parametrize("segment,p", [(16384, 6), (16384, 0), (1024, 8), (777, 2), (4096, 21)])
@pytest.mark.parametrize("eb", [1e-4, 1e-3])
def test_md_prx_matches_oracle(sz, ctx, oracle, segment, p, eb):
    md = synth.md_fcc(cells=25, seed=2)
    f = [md[k] for k in ("xx", "yy", "zz")]
    got, perm = _snapshot_gpu(sz, ctx, f, eb, sz.SZ_EB_REL, segment, p)
    h = oracle.parse_header(got[0])
    ref, rperm = oracle.compress_snapshot([t.numpy() for t in f], eb, 1, h["chunk"], h["sub"], segment, p)
    assert np.array_equal(perm, rperm)
    for g, r in zip(got, ref):
        assert g == r
    assert h["flags"] & 2


def test_md_velocities_follow_the_permutation(sz, ctx, oracle):
    snap = synth.cosmology(50000, 8, 5)
    f = [snap[k] for k in ("xx", "yy", "zz", "vx", "vy", "vz")]
    got, perm = _snapshot_gpu(sz, ctx, f, 1e-4, sz.SZ_EB_REL, 4096, 6)
    h = oracle.parse_header(got[0])
    ref, rperm = oracle.compress_snapshot([t.numpy() for t in f], 1e-4, 1, h["chunk"], h["sub"], 4096, 6)
    assert np.array_equal(perm, rperm)
    assert all(g == r for g, r in zip(got, ref))
    # decompressed fields are the reordered originals, within the bound
    for t, s in zip(f, got):
        y = oracle.decompress(s)
        ea = oracle.parse_header(s)["eb_abs"]
        assert (np.abs(t.numpy()[perm].astype(np.float64) - y) <= ea).all()


def test_md_absolute_bound_and_wide_keys(sz, ctx, oracle):
    """A tiny absolute bound gives more than 21 bits per axis (low bits
    dropped) and keys wider than 32 bits after the shift."""
    md = synth.md_fcc(cells=12, seed=3)
    f = [md[k] for k in ("xx", "yy", "zz")]
    got, perm = _snapshot_gpu(sz, ctx, f, 1e-6, sz.SZ_EB_ABS, 2048, 0)
    h = oracle.parse_header(got[0])
    ref, rperm = oracle.compress_snapshot([t.numpy() for t in f], 1e-6, 0, h["chunk"], h["sub"], 2048, 0)
    assert np.array_equal(perm, rperm)
    assert all(g == r for g, r in zip(got, ref))


def test_md_best_speed_is_plain_lv(sz, ctx, oracle):
    md = synth.md_fcc(cells=20, seed=2)
    f = [md[k] for k in ("xx", "yy", "zz")]
    got, _ = _snapshot_gpu(sz, ctx, f, 1e-4, sz.SZ_EB_REL, 0, 0, mode=sz.SZ_MODE_LV)
    for t, g in zip(f, got):
        h = oracle.parse_header(g)
        assert g == oracle.compress(t.numpy(), 1e-4, 1, h["chunk"], h["sub"])


def test_md_best_compression_round_trip(sz, ctx):
    """best_compression writes one coordinate stream to the first output;
    it decodes to the sorted coordinates within every axis's bound (the
    byte-level parity is in test_gpu_cpc.py)."""
    md = synth.md_fcc(cells=8, seed=2)
    xs = [md[k].cuda() for k in ("xx", "yy", "zz")]
    n = xs[0].numel()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    outs, nb = sz.sz_compress_snapshot(ctx, [0, 1, 2], xs, n, [1e-4] * 3, sz.SZ_EB_REL, sz.SZ_MODE_CPC2000,
                                       perm=perm)
    sz.sz_sync(ctx)
    assert int(nb[1]) == int(nb[2]) == 0 and int(nb[0]) > 160
    ys = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    no = sz.sz_decompress_cpc(ctx, outs[0], int(nb[0]), ys)
    sz.sz_sync(ctx)
    assert no.value == n
    for x, y in zip(xs, ys):
        R = (x.max() - x.min()).double().item()
        assert (x[perm.long()].double() - y.double()).abs().max().item() <= 1e-4 * R * (1 + 1e-12)


@pytest.mark.parametrize("eb", [1e-4, 1e-3])
def test_full_size_md_snapshot(sz, ctx, oracle, eb):
    """The full molecular-dynamics snapshot: 3,920,000 atoms, 3 fields,
    segment 16384, 6 ignored digits (best_tradeoff)."""
    md = synth.md_fcc(seed=2, device="cuda")
    f = [md[k] for k in ("xx", "yy", "zz")]
    got, perm = _snapshot_gpu(sz, ctx, f, eb, sz.SZ_EB_REL, 16384, 6)
    h = oracle.parse_header(got[0])
    ref, rperm = oracle.compress_snapshot([t.cpu().numpy() for t in f], eb, 1, h["chunk"], h["sub"], 16384, 6)
    assert np.array_equal(perm, rperm)
    assert all(g == r for g, r in zip(got, ref))
    raw = 12 * f[0].numel()
    lv = sum(len(oracle.compress(t.cpu().numpy(), eb, 1, h["chunk"], h["sub"])) for t in f)
    assert raw / sum(len(g) for g in got) > raw / lv        # Tables 4-5 trend
