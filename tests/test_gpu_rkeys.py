"""GPU parity of the best_tradeoff reordering with the R-index built from the
velocities or from all six fields (Sec. IV-C, Fig. 3b, Table 6): streams and
permutation identical to the oracle's, including keys that drop low bits
(more than 10 bits per axis) and the largest number of ignored 6-bit digits."""
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


TAGS = None


def _run(sz, ctx, fs, eb, segment, p, key):
    xs = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in fs]
    n = xs[0].numel()
    tags = [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ, sz.SZ_FIELD_VX, sz.SZ_FIELD_VY, sz.SZ_FIELD_VZ]
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    prm = sz._params(0, 0, segment, p, 0, key)
    outs, nb = sz.sz_compress_snapshot(ctx, tags, xs, n, [eb] * 6, sz.SZ_EB_REL, sz.SZ_MODE_LV_PRX, prm, perm=perm)
    sz.sz_sync(ctx)
    return [outs[i][: int(nb[i])].cpu().numpy().tobytes() for i in range(6)], perm.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("key,p,eb", [(1, 6, 1e-4), (1, 0, 1e-3), (2, 3, 1e-4), (2, 0, 1e-3), (2, 10, 1e-4)])
def test_keyed_reordering_matches_oracle(sz, ctx, oracle, key, p, eb):
    snap = synth.cosmology(1 << 16, 16, 2)
    fs = [snap[f].numpy() for f in synth.FIELDS]
    got, perm = _run(sz, ctx, fs, eb, 4096, p, key)
    h = oracle.parse_header(got[0])
    want, operm = oracle.compress_snapshot_keyed(fs, eb, 1, h["chunk"], h["sub"], 4096, p, key)
    assert (perm == operm).all()
    assert got == want


def test_keyed_reordering_arguments(sz, ctx):
    snap = synth.cosmology(1 << 12, 4, 2)
    xs = [snap[f].cuda() for f in synth.FIELDS]
    n = xs[0].numel()
    tags = [sz.SZ_FIELD_XX, sz.SZ_FIELD_YY, sz.SZ_FIELD_ZZ, sz.SZ_FIELD_VX, sz.SZ_FIELD_VY, sz.SZ_FIELD_VZ]
    with pytest.raises(sz.SzError):      # more than 10 ignored 6-bit digits
        sz.sz_compress_snapshot(ctx, tags, xs, n, [1e-4] * 6, 1, sz.SZ_MODE_LV_PRX, sz._params(0, 0, 4096, 11, 0, 2))
    with pytest.raises(sz.SzError):      # a velocity key needs the velocity fields
        sz.sz_compress_snapshot(ctx, tags[:3], xs[:3], n, [1e-4] * 3, 1, sz.SZ_MODE_LV_PRX,
                                sz._params(0, 0, 4096, 6, 0, 1))
    with pytest.raises(sz.SzError):      # best_compression keys on the coordinates only
        sz.sz_compress_snapshot(ctx, tags, xs, n, [1e-4] * 6, 1, sz.SZ_MODE_CPC2000, sz._params(0, 0, 0, 0, 0, 1))
