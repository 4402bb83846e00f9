"""The large cosmology snapshot (2^27 particles x 6 float32 fields, 4096
halos) through the calls the benchmark times: one sz_compress_batch over the
six fields and one sz_decompress_batch over the six streams, at each of the
workload's three relative bounds (1e-3, 1e-4, 1e-5).  A position field and a
velocity field are compared with the CPU oracle: the streams byte for byte,
the reconstructions bit for bit; every field is checked against its error
bound on the GPU."""
import concurrent.futures as cf

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

FIELDS = ("xx", "yy", "zz", "vx", "vy", "vz")
N = 1 << 27


@pytest.fixture(scope="module")
def sz():
    import __graft_entry__ as g
    g.build()
    import paper_1711_03888_gb300 as m
    return m


@pytest.fixture(scope="module")
def snap():
    s = synth.cosmology(N, 4096, 3, device="cuda")
    return [s[f] for f in FIELDS]


def _oracle_pair(oracle, x, eb, chunk):
    ref = oracle.compress(x, eb, 1, chunk, chunk // 64)
    return ref, oracle.decompress(ref)


@pytest.mark.parametrize("eb", [1e-3, 1e-4, 1e-5])
def test_headline_batch_equals_oracle(sz, oracle, snap, eb):
    ctx = sz.Context(0)
    try:
        outs, nb = sz.sz_compress_batch(ctx, snap, [eb] * len(snap), sz.SZ_EB_REL)
        sz.sz_sync(ctx)
        ys = [torch.empty(N, dtype=torch.float32, device="cuda") for _ in snap]
        no = sz.sz_decompress_batch(ctx, outs, [o.numel() for o in outs], ys)
        sz.sz_sync(ctx)
        for i, (x, y) in enumerate(zip(snap, ys)):
            assert no[i] == N
            fin = torch.isfinite(x)
            R = (x[fin].max().double() - x[fin].min().double()).item()
            err = (x.double() - y.double()).abs().max().item()
            assert err <= eb * R, (FIELDS[i], err, eb * R)
        picks = (0, 3)                                  # xx and vx
        streams = [outs[i][: nb[i]].cpu().numpy().tobytes() for i in picks]
        chunks = [oracle.parse_header(s)["chunk"] for s in streams]
        assert all(c in (2048, 4096, 8192, 16384) for c in chunks)
        xs = [snap[i].cpu().numpy() for i in picks]
        with cf.ThreadPoolExecutor(len(picks)) as ex:
            refs = list(ex.map(lambda a: _oracle_pair(oracle, a[0], eb, a[1]), zip(xs, chunks)))
        for i, got, (ref, yr) in zip(picks, streams, refs):
            assert got == ref, f"{FIELDS[i]} at eb {eb}: stream differs from the oracle's"
            yg = ys[i].cpu().numpy()
            assert np.array_equal(yg.view(np.uint32), yr.view(np.uint32)), f"{FIELDS[i]} at eb {eb}"
    finally:
        ctx.close()
