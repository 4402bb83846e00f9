"""GPU parity of the host-memory calls (sz_compress_host / sz_decompress_host):
every stream is byte-identical to the device path's and to the oracle's, and
every decompressed array to the device decoder's, through groups that cycle
both staging slots; capacity and corruption come back as statuses."""
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
    # the host calls use the fixed chunk-size rule; the batched device calls
    # they are compared with use it too when the autotuner is off
    sz.sz_ctx_set_autotune(c, False)
    yield c
    c.close()


def _device_streams(sz, ctx, xs, ebs, kind):
    outs, nb = sz.sz_compress_batch(ctx, [x.cuda() for x in xs], ebs, kind)
    sz.sz_sync(ctx)
    return [outs[i][: nb[i]].cpu().numpy().tobytes() for i in range(len(xs))]


def _host_round_trip(sz, ctx, xs, ebs, kind, pinned=True):
    hx = [x.pin_memory() if pinned else x.clone() for x in xs]
    st, outs, nb = sz.sz_compress_host(ctx, hx, ebs, kind)
    assert st == sz.SZ_OK
    streams = [outs[i][: nb[i]].numpy().tobytes() for i in range(len(xs))]
    ys = [torch.empty(x.numel(), dtype=torch.float32) for x in xs]
    if pinned:
        ys = [y.pin_memory() for y in ys]
    st, n_out = sz.sz_decompress_host(ctx, [o[: max(b, 1)] for o, b in zip(outs, nb)], nb, ys)
    assert st == sz.SZ_OK
    assert n_out == [x.numel() for x in xs]
    return streams, ys


def _edge_arrays():
    rng = np.random.default_rng(5)
    xs = [synth.random_walk_f32(n, int(rng.integers(1 << 20))) for n in (0, 1, 5, 2047, 2049, 70001, 65537)]
    xs.append(torch.full((9000,), 7.0, dtype=torch.float32))          # R = 0: raw
    w = synth.uniform_f32(30000, 7, -1e30, 1e30).numpy().copy()
    w[::97] = np.nan
    w[5::211] = np.inf
    xs.append(torch.from_numpy(w))                                   # NaN / Inf
    s = synth.random_walk_f32(40000, 8, 1e-3).numpy().copy()
    s[::777] = 1e6
    xs.append(torch.from_numpy(s))                                   # escapes
    return xs


def test_host_edge_mix_matches_oracle(sz, ctx, oracle):
    xs = _edge_arrays()
    ebs = [1e-3, 1e-4, 1e-2, 1e-5, 1e-4, 1e-3, 1e-4, 1e-4, 1e-4, 1e-6]
    for kind in (sz.SZ_EB_REL, sz.SZ_EB_ABS):
        streams, ys = _host_round_trip(sz, ctx, xs, ebs, kind)
        for x, e, g, y in zip(xs, ebs, streams, ys):
            h = oracle.parse_header(g)
            assert g == oracle.compress(x.numpy(), e, kind, h["chunk"], h["sub"])
            assert np.array_equal(y.numpy().view(np.uint32), oracle.decompress(g).view(np.uint32))


def test_host_groups_cycle_both_slots(sz, ctx):
    """Five 96 MiB arrays: one group each, so groups 2..4 reuse the slots of
    groups 0..2 (the copy-in waits for the kernels, the kernels for the
    copy-out).  Streams equal the device path's, arrays the device decoder's."""
    snap = synth.cosmology(1 << 23, 64, 11)
    xs = [snap[f].repeat(3) for f in ("xx", "yy", "zz", "vx", "vy")]
    ebs = [1e-4, 1e-3, 1e-4, 1e-5, 1e-4]
    streams, ys = _host_round_trip(sz, ctx, xs, ebs, sz.SZ_EB_REL)
    assert streams == _device_streams(sz, ctx, xs, ebs, sz.SZ_EB_REL)
    for s, y, x in zip(streams, ys, xs):
        d = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
        out = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
        sz.sz_decompress(ctx, d, len(s), out)
        sz.sz_sync(ctx)
        assert torch.equal(out.cpu().view(torch.int32), y.view(torch.int32))


def test_host_many_small_arrays_in_groups(sz, ctx):
    """Several hundred arrays share each group (the batched workload's size
    mix, 2^14..2^20 elements)."""
    arrays = synth.batch_ranks(n_ranks=64, log2_max=20.0)
    xs = [t for _, _, t, _ in arrays]
    ebs = [e for _, _, _, e in arrays]
    streams, ys = _host_round_trip(sz, ctx, xs, ebs, sz.SZ_EB_REL)
    assert streams == _device_streams(sz, ctx, xs, ebs, sz.SZ_EB_REL)
    for x, y, e in zip(xs[::37], ys[::37], ebs[::37]):
        R = float(x.max() - x.min())
        assert float((x.double() - y.double()).abs().max()) <= e * R


def test_host_pageable_buffers(sz, ctx):
    xs = [synth.random_walk_f32(n, n) for n in (100000, 3, 1 << 20)]
    ebs = [1e-4] * 3
    streams, ys = _host_round_trip(sz, ctx, xs, ebs, sz.SZ_EB_REL, pinned=False)
    assert streams == _device_streams(sz, ctx, xs, ebs, sz.SZ_EB_REL)


def test_host_compress_capacity(sz, ctx):
    xs = [synth.random_walk_f32(50000, 1), synth.random_walk_f32(50000, 2)]
    full = _device_streams(sz, ctx, xs, [1e-4, 1e-4], sz.SZ_EB_REL)
    outs = [torch.empty(len(full[0]), dtype=torch.uint8), torch.empty(len(full[1]) - 1, dtype=torch.uint8)]
    st, outs, nb = sz.sz_compress_host(ctx, xs, [1e-4, 1e-4], sz.SZ_EB_REL, outs=outs, check=False)
    assert st == sz.SZ_ERR_CAPACITY
    assert nb == [len(full[0]), len(full[1])]                 # the required size of the one that did not fit
    assert outs[0].numpy().tobytes() == full[0]


def test_host_decompress_capacity_and_corrupt(sz, ctx):
    xs = [synth.random_walk_f32(30000, 3), synth.random_walk_f32(20000, 4)]
    st, outs, nb = sz.sz_compress_host(ctx, xs, [1e-4, 1e-4], sz.SZ_EB_REL)
    streams = [outs[i][: nb[i]].clone() for i in range(2)]
    ys = [torch.empty(30000, dtype=torch.float32), torch.empty(19999, dtype=torch.float32)]
    st, n_out = sz.sz_decompress_host(ctx, streams, nb, ys, check=False)
    assert st == sz.SZ_ERR_CAPACITY
    assert n_out[1] == 20000
    # a stream cut short inside its payload
    st, n_out = sz.sz_decompress_host(ctx, [streams[0]], [nb[0] - 64], [ys[0]], check=False)
    assert st == sz.SZ_ERR_CORRUPT
    # not a stream at all
    junk = torch.zeros(4096, dtype=torch.uint8)
    st, n_out = sz.sz_decompress_host(ctx, [junk], [4096], [ys[0]], check=False)
    assert st == sz.SZ_ERR_CORRUPT
    # the context is still usable
    st, n_out = sz.sz_decompress_host(ctx, streams[:1], nb[:1], ys[:1])
    assert st == sz.SZ_OK and n_out == [30000]
