"""sz_compress_noalloc: compression for callers that cannot let the library
allocate device memory (for example an in-situ simulation whose memory pool
owns the GPU).  Its scratch is a fixed device array inside the library, so
this test checks that its streams are byte-identical to sz_compress's on the
same inputs, over two calls in a row (the second call starts from whatever
the first left in the shared scratch), that they equal the CPU oracle's, at
sizes up to the largest the array accepts (2^26 elements), and that inputs
beyond that limit are refused with an error instead of being run.

Kept in its own file, named to be collected last."""
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


def _plain(sz, ctx, x, eb, kind):
    out, nb = sz.sz_compress(ctx, x, eb, kind)
    sz.sz_sync(ctx)
    return out[: nb.value].cpu().numpy().tobytes()


def _chunk(n):
    # the default chunk size: 2048 elements up to 2^16, else 4096
    return 2048 if n <= (1 << 16) else 4096


def test_noalloc_matches_sz_compress_twice(sz, oracle):
    ctx = sz.Context(0)
    cases = [
        (synth.cosmology(1 << 18, 16, 1)["vx"], 1e-4, sz.SZ_EB_REL),
        (synth.random_walk_f32(3 * 8192 + 77, 5), 1e-3, sz.SZ_EB_REL),
        (synth.md_fcc(cells=20, seed=2)["yy"], 0.01, sz.SZ_EB_ABS),
        (synth.random_walk_f32(65536, 9), 1e-4, sz.SZ_EB_REL),
    ]
    for x_cpu, eb, kind in cases:
        x = x_cpu.cuda()
        ref = _plain(sz, ctx, x, eb, kind)
        C = _chunk(x.numel())
        assert ref == oracle.compress(x_cpu.numpy(), eb, kind, C, C // 64)
        out = torch.empty(sz.sz_max_compressed_bytes(x.numel()), dtype=torch.uint8, device="cuda")
        for call in range(2):
            out.fill_(0x5A)
            st, _, nbytes = sz.sz_compress_noalloc(x, eb, kind, out=out)
            assert st == sz.SZ_OK, sz.sz_status_string(st)
            assert nbytes == len(ref), f"call {call}: {nbytes} vs {len(ref)} bytes"
            assert out[:nbytes].cpu().numpy().tobytes() == ref, f"call {call}: stream differs"
    ctx.close()


def test_noalloc_largest_accepted_size(sz, oracle):
    """Exactly 2^26 elements (256 MB of float32): the fixed per-chunk tables
    are used to their largest extent, and the stream equals the oracle's."""
    n = 1 << 26
    x = synth.cosmology(n, 512, 7, device="cuda")["yy"]
    out = torch.empty(sz.sz_max_compressed_bytes(n), dtype=torch.uint8, device="cuda")
    st, _, nbytes = sz.sz_compress_noalloc(x, 1e-4, sz.SZ_EB_REL, out=out)
    assert st == sz.SZ_OK, sz.sz_status_string(st)
    got = out[:nbytes].cpu().numpy().tobytes()
    ref = oracle.compress(x.cpu().numpy(), 1e-4, 1, 4096, 64)
    assert got == ref
    st, _, nb2 = sz.sz_compress_noalloc(x, 1e-4, sz.SZ_EB_REL, out=out)
    assert st == sz.SZ_OK and out[:nb2].cpu().numpy().tobytes() == ref


def test_noalloc_rejects_inputs_beyond_its_scratch(sz):
    x = torch.zeros((1 << 26) + 1, dtype=torch.float32, device="cuda")
    out = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st, _, _ = sz.sz_compress_noalloc(x, 1e-4, sz.SZ_EB_REL, out=out)
    assert st == sz.SZ_ERR_ARG


def test_noalloc_reports_capacity(sz):
    x = synth.random_walk_f32(50000, 3).cuda()
    out = torch.empty(sz.sz_max_compressed_bytes(x.numel()), dtype=torch.uint8, device="cuda")
    st, _, need = sz.sz_compress_noalloc(x, 1e-4, sz.SZ_EB_REL, out=out)
    assert st == sz.SZ_OK
    st, _, need2 = sz.sz_compress_noalloc(x, 1e-4, sz.SZ_EB_REL, out=out, out_cap=need - 16)
    assert st == sz.SZ_ERR_CAPACITY and need2 == need
