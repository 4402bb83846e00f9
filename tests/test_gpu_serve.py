"""GPU tests of the serving loop (continuous batching of compress and
decompress requests): every result is byte-identical to the CPU oracle's on
the same input (compressed streams byte for byte, reconstructions bit for
bit), alone and in the mix, whatever the admission order, budget and output
ownership; the plain call agrees too; a failing request fails alone."""
import time

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
def plain_ctx(sz):
    c = sz.Context(0)
    yield c
    c.close()


def _plain_compress(sz, ctx, x, eb, kind):
    out, nb = sz.sz_compress(ctx, x, eb, kind)
    sz.sz_sync(ctx)
    return out[: nb.value].cpu().numpy().tobytes()


def _plain_decompress(sz, ctx, stream, n):
    out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    no = sz.sz_decompress(ctx, stream, stream.numel(), out, n)
    sz.sz_sync(ctx)
    return out[: no.value].cpu().numpy().tobytes()


def _pool(n_total, seed):
    snap = synth.cosmology(n_total, 16, seed, device="cuda")
    return [snap["xx"], snap["vz"]]


def _chunk(n):
    # the served and plain calls' chunk size: 2048 elements up to 2^16, else 4096
    return 2048 if n <= (1 << 16) else 4096


def _mix(sz, plain_ctx, seed, sizes):
    """Requests over slices of a device pool: (op, input tensor, n, eb, kind,
    expected bytes).  The expected bytes are the oracle's: its stream for a
    compress request, its reconstruction for a decompress request, whose input
    stream the oracle made too.  The plain call is checked against the same
    bytes."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    pool = _pool(1 << 22, seed)
    reqs = []
    for i, n in enumerate(sizes):
        src = pool[i % 2]
        off = int(rng.integers(0, (src.numel() - n) // 4 + 1)) * 4       # 16-byte aligned slices
        x = src[off: off + n]
        eb = [1e-3, 1e-4][i % 2]
        kind = sz.SZ_EB_REL if i % 3 else sz.SZ_EB_ABS
        if kind == sz.SZ_EB_ABS:
            eb = eb * 100.0
        C = _chunk(n)
        ref = oracle.compress(x.cpu().numpy(), eb, kind, C, C // 64)
        if i % 4 == 3:                        # decompress request of a stream the oracle made
            st = torch.frombuffer(bytearray(ref), dtype=torch.uint8).cuda()
            y = oracle.decompress(ref).tobytes()
            assert _plain_decompress(sz, plain_ctx, st, n) == y
            reqs.append(("d", st, n, eb, kind, y))
        else:
            assert _plain_compress(sz, plain_ctx, x, eb, kind) == ref
            reqs.append(("c", x, n, eb, kind, ref))
    torch.cuda.synchronize()
    return reqs


def _submit(sz, ctx, r, service_out):
    op, inp, n, eb, kind, _ = r
    if op == "c":
        if service_out:
            req = sz.request(sz.SZ_OP_COMPRESS, inp, n, eb=eb, kind=kind)
            return sz.sz_serve_submit(ctx, req), None
        out = torch.empty(sz.sz_max_compressed_bytes(n), dtype=torch.uint8, device="cuda")
        req = sz.request(sz.SZ_OP_COMPRESS, inp, n, out=out, out_cap=out.numel(), eb=eb, kind=kind)
        return sz.sz_serve_submit(ctx, req), out
    if service_out:
        req = sz.request(sz.SZ_OP_DECOMPRESS, inp, n, in_bytes=inp.numel())
        return sz.sz_serve_submit(ctx, req), None
    out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    req = sz.request(sz.SZ_OP_DECOMPRESS, inp, n, out=out, in_bytes=inp.numel())
    return sz.sz_serve_submit(ctx, req), out


def _result_bytes(sz, ctx, r, res, out):
    op = r[0]
    nbytes = res.out_size if op == "c" else 4 * res.out_size
    if out is not None:
        assert res.out == out.data_ptr()
        b = out.view(torch.uint8)[:nbytes].cpu().numpy().tobytes()
    else:
        b = sz.device_bytes(res.out, nbytes).cpu().numpy().tobytes() if nbytes else b""
        sz.sz_serve_release(ctx, res.out)
    return b


SIZES = [1, 0, 4097, 70001, 1 << 20, 3 << 18, 2047, 1 << 16, 123457, (1 << 21) + 3, 500000, 5, 262144, 99999,
         1 << 22, 31]


@pytest.mark.parametrize("slots", [1, 8])
def test_serve_results_equal_plain_alone_and_in_mix(sz, plain_ctx, slots):
    reqs = _mix(sz, plain_ctx, 11, SIZES)
    ctx = sz.Context(0, budget=4 << 30)
    try:
        sz.sz_serve_start(ctx, slots)
        subs = [_submit(sz, ctx, r, service_out=(i % 2 == 0)) for i, r in enumerate(reqs)]
        for r, (t, out) in zip(reqs, subs):
            res = sz.sz_serve_wait(ctx, t, 120.0)
            assert res.status == sz.SZ_OK, (r[0], r[2], res.status)
            assert _result_bytes(sz, ctx, r, res, out) == r[5], (r[0], r[2])
            assert res.latency_s > 0
        st = sz.sz_serve_stats(ctx)
        assert st["submitted"] == st["completed"] == len(reqs)
        assert 1 <= st["peak_inflight"] <= slots
        if slots > 1:
            assert st["peak_inflight"] > 1          # requests really overlapped
        sz.sz_serve_stop(ctx)
    finally:
        ctx.close()


def test_serve_one_request_alone_equals_mix(sz, plain_ctx):
    """The same request served alone (one slot, empty device) and inside a
    crowded mix gives the same bytes."""
    reqs = _mix(sz, plain_ctx, 12, [1 << 20, 777777, 1 << 21, 4096, 65537, 1 << 20, 300001, 1 << 22])
    probe = reqs[1]
    ctx = sz.Context(0, budget=2 << 30)
    try:
        sz.sz_serve_start(ctx, 6)
        t, out = _submit(sz, ctx, probe, False)
        alone = _result_bytes(sz, ctx, probe, sz.sz_serve_wait(ctx, t, 60.0), out)
        subs = [_submit(sz, ctx, r, False) for r in reqs[:4]]
        t2, out2 = _submit(sz, ctx, probe, True)
        subs += [_submit(sz, ctx, r, True) for r in reqs[4:]]
        mixed = _result_bytes(sz, ctx, probe, sz.sz_serve_wait(ctx, t2, 60.0), out2)
        for r, (t, out) in zip(reqs, subs):
            res = sz.sz_serve_wait(ctx, t, 60.0)
            assert res.status == sz.SZ_OK
            assert _result_bytes(sz, ctx, r, res, out) == r[5]
        assert alone == mixed == probe[5]
    finally:
        ctx.close()


def test_serve_budget_admission(sz, plain_ctx):
    """A budget that holds about two requests: admission waits for budget,
    never exceeds it, and the results do not change."""
    n = 1 << 20
    reqs = _mix(sz, plain_ctx, 13, [n] * 12)
    per = 4 * n + sz.sz_max_compressed_bytes(n) + 2 * n + 256
    budget = 2 * per + per // 2
    ctx = sz.Context(0, budget=budget)
    try:
        sz.sz_serve_start(ctx, 8)
        subs = [_submit(sz, ctx, r, service_out=True) for r in reqs]
        for r, (t, out) in zip(reqs, subs):
            res = sz.sz_serve_wait(ctx, t, 60.0)
            assert res.status == sz.SZ_OK
            assert _result_bytes(sz, ctx, r, res, out) == r[5]
        st = sz.sz_serve_stats(ctx)
        assert st["peak_bytes"] <= budget
        assert st["budget_waits"] > 0
        assert 1 <= st["peak_inflight"] <= 4
        # a request that can never fit is refused at submit
        big = torch.zeros(4 * n, dtype=torch.float32, device="cuda")
        with pytest.raises(sz.SzError) as e:
            sz.sz_serve_submit(ctx, sz.request(sz.SZ_OP_COMPRESS, big, big.numel(), eb=1e-4))
        assert e.value.status == sz.SZ_ERR_BUSY
    finally:
        ctx.close()


def test_serve_held_outputs_block_until_released(sz, plain_ctx):
    """Service-owned outputs count against the budget until released: with
    the budget full of unreleased outputs the next request waits, and runs
    once one is released."""
    n = 1 << 18
    reqs = _mix(sz, plain_ctx, 14, [n] * 3)
    keep = (sz.sz_max_compressed_bytes(n) + 255) // 256 * 256
    per = 4 * n + keep + 2 * n + (64 << 10)   # input, output, codes and chunk tables (with slack)
    budget = per + keep          # room for one request in flight plus one held output
    ctx = sz.Context(0, budget=budget)
    try:
        sz.sz_serve_start(ctx, 4)
        t0, _ = _submit(sz, ctx, reqs[0], True)
        r0 = sz.sz_serve_wait(ctx, t0, 60.0)
        assert r0.status == sz.SZ_OK
        t1, _ = _submit(sz, ctx, reqs[1], True)
        r1 = sz.sz_serve_wait(ctx, t1, 60.0)
        assert r1.status == sz.SZ_OK
        t2, _ = _submit(sz, ctx, reqs[2], True)
        time.sleep(0.2)
        assert sz.sz_serve_poll(ctx, t2).status == sz.SZ_ERR_BUSY   # two held outputs: no room
        sz.sz_serve_release(ctx, r0.out)
        r2 = sz.sz_serve_wait(ctx, t2, 60.0)
        assert r2.status == sz.SZ_OK
        assert _result_bytes(sz, ctx, reqs[2], r2, None) == reqs[2][5]
        assert _result_bytes(sz, ctx, reqs[1], r1, None) == reqs[1][5]
        with pytest.raises(sz.SzError):
            sz.sz_serve_release(ctx, r0.out)                          # already released
    finally:
        ctx.close()


def test_serve_failure_is_isolated(sz, plain_ctx):
    """A corrupt stream fails with SZ_ERR_CORRUPT; requests beside it succeed."""
    reqs = _mix(sz, plain_ctx, 15, [1 << 16, 1 << 20, 5000, 1 << 18])
    good = reqs[3]
    assert good[0] == "d"
    bad = good[1].clone()
    bad[0] ^= 1                                # magic
    ctx = sz.Context(0, budget=1 << 30)
    try:
        sz.sz_serve_start(ctx, 4)
        tb, _ = _submit(sz, ctx, ("d", bad, good[2], 0, 0, b""), True)
        subs = [_submit(sz, ctx, r, True) for r in reqs]
        rb = sz.sz_serve_wait(ctx, tb, 60.0)
        assert rb.status == sz.SZ_ERR_CORRUPT and rb.out is None
        for r, (t, out) in zip(reqs, subs):
            res = sz.sz_serve_wait(ctx, t, 60.0)
            assert res.status == sz.SZ_OK
            assert _result_bytes(sz, ctx, r, res, out) == r[5]
        # argument errors
        with pytest.raises(sz.SzError):
            sz.sz_serve_poll(ctx, 10 ** 9)
        with pytest.raises(sz.SzError):
            sz.sz_serve_release(ctx, 12345)
        with pytest.raises(sz.SzError):
            sz.sz_serve_start(ctx, 2)                                 # already running
    finally:
        ctx.close()
    nob = sz.Context(0)
    try:
        sz.sz_serve_start(nob, 2)
        x = reqs[0][1]
        with pytest.raises(sz.SzError):                               # no budget: no arena
            sz.sz_serve_submit(nob, sz.request(sz.SZ_OP_COMPRESS, x, x.numel(), eb=1e-4))
        sz.sz_serve_stop(nob)
        sz.sz_serve_stop(nob)                                         # stopping twice is harmless
    finally:
        nob.close()
