"""The timeout path of the device-side waits.  Every wait in the kernels
polls a bounded number of times and then latches SZ_ERR_TIMEOUT instead of
hanging.  Here the encoder's look-back wait is made to run out on purpose:
one warp waits on a predecessor chunk that never publishes (a status word that
nothing sets), with a limit of a few polls.  sz_sync must report the timeout,
clear it, and leave the context usable: the next call's stream equals the
oracle's."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sz():
    import __graft_entry__ as g
    g.build()
    import paper_1711_03888_gb300 as m
    return m


def test_lookback_wait_times_out_and_context_recovers(sz, oracle):
    ctx = sz.Context(0)
    try:
        x_cpu = synth.cosmology(1 << 16, 8, 1)["vx"]
        ref = oracle.compress(x_cpu.numpy(), 1e-4, 1, 4096, 64)
        x = x_cpu.cuda()
        for spins in (1, 64, 4096):
            sz.sz_check_wait_timeout(ctx, spins)
            assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_TIMEOUT
            assert sz.sz_sync(ctx, check=False) == sz.SZ_OK          # reported once, then cleared
            out, nb = sz.sz_compress(ctx, x, 1e-4, sz.SZ_EB_REL, sz._params(4096))
            assert sz.sz_sync(ctx, check=False) == sz.SZ_OK
            assert out[: nb.value].cpu().numpy().tobytes() == ref
        # a timeout latched between two real calls: both calls' results are
        # still delivered, and the status of that sync is the timeout
        out1, nb1 = sz.sz_compress(ctx, x, 1e-4, sz.SZ_EB_REL, sz._params(4096))
        sz.sz_check_wait_timeout(ctx, 8)
        out2, nb2 = sz.sz_compress(ctx, x, 1e-4, sz.SZ_EB_REL, sz._params(4096))
        assert sz.sz_sync(ctx, check=False) == sz.SZ_ERR_TIMEOUT
        assert out1[: nb1.value].cpu().numpy().tobytes() == ref
        assert out2[: nb2.value].cpu().numpy().tobytes() == ref
        for bad in (0, (1 << 20) + 1):
            with pytest.raises(sz.SzError) as e:
                sz.sz_check_wait_timeout(ctx, bad)
            assert e.value.status == sz.SZ_ERR_ARG
    finally:
        ctx.close()
