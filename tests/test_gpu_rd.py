"""GPU check of the rate-distortion sweep (Fig. 9) that bench.py reports:
its bits per value and PSNR equal those computed from the oracle's streams
and decoded arrays, for both predictors and for the reordered MD mode."""
import math

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


def _oracle_point(oracle, xs, eb, pred):
    bits, psnr = 0, []
    for x in xs:
        x = x.cpu().numpy()
        s = oracle.compress(x, eb, 1, 2048 if x.size <= 65536 else 4096, 32 if x.size <= 65536 else 64, pred=pred)
        y = oracle.decompress(s).astype(np.float64)
        xd = x.astype(np.float64)
        R = xd.max() - xd.min()
        mse = np.mean((xd - y) ** 2)
        bits += 8 * len(s)
        if mse > 0:
            psnr.append(20 * math.log10(R / math.sqrt(mse)))
    return bits / sum(x.numel() for x in xs), (sum(psnr) / len(psnr) if psnr else None)


@pytest.mark.parametrize("pred", [1, 2])
def test_rd_points_match_oracle(sz, oracle, pred):
    import bench
    snap = synth.cosmology(1 << 18, 32, 3)
    xs = [snap[f].cuda() for f in ("xx", "vy")]
    ctx = sz.Context(0)
    try:
        pts = bench.rd_points(sz, ctx, xs, (1e-2, 1e-4, 1e-8), params=sz._params(predictor=pred))
    finally:
        ctx.close()
    for p in pts:
        bits, psnr = _oracle_point(oracle, xs, p["eb"], pred)
        assert p["bits_per_value"] == bits
        if psnr is None:
            assert p["psnr_db"] is None
        else:
            assert abs(p["psnr_db"] - psnr) < 1e-9 * psnr
            assert abs(p["psnr_db"] - p["psnr_closed_form_db"]) < 0.1
        assert p["max_err_over_eb"] <= 1.0 + 1e-12


def test_rd_md_reordered(sz):
    """best_tradeoff reordering changes the order, not the values: same PSNR
    as best_speed at every bound, fewer bits."""
    import bench
    md = synth.md_fcc(cells=25, seed=2)
    xs = [md[f].cuda() for f in ("xx", "yy", "zz")]
    ctx = sz.Context(0)
    try:
        lv = bench.rd_points(sz, ctx, xs, (1e-3, 1e-4))
        prx = bench.rd_points(sz, ctx, xs, (1e-3, 1e-4), params=sz._params(0, 0, 16384, 6),
                              md_mode=sz.SZ_MODE_LV_PRX)
    finally:
        ctx.close()
    for a, b in zip(lv, prx):
        assert abs(a["psnr_db"] - b["psnr_db"]) < 0.05
        assert b["bits_per_value"] < a["bits_per_value"]
        assert b["max_err_over_eb"] <= 1.0 + 1e-12
