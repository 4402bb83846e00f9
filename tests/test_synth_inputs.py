"""The seeded input generators (`synth`): the structure each promises, checked
on the CPU.  They hold no compression arithmetic; these checks keep the
workload recipes honest."""
import numpy as np
import torch

import synth


def test_counter_based_draws_do_not_depend_on_the_split():
    a = synth.bits64(7, 3, 1000)
    b = torch.cat([synth.bits64(7, 3, 400), synth.bits64(7, 3, 600, offset=400)])
    assert torch.equal(a, b)
    u = synth.uniform(7, 3, 1000)
    assert float(u.min()) >= 0.0 and float(u.max()) < 1.0


def test_skewed_steps_counts_and_exactness():
    m, scale, ratio = 26, 3, 1.62
    x = synth.skewed_steps_f32(m, scale, ratio, seed=5)
    counts = [max(1, int(scale * ratio ** k)) for k in range(m)]
    assert x.numel() == sum(counts)
    xd = x.double().numpy()
    assert np.array_equal(xd, np.round(xd)) and np.abs(xd).max() < 2 ** 24
    steps = np.diff(np.concatenate([[0.0], xd])).astype(np.int64)
    vals, cnt = np.unique(steps, return_counts=True)
    assert vals.size == m
    # the most frequent count belongs to step 0, then +1, -1, +2, -2, ...
    want = {}
    for rank, k in enumerate(range(m - 1, -1, -1)):
        want[(rank + 1) // 2 if rank % 2 else -(rank // 2)] = counts[k]
    assert dict(zip(vals.tolist(), cnt.tolist())) == want


def test_cosmology_snapshot_shape_and_box():
    snap = synth.cosmology(1 << 14, 8, 3)
    assert sorted(snap) == sorted(synth.FIELDS)
    for name in ("xx", "yy", "zz"):
        v = snap[name]
        assert v.dtype == torch.float32 and v.numel() == 1 << 14
        assert float(v.min()) >= 0.0 and float(v.max()) < 256.0
    # velocities are O(300 km/s), not positions
    assert 100.0 < float(snap["vx"].std()) < 2000.0
