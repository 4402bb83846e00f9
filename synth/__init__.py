"""Seeded synthetic inputs shaped like the paper's N-body snapshots.

Holds no compression arithmetic: it only makes float32 particle arrays.  Both
the CUDA path and the CPU oracle consume the arrays made here.  The paper's
HACC and AMDF snapshots (Table 1) are not available; these generators stand in
for them with the structure the paper describes: six SoA float32 fields per
particle (Sec. III), cosmology positions in Lagrangian order with halos and a
smooth background (Sec. IV-C), and a disordered molecular-dynamics crystal
(Sec. IV-B).

Random numbers come from a counter-based generator: SplitMix64's output mix
applied to (key(seed, stream) + (counter + 1) * 0x9E3779B97F4A7C15), all in
wrapping 64-bit integer arithmetic, so a value depends only on (seed, stream,
index) and not on the device or on how the work is split.  Uniform doubles take
the top 53 bits; normals use Box-Muller.  Integer draws are identical on every
device; the log/cos of Box-Muller may differ in the last bit between a CPU and
a GPU, so a test that compares two implementations always feeds both the same
tensor.
"""
from __future__ import annotations

import math

import torch

_GOLD = -7046029254386353131          # 0x9E3779B97F4A7C15 as int64
_M1 = -4658895280553007687            # 0xBF58476D1CE4E5B9
_M2 = -7723592293110705685            # 0x94D049BB133111EB
_FNV = 1099511628211                  # 0x100000001B3


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 viewed as uint64."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def _key(seed: int, stream: int) -> int:
    z = torch.tensor([((seed * _FNV) ^ (stream * 0x5851F42D4C957F2D)) & ((1 << 64) - 1)], dtype=torch.uint64)
    z = z.view(torch.int64)
    return int(_mix64(z)[0])


def bits64(seed: int, stream: int, n: int, device="cpu", offset: int = 0) -> torch.Tensor:
    """n raw 64-bit draws (as int64) for counters offset .. offset+n-1."""
    idx = torch.arange(offset + 1, offset + n + 1, dtype=torch.int64, device=device)
    return _mix64(_key(seed, stream) + idx * _GOLD)


def uniform(seed: int, stream: int, n: int, device="cpu", offset: int = 0) -> torch.Tensor:
    """Doubles in [0, 1): top 53 bits of each draw."""
    return _srl(bits64(seed, stream, n, device, offset), 11).to(torch.float64) * (1.0 / (1 << 53))


def normal(seed: int, stream: int, n: int, device="cpu") -> torch.Tensor:
    """Standard normals by Box-Muller from two uniform streams."""
    u1 = uniform(seed, 2 * stream + 1000, n, device)
    u2 = uniform(seed, 2 * stream + 1001, n, device)
    return torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos((2.0 * math.pi) * u2)


def _choose(seed: int, stream: int, pool: int, k: int, device) -> torch.Tensor:
    """k distinct indices of range(pool), in random-key order."""
    keys = _srl(bits64(seed, stream, pool, device), 1)
    return torch.argsort(keys)[:k]


FIELDS = ("xx", "yy", "zz", "vx", "vy", "vz")


def cosmology(n: int, n_halos: int, seed: int, device="cpu", box=(256.0, 256.0, 256.0),
              origin=(0.0, 0.0, 0.0), period: float = 256.0, background: float = 0.3,
              sigma_v: float = 300.0) -> dict:
    """Cosmology-like snapshot: n particles, six float32 fields.

    Particles sit on n of the n_L^3 sites of a Lagrangian lattice spanning the
    box (n_L = 2^ceil(log2(n)/3)), chosen without replacement and stored in site
    order (x slowest).  A fraction `background` stay near their site (uniform
    jitter of one lattice spacing); the rest are drawn around the halo nearest
    to the centre of their site's 4 Mpc/h coarse cell: centre + N(0, s_h^2) per
    axis, s_h ~ U[1, 4], wrapped into the periodic box.  Velocities are
    N(0, sigma_v^2) per axis plus the halo's bulk velocity N(0, sigma_v^2).
    """
    dev = torch.device(device)
    nL = 1 << max(0, math.ceil(math.log2(max(n, 1)) / 3 - 1e-12))
    sites = nL ** 3
    if n == sites:
        site = torch.arange(n, dtype=torch.int64, device=dev)
    else:
        site = torch.sort(_choose(seed, 1, sites, n, dev)).values
    ix = site // (nL * nL)
    iy = (site // nL) % nL
    iz = site % nL
    box_t = torch.tensor(box, dtype=torch.float64, device=dev)
    org_t = torch.tensor(origin, dtype=torch.float64, device=dev)
    spacing = box_t / nL
    centre = org_t + (torch.stack([ix, iy, iz], 1).to(torch.float64) + 0.5) * spacing

    hc = org_t + torch.stack([uniform(seed, 10 + a, n_halos, dev) for a in range(3)], 1) * box_t
    hs = 1.0 + 3.0 * uniform(seed, 13, n_halos, dev)
    hv = torch.stack([normal(seed, 14 + a, n_halos, dev) for a in range(3)], 1) * sigma_v

    # nearest halo (periodic) to each coarse cell centre of the full box
    g = max(1, int(round(period / 4.0)))
    cell = period / g
    cx = torch.floor(centre / cell).clamp(0, g - 1).to(torch.int64)
    cid = (cx[:, 0] * g + cx[:, 1]) * g + cx[:, 2]
    uniq, inv = torch.unique(cid, return_inverse=True)
    cc = torch.stack([uniq // (g * g), (uniq // g) % g, uniq % g], 1).to(torch.float64) * cell + 0.5 * cell
    best = torch.empty(uniq.numel(), dtype=torch.int64, device=dev)
    step = max(1, (1 << 24) // max(n_halos, 1))
    for s in range(0, uniq.numel(), step):
        d = (cc[s:s + step, None, :] - hc[None, :, :]).abs()
        d = torch.minimum(d, period - d)
        best[s:s + step] = torch.argmin((d * d).sum(-1), 1)
    halo = best[inv]

    bg = uniform(seed, 20, n, dev) < background
    jitter = torch.stack([uniform(seed, 21 + a, n, dev) for a in range(3)], 1) - 0.5
    scatter = torch.stack([normal(seed, 24 + a, n, dev) for a in range(3)], 1)
    pos_bg = centre + jitter * spacing
    pos_h = torch.remainder(hc[halo] + scatter * hs[halo, None], period)
    pos = torch.where(bg[:, None], pos_bg, pos_h)
    vel = torch.stack([normal(seed, 30 + a, n, dev) for a in range(3)], 1) * sigma_v
    vel = vel + torch.where(bg[:, None], torch.zeros_like(vel), hv[halo])
    out = {}
    for a, name in enumerate(FIELDS[:3]):
        out[name] = pos[:, a].to(torch.float32).contiguous()
    for a, name in enumerate(FIELDS[3:]):
        out[name] = vel[:, a].to(torch.float32).contiguous()
    return out


def md_fcc(cells: int = 100, a: float = 3.61, sigma: float = 0.1, vacancy: float = 0.02,
           swap: float = 0.10, seed: int = 2, device="cpu") -> dict:
    """Molecular-dynamics snapshot: an FCC crystal of cells^3 unit cells (4
    basis atoms each), a fraction `vacancy` of the sites removed, thermal
    displacement N(0, sigma^2) per axis, stored in lattice order (cell-major,
    basis fastest), then a fraction `swap` of the atoms exchanged in disjoint
    random pairs.  Three float32 position arrays (Angstrom)."""
    dev = torch.device(device)
    sites = 4 * cells ** 3
    n_vac = int(round(vacancy * sites))
    removed = torch.zeros(sites, dtype=torch.bool, device=dev)
    if n_vac:
        removed[_choose(seed, 1, sites, n_vac, dev)] = True
    site = torch.nonzero(~removed).squeeze(1)
    n = site.numel()
    b = site % 4
    c = site // 4
    i, j, k = c // (cells * cells), (c // cells) % cells, c % cells
    basis = torch.tensor([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]],
                         dtype=torch.float64, device=dev)
    pos = (torch.stack([i, j, k], 1).to(torch.float64) + basis[b]) * a
    pos = pos + torch.stack([normal(seed, 5 + ax, n, dev) for ax in range(3)], 1) * sigma
    n_pairs = int(round(swap * n / 2))
    if n_pairs:
        pick = _choose(seed, 9, n, 2 * n_pairs, dev)
        p, q = pick[:n_pairs], pick[n_pairs:]
        tmp = pos[p].clone()
        pos[p] = pos[q]
        pos[q] = tmp
    return {name: pos[:, ax].to(torch.float32).contiguous() for ax, name in enumerate(FIELDS[:3])}


def batch_ranks(n_ranks: int = 128, grid=(8, 4, 4), log2_min: float = 14.0, log2_max: float = 24.0,
                seed: int = 4, device="cpu", ebs=(1e-3, 1e-4), sizes_only: bool = False):
    """Many uneven arrays: n_ranks simulated ranks, each owning a sub-box of
    the 256 Mpc/h box on `grid`, with 2^U[log2_min, log2_max] particles made
    by `cosmology` in its sub-box (max(1, round(64 n / 2^20)) halos).  Returns
    a list of (rank, field, tensor, eb_rel)."""
    dev = torch.device(device)
    u = uniform(seed, 1, n_ranks, "cpu")
    sizes = [int(round(2.0 ** (log2_min + (log2_max - log2_min) * float(v)))) for v in u]
    pick = uniform(seed, 2, 6 * n_ranks, "cpu")
    ebl = [ebs[0] if float(v) < 0.5 else ebs[1] for v in pick]
    if sizes_only:
        return sizes, ebl
    sub = (256.0 / grid[0], 256.0 / grid[1], 256.0 / grid[2])
    out = []
    for r in range(n_ranks):
        gx, gy, gz = r // (grid[1] * grid[2]), (r // grid[2]) % grid[1], r % grid[2]
        origin = (gx * sub[0], gy * sub[1], gz * sub[2])
        nh = max(1, int(round(64 * sizes[r] / (1 << 20))))
        snap = cosmology(sizes[r], nh, seed * 1000003 + r, dev, box=sub, origin=origin)
        for f, name in enumerate(FIELDS):
            out.append((r, name, snap[name], ebl[6 * r + f]))
    return out


def uniform_f32(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, device="cpu") -> torch.Tensor:
    """Plain uniform float32 values (edge-case and stress inputs)."""
    return (lo + (hi - lo) * uniform(seed, 77, n, device)).to(torch.float32)


def random_walk_f32(n: int, seed: int, step: float = 1.0, device="cpu") -> torch.Tensor:
    """Cumulative sum of normal steps: smooth data with a long range."""
    return torch.cumsum(normal(seed, 78, n, device) * step, 0).to(torch.float32)


def skewed_steps_f32(m: int = 26, scale: int = 1, ratio: float = 1.62, seed: int = 5,
                     device="cpu") -> torch.Tensor:
    """Integer-valued walk whose steps take m distinct values with counts
    max(1, floor(scale * ratio^k)), k = 0..m-1, in random order.  Counts that
    grow slightly faster than Fibonacci numbers give the deepest prefix tree a
    given number of elements allows; the most frequent count goes to step 0,
    the next ones to +1, -1, +2, -2, ... .  Values stay integers below 2^24, so
    they are exact in float32."""
    counts = [max(1, int(scale * ratio ** k)) for k in range(m)]
    steps = []
    for rank, k in enumerate(range(m - 1, -1, -1)):
        s = (rank + 1) // 2 if rank % 2 else -(rank // 2)
        steps.append(torch.full((counts[k],), s, dtype=torch.int64))
    seq = torch.cat(steps)
    perm = torch.argsort(_srl(bits64(seed, 79, seq.numel()), 1))
    x = torch.cumsum(seq[perm], 0)
    assert int(x.abs().max()) < (1 << 24)
    return x.to(torch.float32).to(device)
