"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- hand-derived fixtures, exact-rational brute force, textbook
algorithms, closed forms and invariants from the paper (arXiv 1711.03888).
CPU only."""
import heapq
import json
import math
import os
import struct
from fractions import Fraction

import numpy as np
import pytest
import torch

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _f32bits(a):
    return np.asarray(a, np.float32).view(np.uint32)


# --------------------------------------------------------------------------
# Lattice, LV prediction, quantization (Sec. II CPC2000 step 1, Sec. IV-A)
# --------------------------------------------------------------------------

def test_golden_lattice_example(oracle):
    g = _load("lattice_lv_example.json")
    x = np.tile(np.asarray(g["x_pattern"], np.float32), g["repeat"])
    ea, D = oracle.error_bound(x, g["eb_abs"], 0)
    assert ea == g["eb_abs"] and float(D) == g["D"]
    q, v = oracle.lattice(x, D, ea)
    assert q.tolist() == g["q_pattern"] * g["repeat"] and not v.any()
    c, d = oracle.codes(q, v)
    assert d[:8].tolist() == g["delta_head"] and c[:8].tolist() == g["codes_head"]
    s = oracle.compress(x, g["eb_abs"], kind=0, chunk=g["chunk"], sub=g["sub"])
    h = oracle.parse_header(s)
    assert not (h["flags"] & 1)
    syms, lens = oracle.stream_codebook(s)
    assert syms.tolist() == g["codebook_symbols"] and lens.tolist() == g["codebook_lengths"]
    bits = "".join(g["codewords"][str(int(k))] for k in c)
    assert len(bits) == g["payload_bits"]
    assert h["payload_words"] == g["payload_words_padded"]
    bits = bits.ljust(32 * g["payload_words_padded"], "0")
    expect = [int(bits[32 * k:32 * k + 32], 2) for k in range(g["payload_words_padded"])]
    assert list(struct.unpack_from("<%dI" % len(expect), s, h["off_payload"])) == expect
    subl = struct.unpack_from("<4H", s, h["off_sublen"])
    assert list(subl) == g["substream_bits"]
    assert oracle.decompress(s).tolist() == g["recon_pattern"] * g["repeat"]


def _rne(fr: Fraction) -> int:
    fl = fr.numerator // fr.denominator
    rem = fr - fl
    if rem > Fraction(1, 2):
        return fl + 1
    if rem < Fraction(1, 2):
        return fl
    return fl if fl % 2 == 0 else fl + 1


def _sequential_sz_lv(x, D: Fraction):
    """Textbook sequential SZ with the last-value predictor, in exact rational
    arithmetic: the prediction is the previous *reconstructed* value."""
    pred = Fraction(0)
    codes, recon = [], []
    for xi in x:
        k = _rne((Fraction(float(xi)) - pred) / D)
        pred = pred + k * D
        codes.append(k + 32768 if -32767 <= k <= 32767 else 0)
        recon.append(np.float32(float(pred)))   # RN64 then RN32
    return codes, recon


@pytest.mark.parametrize("eb_abs", [2.0 ** -5, 0.0123, 3.7e-3])
def test_bruteforce_sequential_lv(oracle, eb_abs):
    rng = np.random.default_rng(11)
    n = 400
    D = float(oracle.step(eb_abs))
    # a walk on the lattice scale with steps well inside the code radius
    steps = rng.normal(0, 50, n) * D
    x = np.cumsum(steps).astype(np.float32)
    t = np.asarray([Fraction(float(v)) / Fraction(D) for v in x])
    frac = np.asarray([float(ti - math.floor(ti)) for ti in t])
    keep = np.abs(frac - 0.5) > 1e-6                         # no exact half-ties
    x = x[keep]
    codes_bf, recon_bf = _sequential_sz_lv(x, Fraction(D))
    ea, Dd = oracle.error_bound(x, eb_abs, 0)
    q, v = oracle.lattice(x, Dd, ea)
    c, _ = oracle.codes(q, v)
    assert c.tolist() == codes_bf
    s = oracle.compress(x, eb_abs, kind=0, chunk=256, sub=16)
    y = oracle.decompress(s)
    assert (_f32bits(y) == _f32bits(recon_bf)).all()


def test_lattice_power_of_two_exact(oracle):
    """D a power of two and |x| <= 2^20 D: every step is exact, so the lattice
    index is the nearest integer of x/D (ties to even)."""
    rng = np.random.default_rng(3)
    D = 2.0 ** -6
    m = rng.integers(-(1 << 20), 1 << 20, 5000)
    f = rng.integers(0, 64, 5000) / 64.0                    # includes exact halves
    x = ((m + f) * D).astype(np.float32)
    q, v = oracle.lattice(x, np.float32(D), D / 2)
    expect = np.round(x.astype(np.float64) / D)             # numpy rounds half to even
    assert (q == expect.astype(np.int64)).all() and not v.any()


def test_codes_radius_and_escape(oracle):
    q = np.array([0, 32767, 0, -32767, -65534, 5], np.int64)
    v = np.array([0, 0, 0, 0, 0, 1], bool)
    c, d = oracle.codes(q, v)
    assert d.tolist() == [0, 32767, -32767, -32767, -32767, 65539]
    assert c.tolist() == [32768, 65535, 1, 1, 1, 0]
    q2 = np.array([32768, 0, -32768], np.int64)
    c2, _ = oracle.codes(q2, np.zeros(3, bool))
    assert c2.tolist() == [0, 0, 0]                          # |delta| >= 32768 escapes


# --------------------------------------------------------------------------
# Error bound (Sec. III) and its consequences (Sec. V: max error equals eb)
# --------------------------------------------------------------------------

def _inputs():
    snap = synth.cosmology(1 << 14, 8, 1)
    md = synth.md_fcc(cells=12, seed=2)
    yield "cosmo_xx", snap["xx"].numpy()
    yield "cosmo_vz", snap["vz"].numpy()
    yield "md_yy", md["yy"].numpy()
    yield "walk", synth.random_walk_f32(20000, 5).numpy()
    yield "uniform", synth.uniform_f32(20000, 6).numpy()
    w = synth.uniform_f32(3000, 7, -1e30, 1e30).numpy()
    w[::97] = np.nan
    w[5::211] = np.inf
    w[7::223] = -np.inf
    w[9::50] = np.float32(1e-42)                             # subnormal
    w[11::50] = -0.0
    yield "wild", w


@pytest.mark.parametrize("eb", [1e-2, 1e-4, 1e-6])
def test_error_bound_every_element(oracle, eb):
    for name, x in _inputs():
        s = oracle.compress(x, eb, kind=1, chunk=1024, sub=64)
        y = oracle.decompress(s)
        ea, _ = oracle.error_bound(x, eb, 1)
        fin = np.isfinite(x)
        err = np.abs(x[fin].astype(np.float64) - y[fin].astype(np.float64))
        assert err.max(initial=0.0) <= ea, name
        assert (_f32bits(x[~fin]) == _f32bits(y[~fin])).all(), name


def test_nrmse_closed_form_and_max_error(oracle):
    """Uniform dense data: the error is uniform on [-D/2, D/2], so
    NRMSE = D / sqrt(12) / R = eb_rel / sqrt(3) and the largest error reaches
    the bound (Sec. V reports it 'exactly equal' to eb)."""
    x = synth.uniform_f32(1 << 18, 9, 0.0, 1.0).numpy()
    eb = 1e-4
    y = oracle.decompress(oracle.compress(x, eb, kind=1))
    ea, _ = oracle.error_bound(x, eb, 1)
    R = oracle.value_range(x)
    e = x.astype(np.float64) - y.astype(np.float64)
    nrmse = math.sqrt(np.mean(e * e)) / R
    assert abs(nrmse / (eb / math.sqrt(3)) - 1) < 0.01
    psnr = -20 * math.log10(nrmse)
    assert abs(psnr - 84.77) < 0.1
    assert np.abs(e).max() / ea > 0.999


def test_step_rounds_toward_zero(oracle):
    """The lattice step is the largest float not above 2*eb_abs, so the
    rounding error |x - qD| <= D/2 never exceeds eb_abs."""
    for ea in [0.05, 1e-4, 3.3e-7, 0.95, 123.456, 1e-30]:
        D = oracle.step(ea)
        assert float(D) <= 2 * ea < float(np.nextafter(D, np.float32(np.inf)))
    assert float(oracle.step(0.0)) == 0.0


def test_large_lattice_index_reconstructs_exactly(oracle):
    """|q| beyond 2^24: when the float spacing of x exceeds 2*eb, the nearest
    float to q*D is x itself, so reconstruction is exact (and not verbatim)."""
    rng = np.random.default_rng(8)
    x = (1000.0 + np.cumsum(rng.normal(0, 1e-4, 4000))).astype(np.float32)
    s = oracle.compress(x, 1e-6, kind=0, chunk=1024, sub=64)
    h = oracle.parse_header(s)
    assert not (h["flags"] & 1)
    ea, D = oracle.error_bound(x, 1e-6, 0)
    q, v = oracle.lattice(x, D, ea)
    assert np.abs(q).min() > (1 << 24) and not v.any()
    assert (_f32bits(oracle.decompress(s)) == _f32bits(x)).all()


def test_value_range_definition(oracle):
    x = np.array([3.0, np.nan, -2.0, np.inf, 7.5], np.float32)
    assert oracle.value_range(x) == 9.5
    ea, D = oracle.error_bound(x, 0.1, 1)
    assert ea == 0.1 * 9.5
    assert float(D) <= 2 * ea and float(np.nextafter(D, np.float32(np.inf))) > 2 * ea


# --------------------------------------------------------------------------
# Huffman coding of the codes (Sec. II / IV-A / IV-B: tailored Huffman)
# --------------------------------------------------------------------------

def _heap_cost(freq):
    h = [int(f) for f in freq]
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def _heap_lengths(freq, sym, limit=24):
    """Lengths from a heap-ordered Huffman construction whose heap key is
    (weight, leaf-before-internal, order): leaves ordered by (weight, symbol),
    internal nodes by creation.  Picking the heap minimum equals comparing the
    fronts of the two queues, so the tree is the same; the length limit
    rescales every weight to (w >> 1) | 1 and rebuilds."""
    f = [int(v) for v in freq]
    m = len(f)
    if m == 1:
        return [1]
    while True:
        order = sorted(range(m), key=lambda k: (f[k], int(sym[k])))
        heap = [(f[k], 0, r, ("leaf", k)) for r, k in enumerate(order)]
        heapq.heapify(heap)
        parent = {}
        made = 0
        while len(heap) > 1:
            a = heapq.heappop(heap)
            b = heapq.heappop(heap)
            node = ("int", made)
            parent[a[3]] = node
            parent[b[3]] = node
            heapq.heappush(heap, (a[0] + b[0], 1, made, node))
            made += 1
        lens = []
        for k in range(m):
            d, v = 0, ("leaf", k)
            while v in parent:
                v = parent[v]
                d += 1
            lens.append(d)
        if max(lens) <= limit:
            return lens
        f = [(v >> 1) | 1 for v in f]


@pytest.mark.parametrize("seed", range(4))
def test_huffman_lengths_match_heap_construction(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(2, 600))
    freq = rng.integers(1, 6, m).astype(np.uint64) ** rng.integers(1, 4, m).astype(np.uint64)
    sym = np.sort(rng.choice(65536, m, replace=False)).astype(np.uint32)
    assert oracle.huffman_lengths(freq, sym).tolist() == _heap_lengths(freq, sym)


@pytest.mark.parametrize("kind", ["fib", "pow2", "pow3"])
def test_huffman_limit_matches_heap_construction(oracle, kind):
    rng = np.random.default_rng(9)
    if kind == "fib":
        base = [1, 1]
        while len(base) < 40:
            base.append(base[-1] + base[-2])
    elif kind == "pow2":
        base = [1 << k for k in range(34)]
    else:
        base = [3 ** k for k in range(22)]
    extra = [] if kind == "fib" else list(rng.integers(1, 50, 30))
    freq = np.asarray(base + extra, np.uint64)
    sym = np.arange(freq.size, dtype=np.uint32)
    lens = oracle.huffman_lengths(freq, sym)
    assert max(_heap_lengths(freq, sym, limit=64)) > 24      # the limit binds
    assert lens.tolist() == _heap_lengths(freq, sym)


@pytest.mark.parametrize("scale", [1, 3, 6, 12, 48])
def test_huffman_limit_on_repeated_rebuilds(oracle, scale):
    """The step counts of synth.skewed_steps_f32 (m = 26, ratio 1.62) need one
    to seven rescalings before the tree fits 24 bits; the oracle must end on
    the heap construction's tree after every one of them."""
    freq = np.asarray([max(1, int(scale * 1.62 ** k)) for k in range(26)], np.uint64)
    sym = np.arange(freq.size, dtype=np.uint32)
    assert max(_heap_lengths(freq, sym, limit=64)) > 24
    assert oracle.huffman_lengths(freq, sym).tolist() == _heap_lengths(freq, sym)


def _package_merge(freq, L):
    """Optimal lengths under a length limit L (Larmore-Hirschberg)."""
    n = len(freq)
    items = sorted([(int(f), (i,)) for i, f in enumerate(freq)])
    cur = list(items)
    for _ in range(L - 1):
        pk = [(cur[k][0] + cur[k + 1][0], cur[k][1] + cur[k + 1][1]) for k in range(0, len(cur) - 1, 2)]
        cur = sorted(items + pk, key=lambda t: t[0])
    lens = [0] * n
    for _, members in cur[: 2 * (n - 1)]:
        for i in members:
            lens[i] += 1
    return lens


def _check_prefix_free(lens, codes):
    order = sorted(range(len(lens)), key=lambda i: (lens[i], i))
    for a_i, a in enumerate(order):
        for b in order[a_i + 1:]:
            assert (int(codes[b]) >> (int(lens[b]) - int(lens[a]))) != int(codes[a])


def test_golden_huffman(oracle):
    g = _load("huffman_examples.json")
    for case in g["cases"]:
        f = np.asarray(case["freq"], np.uint64)
        lens = oracle.huffman_lengths(f)
        if "lengths" in case:
            assert lens.tolist() == case["lengths"], case["note"]
            assert oracle.canonical_codes(lens).tolist() == case["codes"], case["note"]
        if "cost" in case:
            assert int((f * lens).sum()) == case["cost"]


@pytest.mark.parametrize("seed", range(6))
def test_huffman_optimal_and_kraft(oracle, seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(2, 3000))
    freq = np.maximum(1, (rng.pareto(1.2, m) * 10).astype(np.uint64))
    lens = oracle.huffman_lengths(freq)
    if lens.max() <= 24:
        assert int((freq * lens).sum()) == _heap_cost(freq)
    kraft = sum(Fraction(1, 1 << int(l)) for l in lens)
    assert kraft == 1
    codes = oracle.canonical_codes(lens)
    if m < 400:
        _check_prefix_free(lens, codes)
    # entropy bound: H <= average length < H + 1
    p = freq / freq.sum()
    H = float(-(p * np.log2(p)).sum())
    avg = float((p * lens).sum())
    assert H <= avg + 1e-12 and avg < H + 1


def test_huffman_length_limit(oracle):
    fib = [1, 1]
    while len(fib) < 32:
        fib.append(fib[-1] + fib[-2])
    freq = np.asarray(fib, np.uint64)
    lens = oracle.huffman_lengths(freq)
    assert lens.max() <= 24
    assert sum(Fraction(1, 1 << int(l)) for l in lens) == 1
    opt = _package_merge(fib, 24)
    cost = int((freq * lens).sum())
    best = sum(f * l for f, l in zip(fib, opt))
    assert best <= cost <= 1.01 * best
    assert _heap_cost(fib) < best                             # the limit really binds
    _check_prefix_free(lens, oracle.canonical_codes(lens))


# --------------------------------------------------------------------------
# Stream: round trip, layout invariants, degenerate inputs
# --------------------------------------------------------------------------

def _check_layout(oracle, s, n):
    h = oracle.parse_header(s)
    assert h["magic"] == 0x564C5A53 and h["version"] == 1 and h["header_bytes"] == 160
    assert h["n"] == n and h["total_bytes"] == len(s) and len(s) % 16 == 0
    offs = [h[k] for k in ("off_syms", "off_lens", "off_chunk_word", "off_chunk_anchor",
                           "off_chunk_esc", "off_sublen", "off_escapes", "off_payload")]
    assert all(o % 16 == 0 for o in offs) and offs == sorted(offs)
    assert h["payload_words"] % 4 == 0
    assert len(s) <= oracle.max_bytes(n)
    if h["flags"] & 1 or n == 0:
        return h
    nc = h["n_chunks"]
    assert nc == (n + h["chunk"] - 1) // h["chunk"]
    cw = np.frombuffer(s, np.uint64, nc + 1, h["off_chunk_word"])
    assert cw[0] == 0 and (np.diff(cw.astype(np.int64)) >= 0).all() and cw[-1] == h["payload_words"]
    assert (cw % 4 == 0).all()
    ce = np.frombuffer(s, np.uint64, nc + 1, h["off_chunk_esc"])
    assert ce[0] == 0 and ce[-1] == h["n_escapes"]
    S = h["chunk"] // h["sub"]
    sl = np.frombuffer(s, np.uint16, nc * S, h["off_sublen"]).reshape(nc, S).astype(np.int64)
    per_chunk = sl.sum(1)
    assert ((per_chunk + 127) // 128 * 4 == np.diff(cw.astype(np.int64))).all()
    syms, lens = oracle.stream_codebook(s)
    assert (np.diff(syms.astype(np.int64)) > 0).all() and lens.min() >= 1 and lens.max() <= 24
    return h


@pytest.mark.parametrize("n,chunk,sub", [(1, 256, 16), (2, 256, 16), (255, 256, 16), (257, 256, 16),
                                         (5000, 1024, 32), (70001, 8192, 128), (65536, 65536, 2048)])
def test_roundtrip_layout(oracle, n, chunk, sub):
    x = synth.random_walk_f32(n, 21).numpy()
    s = oracle.compress(x, 1e-3, kind=1, chunk=chunk, sub=sub)
    h = _check_layout(oracle, s, n)
    y = oracle.decompress(s)
    ea = h["eb_abs"]
    assert y.size == n and (np.abs(x.astype(np.float64) - y) <= ea).all()


def test_degenerate_inputs(oracle):
    s = oracle.compress(np.zeros(0, np.float32), 1e-4)
    assert len(s) == 160 and oracle.decompress(s).size == 0
    c = np.full(1000, 3.25, np.float32)                      # R = 0: eb_abs = 0 -> raw, exact
    s = oracle.compress(c, 1e-4)
    assert oracle.parse_header(s)["flags"] & 1
    assert (oracle.decompress(s) == c).all()
    x = synth.uniform_f32(1000, 3).numpy()
    s = oracle.compress(x, 0.0, kind=0)                      # abs eb 0 -> raw
    assert (_f32bits(oracle.decompress(s)) == _f32bits(x)).all()
    allnan = np.full(100, np.nan, np.float32)
    assert np.isnan(oracle.decompress(oracle.compress(allnan, 1e-4))).all()
    with pytest.raises(oracle.OracleError):
        oracle.compress(x, float("nan"))
    with pytest.raises(oracle.OracleError):
        oracle.compress(x, 1e-4, chunk=1000)


def test_far_offsets_and_escapes(oracle):
    """Large jumps (|delta| >= 2^15) and values whose lattice index would
    exceed 2^53 go to escape records; all stay within the bound."""
    rng = np.random.default_rng(4)
    x = np.cumsum(rng.normal(0, 1e-5, 50000)).astype(np.float32)
    x[::1000] = 1e6
    s = oracle.compress(x, 1e-6, kind=0, chunk=2048, sub=64)
    h = _check_layout(oracle, s, x.size)
    assert h["n_escapes"] >= 100 and not (h["flags"] & 1)
    y = oracle.decompress(s)
    assert (np.abs(x.astype(np.float64) - y) <= 1e-6).all()
    big = np.array([1e30, 1.0, -1e30, 2.0], np.float32)     # 1e30 / 2e-10 > 2^53
    s = oracle.compress(np.tile(big, 500), 1e-10, kind=0)
    y = oracle.decompress(s)
    assert (np.abs(np.tile(big, 500).astype(np.float64) - y) <= 1e-10).all()


def test_raw_fallback_when_lossy_is_larger(oracle):
    x = synth.uniform_f32(1 << 14, 8, -1.0, 1.0).numpy()
    s = oracle.compress(x, 1e-9, kind=0)
    h = oracle.parse_header(s)
    assert h["flags"] & 1 and len(s) == oracle.max_bytes(x.size)
    assert (_f32bits(oracle.decompress(s)) == _f32bits(x)).all()


# --------------------------------------------------------------------------
# MD reordering: R-index (Fig. 3a) and the segment-wise PRX sort (Tables 4-5)
# --------------------------------------------------------------------------

def test_golden_rindex(oracle):
    g = _load("rindex_examples.json")
    for c in g["morton"]:
        assert oracle.morton3(*c["u"], c["bits"]) == c["key"]
    for c in g["segment_sort"]:
        perm = oracle.segment_sort(np.asarray(c["keys"], np.uint64), c["segment"], c["ignored_digits"])
        assert perm.tolist() == c["perm"]


def test_morton_order_is_octree_order(oracle):
    """Interleaving makes the key order the depth-first octree order: comparing
    keys equals comparing the (x, y, z) octant digits from the top level down."""
    rng = np.random.default_rng(5)
    u = rng.integers(0, 1 << 7, (400, 3))
    keys = [oracle.morton3(int(a), int(b), int(c), 7) for a, b, c in u]

    def path(t):
        return [((t[0] >> l) & 1, (t[1] >> l) & 1, (t[2] >> l) & 1) for l in range(6, -1, -1)]
    by_key = sorted(range(400), key=lambda i: keys[i])
    by_path = sorted(range(400), key=lambda i: path(u[i]))
    assert [keys[i] for i in by_key] == [keys[i] for i in by_path]
    # de-interleaving gives the coordinates back
    for (a, b, c), k in zip(u[:50], keys[:50]):
        assert sum(((k >> (3 * l + 2)) & 1) << l for l in range(7)) == a
        assert sum(((k >> (3 * l + 1)) & 1) << l for l in range(7)) == b
        assert sum(((k >> (3 * l)) & 1) << l for l in range(7)) == c


@pytest.mark.parametrize("S,p", [(1024, 0), (1024, 6), (4096, 2), (16384, 6), (777, 8)])
def test_segment_sort_properties(oracle, S, p):
    rng = np.random.default_rng(S + p)
    n = 20000
    keys = rng.integers(0, 1 << 40, n, dtype=np.uint64)
    keys[::7] = keys[3]                                      # many ties
    perm = oracle.segment_sort(keys, S, p)
    assert np.array_equal(np.sort(perm), np.arange(n))
    for s0 in range(0, n, S):
        seg = perm[s0:s0 + S]
        assert seg.min() >= s0 and seg.max() < s0 + S
        k = keys[seg] >> np.uint64(3 * p)
        assert (np.diff(k.astype(np.float64)) >= 0).all()
        ref = s0 + np.argsort(keys[s0:s0 + S] >> np.uint64(3 * p), kind="stable")
        assert np.array_equal(seg, ref)


def test_rindex_keys_and_snapshot_consistency(oracle):
    md = synth.md_fcc(cells=14, seed=2)
    x, y, z = (md[k].numpy() for k in ("xx", "yy", "zz"))
    perm, keys = oracle.rindex_perm(x, y, z, 1e-3, 1, 4096, 6)
    # keys rebuilt from the per-axis lattice with a different method
    qs = []
    for a in (x, y, z):
        ea, D = oracle.error_bound(a, 1e-3, 1)
        q, _ = oracle.lattice(a, D, ea)
        qs.append(q - q.min())
    b = int(max(int(q.max()) for q in qs)).bit_length()
    assert b <= 21
    k2 = np.zeros(x.size, np.uint64)
    for l in range(b):
        for sh, q in zip((2, 1, 0), qs):
            k2 |= ((q >> l) & 1).astype(np.uint64) << np.uint64(3 * l + sh)
    assert np.array_equal(keys, k2)
    streams, perm2 = oracle.compress_snapshot([x, y, z], 1e-3, 1, 8192, 128, 4096, 6)
    assert np.array_equal(perm, perm2)
    recon = [oracle.decompress(s) for s in streams]
    for a, r in zip((x, y, z), recon):
        ea, _ = oracle.error_bound(a, 1e-3, 1)
        assert (np.abs(a[perm].astype(np.float64) - r) <= ea).all()   # tuples kept together
        assert oracle.parse_header(streams[0])["flags"] & 2


def test_prx_trend_on_md(oracle):
    """Tables 4-5 trend: reordering raises the ratio on disordered MD data, and
    ignoring 6 digits keeps it (within a few percent of the full R-index sort)."""
    md = synth.md_fcc(cells=25, seed=2)
    f = [md[k].numpy() for k in ("xx", "yy", "zz")]
    raw = 12 * f[0].size
    lv = raw / sum(len(oracle.compress(a, 1e-4)) for a in f)
    rx = raw / sum(len(s) for s in oracle.compress_snapshot(f, 1e-4, 1, 8192, 128, 16384, 0)[0])
    prx = raw / sum(len(s) for s in oracle.compress_snapshot(f, 1e-4, 1, 8192, 128, 16384, 6)[0])
    assert rx > lv * 1.03 and prx > lv * 1.03
    assert abs(prx / rx - 1) < 0.05


# --------------------------------------------------------------------------
# LCF predictor (Sec. IV-A: the original SZ's linear curve fitting,
# pred_i = 2 x_{i-1} - x_{i-2}; Table 3, Fig. 4)
# --------------------------------------------------------------------------

def _sequential_sz_lcf(x, D: Fraction):
    """Textbook sequential SZ with the linear-curve-fitting predictor, in exact
    rational arithmetic: the prediction extrapolates the two previous
    *reconstructed* values (both 0 before the array)."""
    r1 = r2 = Fraction(0)
    codes, recon = [], []
    for xi in x:
        pred = 2 * r1 - r2
        k = _rne((Fraction(float(xi)) - pred) / D)
        r2, r1 = r1, pred + k * D
        codes.append(k + 32768 if -32767 <= k <= 32767 else 0)
        recon.append(np.float32(float(r1)))
    return codes, recon


@pytest.mark.parametrize("eb_abs", [2.0 ** -5, 0.0123, 3.7e-3])
def test_bruteforce_sequential_lcf(oracle, eb_abs):
    rng = np.random.default_rng(12)
    n = 400
    D = float(oracle.step(eb_abs))
    # a smooth trajectory: accelerations of a few lattice steps, one jump that escapes
    acc = rng.normal(0, 20, n) * D
    x = np.cumsum(np.cumsum(acc) * 0.05).astype(np.float32)
    x[200:] += np.float32(70000 * D)
    t = np.asarray([Fraction(float(v)) / Fraction(D) for v in x])
    frac = np.asarray([float(ti - math.floor(ti)) for ti in t])
    # away from half-steps: no ties, and |x| reaches ~600 here, where the float32
    # rounding of q*D could push an element within ulp/2 of D/2 past eb (verbatim)
    x = x[np.abs(frac - 0.5) > 0.02]
    codes_bf, recon_bf = _sequential_sz_lcf(x, Fraction(D))
    assert 0 in codes_bf                                      # the jump is an escape
    ea, Dd = oracle.error_bound(x, eb_abs, 0)
    q, v = oracle.lattice(x, Dd, ea)
    c, _ = oracle.codes_lcf(q, v)
    assert c.tolist() == codes_bf
    s = oracle.compress(x, eb_abs, kind=0, chunk=256, sub=16, pred=oracle.PRED_LCF)
    assert (_f32bits(oracle.decompress(s)) == _f32bits(recon_bf)).all()


def test_lcf_closed_forms(oracle):
    """Second differences: a line on the lattice predicts exactly from its
    third element on, a parabola c i^2 leaves the constant 2c, and a single
    spike J leaves +J, -2J, +J (the sign and index pattern of the formula)."""
    z = np.zeros(12, bool)
    i = np.arange(12, dtype=np.int64)
    _, d = oracle.codes_lcf(7 + 5 * i, z)
    assert d.tolist() == [7, 5 - 7] + [0] * 10
    _, d = oracle.codes_lcf(3 * i * i, z)
    assert d.tolist() == [0, 3] + [6] * 10
    q = np.zeros(12, np.int64)
    q[5] = 40000
    c, d = oracle.codes_lcf(q, z)
    assert d.tolist() == [0] * 5 + [40000, -80000, 40000] + [0] * 4
    assert c.tolist() == [32768] * 5 + [0, 0, 0] + [32768] * 4  # |delta| >= 32768 escapes


@pytest.mark.parametrize("n,chunk,sub", [(1, 256, 16), (2, 256, 16), (3, 256, 16), (257, 256, 16),
                                         (5000, 1024, 16), (70001, 4096, 64)])
def test_lcf_round_trip_equals_lv(oracle, n, chunk, sub):
    """Both predictors code the same lattice losslessly, so their streams
    decode to the same floats bit for bit (verbatim values, escapes and chunk
    anchors included); the LCF stream carries predictor 2 and two anchors
    (q_{b-1}, q_{b-2}) per chunk."""
    x = synth.random_walk_f32(n, n + 17, 0.3).numpy().copy()
    if n > 100:
        x[::53] = np.nan
        x[7::101] = np.inf
        x[30::97] += 5e3
    lv = oracle.compress(x, 1e-4, 1, chunk, sub)
    lcf = oracle.compress(x, 1e-4, 1, chunk, sub, pred=oracle.PRED_LCF)
    assert (_f32bits(oracle.decompress(lcf)) == _f32bits(oracle.decompress(lv))).all()
    h = oracle.parse_header(lcf)
    assert h["predictor"] == 2 and oracle.parse_header(lv)["predictor"] == 1
    if h["flags"] & 1:
        return
    nc = h["n_chunks"]
    anchors = np.frombuffer(lcf, np.int64, 2 * nc, h["off_chunk_anchor"])
    ea, D = oracle.error_bound(x, 1e-4, 1)
    q, _ = oracle.lattice(x, D, ea)
    for c in range(nc):
        b = c * chunk
        assert anchors[2 * c] == (q[b - 1] if b >= 1 else 0)
        assert anchors[2 * c + 1] == (q[b - 2] if b >= 2 else 0)


def test_lcf_rejects_unknown_predictor(oracle):
    s = bytearray(oracle.compress(synth.random_walk_f32(3000, 5).numpy(), 1e-4, 1, 1024, 16))
    s[43] = 3
    with pytest.raises(oracle.OracleError):
        oracle.decompress(bytes(s))


def test_lv_beats_lcf_on_particle_data(oracle):
    """Table 3 / Fig. 4 trend: on particle fields (no smoothness along the
    stored order) the last-value predictor has the smaller prediction error
    and the higher compression ratio than linear curve fitting."""
    snap = synth.cosmology(1 << 16, 16, 1)
    for f in synth.FIELDS:
        x = snap[f].numpy()
        xd = x.astype(np.float64)
        e_lv = np.sqrt(np.mean((xd[1:] - xd[:-1]) ** 2))
        e_lcf = np.sqrt(np.mean((xd[2:] - 2 * xd[1:-1] + xd[:-2]) ** 2))
        assert e_lv < e_lcf
        lv = len(oracle.compress(x, 1e-4, 1, 4096, 64))
        lcf = len(oracle.compress(x, 1e-4, 1, 4096, 64, pred=oracle.PRED_LCF))
        assert lv < lcf


# --------------------------------------------------------------------------
# Rate-distortion (Fig. 9): PSNR of uniform quantization and the rate slope
# --------------------------------------------------------------------------

def _rd_point(oracle, x, eb):
    s = oracle.compress(x, eb, 1, 4096, 64)
    y = oracle.decompress(s).astype(np.float64)
    xd = x.astype(np.float64)
    R = xd.max() - xd.min()
    mse = np.mean((xd - y) ** 2)
    return 8 * len(s) / x.size, (20 * math.log10(R / math.sqrt(mse)) if mse > 0 else None)


def test_rate_distortion_closed_forms(oracle):
    """Lattice step D = 2 eb R with errors spread uniformly over a step: RMSE
    = D / sqrt(12), so PSNR = -20 log10(eb / sqrt 3) (84.77 dB at 1e-4).  At
    high rate each decade of eb costs log2(10) bits, i.e. about 6.02 dB per
    bit.  A bound below the data's resolution falls back to the raw stream:
    32 bits per value, no error."""
    snap = synth.cosmology(1 << 16, 16, 1)
    for f in ("xx", "vx"):
        x = snap[f].numpy()
        pts = {eb: _rd_point(oracle, x, eb) for eb in (1e-2, 1e-3, 1e-4, 1e-5, 1e-8)}
        for eb in (1e-2, 1e-3, 1e-4, 1e-5):
            assert abs(pts[eb][1] - (-20 * math.log10(eb / math.sqrt(3)))) < 0.1
        bits = [pts[eb][0] for eb in (1e-2, 1e-3, 1e-4, 1e-5)]
        assert bits == sorted(bits)
        slope = (pts[1e-3][1] - pts[1e-2][1]) / (pts[1e-3][0] - pts[1e-2][0])
        assert 5.0 < slope < 6.6
        assert pts[1e-8] == (8 * (160 + 4 * x.size) / x.size, None)


# --------------------------------------------------------------------------
# SZ-CPC2000 coordinates (Sec. II CPC2000 steps 1-4; Sec. IV-B; Fig. 2)
# --------------------------------------------------------------------------

def _cpc_fields(s):
    h = struct.unpack_from("<IHHQ3d3IIqqqIIQQQ6Q", s, 0)
    return {"n": h[3], "D": h[7:10], "b": h[10], "qmin": h[11:14], "block": h[14], "subs": h[15], "nb": h[16],
            "ne": h[17], "words": h[18], "off": h[19:25]}


def test_cpc_golden_examples(oracle):
    for case in _load("cpc_examples.json")["cases"]:
        xyz = np.asarray(case["xyz"], np.float32)
        s, perm = oracle.compress_cpc(xyz[:, 0], xyz[:, 1], xyz[:, 2], 0.5, kind=0)
        h = _cpc_fields(s)
        assert list(h["qmin"]) == case["qmin"] and h["b"] == case["b"] and h["ne"] == 0
        assert perm.tolist() == case["perm"]
        assert struct.unpack_from("<Q", s, h["off"][0])[0] == case["first_key"]
        assert s[h["off"][2]] == case["k"]
        subs = struct.unpack_from("<32I", s, h["off"][3])
        assert subs[0] == 0 and all(v == case["bits"] for v in subs[1:])
        assert h["words"] == 1 and struct.unpack_from("<I", s, h["off"][5])[0] == case["word0"]
        back = oracle.decompress_cpc(s)
        for a in range(3):
            assert back[a].tolist() == xyz[perm, a].tolist()


def test_cpc_rice_parameter_is_the_cheapest(oracle):
    """The per-block k gives the fewest bits (smallest k on ties), and for
    geometric differences of mean m it sits near log2(m) (Golomb-Rice)."""
    rng = np.random.default_rng(8)
    for mean in (0.3, 5.0, 300.0, 70000.0):
        d = rng.geometric(1.0 / (mean + 1.0), 4096).astype(np.uint64) - 1
        k = oracle.cpc_choose_k(d)
        cost = [int(np.sum(d >> np.uint64(j))) + d.size * (1 + j) for j in range(64)]
        assert cost[k] == min(cost) and cost.index(min(cost)) == k
        assert abs(k - max(0.0, math.log2(mean))) <= 1.5
    assert oracle.cpc_rice_bits(9, 2) == 5 and oracle.cpc_rice_bits(0, 0) == 1


def _md_xyz(cells, seed=2):
    md = synth.md_fcc(cells=cells, seed=seed)
    return [md[k].numpy() for k in ("xx", "yy", "zz")]


@pytest.mark.parametrize("eb,kind", [(1e-3, 1), (1e-4, 1), (0.01, 0)])
def test_cpc_round_trip_is_the_sorted_lattice(oracle, eb, kind):
    """Decoding gives, at every sorted position j, the lattice reconstruction
    RN32(q D) of particle perm[j] (its verbatim value where the lattice
    misses the bound), and perm is the stable full R-index sort (the segment
    sort with one segment and no ignored digits)."""
    f = _md_xyz(12)
    f[1][::997] = np.nan
    f[2][5::1301] = np.inf
    s, perm = oracle.compress_cpc(*f, eb, kind)
    back = oracle.decompress_cpc(s)
    qs = []
    for a in range(3):
        ea, D = oracle.error_bound(f[a], eb, kind)
        q, v = oracle.lattice(f[a], D, ea)
        qs.append(q)
        want = np.where(v.astype(bool), f[a], np.array([oracle.recon(int(k), D) for k in q], np.float32))
        assert (_f32bits(back[a]) == _f32bits(want[perm])).all()
        fin = np.isfinite(f[a])
        assert (np.abs(f[a][perm][fin[perm]].astype(np.float64) - back[a][fin[perm]]) <= ea).all()
    keys, b = oracle.rindex_keys(*qs)
    assert b <= 21
    assert (perm == oracle.segment_sort(keys, f[0].size, 0)).all()
    assert _cpc_fields(s)["ne"] >= (~np.isfinite(f[1])).sum() + (~np.isfinite(f[2])).sum()


def test_cpc_block_edges_and_limits(oracle):
    for n in (0, 1, 2, 4095, 4096, 4097, 12289):
        f = [synth.uniform_f32(n, 30 + a, 0.0, 100.0).numpy() for a in range(3)]
        s, perm = oracle.compress_cpc(*f, 1e-3)
        h = _cpc_fields(s)
        assert h["n"] == n and h["nb"] == (n + 4095) // 4096
        back = oracle.decompress_cpc(s)
        for a in range(3):
            assert back[a].size == n
    # a bound so fine that a key would need more than 63 bits
    with pytest.raises(oracle.OracleError) as e:
        oracle.compress_cpc(*_md_xyz(5), 1e-8)
    assert e.value.rc == oracle.ERR_UNSUPPORTED


def test_cpc_trend_on_md(oracle):
    """Fig. 2 / Sec. IV-B trend: on disordered MD coordinates CPC2000 beats
    SZ-LV in stored order at both bounds and the segment-sorted SZ-LV-PRX
    at 1e-3."""
    f = _md_xyz(25)
    raw = 12 * f[0].size
    for eb in (1e-3, 1e-4):
        lv = raw / sum(len(oracle.compress(a, eb)) for a in f)
        cpc = raw / len(oracle.compress_cpc(*f, eb)[0])
        assert cpc > lv * 1.1
        if eb == 1e-3:
            prx = raw / sum(len(s) for s in oracle.compress_snapshot(f, eb, 1, 8192, 128, 16384, 6)[0])
            assert cpc > prx


# --------------------------------------------------------------------------
# R-index from velocities and from coordinates + velocities (Sec. IV-C,
# Fig. 3b, Table 6)
# --------------------------------------------------------------------------

def test_morton6_golden(oracle):
    """Hand-derived: bit 6k + (5 - a) holds bit k of axis a (xx leads, vz last)."""
    assert oracle.morton6([1, 0, 0, 0, 0, 1], 1) == 32 + 1
    assert oracle.morton6([0, 1, 0, 0, 0, 0], 2) == 1 << 4
    assert oracle.morton6([2, 0, 0, 0, 0, 0], 2) == 1 << 11
    assert oracle.morton6([0, 0, 0, 3, 0, 0], 2) == (1 << 2) | (1 << 8)


def test_six_axis_key_reduces_to_three_axis_order(oracle):
    """With every velocity equal, the 6-D key orders particles exactly as the
    3-D coordinate key (no bits dropped at this size), and a keyed snapshot
    with the coordinate key is the best_tradeoff snapshot."""
    md = synth.md_fcc(cells=6, seed=4)
    f = [md[k].numpy() for k in ("xx", "yy", "zz")]
    n = f[0].size
    vel = [np.full(n, 1.5, np.float32) for _ in range(3)]
    qs = []
    for a in f + vel:
        ea, D = oracle.error_bound(a, 1e-2, 0)
        qs.append(oracle.lattice(a, D, ea)[0])
    k3, b3 = oracle.rindex_keys(*qs[:3])
    k6, b6 = oracle.rindex_keys6(qs)
    assert b3 <= 10 and b6 == b3
    assert (oracle.segment_sort(k3, n, 0) == oracle.segment_sort(k6, n, 0)).all()
    s1, p1 = oracle.compress_snapshot_keyed(f, 1e-3, 1, 8192, 128, 4096, 6, oracle.KEY_XYZ)
    s2, p2 = oracle.compress_snapshot(f, 1e-3, 1, 8192, 128, 4096, 6)
    assert s1 == s2 and (p1 == p2).all()


def test_table6_per_variable_trend(oracle):
    """Table 6, per variable (segments of 4096): the velocity key raises the
    velocity fields' ratios and lowers the coordinates', and the
    coordinate + velocity key lands between the two single keys for every
    field.  (The table's overall finding on HACC -- no key helps -- comes from
    HACC's nearly sorted yy, which the synthetic snapshot does not have.)"""
    snap = synth.cosmology(1 << 17, 32, 1)
    fs = [snap[k].numpy() for k in synth.FIELDS]
    raw = 4 * fs[0].size
    cr = {}
    for key, p in ((oracle.KEY_XYZ, 6), (oracle.KEY_V, 6), (oracle.KEY_XYZV, 3)):
        streams, _ = oracle.compress_snapshot_keyed(fs, 1e-4, 1, 4096, 64, 4096, p, key)
        cr[key] = [raw / len(s) for s in streams]
    stored = [raw / len(oracle.compress(a, 1e-4, 1, 4096, 64)) for a in fs]
    for i in range(3):
        assert cr[oracle.KEY_V][i] < stored[i]
        assert cr[oracle.KEY_V][i] < cr[oracle.KEY_XYZV][i] < cr[oracle.KEY_XYZ][i]
    for i in range(3, 6):
        assert cr[oracle.KEY_V][i] > stored[i]
        assert cr[oracle.KEY_XYZ][i] < cr[oracle.KEY_XYZV][i] < cr[oracle.KEY_V][i]
