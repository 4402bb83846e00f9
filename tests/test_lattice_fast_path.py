"""The GPU's single-precision shortcut for the value -> lattice conversion
(a2), checked exhaustively on CPU against the oracle's binary64 definition
q = RNE(RN64(x / D)), verbatim iff |x - RN32(RN64(q D))| > eb_abs.

The device code (sz_device.cuh, lattice_q) takes the candidate
qc = rint(RN32(x * RN32(1/D))) and the residual r = fmaf(-qc, D, x).  It keeps
qc when |r| <= thr_lo = RD32(D (1/2 - 2^-20)), tries qc +- 1 when
|r| >= thr_hi = RU32(D (1/2 + 2^-20)), and otherwise (a near-tie) falls back
to binary64.  Kept candidates reconstruct with one float multiply and take the
verbatim test in float against RD32(eb_abs).  The argument that this equals
the binary64 definition is short but easy to get subtly wrong, so this test
replays the single-precision steps exactly in numpy for every float in the
binades where the shortcut runs (|x / D| from 2^-2 to 2^22, every mantissa,
positive values; a random sample of negative ones) and compares q and the
verbatim flag with the oracle's.  It also checks that only near-ties fall back,
and that they are rare for a step with a full 24-bit mantissa.
"""
import numpy as np
import pytest

F32, F64 = np.float32, np.float64


def _rd32(v: float) -> np.float32:
    f = F32(v)
    return np.nextafter(f, F32(-np.inf)) if F64(f) > v else f


def _ru32(v: float) -> np.float32:
    f = F32(v)
    return np.nextafter(f, F32(np.inf)) if F64(f) < v else f


def _fma32(a: np.ndarray, D: np.float32, x: np.ndarray) -> np.ndarray:
    """RN32(a * D + x) with one rounding, for float32 a, D, x.  a * D is exact
    in binary64 (24 + 24 bits); the binary64 sum is checked exact with a
    TwoSum residual, so the final conversion is the only rounding."""
    p = a.astype(F64) * F64(D)
    xd = x.astype(F64)
    s = p + xd
    bp = s - xd
    err = (p - bp) + (xd - (s - bp))
    assert not err.any(), "binary64 sum inexact: the emulation would round twice"
    return s.astype(F32)


def _fast_path(x: np.ndarray, D: np.float32, eb_abs: float):
    """The device shortcut: (taken, q, verbatim) per element."""
    inv = F32(1.0) / D
    thr_lo = _rd32(F64(D) * (0.5 - 2.0 ** -20))
    thr_hi = _ru32(F64(D) * (0.5 + 2.0 ** -20))
    ebf = _rd32(eb_abs)
    t = x * inv
    inside = np.abs(t) < F32(4194304.0)
    qc = np.rint(t)
    r = _fma32(-qc, D, x)
    ar = np.abs(r)
    ok = ar <= thr_lo
    retry = ~ok & (ar >= thr_hi)
    qc2 = qc + np.where(r > 0, F32(1.0), F32(-1.0))
    r2 = _fma32(-qc2, D, x)
    ok2 = retry & (np.abs(r2) <= thr_lo)
    q = np.where(ok2, qc2, qc)
    taken = inside & (ok | ok2)
    xr = q * D
    verb = np.abs(x - xr) > ebf
    return taken, q.astype(np.int64), verb


def _binade(e: int, sign: float = 1.0) -> np.ndarray:
    """Every float32 in [2^e, 2^(e+1)) (times sign)."""
    bits = (np.uint32(e + 127) << np.uint32(23)) | np.arange(1 << 23, dtype=np.uint32)
    return (bits.view(F32) * F32(sign)).astype(F32)


# D = RZ32(2 eb): a power of two; a full 24-bit mantissa, for which exact
# half-ties of x / D are rare; and 3 = 1.5 * 2, whose short mantissa makes
# x = 1.5 (2k + 1) exact ties common again
CASES = [(F32(2.0 ** -9), 2.0 ** -10),
         (F32(0.0512), 0.0256),
         (F32(3.0), 1.5)]
RARE_TIES = {float(F32(0.0512))}


@pytest.mark.parametrize("D,eb_abs", CASES[:2])
def test_fast_path_equals_binary64_definition(oracle, D, eb_abs):
    assert F32(D) == D
    lo = int(np.floor(np.log2(float(D)))) - 2
    hi = int(np.ceil(np.log2(float(D)))) + 22
    taken_total = seen = 0
    for e in range(lo, hi + 1):
        x = _binade(e)
        taken, q, verb = _fast_path(x, D, eb_abs)
        qo, vo = oracle.lattice(x, float(D), eb_abs)
        bad = taken & ((q != qo) | (verb != vo.astype(bool)))
        assert not bad.any(), (f"D={D} binade 2^{e}: {int(bad.sum())} mismatches, first x="
                               f"{x[bad][0]!r} q={q[bad][0]} oracle q={qo[bad][0]}")
        inside = np.abs(x * (F32(1.0) / D)) < F32(4194304.0)
        # the binary64 fallback is taken only for near-ties of x / D
        t = x[inside & ~taken].astype(F64) / F64(D)
        assert (np.abs(np.abs(t - np.floor(t) - 0.5)) <= 2.0 ** -18).all()
        taken_total += int(taken.sum())
        seen += int(inside.sum())
    assert seen > 0
    if float(D) in RARE_TIES:
        # a full-mantissa step: the fallback runs for about 2^-19 of the
        # inputs.  (With a power-of-two step x / D is exact, and the top
        # binades hold many exact half-ties, which the fallback decides by
        # design.)
        assert (seen - taken_total) / seen < 1e-4


@pytest.mark.parametrize("D,eb_abs", CASES)
def test_fast_path_negative_values_sample(oracle, D, eb_abs):
    rng = np.random.default_rng(11)
    lo = int(np.floor(np.log2(float(D)))) - 2
    hi = int(np.ceil(np.log2(float(D)))) + 22
    e = rng.integers(lo, hi + 1, 1 << 22)
    m = rng.integers(0, 1 << 23, 1 << 22).astype(np.uint32)
    bits = ((e + 127).astype(np.uint32) << np.uint32(23)) | m | np.uint32(1 << 31)
    x = bits.view(F32)
    taken, q, verb = _fast_path(x, D, eb_abs)
    qo, vo = oracle.lattice(x, float(D), eb_abs)
    bad = taken & ((q != qo) | (verb != vo.astype(bool)))
    assert not bad.any()
    inside = np.abs(x * (F32(1.0) / D)) < F32(4194304.0)
    assert taken.sum() / inside.sum() > (0.999 if float(D) in RARE_TIES else 0.9)


def test_candidate_alone_is_not_enough(oracle):
    """The comparison has teeth: near |x / D| = 2^22 the float candidate
    rint(RN32(x * RN32(1/D))) alone is off by one for many inputs (the two
    roundings err by up to about 0.4), and the check above would see it.  The
    residual test is what makes the shortcut exact."""
    D, eb_abs = CASES[1]
    x = _binade(int(np.floor(np.log2(float(D)))) + 21)
    qc = np.rint(x * (F32(1.0) / D)).astype(np.int64)
    qo, _ = oracle.lattice(x, float(D), eb_abs)
    wrong = qc != qo
    assert wrong.mean() > 0.01
    taken, q, _ = _fast_path(x[wrong], D, eb_abs)
    assert (q[taken] == qo[wrong][taken]).all() and taken.mean() > 0.99


@pytest.mark.parametrize("D", [F32(2.0 ** -9), F32(0.0512), F32(3.0), F32(2.0 ** -140), F32(1e30)])
def test_reconstruction_shortcut_every_small_q(D):
    """The decoder's shortcut (sz_device.cuh, recon_f; the 32-bit loop of
    k_decode.cu): for |q| <= 2^24 one float multiply RN32(float(q) * D)
    equals the definition RN32(RN64(q * D)), for every such q, a subnormal
    step and a step whose products overflow included."""
    q = np.arange(-(1 << 24), (1 << 24) + 1, dtype=np.int64)
    with np.errstate(over="ignore"):
        short = q.astype(F32) * D
        ref = (q.astype(F64) * F64(D)).astype(F32)
    assert np.array_equal(short.view(np.uint32), ref.view(np.uint32))
