"""CPU oracle for the SZ-LV path of arXiv 1711.03888 (test infrastructure).

This package is test infrastructure, not part of the product: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it.  It wraps ``sz_oracle.c`` (plain single-threaded C,
IEEE binary64, ``-ffp-contract=off``) through ctypes.  It shares no code with
the CUDA path.

Paper anchors (section / table of arXiv 1711.03888):
  * Sec. III, pointwise compression error: |x_i - x'_i| <= eb_abs, eb_rel = eb_abs / R.
  * Sec. II, CPC2000 step 1: floats are turned into integers by dividing by the bound.
  * Sec. IV-A: last-value prediction, linear-scaling quantization, Huffman coding.
  * Sec. IV-B, Fig. 3(a), Tables 4-5: R-index keys and the segment-wise partial radix sort.
"""
from __future__ import annotations

import ctypes as C
import os
import struct
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sz_oracle.c")
_LIB = os.path.join(_HERE, "libsz_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOMEM, ERR_CAPACITY, ERR_CORRUPT, ERR_UNSUPPORTED = 0, 1, 2, 3, 4, 5
HEADER_BYTES = 160
FLAG_RAW, FLAG_REORDERED = 1, 2
PRED_LV, PRED_LCF = 1, 2          # header byte 43


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain C, no contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                            "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        u64, i32, dbl, vp = C.c_uint64, C.c_int, C.c_double, C.c_void_p
        L.szo_value_range.restype = dbl
        L.szo_value_range.argtypes = [vp, u64]
        L.szo_step.restype = C.c_float
        L.szo_step.argtypes = [dbl]
        L.szo_error_bound.restype = i32
        L.szo_error_bound.argtypes = [vp, u64, dbl, i32, vp, vp]
        L.szo_lattice.restype = None
        L.szo_lattice.argtypes = [vp, u64, C.c_float, dbl, vp, vp]
        L.szo_recon.restype = C.c_float
        L.szo_recon.argtypes = [C.c_int64, C.c_float]
        L.szo_codes.restype = None
        L.szo_codes.argtypes = [vp, vp, u64, vp, vp]
        L.szo_huffman_lengths.restype = i32
        L.szo_huffman_lengths.argtypes = [vp, vp, C.c_uint32, vp]
        L.szo_canonical_codes.restype = None
        L.szo_canonical_codes.argtypes = [vp, C.c_uint32, vp]
        L.szo_max_bytes.restype = u64
        L.szo_max_bytes.argtypes = [u64]
        L.szo_codes_lcf.restype = None
        L.szo_codes_lcf.argtypes = [vp, vp, u64, vp, vp]
        L.szo_compress.restype = i32
        L.szo_compress.argtypes = [vp, u64, dbl, i32, C.c_uint32, C.c_uint32, C.c_uint32, vp, u64, vp]
        L.szo_compress_pred.restype = i32
        L.szo_compress_pred.argtypes = [vp, u64, dbl, i32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                        vp, u64, vp]
        L.szo_stream_n.restype = i32
        L.szo_stream_n.argtypes = [vp, u64, vp]
        L.szo_decompress.restype = i32
        L.szo_decompress.argtypes = [vp, u64, vp, u64, vp]
        L.szo_morton3.restype = u64
        L.szo_morton3.argtypes = [u64, u64, u64, i32]
        L.szo_rindex_keys.restype = None
        L.szo_rindex_keys.argtypes = [vp, vp, vp, u64, vp, vp]
        L.szo_segment_sort.restype = i32
        L.szo_segment_sort.argtypes = [vp, u64, C.c_uint32, C.c_uint32, vp]
        L.szo_rindex_perm.restype = i32
        L.szo_rindex_perm.argtypes = [vp, vp, vp, u64, vp, vp, C.c_uint32, C.c_uint32, vp, vp]
        L.szo_morton6.restype = u64
        L.szo_morton6.argtypes = [vp, i32]
        L.szo_rindex_keys6.restype = None
        L.szo_rindex_keys6.argtypes = [vp, u64, vp, vp]
        L.szo_cpc_rice_bits.restype = u64
        L.szo_cpc_rice_bits.argtypes = [u64, i32]
        L.szo_cpc_choose_k.restype = i32
        L.szo_cpc_choose_k.argtypes = [vp, u64]
        L.szo_cpc_max_bytes.restype = i32
        L.szo_cpc_max_bytes.argtypes = [u64, vp]
        L.szo_compress_cpc.restype = i32
        L.szo_compress_cpc.argtypes = [vp, vp, vp, u64, vp, i32, vp, u64, vp, vp]
        L.szo_decompress_cpc.restype = i32
        L.szo_decompress_cpc.argtypes = [vp, u64, vp, vp, vp, u64, vp]
        L.szo_compress_snapshot.restype = i32
        L.szo_compress_snapshot.argtypes = [i32, vp, u64, vp, i32, C.c_uint32, C.c_uint32,
                                            C.c_uint32, C.c_uint32, vp, vp, vp, vp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


class OracleError(RuntimeError):
    def __init__(self, rc: int, what: str):
        super().__init__(f"{what}: oracle status {rc}")
        self.rc = rc


def value_range(x) -> float:
    x = _f32(x)
    return lib().szo_value_range(_p(x), x.size)


def step(eb_abs: float) -> np.float32:
    return np.float32(lib().szo_step(eb_abs))


def error_bound(x, eb: float, kind: int):
    """(eb_abs, D) for an absolute (kind 0) or value-range relative (kind 1) bound."""
    x = _f32(x)
    ea = C.c_double()
    d = C.c_float()
    rc = lib().szo_error_bound(_p(x), x.size, eb, kind, C.byref(ea), C.byref(d))
    if rc:
        raise OracleError(rc, "error_bound")
    return ea.value, np.float32(d.value)


def lattice(x, D: float, eb_abs: float):
    """Per-element lattice index q and verbatim flag."""
    x = _f32(x)
    q = np.zeros(x.size, np.int64)
    v = np.zeros(x.size, np.uint8)
    lib().szo_lattice(_p(x), x.size, np.float32(D), eb_abs, _p(q), _p(v))
    return q, v.astype(bool)


def recon(q: int, D: float) -> np.float32:
    return np.float32(lib().szo_recon(int(q), np.float32(D)))


def codes(q, verbatim):
    q = np.ascontiguousarray(q, np.int64)
    v = np.ascontiguousarray(verbatim, np.uint8)
    c = np.zeros(q.size, np.uint16)
    d = np.zeros(q.size, np.int64)
    lib().szo_codes(_p(q), _p(v), q.size, _p(c), _p(d))
    return c, d


def codes_lcf(q, verbatim):
    """Second-difference (LCF) codes on the lattice: delta_i = q_i - 2 q_{i-1} + q_{i-2}."""
    q = np.ascontiguousarray(q, np.int64)
    v = np.ascontiguousarray(verbatim, np.uint8)
    c = np.zeros(q.size, np.uint16)
    d = np.zeros(q.size, np.int64)
    lib().szo_codes_lcf(_p(q), _p(v), q.size, _p(c), _p(d))
    return c, d


def huffman_lengths(freq, sym=None) -> np.ndarray:
    """Code lengths for used symbols (ascending symbol order) with their counts."""
    f = np.ascontiguousarray(freq, np.uint64)
    s = np.arange(f.size, dtype=np.uint32) if sym is None else np.ascontiguousarray(sym, np.uint32)
    out = np.zeros(f.size, np.uint8)
    rc = lib().szo_huffman_lengths(_p(f), _p(s), f.size, _p(out))
    if rc:
        raise OracleError(rc, "huffman_lengths")
    return out


def canonical_codes(lengths) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, np.uint8)
    out = np.zeros(ln.size, np.uint32)
    lib().szo_canonical_codes(_p(ln), ln.size, _p(out))
    return out


def max_bytes(n: int) -> int:
    return int(lib().szo_max_bytes(n))


def compress(x, eb: float, kind: int = 1, chunk: int = 8192, sub: int = 128, reordered: bool = False,
             pred: int = PRED_LV) -> bytes:
    """Compress one float32 array; returns the stream bytes.  pred: PRED_LV
    (Sec. IV-A last value) or PRED_LCF (the original SZ's curve fitting)."""
    x = _f32(x)
    cap = max_bytes(x.size)
    out = np.zeros(cap, np.uint8)
    nb = C.c_uint64()
    rc = lib().szo_compress_pred(_p(x), x.size, eb, kind, chunk, sub, FLAG_REORDERED if reordered else 0,
                                 pred, _p(out), cap, C.byref(nb))
    if rc:
        raise OracleError(rc, "compress")
    return out[: nb.value].tobytes()


def decompress(stream: bytes) -> np.ndarray:
    buf = np.frombuffer(stream, np.uint8).copy()
    n = C.c_uint64()
    rc = lib().szo_stream_n(_p(buf), buf.size, C.byref(n))
    if rc:
        raise OracleError(rc, "stream_n")
    out = np.zeros(max(n.value, 1), np.float32)
    no = C.c_uint64()
    rc = lib().szo_decompress(_p(buf), buf.size, _p(out), n.value, C.byref(no))
    if rc:
        raise OracleError(rc, "decompress")
    return out[: no.value]


def morton3(ux: int, uy: int, uz: int, bits: int) -> int:
    return int(lib().szo_morton3(ux, uy, uz, bits))


def rindex_keys(qx, qy, qz):
    qx, qy, qz = (np.ascontiguousarray(a, np.int64) for a in (qx, qy, qz))
    k = np.zeros(qx.size, np.uint64)
    b = C.c_int()
    lib().szo_rindex_keys(_p(qx), _p(qy), _p(qz), qx.size, _p(k), C.byref(b))
    return k, b.value


def segment_sort(keys, segment: int, ignored_digits: int) -> np.ndarray:
    k = np.ascontiguousarray(keys, np.uint64)
    perm = np.zeros(k.size, np.uint32)
    rc = lib().szo_segment_sort(_p(k), k.size, segment, ignored_digits, _p(perm))
    if rc:
        raise OracleError(rc, "segment_sort")
    return perm


def rindex_perm(x, y, z, eb: float, kind: int, segment: int, ignored_digits: int):
    """Permutation of the MD reordering (R-index keys of the three coordinates)."""
    xs = [_f32(a) for a in (x, y, z)]
    D = np.zeros(3, np.float32)
    ea = np.zeros(3, np.float64)
    for a in range(3):
        ea[a], D[a] = error_bound(xs[a], eb, kind)
    n = xs[0].size
    perm = np.zeros(n, np.uint32)
    keys = np.zeros(n, np.uint64)
    rc = lib().szo_rindex_perm(_p(xs[0]), _p(xs[1]), _p(xs[2]), n, _p(D), _p(ea), segment,
                               ignored_digits, _p(perm), _p(keys))
    if rc:
        raise OracleError(rc, "rindex_perm")
    return perm, keys


def compress_snapshot(fields, eb, kind: int = 1, chunk: int = 8192, sub: int = 128,
                      segment: int = 16384, ignored_digits: int = 6):
    """MD mode (best_tradeoff): reorder all fields by the R-index segment sort,
    then compress each with LV.  Returns (streams, perm)."""
    fs = [_f32(f) for f in fields]
    n = fs[0].size
    nf = len(fs)
    ebs = np.asarray(eb if np.ndim(eb) else [eb] * nf, np.float64)
    caps = np.full(nf, max_bytes(n), np.uint64)
    outs = [np.zeros(int(caps[0]), np.uint8) for _ in range(nf)]
    in_ptrs = (C.c_void_p * nf)(*[f.ctypes.data for f in fs])
    out_ptrs = (C.c_void_p * nf)(*[o.ctypes.data for o in outs])
    nbytes = np.zeros(nf, np.uint64)
    perm = np.zeros(max(n, 1), np.uint32)
    rc = lib().szo_compress_snapshot(nf, C.cast(in_ptrs, C.c_void_p), n, _p(ebs), kind, chunk, sub,
                                     segment, ignored_digits, C.cast(out_ptrs, C.c_void_p), _p(caps),
                                     _p(nbytes), _p(perm))
    if rc:
        raise OracleError(rc, "compress_snapshot")
    return [outs[f][: int(nbytes[f])].tobytes() for f in range(nf)], perm[:n]


def morton6(u, bits: int) -> int:
    a = np.ascontiguousarray(u, np.uint64)
    return int(lib().szo_morton6(_p(a), bits))


def rindex_keys6(qs):
    """R-index keys from six lattice arrays (xx, yy, zz, vx, vy, vz); returns
    (keys, bits per axis)."""
    arrs = [np.ascontiguousarray(q, np.int64) for q in qs]
    ptrs = (C.c_void_p * 6)(*[a.ctypes.data for a in arrs])
    k = np.zeros(max(arrs[0].size, 1), np.uint64)
    b = C.c_int()
    lib().szo_rindex_keys6(C.cast(ptrs, C.c_void_p), arrs[0].size, _p(k), C.byref(b))
    return k[: arrs[0].size], b.value


KEY_XYZ, KEY_V, KEY_XYZV = 0, 1, 2


def compress_snapshot_keyed(fields, eb, kind: int = 1, chunk: int = 8192, sub: int = 128, segment: int = 16384,
                            ignored_digits: int = 6, key: int = KEY_XYZ):
    """best_tradeoff with the R-index built from the coordinates (Fig. 3a),
    the velocities (fields 3-5) or all six (Fig. 3b; digits of 6 bits):
    every field reordered by the segment sort of that key, then SZ-LV.
    Returns (streams, perm)."""
    fs = [_f32(f) for f in fields]
    nf = len(fs)
    ebs = list(eb) if np.ndim(eb) else [eb] * nf
    axes = {KEY_XYZ: (0, 1, 2), KEY_V: (3, 4, 5), KEY_XYZV: (0, 1, 2, 3, 4, 5)}[key]
    qs = []
    for a in axes:
        ea, D = error_bound(fs[a], ebs[a], kind)
        q, _ = lattice(fs[a], D, ea) if D != 0 else (np.zeros(fs[a].size, np.int64), None)
        qs.append(q)
    if key == KEY_XYZV:
        keys, _ = rindex_keys6(qs)
        perm = segment_sort(keys, segment, 2 * ignored_digits)    # 6-bit digits: shift 6p
    else:
        keys, _ = rindex_keys(*qs)
        perm = segment_sort(keys, segment, ignored_digits)
    return [compress(f[perm], ebs[i], kind, chunk, sub, reordered=True) for i, f in enumerate(fs)], perm


def cpc_rice_bits(d: int, k: int) -> int:
    return int(lib().szo_cpc_rice_bits(d, k))


def cpc_choose_k(deltas) -> int:
    d = np.ascontiguousarray(deltas, np.uint64)
    return int(lib().szo_cpc_choose_k(_p(d), d.size))


def compress_cpc(x, y, z, eb, kind: int = 1):
    """SZ-CPC2000 coordinates (Sec. II CPC2000 steps 1-4): one stream for the
    three coordinate arrays; returns (stream, perm), perm[j] = the original
    index of the particle at sorted position j."""
    f = [_f32(a) for a in (x, y, z)]
    n = f[0].size
    ebs = np.asarray(eb if np.ndim(eb) else [eb] * 3, np.float64)
    cap = C.c_uint64()
    lib().szo_cpc_max_bytes(n, C.byref(cap))
    out = np.zeros(cap.value, np.uint8)
    nb = C.c_uint64()
    perm = np.zeros(max(n, 1), np.uint32)
    rc = lib().szo_compress_cpc(_p(f[0]), _p(f[1]), _p(f[2]), n, _p(ebs), kind, _p(out), cap.value, C.byref(nb),
                                _p(perm))
    if rc:
        raise OracleError(rc, "compress_cpc")
    return out[: nb.value].tobytes(), perm[:n]


def decompress_cpc(stream: bytes):
    buf = np.frombuffer(stream, np.uint8).copy()
    n = struct.unpack_from("<Q", buf, 8)[0] if buf.size >= 16 else 0
    outs = [np.zeros(max(n, 1), np.float32) for _ in range(3)]
    no = C.c_uint64()
    rc = lib().szo_decompress_cpc(_p(buf), buf.size, _p(outs[0]), _p(outs[1]), _p(outs[2]), n, C.byref(no))
    if rc:
        raise OracleError(rc, "decompress_cpc")
    return [o[: no.value] for o in outs]


def compress_snapshot_cpc(fields, eb, kind: int = 1, chunk: int = 8192, sub: int = 128):
    """SZ-CPC2000 (Sec. IV-B, best_compression): the coordinates (fields 0-2)
    by CPC2000, every further field reordered by the same permutation and
    compressed with SZ-LV.  Returns ([coordinate stream, further streams...],
    perm)."""
    nf = len(fields)
    ebs = list(eb) if np.ndim(eb) else [eb] * nf
    s, perm = compress_cpc(fields[0], fields[1], fields[2], ebs[:3], kind)
    rest = [compress(_f32(fields[f])[perm], ebs[f], kind, chunk, sub, reordered=True) for f in range(3, nf)]
    return [s] + rest, perm


_HDR = struct.Struct("<IHHQdIIIIHBBIQQQQ8QQQ")


def parse_header(stream: bytes) -> dict:
    """Decode the 160-byte stream header into a dict (format description)."""
    v = _HDR.unpack_from(stream, 0)
    keys = ["magic", "version", "header_bytes", "n", "eb_abs", "D_bits", "flags", "chunk", "sub",
            "m_bits", "max_len", "predictor", "reserved0", "n_chunks", "n_symbols", "n_escapes",
            "payload_words", "off_syms", "off_lens", "off_chunk_word", "off_chunk_anchor",
            "off_chunk_esc", "off_sublen", "off_escapes", "off_payload", "total_bytes", "reserved1"]
    h = dict(zip(keys, v))
    h["D"] = struct.unpack("<f", struct.pack("<I", h["D_bits"]))[0]
    return h


def stream_codebook(stream: bytes):
    """(symbols, lengths) arrays of the codebook section."""
    h = parse_header(stream)
    m = h["n_symbols"]
    syms = np.frombuffer(stream, np.uint16, m, h["off_syms"]).copy()
    lens = np.frombuffer(stream, np.uint8, m, h["off_lens"]).copy()
    return syms, lens
