"""Python binding of the GB300 SZ-LV compressor (C ABI in include/sz_gb300.h).

Argument marshalling only: tensors become device pointers, the current torch
stream becomes the CUDA stream, and sizes come back through sz_sync().  Every
step of compression and decompression runs in the CUDA kernels of
libsz_gb300.so; there is no CPU fallback.  If the shared library is missing,
importing this package raises.  Build it with build.build() (or
__graft_entry__.build()).

The functions keep the C names.  A `Context` wraps an sz_ctx* and keeps the
host size holders alive until sz_sync().
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsz_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: the GB300 library must be built (paper_1711_03888_gb300.build)")

_lib = C.CDLL(LIB_PATH)

SZ_OK, SZ_ERR_ARG, SZ_ERR_NOMEM, SZ_ERR_CAPACITY, SZ_ERR_CORRUPT, SZ_ERR_CUDA, SZ_ERR_TIMEOUT, \
    SZ_ERR_UNSUPPORTED, SZ_ERR_BUSY = range(9)
SZ_EB_ABS, SZ_EB_REL = 0, 1
SZ_MODE_LV, SZ_MODE_LV_PRX, SZ_MODE_CPC2000 = 0, 1, 2
SZ_PRED_DEFAULT, SZ_PRED_LV, SZ_PRED_LCF = 0, 1, 2
SZ_KEY_XYZ, SZ_KEY_V, SZ_KEY_XYZV = 0, 1, 2
SZ_FIELD_XX, SZ_FIELD_YY, SZ_FIELD_ZZ, SZ_FIELD_VX, SZ_FIELD_VY, SZ_FIELD_VZ, SZ_FIELD_OTHER = range(7)
SZ_OP_COMPRESS, SZ_OP_DECOMPRESS = 0, 1
HEADER_BYTES = 160

EXPORTS = ("sz_ctx_create", "sz_ctx_destroy", "sz_max_compressed_bytes", "sz_compress", "sz_decompress",
           "sz_compress_batch", "sz_decompress_batch", "sz_compress_host", "sz_decompress_host", "sz_compress_snapshot",
           "sz_cpc_max_bytes", "sz_decompress_cpc", "sz_sync", "sz_status_string",
           "sz_profile_enable", "sz_profile_read", "sz_compress_noalloc", "sz_check_wait_timeout",
           "sz_ctx_set_autotune", "sz_batch_tuning",
           "sz_serve_start", "sz_serve_submit", "sz_serve_poll", "sz_serve_wait", "sz_serve_release",
           "sz_serve_stats", "sz_serve_stop")
PHASES = ("range", "quant", "codebook", "encode", "decode_setup", "decode", "reorder", "batch", "encode_sizes")


class sz_params(C.Structure):
    _fields_ = [("chunk_elems", C.c_uint32), ("sub_elems", C.c_uint32),
                ("segment", C.c_uint32), ("ignored_digits", C.c_uint32), ("predictor", C.c_uint32),
                ("key_fields", C.c_uint32)]


class sz_tuning(C.Structure):
    _fields_ = [("chunk_elems", C.c_uint32), ("fixed_chunk_elems", C.c_uint32), ("class_lo", C.c_uint64),
                ("class_hi", C.c_uint64), ("trial_ms", C.c_float * 4), ("range_tile", C.c_uint32),
                ("quant_group", C.c_uint32), ("tile_trial_ms", C.c_float * 4)]


class sz_request(C.Structure):
    _fields_ = [("op", C.c_int), ("input", C.c_void_p), ("n", C.c_size_t), ("in_bytes", C.c_size_t),
                ("out", C.c_void_p), ("out_cap", C.c_size_t), ("eb", C.c_double), ("kind", C.c_int)]


class sz_result(C.Structure):
    _fields_ = [("status", C.c_int), ("out_size", C.c_size_t), ("latency_s", C.c_double), ("out", C.c_void_p)]


class sz_serve_counters(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("peak_inflight", C.c_uint32),
                ("peak_queue", C.c_uint32), ("peak_bytes", C.c_size_t), ("budget_waits", C.c_uint64)]


_vp, _sz, _st = C.c_void_p, C.c_size_t, C.c_int
_sig = {
    "sz_ctx_create": (_st, [C.POINTER(_vp), C.c_int, _sz]),
    "sz_ctx_destroy": (_st, [_vp]),
    "sz_max_compressed_bytes": (_sz, [_sz]),
    "sz_compress": (_st, [_vp, _vp, _sz, C.c_double, C.c_int, C.POINTER(sz_params), _vp, _sz,
                          C.POINTER(_sz), _vp]),
    "sz_decompress": (_st, [_vp, _vp, _sz, _vp, _sz, C.POINTER(_sz), _vp]),
    "sz_compress_batch": (_st, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_sz), C.POINTER(C.c_double), C.c_int,
                                C.POINTER(sz_params), C.POINTER(_vp), C.POINTER(_sz), C.POINTER(_sz), _vp]),
    "sz_decompress_batch": (_st, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_sz), C.POINTER(_vp), C.POINTER(_sz),
                                  C.POINTER(_sz), _vp]),
    "sz_compress_host": (_st, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_sz), C.POINTER(C.c_double), C.c_int,
                               C.POINTER(sz_params), C.POINTER(_vp), C.POINTER(_sz), C.POINTER(_sz), _vp]),
    "sz_decompress_host": (_st, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_sz), C.POINTER(_vp), C.POINTER(_sz),
                                 C.POINTER(_sz), _vp]),
    "sz_compress_snapshot": (_st, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(_vp), _sz, C.POINTER(C.c_double),
                                   C.c_int, C.c_int, C.POINTER(sz_params), C.POINTER(_vp), C.POINTER(_sz),
                                   C.POINTER(_sz), _vp, _vp]),
    "sz_cpc_max_bytes": (_sz, [_sz]),
    "sz_decompress_cpc": (_st, [_vp, _vp, _sz, C.POINTER(_vp), _sz, C.POINTER(_sz), _vp]),
    "sz_sync": (_st, [_vp, _vp]),
    "sz_status_string": (C.c_char_p, [C.c_int]),
    "sz_compress_noalloc": (_st, [_vp, _sz, C.c_double, C.c_int, _vp, _sz, C.POINTER(_sz), _vp]),
    "sz_check_wait_timeout": (_st, [_vp, C.c_uint32, _vp]),
    "sz_ctx_set_autotune": (_st, [_vp, C.c_int]),
    "sz_batch_tuning": (_st, [_vp, _sz, C.POINTER(sz_tuning)]),
    "sz_profile_enable": (_st, [_vp, C.c_int]),
    "sz_profile_read": (_st, [_vp, C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.c_int]),
    "sz_serve_start": (_st, [_vp, C.c_int]),
    "sz_serve_submit": (_st, [_vp, C.POINTER(sz_request), C.POINTER(C.c_uint64)]),
    "sz_serve_poll": (_st, [_vp, C.c_uint64, C.POINTER(sz_result)]),
    "sz_serve_wait": (_st, [_vp, C.c_uint64, C.c_double, C.POINTER(sz_result)]),
    "sz_serve_release": (_st, [_vp, _vp]),
    "sz_serve_stats": (_st, [_vp, C.POINTER(sz_serve_counters)]),
    "sz_serve_stop": (_st, [_vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class SzError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = _lib.sz_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)
        self.status = status


def _check(status: int, what: str):
    if status != SZ_OK:
        raise SzError(status, what)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


_F32, _U8, _I32 = "float32", "uint8", "int32"


def _arg(t, dtype: str, device: str, what: str, min_numel: int = 0):
    """Check a tensor before its address crosses the C ABI, which takes raw
    pointers and element counts: the element type, one contiguous block, the
    memory the call expects ("cuda" for device calls, "cpu" for the host-memory
    calls) and, where a count is passed beside it, enough elements."""
    if str(t.dtype) != "torch." + dtype:
        raise SzError(SZ_ERR_ARG, f"{what}: {t.dtype}, expected torch.{dtype}")
    if not t.is_contiguous():
        raise SzError(SZ_ERR_ARG, f"{what}: not contiguous")
    if t.device.type != device:
        raise SzError(SZ_ERR_ARG, f"{what}: on {t.device}, expected {device} memory")
    min_numel = int(getattr(min_numel, "value", min_numel))
    if t.numel() < min_numel:
        raise SzError(SZ_ERR_ARG, f"{what}: {t.numel()} elements, {min_numel} needed")
    return t


def _cap(t, cap, what: str) -> int:
    """An explicit capacity may not pass the tensor's own size."""
    if cap is None:
        return t.numel()
    cap = int(getattr(cap, "value", cap))
    if cap < 0 or cap > t.numel():
        raise SzError(SZ_ERR_ARG, f"{what}: capacity {cap} outside 0..{t.numel()}")
    return int(cap)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(int(torch.cuda.current_stream().cuda_stream))


def _params(chunk: int = 0, sub: int = 0, segment: int = 0, ignored_digits: int = 0, predictor: int = 0,
            key_fields: int = 0):
    return sz_params(chunk, sub, segment, ignored_digits, predictor, key_fields)


class Context:
    """Owns an sz_ctx* and the host size holders of pending calls."""

    def __init__(self, device: int = 0, budget: int = 0):
        h = C.c_void_p()
        _check(_lib.sz_ctx_create(C.byref(h), device, budget), "sz_ctx_create")
        self.handle = h
        self.device = device
        self._keep = []

    def close(self):
        if self.handle:
            _lib.sz_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hold(self, obj):
        self._keep.append(obj)
        return obj


def sz_ctx_create(device: int = 0, budget: int = 0) -> Context:
    return Context(device, budget)


def sz_ctx_destroy(ctx: Context):
    ctx.close()


def sz_max_compressed_bytes(n: int) -> int:
    return int(_lib.sz_max_compressed_bytes(n))


def sz_compress(ctx: Context, x, eb: float, kind: int = SZ_EB_REL, params=None, out=None, out_cap=None,
                stream=None):
    """Enqueue compression of the float32 CUDA tensor x into `out` (uint8 CUDA
    tensor; allocated with the maximum size when None).  Returns
    (out, size_holder); size_holder.value is valid after sz_sync."""
    import torch
    _arg(x, _F32, "cuda", "sz_compress x")
    n = x.numel()
    if out is None:
        out = torch.empty(sz_max_compressed_bytes(n), dtype=torch.uint8, device=x.device)
    _arg(out, _U8, "cuda", "sz_compress out")
    cap = _cap(out, out_cap, "sz_compress out")
    nb = ctx.hold(C.c_size_t(0))
    p = params if params is not None else _params()
    _check(_lib.sz_compress(ctx.handle, _ptr(x), n, eb, kind, C.byref(p), _ptr(out), cap, C.byref(nb),
                            _stream(stream)), "sz_compress")
    return out, nb


def sz_decompress(ctx: Context, stream_buf, in_bytes: int, out, n_cap=None, stream=None):
    """Enqueue decompression of a stream (uint8 CUDA tensor) into the float32
    CUDA tensor `out`.  Returns a holder whose .value is n after sz_sync."""
    _arg(stream_buf, _U8, "cuda", "sz_decompress stream", in_bytes)
    _arg(out, _F32, "cuda", "sz_decompress out")
    cap = _cap(out, n_cap, "sz_decompress out")
    no = ctx.hold(C.c_size_t(0))
    _check(_lib.sz_decompress(ctx.handle, _ptr(stream_buf), in_bytes, _ptr(out), cap, C.byref(no),
                              _stream(stream)), "sz_decompress")
    return no


def sz_compress_batch(ctx: Context, xs, ebs, kind: int = SZ_EB_REL, params=None, outs=None, stream=None):
    import torch
    k = len(xs)
    for i in range(k):
        _arg(xs[i], _F32, "cuda", f"sz_compress_batch xs[{i}]")
    if outs is None:
        outs = [torch.empty(sz_max_compressed_bytes(x.numel()), dtype=torch.uint8, device=x.device) for x in xs]
    for i in range(k):
        _arg(outs[i], _U8, "cuda", f"sz_compress_batch outs[{i}]")
    ins = (C.c_void_p * k)(*[_ptr(x) for x in xs])
    ns = (C.c_size_t * k)(*[x.numel() for x in xs])
    e = (C.c_double * k)(*ebs)
    o = (C.c_void_p * k)(*[_ptr(t) for t in outs])
    caps = (C.c_size_t * k)(*[t.numel() for t in outs])
    nb = ctx.hold((C.c_size_t * k)())
    p = params if params is not None else _params()
    _check(_lib.sz_compress_batch(ctx.handle, k, ins, ns, e, kind, C.byref(p), o, caps, nb, _stream(stream)),
           "sz_compress_batch")
    return outs, nb


def sz_decompress_batch(ctx: Context, streams, in_bytes, outs, stream=None):
    k = len(streams)
    for i in range(k):
        _arg(streams[i], _U8, "cuda", f"sz_decompress_batch streams[{i}]", in_bytes[i])
        _arg(outs[i], _F32, "cuda", f"sz_decompress_batch outs[{i}]")
    ins = (C.c_void_p * k)(*[_ptr(s) for s in streams])
    ib = (C.c_size_t * k)(*in_bytes)
    o = (C.c_void_p * k)(*[_ptr(t) for t in outs])
    caps = (C.c_size_t * k)(*[t.numel() for t in outs])
    no = ctx.hold((C.c_size_t * k)())
    _check(_lib.sz_decompress_batch(ctx.handle, k, ins, ib, o, caps, no, _stream(stream)), "sz_decompress_batch")
    return no


def sz_compress_host(ctx: Context, xs, ebs, kind: int = SZ_EB_REL, params=None, outs=None, stream=None,
                     check: bool = True):
    """Host tensors in, host streams out (synchronous).  Returns (status,
    outs, sizes); raises on failure when `check`."""
    import torch
    k = len(xs)
    for i in range(k):
        _arg(xs[i], _F32, "cpu", f"sz_compress_host xs[{i}]")
    if outs is None:
        outs = [torch.empty(sz_max_compressed_bytes(x.numel()), dtype=torch.uint8).pin_memory() for x in xs]
    for i in range(k):
        _arg(outs[i], _U8, "cpu", f"sz_compress_host outs[{i}]")
    ins = (C.c_void_p * k)(*[_ptr(x) for x in xs])
    ns = (C.c_size_t * k)(*[x.numel() for x in xs])
    e = (C.c_double * k)(*ebs)
    o = (C.c_void_p * k)(*[_ptr(t) for t in outs])
    caps = (C.c_size_t * k)(*[t.numel() for t in outs])
    nb = (C.c_size_t * k)()
    p = params if params is not None else _params()
    st = _lib.sz_compress_host(ctx.handle, k, ins, ns, e, kind, C.byref(p), o, caps, nb, _stream(stream))
    if check:
        _check(st, "sz_compress_host")
    return st, outs, [int(v) for v in nb]


def sz_decompress_host(ctx: Context, streams, in_bytes, outs, stream=None, check: bool = True):
    """Host streams in, host float32 tensors out (synchronous).  Returns
    (status, element counts); raises on failure when `check`."""
    k = len(streams)
    for i in range(k):
        _arg(streams[i], _U8, "cpu", f"sz_decompress_host streams[{i}]", in_bytes[i])
        _arg(outs[i], _F32, "cpu", f"sz_decompress_host outs[{i}]")
    ins = (C.c_void_p * k)(*[_ptr(s) for s in streams])
    ib = (C.c_size_t * k)(*in_bytes)
    o = (C.c_void_p * k)(*[_ptr(t) for t in outs])
    caps = (C.c_size_t * k)(*[t.numel() for t in outs])
    no = (C.c_size_t * k)()
    st = _lib.sz_decompress_host(ctx.handle, k, ins, ib, o, caps, no, _stream(stream))
    if check:
        _check(st, "sz_decompress_host")
    return st, [int(v) for v in no]


def sz_compress_snapshot(ctx: Context, fields, xs, n: int, ebs, kind: int = SZ_EB_REL, mode: int = SZ_MODE_LV_PRX,
                         params=None, outs=None, perm=None, stream=None):
    import torch
    k = len(xs)
    for i in range(k):
        _arg(xs[i], _F32, "cuda", f"sz_compress_snapshot xs[{i}]", n)
    if outs is None:
        outs = [torch.empty(sz_max_compressed_bytes(n), dtype=torch.uint8, device=xs[0].device) for _ in xs]
        if mode == SZ_MODE_CPC2000:
            outs[0] = torch.empty(sz_cpc_max_bytes(n), dtype=torch.uint8, device=xs[0].device)
    for i in range(k):
        _arg(outs[i], _U8, "cuda", f"sz_compress_snapshot outs[{i}]")
    if perm is not None:
        _arg(perm, _I32, "cuda", "sz_compress_snapshot perm", n)
    f = (C.c_int * k)(*fields)
    ins = (C.c_void_p * k)(*[_ptr(x) for x in xs])
    e = (C.c_double * k)(*ebs)
    o = (C.c_void_p * k)(*[_ptr(t) for t in outs])
    caps = (C.c_size_t * k)(*[t.numel() for t in outs])
    nb = ctx.hold((C.c_size_t * k)())
    p = params if params is not None else _params()
    _check(_lib.sz_compress_snapshot(ctx.handle, k, f, ins, n, e, kind, mode, C.byref(p), o, caps, nb,
                                     _ptr(perm), _stream(stream)), "sz_compress_snapshot")
    return outs, nb


def sz_cpc_max_bytes(n: int) -> int:
    return int(_lib.sz_cpc_max_bytes(n))


def sz_decompress_cpc(ctx: Context, stream_buf, in_bytes: int, outs, n_cap=None, stream=None):
    """Enqueue decoding of an SZ-CPC2000 coordinate stream into three float32
    CUDA tensors (x, y, z).  Returns a holder whose .value is n after sz_sync."""
    _arg(stream_buf, _U8, "cuda", "sz_decompress_cpc stream", in_bytes)
    if len(outs) != 3:
        raise SzError(SZ_ERR_ARG, "sz_decompress_cpc: three output arrays (x, y, z)")
    for i, t in enumerate(outs):
        _arg(t, _F32, "cuda", f"sz_decompress_cpc outs[{i}]", 0 if n_cap is None else n_cap)
    no = ctx.hold(C.c_size_t(0))
    o = ctx.hold((C.c_void_p * 3)(*[_ptr(t) for t in outs]))
    cap = min(t.numel() for t in outs) if n_cap is None else n_cap
    _check(_lib.sz_decompress_cpc(ctx.handle, _ptr(stream_buf), in_bytes, o, cap, C.byref(no), _stream(stream)),
           "sz_decompress_cpc")
    return no


def sz_sync(ctx: Context, stream=None, check: bool = True) -> int:
    st = _lib.sz_sync(ctx.handle, _stream(stream))
    ctx._keep.clear()
    if check:
        _check(st, "sz_sync")
    return st


def sz_status_string(status: int) -> str:
    return _lib.sz_status_string(status).decode()


def sz_compress_noalloc(x, eb: float, kind: int = SZ_EB_REL, out=None, out_cap=None, stream=None):
    """Compression that allocates nothing in the library (fixed device scratch;
    n <= 2^26).  Synchronous; returns (status, out, out_bytes).  `out` is
    allocated here by torch when None -- pass it to allocate nothing at all."""
    import torch
    _arg(x, _F32, "cuda", "sz_compress_noalloc x")
    n = x.numel()
    if out is None:
        out = torch.empty(sz_max_compressed_bytes(n), dtype=torch.uint8, device=x.device)
    _arg(out, _U8, "cuda", "sz_compress_noalloc out")
    cap = _cap(out, out_cap, "sz_compress_noalloc out")
    nb = C.c_size_t(0)
    st = _lib.sz_compress_noalloc(_ptr(x), n, eb, kind, _ptr(out), cap, C.byref(nb), _stream(stream))
    return st, out, nb.value


def sz_ctx_set_autotune(ctx: Context, on: bool = True):
    _check(_lib.sz_ctx_set_autotune(ctx.handle, 1 if on else 0), "sz_ctx_set_autotune")


def sz_batch_tuning(ctx: Context, n: int) -> dict:
    """The batched form's autotuner choice for arrays of n elements."""
    t = sz_tuning()
    _check(_lib.sz_batch_tuning(ctx.handle, int(n), C.byref(t)), "sz_batch_tuning")
    return {"chunk_elems": t.chunk_elems, "fixed_chunk_elems": t.fixed_chunk_elems,
            "class": (t.class_lo, t.class_hi), "trial_ms": {2048 << j: t.trial_ms[j] for j in range(4)},
            "range_tile": t.range_tile, "quant_group": t.quant_group,
            "tile_trial_ms": list(t.tile_trial_ms)}


def sz_check_wait_timeout(ctx: Context, spins: int, stream=None):
    """Enqueue one warp whose look-back wait runs out after `spins` polls; the
    next sz_sync() reports SZ_ERR_TIMEOUT."""
    _check(_lib.sz_check_wait_timeout(ctx.handle, int(spins), _stream(stream)), "sz_check_wait_timeout")


def sz_profile_enable(ctx: Context, on: bool = True):
    _check(_lib.sz_profile_enable(ctx.handle, 1 if on else 0), "sz_profile_enable")


def sz_profile_read(ctx: Context) -> dict:
    """{phase: (launches, milliseconds)} since tracing was enabled or last read."""
    k = len(PHASES)
    n = (C.c_uint64 * k)()
    ms = (C.c_double * k)()
    _check(_lib.sz_profile_read(ctx.handle, n, ms, k), "sz_profile_read")
    return {PHASES[i]: (int(n[i]), float(ms[i])) for i in range(k)}


def sz_serve_start(ctx: Context, slots: int):
    _check(_lib.sz_serve_start(ctx.handle, slots), "sz_serve_start")


def sz_serve_submit(ctx: Context, req: sz_request) -> int:
    t = C.c_uint64(0)
    _check(_lib.sz_serve_submit(ctx.handle, C.byref(req), C.byref(t)), "sz_serve_submit")
    return t.value


def sz_serve_poll(ctx: Context, ticket: int) -> sz_result:
    r = sz_result()
    _check(_lib.sz_serve_poll(ctx.handle, ticket, C.byref(r)), "sz_serve_poll")
    return r


def sz_serve_wait(ctx: Context, ticket: int, timeout_s: float = 60.0) -> sz_result:
    r = sz_result()
    _check(_lib.sz_serve_wait(ctx.handle, ticket, float(timeout_s), C.byref(r)), "sz_serve_wait")
    return r


def sz_serve_release(ctx: Context, out: int):
    _check(_lib.sz_serve_release(ctx.handle, C.c_void_p(out)), "sz_serve_release")


def sz_serve_stats(ctx: Context) -> dict:
    c = sz_serve_counters()
    _check(_lib.sz_serve_stats(ctx.handle, C.byref(c)), "sz_serve_stats")
    return {f: getattr(c, f) for f, _ in sz_serve_counters._fields_}


def request(op: int, inp, n: int, out=None, out_cap: int = 0, in_bytes: int = 0, eb: float = 0.0,
            kind: int = SZ_EB_REL) -> sz_request:
    """Build an sz_request from CUDA tensors or raw device addresses (out=None:
    the service allocates the output).  Tensors are checked like the other
    entry points' (raw addresses are the caller's responsibility): a compress
    request takes n float32 values in and writes uint8 stream bytes, within
    out_cap; a decompress request reads in_bytes stream bytes and writes up to
    n float32 values."""
    comp = op == SZ_OP_COMPRESS
    if not isinstance(inp, int) and inp is not None:
        if comp:
            _arg(inp, _F32, "cuda", "request input", n)
        else:
            _arg(inp, _U8, "cuda", "request stream", in_bytes)
    if not isinstance(out, int) and out is not None:
        if comp:
            _arg(out, _U8, "cuda", "request output")
            _cap(out, out_cap, "request output")
        else:
            _arg(out, _F32, "cuda", "request output", n)

    def addr(t):
        return None if t is None else (t if isinstance(t, int) else t.data_ptr())
    return sz_request(op, addr(inp), n, in_bytes, addr(out), out_cap, eb, kind)


class _DevBuf:
    """Exposes a raw device range through __cuda_array_interface__ (for torch.as_tensor)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def device_bytes(ptr: int, nbytes: int):
    """A uint8 CUDA tensor viewing nbytes at device address ptr (no copy)."""
    import torch
    return torch.as_tensor(_DevBuf(ptr, nbytes), device="cuda")


def sz_serve_stop(ctx: Context):
    _check(_lib.sz_serve_stop(ctx.handle), "sz_serve_stop")


# ---- convenience (still only marshalling) ----------------------------------

def compress(ctx: Context, x, eb: float, kind: int = SZ_EB_REL, chunk: int = 0):
    """Compress and synchronize; returns the stream as a uint8 CUDA tensor."""
    out, nb = sz_compress(ctx, x, eb, kind, _params(chunk))
    sz_sync(ctx)
    return out[: nb.value]


def decompress(ctx: Context, stream_buf, n: int):
    import torch
    out = torch.empty(max(n, 1), dtype=torch.float32, device=stream_buf.device)
    no = sz_decompress(ctx, stream_buf, stream_buf.numel(), out, n)
    sz_sync(ctx)
    return out[: no.value]
