"""The binding's argument checks, on CPU: a tensor whose element type, layout,
memory or size does not fit the call is refused with SZ_ERR_ARG before any
address crosses the C ABI (which takes raw pointers and counts and cannot
check them)."""
import types

import pytest
import torch

import paper_1711_03888_gb300 as sz

# no call below reaches the library: the checks come first
CTX = types.SimpleNamespace(handle=None, hold=lambda o: o)


def _refused(fn, *a, **k):
    with pytest.raises(sz.SzError) as e:
        fn(*a, **k)
    assert e.value.status == sz.SZ_ERR_ARG
    return str(e.value)


def test_device_calls_refuse_host_tensors():
    x = torch.zeros(100, dtype=torch.float32)
    assert "expected cuda" in _refused(sz.sz_compress, CTX, x, 1e-4)
    assert "expected cuda" in _refused(sz.sz_compress_noalloc, x, 1e-4)
    assert "expected cuda" in _refused(sz.sz_compress_batch, CTX, [x], [1e-4])
    s = torch.zeros(400, dtype=torch.uint8)
    assert "expected cuda" in _refused(sz.sz_decompress, CTX, s, 400, x)
    assert "expected cuda" in _refused(sz.sz_decompress_batch, CTX, [s], [400], [x])
    assert "expected cuda" in _refused(sz.sz_decompress_cpc, CTX, s, 400, [x, x, x])
    assert "expected cuda" in _refused(sz.sz_compress_snapshot, CTX, [0], [x], 100, [1e-4],
                                       outs=[s])


def test_wrong_element_types_are_refused():
    assert "expected torch.float32" in _refused(sz.sz_compress, CTX, torch.zeros(8, dtype=torch.float64), 1e-4)
    assert "expected torch.float32" in _refused(sz.sz_compress_host, CTX, [torch.zeros(8, dtype=torch.float16)],
                                                [1e-4])
    assert "expected torch.uint8" in _refused(sz.sz_decompress_host, CTX, [torch.zeros(8, dtype=torch.int8)], [8],
                                              [torch.zeros(8)])
    assert "expected torch.float32" in _refused(sz.sz_decompress_host, CTX, [torch.zeros(8, dtype=torch.uint8)],
                                                [8], [torch.zeros(8, dtype=torch.int32)])


def test_strided_views_are_refused():
    x = torch.zeros(64, dtype=torch.float32)[::2]
    assert "not contiguous" in _refused(sz.sz_compress_host, CTX, [x], [1e-4])
    y = torch.zeros(4, 16, dtype=torch.float32).t()
    assert "not contiguous" in _refused(sz.sz_decompress_host, CTX, [torch.zeros(64, dtype=torch.uint8)], [64], [y])


def test_sizes_beyond_the_buffer_are_refused():
    s = torch.zeros(100, dtype=torch.uint8)
    y = torch.zeros(10, dtype=torch.float32)
    assert "101 needed" in _refused(sz.sz_decompress_host, CTX, [s], [101], [y])
    # a ctypes size holder counts like its value
    import ctypes
    assert "101 needed" in _refused(sz.sz_decompress_host, CTX, [s], [ctypes.c_size_t(101)], [y])


def test_explicit_capacity_may_not_pass_the_tensor():
    t = torch.zeros(50, dtype=torch.uint8)
    assert sz._cap(t, None, "out") == 50
    assert sz._cap(t, 20, "out") == 20
    assert sz._cap(t, 50, "out") == 50
    assert "outside 0..50" in _refused(sz._cap, t, 51, "out")
    assert "outside 0..50" in _refused(sz._cap, t, -1, "out")


def test_coordinate_decoder_takes_three_arrays():
    s = torch.zeros(8, dtype=torch.uint8)
    x = torch.zeros(8, dtype=torch.float32)
    # the memory check of the stream comes first on CPU; with two arrays the count is refused
    _refused(sz.sz_decompress_cpc, CTX, s, 8, [x, x])


class _DevT:
    """Stands in for a contiguous CUDA tensor (dtype, memory kind, size,
    address) so the acceptance side of the checks runs on CPU."""

    def __init__(self, dtype, numel):
        self.dtype, self._n = dtype, numel
        self.device = types.SimpleNamespace(type="cuda")

    def numel(self):
        return self._n

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return 1 << 20


def test_serving_requests_are_checked_like_the_calls():
    n = 5000
    x, st = _DevT(torch.float32, n), _DevT(torch.uint8, 1234)
    out_c, out_d = _DevT(torch.uint8, sz.sz_max_compressed_bytes(n)), _DevT(torch.float32, n)
    # the shapes the serving tests and the bench submit are accepted
    sz.request(sz.SZ_OP_COMPRESS, x, n, eb=1e-4)
    sz.request(sz.SZ_OP_COMPRESS, x, n, out=out_c, out_cap=out_c.numel(), eb=1e-4)
    sz.request(sz.SZ_OP_DECOMPRESS, st, n, in_bytes=st.numel())
    sz.request(sz.SZ_OP_DECOMPRESS, st, n, out=out_d, in_bytes=st.numel())
    r = sz.request(sz.SZ_OP_COMPRESS, 123456, n, out=654321, out_cap=10)     # raw addresses pass
    assert r.input == 123456 and r.out == 654321
    # and the ones that do not fit are refused
    _refused(sz.request, sz.SZ_OP_COMPRESS, torch.zeros(n), n)                # host memory
    _refused(sz.request, sz.SZ_OP_COMPRESS, _DevT(torch.uint8, n), n)         # a stream as input
    _refused(sz.request, sz.SZ_OP_COMPRESS, _DevT(torch.float32, n - 1), n)   # too short
    _refused(sz.request, sz.SZ_OP_COMPRESS, x, n, out=out_c, out_cap=out_c.numel() + 1)
    _refused(sz.request, sz.SZ_OP_DECOMPRESS, st, n, in_bytes=st.numel() + 1)
    _refused(sz.request, sz.SZ_OP_DECOMPRESS, st, n, out=_DevT(torch.float32, n - 1), in_bytes=10)
