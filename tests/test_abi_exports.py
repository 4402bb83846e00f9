"""CPU checks of the boundary: the shared library builds for sm_103a, loads,
and exports every function include/sz_gb300.h declares (no GPU calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sz_gb300.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:sz_status|size_t|const char\*)\s+(sz_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__ as g
    g._load_build_module().build()
    return os.path.join(ROOT, "paper_1711_03888_gb300", "libsz_gb300.so")


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("sz_compress", "sz_decompress", "sz_compress_batch", "sz_decompress_batch",
                 "sz_compress_snapshot", "sz_sync", "sz_ctx_create", "sz_ctx_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (sz_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_names_match_header(lib_path):
    import paper_1711_03888_gb300 as sz
    assert set(sz.EXPORTS) == set(_declared())
    for name in _declared():
        assert callable(getattr(sz, name))


def test_host_only_calls(lib_path):
    import paper_1711_03888_gb300 as sz
    assert sz.sz_max_compressed_bytes(0) == 160
    assert sz.sz_max_compressed_bytes(5) == 160 + 32
    assert sz.sz_status_string(sz.SZ_ERR_CORRUPT) == "corrupt stream"


def test_built_for_sm103a_only():
    import __graft_entry__ as g
    b = g._load_build_module()
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "--use_fast_math" not in b.FLAGS and "-ftz=true" not in b.FLAGS
