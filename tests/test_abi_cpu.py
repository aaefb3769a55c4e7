"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry
point that include/cbc.h declares; argument errors are reported without any GPU work."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2601_19650_gb300 import _cbc, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cbc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ttn_create", "ttno_create", "cbc_apply", "ttn_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_rejects_bad_arguments(libpath):
    L = _cbc.lib()
    out = ctypes.c_void_p()
    # n_nodes = 0: rejected before any device work
    rc = L.ttn_create(0, None, None, None, 0, None, 0, None, ctypes.byref(out))
    assert rc == 1 and out.value is None
    assert "n_nodes" in _cbc.cbc_last_error()
    rc = L.cbc_apply(None, None, 8, 0.0, None, ctypes.byref(out))
    assert rc == 1
    # two roots
    n = 2
    par = (ctypes.c_int32 * n)(-1, -1)
    dims = (ctypes.c_int64 * n)(2, 2)
    ptrs = (ctypes.c_void_p * n)(1, 1)
    rc = L.ttn_create(n, par, dims, dims, 1, ptrs, 1, None, ctypes.byref(out))
    assert rc == 1 and "roots" in _cbc.cbc_last_error()
    # a cycle
    par = (ctypes.c_int32 * 3)(-1, 2, 1)
    d3 = (ctypes.c_int64 * 3)(2, 2, 2)
    p3 = (ctypes.c_void_p * 3)(1, 1, 1)
    rc = L.ttn_create(3, par, d3, d3, 1, p3, 1, None, ctypes.byref(out))
    assert rc == 1 and "cycle" in _cbc.cbc_last_error()
    # bad dtype
    par = (ctypes.c_int32 * 1)(-1)
    d1 = (ctypes.c_int64 * 1)(2)
    p1 = (ctypes.c_void_p * 1)(1)
    rc = L.ttn_create(1, par, d1, d1, 9, p1, 1, None, ctypes.byref(out))
    assert rc == 1 and "dtype" in _cbc.cbc_last_error()
    assert L.ttn_destroy(None) == 0 and L.ttno_destroy(None) == 0
    # fetching from a NULL handle, into a NULL buffer
    buf = (ctypes.c_double * 4)()
    assert L.ttn_get_network(None, buf, 0, 1) == 1
    assert "NULL" in _cbc.cbc_last_error()
    assert L.ttn_get_node(None, 0, buf, 0, 1) == 1
    # an empty batch is a no-op; a batch with NULL arrays is rejected
    assert L.cbc_apply_batched(0, None, None, None, None, None, 0, None) == 0
    assert L.cbc_apply_batched(2, None, None, None, None, None, 0, None) == 1
    # the comparison methods check their handles before any device work
    assert L.zipup_apply(None, None, 4, 0.0, None, ctypes.byref(out)) == 1
    assert "zipup_apply" in _cbc.cbc_last_error() and out.value is None
    assert L.direct_apply(None, None, 4, 0.0, None, ctypes.byref(out)) == 1
    assert "direct_apply" in _cbc.cbc_last_error() and out.value is None
    assert L.src_apply(None, None, 4, None, 1, 0, None, ctypes.byref(out)) == 1
    assert "src_apply" in _cbc.cbc_last_error() and out.value is None


def test_build_targets_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
