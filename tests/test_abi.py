"""The C ABI boundary on the CPU: the library loads, exports every declared
entry point, and rejects malformed input before touching a GPU."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "smx.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(smx_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_14741_gb300 import _lib

    if not os.path.exists(_lib.LIB_PATH):
        import paper_2205_14741_gb300.build as b

        b.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["smx_create", "smx_set_values", "smx_set_filter_threshold", "smx_set_mu",
                     "smx_set_electron_count", "smx_set_precision", "smx_build_density", "smx_solve_mu",
                     "smx_get_trace", "smx_get_density", "smx_get_pattern", "smx_get_stats", "smx_destroy",
                     "smx_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2205_14741_gb300 import _lib

    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_status_strings(lib):
    for s in range(11):
        assert lib.smx_status_string(s)
    assert lib.smx_status_string(0) == b"ok"
    assert lib.smx_status_string(2) == b"malformed block pattern"


def _create(lib, bs, cp, ri, vals):
    ctx = C.c_void_p()
    arrs = [np.ascontiguousarray(bs, np.int32), np.ascontiguousarray(cp, np.int64),
            np.ascontiguousarray(ri, np.int32), np.ascontiguousarray(vals, np.float64)]
    st = lib.smx_create(C.byref(ctx), len(arrs[0]), *[a.ctypes.data_as(C.c_void_p) for a in arrs], None)
    return st, ctx


def test_malformed_patterns_rejected_on_host(lib):
    from paper_2205_14741_gb300 import _lib

    vals = np.zeros(100)
    # missing diagonal block in column 1
    assert _create(lib, [1, 1], [0, 2, 3], [0, 1, 0], vals)[0] == _lib.ERR_PATTERN
    # unsorted rows
    assert _create(lib, [1, 1], [0, 2, 4], [1, 0, 0, 1], vals)[0] == _lib.ERR_PATTERN
    # asymmetric pattern: (1,0) present, (0,1) absent
    assert _create(lib, [1, 1], [0, 2, 3], [0, 1, 1], vals)[0] == _lib.ERR_PATTERN
    # row index out of range
    assert _create(lib, [1, 1], [0, 1, 3], [0, 1, 2], vals)[0] == _lib.ERR_PATTERN
    # block size out of range, non-positive count
    assert _create(lib, [0, 1], [0, 1, 2], [0, 1], vals)[0] == _lib.ERR_ARG
    assert _create(lib, [65], [0, 1], [0], vals)[0] == _lib.ERR_ARG
    ctx = C.c_void_p()
    assert lib.smx_create(C.byref(ctx), 0, None, None, None, None, None) == _lib.ERR_ARG
    assert lib.smx_create(None, 1, None, None, None, None, None) == _lib.ERR_ARG


def test_null_context_is_rejected(lib):
    from paper_2205_14741_gb300 import _lib

    assert lib.smx_build_density(None) == _lib.ERR_ARG
    assert lib.smx_set_mu(None, 0.0) == _lib.ERR_ARG
    assert lib.smx_get_trace(None, None, None, None) == _lib.ERR_ARG
    lib.smx_destroy(None)
