"""The allocation-free dense entry point, through the C ABI.

smx_dense_density_noalloc is for callers that cannot allocate device memory
when they need a density matrix (plug-ins whose host framework owns the
device pool, loops that must not enter the allocator).  Its result must match
the regular entry point, smx_build_density, on a system whose single
submatrix is the whole matrix, and the oracle's dense density matrix, call
after call: the shared fixed work array keeps the previous call's contents,
which must not leak into the next result.

This file is named so that pytest collects it after every other test file.
"""

import ctypes as C

import numpy as np
import pytest

import oracle as O
from synth import make_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10  # the FP64 parity tolerance of the other GPU tests


def test_no_alloc_matches_build_density_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_14741_gb300 import SubmatrixDensity, _lib

    lib = _lib.load()
    s = make_workload("water32_full")  # one 192 x 192 submatrix = the whole matrix
    n = s.n
    h = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)  # layout conversion only
    h_dev = torch.from_numpy(h).cuda()
    d_dev = torch.empty_like(h_dev)
    stream = torch.cuda.current_stream().cuda_stream

    for call, mu in enumerate([0.1, -0.2]):
        with SubmatrixDensity.from_system(s) as ctx:
            ctx.set_precision("fp64")
            ctx.set_mu(mu)
            ctx.build_density()
            d_ref = O.to_dense(s.block_size, s.col_ptr, s.row_idx, ctx.get_density())
        d_dev.fill_(float("nan"))
        st = lib.smx_dense_density_noalloc(C.c_void_p(h_dev.data_ptr()), n, mu, C.c_void_p(d_dev.data_ptr()),
                                           C.c_void_p(stream))
        assert st == _lib.OK, f"call {call}: status {st}"
        d = d_dev.cpu().numpy()
        err = float(np.max(np.abs(d - d_ref)))
        assert err <= TOL_FP64, f"call {call}: max|D_noalloc - D_build| = {err:.3e}"
        err_or = float(np.max(np.abs(d - O.dense_density(h, mu))))
        assert err_or <= TOL_FP64, f"call {call}: max|D_noalloc - D_oracle| = {err_or:.3e}"


def test_no_alloc_reports_nonfinite_input_then_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_14741_gb300 import _lib

    lib = _lib.load()
    s = make_workload("water32")
    h = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    bad = h.copy()
    bad[3, 5] = bad[5, 3] = np.nan
    d_dev = torch.empty(h.shape, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for hh, want in [(bad, _lib.ERR_NONFINITE), (h, _lib.OK)]:
        h_dev = torch.from_numpy(hh).cuda()
        st = lib.smx_dense_density_noalloc(C.c_void_p(h_dev.data_ptr()), s.n, 0.0, C.c_void_p(d_dev.data_ptr()),
                                           stream)
        assert st == want
    err = float(np.max(np.abs(d_dev.cpu().numpy() - O.dense_density(h, 0.0))))
    assert err <= TOL_FP64


def test_no_alloc_rejects_oversized_input():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_14741_gb300 import _lib

    lib = _lib.load()
    buf = torch.zeros(257 * 257, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    assert lib.smx_dense_density_noalloc(p, 257, 0.0, p, None) == _lib.ERR_ARG
    assert lib.smx_dense_density_noalloc(p, 0, 0.0, p, None) == _lib.ERR_ARG
    assert lib.smx_dense_density_noalloc(None, 8, 0.0, p, None) == _lib.ERR_ARG
