"""GPU parity of the function forms (FP64): per-submatrix A^-1/2, A^1/2 and A^-1 of an overlap-like
symmetric positive definite matrix against oracle/functions.py (eigendecomposition), and the
error paths.  Tolerance: the FP64 form's 1e-10 max-abs, as for the density matrix."""

import numpy as np
import pytest

import oracle as O
from synth import make_overlap_system, make_workload
from tests.helpers import max_abs_on_columns, sample_columns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ctx(sysm, f, prec="fp64"):
    from paper_2205_14741_gb300 import SubmatrixDensity

    c = SubmatrixDensity.from_system(sysm)
    c.set_precision(prec)
    c.set_function(f)
    c.set_mu(0.0)
    return c


@pytest.mark.parametrize("f", ["inv_sqrt", "sqrt", "inv"])
def test_functions_match_oracle(f):
    s = make_overlap_system(64, 6, 5.0, 1.5, 31)
    with _ctx(s, f) as c:
        c.build_density()
        got = c.get_density()
        tr, en, _ = c.get_trace()
        st = c.get_stats()
    res = O.function_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, f)
    assert np.max(np.abs(got - res.values)) <= 1e-10
    assert abs(tr - res.trace) <= 1e-10 * abs(res.trace)
    assert abs(en - res.energy) <= 1e-10 * abs(res.energy)
    assert st["n_noconv"] == 0 and st["iters_max"] < 20


def test_inv_sqrt_1024_molecules_sampled_columns():
    s = make_overlap_system(1024, 6, 6.0, 1.5, 41)
    with _ctx(s, "inv_sqrt") as c:
        c.build_density()
        got = c.get_density()
        dims, iters, _ = c.get_submatrix_info()
    cols = sample_columns(dims, 16)
    res = O.function_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, "inv_sqrt", columns=cols)
    assert max_abs_on_columns(got, res.values, s, cols) <= 1e-10
    assert dims.min() >= 96 and iters.max() < 20


def test_function_errors_and_switching_back():
    from paper_2205_14741_gb300 import SmxError, _lib

    s = make_overlap_system(32, 6, 5.0, 1.5, 7)
    with _ctx(s, "inv_sqrt", prec="fp16x3") as c:
        with pytest.raises(SmxError) as ei:
            c.build_density()  # the function forms run in FP64
        assert ei.value.status == _lib.ERR_UNSUPPORTED
        c.set_precision("fp64")
        c.set_electron_count(48.0, 30, 0.5)
        with pytest.raises(SmxError) as ei:
            c.solve_mu()  # bisection needs the density matrix
        assert ei.value.status == _lib.ERR_STATE
        c.build_density()
        c.set_function("density")
        c.build_density()
        d = c.get_density()
    with _ctx(s, "density") as f:
        f.build_density()
        assert np.array_equal(f.get_density(), d)
    # a submatrix that is not positive definite (the Hamiltonian stand-in at mu = 0)
    h = make_workload("water32")
    with _ctx(h, "inv_sqrt") as c:
        with pytest.raises(SmxError) as ei:
            c.build_density()
            c.get_trace()
        assert ei.value.status in (_lib.ERR_NOCONV, _lib.ERR_NONFINITE)
