"""Failure detection, exercised without faulting the GPU.

* The bounded device waits: a self-test kernel waits on an mbarrier that
  nothing arrives at (no copies or tensor-core work in flight) and gives up
  after a short poll limit; the context reports SMX_ERR_TIMEOUT, keeps it
  latched until the next build, and then builds the correct density matrix.
* The learned bound's safe check: parameters that predict a far too small
  spectral radius (or an impossible gap) must all fail the check, fall back to
  the guaranteed start, and still give the oracle's D (Section 4's learning on
  the fly may only cost speed, never correctness).
* The scaled schedule with a wrong gap: any lower bound in (0, 1] converges
  (tiny gaps cost steps), so D still matches the oracle.
* Guard bands: results written to caller-owned device memory touch nothing
  outside the requested range.
"""

import ctypes as C

import numpy as np
import pytest

import oracle as O
from synth import make_workload
from tests.helpers import oracle_in_input_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_D = {"fp64": 1e-10, "fp16x3": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _params(rho_over_g, delta_over_g):
    """Bound-model parameters whose outputs are the given constants (output layer bias only)."""
    from paper_2205_14741_gb300 import BOUND_MODEL_PARAMS

    p = np.zeros(BOUND_MODEL_PARAMS, dtype=np.float32)
    p[-2:] = [rho_over_g, delta_over_g]
    return p


def _built(sysm, prec, mu, params=None, mode=True):
    from paper_2205_14741_gb300 import SubmatrixDensity

    c = SubmatrixDensity.from_system(sysm)
    c.set_precision(prec)
    c.set_mu(mu)
    if params is not None:
        c.bound_model_init(0)
        c.bound_model_set_params(params)
        c.set_bound_model(mode)
    c.build_density()
    return c


def test_bounded_wait_times_out_and_the_context_recovers():
    from paper_2205_14741_gb300 import SmxError, _lib

    s = make_workload("water32")
    d_or, res, _ = oracle_in_input_layout(s, 0.0, 0.0)
    with _built(s, "fp16x3", 0.0) as c:
        assert c.selftest_wait_timeout(1 << 16) == _lib.ERR_TIMEOUT
        with pytest.raises(SmxError) as e:
            c.get_trace()  # latched until the next build
        assert e.value.status == _lib.ERR_TIMEOUT
        assert c.selftest_wait_timeout(1) == _lib.ERR_TIMEOUT
        c.build_density()
        d = c.get_density()
        tr, _, _ = c.get_trace()
    assert float(np.max(np.abs(d - d_or))) <= TOL_D["fp16x3"]
    assert abs(tr - res.trace) <= 1e-6 * abs(res.trace)


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
@pytest.mark.parametrize("mode", ["rho", "gap"])
def test_forced_bad_learned_bound_falls_back(prec, mode):
    # rho_hat / G = -5 is clamped to 0.02: X0 = A / b is far too large, the guaranteed bound s
    # fails every check; the gap output is negative (no scaled schedule)
    s = make_workload("water32")
    d_or, _, _ = oracle_in_input_layout(s, 0.0, 0.0)
    with _built(s, prec, 0.0, _params(-5.0, -5.0), mode) as c:
        d = c.get_density()
        st = c.get_stats()
    assert st["n_bound_fallback"] == s.n_blocks
    assert float(np.max(np.abs(d - d_or))) <= TOL_D[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_impossible_gap_fails_the_check(prec):
    # a predicted gap above the guaranteed spectral bound cannot be right: every column falls back
    s = make_workload("water32")
    d_or, _, _ = oracle_in_input_layout(s, 0.0, 0.0)
    with _built(s, prec, 0.0, _params(0.33, 5.0), "gap") as c:
        d = c.get_density()
        st = c.get_stats()
    assert st["n_bound_fallback"] == s.n_blocks
    assert float(np.max(np.abs(d - d_or))) <= TOL_D[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
@pytest.mark.parametrize("delta", [1e-4, 0.02, 0.3])
def test_scaled_schedule_converges_for_any_gap_guess(prec, delta):
    # the true delta/G of these submatrices is about 0.16: a thousandfold underestimate costs
    # steps, an overestimate (still below s) costs little; D is the oracle's in every case
    s = make_workload("water32")
    d_or, _, _ = oracle_in_input_layout(s, 0.0, 0.0)
    with _built(s, prec, 0.0, _params(0.33, delta), "gap") as c:
        d = c.get_density()
        st = c.get_stats()
    assert st["n_noconv"] == 0 and st["n_bound_fallback"] == 0
    assert float(np.max(np.abs(d - d_or))) <= TOL_D[prec]
    assert st["iters_max"] <= 30


def test_device_outputs_respect_guard_bands():
    from paper_2205_14741_gb300 import _lib

    s = make_workload("water32")
    guard = 4096
    canary = 12345.678
    with _built(s, "fp16x3", 0.0) as c:
        d_host = c.get_density()
        buf = torch.full((s.values.shape[0] + 2 * guard,), canary, dtype=torch.float64, device="cuda")
        c.get_density(buf[guard:guard + s.values.shape[0]])
        torch.cuda.synchronize()
    out = buf.cpu().numpy()
    assert np.all(out[:guard] == canary) and np.all(out[-guard:] == canary)
    assert np.array_equal(out[guard:-guard], d_host)
    # the allocation-free dense entry point on a caller buffer with guard bands
    h = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    n = h.shape[0]
    h_dev = torch.from_numpy(h).cuda()
    dbuf = torch.full((n * n + 2 * guard,), canary, dtype=torch.float64, device="cuda")
    lib = _lib.load()
    st = lib.smx_dense_density_noalloc(C.c_void_p(h_dev.data_ptr()), n, 0.0,
                                       C.c_void_p(dbuf[guard:].data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.OK
    out = dbuf.cpu().numpy()
    assert np.all(out[:guard] == canary) and np.all(out[guard + n * n:] == canary)
    assert float(np.max(np.abs(out[guard:guard + n * n].reshape(n, n) - O.dense_density(h, 0.0)))) <= 1e-10
