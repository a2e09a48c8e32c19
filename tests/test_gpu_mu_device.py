"""The bisection for Eq. 14's mu with its decisions on the device (smx_solve_mu_device): the
same mu, D, trace and step count as the host loop of smx_solve_mu, bit for bit, with new values
(filter first), on an analysed context, when the stopping rule ends early, and when every step
runs."""

import numpy as np
import pytest

from synth import make_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _solve(sysm, prec, n_e, max_steps, tol, device, eps=1e-5, repeat_values=False, symmetrize=False):
    from paper_2205_14741_gb300 import SubmatrixDensity

    with SubmatrixDensity.from_system(sysm) as c:
        c.set_precision(prec)
        c.set_filter_threshold(eps)
        if symmetrize:
            c.set_symmetrize(True)
        c.set_electron_count(n_e, max_steps=max_steps, tol=tol)
        if repeat_values:  # an analysed context given new values (the filter runs first)
            c.set_mu(0.0)
            c.build_density()
            c.set_values(sysm.values)
        (c.solve_mu_device if device else c.solve_mu)()
        tr, en, mu = c.get_trace()
        return c.get_density().copy(), tr, en, mu, c.get_stats()["bisection_steps"]


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
@pytest.mark.parametrize("case", ["early", "all_steps", "new_values"])
def test_device_bisection_matches_the_host_loop(prec, case):
    name = "water1024" if case == "early" else "water32"
    s = make_workload(name)
    n_e, steps, tol = {"early": (3072.0, 30, 1e-2), "all_steps": (90.5, 12, 0.0), "new_values": (96.0, 40, 1e-3)}[case]
    host = _solve(s, prec, n_e, steps, tol, False, repeat_values=case == "new_values")
    dev = _solve(s, prec, n_e, steps, tol, True, repeat_values=case == "new_values")
    assert dev[3] == host[3] and dev[4] == host[4]
    assert dev[1] == host[1] and dev[2] == host[2]
    assert np.array_equal(dev[0], host[0])
    if case == "all_steps":
        assert host[4] == steps


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_device_bisection_with_symmetrised_result(prec):
    # The symmetrisation runs after every build of the solve, and the skipped builds after
    # the stopping step skip it too: the device loop's D is the host loop's, bit for bit,
    # and it is exactly symmetric on the pattern.
    import oracle as O

    s = make_workload("water32")
    host = _solve(s, prec, 96.0, 40, 1e-3, False, symmetrize=True)
    dev = _solve(s, prec, 96.0, 40, 1e-3, True, symmetrize=True)
    assert dev[3] == host[3] and dev[4] == host[4] and dev[4] < 40
    assert np.array_equal(dev[0], host[0])
    dense = O.to_dense(s.block_size, s.col_ptr, s.row_idx, dev[0])
    assert np.array_equal(dense, dense.T)

