"""FP64 finishing steps after a low-precision bulk phase (the bulk's last iterate, then plain
FP64 Newton-Schulz steps on the CUDA cores, then the scatter): parity against the oracle in every
bulk precision, the step count and the flop counter, and the plain FP64 form unaffected."""

import numpy as np
import pytest

from synth import make_workload
from tests.helpers import oracle_in_input_layout

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the bulk precision sets the error (the finishing steps do not repair a single-pass bulk's
# rotated subspace); the split form keeps the 1e-5 bound on D of the mixed forms
BOUND = {"fp16x3": 1e-5, "fp16": 2e-2, "bf16": 1e-1}


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("bulk", ["fp16x3", "fp16", "bf16"])
@pytest.mark.parametrize("final", [1, 2])
def test_fp64_finish_parity(bulk, final):
    from paper_2205_14741_gb300 import SubmatrixDensity

    s = make_workload("water32")
    d_or, res, _ = oracle_in_input_layout(s, 0.0, 0.0)
    with SubmatrixDensity.from_system(s) as c:
        c.set_precision(bulk)
        c.set_mu(0.0)
        c.build_density()
        it0 = c.get_submatrix_info()[1].copy()
        c.set_precision(bulk, final)
        c.reset_counters()
        c.build_density()
        d = c.get_density()
        tr, en, _ = c.get_trace()
        st = c.get_stats()
        dims, it1, _ = c.get_submatrix_info()
    assert st["fp64_final_iters"] == final
    assert np.array_equal(it1, it0 + final)
    assert st["ns_work_n3"] == float(np.sum(dims.astype(np.float64) ** 3 * it1))
    assert float(np.max(np.abs(d - d_or))) <= BOUND[bulk]
    if bulk == "fp16x3":
        assert abs(en - res.energy) <= 1e-6 * abs(res.energy)
        assert abs(tr - res.trace) <= 1e-6 * abs(res.trace)


def test_fp64_finish_on_the_streamed_form():
    # a single 224 x 224 submatrix (kpad > 192): the final iterate comes from the workspace
    from paper_2205_14741_gb300 import SubmatrixDensity
    from synth import make_mixed_block_system

    s = make_mixed_block_system([32] * 7, r_c=np.inf, ell=1.5, seed=7)
    d_or, _, _ = oracle_in_input_layout(s, 0.0, 0.0)
    with SubmatrixDensity.from_system(s) as c:
        c.set_precision("fp16x3", 1)
        c.set_mu(0.0)
        c.build_density()
        d = c.get_density()
        assert c.get_stats()["dim_min"] == 224
    assert float(np.max(np.abs(d - d_or))) <= BOUND["fp16x3"]


def test_plain_fp64_ignores_final_iters():
    from paper_2205_14741_gb300 import SubmatrixDensity

    s = make_workload("water32")
    out = []
    for final in [0, 3]:
        with SubmatrixDensity.from_system(s) as c:
            c.set_precision("fp64", final)
            c.set_mu(0.0)
            c.build_density()
            out.append((c.get_density().copy(), c.get_stats()["fp64_final_iters"]))
    assert np.array_equal(out[0][0], out[1][0]) and out[1][1] == 0
