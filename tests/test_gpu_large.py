"""GPU parity at the larger workloads and chunked staging.

* chunked staging (block columns processed in several passes over a bounded
  staging buffer) gives bitwise the same result as one pass;
* 4096 molecules x 23 orbitals (N = 94208, submatrices 920-1242) at its
  fixed mu, split FP16, on sampled columns against the oracle;
* the water/vacuum slab of 6000 molecules: the literal variant (cutoff 6 A,
  dimensions 6-252) solved for mu in both forms, and the wide variant
  (cutoff 15.3 A, dimensions 36-3024, ~300 GB of FP64 staging, so built in
  chunks) at mu = 0, on sampled columns.
"""

import numpy as np
import pytest

from synth import WORKLOADS, make_workload
from tests.helpers import max_abs_on_columns, oracle_in_input_layout, sample_columns

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_D = {"fp64": 1e-10, "fp16x3": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ctx(sysm, prec, eps):
    from paper_2205_14741_gb300 import SubmatrixDensity

    c = SubmatrixDensity.from_system(sysm)
    c.set_precision(prec)
    c.set_filter_threshold(eps)
    return c


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_chunked_staging_is_invisible(prec):
    s = make_workload("water1024")
    out = []
    for limit in [None, 16 << 20]:  # one pass / about a dozen chunks
        with _ctx(s, prec, 1e-5) as c:
            if limit:
                c.set_staging_limit(limit)
            c.set_mu(0.012)
            c.build_density()
            d = c.get_density().copy()
            tr = c.get_trace()
            c.bound_model_init(3)
            f, p, _ = c.bound_model_predict()
            out.append((d, tr, f, p))
    (d0, t0, f0, p0), (d1, t1, f1, p1) = out
    assert np.array_equal(d0, d1) and t0 == t1
    assert np.array_equal(f0, f1) and np.array_equal(p0, p1)


def test_water4096x23_sampled_columns():
    w = WORKLOADS["water4096x23"]
    s = make_workload("water4096x23")
    with _ctx(s, "fp16x3", w["eps"]) as c:
        c.set_mu(w["mu"])
        c.build_density()
        d = c.get_density()
        tr, en, _ = c.get_trace()
        st = c.get_stats()
        dims, iters, _ = c.get_submatrix_info()
    assert st["n_noconv"] == 0 and dims.min() >= 900 and dims.max() <= 1300
    # mu in the gap: the submatrix trace is close to, not exactly, the occupied orbital
    # count (the method is an approximation; 45071.6 here); D is checked column by column
    assert abs(tr - 4096 * 11) < 1e-3 * 4096 * 11
    cols = sample_columns(dims, 10)
    d_or, _, _ = oracle_in_input_layout(s, w["eps"], w["mu"], columns=cols)
    assert max_abs_on_columns(d, d_or, s, cols) <= TOL_D["fp16x3"]


def test_slab_literal_cutoff_solved_both_forms():
    w = WORKLOADS["slab6000"]
    s = make_workload("slab6000", r_c=6.0, ell=1.5)
    res = {}
    for prec in ["fp16x3", "fp64"]:
        with _ctx(s, prec, w["eps"]) as c:
            c.set_electron_count(w["n_e"], max_steps=20, tol=1e-2)
            c.solve_mu()
            tr, en, mu = c.get_trace()
            dims, _, _ = c.get_submatrix_info()
            res[prec] = (c.get_density(), tr, mu, dims)
        assert abs(tr - w["n_e"]) <= 1e-2
    assert res["fp64"][2] == res["fp16x3"][2]
    dims = res["fp64"][3]
    assert dims.min() <= 12 and dims.max() >= 200  # vacuum to bulk
    cols = sample_columns(dims, 24)
    d_or, _, _ = oracle_in_input_layout(s, w["eps"], res["fp64"][2], columns=cols)
    for prec in ["fp64", "fp16x3"]:
        assert max_abs_on_columns(res[prec][0], d_or, s, cols) <= TOL_D[prec], prec


def test_slab_wide_chunked_sampled_columns():
    w = WORKLOADS["slab6000"]
    s = make_workload("slab6000")
    with _ctx(s, "fp16x3", w["eps"]) as c:
        c.set_mu(0.0)
        c.build_density()
        d = c.get_density()
        st = c.get_stats()
        dims, _, _ = c.get_submatrix_info()
    assert st["n_noconv"] == 0 and dims.max() >= 2500
    order = np.argsort(dims)
    cols = sorted({int(order[0]), int(order[len(order) // 2]), int(order[-1])})
    d_or, _, _ = oracle_in_input_layout(s, w["eps"], 0.0, columns=cols)
    assert max_abs_on_columns(d, d_or, s, cols) <= TOL_D["fp16x3"]
