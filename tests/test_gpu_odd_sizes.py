"""Odd submatrix sizes: n = 1, 7, 127, 129 and 3001, each as the single submatrix of a
complete pattern (every block column's submatrix is the whole matrix), so the result is the
dense projector of Eq. 14.  n = 1 and 7 sit far below a tile, 127 / 129 straddle the 128-row
tile, 3001 spans 24 row tiles of the streamed form with a ragged tail."""

import numpy as np
import pytest

import oracle as O
from synth import make_mixed_block_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = {1: [1], 7: [7], 127: [64, 63], 129: [64, 64, 1], 3001: [64] * 46 + [57]}
# the split form's error grows with the accumulation length (about 1e-5 near n = 3000)
TOL = {"fp64": 1e-10, "fp16x3": 1e-5}
TOL_3001 = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("n", sorted(SIZES))
@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_odd_sizes_against_the_dense_projector(n, prec):
    if prec == "fp64" and n > 200:
        pytest.skip("one FP64 CTA per submatrix: minutes at n = 3001")
    from paper_2205_14741_gb300 import SubmatrixDensity

    s = make_mixed_block_system(SIZES[n], r_c=np.inf, ell=1.5, seed=60 + n)
    assert s.n == n
    h = O.to_dense(s.block_size, s.col_ptr, s.row_idx, s.values)
    d_ref = O.dense_density(h, 0.0)
    with SubmatrixDensity.from_system(s) as c:
        c.set_precision(prec)
        c.set_mu(0.0)
        c.build_density()
        d = O.to_dense(s.block_size, s.col_ptr, s.row_idx, c.get_density())
        tr, _, _ = c.get_trace()
        st = c.get_stats()
    assert st["dim_min"] == n and st["dim_max"] == n and st["n_noconv"] == 0
    tol = TOL_3001 if (n == 3001 and prec == "fp16x3") else TOL[prec]
    assert float(np.max(np.abs(d - d_ref))) <= tol
    assert abs(tr - np.trace(d_ref)) <= max(1e-6, tol) * n
