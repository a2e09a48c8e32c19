"""The finite-temperature Fermi function on the submatrix machinery (Fig. 2 is generic in f):
F[R_j, j] = (I + exp(beta (T_j - mu I)))^-1 [:, own_j] in FP64 on the GPU (tanh doublings with
Newton-Schulz inverses, products only) against the oracle's eigendecomposition, element by
element, over temperatures from infinite to low, two chemical potentials and ragged blocks."""

import numpy as np
import pytest

import oracle as O
from synth import make_mixed_block_system, make_workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _fermi(sysm, mu, beta, prec="fp64"):
    from paper_2205_14741_gb300 import SubmatrixDensity

    with SubmatrixDensity.from_system(sysm) as c:
        c.set_precision(prec)
        c.set_function("fermi")
        c.set_fermi_beta(beta)
        c.set_mu(mu)
        c.build_density()
        tr, en, _ = c.get_trace()
        return c.get_density(), tr, en, c.get_stats()


@pytest.mark.parametrize("beta", [0.0, 1.0, 10.0, 50.0, 400.0])
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_fermi_matches_the_oracle(beta, mu):
    s = make_workload("water32")
    f, tr, en, st = _fermi(s, mu, beta)
    ref = O.fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, mu, beta)
    assert float(np.max(np.abs(f - ref.values))) <= TOL
    assert abs(tr - ref.trace) <= TOL * max(1.0, abs(ref.trace))
    assert abs(en - ref.energy) <= TOL * max(1.0, abs(ref.energy))
    assert st["n_noconv"] == 0
    if beta == 0.0:  # infinite temperature: one half on the diagonal, zero elsewhere
        assert abs(tr - 0.5 * s.n) <= 1e-12


def test_fermi_ragged_blocks():
    s = make_mixed_block_system([1, 5, 13, 7, 2, 9, 4, 11], r_c=6.0, ell=1.5, seed=5)
    f, _, _, _ = _fermi(s, 0.05, 20.0)
    ref = O.fermi_submatrix(s.block_size, s.col_ptr, s.row_idx, s.values, 0.05, 20.0)
    assert float(np.max(np.abs(f - ref.values))) <= TOL


def test_fermi_needs_fp64_and_a_valid_beta():
    from paper_2205_14741_gb300 import SmxError, SubmatrixDensity, _lib

    s = make_workload("water32")
    with SubmatrixDensity.from_system(s) as c:
        with pytest.raises(SmxError) as e:
            c.set_fermi_beta(-1.0)
        assert e.value.status == _lib.ERR_ARG
        c.set_function("fermi")
        c.set_precision("fp16x3")
        with pytest.raises(SmxError) as e:
            c.build_density()
        assert e.value.status == _lib.ERR_UNSUPPORTED
