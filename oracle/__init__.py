"""CPU FP64 oracle for the submatrix density-matrix method.

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
reference that the CUDA path is checked against. Only the test suite, the
package's smoke check and the benchmark's CPU-baseline leg may import it; the
product path never does, and shares no code with it.

Parity status of each function is listed in ``oracle/submatrix.py``,
``oracle/functions.py``, ``oracle/nonorth.py``, ``oracle/fermi.py`` and ``oracle/mlp.py``; every function there is pinned by tests in
``tests/test_oracle_*.py`` against closed forms, invariants, brute force or
independent algorithms.
"""

from .submatrix import (  # noqa: F401
    block_value_offsets,
    filter_blocks,
    to_dense,
    submatrix_rows,
    gather_submatrix,
    sign_eig,
    sign_newton,
    gershgorin_bounds,
    global_gershgorin,
    density_submatrix,
    bisect_mu,
    dense_density,
    SubmatrixResult,
)
from .functions import FUNCTIONS, apply_eig, coupled_newton_schulz, function_submatrix  # noqa: F401
from .nonorth import (  # noqa: F401
    sign_pencil,
    density_pencil,
    density_nonorth_submatrix,
    nonorth_bracket,
    bisect_mu_nonorth,
    take_blocks,
)
from .fermi import fermi_dense, fermi_submatrix  # noqa: F401
