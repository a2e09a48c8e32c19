"""Other matrix functions on the submatrix machinery (Fig. 2 is generic in f): A^-1/2, A^1/2, A^-1.

TEST INFRASTRUCTURE ONLY: the reference the CUDA path's function forms are
checked against.  Only tests, the smoke check and the benchmark's CPU-baseline
leg use it.

For a symmetric positive definite H (an overlap matrix, say) the submatrix
method gives sparse approximations of H^(-1/2), H^(1/2) and H^(-1): for every block
column j the dense submatrix A_j = T_j - mu I (Fig. 2 step (i)), f(A_j) by
eigendecomposition (step (ii)), and the columns of block j of f(A_j) into the
result (step (iii)).  Section 3 obtains these functions from the sign function
through Eq. 12, sign([[0, A], [I, 0]]) = [[0, A^1/2], [A^-1/2, 0]] (the inverse
as the square of A^-1/2); the GPU path iterates that identity, this oracle
evaluates f on the eigenvalues.

Readings: f acts on T_j - mu I (mu = 0 for H itself); the result has exactly
the filtered pattern of H; its "trace" is the sum of the diagonal entries of
the diagonal blocks and its "energy" the sum over stored entries F_pq H_pq
(the same bookkeeping as the density matrix).

Parity status: pinned by tests/test_oracle_functions.py (diagonal and
block-diagonal inputs, a full pattern against the dense function computed
from numpy's eigh, F A F = I and F A = I on a full pattern, the inverse
against a library solve, and an independent coupled Newton-Schulz iteration
of Eq. 12 on small submatrices).
"""

from __future__ import annotations

import numpy as np

from .submatrix import SubmatrixResult, _block, block_value_offsets, gather_submatrix, submatrix_rows

FUNCTIONS = ("inv_sqrt", "sqrt", "inv")


def apply_eig(a: np.ndarray, f: str) -> np.ndarray:
    """f(A) for a symmetric positive definite A from its eigendecomposition."""
    lam, v = np.linalg.eigh(a)
    if np.min(lam) <= 0.0:
        raise ValueError("the matrix is not positive definite")
    g = {"inv_sqrt": lam ** -0.5, "sqrt": np.sqrt(lam), "inv": 1.0 / lam}[f]
    return (v * g) @ v.T


def coupled_newton_schulz(a: np.ndarray, c: float, tol: float = 1e-14, max_iter: int = 100):
    """(A^1/2, A^-1/2) by the coupled Newton-Schulz iteration: the sign iteration
    X <- X (3I - X^2)/2 of the block matrix [[0, A/c], [I, 0]] (Eq. 12) written per block,
    Y <- Y T, Z <- T Z with T = (3I - Z Y)/2 from Y = A/c, Z = I (c >= rho(A)).  An algorithm
    independent of the eigendecomposition, used only to pin :func:`apply_eig`."""
    n = a.shape[0]
    y = a / c
    z = np.eye(n)
    for _ in range(max_iter):
        t = 0.5 * (3.0 * np.eye(n) - z @ y)
        y, z = y @ t, t @ z
        if np.linalg.norm(z @ y - np.eye(n)) <= tol:
            break
    return y * np.sqrt(c), z / np.sqrt(c)


def function_submatrix(block_size, col_ptr, row_idx, values, f: str, mu: float = 0.0,
                       columns=None) -> SubmatrixResult:
    """F[R_j, j] = f(T_j - mu I)[:, cols of j] for every block column j, in the pattern of H
    (already filtered).  ``columns`` restricts the work to a subset of block columns."""
    if f not in FUNCTIONS:
        raise ValueError(f"unknown function {f!r}")
    block_size = np.asarray(block_size, dtype=np.int64)
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    values = np.asarray(values, dtype=np.float64)
    off = block_value_offsets(block_size, col_ptr, row_idx)
    n_cols = block_size.shape[0]
    cols = range(n_cols) if columns is None else list(columns)
    f_vals = np.zeros_like(values)
    dims = np.zeros(n_cols, dtype=np.int64)
    for j in cols:
        a, rows, local = gather_submatrix(block_size, col_ptr, row_idx, values, j, mu, off)
        fa = apply_eig(a, f)
        own = int(np.searchsorted(rows, j))
        o0, o1 = local[own], local[own + 1]
        dims[j] = a.shape[0]
        for q, k in enumerate(range(col_ptr[j], col_ptr[j + 1])):
            blk = fa[local[q]:local[q + 1], o0:o1]  # rows of block R_j[q], columns of j
            f_vals[off[k]:off[k + 1]] = blk.T.reshape(-1)  # column-major
    trace = 0.0
    for j in cols:
        rows = submatrix_rows(col_ptr, row_idx, j)
        k = col_ptr[j] + int(np.searchsorted(rows, j))
        trace += float(np.trace(_block(f_vals, off, k, block_size[j], block_size[j])))
    mask = np.zeros(values.shape[0], dtype=bool)
    for j in cols:
        mask[off[col_ptr[j]]:off[col_ptr[j + 1]]] = True
    energy = float(np.sum(f_vals[mask] * values[mask]))
    nan = np.full(n_cols, np.nan)
    return SubmatrixResult(f_vals, trace, energy, dims, nan, np.zeros(n_cols, dtype=np.int64), float(mu))
