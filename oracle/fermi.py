"""The finite-temperature Fermi function on the submatrix machinery (Fig. 2 is generic in f).

TEST INFRASTRUCTURE ONLY: the reference a GPU form of this function will be checked against.
Only tests, the smoke check and the benchmark's CPU-baseline leg use it.

For a symmetric H, an inverse temperature beta (in inverse units of H) and a chemical
potential mu, the Fermi-Dirac density matrix is F = (I + exp(beta (H - mu I)))^-1, the
finite-temperature counterpart of D = 1/2 (I - sign(H - mu I)) of Eq. 14: both are functions of
H with occupations 1 / (1 + exp(beta (lambda - mu))), which tend to the step function (one
half at lambda = mu) as beta grows.  The submatrix method applies it to T_j = H[R_j, R_j] and
keeps the owner columns, F[R_j, j] = f(T_j)[:, own_j].  This oracle evaluates f on the
eigenvalues of each submatrix (LAPACK through numpy as a library step; the occupations through
scipy's logistic function, which stays finite for any beta (lambda - mu)).

Readings: no spin factor (the trace counts orbitals, as for D); "trace" is the sum of the
diagonal entries of the diagonal blocks and "energy" the sum over stored entries F_pq H_pq.

Parity status: pinned by tests/test_oracle_fermi.py (diagonal inputs against the logistic
function; the large-beta limit against the density-matrix oracle; a full pattern against
(I + expm(beta (H - mu I)))^-1 from scipy's matrix exponential and a solve; particle-hole
symmetry F(2 mu I - H) = I - F(H) block column by block column on a truncated pattern; the
beta -> 0 limit 1/2 I; the trace increasing in mu).
"""

from __future__ import annotations

import numpy as np
import scipy.special

from .submatrix import SubmatrixResult, _block, block_value_offsets, gather_submatrix, submatrix_rows


def fermi_dense(a: np.ndarray, mu: float, beta: float) -> np.ndarray:
    """(I + exp(beta (A - mu I)))^-1 of a symmetric A from its eigendecomposition."""
    lam, v = np.linalg.eigh(a)
    occ = scipy.special.expit(-beta * (lam - mu))
    return (v * occ[None, :]) @ v.T


def fermi_submatrix(block_size, col_ptr, row_idx, values, mu: float, beta: float,
                    columns=None) -> SubmatrixResult:
    """F[R_j, j] = f(T_j)[:, own_j] with f the Fermi function at (mu, beta), for every block
    column j of the (already filtered) H, in its pattern.  ``columns`` restricts the work to
    a subset of block columns."""
    if not beta >= 0.0:
        raise ValueError("beta must be non-negative")
    block_size = np.asarray(block_size, dtype=np.int64)
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    values = np.asarray(values, dtype=np.float64)
    off = block_value_offsets(block_size, col_ptr, row_idx)
    n_cols = block_size.shape[0]
    cols = range(n_cols) if columns is None else list(columns)
    f_vals = np.zeros_like(values)
    dims = np.zeros(n_cols, dtype=np.int64)
    for j in cols:
        t, rows, local = gather_submatrix(block_size, col_ptr, row_idx, values, j, 0.0, off)
        f = fermi_dense(t, mu, beta)
        own = int(np.searchsorted(rows, j))
        o0, o1 = local[own], local[own + 1]
        dims[j] = t.shape[0]
        for q, k in enumerate(range(col_ptr[j], col_ptr[j + 1])):
            blk = f[local[q]:local[q + 1], o0:o1]  # rows of block R_j[q], columns of j
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
