"""The non-orthogonal form of the purification formula (Eq. 14) on the submatrix machinery.

TEST INFRASTRUCTURE ONLY: the reference the CUDA path's non-orthogonal form is
checked against.  Only tests, the smoke check and the benchmark's CPU-baseline
leg use it.

Eq. 14 gives the density matrix of a Kohn-Sham matrix H in a non-orthogonal
basis with overlap S as P = 1/2 (I - sign(S^-1 H - mu I)) S^-1.  The submatrix
method (Fig. 2) applies this function of the pair (H, S) to the dense
submatrices of both on the same index set: for block column j,
A_H = H[R_j, R_j], A_S = S[R_j, R_j] and

    P_j = 1/2 (I - sign(A_S^-1 A_H - mu I)) A_S^-1,      P[R_j, j] = P_j[:, own_j].

S^-1 H is not symmetric, but it is similar to the symmetric S^-1/2 H S^-1/2,
so it has a real spectrum and its sign is V sign(Lambda - mu) V^-1 for its
eigenvector matrix V (Eq. 13 applied to a diagonalisable matrix).  The oracle
takes V from the symmetric-definite pencil (A_H, A_S), whose eigenvectors
satisfy V^T A_S V = I, so V^-1 = V^T A_S; the inverse A_S^-1 is a library
inverse.  Both are library steps; the rest follows Eq. 14 as written.

Readings (the paper does not spell these out): the kept pattern is the
filtered pattern of H and S is taken on it (S blocks outside it are dropped);
the electron count that the bisection matches is tr(P S), evaluated like the
energy over the stored entries, sum_pq P_pq S_pq; the energy is
sum_pq P_pq H_pq; the bisection bracket is the smallest interval holding the
Gershgorin intervals of all A_S^-1/2 A_H A_S^-1/2 (their eigenvalues are the
pencil's), so that P is zero below it and A_S^-1 above it.

Parity status: pinned by tests/test_oracle_nonorth.py (S = I gives the
orthogonal oracle; on a full pattern the dense Loewdin form
S^-1/2 D(S^-1/2 H S^-1/2) S^-1/2, idempotency P S P = P and tr(P S) equal to
the inertia of H - mu S from an LDL^T factorisation; congruence with a
block-diagonal transformation; the bracket's end points).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg

from .functions import apply_eig
from .submatrix import SubmatrixResult, block_value_offsets, gather_submatrix, gershgorin_bounds


def sign_pencil(a_h: np.ndarray, a_s: np.ndarray, mu: float) -> np.ndarray:
    """sign(A_S^-1 A_H - mu I) for symmetric A_H and symmetric positive definite A_S
    (Eq. 13 for a matrix with real spectrum): V sign(Lambda - mu) V^-1 with the pencil's
    eigenvectors V (V^T A_S V = I, hence V^-1 = V^T A_S); sign(0) = 0."""
    lam, v = scipy.linalg.eigh(a_h, a_s)
    return (v * np.sign(lam - mu)[None, :]) @ (v.T @ a_s)


def density_pencil(a_h: np.ndarray, a_s: np.ndarray, mu: float) -> np.ndarray:
    """Eq. 14 for one dense pair: 1/2 (I - sign(A_S^-1 A_H - mu I)) A_S^-1."""
    n = a_h.shape[0]
    return 0.5 * (np.eye(n) - sign_pencil(a_h, a_s, mu)) @ np.linalg.inv(a_s)


def density_nonorth_submatrix(block_size, col_ptr, row_idx, h_values, s_values, mu: float,
                              columns=None) -> SubmatrixResult:
    """P[R_j, j] = P_j[:, own_j] for every block column j (see the module docstring), in the
    (already filtered) pattern of H; S holds values on the same pattern.  ``trace`` is
    tr(P S) = sum_pq P_pq S_pq and ``energy`` sum_pq P_pq H_pq over the stored entries;
    ``n_negative`` counts the pencil eigenvalues below mu per submatrix.  ``columns``
    restricts the work to a subset of block columns."""
    block_size = np.asarray(block_size, dtype=np.int64)
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    h_values = np.asarray(h_values, dtype=np.float64)
    s_values = np.asarray(s_values, dtype=np.float64)
    off = block_value_offsets(block_size, col_ptr, row_idx)
    n_cols = block_size.shape[0]
    cols = range(n_cols) if columns is None else list(columns)
    p_vals = np.zeros_like(h_values)
    dims = np.zeros(n_cols, dtype=np.int64)
    gaps = np.full(n_cols, np.nan)
    nneg = np.zeros(n_cols, dtype=np.int64)
    for j in cols:
        a_h, rows, local = gather_submatrix(block_size, col_ptr, row_idx, h_values, j, 0.0, off)
        a_s, _, _ = gather_submatrix(block_size, col_ptr, row_idx, s_values, j, 0.0, off)
        p = density_pencil(a_h, a_s, mu)
        lam = scipy.linalg.eigh(a_h, a_s, eigvals_only=True)
        dims[j], gaps[j], nneg[j] = a_h.shape[0], float(np.min(np.abs(lam - mu))), int(np.count_nonzero(lam < mu))
        own = int(np.searchsorted(rows, j))
        o0, o1 = local[own], local[own + 1]
        for q, k in enumerate(range(col_ptr[j], col_ptr[j + 1])):
            blk = p[local[q]:local[q + 1], o0:o1]  # rows of block R_j[q], columns of j
            p_vals[off[k]:off[k + 1]] = blk.T.reshape(-1)  # column-major
    mask = np.zeros(h_values.shape[0], dtype=bool)
    for j in cols:
        mask[off[col_ptr[j]]:off[col_ptr[j + 1]]] = True
    trace = float(np.sum(p_vals[mask] * s_values[mask]))
    energy = float(np.sum(p_vals[mask] * h_values[mask]))
    return SubmatrixResult(p_vals, trace, energy, dims, gaps, nneg, float(mu))


def nonorth_bracket(block_size, col_ptr, row_idx, h_values, s_values):
    """[min_j lo_j, max_j hi_j] over the Gershgorin intervals (lo_j, hi_j) of
    M_j = A_S^-1/2 A_H A_S^-1/2, whose eigenvalues are those of the pencil (A_H, A_S)."""
    block_size = np.asarray(block_size, dtype=np.int64)
    off = block_value_offsets(block_size, col_ptr, row_idx)
    lo, hi = np.inf, -np.inf
    for j in range(block_size.shape[0]):
        a_h, _, _ = gather_submatrix(block_size, col_ptr, row_idx, h_values, j, 0.0, off)
        a_s, _, _ = gather_submatrix(block_size, col_ptr, row_idx, s_values, j, 0.0, off)
        li = apply_eig(a_s, "inv_sqrt")
        a, b = gershgorin_bounds(li @ a_h @ li)
        lo, hi = min(lo, a), max(hi, b)
    return float(lo), float(hi)


def bisect_mu_nonorth(block_size, col_ptr, row_idx, h_values, s_values, n_e: float, max_steps: int = 30,
                      tol: float = 0.5, bracket=None):
    """mu by bisection on tr(P(mu) S) = n_e, P by :func:`density_nonorth_submatrix`; the
    same stepping rule as the orthogonal bisection.  Returns (mu, result, history)."""
    lo, hi = nonorth_bracket(block_size, col_ptr, row_idx, h_values, s_values) if bracket is None else bracket
    history = []
    res = None
    for _ in range(max_steps):
        mid = 0.5 * (lo + hi)
        res = density_nonorth_submatrix(block_size, col_ptr, row_idx, h_values, s_values, mid)
        history.append((mid, res.trace))
        if abs(res.trace - n_e) <= tol:
            break
        if res.trace < n_e:
            lo = mid
        else:
            hi = mid
    return res.mu, res, history


def take_blocks(block_size, col_ptr, row_idx, values, keep) -> np.ndarray:
    """The values of the blocks marked in ``keep`` (the filter's flags of H), in order: S on
    the filtered pattern of H."""
    off = block_value_offsets(block_size, col_ptr, row_idx)
    pieces = [values[off[k]:off[k + 1]] for k in range(len(keep)) if keep[k]]
    return np.concatenate(pieces) if pieces else np.zeros(0)


__all__ = ["sign_pencil", "density_pencil", "density_nonorth_submatrix", "nonorth_bracket", "bisect_mu_nonorth",
           "take_blocks"]
