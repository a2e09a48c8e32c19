"""Submatrix method for the density matrix, plain FP64 on the CPU.

TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.
Only tests, the smoke check and the benchmark's CPU-baseline leg use it.

What it computes (the paper, Section 2 and Section 3):

* Eq. 14, purification by the matrix sign function, with an orthogonalised
  input (S = I):  D = 1/2 (I - sign(H - mu I)).
* Eq. 13, the matrix sign function sign(A) = A (A^2)^(-1/2).  For a symmetric
  A = V diag(lambda) V^T this equals V diag(sign(lambda)) V^T, which is how
  this oracle evaluates it (eigendecomposition by LAPACK through numpy; the
  iterative methods are the GPU path's business).
* Fig. 2, the submatrix method: (i) one dense submatrix per column, made of
  the rows stored in that column, (ii) the matrix function of each dense
  submatrix, (iii) the columns of each result that belong to its column
  written back into the sparse result.

Readings where the paper is silent (the same readings bind the GPU path):

* granularity is the block column: block column j gives the submatrix
  T_j = H[R_j, R_j], R_j = sorted block rows stored in column j of the
  filtered H; blocks of H[R_j, R_j] that are not stored are zero;
* the result columns kept are the columns of block j only, over all rows
  of R_j: D[R_j, j] = 1/2 (E_j - sign(T_j - mu I)[:, cols of j]);
* filtering drops an off-diagonal block when its Frobenius norm is strictly
  below eps; diagonal blocks are always kept;
* D has exactly the filtered pattern of H and is not symmetrised (an explicit
  option symmetrises it);
* sign(0) = 0, so an eigenvalue exactly at mu contributes one half;
* trace(D) = sum of the diagonal entries of the diagonal blocks of D, and the
  band-structure energy is E = trace(D H) = sum over stored entries D_pq H_pq
  (H symmetric);
* mu by bisection on trace(D) = n_e inside the global Gershgorin interval of
  the filtered H, stopping when |trace(D) - n_e| <= tol or after max_steps
  steps; the result is the last evaluated midpoint and its D.

Parity status: every function below is pinned by tests/test_oracle_*.py
(closed-form 2x2 sign, diagonal and block-diagonal cases, sign(A)^2 = I,
commutation and positivity, an independent Newton sign iteration, exact
equality with the dense spectral projector when the pattern is complete,
brute force on tiny systems, monotonicity of trace(D) in mu).
"""

from __future__ import annotations

import concurrent.futures as _cf
import dataclasses

import numpy as np


# --------------------------------------------------------------------------
# block-CSC helpers
# --------------------------------------------------------------------------

def block_value_offsets(block_size, col_ptr, row_idx) -> np.ndarray:
    """Offset of every stored block inside ``values`` (length nnzb + 1)."""
    block_size = np.asarray(block_size, dtype=np.int64)
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    row_idx = np.asarray(row_idx, dtype=np.int64)
    n_cols = block_size.shape[0]
    col_of = np.repeat(np.arange(n_cols), np.diff(col_ptr))
    sizes = block_size[row_idx] * block_size[col_of]
    off = np.zeros(row_idx.shape[0] + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return off


def _block(values, off, k, br, bc):
    """Block k as a dense br x bc array (stored column-major)."""
    return values[off[k]:off[k + 1]].reshape(bc, br).T


def filter_blocks(block_size, col_ptr, row_idx, values, eps: float):
    """Drop off-diagonal blocks whose Frobenius norm is strictly below ``eps``.

    Returns (col_ptr, row_idx, values, keep) of the filtered matrix; ``keep``
    marks the surviving blocks of the input.  Diagonal blocks are always kept.
    """
    block_size = np.asarray(block_size)
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    row_idx = np.asarray(row_idx)
    values = np.asarray(values, dtype=np.float64)
    off = block_value_offsets(block_size, col_ptr, row_idx)
    n_cols = block_size.shape[0]
    keep = np.zeros(row_idx.shape[0], dtype=bool)
    for j in range(n_cols):
        for k in range(col_ptr[j], col_ptr[j + 1]):
            r = int(row_idx[k])
            norm = np.sqrt(np.sum(values[off[k]:off[k + 1]] ** 2))
            keep[k] = (r == j) or not (norm < eps)
    new_ptr = np.zeros(n_cols + 1, dtype=np.int64)
    for j in range(n_cols):
        new_ptr[j + 1] = new_ptr[j] + int(np.count_nonzero(keep[col_ptr[j]:col_ptr[j + 1]]))
    new_rows = np.asarray(row_idx)[keep].astype(np.int32)
    pieces = [values[off[k]:off[k + 1]] for k in range(row_idx.shape[0]) if keep[k]]
    new_vals = np.concatenate(pieces) if pieces else np.zeros(0)
    return new_ptr, new_rows, new_vals, keep


def to_dense(block_size, col_ptr, row_idx, values) -> np.ndarray:
    """Dense N x N matrix of a block-CSC matrix (absent blocks are zero)."""
    block_size = np.asarray(block_size, dtype=np.int64)
    start = np.zeros(block_size.shape[0] + 1, dtype=np.int64)
    start[1:] = np.cumsum(block_size)
    off = block_value_offsets(block_size, col_ptr, row_idx)
    a = np.zeros((start[-1], start[-1]))
    for j in range(block_size.shape[0]):
        for k in range(col_ptr[j], col_ptr[j + 1]):
            r = int(row_idx[k])
            a[start[r]:start[r + 1], start[j]:start[j + 1]] = _block(values, off, k, block_size[r], block_size[j])
    return a


def submatrix_rows(col_ptr, row_idx, j: int) -> np.ndarray:
    """R_j: the block rows stored in block column j, ascending (Fig. 2, step (i))."""
    return np.asarray(row_idx[col_ptr[j]:col_ptr[j + 1]], dtype=np.int64)


def gather_submatrix(block_size, col_ptr, row_idx, values, j: int, mu: float = 0.0, off=None):
    """Dense T_j - mu I with T_j = H[R_j, R_j] (Fig. 2 step (i); shift of Eq. 14).

    Returns (A, R_j, local_start) where local_start[a] is the first row of
    block R_j[a] inside A (length |R_j| + 1).
    """
    block_size = np.asarray(block_size, dtype=np.int64)
    if off is None:
        off = block_value_offsets(block_size, col_ptr, row_idx)
    rows = submatrix_rows(col_ptr, row_idx, j)
    local = np.zeros(rows.shape[0] + 1, dtype=np.int64)
    local[1:] = np.cumsum(block_size[rows])
    a = np.zeros((local[-1], local[-1]))
    for cb, c in enumerate(rows):
        col_rows = np.asarray(row_idx[col_ptr[c]:col_ptr[c + 1]], dtype=np.int64)
        for rb, r in enumerate(rows):
            pos = np.searchsorted(col_rows, r)
            if pos < col_rows.shape[0] and col_rows[pos] == r:
                k = col_ptr[c] + pos
                a[local[rb]:local[rb + 1], local[cb]:local[cb + 1]] = _block(values, off, k, block_size[r], block_size[c])
    a -= mu * np.eye(a.shape[0])
    return a, rows, local


# --------------------------------------------------------------------------
# matrix sign (Eq. 13)
# --------------------------------------------------------------------------

def sign_eig(a: np.ndarray):
    """sign(A) of a symmetric A as V diag(sign(lambda)) V^T (Eq. 13); sign(0) = 0.

    Returns (S, lambda) with the eigenvalues ascending.
    """
    lam, v = np.linalg.eigh(a)
    return (v * np.sign(lam)[None, :]) @ v.T, lam


def sign_newton(a: np.ndarray, tol: float = 1e-15, max_iter: int = 100) -> np.ndarray:
    """sign(A) by the Newton iteration X <- (X + X^-1)/2 from X0 = A.

    An algorithm independent of the eigendecomposition, used only to pin
    :func:`sign_eig`.  A must be non-singular.
    """
    x = np.array(a, dtype=np.float64)
    for _ in range(max_iter):
        x_new = 0.5 * (x + np.linalg.inv(x))
        if np.max(np.abs(x_new - x)) <= tol * max(1.0, np.max(np.abs(x_new))):
            return x_new
        x = x_new
    return x


def gershgorin_bounds(a: np.ndarray):
    """(lo, hi) = (min_r a_rr - R_r, max_r a_rr + R_r), R_r = sum_{c != r} |a_rc|."""
    d = np.diag(a)
    radius = np.sum(np.abs(a), axis=1) - np.abs(d)
    return float(np.min(d - radius)), float(np.max(d + radius))


# --------------------------------------------------------------------------
# the submatrix method (Fig. 2 + Eq. 14)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SubmatrixResult:
    values: np.ndarray  # D in the (filtered) pattern of H, column-major blocks
    trace: float  # trace(D)
    energy: float  # trace(D H)
    dims: np.ndarray  # n_j per block column
    min_abs_eig: np.ndarray  # min |lambda(T_j - mu I)| per block column (the gap)
    n_negative: np.ndarray  # number of eigenvalues of T_j - mu I below zero
    mu: float


def _one_column(block_size, col_ptr, row_idx, values, off, j, mu):
    a, rows, local = gather_submatrix(block_size, col_ptr, row_idx, values, j, mu, off)
    s, lam = sign_eig(a)
    own = int(np.searchsorted(rows, j))
    o0, o1 = local[own], local[own + 1]
    e = np.zeros((a.shape[0], o1 - o0))
    e[o0:o1, :] = np.eye(o1 - o0)
    dcol = 0.5 * (e - s[:, o0:o1])  # D[R_j, j] = 1/2 (E_j - sign(T_j - mu I)[:, own])
    return j, dcol, rows, local, a.shape[0], float(np.min(np.abs(lam))), int(np.count_nonzero(lam < 0))


def density_submatrix(block_size, col_ptr, row_idx, values, mu: float, workers: int = 1,
                      symmetrize: bool = False, columns=None) -> SubmatrixResult:
    """D = 1/2 (I - sign(H - mu I)) by the submatrix method, in the pattern of H.

    ``H`` must already be filtered (see :func:`filter_blocks`).  ``columns``
    restricts the work to a subset of block columns (the other columns of D
    stay zero and do not enter trace and energy); used to time a bounded
    sample.
    """
    block_size = np.asarray(block_size, dtype=np.int64)
    col_ptr = np.asarray(col_ptr, dtype=np.int64)
    values = np.asarray(values, dtype=np.float64)
    off = block_value_offsets(block_size, col_ptr, row_idx)
    n_cols = block_size.shape[0]
    cols = range(n_cols) if columns is None else list(columns)
    d_vals = np.zeros_like(values)
    dims = np.zeros(n_cols, dtype=np.int64)
    gaps = np.full(n_cols, np.nan)
    nneg = np.zeros(n_cols, dtype=np.int64)

    def place(res):
        j, dcol, rows, local, n_j, gap, neg = res
        dims[j], gaps[j], nneg[j] = n_j, gap, neg
        for a, k in enumerate(range(col_ptr[j], col_ptr[j + 1])):
            blk = dcol[local[a]:local[a + 1], :]  # rows of block R_j[a], columns of j
            d_vals[off[k]:off[k + 1]] = blk.T.reshape(-1)  # column-major

    if workers > 1:
        with _cf.ThreadPoolExecutor(max_workers=workers) as ex:
            for res in ex.map(lambda j: _one_column(block_size, col_ptr, row_idx, values, off, j, mu), cols):
                place(res)
    else:
        for j in cols:
            place(_one_column(block_size, col_ptr, row_idx, values, off, j, mu))

    if symmetrize:
        d_vals = _symmetrize(block_size, col_ptr, row_idx, d_vals, off)

    trace = 0.0
    for j in cols:
        rows = submatrix_rows(col_ptr, row_idx, j)
        k = col_ptr[j] + int(np.searchsorted(rows, j))
        trace += float(np.trace(_block(d_vals, off, k, block_size[j], block_size[j])))
    mask = np.zeros(values.shape[0], dtype=bool)
    for j in cols:
        mask[off[col_ptr[j]]:off[col_ptr[j + 1]]] = True
    energy = float(np.sum(d_vals[mask] * values[mask]))
    return SubmatrixResult(d_vals, trace, energy, dims, gaps, nneg, float(mu))


def _symmetrize(block_size, col_ptr, row_idx, d_vals, off):
    """1/2 (D + D^T) in the (symmetric) pattern."""
    out = np.empty_like(d_vals)
    n_cols = block_size.shape[0]
    for j in range(n_cols):
        for k in range(col_ptr[j], col_ptr[j + 1]):
            r = int(row_idx[k])
            rows_r = np.asarray(row_idx[col_ptr[r]:col_ptr[r + 1]])
            kt = col_ptr[r] + int(np.searchsorted(rows_r, j))
            blk = _block(d_vals, off, k, block_size[r], block_size[j])
            blk_t = _block(d_vals, off, kt, block_size[j], block_size[r]).T
            out[off[k]:off[k + 1]] = (0.5 * (blk + blk_t)).T.reshape(-1)
    return out


def global_gershgorin(block_size, col_ptr, row_idx, values):
    """Gershgorin interval of the whole block-sparse H without forming it densely."""
    block_size = np.asarray(block_size, dtype=np.int64)
    start = np.zeros(block_size.shape[0] + 1, dtype=np.int64)
    start[1:] = np.cumsum(block_size)
    off = block_value_offsets(block_size, col_ptr, row_idx)
    n = int(start[-1])
    abs_sum = np.zeros(n)
    diag = np.zeros(n)
    for j in range(block_size.shape[0]):
        for k in range(col_ptr[j], col_ptr[j + 1]):
            r = int(row_idx[k])
            blk = _block(values, off, k, block_size[r], block_size[j])
            abs_sum[start[r]:start[r + 1]] += np.sum(np.abs(blk), axis=1)
            if r == j:
                diag[start[r]:start[r + 1]] = np.diag(blk)
    radius = abs_sum - np.abs(diag)
    return float(np.min(diag - radius)), float(np.max(diag + radius))


def bisect_mu(block_size, col_ptr, row_idx, values, n_e: float, max_steps: int = 30, tol: float = 0.5,
              workers: int = 1, bracket=None):
    """mu by bisection on trace(D(mu)) = n_e (D by :func:`density_submatrix`).

    Bracket: the global Gershgorin interval of H unless given.  Each step
    evaluates the midpoint; it stops when |trace - n_e| <= tol or after
    ``max_steps`` steps.  Returns (mu, result, history) where ``result`` is
    the last evaluation and history lists (mu, trace) per step.
    """
    lo, hi = global_gershgorin(block_size, col_ptr, row_idx, values) if bracket is None else bracket
    history = []
    res = None
    for _ in range(max_steps):
        mid = 0.5 * (lo + hi)
        res = density_submatrix(block_size, col_ptr, row_idx, values, mid, workers=workers)
        history.append((mid, res.trace))
        if abs(res.trace - n_e) <= tol:
            break
        if res.trace < n_e:
            lo = mid
        else:
            hi = mid
    return res.mu, res, history


def dense_density(h: np.ndarray, mu: float) -> np.ndarray:
    """Exact density matrix of a dense symmetric H as the spectral projector.

    D = sum_{lambda_k < mu} v_k v_k^T + 1/2 sum_{lambda_k = mu} v_k v_k^T,
    which equals 1/2 (I - sign(H - mu I)) (Eq. 14 with S = I).
    """
    lam, v = np.linalg.eigh(h)
    w = np.where(lam < mu, 1.0, np.where(lam == mu, 0.5, 0.0))
    return (v * w[None, :]) @ v.T
