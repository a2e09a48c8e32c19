// Scatter of the owner columns into D and the per-column partial sums
// (Fig. 2 step (iii); Eq. 14).
#pragma once

#include "smx_device.cuh"

namespace smx {

// For submatrix s with converged X ~ sign(T_j - mu I):
//   D[R_j, j] = 1/2 (E_j - X[:, own .. own + b_j))
// written into D laid out like the input values (block (R_j[a], j) at
// pv.fvoff[s.fptr + a], column-major).  X is symmetric, so column own + q is
// read as row own + q (contiguous).  Returns nothing; writes
// partial[col] = (trace of the diagonal block of D, sum over column j of D .* H).
//
// xrow(q, i) must return X[own + q][i] as double.  All threads of the block
// call this function; smem_ls must hold room for s.nblk + 1 ints.  With
// density = false the columns of X themselves are written (another matrix
// function f on the same machinery: F[R_j, j] = f(T_j)[:, own ..]).  With a
// trace_weight W (laid out like H) the first partial is sum over the column of
// D .* W instead of the diagonal's trace (tr(P S) of the non-orthogonal form).
template <class XRow>
__device__ void finish_column(const SubDesc& s, const PatternView& pv, const double* __restrict__ H,
                              double* __restrict__ D, double2* __restrict__ partial, XRow xrow, int* smem_ls,
                              double* red_scratch, bool density = true,
                              const double* __restrict__ trace_weight = nullptr) {
    for (int a = threadIdx.x; a < s.nblk; a += blockDim.x) smem_ls[a] = pv.lstart[s.fptr + a];
    if (threadIdx.x == 0) smem_ls[s.nblk] = s.n;
    __syncthreads();
    double tr = 0.0, en = 0.0;
    const int total = s.n * s.bown;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int q = e / s.n;
        const int i = e - q * s.n;
        // block a of R_j that contains local row i
        int lo = 0, hi = s.nblk - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (smem_ls[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const int64_t k = s.fptr + lo;
        const int br = smem_ls[lo + 1] - smem_ls[lo];
        const int p = i - smem_ls[lo];
        const int64_t off = pv.fvoff[k] + static_cast<int64_t>(q) * br + p;
        const bool diag = (i == s.own + q);
        const double d = density ? 0.5 * ((diag ? 1.0 : 0.0) - xrow(q, i)) : xrow(q, i);
        D[off] = d;
        if (trace_weight) tr += d * trace_weight[off];
        else if (diag) tr += d;
        en += d * H[off];
    }
    tr = block_sum(tr, red_scratch);
    en = block_sum(en, red_scratch);
    if (threadIdx.x == 0) partial[s.col] = make_double2(tr, en);
}

}  // namespace smx
