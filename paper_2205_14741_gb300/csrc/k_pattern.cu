// Filter, gather + spectral bound, Gershgorin bracket and reductions.
//
//  a1  block filter (Frobenius norm per block; diagonal blocks kept) and the
//      Gershgorin bracket of the filtered H (mu bisection)
//  a3  gather T_j = H[R_j, R_j] - mu I (Fig. 2 step (i), shift of Eq. 14)
//  a4  Gershgorin bound b_j >= spectral radius of T_j - mu I
//  a8  deterministic FP64 sums of trace(D) and trace(D H)
#include <algorithm>

#include <cuda_fp16.h>

#include "smx_finish.cuh"
#include "smx_kernels.h"

namespace smx {

// a1 + the Gershgorin bracket of a9 in one pass: one CTA per block column j of
// the input pattern, G groups of eight lanes (G = blockDim / 8).  The column's
// block rows, block sizes and value offsets are first staged in shared memory
// (one round of dependent loads for the whole column); then group g takes the
// blocks k0 + g, k0 + g + G, ... and lane q0 of a group the block's columns q0,
// q0 + 8, ...  Per (block, column): the values are checked for finiteness and
// copied to FP32, their sum of squares and of absolute values taken; the
// block's Frobenius norm (squares summed over its columns in a fixed tree over
// the group) decides whether it is kept (diagonal blocks always), against
// keep_prev when given.  The absolute column sums of the kept blocks go into
// per-group accumulators in shared memory (each lane owns its entries), then
// are summed over the groups in order: with the diagonal block's diagonal d_q,
// column q's Gershgorin interval is [d_q - r_q, d_q + r_q], r_q = sum - |d_q|
// (H symmetric: column sums are row sums).  The column's minimum and maximum
// reach the bracket through atomic maxima of order-preserving integer images
// (independent of the order of the CTAs), and the last CTA writes the bracket
// and its midpoint.
constexpr int kFilterGroups = 8;

// Order-preserving image of a double in the unsigned integers: x < y <=> enc(x) < enc(y)
// for non-NaN x, y, and enc(x) > 0 for every x, so 0 is below every value.
__device__ __forceinline__ unsigned long long ord_enc(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_dec(unsigned long long e) {
    const unsigned long long b = (e >> 63) ? (e & 0x7fffffffffffffffull) : ~e;
    return __longlong_as_double(static_cast<long long>(b));
}

__global__ void __launch_bounds__(8 * kFilterGroups) k_filter(const double* __restrict__ H, const int64_t* __restrict__ col_ptr,
                                                              const int32_t* __restrict__ row_idx,
                                                              const int64_t* __restrict__ voff,
                                                              const int32_t* __restrict__ bsize, int bmax, int max_col_blocks,
                                                              double eps, uint8_t* __restrict__ keep,
                                                              const uint8_t* __restrict__ keep_prev, float* __restrict__ H32,
                                                              DevScalars* sc) {
    // cs[G][bmax] kept column sums, ca[G][bmax] this block's, dg[bmax]; the column's block
    // offsets, rows and sizes
    extern __shared__ double fsm[];
    __shared__ bool last_s;
    const int G = blockDim.x >> 3, nt = blockDim.x;
    double* cs = fsm;
    double* ca = cs + G * bmax;
    double* dg = ca + G * bmax;
    int64_t* mvo = reinterpret_cast<int64_t*>(dg + bmax);
    int* mr = reinterpret_cast<int*>(mvo + max_col_blocks);
    int* mbr = mr + max_col_blocks;
    const int j = blockIdx.x, tid = threadIdx.x, g = tid >> 3, q0 = tid & 7;
    const int bc = bsize[j];
    const int64_t k0 = col_ptr[j], k1 = col_ptr[j + 1];
    const int nk = static_cast<int>(k1 - k0);
    for (int i = tid; i < nk; i += nt) {
        const int r = row_idx[k0 + i];
        mr[i] = r;
        mvo[i] = voff[k0 + i];
        mbr[i] = bsize[r];
    }
    const unsigned gmask = 0xffu << (tid & 24);  // this group's lanes (groups differ in their block counts)
    // keep decisions: sum of squares in FP32 unless it lies within its rounding bound of eps^2
    // (then again in FP64, as the oracle takes it); eps <= 0 keeps every block
    const bool keep_all = !(eps > 0.0);
    const float eps2f = keep_all ? 0.0f : d2f_rn(eps * eps);
    const bool fp32_ok = eps2f >= 1e-30f;  // far from FP32 underflow
    for (int i = tid; i < G * bmax; i += nt) cs[i] = 0.0;
    for (int q = tid; q < bc; q += nt) dg[q] = 0.0;
    __syncthreads();
    bool finite = true;
    for (int i = g; i < nk; i += G) {  // the group is uniform
        const int64_t k = k0 + i;
        const int r = mr[i];
        const int br = mbr[i];
        const double* blk = H + mvo[i];
        float* blk32 = H32 + mvo[i];
        float ss = 0.0f;
        for (int q = q0; q < bc; q += 8) {
            const double* col = blk + static_cast<int64_t>(q) * br;
            float* col32 = blk32 + static_cast<int64_t>(q) * br;
            double a = 0.0;  // FP64: the Gershgorin bracket
            for (int p0 = 0; p0 < br; p0 += 8) {  // eight loads in flight, then their use
                double v[8];
#pragma unroll
                for (int p = 0; p < 8; ++p) v[p] = p0 + p < br ? col[p0 + p] : 0.0;
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    if (p0 + p >= br) break;
                    const float f = d2f_rn(v[p]);
                    ss = fmaf(f, f, ss);
                    a += fabs(v[p]);
                    finite = finite && finite_bits(v[p]);
                    col32[p0 + p] = f;
                }
            }
            ca[g * bmax + q] = a;
            if (r == j) dg[q] = col[q];
        }
        // the block's sum of squares over its eight lanes (a fixed tree: every lane ends
        // with the same bits, so the decision is uniform over the group)
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) ss += __shfl_xor_sync(gmask, ss, o, 8);
        bool kept = keep_all || r == j;
        if (!kept) {
            // |ss - sum v^2| <= (n_elem + 5) 2^-24 sum v^2 (conversion, FMA chain, tree); twice that
            const float tol = static_cast<float>(br * bc + 8) * 0x1p-23f * eps2f;
            if (fp32_ok && fabsf(ss - eps2f) > tol) {
                kept = !(ss < eps2f);
            } else {
                double sd = 0.0;
                for (int q = q0; q < bc; q += 8)
                    for (int p = 0; p < br; ++p) {
                        const double x = blk[static_cast<int64_t>(q) * br + p];
                        sd = fma(x, x, sd);
                    }
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) sd += __shfl_xor_sync(gmask, sd, o, 8);
                kept = !(sqrt(sd) < eps);
            }
        }
        if (kept)
            for (int q = q0; q < bc; q += 8) cs[g * bmax + q] += ca[g * bmax + q];
        if (q0 == 0) {
            keep[k] = kept ? 1 : 0;
            if (keep_prev && kept != (keep_prev[k] != 0)) atomicOr(&sc->changed, 1);
        }
    }
    if (!finite) atomicCAS(&sc->status, kOk, kErrNonfinite);
    __syncthreads();
    // column q: the kept blocks' sums over the groups in order, then its interval
    double lo = INFINITY, hi = -INFINITY;
    for (int q = tid; q < bc; q += nt) {
        double c_ = 0.0;
        for (int gg = 0; gg < G; ++gg) c_ += cs[gg * bmax + q];
        const double d = dg[q], rad = c_ - fabs(d);
        lo = fmin(lo, d - rad);
        hi = fmax(hi, d + rad);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((tid & 31) == 0 && lo <= hi) {  // a warp without columns has nothing to add
        atomicMax(&sc->nlo_enc, ord_enc(-lo));
        atomicMax(&sc->hi_enc, ord_enc(hi));
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last_s = atomicAdd(&sc->filter_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_s || tid != 0) return;
    __threadfence();
    const double blo = -ord_dec(atomicExch(&sc->nlo_enc, 0ull)), bhi = ord_dec(atomicExch(&sc->hi_enc, 0ull));
    sc->br_lo = blo;
    sc->br_hi = bhi;
    sc->mu0 = 0.5 * (blo + bhi);
    sc->filter_done = 0u;
}

cudaError_t launch_filter_gershgorin(const double* H, const int64_t* col_ptr, const int32_t* row_idx, const int64_t* voff,
                                     const int32_t* bsize, int n_cols, int bmax, int max_col_blocks, double eps,
                                     uint8_t* keep, const uint8_t* keep_prev, float* H32, DevScalars* sc, cudaStream_t st) {
    if (n_cols <= 0) return cudaSuccess;
    // as many groups as fit 48 KB of column sums next to the staged block information
    const size_t meta = static_cast<size_t>(max_col_blocks) * (sizeof(int64_t) + 2 * sizeof(int));
    int groups = kFilterGroups;
    while (groups > 1 && sizeof(double) * static_cast<size_t>(2 * groups + 1) * bmax + meta > (48u << 10)) groups >>= 1;
    const size_t smem = sizeof(double) * static_cast<size_t>(2 * groups + 1) * bmax + meta;
    if (smem > (48u << 10)) {
        cudaError_t e = cudaFuncSetAttribute(k_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_filter<<<n_cols, 8 * groups, smem, st>>>(H, col_ptr, row_idx, voff, bsize, bmax, max_col_blocks, eps, keep, keep_prev,
                                               H32, sc);
    return cudaGetLastError();
}

// The end of both gather forms: the per-warp row statistics (Gershgorin maximum
// m and the feature sums of this warp's rows) reduced over the 8 warps in
// order, the bound b_j (Gershgorin, or the learned model's), the features and
// predictions.  All 256 threads call it; the FP64 scalar work is thread 0's
// (on every thread it would queue eight warps on the narrow FP64 pipe).
template <class R>
__device__ void gather_finish(const SubDesc& s, R m, float f2, float da, float ds, float dq, float rs, float dm,
                              float rm, double* __restrict__ bound, const GatherExtras& ex) {
    __shared__ R warp_max_s[8];
    __shared__ float stat_s[8][7];  // per warp: F2, Da, Ds, Dq, Rs (sums), Dm, Rm (maxima)
    __shared__ float x_s[kModelFeatures], h1_s[kModelHidden], y_s[2][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        warp_max_s[warp] = m;
        stat_s[warp][0] = f2;
        stat_s[warp][1] = da;
        stat_s[warp][2] = ds;
        stat_s[warp][3] = dq;
        stat_s[warp][4] = rs;
        stat_s[warp][5] = dm;
        stat_s[warp][6] = rm;
    }
    __syncthreads();
    // G = the largest row sum (the maximum is exact in the staging type)
    auto gmax = [&]() -> double {
        R g = R(0);
        for (int w = 0; w < 8; ++w) g = fmax(g, warp_max_s[w]);
        return static_cast<double>(g);
    };
    if (ex.feat || ex.params) {
        if (tid == 0) {
            float F2 = 0.f, Da = 0.f, Ds = 0.f, Dq = 0.f, Rs = 0.f, Dm = 0.f, Rm = 0.f;
            for (int w = 0; w < 8; ++w) {
                F2 += stat_s[w][0];
                Da += stat_s[w][1];
                Ds += stat_s[w][2];
                Dq += stat_s[w][3];
                Rs += stat_s[w][4];
                Dm = fmaxf(Dm, stat_s[w][5]);
                Rm = fmaxf(Rm, stat_s[w][6]);
            }
            const float n = static_cast<float>(s.n), G = static_cast<float>(gmax());
            const float ig = G > 0.f ? 1.f / G : 0.f, mean = Ds / n;
            x_s[0] = sqrtf(F2 / n) * ig;
            x_s[1] = Dm * ig;
            x_s[2] = Da / n * ig;
            x_s[3] = sqrtf(fmaxf(Dq / n - mean * mean, 0.f)) * ig;
            x_s[4] = Rm * ig;
            x_s[5] = Rs / n * ig;
            x_s[6] = n / 256.f;
            x_s[7] = mean * ig;
            x_s[8] = ex.prev_ratio ? ex.prev_ratio[blockIdx.x] : 0.f;
            if (ex.feat)
                for (int k = 0; k < kModelFeatures; ++k) ex.feat[static_cast<int64_t>(blockIdx.x) * kModelFeatures + k] = x_s[k];
        }
        __syncthreads();
    }
    const float* p = ex.params;
    auto w16 = [](float v) { return __half2float(__float2half_rn(v)); };
    if (p) {
        // the network, weights rounded to FP16 (threads 0..63: one hidden unit each)
        if (tid < kModelHidden) {
            float acc = w16(p[kOffB1 + tid]);
            for (int k = 0; k < kModelFeatures; ++k) acc = fmaf(w16(p[tid * kModelFeatures + k]), x_s[k], acc);
            h1_s[tid] = tanhf(acc);
        }
        __syncthreads();
        if (tid < kModelHidden) {
            float acc = w16(p[kOffB2 + tid]);
            for (int k = 0; k < kModelHidden; ++k) acc = fmaf(w16(p[kOffW2 + tid * kModelHidden + k]), h1_s[k], acc);
            const float h2 = tanhf(acc);
            float y0 = w16(p[kOffW3 + tid]) * h2, y1 = w16(p[kOffW3 + kModelHidden + tid]) * h2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                y0 += __shfl_xor_sync(0xffffffffu, y0, o);
                y1 += __shfl_xor_sync(0xffffffffu, y1, o);
            }
            if (lane == 0) {
                y_s[warp][0] = y0;
                y_s[warp][1] = y1;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        double g = gmax();
        // in FP32 the row sums carry a relative error below n 2^-24, covered by the 1e-5 margin
        if (sizeof(R) == 4) g *= 1.0 + 1e-5;
        if (!(g > 0.0)) g = 1.0;
        double b = g;
        if (p) {
            const float y0 = (y_s[0][0] + y_s[1][0]) + w16(p[kOffB3]);
            const float y1 = (y_s[0][1] + y_s[1][1]) + w16(p[kOffB3 + 1]);
            if (ex.pred) {
                ex.pred[2 * static_cast<int64_t>(blockIdx.x)] = y0;
                ex.pred[2 * static_cast<int64_t>(blockIdx.x) + 1] = y1;
            }
            b = g * fmin(fmax(static_cast<double>(y0), 0.02), 1.0) * (1.0 + ex.margin) / 1.2;
        }
        bound[blockIdx.x] = b;
        if (ex.gersh) ex.gersh[blockIdx.x] = g;
    }
}

// One CTA per submatrix; T_j is row-major with leading dimension s.ld (zero
// in columns [n, ld)).  Warp w takes the block rows c = w, w + 8, ... of T_j.
// T_j is symmetric, so block row c is block column c transposed: the blocks
// of H's column R_j[c] whose rows lie in R_j, listed by local block a in a
// per-warp table (value offset, or -1 for a block dropped by the filter).
// Rows x = start(c) + q are then written column by column: the lane of
// column y reads element (y - start(a), q) of block (R_j[a], R_j[c]) straight
// from H (a = the local block of y; consecutive y of a block are consecutive
// in memory) for up to eight rows q at once, and the stores are coalesced.
// Each row's absolute sum (Gershgorin bound b_j = max_x sum_y |T[x][y]|) and
// the feature statistics are taken as the row is written, lane-strided over
// y, then reduced over the warp (a fixed order).
//
// Learned bound (optional): features of A = T_j - mu I (all over G except f6,
// f8): f0 ||A||_F/sqrt(n), f1 max|A_rr|, f2 mean|A_rr|, f3 std(A_rr), f4 max_r
// R_r, f5 mean_r R_r (R_r = sum_{c != r} |A_rc|), f6 n/256, f7 mean A_rr, f8
// the previous step's ratio; then the 9 -> 64 -> 64 -> 2 tanh network with the
// parameters rounded to FP16, and b_j = G clamp(rho_hat/G, 0.02, 1) (1 + margin)/1.2.
constexpr int kGatherRows = 8;  // rows of a block row written together

template <class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_gather_bound(const SubDesc* __restrict__ subs, PatternView pv,
                                                      const R* __restrict__ H, double mu_d, R* __restrict__ T,
                                                      double* __restrict__ bound, int nblk_max, int n_max,
                                                      GatherExtras ex) {
    extern __shared__ __align__(16) unsigned char gsm[];
    if (ex.skip && *ex.skip) return;
    const R mu = static_cast<R>(ex.mu_dev ? *ex.mu_dev : mu_d);
    const SubDesc s = subs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t* tab = reinterpret_cast<int64_t*>(gsm) + static_cast<size_t>(warp) * nblk_max;  // per warp
    int* rows = reinterpret_cast<int*>(reinterpret_cast<int64_t*>(gsm) + static_cast<size_t>(8) * nblk_max);  // R_j
    int* ls = rows + nblk_max;      // local starts, nblk + 1 entries
    int* cinfo = ls + nblk_max + 1;  // per local column y: local block a (bits 16-31), its size (8-15), y - start(a) (0-7)
    for (int a = tid; a < s.nblk; a += blockDim.x) {
        rows[a] = pv.frow_idx[s.fptr + a];
        ls[a] = pv.lstart[s.fptr + a];
    }
    if (tid == 0) ls[s.nblk] = s.n;
    __syncthreads();
    for (int y = tid; y < s.n; y += blockDim.x) {
        int lo = 0, hi = s.nblk - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ls[mid] <= y) lo = mid; else hi = mid - 1;
        }
        cinfo[y] = (lo << 16) | ((ls[lo + 1] - ls[lo]) << 8) | (y - ls[lo]);
    }
    __syncthreads();

    R* t = T + s.t_off;
    R m = R(0);  // largest row sum so far (in the staging type: no FP64 work per row in FP32)
    float f2 = 0.f, da = 0.f, ds = 0.f, dq = 0.f, rs = 0.f, dm = 0.f, rm = 0.f;  // feature statistics
    for (int c = warp; c < s.nblk; c += 8) {
        const int col = rows[c];
        const int bc = ls[c + 1] - ls[c];
        // tab[a] = value offset of block (R_j[a], col), -1 when the filter dropped it
        for (int a = lane; a < s.nblk; a += 32) tab[a] = -1;
        __syncwarp();
        const int64_t k0 = pv.fcol_ptr[col], k1 = pv.fcol_ptr[col + 1];
        for (int64_t k = k0 + lane; k < k1; k += 32) {
            const int r = pv.frow_idx[k];
            int lo = 0, hi = s.nblk - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (rows[mid] < r) lo = mid + 1; else hi = mid;
            }
            if (rows[lo] == r) tab[lo] = pv.fvoff[k];
        }
        __syncwarp();
        for (int q0 = 0; q0 < bc; q0 += kGatherRows) {
            const int nq = min(kGatherRows, bc - q0);
            R acc[kGatherRows];
            float sq[kGatherRows];
            R dsel = R(0);  // this lane's diagonal entry of the group, if it holds one
#pragma unroll
            for (int qq = 0; qq < kGatherRows; ++qq) {
                acc[qq] = R(0);
                sq[qq] = 0.f;
            }
            const int dcol = ls[c] + q0;  // column of row q0's diagonal entry
            for (int y = lane; y < s.ld; y += 32) {
                R v[kGatherRows];
#pragma unroll
                for (int qq = 0; qq < kGatherRows; ++qq) v[qq] = R(0);
                if (y < s.n) {
                    const int ci = cinfo[y];
                    const int64_t vo = tab[ci >> 16];
                    if (vo >= 0) {
                        const int br = (ci >> 8) & 0xff;
                        const R* src = H + vo + (ci & 0xff) + static_cast<int64_t>(q0) * br;
#pragma unroll
                        for (int qq = 0; qq < kGatherRows; ++qq)
                            if (qq < nq) v[qq] = src[static_cast<int64_t>(qq) * br];
                    }
                }
                const int dq_ = y - dcol;  // row of the group whose diagonal is column y
                if (dq_ >= 0 && dq_ < nq) {
#pragma unroll
                    for (int qq = 0; qq < kGatherRows; ++qq)
                        if (qq == dq_) {
                            v[qq] -= mu;
                            dsel = v[qq];
                        }
                }
#pragma unroll
                for (int qq = 0; qq < kGatherRows; ++qq)
                    if (qq < nq) {
                        t[static_cast<int64_t>(dcol + qq) * s.ld + y] = v[qq];
                        acc[qq] += fabs(v[qq]);
                        sq[qq] = fmaf(static_cast<float>(v[qq]), static_cast<float>(v[qq]), sq[qq]);
                    }
            }
#pragma unroll
            for (int qq = 0; qq < kGatherRows; ++qq) {
                if (qq >= nq) break;
                R a_ = acc[qq];
                float s_ = sq[qq];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a_ += __shfl_xor_sync(0xffffffffu, a_, o);
                    s_ += __shfl_xor_sync(0xffffffffu, s_, o);
                }
                const float d = static_cast<float>(__shfl_sync(0xffffffffu, dsel, (dcol + qq) & 31));
                m = fmax(m, a_);
                const float ad = fabsf(d), rr = static_cast<float>(a_) - ad;
                f2 += s_;
                da += ad;
                ds += d;
                dq = fmaf(d, d, dq);
                rs += rr;
                dm = fmaxf(dm, ad);
                rm = fmaxf(rm, rr);
            }
        }
        __syncwarp();
    }
    gather_finish<R>(s, m, f2, da, ds, dq, rs, dm, rm, bound, ex);
}

// Staged form of the same gather, for patterns whose block rows fit a per-warp
// shared-memory buffer (bmax x round_up(max n, 4) elements) and whose
// submatrices have at most kStagedMaxBlocks blocks; one CTA per submatrix,
// same outputs bit for bit (same values, same per-lane and per-warp orders of
// the row sums and feature sums).
//
// 1. The block map of T_j in shared memory, built once for the submatrix by
//    all warps: map[a][c] = value offset of block (R_j[c], R_j[a]), the block
//    of H's column R_j[a] in block row R_j[c] (-1 when the filter dropped it).
//    T_j is symmetric, so block row a of T_j is that column transposed: the
//    column-major block (R_j[c], R_j[a]) holds tile (a, c) of T_j row-major.
// 2. Warp w assembles block rows a = w, w + 8, ... in its buffer: up to eight
//    rows at once, 32 columns per lane-step and four lane-steps per batch
//    (all loads of a batch issued before its shared-memory stores), -mu on the
//    diagonal, row sums and feature sums as the values go in.
// 3. The block row's b_a x ld elements are one contiguous, 16-byte aligned
//    range of the staging buffer: one lane writes it with a bulk copy
//    (cp.async.bulk shared -> global) and the warp goes on to the next block
//    row; the buffer is reused once that copy has read it.
constexpr int kStagedMaxBlocks = 64;
constexpr size_t kStagedSmemLimit = 100u << 10;  // at least two CTAs per SM
constexpr int kStagedBatch = 4;  // lane-steps of 32 columns whose loads are issued together
constexpr int kPairBatch = 1;    // uniform 6 x 6 blocks: lane-steps of 32 pairs whose loads are issued together

template <class R> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// BS = 6: every block is 6 x 6 (the water workloads): a block row is taken as pairs of
// consecutive elements (float2 / double2 loads and stores), six rows per pair of columns;
// BS = 0: any block sizes, one element per lane and row group of up to eight rows.
template <class R, int BS>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? (BS == 6 ? 4 : 3) : 2) k_gather_staged(const SubDesc* __restrict__ subs, PatternView pv,
                                                       const R* __restrict__ H, double mu_d, R* __restrict__ T,
                                                       double* __restrict__ bound, int nblk_max, int stage_elems,
                                                       GatherExtras ex) {
    extern __shared__ __align__(128) unsigned char gsm[];
    if (ex.skip && *ex.skip) return;
    const R mu = static_cast<R>(ex.mu_dev ? *ex.mu_dev : mu_d);
    const SubDesc s = subs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = s.nblk, ld = s.ld;
    R* stage = reinterpret_cast<R*>(gsm) + static_cast<size_t>(warp) * stage_elems;  // this warp's block-row buffer
    int64_t* map = reinterpret_cast<int64_t*>(gsm + static_cast<size_t>(8) * stage_elems * sizeof(R));
    int64_t* kcol = map + static_cast<size_t>(nblk_max) * nblk_max;  // filtered blocks of column R_j[a]: [kcol[2a], kcol[2a + 1])
    int* rows = reinterpret_cast<int*>(kcol + 2 * nblk_max);  // R_j
    int* ls = rows + nblk_max;        // local starts, nb + 1 entries
    int* cinfo = ls + nblk_max + 1;   // per local column y: local block (bits 16-31), its size (8-15), y - start (0-7)
    const bool premap = pv.maps != nullptr;  // the map built once per pattern: one coalesced read
    if (premap) {
        const int32_t* gm = pv.maps + pv.map_off[s.col];
        for (int a = tid; a < nb; a += blockDim.x) ls[a] = pv.lstart[s.fptr + a];
        for (int i = tid; i < nb * nb; i += blockDim.x) map[i] = gm[i];
    } else {
        for (int a = tid; a < nb; a += blockDim.x) {
            const int r = pv.frow_idx[s.fptr + a];
            rows[a] = r;
            ls[a] = pv.lstart[s.fptr + a];
            kcol[2 * a] = pv.fcol_ptr[r];
            kcol[2 * a + 1] = pv.fcol_ptr[r + 1];
        }
        for (int i = tid; i < nb * nb; i += blockDim.x) map[i] = -1;
    }
    if (tid == 0) ls[nb] = s.n;
    __syncthreads();
    if constexpr (BS == 0) {
        for (int y = tid; y < s.n; y += blockDim.x) {
            int lo = 0, hi = nb - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ls[mid] <= y) lo = mid; else hi = mid - 1;
            }
            cinfo[y] = (lo << 16) | ((ls[lo + 1] - ls[lo]) << 8) | (y - ls[lo]);
        }
    }
    for (int a = premap ? nb : warp; a < nb; a += 8) {
        for (int64_t k = kcol[2 * a] + lane; k < kcol[2 * a + 1]; k += 32) {
            const int r = pv.frow_idx[k];
            const int64_t vo = pv.fvoff[k];
            int lo = 0, hi = nb - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (rows[mid] < r) lo = mid + 1; else hi = mid;
            }
            if (rows[lo] == r) map[a * nb + lo] = vo;
        }
    }
    __syncthreads();

    R* tj = T + s.t_off;
    R m = R(0);  // largest row sum so far (in the staging type: no FP64 work per row in FP32)
    float f2 = 0.f, da = 0.f, ds = 0.f, dq = 0.f, rs = 0.f, dm = 0.f, rm = 0.f;  // feature statistics
    for (int a = warp; a < nb; a += 8) {
        const int x0 = ls[a], ba = ls[a + 1] - x0;
        const int64_t* mrow = map + a * nb;
        if (lane == 0) bulk_wait_read_all();  // the buffer's previous bulk copy has read it
        __syncwarp();
        if constexpr (BS == 6) {
            // pair unit t of a row: tile c = t / 3, columns 6c + p2, p2 + 1 (p2 = 2 (t mod 3)); tile
            // (a, c) is H's block (R_j[c], R_j[a]) holding the 6 x 6 tile row-major, so row q of
            // the pair is at vo + 6q + p2; pairs past the 3 nb of data are the zero padding
            using V2 = typename Pair<R>::type;
            const int units = ld >> 1, uvalid = 3 * nb;
            R acc[6];
            float sq[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                acc[q] = R(0);
                sq[q] = 0.f;
            }
            for (int t0 = 0; t0 < units; t0 += 32 * kPairBatch) {
                V2 v[kPairBatch][6];
#pragma unroll
                for (int i = 0; i < kPairBatch; ++i) {
                    const int t = t0 + lane + 32 * i;
                    const int c = t / 3, p2 = 2 * (t - 3 * c);
                    const int64_t vo = t < uvalid ? mrow[c] : -1;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        v[i][q].x = R(0);
                        v[i][q].y = R(0);
                        if (vo >= 0) v[i][q] = *reinterpret_cast<const V2*>(H + vo + 6 * q + p2);
                    }
                }
#pragma unroll
                for (int i = 0; i < kPairBatch; ++i) {
                    const int t = t0 + lane + 32 * i;
                    if (t >= units) break;
                    const int c = t / 3, p2 = 2 * (t - 3 * c);
                    const bool dtile = c == a;  // the diagonal tile of block row a
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        V2 w = v[i][q];
                        if (dtile && p2 == (q & ~1)) {
                            if (q & 1) w.y -= mu;
                            else w.x -= mu;
                        }
                        *reinterpret_cast<V2*>(stage + q * ld + 2 * t) = w;
                        acc[q] += fabs(w.x) + fabs(w.y);
                        sq[q] = fmaf(static_cast<float>(w.x), static_cast<float>(w.x), sq[q]);
                        sq[q] = fmaf(static_cast<float>(w.y), static_cast<float>(w.y), sq[q]);
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                R a_ = acc[q];
                float s_ = sq[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a_ += __shfl_xor_sync(0xffffffffu, a_, o);
                    s_ += __shfl_xor_sync(0xffffffffu, s_, o);
                }
                const float d = static_cast<float>(stage[q * ld + x0 + q]);  // the diagonal entry of row x0 + q
                m = fmax(m, a_);
                const float ad = fabsf(d), rr = static_cast<float>(a_) - ad;
                f2 += s_;
                da += ad;
                ds += d;
                dq = fmaf(d, d, dq);
                rs += rr;
                dm = fmaxf(dm, ad);
                rm = fmaxf(rm, rr);
            }
        } else
        for (int q0 = 0; q0 < ba; q0 += kGatherRows) {
            const int nq = min(kGatherRows, ba - q0);
            R acc[kGatherRows];
            float sq[kGatherRows];
            R dsel = R(0);  // this lane's diagonal entry of the group, if it holds one
#pragma unroll
            for (int qq = 0; qq < kGatherRows; ++qq) {
                acc[qq] = R(0);
                sq[qq] = 0.f;
            }
            const int dcol = x0 + q0;  // column of row q0's diagonal entry
            R* srow = stage + static_cast<size_t>(q0) * ld;
            for (int y0 = 0; y0 < ld; y0 += 32 * kStagedBatch) {
                R v[kStagedBatch][kGatherRows];
#pragma unroll
                for (int i = 0; i < kStagedBatch; ++i) {
                    const int y = y0 + lane + 32 * i;
                    const R* src = nullptr;
                    int br = 0;
                    if (y < s.n) {
                        const int ci = cinfo[y];
                        const int64_t vo = mrow[ci >> 16];
                        if (vo >= 0) {
                            br = (ci >> 8) & 0xff;
                            src = H + vo + (ci & 0xff) + q0 * br;
                        }
                    }
#pragma unroll
                    for (int qq = 0; qq < kGatherRows; ++qq) v[i][qq] = (src != nullptr && qq < nq) ? src[qq * br] : R(0);
                }
#pragma unroll
                for (int i = 0; i < kStagedBatch; ++i) {
                    const int y = y0 + lane + 32 * i;
                    if (y >= ld) break;
                    const int dq_ = y - dcol;  // row of the group whose diagonal is column y
#pragma unroll
                    for (int qq = 0; qq < kGatherRows; ++qq) {
                        if (qq >= nq) break;
                        R val = v[i][qq];
                        if (qq == dq_) {
                            val -= mu;
                            dsel = val;
                        }
                        srow[qq * ld + y] = val;
                        acc[qq] += fabs(val);
                        sq[qq] = fmaf(static_cast<float>(val), static_cast<float>(val), sq[qq]);
                    }
                }
            }
#pragma unroll
            for (int qq = 0; qq < kGatherRows; ++qq) {
                if (qq >= nq) break;
                R a_ = acc[qq];
                float s_ = sq[qq];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a_ += __shfl_xor_sync(0xffffffffu, a_, o);
                    s_ += __shfl_xor_sync(0xffffffffu, s_, o);
                }
                const float d = static_cast<float>(__shfl_sync(0xffffffffu, dsel, (dcol + qq) & 31));
                m = fmax(m, a_);
                const float ad = fabsf(d), rr = static_cast<float>(a_) - ad;
                f2 += s_;
                da += ad;
                ds += d;
                dq = fmaf(d, d, dq);
                rs += rr;
                dm = fmaxf(dm, ad);
                rm = fmaxf(rm, rr);
            }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            bulk_store(tj + static_cast<int64_t>(x0) * ld, stage, static_cast<uint32_t>(ba * ld * sizeof(R)));
            bulk_commit();
        }
    }
    if (lane == 0) bulk_wait_all();
    gather_finish<R>(s, m, f2, da, ds, dq, rs, dm, rm, bound, ex);
}

template <class R, int BS>
static cudaError_t launch_staged(const SubDesc* subs, int n_subs, int max_nblk, int stage_elems, size_t smem,
                                 const PatternView& pv, const R* H, double mu, R* T, double* bound, const GatherExtras& ex,
                                 cudaStream_t st) {
    if (smem > (48u << 10)) {
        cudaError_t e = cudaFuncSetAttribute(k_gather_staged<R, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_gather_staged<R, BS><<<n_subs, 256, smem, st>>>(subs, pv, H, mu, T, bound, max_nblk, stage_elems, ex);
    return cudaGetLastError();
}

template <class R>
static cudaError_t launch_gather(const SubDesc* subs, int n_subs, int max_nblk, int max_n, int bmax, bool uniform,
                                 const PatternView& pv, const R* H, double mu, R* T, double* bound, const GatherExtras& ex,
                                 cudaStream_t st) {
    if (n_subs <= 0) return cudaSuccess;
    // staged form: eight block-row buffers, the block map, R_j, local starts, column ranges, column info
    const int stage_elems = static_cast<int>((static_cast<int64_t>(bmax) * ((max_n + 3) / 4 * 4) + 31) / 32 * 32);
    const size_t staged_smem = static_cast<size_t>(8) * stage_elems * sizeof(R) +
                               (static_cast<size_t>(max_nblk) * max_nblk + 2 * max_nblk) * sizeof(int64_t) +
                               (static_cast<size_t>(2 * max_nblk + 1) + static_cast<size_t>(max_n)) * sizeof(int);
    if (max_nblk <= kStagedMaxBlocks && staged_smem <= kStagedSmemLimit) {
        if (uniform && bmax == 6)
            return launch_staged<R, 6>(subs, n_subs, max_nblk, stage_elems, staged_smem, pv, H, mu, T, bound, ex, st);
        return launch_staged<R, 0>(subs, n_subs, max_nblk, stage_elems, staged_smem, pv, H, mu, T, bound, ex, st);
    }
    // per-warp block tables, R_j, local starts and the local block of every column
    const size_t smem = static_cast<size_t>(8) * max_nblk * sizeof(int64_t) +
                        (static_cast<size_t>(2 * max_nblk + 1) + static_cast<size_t>(max_n)) * sizeof(int);
    if (smem > (48u << 10)) {
        cudaError_t e = cudaFuncSetAttribute(k_gather_bound<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_gather_bound<R><<<n_subs, 256, smem, st>>>(subs, pv, H, mu, T, bound, max_nblk, max_n, ex);
    return cudaGetLastError();
}

cudaError_t launch_gather_bound(const SubDesc* subs, int n_subs, int max_nblk, int max_n, int bmax, bool uniform,
                                const PatternView& pv, const double* H, double mu, double* T, double* bound,
                                const GatherExtras& ex, cudaStream_t st) {
    return launch_gather<double>(subs, n_subs, max_nblk, max_n, bmax, uniform, pv, H, mu, T, bound, ex, st);
}

cudaError_t launch_gather_bound_f32(const SubDesc* subs, int n_subs, int max_nblk, int max_n, int bmax, bool uniform,
                                    const PatternView& pv, const float* H32, double mu, float* T32, double* bound,
                                    const GatherExtras& ex, cudaStream_t st) {
    return launch_gather<float>(subs, n_subs, max_nblk, max_n, bmax, uniform, pv, H32, mu, T32, bound, ex, st);
}

// Deterministic sums of partial[0, n_cols) by one block (each thread adds a fixed
// strided subset in order, then a fixed tree) into sc->trace, sc->energy.
__device__ void sum_partials(const double2* partial, int n_cols, DevScalars* sc, double* scratch) {
    double tr = 0.0, en = 0.0;
    for (int c = threadIdx.x; c < n_cols; c += blockDim.x) {
        const double2 p = __ldcg(partial + c);
        tr += p.x;
        en += p.y;
    }
    tr = block_sum(tr, scratch);
    en = block_sum(en, scratch);
    if (threadIdx.x == 0) {
        sc->trace = tr;
        sc->energy = en;
    }
}

// One CTA per submatrix: scatter of the saved owner columns (Fig. 2 step (iii);
// Eq. 14: D[R_j, j] = 1/2 (E_j - X[:, own]), X symmetric, so the saved column q
// is X's row own + q), then (the last CTA) the sums of a8.
//
// The elements are taken in the order of D's own layout: the kept blocks
// (R_j[a], j) of column j, each column-major b_a x b_j, so element e of the
// packed column lies in block a (the blocks' packed starts are ls[a] b_j) at
// e' = e - ls[a] b_j, row p = e' mod b_a of column q = e' / b_a.  With uniform
// b x b blocks (BS = b) a = e / b^2 and no tables are needed; otherwise block
// a = blk[e / b_j] from shared-memory tables.  Consecutive threads store
// consecutive D entries and read runs of b_a consecutive saved values; each
// thread issues the loads of up to kScatterBatch elements before their stores.
//
// Arithmetic (GB300's FP64 pipe is narrow): an off-diagonal entry -x/2 is exact
// in FP32 and widened on the integer pipes; the b_j diagonal entries (1 - x)/2
// are formed in FP64 by the first b_j threads after the sweep (which skips
// them), and only they add to the trace (FP64).  The energy sum trace(D H)
// takes FP32 products of D and the FP32 copy of H, summed in FP32 per thread
// and warp, then in FP64 over the warps and the columns.
constexpr int kScatterBatch = 4;

template <int BS>
__global__ void __launch_bounds__(256) k_scatter_owner(const SubDesc* __restrict__ subs, PatternView pv,
                                                       const float* __restrict__ xown, const float* __restrict__ H32,
                                                       double* __restrict__ D, double2* __restrict__ partial, int n_cols,
                                                       DevScalars* sc, const int* skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char ssm[];
    __shared__ double scratch[32];
    __shared__ double tr_s[8];
    __shared__ float en_s[8];
    __shared__ bool last_s;
    const SubDesc s = subs[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = s.nblk, n = s.n, bj = s.bown;
    const int64_t* fvoff = pv.fvoff + s.fptr;
    int64_t* fvo = reinterpret_cast<int64_t*>(ssm);  // generic form: value offset of block (R_j[a], j)
    int* ls = reinterpret_cast<int*>(fvo + nb);      // ... local starts, nb + 1 entries
    int* blk = ls + nb + 1;                          // ... local block of every row of T_j
    if constexpr (BS == 0) {
        for (int a = tid; a < nb; a += blockDim.x) {
            fvo[a] = fvoff[a];
            ls[a] = pv.lstart[s.fptr + a];
        }
        if (tid == 0) ls[nb] = n;
        __syncthreads();
        for (int a = warp; a < nb; a += 8)
            for (int r = ls[a] + lane; r < ls[a + 1]; r += 32) blk[r] = a;
        __syncthreads();
    }
    const float* x = xown + s.x_off;
    float en = 0.0f;
    const int total = n * bj;
    for (int e0 = tid; e0 < total; e0 += kScatterBatch * 256) {
        float xv[kScatterBatch], hv[kScatterBatch];
        int64_t off[kScatterBatch];
#pragma unroll
        for (int i = 0; i < kScatterBatch; ++i) {
            const int e = e0 + i * 256;
            off[i] = -1;
            xv[i] = 0.f;
            hv[i] = 0.f;
            if (e < total) {
                int a, ba, ep, row0;
                if constexpr (BS > 0) {
                    a = e / (BS * BS);
                    ba = BS;
                    ep = e - a * (BS * BS);
                    row0 = BS * a;
                } else {
                    a = blk[e / bj];
                    ba = ls[a + 1] - ls[a];
                    ep = e - ls[a] * bj;
                    row0 = ls[a];
                }
                const int q = ep / ba, row = row0 + (ep - q * ba);
                if (row != s.own + q) {  // diagonal entries after the sweep
                    off[i] = (BS > 0 ? fvoff[a] : fvo[a]) + ep;
                    xv[i] = x[static_cast<int64_t>(q) * n + row];
                    hv[i] = H32[off[i]];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kScatterBatch; ++i) {
            if (off[i] < 0) continue;
            const float d32 = -0.5f * xv[i];
            D[off[i]] = f2d(d32);
            en = fmaf(d32, hv[i], en);
        }
    }
    double tr = 0.0;
    int a_own;
    if constexpr (BS > 0) a_own = s.own / BS;
    else a_own = blk[s.own];
    const int64_t own_off = BS > 0 ? fvoff[a_own] : fvo[a_own];
    for (int q = tid; q < bj; q += blockDim.x) {  // the diagonal entry of the owner block's column q
        const int64_t off = own_off + static_cast<int64_t>(q) * bj + q;
        const double d = 0.5 * (1.0 - f2d(x[static_cast<int64_t>(q) * n + s.own + q]));
        D[off] = d;
        tr += d;
        en = fmaf(d2f_rn(d), H32[off], en);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) en += __shfl_xor_sync(0xffffffffu, en, o);
    if (warp * 32 < bj) tr = warp_sum(tr);  // only the warps holding diagonal entries (warp-uniform)
    if (lane == 0) {
        en_s[warp] = en;
        tr_s[warp] = tr;
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0, e = 0.0;
        for (int w = 0; w < 8; ++w) {
            t += tr_s[w];
            e += f2d(en_s[w]);
        }
        partial[s.col] = make_double2(t, e);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last_s = atomicAdd(&sc->scatter_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    sum_partials(partial, n_cols, sc, scratch);
    if (tid == 0) {
        sc->scatter_done = 0u;
        sc->ns_counter = 0;  // the Newton-Schulz launch before this one is complete
    }
}

cudaError_t launch_scatter_owner(const SubDesc* subs, int n_subs, int max_nblk, int max_n, int bmax, bool uniform,
                                 const PatternView& pv, const float* xown, const float* H32, double* D, double2* partial,
                                 int n_cols, DevScalars* sc, cudaStream_t st, const int* skip) {
    if (n_subs <= 0) return cudaSuccess;
    if (uniform && bmax == 6) {
        k_scatter_owner<6><<<n_subs, 256, 0, st>>>(subs, pv, xown, H32, D, partial, n_cols, sc, skip);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(int64_t) * static_cast<size_t>(max_nblk) +
                        sizeof(int) * (static_cast<size_t>(max_nblk) + 1 + static_cast<size_t>(max_n));
    if (smem > (48u << 10)) {
        cudaError_t e = cudaFuncSetAttribute(k_scatter_owner<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_scatter_owner<0><<<n_subs, 256, smem, st>>>(subs, pv, xown, H32, D, partial, n_cols, sc, skip);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_reduce(const double2* __restrict__ partial, int n_cols, DevScalars* sc,
                                                 const int* skip) {
    if (skip && *skip) return;
    __shared__ double scratch[32];
    sum_partials(partial, n_cols, sc, scratch);
}

cudaError_t launch_reduce(const double2* partial, int n_cols, DevScalars* sc, cudaStream_t st, const int* skip) {
    k_reduce<<<1, 256, 0, st>>>(partial, n_cols, sc, skip);
    return cudaGetLastError();
}

// The symmetrised D (the option of taking 1/2 (D + D^T): the submatrix method's D is not
// symmetric).  Warp w of the grid takes pair w; its lanes stride over the pair's elements.
__global__ void __launch_bounds__(256) k_symmetrize(const SymPair* __restrict__ pairs, int n_pairs,
                                                    const uint8_t* __restrict__ keep, double* __restrict__ D,
                                                    const int* skip) {
    if (skip && *skip) return;
    const int w = static_cast<int>((blockIdx.x * static_cast<unsigned>(blockDim.x) + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= n_pairs) return;
    const SymPair p = pairs[w];
    const int br = p.br, bj = p.bj;
    if (p.k == p.kt) {  // a diagonal block (br == bj): element (r, c) with r < c and its mirror (c, r)
        if (!keep[p.k]) return;
        double* blk = D + p.off_k;
        for (int e = lane; e < br * br; e += 32) {
            const int c = e / br, r = e - c * br;  // column-major: element (r, c) at c br + r
            if (r < c) {
                const double v = 0.5 * (blk[e] + blk[r * br + c]);
                blk[e] = v;
                blk[r * br + c] = v;
            }
        }
        return;
    }
    const bool kk = keep[p.k] != 0, kt = keep[p.kt] != 0;
    double* bk = D + p.off_k;    // br x bj: rows of block row r, columns of block column j
    double* bt = D + p.off_kt;   // bj x br: its transpose position
    for (int e = lane; e < br * bj; e += 32) {
        const int c = e / br, r = e - c * br;  // element (r, c) of block k; (c, r) of block kt
        const int et = r * bj + c;
        const double v = 0.5 * (bk[e] + bt[et]);  // a dropped block holds zeros
        bk[e] = kk ? v : 0.0;
        bt[et] = kt ? v : 0.0;
    }
}

cudaError_t launch_symmetrize(const SymPair* pairs, int n_pairs, const uint8_t* keep, double* D, cudaStream_t st,
                              const int* skip) {
    if (n_pairs <= 0) return cudaSuccess;
    const int blocks = (n_pairs + 7) / 8;  // eight warps (pairs) per CTA
    k_symmetrize<<<blocks, 256, 0, st>>>(pairs, n_pairs, keep, D, skip);
    return cudaGetLastError();
}

// a9 on the device: the bisection's state lives in the device scalars, so a whole mu solve is
// enqueued at once (the same decisions as the host loop, in the same FP64 arithmetic).
__global__ void k_bisect_init(DevScalars* sc, double lo, double hi) {
    sc->bis_lo = lo;
    sc->bis_hi = hi;
    sc->bis_mid = 0.5 * (lo + hi);
    sc->bis_done = 0;
    sc->bis_steps = 0;
}

__global__ void k_bisect_step(DevScalars* sc, double n_e, double tol, int max_steps) {
    if (sc->bis_done) return;
    const int steps = ++sc->bis_steps;
    const double tr = sc->trace, mid = sc->bis_mid;
    if (sc->status != kOk || fabs(tr - n_e) <= tol || steps >= max_steps) {
        sc->bis_done = 1;  // the result is the last evaluated mu (and its D)
        return;
    }
    if (tr < n_e) sc->bis_lo = mid;
    else sc->bis_hi = mid;
    sc->bis_mid = 0.5 * (sc->bis_lo + sc->bis_hi);
}

cudaError_t launch_bisect_init(DevScalars* sc, double lo, double hi, cudaStream_t st) {
    k_bisect_init<<<1, 1, 0, st>>>(sc, lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_bisect_step(DevScalars* sc, double n_e, double tol, int max_steps, cudaStream_t st) {
    k_bisect_step<<<1, 1, 0, st>>>(sc, n_e, tol, max_steps);
    return cudaGetLastError();
}

// Failure-detection self-test: one thread waits on a fresh mbarrier that nothing
// arrives at, with the library's bounded wait at a caller-given poll limit.  No
// asynchronous copy or tensor-core operation is in flight, so giving up is
// clean: the wait records kErrTimeout in *status and the kernel returns.
__global__ void k_wait_selftest(int* status, uint32_t poll_limit, int* polls_out) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_barrier_init();
    uint32_t i = 0;
    for (; i < poll_limit; ++i)
        if (mbar_try_wait(&bar, 0)) break;
    if (i == poll_limit) atomicCAS(status, kOk, kErrTimeout);
    if (polls_out) *polls_out = static_cast<int>(i);
}

cudaError_t launch_wait_selftest(int* status, uint32_t poll_limit, int* polls_out, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(status, poll_limit, polls_out);
    return cudaGetLastError();
}

}  // namespace smx
