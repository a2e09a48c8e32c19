// Newton-Schulz sign iteration in FP64 on the CUDA cores (the plain form).
//
// Eq. 13 defines sign(A) = A (A^2)^(-1/2).  The iteration
//     X_{k+1} = 1/2 X_k (3 I - X_k^2),   X_0 = (T_j - mu I) / b_j,
// converges to sign(T_j - mu I) when every eigenvalue of X_0 lies in
// (-sqrt 3, 0) u (0, sqrt 3); b_j >= spectral radius guarantees |lambda| <= 1.
// Each step is two products: Y = 3/2 I - 1/2 X X (which also yields the
// residual ||X^2 - I||_F) and X' = X Y.  Stopping rule: after the step whose
// residual is <= tau (the next residual is ~0.75 tau^2).
//
// One CTA per submatrix; FP64 throughput on this part is about 1.2 TFLOP/s
// for the whole GPU, so the kernel is bound by the FP64 pipes and a plain
// shared-memory tiled product with 4x4 register blocking suffices.
#include "smx_finish.cuh"
#include "smx_kernels.h"

namespace smx {

namespace {

constexpr int kTile = 64;
constexpr int kKc = 16;

// C = A B (n x n, row-major, leading dimension ld).  mode 1 writes
// dg I + cf A B (3/2 I - 1/2 A B by default) and returns this thread's share of
// ||A B - I||_F^2; mode 2 writes oscale * A B.
__device__ double gemm_fp64(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C, int n,
                            int ld, int mode, double (*As)[kTile + 1], double (*Bs)[kTile + 1], double oscale = 1.0,
                            double cf = -0.5, double dg = 1.5) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double r2 = 0.0;
    for (int r0 = 0; r0 < n; r0 += kTile) {
        for (int c0 = 0; c0 < n; c0 += kTile) {
            double acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
            for (int k0 = 0; k0 < n; k0 += kKc) {
                for (int e = tid; e < kTile * kKc; e += 256) {
                    const int rr = e / kKc, kk = e - rr * kKc;
                    const int row = r0 + rr, col = k0 + kk;
                    As[kk][rr] = (row < n && col < n) ? A[static_cast<int64_t>(row) * ld + col] : 0.0;
                }
                for (int e = tid; e < kTile * kKc; e += 256) {
                    const int kk = e / kTile, cc = e - kk * kTile;
                    const int row = k0 + kk, col = c0 + cc;
                    Bs[kk][cc] = (row < n && col < n) ? B[static_cast<int64_t>(row) * ld + col] : 0.0;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < kKc; ++kk) {
                    double a[4], b[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = r0 + ty * 4 + i;
                if (row >= n) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int col = c0 + tx * 4 + j;
                    if (col >= n) continue;
                    const double v = acc[i][j];
                    if (mode == 1) {
                        const double dlt = (row == col) ? 1.0 : 0.0;
                        C[static_cast<int64_t>(row) * ld + col] = dg * dlt + cf * v;
                        r2 += (v - dlt) * (v - dlt);
                    } else {
                        C[static_cast<int64_t>(row) * ld + col] = oscale * v;
                    }
                }
            }
        }
    }
    return r2;
}

// The sign iteration of the Eq. 12 block matrix [[0, A], [I, 0]] written per block (the
// coupled Newton-Schulz iteration): T = 3/2 I - 1/2 Z Y, Y <- Y T, Z <- T Z from Y = A (in Yb,
// eigenvalues in (0, 1]) and Z = I (set here); Y -> A^1/2, Z -> A^-1/2.  The residual
// ||Z Y - I||_F comes with the first product; the stopping rule is the sign iteration's.  On
// return Yb and Zb point to the final iterates; the four n x n buffers rotate.  Returns the
// number of steps.
__device__ int coupled_ns(double*& Yb, double*& Zb, double*& Tb, double*& Nb, int n, int ld, int max_iter, double tau,
                          double (*As)[kTile + 1], double (*Bs)[kTile + 1], double* scratch, bool& conv, bool& bad) {
    for (int r = threadIdx.x / 32; r < n; r += 8)
        for (int c = threadIdx.x & 31; c < n; c += 32) Zb[static_cast<int64_t>(r) * ld + c] = r == c ? 1.0 : 0.0;
    __syncthreads();
    int done = 0;
    conv = bad = false;
    for (int it = 0; it < max_iter; ++it) {
        double r2 = gemm_fp64(Zb, Yb, Tb, n, ld, 1, As, Bs);  // T = 3/2 I - 1/2 Z Y
        r2 = block_sum(r2, scratch);
        gemm_fp64(Yb, Tb, Nb, n, ld, 2, As, Bs);  // Y' = Y T
        __syncthreads();
        gemm_fp64(Tb, Zb, Yb, n, ld, 2, As, Bs);  // Z' = T Z into Y's buffer
        __syncthreads();
        double* old_z = Zb;
        Zb = Yb;
        Yb = Nb;
        Nb = old_z;
        done = it + 1;
        if (!isfinite(r2)) { bad = true; break; }
        if (it > 0 && sqrt(r2) <= tau) { conv = true; break; }
    }
    return done;
}

// The finite-temperature Fermi function F = (I + exp(beta A))^-1 = 1/2 (I - tanh(beta A / 2)) of
// a symmetric A, from X = A / g (g >= the spectral radius of A), in products only:
//   B = (beta g / 2) X / 2^k with k such that ||B|| <= 1/16;
//   T = tanh(B) by its odd Taylor series to degree 11 (the next term is below 1e-18 there);
//   k doublings tanh(2x) = 2 tanh(x) / (1 + tanh(x)^2): T <- 2 T (I + T^2)^-1, the inverse by
//   Newton-Schulz V <- V + V (I - M V) from V = 4/3 I - 4/9 M (the first step from 2/3 I in
//   closed form; M = I + T^2 has its eigenvalues in [1, 2], so the residual I - M V starts
//   below 1/9 and squares every step) until ||I - M V||_F <= 1e-15 sqrt(n);
//   F = 1/2 (I - T).
// A doubling at most doubles an error in T, so k doublings cost about 2^k rounding errors
// (k = 11 at beta g = 150).  Five n x n buffers (X first); returns the one holding F and counts
// the products in nprod.
__device__ double* fermi_tanh(double* X, double* B1, double* B2, double* B3, double* B4, int n, int ld, double beta_g,
                              double (*As)[kTile + 1], double (*Bs)[kTile + 1], double* scratch, int& nprod, bool& bad) {
    int k = 0;
    double sc = 0.5 * beta_g;
    while (sc > 1.0 / 16.0 && k < 60) {
        sc *= 0.5;
        ++k;
    }
    // M <- alpha M + d I
    auto axpy_diag = [&](double* M, double alpha, double d) {
        for (int r = threadIdx.x / 32; r < n; r += 8)
            for (int c = threadIdx.x & 31; c < n; c += 32) {
                double& v = M[static_cast<int64_t>(r) * ld + c];
                v = alpha * v + (r == c ? d : 0.0);
            }
        __syncthreads();
    };
    auto prod = [&](const double* A, const double* B, double* C) {
        gemm_fp64(A, B, C, n, ld, 2, As, Bs);
        __syncthreads();
        ++nprod;
    };
    nprod = 0;
    bad = false;
    // T = tanh(B): X <- B in place, Y = B^2, Horner in Y, T = B p(B^2)
    axpy_diag(X, sc, 0.0);
    double* Y = B1;
    double* P = B2;
    double* Q = B3;
    prod(X, X, Y);
    const double c[6] = {1.0, -1.0 / 3.0, 2.0 / 15.0, -17.0 / 315.0, 62.0 / 2835.0, -1382.0 / 155925.0};
    for (int r = threadIdx.x / 32; r < n; r += 8)
        for (int cc = threadIdx.x & 31; cc < n; cc += 32) {
            const int64_t o = static_cast<int64_t>(r) * ld + cc;
            P[o] = c[5] * Y[o] + (r == cc ? c[4] : 0.0);
        }
    __syncthreads();
    for (int i = 3; i >= 0; --i) {
        prod(P, Y, Q);
        axpy_diag(Q, 1.0, c[i]);
        double* t = P; P = Q; Q = t;
    }
    prod(X, P, Q);
    double* T = Q;
    double* fr[4] = {X, Y, P, B4};  // free buffers
    for (int d = 0; d < k && !bad; ++d) {
        double *M = fr[0], *V = fr[1], *R = fr[2], *Vn = fr[3];
        prod(T, T, M);  // M = I + T^2
        axpy_diag(M, 1.0, 1.0);
        for (int r = threadIdx.x / 32; r < n; r += 8)
            for (int cc = threadIdx.x & 31; cc < n; cc += 32) {
                const int64_t o = static_cast<int64_t>(r) * ld + cc;
                V[o] = (r == cc ? 4.0 / 3.0 : 0.0) - 4.0 / 9.0 * M[o];
            }
        __syncthreads();
        for (int m = 0; m < 12; ++m) {
            prod(M, V, R);  // R = I - M V
            double r2 = 0.0;
            for (int r = threadIdx.x / 32; r < n; r += 8)
                for (int cc = threadIdx.x & 31; cc < n; cc += 32) {
                    const int64_t o = static_cast<int64_t>(r) * ld + cc;
                    const double e = (r == cc ? 1.0 : 0.0) - R[o];
                    R[o] = e;
                    r2 += e * e;
                }
            r2 = block_sum(r2, scratch);
            if (!isfinite(r2)) { bad = true; break; }
            if (sqrt(r2) <= 1e-15 * sqrt(static_cast<double>(n))) break;
            prod(V, R, Vn);  // V <- V + V R
            for (int r = threadIdx.x / 32; r < n; r += 8)
                for (int cc = threadIdx.x & 31; cc < n; cc += 32) {
                    const int64_t o = static_cast<int64_t>(r) * ld + cc;
                    Vn[o] += V[o];
                }
            __syncthreads();
            double* t = V; V = Vn; Vn = t;
        }
        prod(T, V, R);  // T <- 2 T V
        axpy_diag(R, 2.0, 0.0);
        double* oldT = T;
        T = R;
        fr[0] = oldT;
        fr[1] = M;
        fr[2] = V;
        fr[3] = Vn;
    }
    axpy_diag(T, -0.5, 0.5);  // F = 1/2 (I - T)
    return T;
}

// Gershgorin interval (lo, hi) of an n x n matrix held row by row.
__device__ double2 gershgorin_interval(const double* M, int n, int ld, double* scratch) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    double lo = INFINITY, hi = -INFINITY;
    for (int r = warp; r < n; r += 8) {
        double acc = 0.0;
        for (int c = lane; c < n; c += 32) acc += c == r ? 0.0 : fabs(M[static_cast<int64_t>(r) * ld + c]);
        acc = warp_sum(acc);
        const double d = M[static_cast<int64_t>(r) * ld + r];
        lo = fmin(lo, d - acc);
        hi = fmax(hi, d + acc);
    }
    lo = -warp_max(-lo);
    hi = warp_max(hi);
    if (lane == 0) {
        scratch[warp] = lo;
        scratch[8 + warp] = hi;
    }
    __syncthreads();
    double2 out = make_double2(INFINITY, -INFINITY);
    for (int w = 0; w < 8; ++w) {
        out.x = fmin(out.x, scratch[w]);
        out.y = fmax(out.y, scratch[8 + w]);
    }
    __syncthreads();
    return out;
}

// C[i][q] = sum_k A[i][k] Bt[q][k] for i < n, q < m: a product with a thin right factor given
// by its rows (Bt = the transposed factor, m rows of length n, leading dimension ldb), C with
// leading dimension m.  mode 1 writes Bt[q][i] - C[i][q] instead; scale multiplies the result.
// A warp per row i, eight columns q at a time.
__device__ void thin_product(const double* __restrict__ A, int lda, const double* __restrict__ Bt, int ldb, int n, int m,
                             double* __restrict__ C, int mode, double scale) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    for (int i = warp; i < n; i += 8) {
        const double* ai = A + static_cast<int64_t>(i) * lda;
        for (int q0 = 0; q0 < m; q0 += 8) {
            double acc[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) acc[t] = 0.0;
            for (int k = lane; k < n; k += 32) {
                const double x = ai[k];
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (q0 + t < m) acc[t] = fma(x, Bt[static_cast<int64_t>(q0 + t) * ldb + k], acc[t]);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const double v = warp_sum(acc[t]);
                if (lane == 0 && q0 + t < m) {
                    const double r = mode == 1 ? Bt[static_cast<int64_t>(q0 + t) * ldb + i] - v : v;
                    C[static_cast<int64_t>(i) * m + q0 + t] = scale * r;
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(256) k_ns_fp64(NsFp64Args a) {
    __shared__ double As[kKc][kTile + 1];
    __shared__ double Bs[kKc][kTile + 1];
    __shared__ double scratch[32];
    extern __shared__ int ls_smem[];
    if (a.skip && *a.skip) return;
    const SubDesc s = a.subs[blockIdx.x];
    const int n = s.n, ld = s.ld;
    double* X = a.T + s.t_off;
    double* Y = a.W1 + s.t_off;
    double* Z = a.W2 + s.t_off;
    if (a.Mc) {
        // non-orthogonal form: the sign iteration runs on M_j - mu I with M_j = L_j A_H L_j
        // (L_j = A_S^-1/2, from the setup kernel); its Gershgorin bound starts the iteration
        const double* M = a.Mc + s.t_off;
        const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
        double rmax = 0.0;
        for (int r = warp; r < n; r += 8) {
            double acc = 0.0;
            for (int c = lane; c < n; c += 32) {
                const double v = M[static_cast<int64_t>(r) * ld + c] - (r == c ? a.mu : 0.0);
                X[static_cast<int64_t>(r) * ld + c] = v;
                acc += fabs(v);
            }
            rmax = fmax(rmax, warp_sum(acc));
        }
        rmax = warp_max(rmax);
        if (lane == 0) scratch[warp] = rmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int w = 0; w < 8; ++w) b = fmax(b, scratch[w]);
            b = b > 0.0 ? b : 1.0;
            a.bound[blockIdx.x] = b;
            a.gersh[blockIdx.x] = b;
        }
        __syncthreads();
    }
    if (a.finish_iters > 0) {
        // FP64 finishing steps after a low-precision bulk phase: X (in T) is that phase's last
        // iterate; plain Newton-Schulz steps in FP64, then the scatter of the owner columns
        bool bad = false;
        for (int it = 0; it < a.finish_iters; ++it) {
            double r2 = gemm_fp64(X, X, Y, n, ld, 1, As, Bs);  // Y = 3/2 I - 1/2 X^2
            r2 = block_sum(r2, scratch);
            gemm_fp64(X, Y, Z, n, ld, 2, As, Bs);
            __syncthreads();
            double* tmp = X; X = Z; Z = tmp;
            if (!isfinite(r2)) bad = true;
        }
        if (threadIdx.x == 0) {
            a.iters[s.col] += a.finish_iters;
            atomicAdd(a.work_n3, static_cast<unsigned long long>(n) * n * n * a.finish_iters);
            if (bad) atomicCAS(a.status, kOk, kErrNonfinite);
        }
        const double* Xf = X;
        auto xrow = [&](int q, int i) -> double { return Xf[static_cast<int64_t>(s.own + q) * ld + i]; };
        finish_column(s, a.pv, a.H, a.D, a.partial, xrow, ls_smem, scratch);
        return;
    }
    const double inv_b = 1.0 / a.bound[blockIdx.x];
    // learned bound: the predicted smallest |eigenvalue| of X0 = (T_j - mu I) / b_j (negative:
    // no prediction), and the lower end the scaled schedule assumes (1 = plain steps)
    const double dhat = a.pred ? a.pred[2 * blockIdx.x + 1] * a.gersh[blockIdx.x] * inv_b : -1.0;
    double lsch = 1.0, acur = 1.0;
    for (int r = threadIdx.x / 32; r < n; r += 8)
        for (int c = threadIdx.x & 31; c < n; c += 32) X[static_cast<int64_t>(r) * ld + c] *= inv_b;
    __syncthreads();

    int done = 0;
    bool conv = false, bad = false;
    if (a.function == kFnFermi) {
        // the Fermi function of A = T_j - mu I (now A / b in X, b its Gershgorin bound)
        int nprod = 0;
        bool bad = false;
        const double* F = fermi_tanh(X, Y, Z, a.W3 + s.t_off, a.W4 + s.t_off, n, ld,
                                     a.beta * a.bound[blockIdx.x], As, Bs, scratch, nprod, bad);
        if (threadIdx.x == 0) {
            a.iters[s.col] = nprod;
            atomicAdd(a.work_n3, static_cast<unsigned long long>(n) * n * n * nprod);
            if (bad) atomicCAS(a.status, kOk, kErrNonfinite);
        }
        auto frow = [&](int q, int i) -> double { return F[static_cast<int64_t>(s.own + q) * ld + i]; };
        finish_column(s, a.pv, a.H, a.D, a.partial, frow, ls_smem, scratch, false);
        return;
    }
    if (a.function != kFnDensity) {
        // f = A^-1/2 or A^1/2 for a symmetric positive definite A = T_j - mu I (now A/b in X)
        double* Yb = X;
        double* Zb = Y;
        double* Tb = Z;
        double* Nb = a.W3 + s.t_off;
        done = coupled_ns(Yb, Zb, Tb, Nb, n, ld, a.max_iter, a.tau, As, Bs, scratch, conv, bad);
        if (threadIdx.x == 0) {
            a.iters[s.col] = done;
            atomicAdd(a.work_n3, static_cast<unsigned long long>(n) * n * n * done);
            if (bad) atomicCAS(a.status, kOk, kErrNonfinite);
            else if (!conv) atomicCAS(a.status, kOk, kErrNoconv);
        }
        if (a.function == kFnInv) {
            // A^-1 = (A^-1/2)^2 = Z Z / b: its owner columns Z Z[:, own] / b (Z symmetric, so
            // the thin factor is given by rows own ..), into the free buffer T
            thin_product(Zb, ld, Zb + static_cast<int64_t>(s.own) * ld, ld, n, s.bown, Tb, 0,
                         1.0 / a.bound[blockIdx.x]);
            const double* U = Tb;
            auto irow = [&](int q, int i) -> double { return U[static_cast<int64_t>(i) * s.bown + q]; };
            finish_column(s, a.pv, a.H, a.D, a.partial, irow, ls_smem, scratch, false);
            return;
        }
        // A^-1/2 = Z / sqrt(b), A^1/2 = sqrt(b) Y (both symmetric: row own + q is column own + q)
        const double* F = a.function == kFnInvSqrt ? Zb : Yb;
        const double fs = a.function == kFnInvSqrt ? 1.0 / sqrt(a.bound[blockIdx.x]) : sqrt(a.bound[blockIdx.x]);
        auto frow = [&](int q, int i) -> double { return fs * F[static_cast<int64_t>(s.own + q) * ld + i]; };
        finish_column(s, a.pv, a.H, a.D, a.partial, frow, ls_smem, scratch, false);
        return;
    }
    for (int it = 0; it < a.max_iter; ++it) {
        double r2 = 1.0, oscale = 1.0;
        if (it == 0) {
            // a-posteriori scaling (as in the tensor-core kernel): with Y = X0^2,
            // rho(X0)^2 = rho(Y) <= rho(|Y|) <= max_r (|Y| w)_r / w_r for any
            // positive w (Collatz-Wielandt): w = 1 (the max row sum) and two
            // power steps of |Y| from it; continue from X0' = (1.2/s) X0
            gemm_fp64(X, X, Y, n, ld, 2, As, Bs);
            __syncthreads();
            double* wv = Z;  // the output buffer of this iteration is free until the second product
            double* wn = Z + n;
            const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
            auto block_max2 = [&](double x, double y) -> double2 {
                x = warp_max(x);
                y = warp_max(y);
                if (lane == 0) {
                    scratch[warp] = x;
                    scratch[8 + warp] = y;
                }
                __syncthreads();
                double2 m = make_double2(0.0, 0.0);
                for (int w = 0; w < 8; ++w) {
                    m.x = fmax(m.x, scratch[w]);
                    m.y = fmax(m.y, scratch[8 + w]);
                }
                __syncthreads();
                return m;
            };
            double rmax = 0.0;
            for (int r = warp; r < n; r += 8) {
                double acc = 0.0;
                for (int c = lane; c < n; c += 32) acc += fabs(Y[static_cast<int64_t>(r) * ld + c]);
                acc = warp_sum(acc);
                if (lane == 0) wv[r] = acc;
                rmax = fmax(rmax, acc);
            }
            rmax = block_max2(rmax, 0.0).x;
            double best = rmax, wtop = rmax;
            for (int pass = 0; pass < 2 && best > 0.0; ++pass) {
                for (int c = threadIdx.x; c < n; c += blockDim.x) wv[c] = fmax(wv[c], 1e-30 * wtop);
                __syncthreads();
                double q = 0.0, wm = 0.0;
                for (int r = warp; r < n; r += 8) {
                    double acc = 0.0;
                    for (int c = lane; c < n; c += 32) acc = fma(fabs(Y[static_cast<int64_t>(r) * ld + c]), wv[c], acc);
                    acc = warp_sum(acc);
                    if (lane == 0) wn[r] = acc;
                    q = fmax(q, acc / wv[r]);
                    wm = fmax(wm, acc);
                }
                const double2 m2 = block_max2(q, wm);
                best = fmin(best, m2.x);
                if (!(m2.y > 0.0)) break;
                for (int c = threadIdx.x; c < n; c += blockDim.x) wv[c] = wn[c] / m2.y;
                wtop = 1.0;
            }
            const double smax = sqrt(best * (1.0 + 1e-12));
            double scale = smax > 0.0 ? 1.2 / smax : 1.0;
            if (a.use_model && smax > 0.0) {  // same rule as the tensor-core kernel
                const bool gap = dhat > 0.0;
                if (gap ? dhat <= smax : smax <= 1.7) {
                    if (gap) {  // the scaled schedule from l0 = dhat / s
                        const double l0 = dhat / smax;
                        const double a0 = ns_scale(l0);
                        scale = a0 / smax;
                        lsch = ns_next_lower(a0, l0);
                    } else {
                        scale = fmax(1.0, scale);
                    }
                } else if (threadIdx.x == 0) {
                    atomicAdd(a.fallbacks, 1);
                }
            }
            const double sc2 = scale * scale;
            for (int r = threadIdx.x / 32; r < n; r += 8)
                for (int c = threadIdx.x & 31; c < n; c += 32) {
                    double& y = Y[static_cast<int64_t>(r) * ld + c];
                    y = (r == c ? 1.5 : 0.0) - 0.5 * sc2 * y;
                }
            if (threadIdx.x == 0) {
                // feature of the next snapshot: the Gershgorin bound of A^2, over G
                a.sq_ratio[blockIdx.x] = static_cast<float>(sqrt(rmax) * a.bound[blockIdx.x] / a.gersh[blockIdx.x]);
                a.bound[blockIdx.x] = a.bound[blockIdx.x] / scale;
            }
            __syncthreads();
            oscale = scale;
        } else {
            // Y = a (3/2 I - a^2/2 X^2) on the scaled schedule (a = 1: a plain step)
            double cf = -0.5, dg = 1.5;
            acur = 1.0;
            if (lsch < 1.0) {
                const double f = ns_scale(lsch);
                cf = -0.5 * f * f * f;
                dg = 1.5 * f;
                lsch = ns_next_lower(f, lsch);
                acur = f;
            }
            r2 = gemm_fp64(X, X, Y, n, ld, 1, As, Bs, 1.0, cf, dg);
            r2 = block_sum(r2, scratch);
        }
        gemm_fp64(X, Y, Z, n, ld, 2, As, Bs, oscale);
        __syncthreads();
        double* tmp = X; X = Z; Z = tmp;
        done = it + 1;
        if (!isfinite(r2)) { bad = true; break; }
        if (it > 0 && sqrt(r2) <= a.tau) {
            // stop after this step unless it was a scaled step whose factor moves converged
            // eigenvalues off 1 (p(a) ~ 1 - 1.5 (a - 1)^2): then plain steps from here
            if (acur - 1.0 <= 2e-6) { conv = true; break; }
            lsch = 1.0;
        }
    }
    if (threadIdx.x == 0) {
        a.iters[s.col] = done;
        atomicAdd(a.work_n3, static_cast<unsigned long long>(n) * n * n * done);
        if (bad) atomicCAS(a.status, kOk, kErrNonfinite);
        else if (!conv) atomicCAS(a.status, kOk, kErrNoconv);
    }
    const double* Xf = X;
    if (a.Mc) {
        // P_j[:, own] = 1/2 L (I - X) L[:, own] = 1/2 L (W - X W), W = L[:, own] (rows own..
        // of the symmetric L): Eq. 14 with sign(A_S^-1 A_H - mu I) = L sign(M - mu I) L^-1
        // and A_S^-1 = L L.  Two thin products into the free buffers Y (U) and Z (P_own).
        const double* L = a.Lc + s.t_off;
        double* U = Y;
        double* Pown = Z;
        thin_product(Xf, ld, L + static_cast<int64_t>(s.own) * ld, ld, n, s.bown, U, 1, 1.0);
        // second factor given by rows: U^T (bown x n) is U read with stride bown
        const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
        for (int i = warp; i < n; i += 8) {
            const double* li = L + static_cast<int64_t>(i) * ld;
            for (int q0 = 0; q0 < s.bown; q0 += 8) {
                double acc[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[t] = 0.0;
                for (int k = lane; k < n; k += 32) {
                    const double x = li[k];
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        if (q0 + t < s.bown) acc[t] = fma(x, U[static_cast<int64_t>(k) * s.bown + q0 + t], acc[t]);
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const double v = warp_sum(acc[t]);
                    if (lane == 0 && q0 + t < s.bown) Pown[static_cast<int64_t>(i) * s.bown + q0 + t] = 0.5 * v;
                }
            }
        }
        __syncthreads();
        auto prow = [&](int q, int i) -> double { return Pown[static_cast<int64_t>(i) * s.bown + q]; };
        finish_column(s, a.pv, a.H, a.D, a.partial, prow, ls_smem, scratch, false, a.Sv);
        return;
    }
    auto xrow = [&](int q, int i) -> double { return Xf[static_cast<int64_t>(s.own + q) * ld + i]; };
    finish_column(s, a.pv, a.H, a.D, a.partial, xrow, ls_smem, scratch);
}

// Setup of the non-orthogonal form for one (H, S) pair, a CTA per submatrix: from A_S (in Lc)
// and A_H (in Mc), both gathered without shift, L = A_S^-1/2 by the coupled iteration (into
// Lc) and M = L A_H L, symmetrised (into Mc), and the Gershgorin interval of M.
__global__ void __launch_bounds__(256) k_nonorth_setup(NonorthSetupArgs a) {
    __shared__ double As[kKc][kTile + 1];
    __shared__ double Bs[kKc][kTile + 1];
    __shared__ double scratch[32];
    const SubDesc s = a.subs[blockIdx.x];
    const int n = s.n, ld = s.ld;
    double* Lc = a.Lc + s.t_off;
    double* Mc = a.Mc + s.t_off;
    double* Yb = a.T + s.t_off;
    double* Zb = a.W1 + s.t_off;
    double* Tb = a.W2 + s.t_off;
    double* Nb = a.W3 + s.t_off;
    const double b = a.bound_s[blockIdx.x];
    const double inv_b = b > 0.0 ? 1.0 / b : 0.0;
    for (int r = threadIdx.x / 32; r < n; r += 8)
        for (int c = threadIdx.x & 31; c < n; c += 32)
            Yb[static_cast<int64_t>(r) * ld + c] = Lc[static_cast<int64_t>(r) * ld + c] * inv_b;
    __syncthreads();
    bool conv = false, bad = false;
    const int done = coupled_ns(Yb, Zb, Tb, Nb, n, ld, a.max_iter, a.tau, As, Bs, scratch, conv, bad);
    if (threadIdx.x == 0) {
        a.iters[s.col] = done;
        if (bad || !(b > 0.0)) atomicCAS(a.status, kOk, kErrNonfinite);
        else if (!conv) atomicCAS(a.status, kOk, kErrNoconv);
    }
    const double ls = b > 0.0 ? 1.0 / sqrt(b) : 0.0;  // A_S^-1/2 = Z / sqrt(b)
    for (int r = threadIdx.x / 32; r < n; r += 8)
        for (int c = threadIdx.x & 31; c < n; c += 32)
            Lc[static_cast<int64_t>(r) * ld + c] = ls * Zb[static_cast<int64_t>(r) * ld + c];
    __syncthreads();
    gemm_fp64(Mc, Lc, Tb, n, ld, 2, As, Bs);  // A_H L
    __syncthreads();
    gemm_fp64(Lc, Tb, Nb, n, ld, 2, As, Bs);  // L A_H L
    __syncthreads();
    for (int r = threadIdx.x / 32; r < n; r += 8)
        for (int c = threadIdx.x & 31; c < n; c += 32)
            Mc[static_cast<int64_t>(r) * ld + c] =
                0.5 * (Nb[static_cast<int64_t>(r) * ld + c] + Nb[static_cast<int64_t>(c) * ld + r]);
    __syncthreads();
    const double2 g = gershgorin_interval(Mc, n, ld, scratch);
    if (threadIdx.x == 0) {
        a.lohi[2 * blockIdx.x] = g.x;
        a.lohi[2 * blockIdx.x + 1] = g.y;
    }
}

cudaError_t launch_ns_fp64(const NsFp64Args& a, int max_nblk, cudaStream_t st) {
    const size_t smem = sizeof(int) * (static_cast<size_t>(max_nblk) + 1);
    k_ns_fp64<<<a.n_subs, 256, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nonorth_setup(const NonorthSetupArgs& a, cudaStream_t st) {
    k_nonorth_setup<<<a.n_subs, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace smx

// ---------------------------------------------------------------------------
// Allocation-free dense entry point (no counterpart in the paper).
//
// Some callers cannot allocate device memory when they need a result:
// plug-ins inside a host framework whose caching allocator already owns the
// whole device pool (a cudaMalloc of their own would fail or fragment it),
// and latency-critical loops that must never enter the driver's allocator
// (cudaMalloc/cudaFree can synchronise the device and take milliseconds).
// smx_dense_density_noalloc serves them: it takes caller-owned input and
// output buffers and keeps its Newton-Schulz work matrices in the fixed
// device array below, which every GPU that loads this library holds until the
// process exits.  The call itself synchronises its stream to return the status.
// ---------------------------------------------------------------------------

#include <cmath>
#include <mutex>

#include "smx.h"

namespace smx {

namespace {
constexpr int kNoAllocMaxN = 256;                          // largest n accepted
constexpr int64_t kNoAllocMat = int64_t(kNoAllocMaxN) * kNoAllocMaxN;
constexpr int kNoAllocMaxDevices = 64;
}  // namespace

// X, Y, Z work matrices (n x n each, leading dimension n) followed by a small
// header: [0] status, [1] iterations.  3 * 256^2 + 4 doubles, about 1.5 MiB.
static __device__ __align__(256) double g_noalloc_scratch[3 * kNoAllocMat + 4];

// One CTA: D = 1/2 (I - sign(H - mu I)) of a dense symmetric H by the FP64
// Newton-Schulz iteration of k_ns_fp64, with the Gershgorin bound for X0.
__global__ void __launch_bounds__(256) k_dense_density_noalloc(const double* __restrict__ H, int n, double mu,
                                                               double* __restrict__ Dout, double* scratch,
                                                               double tau, int max_iter) {
    __shared__ double As[kKc][kTile + 1];
    __shared__ double Bs[kKc][kTile + 1];
    __shared__ double red[32];
    double* X = scratch;
    double* Y = scratch + kNoAllocMat;
    double* Z = scratch + 2 * kNoAllocMat;
    int* hdr = reinterpret_cast<int*>(scratch + 3 * kNoAllocMat);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // every call overwrites the work matrices in full; nothing is carried over

    // Gershgorin bound b = max_r sum_c |H_rc - mu delta_rc| (>= spectral radius)
    double m = 0.0;
    for (int r = warp; r < n; r += 8) {
        double acc = 0.0;
        for (int c = lane; c < n; c += 32) acc += fabs(H[static_cast<int64_t>(r) * n + c] - (r == c ? mu : 0.0));
        m = fmax(m, warp_sum(acc));
    }
    if (lane == 0) red[warp] = m;
    __syncthreads();
    double b = 0.0;
    for (int w = 0; w < 8; ++w) b = fmax(b, red[w]);
    if (b == 0.0) b = 1.0;
    __syncthreads();
    const double inv_b = 1.0 / b;
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(n) * n; e += blockDim.x) {
        const int r = static_cast<int>(e / n), c = static_cast<int>(e - static_cast<int64_t>(r) * n);
        X[e] = (H[e] - (r == c ? mu : 0.0)) * inv_b;
    }
    __syncthreads();

    int done = 0;
    bool conv = false, bad = false;
    for (int it = 0; it < max_iter; ++it) {
        double r2 = gemm_fp64(X, X, Y, n, n, 1, As, Bs);
        r2 = block_sum(r2, red);
        gemm_fp64(X, Y, Z, n, n, 2, As, Bs);
        __syncthreads();
        double* t = X; X = Z; Z = t;
        done = it + 1;
        if (!isfinite(r2)) { bad = true; break; }
        if (sqrt(r2) <= tau) { conv = true; break; }
    }
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(n) * n; e += blockDim.x) {
        const int r = static_cast<int>(e / n), c = static_cast<int>(e - static_cast<int64_t>(r) * n);
        Dout[e] = 0.5 * ((r == c ? 1.0 : 0.0) - X[e]);
    }
    if (threadIdx.x == 0) {
        hdr[0] = bad ? kErrNonfinite : (conv ? kOk : kErrNoconv);
        hdr[1] = done;
    }
}

}  // namespace smx

namespace {
std::mutex g_noalloc_mutex;
// per device: the array's device address and the context it was looked up in
double* g_noalloc_ptr[smx::kNoAllocMaxDevices] = {};
CUcontext g_noalloc_ctx[smx::kNoAllocMaxDevices] = {};

// The current driver context, through the runtime's driver entry point (no link to libcuda).
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(p);
    });
    CUcontext c = nullptr;
    if (fn) fn(&c);
    return c;
}
}  // namespace

extern "C" smx_status smx_dense_density_noalloc(const double* h_dev, int32_t n, double mu, double* d_dev,
                                                void* cuda_stream) {
    if (!h_dev || !d_dev || n < 1 || n > smx::kNoAllocMaxN || !std::isfinite(mu)) return SMX_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SMX_ERR_CUDA;
    if (dev < 0 || dev >= smx::kNoAllocMaxDevices) return SMX_ERR_UNSUPPORTED;
    double* scratch = nullptr;
    {
        // set-up once per device, with that device current: the host-side name
        // of a __device__ array is not a device address, so look the address up.
        // A device reset (cudaDeviceReset) replaces the context and reloads the
        // module, so the lookup is repeated when the current context changed.
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        const CUcontext cur = current_context();
        if (!g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != cur) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, smx::g_noalloc_scratch) != cudaSuccess || !p) return SMX_ERR_CUDA;
            g_noalloc_ptr[dev] = static_cast<double*>(p);
            g_noalloc_ctx[dev] = cur;
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    smx::k_dense_density_noalloc<<<1, 256, 0, st>>>(h_dev, n, mu, d_dev, scratch, 1e-7, 100);
    if (cudaGetLastError() != cudaSuccess) return SMX_ERR_CUDA;
    int hdr[2] = {0, 0};
    if (cudaMemcpyAsync(hdr, scratch + 3 * smx::kNoAllocMat, sizeof(hdr), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SMX_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SMX_ERR_CUDA;
    return static_cast<smx_status>(hdr[0]);
}
