// Learned spectral bound: Lanczos labels and MLP training (the features and the
// inference run inside the gather kernel, k_pattern.cu).
//
// The network predicts, per submatrix A = T_j - mu I, the ratios rho/G and
// delta/G (spectral radius and smallest |eigenvalue| over the Gershgorin
// bound G) from nine cheap features; the Newton-Schulz start is then scaled
// with the predicted radius and checked against the guaranteed bound that the
// first product yields (see the Newton-Schulz kernels).  The paper's Section 4
// names learning on the fly (a network trained on data the simulation itself
// produces) as a direction; this is that reading for the sign iteration.
//
// Conventions shared with the FP64 oracle of the model (written separately):
//   features f0..f8 (all over G except f6 and f8):
//     ||A||_F/sqrt(n), max|A_rr|, mean|A_rr|, std(A_rr), max R_r, mean R_r,
//     n/256, mean A_rr, previous-step ratio;  R_r = sum_{c != r} |A_rc|
//   network F=9 -> 64 (tanh) -> 64 (tanh) -> 2, loss 1/(2m) sum (y - t)^2
//   flat parameters: W1 (64 x 9), b1, W2 (64 x 64), b2, W3 (2 x 64), b3
#include "smx_kernels.h"

namespace smx {

namespace {

constexpr int kF = kModelFeatures, kH = kModelHidden, kO = 2;

constexpr int kChunk = 64;  // samples per gradient block

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

// ---------------------------------------------------------------------------
// Lanczos labels (one CTA per submatrix): rho from A, delta from A^2
// ---------------------------------------------------------------------------
namespace {

// number of eigenvalues below x of the symmetric tridiagonal (a, b), b[0] unused
__device__ int sturm_count(const double* a, const double* b, int k, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
        const double bb = i ? b[i] * b[i] : 0.0;
        q = (a[i] - x) - (i ? bb / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// i-th smallest eigenvalue (0-based) of the tridiagonal by bisection
__device__ double tridiag_eig(const double* a, const double* b, int k, int i) {
    double lo = 1e300, hi = -1e300;
    for (int j = 0; j < k; ++j) {
        const double r = (j ? fabs(b[j]) : 0.0) + (j + 1 < k ? fabs(b[j + 1]) : 0.0);
        lo = fmin(lo, a[j] - r);
        hi = fmax(hi, a[j] + r);
    }
    for (int it = 0; it < 100; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, k, mid) > i) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

template <class R>
__global__ void __launch_bounds__(256) k_lanczos(const SubDesc* __restrict__ subs, const R* __restrict__ T, int ksteps,
                                                 float* __restrict__ labels) {
    extern __shared__ float lz[];  // 4 vectors of max_n
    __shared__ double alpha[kMaxLanczos], beta[kMaxLanczos + 1];
    __shared__ float red[8];
    __shared__ float gmax_s;
    const SubDesc s = subs[blockIdx.x];
    const R* t = T + s.t_off;
    const int n = s.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* v = lz;
    float* w = lz + n;
    float* vp = lz + 2 * n;
    float* u = lz + 3 * n;

    auto block_sum_f = [&](float x) -> float {
        x = warp_sum_f(x);
        __syncthreads();
        if (lane == 0) red[warp] = x;
        __syncthreads();
        float r = 0.f;
        for (int i = 0; i < 8; ++i) r += red[i];
        __syncthreads();
        return r;
    };
    // y = A x (a warp per row)
    auto matvec = [&](const float* x, float* y) {
        for (int r = warp; r < n; r += 8) {
            float acc = 0.f;
            for (int c = lane; c < n; c += 32) acc = fmaf(static_cast<float>(t[static_cast<int64_t>(r) * s.ld + c]), x[c], acc);
            acc = warp_sum_f(acc);
            if (lane == 0) y[r] = acc;
        }
        __syncthreads();
    };
    // Gershgorin bound G
    {
        float g = 0.f;
        for (int r = warp; r < n; r += 8) {
            float acc = 0.f;
            for (int c = lane; c < n; c += 32) acc += fabsf(static_cast<float>(t[static_cast<int64_t>(r) * s.ld + c]));
            g = fmaxf(g, warp_sum_f(acc));
        }
        if (lane == 0) red[warp] = g;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int i = 0; i < 8; ++i) m = fmaxf(m, red[i]);
            gmax_s = m;
        }
        __syncthreads();
    }
    const int K = min(ksteps, min(n, kMaxLanczos));
    double lam_lo = 0.0, lam_hi = 0.0, sq_lo = 0.0;
    for (int pass = 0; pass < 2; ++pass) {  // pass 0: A, pass 1: A^2
        // deterministic start vector with all components non-zero
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            v[i] = 1.0f + 0.5f * __sinf(1.7f * static_cast<float>(i) + 0.3f * pass);
            vp[i] = 0.f;
        }
        __syncthreads();
        float nv = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) nv += v[i] * v[i];
        nv = sqrtf(block_sum_f(nv));
        for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] /= nv;
        __syncthreads();
        float bprev = 0.f;
        int k = 0;
        for (; k < K; ++k) {
            if (pass == 0) matvec(v, w);
            else { matvec(v, u); matvec(u, w); }
            float al = 0.f;
            for (int i = threadIdx.x; i < n; i += blockDim.x) al += v[i] * w[i];
            al = block_sum_f(al);
            float nw = 0.f;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const float x = w[i] - al * v[i] - bprev * vp[i];
                w[i] = x;
                nw += x * x;
            }
            nw = sqrtf(block_sum_f(nw));
            if (threadIdx.x == 0) { alpha[k] = al; beta[k + 1] = nw; }
            if (nw <= 1e-12f * gmax_s || k + 1 == K) { ++k; break; }
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                vp[i] = v[i];
                v[i] = w[i] / nw;
            }
            bprev = nw;
            __syncthreads();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (pass == 0) {
                lam_lo = tridiag_eig(alpha, beta, k, 0);
                lam_hi = tridiag_eig(alpha, beta, k, k - 1);
            } else {
                sq_lo = tridiag_eig(alpha, beta, k, 0);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double G = gmax_s > 0.f ? gmax_s : 1.f;
        labels[2 * blockIdx.x] = static_cast<float>(fmax(fabs(lam_lo), fabs(lam_hi)) / G);
        labels[2 * blockIdx.x + 1] = static_cast<float>(sqrt(fmax(sq_lo, 0.0)) / G);
    }
}

// ---------------------------------------------------------------------------
// MLP
// ---------------------------------------------------------------------------

// Forward + backward for samples [blockIdx.x * 64, +64): per-block gradient sums
// (sum over the block's samples, in sample order) and half the squared residual.
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ params, const float* __restrict__ X,
                                                  const float* __restrict__ Tg, int m, float* __restrict__ partial,
                                                  float* __restrict__ partial_loss) {
    extern __shared__ float sm[];
    float* p = sm;                              // kModelParams
    float* xs = p + kModelParams;               // [64][kF]
    float* h1 = xs + kChunk * kF;               // [64][64]
    float* h2 = h1 + kChunk * kH;               // [64][64]
    float* d1 = h2 + kChunk * kH;               // [64][64]  dL/d(pre-activation 1)
    float* d2 = d1 + kChunk * kH;               // [64][64]
    float* dy = d2 + kChunk * kH;               // [64][2]
    float* ls = dy + kChunk * kO;               // [64] half squared residual per sample
    const int s0 = blockIdx.x * kChunk;
    const int cnt = min(kChunk, m - s0);
    for (int i = threadIdx.x; i < kModelParams; i += blockDim.x) p[i] = params[i];
    for (int i = threadIdx.x; i < kChunk * kF; i += blockDim.x) {
        const int sidx = i / kF;
        xs[i] = sidx < cnt ? X[static_cast<int64_t>(s0) * kF + i] : 0.f;
    }
    __syncthreads();
    // layer 1 and 2 forward: thread handles (sample, unit) pairs
    for (int e = threadIdx.x; e < kChunk * kH; e += blockDim.x) {
        const int sidx = e / kH, i = e - sidx * kH;
        float a = p[kOffB1 + i];
        for (int k = 0; k < kF; ++k) a = fmaf(p[i * kF + k], xs[sidx * kF + k], a);
        h1[e] = tanhf(a);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kChunk * kH; e += blockDim.x) {
        const int sidx = e / kH, i = e - sidx * kH;
        float a = p[kOffB2 + i];
        for (int k = 0; k < kH; ++k) a = fmaf(p[kOffW2 + i * kH + k], h1[sidx * kH + k], a);
        h2[e] = tanhf(a);
    }
    __syncthreads();
    if (threadIdx.x < kChunk) {
        const int sidx = threadIdx.x;
        float l = 0.f;
        for (int o = 0; o < kO; ++o) {
            float y = p[kOffB3 + o];
            for (int k = 0; k < kH; ++k) y = fmaf(p[kOffW3 + o * kH + k], h2[sidx * kH + k], y);
            const float r = sidx < cnt ? y - Tg[2 * static_cast<int64_t>(s0 + sidx) + o] : 0.f;
            dy[sidx * kO + o] = r;
            l = fmaf(r, r, l);
        }
        ls[sidx] = 0.5f * l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // summed in sample order
        float l = 0.f;
        for (int i = 0; i < kChunk; ++i) l += ls[i];
        partial_loss[blockIdx.x] = l;
    }
    // backward: d2 = (dy W3) * (1 - h2^2); d1 = (d2 W2) * (1 - h1^2)
    for (int e = threadIdx.x; e < kChunk * kH; e += blockDim.x) {
        const int sidx = e / kH, i = e - sidx * kH;
        const float g = dy[sidx * kO] * p[kOffW3 + i] + dy[sidx * kO + 1] * p[kOffW3 + kH + i];
        d2[e] = g * (1.f - h2[e] * h2[e]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kChunk * kH; e += blockDim.x) {
        const int sidx = e / kH, k = e - sidx * kH;
        float g = 0.f;
        for (int i = 0; i < kH; ++i) g = fmaf(d2[sidx * kH + i], p[kOffW2 + i * kH + k], g);
        d1[e] = g * (1.f - h1[e] * h1[e]);
    }
    __syncthreads();
    // parameter gradients, each a sum over the block's samples in order
    float* gout = partial + static_cast<int64_t>(blockIdx.x) * kModelParams;
    for (int q = threadIdx.x; q < kModelParams; q += blockDim.x) {
        float g = 0.f;
        if (q < kOffB1) {
            const int i = q / kF, k = q - i * kF;
            for (int sidx = 0; sidx < kChunk; ++sidx) g = fmaf(d1[sidx * kH + i], xs[sidx * kF + k], g);
        } else if (q < kOffW2) {
            const int i = q - kOffB1;
            for (int sidx = 0; sidx < kChunk; ++sidx) g += d1[sidx * kH + i];
        } else if (q < kOffB2) {
            const int i = (q - kOffW2) / kH, k = (q - kOffW2) - i * kH;
            for (int sidx = 0; sidx < kChunk; ++sidx) g = fmaf(d2[sidx * kH + i], h1[sidx * kH + k], g);
        } else if (q < kOffW3) {
            const int i = q - kOffB2;
            for (int sidx = 0; sidx < kChunk; ++sidx) g += d2[sidx * kH + i];
        } else if (q < kOffB3) {
            const int o = (q - kOffW3) / kH, k = (q - kOffW3) - o * kH;
            for (int sidx = 0; sidx < kChunk; ++sidx) g = fmaf(dy[sidx * kO + o], h2[sidx * kH + k], g);
        } else {
            const int o = q - kOffB3;
            for (int sidx = 0; sidx < kChunk; ++sidx) g += dy[sidx * kO + o];
        }
        gout[q] = g;
    }
}

// Ordered sum of the block partials, divided by m; optional gradient output and
// optional Adam update (step t >= 1, lr > 0).
__global__ void k_mlp_reduce_adam(const float* __restrict__ partial, const float* __restrict__ partial_loss,
                                  int nblocks, int m, float* __restrict__ params, float* __restrict__ mst,
                                  float* __restrict__ vst, int t, float lr, float* __restrict__ grad_out,
                                  float* __restrict__ loss_out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const float inv_m = 1.f / static_cast<float>(m);
    if (q == 0 && loss_out) {
        float l = 0.f;
        for (int b = 0; b < nblocks; ++b) l += partial_loss[b];
        *loss_out = l * inv_m;
    }
    if (q >= kModelParams) return;
    float g = 0.f;
    for (int b = 0; b < nblocks; ++b) g += partial[static_cast<int64_t>(b) * kModelParams + q];
    g *= inv_m;
    if (grad_out) grad_out[q] = g;
    if (lr > 0.f) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float mm = b1 * mst[q] + (1.f - b1) * g;
        const float vv = b2 * vst[q] + (1.f - b2) * g * g;
        mst[q] = mm;
        vst[q] = vv;
        const float mh = mm / (1.f - powf(b1, static_cast<float>(t)));
        const float vh = vv / (1.f - powf(b2, static_cast<float>(t)));
        params[q] -= lr * mh / (sqrtf(vh) + eps);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_lanczos(const SubDesc* subs, int n_subs, int max_n, const void* T, bool fp32, int ksteps,
                           float* labels, cudaStream_t st) {
    const size_t smem = sizeof(float) * 4 * static_cast<size_t>(max_n);
    if (fp32) {
        cudaError_t e = cudaFuncSetAttribute(k_lanczos<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        k_lanczos<float><<<n_subs, 256, smem, st>>>(subs, static_cast<const float*>(T), ksteps, labels);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_lanczos<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        k_lanczos<double><<<n_subs, 256, smem, st>>>(subs, static_cast<const double*>(T), ksteps, labels);
    }
    return cudaGetLastError();
}

size_t mlp_partial_floats(int m) { return static_cast<size_t>((m + kChunk - 1) / kChunk) * (kModelParams + 1); }

cudaError_t launch_mlp_step(const float* params_in, const float* X, const float* Tg, int m, float* partial,
                            float* params, float* mst, float* vst, int t, float lr, float* grad_out, float* loss_out,
                            cudaStream_t st) {
    if (m <= 0) return cudaErrorInvalidValue;
    const int nb = (m + kChunk - 1) / kChunk;
    float* partial_loss = partial + static_cast<size_t>(nb) * kModelParams;
    const size_t smem = sizeof(float) * (kModelParams + kChunk * kF + 4 * kChunk * kH + kChunk * kO + kChunk);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<nb, 256, smem, st>>>(params_in, X, Tg, m, partial, partial_loss);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mlp_reduce_adam<<<(kModelParams + 255) / 256, 256, 0, st>>>(partial, partial_loss, nb, m, params, mst, vst, t, lr,
                                                                  grad_out, loss_out);
    return cudaGetLastError();
}

}  // namespace smx
