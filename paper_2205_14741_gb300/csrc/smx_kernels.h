// Host-side launchers of the library's CUDA kernels (internal interface).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "smx_device.cuh"

namespace smx {

// Small device-side state of a context, read back by the host in one copy.
struct DevScalars {
    double trace, energy;  // a8: trace(D) and trace(D H) of the last build
    double br_lo, br_hi;   // Gershgorin bracket of the filtered H (a9)
    double mu0;            // 0.5 (br_lo + br_hi): the first bisection step
    double bis_mid;        // device-side bisection: the mu of the current step
    double bis_lo, bis_hi; // ... and its bracket
    int status;            // first error recorded by a kernel (kOk = 0)
    int changed;           // the keep flags differ from the current filtered pattern
    int fallbacks;         // learned-bound fallbacks since the last reset
    int ns_counter;        // job counter of the tensor-core Newton-Schulz kernel (reset by the scatter)
    unsigned int filter_done, scatter_done;  // last-block tickets (each reset by its last block)
    unsigned long long nlo_enc, hi_enc;      // filter: running bracket as order-preserving images (reset by its last block)
    int bis_done;          // device-side bisection: stopped (the later builds are skipped)
    int bis_steps;         // ... builds evaluated
};

// Device-side bisection for mu (a9): start at the bracket's midpoint (one thread).
cudaError_t launch_bisect_init(DevScalars* sc, double lo, double hi, cudaStream_t st);
// After a build at sc->bis_mid: stop when |trace - n_e| <= tol or after max_steps builds (the
// result is the last evaluated mu), else halve the bracket and set the next midpoint.  Once
// stopped, the following steps change nothing (and the kernels of their builds return early).
cudaError_t launch_bisect_step(DevScalars* sc, double n_e, double tol, int max_steps, cudaStream_t st);

// a1 + bracket: keep flags of every block (Frobenius norm >= eps, diagonal
// always), non-finite check (sc->status), FP32 copy of H; with keep_prev,
// sc->changed = 1 when a flag differs from it.  The Gershgorin bracket of the
// filtered H (minimum and maximum over its columns' intervals) and its
// midpoint go to sc->br_lo, br_hi, mu0.
// max_col_blocks: the largest number of blocks in a column of the input pattern.
cudaError_t launch_filter_gershgorin(const double* H, const int64_t* col_ptr, const int32_t* row_idx, const int64_t* voff,
                                     const int32_t* bsize, int n_cols, int bmax, int max_col_blocks, double eps,
                                     uint8_t* keep, const uint8_t* keep_prev, float* H32, DevScalars* sc, cudaStream_t st);

// Optional outputs of the gather, per submatrix (pointers offset like subs; null = not wanted).
struct GatherExtras {
    double* gersh = nullptr;             // the Gershgorin bound G_j
    const float* prev_ratio = nullptr;   // learned bound: previous-step feature (null = 0)
    float* feat = nullptr;               // learned bound: the 9 features of T_j - mu I
    const float* params = nullptr;       // learned bound: parameters; when set, b_j is the model's
    float* pred = nullptr;               // ... and its two predictions
    float margin = 0.0f;                 // ... b_j = G_j clamp(pred_0, 0.02, 1) (1 + margin) / 1.2
    const double* mu_dev = nullptr;      // when set, mu is read from here (on the device) instead
    const int* skip = nullptr;           // when set and non-zero at launch, the kernel does nothing
};

// a3 + a4: T_j = H[R_j, R_j] - mu I into the FP64 staging buffer, then the
// Gershgorin bound b_j = max row abs-sum of T_j (>= spectral radius), or the
// learned bound (extras.params).
// bmax: the largest block size; uniform: every block has that size.
cudaError_t launch_gather_bound(const SubDesc* subs, int n_subs, int max_nblk, int max_n, int bmax, bool uniform,
                                const PatternView& pv, const double* H, double mu, double* T, double* bound,
                                const GatherExtras& ex, cudaStream_t st);
// The same in FP32 (tensor-core path): T32 from the FP32 copy of H; the bound
// is enlarged by 1e-5 relative to cover FP32 summation.
cudaError_t launch_gather_bound_f32(const SubDesc* subs, int n_subs, int max_nblk, int max_n, int bmax, bool uniform,
                                    const PatternView& pv, const float* H32, double mu, float* T32, double* bound,
                                    const GatherExtras& ex, cudaStream_t st);

// a8 (FP64 form): deterministic sums of the per-column partials ->
// sc->trace = trace(D), sc->energy = trace(D H).
cudaError_t launch_reduce(const double2* partial, int n_cols, DevScalars* sc, cudaStream_t st,
                          const int* skip = nullptr);

// D <- 1/2 (D + D^T) on the filtered pattern, in place, in the input layout: for each block
// pair both blocks get the mean of the block and the transpose of its partner, and a block the
// filter dropped (keep[k] == 0) stays zero.  One warp per pair; every element is read and
// written by one thread.
cudaError_t launch_symmetrize(const SymPair* pairs, int n_pairs, const uint8_t* keep, double* D, cudaStream_t st,
                              const int* skip = nullptr);

// Failure-detection self-test: a wait on an mbarrier nothing arrives at, given up after
// poll_limit polls (records kErrTimeout in *status; *polls_out, if set, the polls made).
cudaError_t launch_wait_selftest(int* status, uint32_t poll_limit, int* polls_out, cudaStream_t st);

// a5/a6 (FP64 plain form) + a7: Newton-Schulz in FP64, then scatter.
// Matrix function of a build (values of smx_function): 0 = the density matrix
// 1/2 (I - sign(A)), 1 = A^-1/2, 2 = A^1/2 (A = T_j - mu I symmetric positive definite).
enum : int { kFnDensity = 0, kFnInvSqrt = 1, kFnSqrt = 2, kFnInv = 3, kFnFermi = 4 };

struct NsFp64Args {
    const SubDesc* subs;
    int n_subs;
    double* T;   // FP64 staging buffer (overwritten: X0 = T / b)
    double* W1;  // FP64 work buffers laid out like T
    double* W2;
    double* W3;  // a third one for the function forms (coupled iteration), else unused
    double* W4 = nullptr;  // a fourth one for the Fermi function
    int function;  // kFnDensity, kFnInvSqrt or kFnSqrt
    double* bound;  // in: initial bound b_j; out: effective bound after the a-posteriori rescale
    double tau;
    int max_iter;
    int32_t* iters;
    unsigned long long* work_n3;  // += n_j^3 * iters_j per submatrix
    double* gersh;         // Gershgorin bound G_j of T_j - mu I (written here in the non-orthogonal form)
    float* sq_ratio;       // out: sqrt(max_r sum_c |(A^2)_rc|) / G_j, the Gershgorin bound of A^2 (next-step feature)
    int use_model;         // the initial bound came from the learned model: keep it when the check passes
    int* fallbacks;        // count of submatrices whose learned bound failed the check
    int* status;
    PatternView pv;
    const double* H;
    double* D;
    double2* partial;
    // non-orthogonal form (Eq. 14 with S != I), all null otherwise: the iteration starts from
    // M_j - mu I (T is not read; bound and gersh are written), the owner columns of
    // P_j = 1/2 L_j (I - X) L_j are scattered, and the trace is sum P_pq S_pq
    const double* Mc = nullptr;  // M_j = L_j A_H L_j, laid out like T
    const double* Lc = nullptr;  // L_j = A_S^-1/2, laid out like T
    const double* Sv = nullptr;  // S in the input value layout
    double mu = 0.0;
    // learned bound: predictions of this chunk ([2 i + 1] = delta_hat / G for the i-th
    // submatrix); see NsTcArgs::pred
    const float* pred = nullptr;
    // FP64 finishing steps after a low-precision bulk phase (> 0): T holds the bulk phase's last
    // iterate X (not T_j - mu I); exactly this many plain steps in FP64, then the scatter; the
    // steps are added to iters
    int finish_iters = 0;
    const int* skip = nullptr;  // when set and non-zero at launch, the kernel does nothing
    double beta = 0.0;          // kFnFermi: the inverse temperature (in inverse units of H)
};
cudaError_t launch_ns_fp64(const NsFp64Args& a, int max_nblk, cudaStream_t st);

// Setup of the non-orthogonal form, once per (H, S): L_j = A_S^-1/2 (coupled iteration) and
// M_j = L_j A_H L_j with its Gershgorin interval, a CTA per submatrix.
struct NonorthSetupArgs {
    const SubDesc* subs;
    int n_subs;
    double* Lc;             // in: A_S = S[R_j, R_j]; out: L_j
    double* Mc;             // in: A_H = H[R_j, R_j]; out: M_j (symmetrised)
    double* T;              // work buffers laid out like Lc
    double* W1;
    double* W2;
    double* W3;
    const double* bound_s;  // Gershgorin bound of A_S (>= its largest eigenvalue)
    double tau;
    int max_iter;
    int32_t* iters;         // out: steps of the coupled iteration per block column
    double* lohi;           // out: [2 * n_subs] Gershgorin interval of M_j
    int* status;
};
cudaError_t launch_nonorth_setup(const NonorthSetupArgs& a, cudaStream_t st);

// a5 (tcgen05 tensor cores) + a7.
struct NsTcArgs {
    const SubDesc* subs;
    const int32_t* order;  // processing order (largest first)
    int n_subs;
    int* work_counter;     // zero at launch (the scatter that follows resets it)
    const float* T;        // FP32 staging of T_j - mu I (leading dimension SubDesc::ld)
    double* bound;         // in: initial bound b_j (X0 = T_j / b_j); out: effective bound after rescaling
    void* ws;              // 16-bit workspace: n_slots * 6 buffers of ld x ld
    int ld;                // multiple of 64, >= every padded n_j
    int n_slots;           // persistent CTAs (one per SM)
    float tau;
    // single-pass forms: also stop after a step whose residual lies below this level but is
    // more than half the previous one (the rounding floor; 0 = off)
    float stall_level;
    int max_iter;
    int32_t* iters;
    unsigned long long* work_n3;  // += n_j^3 * iters_j per submatrix
    const double* gersh;   // Gershgorin bound G_j of T_j - mu I
    float* sq_ratio;       // out: sqrt(max_r sum_c |(A^2)_rc|) / G_j, the Gershgorin bound of A^2 (next-step feature)
    int use_model;         // the initial bound came from the learned model: keep it when the check passes
    int* fallbacks;        // count of submatrices whose learned bound failed the check
    int* status;
    PatternView pv;
    const double* H;
    double* D;
    double2* partial;
    float* xown;           // receives columns own .. own + bown of each final X
    // learned bound: predictions per block column ([2 j + 1] = delta_hat / G_j); with the
    // prediction accepted, the steps follow the scaled schedule from the lower bound
    // delta_hat / (b_j s) (null: plain steps after the a-posteriori start)
    const float* pred = nullptr;
    // when set, the final X of every submatrix (n_j x n_j, row-major with leading dimension
    // SubDesc::ld at SubDesc::t_off, as FP64) for FP64 finishing steps
    double* xfull = nullptr;
    const int* skip = nullptr;  // when set and non-zero at launch, the kernel does nothing
};
// precision: 1 = FP16 split hi/lo (3 products), 2 = FP16, 3 = BF16 (values of smx_precision)
cudaError_t launch_ns_tc(const NsTcArgs& a, int precision, const CUtensorMap& tmap, int max_nblk, cudaStream_t st);

// a7 + a8 for the tensor-core path: D[R_j, j] = 1/2 (E_j - X[:, own]) from the
// saved owner columns, with the per-column trace (FP64) and energy (FP32 terms
// against the FP32 copy H32 of H, FP64 over warps and columns) partials; the
// last block sums partial[0, n_cols) in a fixed order into sc->trace,
// sc->energy and resets sc->ns_counter for the next Newton-Schulz launch.
cudaError_t launch_scatter_owner(const SubDesc* subs, int n_subs, int max_nblk, int max_n, int bmax, bool uniform,
                                 const PatternView& pv, const float* xown, const float* H32, double* D, double2* partial, int n_cols,
                                 DevScalars* sc, cudaStream_t st, const int* skip = nullptr);

// ---------------------------------------------------------------------------
// learned spectral bound (k_bound_model.cu)
// ---------------------------------------------------------------------------
constexpr int kModelFeatures = 9;
constexpr int kModelHidden = 64;
constexpr int kModelParams = 64 * kModelFeatures + 64 + 64 * 64 + 64 + 2 * 64 + 2;  // 4930
// flat parameter layout: W1 (64 x 9, row-major), b1, W2 (64 x 64), b2, W3 (2 x 64), b3
constexpr int kOffB1 = kModelHidden * kModelFeatures, kOffW2 = kOffB1 + kModelHidden,
              kOffB2 = kOffW2 + kModelHidden * kModelHidden, kOffW3 = kOffB2 + kModelHidden,
              kOffB3 = kOffW3 + 2 * kModelHidden;
static_assert(kOffB3 + 2 == kModelParams, "parameter layout");
constexpr int kMaxLanczos = 64;
// b_j = rho_hat (1 + margin) / 1.2: the margin covers the model's typical
// under-prediction (a few percent) so that the first-product check passes
constexpr float kModelMargin = 0.05f;

// labels[2j] = rho/G, labels[2j+1] = delta/G by Lanczos on A and A^2
cudaError_t launch_lanczos(const SubDesc* subs, int n_subs, int max_n, const void* T, bool fp32, int ksteps,
                           float* labels, cudaStream_t st);
// floats of scratch one gradient/Adam step on m samples needs
size_t mlp_partial_floats(int m);
// gradient at params_in on (X, Tg); grad_out/loss_out optional; Adam update of params when lr > 0
cudaError_t launch_mlp_step(const float* params_in, const float* X, const float* Tg, int m, float* partial,
                            float* params, float* mst, float* vst, int t, float lr, float* grad_out, float* loss_out,
                            cudaStream_t st);

// Dynamic shared memory the tcgen05 kernel needs for a precision.
size_t ns_tc_smem_bytes(int precision);

}  // namespace smx
