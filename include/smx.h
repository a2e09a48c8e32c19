/*
 * smx.h -- C ABI of the GB300 submatrix density-matrix library.
 *
 * The library computes the density matrix of a sparse, filtered, orthogonalised
 * Kohn-Sham-like matrix H by sign-function purification (the paper's Eq. 14
 * with S = I),
 *
 *        D = 1/2 (I - sign(H - mu I)),
 *
 * using the submatrix method (the paper's Fig. 2): for every block column j the
 * block rows R_j stored in that column of the filtered H form a dense principal
 * submatrix T_j = H[R_j, R_j]; its sign function (Eq. 13) is computed by
 * Newton-Schulz iteration on the GPU; only the columns of block j are kept,
 * D[R_j, j] = 1/2 (E_j - sign(T_j - mu I)[:, cols of j]).  mu is either fixed
 * or found by bisection on trace(D) = n_e.
 *
 * Conventions (all entry points):
 *  - Every function returns an smx_status and never throws or aborts.
 *  - Arrays passed in are borrowed for the duration of the call only; the
 *    library copies what it keeps.  The library owns all device memory it
 *    allocates and frees it in smx_destroy.
 *  - "Host pointer" means ordinary CPU memory (pinned or pageable); "device
 *    pointer" means memory of the current CUDA device.
 *  - Work is enqueued on the stream given to smx_create (NULL = legacy default
 *    stream).  Calls that return results to the host synchronise that stream.
 *  - A failure inside asynchronous device work (non-finite numbers, a
 *    submatrix that did not converge, a device wait that timed out) is latched
 *    in the context and reported by the next smx_get_* call; it stays latched
 *    until the next successful smx_build_density / smx_solve_mu.
 *  - Matrix layout ("block-CSC"): n_block_cols block columns; block i has
 *    block_size[i] rows and columns.  Column j stores blocks for the block
 *    rows row_idx[col_ptr[j] .. col_ptr[j+1]-1], strictly ascending; the
 *    diagonal block must be present and the block pattern must be symmetric.
 *    values holds the blocks in that order, each block (b_r x b_c) stored
 *    column-major, so block k starts at sum_{k' < k} b_r(k') b_c(k').
 *  - The values of H are assumed symmetric (H_ij = H_ji^T); they are not
 *    checked for symmetry.
 *
 * Thread safety: a context must not be used from two host threads at once.
 * Different contexts are independent.
 */
#ifndef SMX_H
#define SMX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smx_ctx smx_ctx;

typedef enum {
    SMX_OK = 0,
    SMX_ERR_ARG = 1,         /* null pointer, size out of range, unknown enum value */
    SMX_ERR_PATTERN = 2,     /* malformed block-CSC pattern */
    SMX_ERR_NONFINITE = 3,   /* NaN/Inf in the input values or in a submatrix iteration */
    SMX_ERR_CUDA = 4,        /* a CUDA runtime call failed (the context should be destroyed) */
    SMX_ERR_OOM = 5,         /* device allocation failed */
    SMX_ERR_NOCONV = 6,      /* a submatrix did not converge within the iteration cap */
    SMX_ERR_NOBRACKET = 7,   /* the electron count lies outside [0, N] */
    SMX_ERR_TIMEOUT = 8,     /* a device-side wait exceeded its limit and the kernel gave up */
    SMX_ERR_STATE = 9,       /* call order violated (e.g. results requested before a build) */
    SMX_ERR_UNSUPPORTED = 10 /* valid request this build cannot serve (e.g. submatrix too large) */
} smx_status;

/* Arithmetic of the Newton-Schulz bulk phase (Eq. 13 iteration).
 *  SMX_FP64   : FP64 on the CUDA cores ("plain" form).
 *  SMX_FP16X3 : tcgen05 tensor cores, FP16 operands split as hi + lo with three
 *               products (hi*hi + hi*lo + lo*hi) per step and FP32 accumulation
 *               in tensor memory; about 22 significant bits per operand.
 *  SMX_FP16   : tcgen05, one FP16 product per step, FP32 accumulation.
 *  SMX_BF16   : tcgen05, one BF16 product per step, FP32 accumulation.
 * The scaling X0 = (T - mu I)/b per submatrix, the trace and the energy are
 * always FP64. */
typedef enum {
    SMX_FP64 = 0,
    SMX_FP16X3 = 1,
    SMX_FP16 = 2,
    SMX_BF16 = 3
} smx_precision;

/* Matrix function a build computes (Fig. 2 is generic in f).
 *   SMX_FN_DENSITY  D = 1/2 (I - sign(H - mu I)) (Eq. 14 with S = I), the default;
 *   SMX_FN_INV_SQRT (H - mu I)^(-1/2) and SMX_FN_SQRT (H - mu I)^(1/2) for a
 *                   symmetric positive definite H - mu I (an overlap matrix with
 *                   mu = 0, the step before the non-orthogonal form of Eq. 14):
 *                   per block column the owner columns of f(T_j - mu I), by the
 *                   sign iteration of the Eq. 12 block matrix [[0, A], [I, 0]]
 *                   written per block (coupled Newton-Schulz);
 *   SMX_FN_INV      (H - mu I)^(-1) for the same inputs: the square of the
 *                   iteration's (H - mu I)^(-1/2), owner columns only;
 *   SMX_FN_FERMI    the finite-temperature Fermi function
 *                   (I + exp(beta (H - mu I)))^(-1) = 1/2 (I - tanh(beta (H - mu I)/2)),
 *                   the finite-temperature counterpart of Eq. 14 (beta from
 *                   smx_set_fermi_beta): per submatrix, tanh by a Taylor start at
 *                   a small argument and k doublings tanh(2x) = 2 tanh(x)/(1 + tanh^2 x),
 *                   each with a Newton-Schulz inverse of I + T^2 (products only;
 *                   about 7 + 11 k products, k = log2(8 beta G_j)). */
typedef enum {
    SMX_FN_DENSITY = 0,
    SMX_FN_INV_SQRT = 1,
    SMX_FN_SQRT = 2,
    SMX_FN_INV = 3,
    SMX_FN_FERMI = 4
} smx_function;

/* Statistics of the last build (or the last bisection step). */
typedef struct {
    int32_t n_block_cols;       /* number of submatrices */
    int64_t n;                  /* scalar dimension of H */
    int64_t nnzb_input;         /* stored blocks of the input pattern */
    int64_t nnzb_filtered;      /* stored blocks after filtering */
    int32_t dim_min, dim_max;   /* smallest / largest submatrix dimension n_j */
    double dim_mean;
    int32_t iters_min, iters_max; /* Newton-Schulz iterations per submatrix */
    double iters_mean;
    int32_t n_noconv;           /* submatrices that hit the iteration cap */
    int32_t n_bound_fallback;   /* submatrices whose learned bound failed the safe check */
    int32_t bisection_steps;    /* builds done by the last smx_solve_mu (a first step taken again counts twice) */
    double flops_ns;            /* algorithmic flops of the last build: sum_j 4 n_j^3 iters_j
                                   (6 n_j^3 iters_j for the function forms: three products a step) */
    double ms_last_build;       /* device time of the last build (CUDA events), ms */
    double mu;                  /* mu of the last build */
    int32_t precision;          /* smx_precision of the bulk phase */
    int32_t fp64_final_iters;
    /* Counters accumulated since smx_create or the last smx_reset_counters: */
    int64_t kernel_launches;    /* CUDA kernels this library launched */
    int64_t ns_launches;        /* launches of the Newton-Schulz kernel */
    double ns_ms_total;         /* their summed device time (CUDA events on the context stream), ms */
    double ns_work_n3;          /* sum over submatrices and launches of n_j^3 * iterations_j;
                                   4 * ns_work_n3 is the algorithmic Newton-Schulz flop count
                                   (6 * for the function forms) */
} smx_stats;

/* Human-readable name of a status code (static string, never NULL). */
const char* smx_status_string(smx_status s);

/* Creates a context for a block-sparse symmetric H (Fig. 2 input).
 *  out          : receives the new context (set to NULL on failure).
 *  n_block_cols : number of block rows/columns B (>= 1).
 *  block_size   : host int32[B], each >= 1 and <= 64.
 *  col_ptr      : host int64[B+1], col_ptr[0] = 0, non-decreasing.
 *  row_idx      : host int32[col_ptr[B]], see the layout convention above.
 *  values       : host double[sum of block areas], the blocks of H.
 *  cuda_stream  : cudaStream_t to enqueue work on, or NULL.
 * Errors: SMX_ERR_ARG, SMX_ERR_PATTERN, SMX_ERR_NONFINITE, SMX_ERR_OOM, SMX_ERR_CUDA.
 * Defaults: filter threshold 0, mu = 0 (fixed), precision SMX_FP64. */
smx_status smx_create(smx_ctx** out, int32_t n_block_cols, const int32_t* block_size,
                      const int64_t* col_ptr, const int32_t* row_idx, const double* values,
                      void* cuda_stream);

/* Replaces the values of H (same input pattern, e.g. the next MD snapshot;
 * the input of Fig. 2, which Section 4 revisits at every step of a run).
 *  values    : double[] of the same length as in smx_create.
 *  on_device : 0 = host pointer, 1 = device pointer (read on the context stream).
 * The filter is re-applied at the next build.  Errors: SMX_ERR_ARG, SMX_ERR_CUDA. */
smx_status smx_set_values(smx_ctx* ctx, const double* values, int32_t on_device);

/* Block filter (the sparse, filtered matrices of Section 3 that Fig. 2 takes
 * as input; the paper prints no rule, so this library reads it as): an
 * off-diagonal block whose Frobenius norm is strictly below eps is dropped
 * from H (and from D); diagonal blocks are always kept.
 * eps >= 0.  Errors: SMX_ERR_ARG. */
smx_status smx_set_filter_threshold(smx_ctx* ctx, double eps);

/* Upper bound (bytes, >= 1 MiB) on the device staging of the gathered
 * submatrices T_j - mu I (counted as FP64).  Block columns are processed in
 * consecutive chunks whose staging fits; one chunk when everything fits.
 * Default (no call): automatic, a tenth of the device memory for each FP64
 * staging buffer of the plain form (which keeps up to five of that size) and
 * half of it for the FP32 staging of the tensor-core forms (which keep one).
 * Results do not depend on the chunking.  Errors: SMX_ERR_ARG. */
smx_status smx_set_staging_limit(smx_ctx* ctx, uint64_t bytes);

/* Restricts the context to block columns [j0, j1) (one shard of a multi-GPU
 * run; 0 <= j0 < j1 <= n_block_cols, the full range restores the default).
 * Builds then compute D, trace(D) and trace(DH) over those columns only (D
 * is zero elsewhere); the shards' traces add up to the full build's.  The
 * bisection across shards is the caller's (smx_get_gershgorin_interval, a
 * build per midpoint and a sum of the 16-byte traces over the shards);
 * smx_solve_mu returns SMX_ERR_STATE on a shard.  Errors: SMX_ERR_ARG. */
smx_status smx_set_column_range(smx_ctx* ctx, int32_t j0, int32_t j1);

/* Gershgorin interval [lo, hi] of the whole filtered H (Eq. 14's mu lies in
 * it): the bisection bracket.  With an overlap set (smx_set_overlap) the
 * bracket of the non-orthogonal form instead: the union of the Gershgorin
 * intervals of all M_j (runs the setup if needed); SMX_ERR_UNSUPPORTED on a
 * column-range shard (the shard knows only its own M_j) or outside FP64.
 * Synchronises.  Errors: SMX_ERR_ARG, SMX_ERR_CUDA, SMX_ERR_UNSUPPORTED. */
smx_status smx_get_gershgorin_interval(smx_ctx* ctx, double* lo, double* hi);

/* Fixed chemical potential mu (Eq. 14) for smx_build_density.  Errors: SMX_ERR_ARG (non-finite). */
smx_status smx_set_mu(smx_ctx* ctx, double mu);

/* Electron count for smx_solve_mu, which sets Eq. 14's mu (the paper does not
 * say how; this library reads it as a bisection): bisection on
 * trace(D(mu)) = n_e inside the Gershgorin interval of the filtered H, with
 * trace(D) counting orbitals (no spin factor); stops when |trace - n_e| <= tol or
 * after max_steps builds (1..200).  The result is the last evaluated mu.
 * Errors: SMX_ERR_ARG. */
smx_status smx_set_electron_count(smx_ctx* ctx, double n_e, int32_t max_steps, double tol);

/* Arithmetic of the Newton-Schulz iteration (Eq. 13; Section 3's low-precision
 * units).  fp64_final_iters (0..4): when bulk != SMX_FP64, that many plain
 * Newton-Schulz steps in FP64 (CUDA cores) follow the bulk phase's stopping
 * rule, on its last iterate, before the owner columns are scattered (the
 * density matrix only; ignored for SMX_FP64).  Note that they restore
 * X^2 = I but not the occupied subspace a single-pass bulk phase has rotated
 * (a rounding error that anticommutes with the sign persists through later
 * steps), so D keeps an error of the bulk's order.  Errors: SMX_ERR_ARG. */
smx_status smx_set_precision(smx_ctx* ctx, smx_precision bulk, int32_t fp64_final_iters);

/* The matrix function of the following builds.  The function forms run in
 * FP64 only (a build in another precision returns SMX_ERR_UNSUPPORTED) and
 * ignore the learned bound; their result is read with smx_get_density, and
 * smx_get_trace reports its trace and its sum of products with H over the
 * stored entries.  A submatrix that is not positive definite ends in
 * SMX_ERR_NOCONV or SMX_ERR_NONFINITE.  smx_solve_mu needs SMX_FN_DENSITY
 * (SMX_ERR_STATE otherwise).  Errors: SMX_ERR_ARG (unknown f). */
smx_status smx_set_function(smx_ctx* ctx, smx_function f);

/* Inverse temperature beta >= 0 (in inverse units of H) of SMX_FN_FERMI.
 * Default 0 (F = I/2).  Errors: SMX_ERR_ARG (negative or non-finite). */
smx_status smx_set_fermi_beta(smx_ctx* ctx, double beta);

/* Symmetrised result (off by default).  Fig. 2 keeps only the owner columns of
 * each submatrix's f(T_j), so the assembled D is not symmetric (each block
 * D_ij comes from column j's submatrix, D_ji from column i's).  With enable != 0
 * every later build returns 1/2 (D + D^T) on the filtered pattern: both blocks
 * of a pair (i, j), (j, i) get the mean of D_ij and D_ji^T, a diagonal block its
 * symmetric part, and blocks the filter dropped stay zero.  The trace and
 * energy of smx_get_trace stay those of D as built (for the symmetric pattern
 * of a symmetric H they are unchanged).  The pair list of the input pattern is
 * built on the first enable (host work and one upload, synchronous).
 * Errors: SMX_ERR_UNSUPPORTED with a column range set (smx_set_column_range:
 * a shard holds only its own columns of D; also returned by a build if a range
 * is set later). */
smx_status smx_set_symmetrize(smx_ctx* ctx, int32_t enable);

/* Non-orthogonal basis (Eq. 14 with an overlap S != I).  values: S on the
 * block pattern given to smx_create, in the same layout as H (n_values
 * doubles, host or device memory per on_device; copied, the caller keeps
 * ownership); NULL returns the context to S = I.  The following builds
 * compute, per block column j on the filtered pattern of H (S is taken on the
 * same pattern), P_j = 1/2 (I - sign(A_S^-1 A_H - mu I)) A_S^-1 with
 * A_H = H[R_j, R_j], A_S = S[R_j, R_j], as P_j = 1/2 L (I - sign(M - mu I)) L
 * with L = A_S^-1/2 (coupled Newton-Schulz iteration, Eq. 12) and
 * M = L A_H L, and write the owner columns P[R_j, j].  L and M are computed once
 * per (H, S, filtered pattern) and kept (2 sum_j n_j ld_j doubles); each
 * bisection step then runs the sign iteration on M - mu I.  smx_get_trace
 * reports tr(P S) = sum_pq P_pq S_pq over the stored entries (the electron
 * count that smx_solve_mu matches) and sum_pq P_pq H_pq; the bisection
 * bracket is the union of the Gershgorin intervals of the M_j.  Supported for
 * SMX_FN_DENSITY in SMX_FP64 on a single staging chunk (SMX_ERR_UNSUPPORTED
 * from the build otherwise).  An S whose submatrices are not positive definite
 * ends in SMX_ERR_NOCONV or SMX_ERR_NONFINITE.  Errors: SMX_ERR_ARG,
 * SMX_ERR_NONFINITE (host values), SMX_ERR_OOM, SMX_ERR_CUDA. */
smx_status smx_set_overlap(smx_ctx* ctx, const double* values, int32_t on_device);

/* Builds D at the current fixed mu (Fig. 2 steps (i)-(iii) and Eq. 14):
 * filter (if values or threshold changed), gather, spectral bound, scaling,
 * Newton-Schulz, scatter, trace and energy.  Asynchronous on the context
 * stream except for a small host round trip when the filtered pattern must
 * be recomputed.  Errors: SMX_ERR_NONFINITE (input), SMX_ERR_OOM, SMX_ERR_CUDA,
 * SMX_ERR_UNSUPPORTED (a submatrix larger than this build handles). */
smx_status smx_build_density(smx_ctx* ctx);

/* Finds Eq. 14's mu by bisection (see smx_set_electron_count) and leaves the
 * last build's D in the context.  Synchronises once per bisection step.  With new
 * values on an analysed context the filter and the first step (at the
 * bracket's midpoint, computed on the device) are issued together and read
 * back once; if the filter changed the filtered pattern, that step is taken
 * again on the new pattern (and counted in bisection_steps).
 * Errors: as smx_build_density, plus SMX_ERR_STATE (no electron count set),
 * SMX_ERR_NOBRACKET, and latched device errors. */
smx_status smx_solve_mu(smx_ctx* ctx);

/* The same bisection as smx_solve_mu with its decisions taken on the device
 * (Eq. 14's mu; a device-side loop): the bracket and the current midpoint live
 * in device memory, every step is a build reading mu from there followed by a
 * one-thread update, and all max_steps steps are enqueued at once; once the
 * stopping rule holds (or after max_steps builds) the later steps' kernels
 * return at once.  The result (mu, D, trace) is that of smx_solve_mu from the
 * same state, bit for bit, and the host waits once (plus once for the filter
 * when the values are new: the filtered pattern must be known before the
 * builds are enqueued).  Not for the non-orthogonal form
 * (SMX_ERR_UNSUPPORTED).  Errors: as smx_solve_mu. */
smx_status smx_solve_mu_device(smx_ctx* ctx);

/* trace(D), trace(D H) (the band-structure energy, unshifted H) and mu of the
 * last build, D being Eq. 14's density matrix assembled by Fig. 2 (trace(D)
 * sums the diagonals of the diagonal blocks; trace(D H) sums D_pq H_pq over
 * the stored entries of the filtered pattern).  Any argument may be NULL.  Synchronises the stream and returns
 * latched device errors.  Errors: SMX_ERR_STATE (no build yet). */
smx_status smx_get_trace(smx_ctx* ctx, double* trace_D, double* trace_DH, double* mu);

/* Copies D of the last build (Fig. 2 step (iii): the kept columns of each
 * f(T_j), inserted into D, which has the filtered pattern of H and no fill-in
 * of its own), laid out exactly like the input values (input pattern; blocks
 * dropped by the filter are zero).
 *  values_out : double[] of the input value count; host or device pointer.
 *  on_device  : 0 = host pointer (synchronises), 1 = device pointer (async).
 * Errors: SMX_ERR_ARG, SMX_ERR_STATE, SMX_ERR_CUDA, latched device errors. */
smx_status smx_get_density(smx_ctx* ctx, double* values_out, int32_t on_device);

/* Filtered pattern of the last build (the pattern of H after the block filter
 * of smx_set_filter_threshold, which D shares; it fixes the index sets R_j of
 * Fig. 2).  col_ptr: host int64[B+1]; row_idx: host int32[nnzb_filtered]
 * (size from smx_get_stats), either may be NULL. */
smx_status smx_get_pattern(smx_ctx* ctx, int64_t* col_ptr, int32_t* row_idx);

/* Statistics of the last build (see smx_stats): the submatrix dimensions of
 * Fig. 2, the iterations of the Eq. 13 iteration (two products of n_j x n_j
 * matrices each, hence 4 n_j^3 flops), fallbacks of the learned bound
 * (Section 4) and device timings.  Synchronises. */
smx_status smx_get_stats(smx_ctx* ctx, smx_stats* out);

/* ---------------------------------------------------------------------------
 * Learned spectral bound (the paper's Section 4: a network trained on data the
 * simulation itself produces, consulted during the run).
 *
 * Per submatrix A = T_j - mu I the model maps nine features (all over the
 * Gershgorin bound G = max_r sum_c |A_rc|, except f6 and f8):
 *   f0 ||A||_F/sqrt(n)  f1 max|A_rr|  f2 mean|A_rr|  f3 std(A_rr)  f4 max_r R_r
 *   f5 mean_r R_r  f6 n/256  f7 mean A_rr  f8 previous-step ratio
 * (R_r = sum_{c != r} |A_rc|; f8 = sqrt(max_r sum_c |(A^2)_rc|)/G of the same
 * block column at the build before the last smx_set_values, 0 before any)
 * through
 * 9 -> 64 -> 64 -> 2 (tanh hidden layers) to predictions of rho/G and delta/G
 * (rho = max |lambda(A)|, delta = min |lambda(A)|).  When enabled, a build
 * starts Newton-Schulz from X0 = A / b with b = rho_hat (1.05) / 1.2; the first
 * product Z = X0^2 gives the guaranteed bound s >= rho(X0) (s^2 =
 * max_r (|Z| w)_r / w_r, the smallest over w = 1 and power steps of |Z| from
 * it, one in the tensor-core forms and two in FP64: a Collatz-Wielandt bound
 * on rho(Z)) and the prediction is kept only if s <= 1.7 (the iteration
 * converges for rho(X0) < sqrt 3 = 1.732), otherwise X0 is rescaled by 1.2/s
 * as without the model (counted in n_bound_fallback).
 * Parameters: SMX_BOUND_MODEL_PARAMS floats, layout W1 (64 x 9, row-major),
 * b1 (64), W2 (64 x 64), b2 (64), W3 (2 x 64), b3 (2).  Inference uses the
 * parameters rounded to FP16; training keeps FP32 master weights (Adam,
 * beta1 0.9, beta2 0.999, eps 1e-8) and minimises 1/(2m) sum (y - t)^2.
 * ------------------------------------------------------------------------- */
#define SMX_BOUND_MODEL_FEATURES 9
#define SMX_BOUND_MODEL_PARAMS 4930

/* Initialises the parameters (uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a
 * counter-based generator seeded by seed, zero biases) and clears the Adam
 * state and the collected samples. */
smx_status smx_bound_model_init(smx_ctx* ctx, uint64_t seed);

/* Copies count (= SMX_BOUND_MODEL_PARAMS) parameters from / to host memory.
 * Setting parameters clears the Adam state.  Errors: SMX_ERR_ARG. */
smx_status smx_bound_model_set_params(smx_ctx* ctx, const float* params, int32_t count);
smx_status smx_bound_model_get_params(smx_ctx* ctx, float* params, int32_t count);

/* Appends one training sample per submatrix of the current H at the fixed mu
 * of smx_set_mu: the features and Lanczos labels (lanczos_steps 8..64 steps on
 * A for rho and on A^2 for delta).  Synchronises. */
smx_status smx_bound_model_collect(smx_ctx* ctx, int32_t lanczos_steps);

/* Trains on the collected samples: epochs passes of contiguous mini-batches of
 * batch samples, Adam with learning rate lr; final_loss (may be NULL) receives
 * the loss of the last mini-batch.  Synchronises. */
smx_status smx_bound_model_train(smx_ctx* ctx, int32_t epochs, int32_t batch, float lr, double* final_loss);

/* steps full-batch Adam steps on caller data (host x[m*9], t[m*2]); grad (host,
 * SMX_BOUND_MODEL_PARAMS floats, may be NULL) receives the gradient at the
 * parameters before the first step, loss (may be NULL) the loss there.
 * steps = 0 only evaluates loss and gradient.  Synchronises. */
smx_status smx_bound_model_fit(smx_ctx* ctx, const float* x, const float* t, int32_t m, int32_t steps, float lr,
                               float* grad, double* loss);

/* For the current H at the fixed mu: host arrays features[B*9], pred[B*2] and
 * Lanczos labels[B*2] (any may be NULL; labels cost lanczos_steps steps).
 * Synchronises. */
smx_status smx_bound_model_predict(smx_ctx* ctx, float* features, float* pred, float* labels, int32_t lanczos_steps);

/* Enables or disables the model in builds; weights_path, if not NULL, loads
 * parameters saved by smx_bound_model_save.
 *  enable = 0: off (X0 = A / G, first step scaled by 1.2/s, plain steps).
 *  enable = 1: on, with both predictions: after the check on rho_hat passes,
 *              the predicted gap sets the scaled schedule of the Newton-Schulz
 *              steps, X_{k+1} = p(a_k X_k) with p(x) = x (3 - x^2)/2,
 *              a_k = min(sqrt(3 / (1 + l_k + l_k^2)), 1.72), l_0 =
 *              delta_hat / (b s) and l_{k+1} = p(a_k l_k) (the interval
 *              [l_k, 1] of |eigenvalues| maps into [l_{k+1}, 1]); any l_0 in
 *              (0, 1] converges, a poor prediction only costs steps.
 *  enable = 2: on, rho_hat only (the start scaling; plain steps).
 * The sign the iteration converges to does not depend on the mode (Eq. 13).
 * Errors: SMX_ERR_ARG (bad file, enable outside 0..2), SMX_ERR_STATE
 * (enabling a model that was never initialised). */
smx_status smx_set_bound_model(smx_ctx* ctx, int32_t enable, const char* weights_path);

/* Writes the parameters to a binary file: 8-byte magic "SMXBNDM1", int32
 * count, count floats, uint64 checksum (FNV-1a of the float bytes). */
smx_status smx_bound_model_save(smx_ctx* ctx, const char* path);

/* Failure-detection self-test of the bounded device waits (the paper has no
 * counterpart).  Every wait of the library's kernels on an mbarrier gives up
 * after a fixed number of polls, records SMX_ERR_TIMEOUT in the context's
 * status word and lets the kernel return (after draining its own copies and
 * tensor-core work), so that a lost arrival surfaces as an error instead of a
 * hung GPU.  This call exercises that path safely: one thread of a one-CTA
 * kernel waits on a fresh mbarrier that nothing arrives at, with no
 * asynchronous copy or tensor-core operation in flight, and gives up after
 * poll_limit polls (1 .. 2^26).  Synchronises and returns SMX_ERR_TIMEOUT
 * (SMX_OK would mean the wait completed, which cannot happen); the error stays
 * latched until the next smx_build_density / smx_solve_mu, and the context
 * stays usable.  Errors: SMX_ERR_ARG, SMX_ERR_CUDA. */
smx_status smx_selftest_wait_timeout(smx_ctx* ctx, uint32_t poll_limit);

/* Zeroes the accumulated counters of smx_stats.  Synchronises the stream. */
smx_status smx_reset_counters(smx_ctx* ctx);

/* Per-submatrix details of the last build, host arrays of length B (any may
 * be NULL): dimension n_j, Newton-Schulz iterations, and the scaling bound
 * b_j used for X0 = (T_j - mu I)/b_j.  Synchronises. */
smx_status smx_get_submatrix_info(smx_ctx* ctx, int32_t* dims, int32_t* iters, double* bounds);

/* Dense density matrix without any device allocation.  The paper has no
 * counterpart: this call serves callers that cannot allocate device memory
 * when they need the result, such as plug-ins whose host framework's caching
 * allocator owns the whole device pool, and latency-critical loops that must
 * not enter the driver's allocator (cudaMalloc/cudaFree can synchronise the
 * device).
 * Computes D = 1/2 (I - sign(H - mu I)) of one dense symmetric H by FP64
 * Newton-Schulz iteration with a Gershgorin scaling (Eq. 13 and Eq. 14 with
 * S = I on a single dense matrix; one CTA; same arithmetic as the FP64 form
 * of smx_build_density).
 *  h_dev       : device double[n*n], row-major, symmetric (read only).
 *  n           : 1 <= n <= 256; larger n returns SMX_ERR_ARG.
 *  mu          : finite chemical potential.
 *  d_dev       : device double[n*n], row-major, receives D (caller-owned).
 *  cuda_stream : stream to run on (NULL = legacy default stream).
 * Work matrices live in one fixed __device__ array of 3*256*256 + 4 doubles
 * (about 1.5 MiB) that every GPU which loads the library keeps until the
 * process exits.  The first call on a device (and the first after a device
 * reset) looks up that array's device address (cudaGetSymbolAddress), so
 * make the first call on each device before any stream capture.  All calls
 * share the array and it keeps the last call's contents (every call
 * overwrites what it reads): calls whose work overlaps on a GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The call waits for its stream (a copy of the status to the host and a
 * stream synchronisation) and returns: SMX_ERR_ARG, SMX_ERR_CUDA,
 * SMX_ERR_UNSUPPORTED (device index >= 64), SMX_ERR_NONFINITE,
 * SMX_ERR_NOCONV. */
smx_status smx_dense_density_noalloc(const double* h_dev, int32_t n, double mu, double* d_dev,
                                     void* cuda_stream);

/* Releases the context and all device memory it owns.  NULL is ignored. */
void smx_destroy(smx_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SMX_H */
