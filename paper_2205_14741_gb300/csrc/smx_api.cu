// C ABI of the submatrix density-matrix library (declared in include/smx.h).
//
// Host responsibilities: validation of the block-CSC pattern, the symbolic
// analysis of the filtered pattern (R_j, n_j, owner offsets; Fig. 2 step
// (i)), device memory, the TMA tensor map of the tensor-core workspace, the
// launch sequence of one build, the mu bisection loop and the statistics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "smx.h"
#include "smx_kernels.h"

namespace {
// NVTX range over a host scope (filter, each build and its phases, each bisection step), so that
// profiler timelines group the library's launches; free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace


using namespace smx;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
        dev_ = dev;
    }
    ~DeviceGuard() {
        if (prev_ != dev_) cudaSetDevice(prev_);
    }

   private:
    int prev_ = 0, dev_ = 0;
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct smx_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;

    // input pattern
    int32_t B = 0;
    int32_t bmax = 0;  // largest block size
    bool bsize_uniform = false;  // every block has size bmax
    int32_t max_col_blocks = 0;  // most blocks in one column of the input pattern
    int64_t N = 0, nnzb = 0, n_values = 0;
    std::vector<int32_t> bs, row_idx;
    std::vector<int64_t> col_ptr, voff, row_start;

    // settings
    double eps = 0.0, mu = 0.0;
    bool have_ne = false;
    double n_e = 0.0, tol = 0.5;
    int max_steps = 30;
    int precision = SMX_FP64;
    int function = SMX_FN_DENSITY;
    int fp64_final = 0;

    // filtered pattern + submatrices
    bool analysed = false, dirty = true;
    std::vector<uint8_t> keep;
    std::vector<int64_t> fcol_ptr, fvoff;
    std::vector<int32_t> frow_idx, lstart, order;
    std::vector<int32_t> maps;     // block maps of the submatrices (empty: built by the gather)
    std::vector<int64_t> map_off;
    std::vector<SubDesc> subs;
    int max_nblk = 0, max_n = 0;
    int64_t t_elems = 0, x_elems = 0;

    // device buffers
    DevBuf d_H, d_H32, d_voff, d_row_idx, d_col_ptr, d_bs, d_keep, d_keep_prev;
    double br_lo = 0.0, br_hi = 0.0;  // Gershgorin bracket of the filtered H (from the last filter)
    bool filter_compared = false;     // the last filter launch compared its flags with the current pattern
    DevBuf d_sc;                      // DevScalars: status, flags, bracket, trace and energy
    DevScalars* h_sc = nullptr;       // pinned copy, filled by fetch()
    DevBuf d_fcol_ptr, d_frow_idx, d_fvoff, d_lstart, d_subs, d_order, d_maps, d_map_off;
    DevBuf d_T, d_W1, d_W2, d_W3, d_W4, d_ws, d_D, d_xown;
    DevBuf d_bound, d_iters, d_partial, d_work_n3;
    uint8_t* h_keep_pinned = nullptr;

    // tensor-core workspace
    CUtensorMap tmap;
    int ws_ld = 0, ws_slots = 0, ws_prec = -1;
    EncodeTiledFn encode = nullptr;

    // results
    bool built = false;
    double last_mu = 0.0;
    int bisection_steps = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    // counters (see smx_stats)
    int64_t kernel_launches = 0, ns_launches = 0;
    double ns_ms_total = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ns_events;  // pool, one pair per pending launch
    size_t ns_pending = 0;

    // staging of the submatrices T_j in chunks of consecutive block columns
    size_t staging_limit = 0;  // bytes counted as FP64 elements; 0 = automatic from the device memory
    size_t mem_total = 0;      // device memory at creation
    size_t chunk_elem = 0;     // element size the chunks were laid out for (automatic limit)
    std::vector<int32_t> chunk_start;         // chunk c = block columns [chunk_start[c], chunk_start[c + 1])
    int32_t col_lo = 0, col_hi = -1;          // block columns this context builds (a shard); col_hi < 0: all
    int64_t t_chunk_max = 0;                  // elements of the largest chunk

    // non-orthogonal form (Eq. 14 with an overlap S on the pattern of H)
    bool have_S = false, nonorth_ready = false;
    DevBuf d_S, d_Lc, d_Mc, d_nlohi, d_setup_iters;
    double nbr_lo = 0.0, nbr_hi = 0.0;  // bracket: the Gershgorin intervals of all M_j

    // learned spectral bound
    bool model_ready = false, model_on = false, sq_valid = false;
    bool model_gap = false;  // the learned gap drives the scaled Newton-Schulz schedule
    double beta = 0.0;       // inverse temperature of SMX_FN_FERMI
    // the symmetrised D: the block pairs of the input pattern (built on first use)
    bool symmetrize = false;
    int32_t n_pairs = -1;
    DevBuf d_pairs;
    int adam_t = 0;
    int64_t n_samples = 0, cap_samples = 0;
    DevBuf d_params, d_mst, d_vst, d_partial_mlp, d_feat, d_pred, d_labels, d_gersh, d_prev_ratio, d_sq_ratio,
        d_loss, d_sx, d_st, d_fit_x, d_fit_t, d_grad;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

static smx_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SMX_OK;
    if (e == cudaErrorMemoryAllocation) return SMX_ERR_OOM;
    return SMX_ERR_CUDA;
}

#define SMX_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_status(e_);      \
    } while (0)

#define SMX_TRY(call)                          \
    do {                                       \
        smx_status s_ = (call);                \
        if (s_ != SMX_OK) return s_;           \
    } while (0)

static smx_status ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return SMX_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    SMX_CUDA(cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
    return SMX_OK;
}

static void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

template <class T>
static smx_status upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
    SMX_TRY(ensure(b, v.size() * sizeof(T)));
    if (!v.empty()) SMX_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return SMX_OK;
}

template <class T>
static T* dp(DevBuf& b) {
    return static_cast<T*>(b.p);
}

static PatternView pattern_view(smx_ctx* c) {
    PatternView pv;
    pv.fcol_ptr = dp<int64_t>(c->d_fcol_ptr);
    pv.frow_idx = dp<int32_t>(c->d_frow_idx);
    pv.fvoff = dp<int64_t>(c->d_fvoff);
    pv.lstart = dp<int32_t>(c->d_lstart);
    pv.bsize = dp<int32_t>(c->d_bs);
    if (!c->maps.empty()) {
        pv.maps = dp<int32_t>(c->d_maps);
        pv.map_off = dp<int64_t>(c->d_map_off);
    }
    return pv;
}

// Pattern checks: monotone col_ptr, strictly ascending in-range rows, diagonal
// present, symmetric block pattern.
static smx_status validate_pattern(int32_t B, const int32_t* bs, const int64_t* col_ptr, const int32_t* row_idx) {
    if (col_ptr[0] != 0) return SMX_ERR_PATTERN;
    for (int32_t j = 0; j < B; ++j) {
        if (bs[j] < 1 || bs[j] > 64) return SMX_ERR_ARG;
        if (col_ptr[j + 1] < col_ptr[j]) return SMX_ERR_PATTERN;
    }
    for (int32_t j = 0; j < B; ++j) {
        bool diag = false;
        for (int64_t k = col_ptr[j]; k < col_ptr[j + 1]; ++k) {
            const int32_t r = row_idx[k];
            if (r < 0 || r >= B) return SMX_ERR_PATTERN;
            if (k > col_ptr[j] && row_idx[k - 1] >= r) return SMX_ERR_PATTERN;
            if (r == j) diag = true;
            // symmetric pattern: block (j, r) must exist, i.e. j in column r
            const int32_t* b0 = row_idx + col_ptr[r];
            const int32_t* b1 = row_idx + col_ptr[r + 1];
            const int32_t* f = std::lower_bound(b0, b1, j);
            if (f == b1 || *f != j) return SMX_ERR_PATTERN;
        }
        if (!diag) return SMX_ERR_PATTERN;
    }
    return SMX_OK;
}

static smx_status get_encoder(smx_ctx* c) {
    if (c->encode) return SMX_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    SMX_CUDA(cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return SMX_ERR_CUDA;
    c->encode = reinterpret_cast<EncodeTiledFn>(fn);
    return SMX_OK;
}

// Filter (a1), the Gershgorin bracket of the filtered H, and symbolic analysis (a2).
static DevScalars* scalars(smx_ctx* c) { return dp<DevScalars>(c->d_sc); }

// Clears the status word, the change flag and the fallback count (once per call that launches work).
static smx_status reset_flags(smx_ctx* c) {
    SMX_CUDA(cudaMemsetAsync(&scalars(c)->status, 0, 3 * sizeof(int), c->stream));
    return SMX_OK;
}

static void accumulate_timers(smx_ctx* c);

// Copies the device scalars to h_sc (one copy) and waits for the stream.
static smx_status fetch(smx_ctx* c) {
    SMX_CUDA(cudaMemcpyAsync(c->h_sc, c->d_sc.p, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    accumulate_timers(c);
    return SMX_OK;
}

// a1 on the device (asynchronous): keep flags, FP32 copy of H, the bracket and,
// against the current filtered pattern, the change flag.
static smx_status launch_filter(smx_ctx* c) {
    NvtxRange nv("smx filter");
    c->filter_compared = c->analysed && c->eps > 0.0;  // without a threshold every block is kept
    SMX_CUDA(launch_filter_gershgorin(dp<double>(c->d_H), dp<int64_t>(c->d_col_ptr), dp<int32_t>(c->d_row_idx),
                                      dp<int64_t>(c->d_voff), dp<int32_t>(c->d_bs), c->B, c->bmax, c->max_col_blocks, c->eps,
                                      dp<uint8_t>(c->d_keep), c->filter_compared ? dp<uint8_t>(c->d_keep_prev) : nullptr,
                                      dp<float>(c->d_H32), scalars(c), c->stream));
    c->kernel_launches += 1;
    return SMX_OK;
}

static smx_status compact(smx_ctx* c);

// After a filter launch and a fetch: errors, the bracket, and the host-side
// compaction of the filtered pattern when it changed (or the first time).
static smx_status after_filter(smx_ctx* c) {
    if (c->h_sc->status == kErrNonfinite) return SMX_ERR_NONFINITE;
    c->br_lo = c->h_sc->br_lo;
    c->br_hi = c->h_sc->br_hi;
    if (c->analysed && (!c->filter_compared || c->h_sc->changed == 0)) {
        c->dirty = false;
        return SMX_OK;  // same filtered pattern
    }
    return compact(c);
}

// a1 + a2, synchronous (clears the flags first).
static smx_status analyse(smx_ctx* c) {
    c->nonorth_ready = false;  // L_j and M_j follow the values of H and the filtered pattern
    SMX_TRY(reset_flags(c));
    SMX_TRY(launch_filter(c));
    SMX_TRY(fetch(c));
    return after_filter(c);
}

// Bytes per staged element: FP64 for the plain form, FP32 for the tensor-core forms.
static size_t staging_elem(const smx_ctx* c) { return c->precision == SMX_FP64 ? sizeof(double) : sizeof(float); }

// Elements of staging per chunk.  An explicit limit counts bytes as FP64 elements.  The
// automatic one takes a tenth of the device memory for each FP64 staging buffer (the plain form
// keeps up to five of that size) and half of it for the FP32 staging of the tensor-core forms,
// which keep one; it follows the precision (the chunks are laid out again when it changes).
static int64_t staging_chunk_elems(smx_ctx* c) {
    if (c->staging_limit) {
        c->chunk_elem = 0;
        return static_cast<int64_t>(c->staging_limit / sizeof(double));
    }
    const size_t elem = staging_elem(c);
    c->chunk_elem = elem;
    const size_t mem = c->mem_total ? c->mem_total : (size_t(24) << 30) * 4;
    return static_cast<int64_t>((elem == sizeof(double) ? mem / 10 : mem / 2) / elem);
}

// a2: the filtered pattern from the keep flags on the device, symbolic sets of
// every submatrix, chunks and processing order (host), uploaded.
static smx_status compact(smx_ctx* c) {
    cudaStream_t st = c->stream;
    SMX_CUDA(cudaMemcpyAsync(c->h_keep_pinned, c->d_keep.p, c->nnzb, cudaMemcpyDeviceToHost, st));
    SMX_CUDA(cudaStreamSynchronize(st));
    c->keep.assign(c->h_keep_pinned, c->h_keep_pinned + c->nnzb);

    const int32_t B = c->B;
    c->fcol_ptr.assign(B + 1, 0);
    c->frow_idx.clear();
    c->fvoff.clear();
    for (int32_t j = 0; j < B; ++j) {
        for (int64_t k = c->col_ptr[j]; k < c->col_ptr[j + 1]; ++k)
            if (c->keep[k]) {
                c->frow_idx.push_back(c->row_idx[k]);
                c->fvoff.push_back(c->voff[k]);
            }
        c->fcol_ptr[j + 1] = static_cast<int64_t>(c->frow_idx.size());
    }
    const int64_t nnzf = static_cast<int64_t>(c->frow_idx.size());
    c->lstart.assign(nnzf, 0);
    c->subs.assign(B, SubDesc{});
    c->max_nblk = 0;
    c->max_n = 0;
    int64_t t_off = 0, x_off = 0;
    const int64_t chunk_elems = std::max<int64_t>(1, staging_chunk_elems(c));
    const int32_t lo = c->col_lo, hi = c->col_hi < 0 ? B : c->col_hi;
    c->chunk_start.assign(1, lo);
    c->t_chunk_max = 0;
    for (int32_t j = 0; j < B; ++j) {
        SubDesc& s = c->subs[j];
        s.col = j;
        s.fptr = c->fcol_ptr[j];
        s.nblk = static_cast<int32_t>(c->fcol_ptr[j + 1] - c->fcol_ptr[j]);
        int32_t acc = 0;
        s.own = -1;
        for (int32_t a = 0; a < s.nblk; ++a) {
            const int32_t r = c->frow_idx[s.fptr + a];
            c->lstart[s.fptr + a] = acc;
            if (r == j) s.own = acc;
            acc += c->bs[r];
        }
        if (s.own < 0) return SMX_ERR_PATTERN;
        s.n = acc;
        s.ld = static_cast<int32_t>(round_up(acc, 4));  // 16-byte aligned FP32 rows
        s.bown = c->bs[j];
        const int64_t t_size = round_up(static_cast<int64_t>(s.n) * s.ld, 32);
        s.x_off = x_off;
        s.t_off = 0;
        if (j >= lo && j < hi) {
            if (t_off > 0 && t_off + t_size > chunk_elems) {  // start a new chunk (staging offsets restart at 0)
                c->chunk_start.push_back(j);
                t_off = 0;
            }
            s.t_off = t_off;
            t_off += t_size;
            c->t_chunk_max = std::max(c->t_chunk_max, t_off);
        }
        x_off += round_up(static_cast<int64_t>(s.n) * s.bown, 32);
        c->max_nblk = std::max(c->max_nblk, s.nblk);
        c->max_n = std::max(c->max_n, s.n);
    }
    c->chunk_start.push_back(hi);
    c->t_elems = c->t_chunk_max;
    c->x_elems = x_off;
    // processing order: largest first within each chunk
    c->order.resize(B);
    for (int32_t j = 0; j < B; ++j) c->order[j] = j;
    for (size_t k = 0; k + 1 < c->chunk_start.size(); ++k)
        std::stable_sort(c->order.begin() + c->chunk_start[k], c->order.begin() + c->chunk_start[k + 1],
                         [&](int32_t x, int32_t y) { return c->subs[x].n > c->subs[y].n; });

    // The block maps of the submatrices (what the shared-memory gather would otherwise build at
    // every gather from the pattern): for submatrices of at most 64 blocks (the gather's staged
    // form), 32-bit value offsets, at most 2^26 entries in all
    c->maps.clear();
    c->map_off.assign(B + 1, 0);
    for (int32_t j = 0; j < B; ++j) {
        const int64_t nb = c->fcol_ptr[j + 1] - c->fcol_ptr[j];
        c->map_off[j + 1] = c->map_off[j] + nb * nb;
    }
    if (c->max_nblk <= 64 && c->map_off[B] <= (int64_t(1) << 26) && c->n_values < (int64_t(1) << 31)) {
        c->maps.assign(static_cast<size_t>(c->map_off[B]), -1);
        for (int32_t j = 0; j < B; ++j) {
            const int32_t* R = c->frow_idx.data() + c->fcol_ptr[j];
            const int32_t nb = static_cast<int32_t>(c->fcol_ptr[j + 1] - c->fcol_ptr[j]);
            int32_t* m = c->maps.data() + c->map_off[j];
            for (int32_t a = 0; a < nb; ++a) {
                const int32_t col = R[a];
                for (int64_t k = c->fcol_ptr[col]; k < c->fcol_ptr[col + 1]; ++k) {
                    const int32_t* f = std::lower_bound(R, R + nb, c->frow_idx[k]);
                    if (f != R + nb && *f == c->frow_idx[k]) m[static_cast<int64_t>(a) * nb + (f - R)] = static_cast<int32_t>(c->fvoff[k]);
                }
            }
        }
        SMX_TRY(upload(c->d_maps, c->maps, st));
        SMX_TRY(upload(c->d_map_off, c->map_off, st));
    }
    SMX_TRY(upload(c->d_fcol_ptr, c->fcol_ptr, st));
    SMX_TRY(upload(c->d_frow_idx, c->frow_idx, st));
    SMX_TRY(upload(c->d_fvoff, c->fvoff, st));
    SMX_TRY(upload(c->d_lstart, c->lstart, st));
    SMX_TRY(upload(c->d_subs, c->subs, st));
    SMX_TRY(upload(c->d_order, c->order, st));
    SMX_TRY(ensure(c->d_T, static_cast<size_t>(c->t_elems) * staging_elem(c)));
    SMX_CUDA(cudaMemsetAsync(c->d_D.p, 0, c->n_values * sizeof(double), st));
    SMX_CUDA(cudaMemsetAsync(c->d_partial.p, 0, sizeof(double2) * B, st));  // columns outside the shard add zero
    SMX_CUDA(cudaMemsetAsync(c->d_iters.p, 0, sizeof(int32_t) * B, st));
    SMX_CUDA(cudaMemcpyAsync(c->d_keep_prev.p, c->d_keep.p, c->nnzb, cudaMemcpyDeviceToDevice, st));
    c->analysed = true;
    c->dirty = false;
    c->ws_prec = -1;  // tensor-core workspace must be re-checked
    return SMX_OK;
}

static smx_status prepare_tc_workspace(smx_ctx* c) {
    const int ld = static_cast<int>(round_up(c->max_n, 64));
    const int slots = std::max(1, std::min(c->num_sms, c->B));
    if (c->ws_prec == c->precision && c->ws_ld >= ld && c->ws_slots == slots) return SMX_OK;
    SMX_TRY(get_encoder(c));
    const size_t bytes = static_cast<size_t>(slots) * 6 * ld * ld * 2;
    SMX_TRY(ensure(c->d_ws, bytes));
    SMX_CUDA(cudaMemsetAsync(c->d_ws.p, 0, bytes, c->stream));
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(ld), static_cast<cuuint64_t>(ld), static_cast<cuuint64_t>(slots) * 6};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * 2, static_cast<cuuint64_t>(ld) * ld * 2};
    cuuint32_t box[3] = {64, 64, 1};
    cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        c->precision == SMX_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUresult r = c->encode(&c->tmap, dt, 3, c->d_ws.p, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return SMX_ERR_CUDA;
    c->ws_ld = ld;
    c->ws_slots = slots;
    c->ws_prec = c->precision;
    return SMX_OK;
}

// Single-pass forms stop at their rounding floor: once ||X^2 - I||_F < 1/2 every eigenvalue
// of X^2 lies within 1/2 of 1, where a Newton-Schulz step shrinks each |lambda^2 - 1| at least
// 2.5-fold; a residual there that does not halve is rounding, not progress.
constexpr float kStallLevel = 0.5f;

static double tau_for(int precision) {
    switch (precision) {
        case SMX_FP64: return 1e-7;
        case SMX_FP16X3: return 2e-3;
        default: return 5e-2;
    }
}

// Adds the device time of the Newton-Schulz launches recorded since the last
// call; the stream must be synchronised.
void accumulate_timers(smx_ctx* c) {
    for (size_t i = 0; i < c->ns_pending; ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->ns_events[i].first, c->ns_events[i].second) == cudaSuccess)
            c->ns_ms_total += ms;
    }
    c->ns_pending = 0;
}

static smx_status ns_event_pair(smx_ctx* c, cudaEvent_t* e0, cudaEvent_t* e1) {
    if (c->ns_pending == c->ns_events.size()) {
        cudaEvent_t a, b;
        SMX_CUDA(cudaEventCreate(&a));
        SMX_CUDA(cudaEventCreate(&b));
        c->ns_events.emplace_back(a, b);
    }
    *e0 = c->ns_events[c->ns_pending].first;
    *e1 = c->ns_events[c->ns_pending].second;
    ++c->ns_pending;
    return SMX_OK;
}

// One build at chemical potential mu (a3 - a8).
// a3 + a4 for block columns [j0, j0 + m) into the staging buffer.
static smx_status gather_chunk(smx_ctx* c, int j0, int m, double mu, const GatherExtras& ex) {
    SMX_TRY(ensure(c->d_T, static_cast<size_t>(c->t_elems) * staging_elem(c)));  // after a precision change
    const PatternView pv = pattern_view(c);
    SubDesc* subs = dp<SubDesc>(c->d_subs);
    if (c->precision == SMX_FP64) {
        SMX_CUDA(launch_gather_bound(subs + j0, m, c->max_nblk, c->max_n, c->bmax, c->bsize_uniform, pv, dp<double>(c->d_H), mu, dp<double>(c->d_T),
                                     dp<double>(c->d_bound) + j0, ex, c->stream));
    } else {
        SMX_CUDA(launch_gather_bound_f32(subs + j0, m, c->max_nblk, c->max_n, c->bmax, c->bsize_uniform, pv, dp<float>(c->d_H32), mu, dp<float>(c->d_T),
                                         dp<double>(c->d_bound) + j0, ex, c->stream));
    }
    c->kernel_launches += 1;
    return SMX_OK;
}

static smx_status read_status(smx_ctx* c);

// Setup of the non-orthogonal form for the current (H, S) and filtered pattern:
// A_S and A_H gathered without shift, L_j = A_S^-1/2 and M_j = L_j A_H L_j kept
// for every block column, and the bisection bracket from the Gershgorin
// intervals of the M_j.  Synchronous (reads the bracket back).
static smx_status nonorth_setup(smx_ctx* c) {
    if (c->chunk_start.size() != 2) return SMX_ERR_UNSUPPORTED;  // L_j and M_j of every column stay resident
    cudaStream_t st = c->stream;
    const size_t tb = static_cast<size_t>(c->t_elems) * sizeof(double);
    SMX_TRY(ensure(c->d_T, tb));
    SMX_TRY(ensure(c->d_W1, tb));
    SMX_TRY(ensure(c->d_W2, tb));
    SMX_TRY(ensure(c->d_W3, tb));
    SMX_TRY(ensure(c->d_Lc, tb));
    SMX_TRY(ensure(c->d_Mc, tb));
    SMX_TRY(ensure(c->d_nlohi, sizeof(double) * 2 * c->B));
    SMX_TRY(ensure(c->d_setup_iters, sizeof(int32_t) * c->B));
    const int j0 = c->chunk_start[0], m = c->chunk_start[1] - j0;
    const PatternView pv = pattern_view(c);
    SubDesc* subs = dp<SubDesc>(c->d_subs) + j0;
    GatherExtras ex;
    SMX_CUDA(launch_gather_bound(subs, m, c->max_nblk, c->max_n, c->bmax, c->bsize_uniform, pv, dp<double>(c->d_S), 0.0, dp<double>(c->d_Lc),
                                 dp<double>(c->d_bound) + j0, ex, st));
    SMX_CUDA(launch_gather_bound(subs, m, c->max_nblk, c->max_n, c->bmax, c->bsize_uniform, pv, dp<double>(c->d_H), 0.0, dp<double>(c->d_Mc),
                                 dp<double>(c->d_gersh) + j0, ex, st));
    NonorthSetupArgs a;
    a.subs = subs;
    a.n_subs = m;
    a.Lc = dp<double>(c->d_Lc);
    a.Mc = dp<double>(c->d_Mc);
    a.T = dp<double>(c->d_T);
    a.W1 = dp<double>(c->d_W1);
    a.W2 = dp<double>(c->d_W2);
    a.W3 = dp<double>(c->d_W3);
    a.bound_s = dp<double>(c->d_bound) + j0;
    a.tau = tau_for(SMX_FP64);
    a.max_iter = 100;
    a.iters = dp<int32_t>(c->d_setup_iters);
    a.lohi = dp<double>(c->d_nlohi);
    a.status = &scalars(c)->status;
    SMX_CUDA(launch_nonorth_setup(a, st));
    c->kernel_launches += 3;
    std::vector<double> lohi(2 * static_cast<size_t>(m));
    SMX_CUDA(cudaMemcpyAsync(lohi.data(), c->d_nlohi.p, sizeof(double) * lohi.size(), cudaMemcpyDeviceToHost, st));
    const smx_status ds = read_status(c);  // synchronises
    if (ds != SMX_OK) return ds;
    double lo = lohi[0], hi = lohi[1];
    for (int j = 1; j < m; ++j) {
        lo = std::min(lo, lohi[2 * j]);
        hi = std::max(hi, lohi[2 * j + 1]);
    }
    if (!std::isfinite(lo) || !std::isfinite(hi)) return SMX_ERR_NONFINITE;
    c->nbr_lo = lo;
    c->nbr_hi = hi;
    c->nonorth_ready = true;
    return SMX_OK;
}

// mu_dev: when set, the gather reads mu from this device address (the midpoint the filter just
// computed, or the device-side bisection's current one) instead of the argument.  skip: when
// set, every kernel of the build returns at once if *skip is non-zero at its launch (the steps
// after the stopping step of a device-side bisection).
static smx_status build_at(smx_ctx* c, double mu, const double* mu_dev = nullptr, const int* skip = nullptr) {
    NvtxRange nv("smx build");
    if (c->function != SMX_FN_DENSITY && c->precision != SMX_FP64) return SMX_ERR_UNSUPPORTED;
    if (c->have_S && (c->function != SMX_FN_DENSITY || c->precision != SMX_FP64 || mu_dev))
        return SMX_ERR_UNSUPPORTED;  // the non-orthogonal form: density matrix, FP64
    if (c->symmetrize && c->col_hi >= 0) return SMX_ERR_UNSUPPORTED;  // a shard holds only its columns of D
    if (c->dirty || !c->analysed) SMX_TRY(analyse(c));
    if (c->have_S && !c->nonorth_ready) SMX_TRY(nonorth_setup(c));
    cudaStream_t st = c->stream;
    const int B = c->B;
    DevScalars* sc = scalars(c);
    const bool model = c->model_on && c->function == SMX_FN_DENSITY && !c->have_S;  // other forms start from G_j
    SMX_CUDA(cudaEventRecord(c->ev0, st));
    const PatternView pv = pattern_view(c);
    if (c->precision == SMX_FP64) {
        const size_t tb = static_cast<size_t>(c->t_elems) * sizeof(double);
        SMX_TRY(ensure(c->d_T, tb));
        SMX_TRY(ensure(c->d_W1, tb));
        SMX_TRY(ensure(c->d_W2, tb));
        if (c->function != SMX_FN_DENSITY) SMX_TRY(ensure(c->d_W3, tb));
        if (c->function == SMX_FN_FERMI) SMX_TRY(ensure(c->d_W4, tb));
    } else {
        SMX_TRY(prepare_tc_workspace(c));
        SMX_TRY(ensure(c->d_xown, static_cast<size_t>(c->x_elems) * sizeof(float)));
        if (c->fp64_final > 0) {  // the bulk phase's last iterate in FP64, and two work buffers
            const size_t tb = static_cast<size_t>(c->t_elems) * sizeof(double);
            SMX_TRY(ensure(c->d_W1, tb));
            SMX_TRY(ensure(c->d_W2, tb));
            SMX_TRY(ensure(c->d_W3, tb));
        }
    }
    SubDesc* subs = dp<SubDesc>(c->d_subs);
    // one pass of a3-a7 per chunk of block columns (the staging of T_j is reused)
    for (size_t k = 0; k + 1 < c->chunk_start.size(); ++k) {
        const int j0 = c->chunk_start[k], m = c->chunk_start[k + 1] - j0;
        GatherExtras ex;
        ex.gersh = dp<double>(c->d_gersh) + j0;
        ex.mu_dev = mu_dev;
        ex.skip = skip;
        if (model) {  // learned bound: features and prediction inside the gather (checked in the NS kernel)
            ex.prev_ratio = dp<float>(c->d_prev_ratio) + j0;
            ex.params = dp<float>(c->d_params);
            ex.margin = kModelMargin;
            if (c->model_gap) ex.pred = dp<float>(c->d_pred) + 2 * j0;  // 2 per column
        }
        if (!c->have_S) SMX_TRY(gather_chunk(c, j0, m, mu, ex));  // the non-orthogonal form starts from M_j
        cudaEvent_t ns0, ns1;
        SMX_TRY(ns_event_pair(c, &ns0, &ns1));
        if (c->precision == SMX_FP64) {
            NsFp64Args a;
            a.subs = subs + j0;
            a.n_subs = m;
            a.T = dp<double>(c->d_T);
            a.W1 = dp<double>(c->d_W1);
            a.W2 = dp<double>(c->d_W2);
            a.W3 = c->function != SMX_FN_DENSITY ? dp<double>(c->d_W3) : nullptr;
            a.W4 = c->function == SMX_FN_FERMI ? dp<double>(c->d_W4) : nullptr;
            a.beta = c->beta;
            a.function = c->function;
            a.bound = dp<double>(c->d_bound) + j0;
            a.tau = tau_for(SMX_FP64);
            a.max_iter = 100;
            a.iters = dp<int32_t>(c->d_iters);
            a.work_n3 = dp<unsigned long long>(c->d_work_n3);
            a.gersh = dp<double>(c->d_gersh) + j0;
            a.sq_ratio = dp<float>(c->d_sq_ratio) + j0;
            a.use_model = model ? 1 : 0;
            if (model && c->model_gap) a.pred = dp<float>(c->d_pred) + 2 * j0;
            a.skip = skip;
            a.fallbacks = &sc->fallbacks;
            a.status = &sc->status;
            a.pv = pv;
            a.H = dp<double>(c->d_H);
            a.D = dp<double>(c->d_D);
            a.partial = dp<double2>(c->d_partial);
            if (c->have_S) {
                a.Mc = dp<double>(c->d_Mc);
                a.Lc = dp<double>(c->d_Lc);
                a.Sv = dp<double>(c->d_S);
                a.mu = mu;
            }
            SMX_CUDA(cudaEventRecord(ns0, st));
            SMX_CUDA(launch_ns_fp64(a, c->max_nblk, st));
            SMX_CUDA(cudaEventRecord(ns1, st));
        } else {
            NsTcArgs a;
            a.subs = subs;  // indexed by block column through the order slice
            a.order = dp<int32_t>(c->d_order) + j0;
            a.n_subs = m;
            a.work_counter = &sc->ns_counter;
            a.T = dp<float>(c->d_T);
            a.bound = dp<double>(c->d_bound);
            a.ws = c->d_ws.p;
            a.ld = c->ws_ld;
            a.n_slots = std::min(c->ws_slots, m);
            a.tau = static_cast<float>(tau_for(c->precision));
            a.stall_level = (c->precision == SMX_FP16 || c->precision == SMX_BF16) ? kStallLevel : 0.0f;
            a.max_iter = 100;
            a.iters = dp<int32_t>(c->d_iters);
            a.work_n3 = dp<unsigned long long>(c->d_work_n3);
            a.gersh = dp<double>(c->d_gersh);
            a.sq_ratio = dp<float>(c->d_sq_ratio);
            a.use_model = model ? 1 : 0;
            if (model && c->model_gap) a.pred = dp<float>(c->d_pred);
            a.skip = skip;
            a.fallbacks = &sc->fallbacks;
            a.status = &sc->status;
            a.pv = pv;
            a.H = dp<double>(c->d_H);
            a.D = dp<double>(c->d_D);
            a.partial = dp<double2>(c->d_partial);
            a.xown = dp<float>(c->d_xown);
            const bool finish = c->fp64_final > 0 && c->function == SMX_FN_DENSITY;
            if (finish) a.xfull = dp<double>(c->d_W1);
            SMX_CUDA(cudaEventRecord(ns0, st));
            SMX_CUDA(launch_ns_tc(a, c->precision, c->tmap, c->max_nblk, st));
            if (finish) {
                // FP64 finishing steps on the bulk phase's last iterate, then the scatter (the
                // tensor-core scatter, which also resets the job counter, is not run)
                SMX_CUDA(cudaMemsetAsync(&sc->ns_counter, 0, sizeof(int), st));
                NsFp64Args f;
                f.subs = subs + j0;
                f.n_subs = m;
                f.T = dp<double>(c->d_W1);
                f.W1 = dp<double>(c->d_W2);
                f.W2 = dp<double>(c->d_W3);
                f.W3 = nullptr;
                f.function = SMX_FN_DENSITY;
                f.bound = dp<double>(c->d_bound) + j0;
                f.tau = tau_for(SMX_FP64);
                f.max_iter = c->fp64_final;
                f.iters = dp<int32_t>(c->d_iters);
                f.work_n3 = dp<unsigned long long>(c->d_work_n3);
                f.gersh = dp<double>(c->d_gersh) + j0;
                f.sq_ratio = dp<float>(c->d_sq_ratio) + j0;
                f.use_model = 0;
                f.fallbacks = &sc->fallbacks;
                f.status = &sc->status;
                f.pv = pv;
                f.H = dp<double>(c->d_H);
                f.D = dp<double>(c->d_D);
                f.partial = dp<double2>(c->d_partial);
                f.finish_iters = c->fp64_final;
                f.skip = skip;
                SMX_CUDA(launch_ns_fp64(f, c->max_nblk, st));
                c->kernel_launches += 1;
            }
            SMX_CUDA(cudaEventRecord(ns1, st));
            if (!finish) {
                SMX_CUDA(launch_scatter_owner(subs + j0, m, c->max_nblk, c->max_n, c->bmax, c->bsize_uniform, pv, dp<float>(c->d_xown), dp<float>(c->d_H32),
                                              dp<double>(c->d_D), dp<double2>(c->d_partial), B, sc, st, skip));
                c->kernel_launches += 1;
            }
        }
        c->kernel_launches += 1;
        c->ns_launches += 1;
    }
    if (c->precision == SMX_FP64 || (c->fp64_final > 0 && c->function == SMX_FN_DENSITY)) {
        // the tensor-core scatter sums the partials itself
        SMX_CUDA(launch_reduce(dp<double2>(c->d_partial), B, sc, st, skip));
        c->kernel_launches += 1;
    }
    if (c->symmetrize) {  // after the sums: trace and energy are those of D as built
        SMX_CUDA(launch_symmetrize(dp<SymPair>(c->d_pairs), c->n_pairs, dp<uint8_t>(c->d_keep), dp<double>(c->d_D), st,
                                   skip));
        c->kernel_launches += 1;
    }
    SMX_CUDA(cudaEventRecord(c->ev1, st));
    c->sq_valid = true;
    c->built = true;
    c->last_mu = mu;
    return SMX_OK;
}

static smx_status read_status(smx_ctx* c) {
    SMX_TRY(fetch(c));
    return static_cast<smx_status>(c->h_sc->status);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* smx_status_string(smx_status s) {
    switch (s) {
        case SMX_OK: return "ok";
        case SMX_ERR_ARG: return "invalid argument";
        case SMX_ERR_PATTERN: return "malformed block pattern";
        case SMX_ERR_NONFINITE: return "non-finite value";
        case SMX_ERR_CUDA: return "CUDA error";
        case SMX_ERR_OOM: return "device out of memory";
        case SMX_ERR_NOCONV: return "Newton-Schulz did not converge";
        case SMX_ERR_NOBRACKET: return "electron count outside [0, N]";
        case SMX_ERR_TIMEOUT: return "device wait timed out";
        case SMX_ERR_STATE: return "invalid call order";
        case SMX_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

smx_status smx_create(smx_ctx** out, int32_t n_block_cols, const int32_t* block_size, const int64_t* col_ptr,
                      const int32_t* row_idx, const double* values, void* cuda_stream) {
    if (!out) return SMX_ERR_ARG;
    *out = nullptr;
    if (n_block_cols < 1 || !block_size || !col_ptr || !row_idx || !values) return SMX_ERR_ARG;
    SMX_TRY(validate_pattern(n_block_cols, block_size, col_ptr, row_idx));
    smx_ctx* c = new (std::nothrow) smx_ctx();
    if (!c) return SMX_ERR_OOM;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) c->mem_total = total_b;
    }
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->B = n_block_cols;
    c->bs.assign(block_size, block_size + n_block_cols);
    c->bmax = *std::max_element(c->bs.begin(), c->bs.end());
    c->bsize_uniform = *std::min_element(c->bs.begin(), c->bs.end()) == c->bmax;
    c->col_ptr.assign(col_ptr, col_ptr + n_block_cols + 1);
    c->nnzb = col_ptr[n_block_cols];
    c->row_idx.assign(row_idx, row_idx + c->nnzb);
    c->voff.assign(c->nnzb + 1, 0);
    c->row_start.assign(n_block_cols + 1, 0);
    for (int32_t j = 0; j < n_block_cols; ++j) c->row_start[j + 1] = c->row_start[j] + block_size[j];
    c->N = c->row_start[n_block_cols];
    for (int32_t j = 0; j < n_block_cols; ++j)
        for (int64_t k = col_ptr[j]; k < col_ptr[j + 1]; ++k)
            c->voff[k + 1] = c->voff[k] + static_cast<int64_t>(block_size[row_idx[k]]) * block_size[j];
    c->n_values = c->voff[c->nnzb];
    for (int32_t j = 0; j < n_block_cols; ++j)
        c->max_col_blocks = std::max(c->max_col_blocks, static_cast<int32_t>(col_ptr[j + 1] - col_ptr[j]));
    smx_status s = SMX_OK;
    auto fail = [&](smx_status e) {
        smx_destroy(c);
        return e;
    };
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) return fail(SMX_ERR_CUDA);
    if ((s = upload(c->d_voff, c->voff, c->stream)) != SMX_OK) return fail(s);
    if ((s = upload(c->d_row_idx, c->row_idx, c->stream)) != SMX_OK) return fail(s);
    if ((s = upload(c->d_col_ptr, c->col_ptr, c->stream)) != SMX_OK) return fail(s);
    if ((s = upload(c->d_bs, c->bs, c->stream)) != SMX_OK) return fail(s);
    const size_t vb = static_cast<size_t>(c->n_values) * sizeof(double);
    if ((s = ensure(c->d_H, vb)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_H32, vb / 2)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_D, vb)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_keep, c->nnzb)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_keep_prev, c->nnzb)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_sc, sizeof(DevScalars))) != SMX_OK) return fail(s);
    if (cudaMallocHost(&c->h_sc, sizeof(DevScalars)) != cudaSuccess) return fail(SMX_ERR_OOM);
    if (cudaMemsetAsync(c->d_sc.p, 0, sizeof(DevScalars), c->stream) != cudaSuccess) return fail(SMX_ERR_CUDA);
    if ((s = ensure(c->d_bound, sizeof(double) * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_iters, sizeof(int32_t) * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_partial, sizeof(double2) * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_work_n3, sizeof(unsigned long long))) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_gersh, sizeof(double) * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_sq_ratio, sizeof(float) * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_prev_ratio, sizeof(float) * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_feat, sizeof(float) * kModelFeatures * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_pred, sizeof(float) * 2 * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_labels, sizeof(float) * 2 * n_block_cols)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_loss, sizeof(float))) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_params, sizeof(float) * kModelParams)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_mst, sizeof(float) * kModelParams)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_vst, sizeof(float) * kModelParams)) != SMX_OK) return fail(s);
    if ((s = ensure(c->d_grad, sizeof(float) * kModelParams)) != SMX_OK) return fail(s);
    if (cudaMemsetAsync(c->d_prev_ratio.p, 0, sizeof(float) * n_block_cols, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_sq_ratio.p, 0, sizeof(float) * n_block_cols, c->stream) != cudaSuccess)
        return fail(SMX_ERR_CUDA);
    if (cudaMemsetAsync(c->d_work_n3.p, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) return fail(SMX_ERR_CUDA);
    if (cudaMallocHost(&c->h_keep_pinned, c->nnzb > 0 ? c->nnzb : 1) != cudaSuccess) return fail(SMX_ERR_OOM);
    if (cudaMemcpyAsync(c->d_H.p, values, vb, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) return fail(SMX_ERR_CUDA);
    if (cudaMemsetAsync(c->d_iters.p, 0, sizeof(int32_t) * n_block_cols, c->stream) != cudaSuccess)
        return fail(SMX_ERR_CUDA);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(SMX_ERR_CUDA);
    *out = c;
    return SMX_OK;
}

smx_status smx_set_values(smx_ctx* c, const double* values, int32_t on_device) {
    if (!c || !values) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    SMX_CUDA(cudaMemcpyAsync(c->d_H.p, values, static_cast<size_t>(c->n_values) * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (c->sq_valid) {  // the ratio of the last build becomes the previous-step feature
        SMX_CUDA(cudaMemcpyAsync(c->d_prev_ratio.p, c->d_sq_ratio.p, sizeof(float) * c->B, cudaMemcpyDeviceToDevice,
                                 c->stream));
        c->sq_valid = false;
    }
    c->dirty = true;
    c->built = false;
    return SMX_OK;
}

smx_status smx_set_filter_threshold(smx_ctx* c, double eps) {
    if (!c || !(eps >= 0.0) || !std::isfinite(eps)) return SMX_ERR_ARG;
    if (eps != c->eps) {
        c->eps = eps;
        c->dirty = true;
        c->analysed = false;  // force the keep flags to be read back
    }
    return SMX_OK;
}

smx_status smx_set_staging_limit(smx_ctx* c, uint64_t bytes) {
    if (!c || bytes < (uint64_t(1) << 20)) return SMX_ERR_ARG;
    if (bytes != c->staging_limit) {
        c->staging_limit = static_cast<size_t>(bytes);
        c->dirty = true;
        c->analysed = false;  // re-chunk
    }
    return SMX_OK;
}

smx_status smx_set_column_range(smx_ctx* c, int32_t j0, int32_t j1) {
    if (!c || j0 < 0 || j1 > c->B || j0 >= j1) return SMX_ERR_ARG;
    const int32_t hi = (j0 == 0 && j1 == c->B) ? -1 : j1;
    if (j0 != c->col_lo || hi != c->col_hi) {
        c->col_lo = j0;
        c->col_hi = hi;
        c->dirty = true;
        c->analysed = false;
        c->built = false;
    }
    return SMX_OK;
}

smx_status smx_get_gershgorin_interval(smx_ctx* c, double* lo, double* hi) {
    if (!c || !lo || !hi) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    if (c->dirty || !c->analysed) SMX_TRY(analyse(c));  // the bracket comes with the filter
    if (c->have_S) {
        // the non-orthogonal form brackets mu by the Gershgorin intervals of its M_j, known only
        // for the context's own block columns: no common bracket for shards
        if (c->col_hi >= 0 || c->precision != SMX_FP64) return SMX_ERR_UNSUPPORTED;
        if (!c->nonorth_ready) SMX_TRY(nonorth_setup(c));
        *lo = c->nbr_lo;
        *hi = c->nbr_hi;
        return SMX_OK;
    }
    *lo = c->br_lo;
    *hi = c->br_hi;
    return SMX_OK;
}

smx_status smx_set_mu(smx_ctx* c, double mu) {
    if (!c || !std::isfinite(mu)) return SMX_ERR_ARG;
    c->mu = mu;
    return SMX_OK;
}

smx_status smx_set_electron_count(smx_ctx* c, double n_e, int32_t max_steps, double tol) {
    if (!c || !std::isfinite(n_e) || max_steps < 1 || max_steps > 200 || !(tol >= 0.0)) return SMX_ERR_ARG;
    c->have_ne = true;
    c->n_e = n_e;
    c->max_steps = max_steps;
    c->tol = tol;
    return SMX_OK;
}

smx_status smx_set_precision(smx_ctx* c, smx_precision bulk, int32_t fp64_final_iters) {
    if (!c) return SMX_ERR_ARG;
    if (bulk != SMX_FP64 && bulk != SMX_FP16X3 && bulk != SMX_FP16 && bulk != SMX_BF16) return SMX_ERR_ARG;
    if (fp64_final_iters < 0 || fp64_final_iters > 4) return SMX_ERR_ARG;
    if (bulk == SMX_FP64) fp64_final_iters = 0;  // the plain form is FP64 throughout
    c->precision = bulk;
    c->fp64_final = fp64_final_iters;
    // with the automatic staging limit the chunks follow the staged element size
    if (!c->staging_limit && c->chunk_elem && c->chunk_elem != staging_elem(c)) c->analysed = false;
    return SMX_OK;
}

smx_status smx_set_overlap(smx_ctx* c, const double* values, int32_t on_device) {
    if (!c) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    c->nonorth_ready = false;
    c->built = false;
    if (!values) {
        c->have_S = false;
        release(c->d_Lc);
        release(c->d_Mc);
        return SMX_OK;
    }
    if (!on_device)
        for (int64_t i = 0; i < c->n_values; ++i)
            if (!std::isfinite(values[i])) return SMX_ERR_NONFINITE;
    SMX_TRY(ensure(c->d_S, static_cast<size_t>(c->n_values) * sizeof(double)));
    SMX_CUDA(cudaMemcpyAsync(c->d_S.p, values, static_cast<size_t>(c->n_values) * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    c->have_S = true;
    return SMX_OK;
}

smx_status smx_set_function(smx_ctx* c, smx_function f) {
    if (!c || (f != SMX_FN_DENSITY && f != SMX_FN_INV_SQRT && f != SMX_FN_SQRT && f != SMX_FN_INV &&
               f != SMX_FN_FERMI))
        return SMX_ERR_ARG;
    c->function = f;
    return SMX_OK;
}

smx_status smx_set_fermi_beta(smx_ctx* c, double beta) {
    if (!c || !std::isfinite(beta) || beta < 0.0) return SMX_ERR_ARG;
    c->beta = beta;
    return SMX_OK;
}

smx_status smx_set_symmetrize(smx_ctx* c, int32_t enable) {
    if (!c) return SMX_ERR_ARG;
    if (enable && c->col_hi >= 0) return SMX_ERR_UNSUPPORTED;  // a shard holds only its own columns of D
    if (enable && c->n_pairs < 0) {
        // block k = (r, j) with r <= j and its transpose; the input pattern is symmetric with
        // sorted rows (checked at creation), so the partner is found by bisection
        std::vector<SymPair> pairs;
        for (int32_t j = 0; j < c->B; ++j) {
            for (int64_t k = c->col_ptr[j]; k < c->col_ptr[j + 1]; ++k) {
                const int32_t r = c->row_idx[k];
                if (r > j) break;
                const int32_t* b0 = c->row_idx.data() + c->col_ptr[r];
                const int32_t* b1 = c->row_idx.data() + c->col_ptr[r + 1];
                const int32_t* f = std::lower_bound(b0, b1, j);
                if (f == b1 || *f != j) return SMX_ERR_PATTERN;
                SymPair p;
                p.k = static_cast<int32_t>(k);
                p.kt = static_cast<int32_t>(f - c->row_idx.data());
                p.off_k = c->voff[k];
                p.off_kt = c->voff[p.kt];
                p.br = c->bs[r];
                p.bj = c->bs[j];
                pairs.push_back(p);
            }
        }
        DeviceGuard g(c->device);
        SMX_TRY(upload(c->d_pairs, pairs, c->stream));
        SMX_CUDA(cudaStreamSynchronize(c->stream));
        c->n_pairs = static_cast<int32_t>(pairs.size());
    }
    c->symmetrize = enable != 0;
    c->built = false;
    return SMX_OK;
}

smx_status smx_build_density(smx_ctx* c) {
    if (!c) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    c->bisection_steps = 0;
    SMX_TRY(reset_flags(c));
    return build_at(c, c->mu);
}

smx_status smx_solve_mu(smx_ctx* c) {
    if (!c) return SMX_ERR_ARG;
    if (!c->have_ne || c->col_hi >= 0) return SMX_ERR_STATE;  // a shard's trace is partial
    if (c->function != SMX_FN_DENSITY) return SMX_ERR_STATE;  // bisection on the density matrix only
    DeviceGuard g(c->device);
    if (c->n_e < 0.0 || c->n_e > static_cast<double>(c->N)) return SMX_ERR_NOBRACKET;
    SMX_TRY(reset_flags(c));
    c->bisection_steps = 0;
    double lo = 0.0, hi = 0.0;
    int step = 0;
    if (c->analysed && c->dirty && !c->have_S) {
        // New values on a known pattern: the filter and the first bisection step (at the
        // midpoint the filter leaves on the device, on the current filtered pattern) go
        // out together and come back in one read.  If the filter changed the pattern,
        // the step is discarded and taken again on the new one.
        SMX_TRY(launch_filter(c));
        c->dirty = false;  // the build below runs on the current filtered pattern
        SMX_TRY(build_at(c, 0.0, &scalars(c)->mu0));
        SMX_TRY(fetch(c));
        const bool changed = c->filter_compared && c->h_sc->changed != 0;
        SMX_TRY(after_filter(c));  // errors of the filter, bracket, compaction when changed
        lo = c->br_lo;
        hi = c->br_hi;
        c->bisection_steps = 1;
        if (changed) {
            SMX_TRY(reset_flags(c));  // the step is taken again on the new pattern
        } else {
            c->last_mu = c->h_sc->mu0;  // the device's 0.5 (lo + hi)
            step = 1;
            if (c->h_sc->status != SMX_OK) return static_cast<smx_status>(c->h_sc->status);
            const double tr = c->h_sc->trace;
            if (std::fabs(tr - c->n_e) <= c->tol) return SMX_OK;
            if (tr < c->n_e) lo = c->last_mu; else hi = c->last_mu;
        }
    } else {
        if (c->dirty || !c->analysed) SMX_TRY(analyse(c));  // the bracket comes with the filter
        lo = c->br_lo;
        hi = c->br_hi;
        if (c->have_S) {  // the pencil's bracket comes with the setup
            if (c->function != SMX_FN_DENSITY || c->precision != SMX_FP64) return SMX_ERR_UNSUPPORTED;
            if (!c->nonorth_ready) SMX_TRY(nonorth_setup(c));
            lo = c->nbr_lo;
            hi = c->nbr_hi;
        }
    }
    for (; step < c->max_steps; ++step) {
        NvtxRange nv("smx bisection step");
        const double mid = 0.5 * (lo + hi);
        SMX_TRY(build_at(c, mid));
        ++c->bisection_steps;
        const smx_status ds = read_status(c);
        if (ds != SMX_OK) return ds;
        const double tr = c->h_sc->trace;
        if (std::fabs(tr - c->n_e) <= c->tol) break;
        if (tr < c->n_e) lo = mid; else hi = mid;
    }
    return SMX_OK;
}

smx_status smx_solve_mu_device(smx_ctx* c) {
    if (!c) return SMX_ERR_ARG;
    if (!c->have_ne || c->col_hi >= 0) return SMX_ERR_STATE;
    if (c->function != SMX_FN_DENSITY) return SMX_ERR_STATE;
    if (c->have_S) return SMX_ERR_UNSUPPORTED;  // the non-orthogonal form: smx_solve_mu
    DeviceGuard g(c->device);
    if (c->n_e < 0.0 || c->n_e > static_cast<double>(c->N)) return SMX_ERR_NOBRACKET;
    SMX_TRY(reset_flags(c));
    c->bisection_steps = 0;
    // the filtered pattern and its bracket first (one read when the values are new)
    if (c->dirty || !c->analysed) SMX_TRY(analyse(c));
    DevScalars* sc = scalars(c);
    SMX_CUDA(launch_bisect_init(sc, c->br_lo, c->br_hi, c->stream));
    c->kernel_launches += 1;
    for (int step = 0; step < c->max_steps; ++step) {
        SMX_TRY(build_at(c, 0.0, &sc->bis_mid, &sc->bis_done));
        SMX_CUDA(launch_bisect_step(sc, c->n_e, c->tol, c->max_steps, c->stream));
        c->kernel_launches += 1;
    }
    SMX_TRY(fetch(c));  // the one read of the solve
    c->bisection_steps = c->h_sc->bis_steps;
    c->last_mu = c->h_sc->bis_mid;
    return static_cast<smx_status>(c->h_sc->status);
}

smx_status smx_get_trace(smx_ctx* c, double* trace_D, double* trace_DH, double* mu) {
    if (!c) return SMX_ERR_ARG;
    if (!c->built) return SMX_ERR_STATE;
    DeviceGuard g(c->device);
    const smx_status ds = read_status(c);
    if (ds != SMX_OK) return ds;
    if (trace_D) *trace_D = c->h_sc->trace;
    if (trace_DH) *trace_DH = c->h_sc->energy;
    if (mu) *mu = c->last_mu;
    return SMX_OK;
}

smx_status smx_get_density(smx_ctx* c, double* values_out, int32_t on_device) {
    if (!c || !values_out) return SMX_ERR_ARG;
    if (!c->built) return SMX_ERR_STATE;
    DeviceGuard g(c->device);
    SMX_CUDA(cudaMemcpyAsync(values_out, c->d_D.p, static_cast<size_t>(c->n_values) * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) return read_status(c);
    return SMX_OK;
}

smx_status smx_get_pattern(smx_ctx* c, int64_t* col_ptr, int32_t* row_idx) {
    if (!c) return SMX_ERR_ARG;
    if (!c->analysed) return SMX_ERR_STATE;
    if (col_ptr) std::copy(c->fcol_ptr.begin(), c->fcol_ptr.end(), col_ptr);
    if (row_idx) std::copy(c->frow_idx.begin(), c->frow_idx.end(), row_idx);
    return SMX_OK;
}

smx_status smx_get_submatrix_info(smx_ctx* c, int32_t* dims, int32_t* iters, double* bounds) {
    if (!c) return SMX_ERR_ARG;
    if (!c->built) return SMX_ERR_STATE;
    DeviceGuard g(c->device);
    if (iters) SMX_CUDA(cudaMemcpyAsync(iters, c->d_iters.p, sizeof(int32_t) * c->B, cudaMemcpyDeviceToHost, c->stream));
    if (bounds) SMX_CUDA(cudaMemcpyAsync(bounds, c->d_bound.p, sizeof(double) * c->B, cudaMemcpyDeviceToHost, c->stream));
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    if (dims)
        for (int32_t j = 0; j < c->B; ++j) dims[j] = c->subs[j].n;
    return SMX_OK;
}

smx_status smx_get_stats(smx_ctx* c, smx_stats* out) {
    if (!c || !out) return SMX_ERR_ARG;
    if (!c->built) return SMX_ERR_STATE;
    DeviceGuard g(c->device);
    std::vector<int32_t> it(c->B);
    unsigned long long work = 0;
    SMX_CUDA(cudaMemcpyAsync(it.data(), c->d_iters.p, sizeof(int32_t) * c->B, cudaMemcpyDeviceToHost, c->stream));
    SMX_CUDA(cudaMemcpyAsync(&work, c->d_work_n3.p, sizeof(work), cudaMemcpyDeviceToHost, c->stream));
    SMX_TRY(fetch(c));
    const int fallbacks = c->h_sc->fallbacks;
    std::memset(out, 0, sizeof(*out));
    out->n_block_cols = c->B;
    const int32_t lo = c->col_lo, hi = c->col_hi < 0 ? c->B : c->col_hi;
    out->n = c->N;
    out->nnzb_input = c->nnzb;
    out->nnzb_filtered = static_cast<int64_t>(c->frow_idx.size());
    out->dim_min = 1 << 30;
    out->iters_min = 1 << 30;
    double dsum = 0.0, isum = 0.0, flops = 0.0;
    int noconv = 0;
    for (int32_t j = lo; j < hi; ++j) {  // the context's block columns
        const int n = c->subs[j].n;
        out->dim_min = std::min(out->dim_min, n);
        out->dim_max = std::max(out->dim_max, n);
        out->iters_min = std::min(out->iters_min, it[j]);
        out->iters_max = std::max(out->iters_max, it[j]);
        dsum += n;
        isum += it[j];
        // two products per step for the sign iteration, three for the coupled one of the function forms
        flops += (c->function == SMX_FN_DENSITY ? 4.0 : c->function == SMX_FN_FERMI ? 2.0 : 6.0) * n *
                 static_cast<double>(n) * n * it[j];
        // the iteration cap of the sign and coupled iterations (the Fermi form counts products;
        // FP64 finishing steps come on top of the bulk phase's count)
        const int capped = it[j] - (c->precision != SMX_FP64 && c->function == SMX_FN_DENSITY ? c->fp64_final : 0);
        if (c->function != SMX_FN_FERMI && capped >= 100) ++noconv;
    }
    out->dim_mean = dsum / (hi - lo);
    out->iters_mean = isum / (hi - lo);
    out->n_noconv = noconv;
    out->n_bound_fallback = fallbacks;
    out->bisection_steps = c->bisection_steps;
    out->flops_ns = flops;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) out->ms_last_build = ms;
    out->mu = c->last_mu;
    out->precision = c->precision;
    out->fp64_final_iters = c->fp64_final;
    out->kernel_launches = c->kernel_launches;
    out->ns_launches = c->ns_launches;
    out->ns_ms_total = c->ns_ms_total;
    out->ns_work_n3 = static_cast<double>(work);
    return SMX_OK;
}

smx_status smx_selftest_wait_timeout(smx_ctx* c, uint32_t poll_limit) {
    if (!c || poll_limit == 0 || poll_limit > kSpinLimit) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    SMX_TRY(reset_flags(c));
    SMX_CUDA(launch_wait_selftest(&scalars(c)->status, poll_limit, nullptr, c->stream));
    c->kernel_launches += 1;
    return read_status(c);
}

smx_status smx_reset_counters(smx_ctx* c) {
    if (!c) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    c->ns_pending = 0;
    c->kernel_launches = 0;
    c->ns_launches = 0;
    c->ns_ms_total = 0.0;
    SMX_CUDA(cudaMemsetAsync(c->d_work_n3.p, 0, sizeof(unsigned long long), c->stream));
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    return SMX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// learned spectral bound
// ---------------------------------------------------------------------------

static uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static smx_status model_upload(smx_ctx* c, const std::vector<float>& p) {
    SMX_CUDA(cudaMemcpyAsync(c->d_params.p, p.data(), sizeof(float) * kModelParams, cudaMemcpyHostToDevice, c->stream));
    SMX_CUDA(cudaMemsetAsync(c->d_mst.p, 0, sizeof(float) * kModelParams, c->stream));
    SMX_CUDA(cudaMemsetAsync(c->d_vst.p, 0, sizeof(float) * kModelParams, c->stream));
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    c->adam_t = 0;
    c->model_ready = true;
    return SMX_OK;
}

// Per chunk of block columns: gather T (staging of the context's precision),
// the Gershgorin bound and the features (d_feat) at the fixed mu, the model's
// predictions (d_pred) when asked, and, when lanczos_steps > 0, the Lanczos
// labels (d_labels) of every submatrix.
static smx_status features_labels(smx_ctx* c, int32_t lanczos_steps, bool predict) {
    if (c->dirty || !c->analysed) SMX_TRY(analyse(c));
    const bool f32 = c->precision != SMX_FP64;
    SubDesc* subs = dp<SubDesc>(c->d_subs);
    for (size_t k = 0; k + 1 < c->chunk_start.size(); ++k) {
        const int j0 = c->chunk_start[k], m = c->chunk_start[k + 1] - j0;
        GatherExtras ex;
        ex.gersh = dp<double>(c->d_gersh) + j0;
        ex.prev_ratio = dp<float>(c->d_prev_ratio) + j0;
        ex.feat = dp<float>(c->d_feat) + kModelFeatures * j0;
        if (predict) {
            ex.params = dp<float>(c->d_params);
            ex.pred = dp<float>(c->d_pred) + 2 * j0;
            ex.margin = kModelMargin;
        }
        SMX_TRY(gather_chunk(c, j0, m, c->mu, ex));
        if (lanczos_steps > 0) {
            SMX_CUDA(launch_lanczos(subs + j0, m, c->max_n, c->d_T.p, f32, lanczos_steps, dp<float>(c->d_labels) + 2 * j0,
                                    c->stream));
            c->kernel_launches += 1;
        }
    }
    return SMX_OK;
}

extern "C" {

smx_status smx_bound_model_init(smx_ctx* c, uint64_t seed) {
    if (!c) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    std::vector<float> p(kModelParams, 0.0f);
    const int F = kModelFeatures;
    const int shapes[3][3] = {{0, 64, F}, {64 * F + 64, 64, 64}, {64 * F + 64 + 4096 + 64, 2, 64}};  // offset, out, in
    uint64_t ctr = 0;
    for (const auto& sh : shapes) {
        const float lim = 1.0f / std::sqrt(static_cast<float>(sh[2]));
        for (int i = 0; i < sh[1] * sh[2]; ++i) {
            const double u = static_cast<double>(splitmix64(seed * 0x100000001B3ull + (ctr++)) >> 11) * (1.0 / 9007199254740992.0);
            p[sh[0] + i] = static_cast<float>((2.0 * u - 1.0) * lim);
        }
    }
    c->n_samples = 0;
    return model_upload(c, p);
}

smx_status smx_bound_model_set_params(smx_ctx* c, const float* params, int32_t count) {
    if (!c || !params || count != kModelParams) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    return model_upload(c, std::vector<float>(params, params + count));
}

smx_status smx_bound_model_get_params(smx_ctx* c, float* params, int32_t count) {
    if (!c || !params || count != kModelParams) return SMX_ERR_ARG;
    if (!c->model_ready) return SMX_ERR_STATE;
    DeviceGuard g(c->device);
    SMX_CUDA(cudaMemcpyAsync(params, c->d_params.p, sizeof(float) * kModelParams, cudaMemcpyDeviceToHost, c->stream));
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    return SMX_OK;
}

smx_status smx_bound_model_collect(smx_ctx* c, int32_t lanczos_steps) {
    if (!c || lanczos_steps < 8 || lanczos_steps > kMaxLanczos) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    SMX_TRY(features_labels(c, lanczos_steps, false));
    const int B = c->B;
    if (c->n_samples + B > c->cap_samples) {  // grow the sample store, keeping its contents
        const int64_t cap = std::max<int64_t>(2 * c->cap_samples, c->n_samples + B);
        DevBuf nx, nt;
        smx_status e = ensure(nx, sizeof(float) * kModelFeatures * cap);
        if (e == SMX_OK) e = ensure(nt, sizeof(float) * 2 * cap);
        if (e != SMX_OK) {
            release(nx);
            release(nt);
            return e;
        }
        if (c->n_samples) {
            SMX_CUDA(cudaMemcpyAsync(nx.p, c->d_sx.p, sizeof(float) * kModelFeatures * c->n_samples, cudaMemcpyDeviceToDevice, c->stream));
            SMX_CUDA(cudaMemcpyAsync(nt.p, c->d_st.p, sizeof(float) * 2 * c->n_samples, cudaMemcpyDeviceToDevice, c->stream));
        }
        SMX_CUDA(cudaStreamSynchronize(c->stream));
        release(c->d_sx);
        release(c->d_st);
        c->d_sx = nx;
        c->d_st = nt;
        c->cap_samples = cap;
    }
    SMX_CUDA(cudaMemcpyAsync(dp<float>(c->d_sx) + kModelFeatures * c->n_samples, c->d_feat.p,
                             sizeof(float) * kModelFeatures * B, cudaMemcpyDeviceToDevice, c->stream));
    SMX_CUDA(cudaMemcpyAsync(dp<float>(c->d_st) + 2 * c->n_samples, c->d_labels.p, sizeof(float) * 2 * B,
                             cudaMemcpyDeviceToDevice, c->stream));
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    c->n_samples += B;
    return SMX_OK;
}

static smx_status mlp_steps(smx_ctx* c, const float* X, const float* T, int64_t m_total, int batch, int steps_or_epochs,
                            bool epochs, float lr, float* grad_host, double* loss_out) {
    SMX_TRY(ensure(c->d_partial_mlp, sizeof(float) * mlp_partial_floats(static_cast<int>(std::min<int64_t>(batch, m_total)))));
    float loss = 0.0f;
    const int64_t nbatch = (m_total + batch - 1) / batch;
    const int64_t total = epochs ? nbatch * steps_or_epochs : steps_or_epochs;
    for (int64_t s = 0; s < total; ++s) {
        const int64_t b0 = epochs ? (s % nbatch) * batch : 0;
        const int m = static_cast<int>(std::min<int64_t>(batch, m_total - b0));
        ++c->adam_t;
        SMX_CUDA(launch_mlp_step(dp<float>(c->d_params), X + kModelFeatures * b0, T + 2 * b0, m, dp<float>(c->d_partial_mlp),
                                 dp<float>(c->d_params), dp<float>(c->d_mst), dp<float>(c->d_vst), c->adam_t, lr,
                                 nullptr, dp<float>(c->d_loss), c->stream));
        c->kernel_launches += 2;
    }
    (void)grad_host;
    if (total > 0) {
        SMX_CUDA(cudaMemcpyAsync(&loss, c->d_loss.p, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        SMX_CUDA(cudaStreamSynchronize(c->stream));
        if (loss_out) *loss_out = loss;
    }
    return SMX_OK;
}

smx_status smx_bound_model_train(smx_ctx* c, int32_t epochs, int32_t batch, float lr, double* final_loss) {
    if (!c || epochs < 1 || batch < 1 || !(lr > 0.0f)) return SMX_ERR_ARG;
    if (!c->model_ready || c->n_samples == 0) return SMX_ERR_STATE;
    DeviceGuard g(c->device);
    return mlp_steps(c, dp<float>(c->d_sx), dp<float>(c->d_st), c->n_samples, batch, epochs, true, lr, nullptr, final_loss);
}

smx_status smx_bound_model_fit(smx_ctx* c, const float* x, const float* t, int32_t m, int32_t steps, float lr,
                               float* grad, double* loss) {
    if (!c || !x || !t || m < 1 || steps < 0 || (steps > 0 && !(lr > 0.0f))) return SMX_ERR_ARG;
    if (!c->model_ready) return SMX_ERR_STATE;
    DeviceGuard g(c->device);
    SMX_TRY(ensure(c->d_fit_x, sizeof(float) * kModelFeatures * m));
    SMX_TRY(ensure(c->d_fit_t, sizeof(float) * 2 * m));
    SMX_CUDA(cudaMemcpyAsync(c->d_fit_x.p, x, sizeof(float) * kModelFeatures * m, cudaMemcpyHostToDevice, c->stream));
    SMX_CUDA(cudaMemcpyAsync(c->d_fit_t.p, t, sizeof(float) * 2 * m, cudaMemcpyHostToDevice, c->stream));
    SMX_TRY(ensure(c->d_partial_mlp, sizeof(float) * mlp_partial_floats(m)));
    // gradient and loss at the current parameters (no update)
    SMX_CUDA(launch_mlp_step(dp<float>(c->d_params), dp<float>(c->d_fit_x), dp<float>(c->d_fit_t), m,
                             dp<float>(c->d_partial_mlp), dp<float>(c->d_params), dp<float>(c->d_mst), dp<float>(c->d_vst),
                             0, 0.0f, dp<float>(c->d_grad), dp<float>(c->d_loss), c->stream));
    c->kernel_launches += 2;
    float l0 = 0.0f;
    SMX_CUDA(cudaMemcpyAsync(&l0, c->d_loss.p, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (grad) SMX_CUDA(cudaMemcpyAsync(grad, c->d_grad.p, sizeof(float) * kModelParams, cudaMemcpyDeviceToHost, c->stream));
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    if (loss) *loss = l0;
    if (steps > 0)
        SMX_TRY(mlp_steps(c, dp<float>(c->d_fit_x), dp<float>(c->d_fit_t), m, m, steps, false, lr, nullptr, nullptr));
    return SMX_OK;
}

smx_status smx_bound_model_predict(smx_ctx* c, float* features, float* pred, float* labels, int32_t lanczos_steps) {
    if (!c || (labels && (lanczos_steps < 8 || lanczos_steps > kMaxLanczos))) return SMX_ERR_ARG;
    if (pred && !c->model_ready) return SMX_ERR_STATE;
    DeviceGuard g(c->device);
    SMX_TRY(features_labels(c, labels ? lanczos_steps : 0, pred != nullptr));
    const int B = c->B;
    if (pred) SMX_CUDA(cudaMemcpyAsync(pred, c->d_pred.p, sizeof(float) * 2 * B, cudaMemcpyDeviceToHost, c->stream));
    if (labels)
        SMX_CUDA(cudaMemcpyAsync(labels, c->d_labels.p, sizeof(float) * 2 * B, cudaMemcpyDeviceToHost, c->stream));
    if (features)
        SMX_CUDA(cudaMemcpyAsync(features, c->d_feat.p, sizeof(float) * kModelFeatures * B, cudaMemcpyDeviceToHost, c->stream));
    SMX_CUDA(cudaStreamSynchronize(c->stream));
    return SMX_OK;
}

static uint64_t fnv1a(const void* data, size_t n) {
    const unsigned char* p = static_cast<const unsigned char*>(data);
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

smx_status smx_bound_model_save(smx_ctx* c, const char* path) {
    if (!c || !path) return SMX_ERR_ARG;
    if (!c->model_ready) return SMX_ERR_STATE;
    std::vector<float> p(kModelParams);
    SMX_TRY(smx_bound_model_get_params(c, p.data(), kModelParams));
    FILE* f = std::fopen(path, "wb");
    if (!f) return SMX_ERR_ARG;
    const int32_t cnt = kModelParams;
    const uint64_t sum = fnv1a(p.data(), sizeof(float) * p.size());
    bool ok = std::fwrite("SMXBNDM1", 1, 8, f) == 8 && std::fwrite(&cnt, 4, 1, f) == 1 &&
              std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size() && std::fwrite(&sum, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SMX_OK : SMX_ERR_ARG;
}

smx_status smx_set_bound_model(smx_ctx* c, int32_t enable, const char* weights_path) {
    if (!c) return SMX_ERR_ARG;
    DeviceGuard g(c->device);
    if (weights_path) {
        FILE* f = std::fopen(weights_path, "rb");
        if (!f) return SMX_ERR_ARG;
        char magic[8];
        int32_t cnt = 0;
        uint64_t sum = 0;
        std::vector<float> p(kModelParams);
        bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "SMXBNDM1", 8) == 0 &&
                  std::fread(&cnt, 4, 1, f) == 1 && cnt == kModelParams &&
                  std::fread(p.data(), sizeof(float), p.size(), f) == p.size() && std::fread(&sum, 8, 1, f) == 1 &&
                  sum == fnv1a(p.data(), sizeof(float) * p.size());
        std::fclose(f);
        if (!ok) return SMX_ERR_ARG;
        SMX_TRY(model_upload(c, p));
    }
    if (enable < 0 || enable > 2) return SMX_ERR_ARG;
    if (enable && !c->model_ready) return SMX_ERR_STATE;
    c->model_on = enable != 0;
    c->model_gap = enable == 1;
    return SMX_OK;
}

}  // extern "C"

extern "C" {

void smx_destroy(smx_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    DevBuf* bufs[] = {&c->d_H, &c->d_H32, &c->d_voff, &c->d_row_idx, &c->d_col_ptr, &c->d_bs, &c->d_keep_prev, &c->d_sc, &c->d_keep, &c->d_fcol_ptr,
                      &c->d_frow_idx, &c->d_fvoff, &c->d_lstart, &c->d_subs, &c->d_order, &c->d_T, &c->d_W1,
                      &c->d_W2, &c->d_W3, &c->d_W4, &c->d_ws, &c->d_D, &c->d_xown, &c->d_bound, &c->d_iters, &c->d_partial,
                      &c->d_work_n3,
                      &c->d_params, &c->d_mst, &c->d_vst, &c->d_partial_mlp, &c->d_feat, &c->d_pred, &c->d_labels,
                      &c->d_gersh, &c->d_prev_ratio, &c->d_sq_ratio, &c->d_loss, &c->d_sx, &c->d_st,
                      &c->d_fit_x, &c->d_fit_t, &c->d_grad, &c->d_S, &c->d_Lc, &c->d_Mc, &c->d_nlohi,
                      &c->d_setup_iters};
    for (DevBuf* b : bufs) release(*b);
    for (auto& pr : c->ns_events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    if (c->h_keep_pinned) cudaFreeHost(c->h_keep_pinned);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

}  // extern "C"
