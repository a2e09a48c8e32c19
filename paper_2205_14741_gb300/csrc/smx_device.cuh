// Device-side building blocks shared by the kernels of the submatrix library:
// per-submatrix descriptors, bounded mbarrier waits, TMA and tcgen05 wrappers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace smx {

// Status codes written by kernels into the context's device status word
// (values match smx_status in smx.h).
enum : int { kOk = 0, kErrNonfinite = 3, kErrNoconv = 6, kErrTimeout = 8 };

// One submatrix T_j = H[R_j, R_j] (Fig. 2 step (i)).
struct SubDesc {
    int32_t col;    // block column j (owner)
    int32_t n;      // n_j = sum of the block sizes of R_j
    int32_t ld;     // leading dimension of T_j in the FP64 staging buffer
    int32_t own;    // first row of block j inside T_j
    int32_t bown;   // block size of j
    int32_t nblk;   // |R_j|
    int64_t fptr;   // first filtered block of column j (R_j = frow_idx[fptr .. fptr + nblk))
    int64_t t_off;  // offset of T_j (elements) in the staging buffer
    int64_t x_off;  // offset of the saved owner columns (n x bown, column by column)
};

// One block pair of the symmetric input pattern for the symmetrised D: block k = (row r,
// column j) with r <= j and its transpose kt = (row j, column r) (kt == k on the diagonal);
// value offsets of both in the input layout (column-major blocks of br x bj and bj x br).
struct SymPair {
    int64_t off_k, off_kt;
    int32_t k, kt;
    int32_t br, bj;
};

// Filtered pattern and value addressing shared by gather and scatter.
struct PatternView {
    const int64_t* fcol_ptr;  // [B+1] filtered block-CSC column pointers
    const int32_t* frow_idx;  // [nnzb_f] filtered block rows
    const int64_t* fvoff;     // [nnzb_f] offset of each filtered block in the input value array
    const int32_t* lstart;    // [nnzb_f] first row of the block inside its column's submatrix
    const int32_t* bsize;     // [B] block sizes
    // Block maps of the submatrices, built once per filtered pattern (null: the gather builds
    // them): for block column j, nblk_j x nblk_j value offsets from maps + map_off[j], entry
    // (a, c) the offset of block (R_j[c], R_j[a]) of H, -1 when the filter dropped it
    const int32_t* maps = nullptr;
    const int64_t* map_off = nullptr;
};

// Conversions between FP64 and FP32 on the integer pipes.  GB300's FP64 pipe
// takes about 16 cycles per warp instruction per SM, and conversions with an
// FP64 operand run on it; these give the same results as the conversion
// instructions for normal values (round to nearest even for FP64 -> FP32) and
// leave the others (zero, subnormal, overflow, inf, NaN) to them.
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t hi = static_cast<uint32_t>(b >> 32), lo = static_cast<uint32_t>(b);
    const int ef = static_cast<int>((hi >> 20) & 0x7ffu) - 896;  // FP32 exponent field (1023 - 127)
    if (ef >= 1 && ef <= 254) {
        uint32_t r = (hi & 0x80000000u) | (static_cast<uint32_t>(ef) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t rem = lo & 0x1fffffffu;  // the 29 bits dropped; half = 2^28
        if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ++r;  // a carry may reach inf: correct
        return __uint_as_float(r);
    }
    return __double2float_rn(x);
}
__device__ __forceinline__ double f2d(float f) {
    const uint32_t u = __float_as_uint(f), e = (u >> 23) & 0xffu;
    if (e != 0u && e != 0xffu) {
        const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
        return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(hi) << 32) | (u << 29)));
    }
    return static_cast<double>(f);
}
// false for inf and NaN (the exponent field of the high word)
__device__ __forceinline__ bool finite_bits(double x) {
    return (static_cast<uint32_t>(static_cast<unsigned long long>(__double_as_longlong(x)) >> 32) & 0x7ff00000u) !=
           0x7ff00000u;
}

// Bounded waits: every spin in the library gives up after this many polls,
// records kErrTimeout and returns false.
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the completion of the phase with the given parity.  Gives up when
// *abort becomes non-zero (another role timed out) or after kSpinLimit polls,
// in which case it raises *abort and records the timeout in *status.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && *abort) return false;
    }
    *abort = 1;
    atomicCAS(status, kOk, kErrTimeout);
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's generic-proxy global writes before later async-proxy
// (TMA) reads issued by other threads of the CTA after a barrier.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy reads of them (tensor-core operands, bulk copies) issued after a
// barrier.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Untiled bulk copy shared -> global (both addresses 16-byte aligned, bytes a
// multiple of 16), tracked by this thread's bulk async-groups.
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until this thread's committed bulk copies have read their shared-memory source.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Waits until this thread's committed bulk copies are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 3-D tiled TMA load (box given by the tensor map) into shared memory,
// completing on an mbarrier transaction count.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// tcgen05 (5th-generation tensor cores, tensor memory)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major operand tile stored in the
// 128-byte-swizzled canonical layout (rows of 128 B, 8-row atoms of 1 KB).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(16 >> 4) << 16;    // leading byte offset (unused for swizzled K-major)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;  // stride byte offset: one 8-row atom
    d |= static_cast<uint64_t>(1) << 46;          // descriptor version
    d |= static_cast<uint64_t>(2) << 61;          // 128-byte swizzle
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16 with FP32 accumulation,
// both operands K-major; ab_fmt 0 = FP16, 1 = BF16.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n, int ab_fmt) {
    return (1u << 4) | (static_cast<uint32_t>(ab_fmt) << 7) | (static_cast<uint32_t>(ab_fmt) << 10) |
           (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

// Arrives on an mbarrier when all tcgen05 operations issued so far by this
// thread have completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
        "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// Scaled Newton-Schulz schedule
// ---------------------------------------------------------------------------
// With every |eigenvalue| of X in [l, 1] (0 < l <= 1), one step of the sign
// iteration applied to a X, p(a X) with p(x) = x (3 - x^2) / 2, maps that
// interval into [p(a l), 1] when a = sqrt(3 / (1 + l + l^2)): this a makes
// p(a l) = p(a), and p peaks at 1 inside the interval.  Small eigenvalues thus
// grow by about 1.5 a (up to 2.6) per step instead of 1.5.  Any l in (0, 1]
// keeps every eigenvalue in (0, 1] with its sign (a l underestimated only
// costs steps), so the schedule is safe for any lower bound the caller
// guesses.  a is capped at kScaleCap < sqrt 3 so that rounding in X or in the
// upper bound cannot carry an eigenvalue past sqrt 3, where p changes sign.
constexpr double kScaleCap = 1.72;
template <typename T>
__device__ __forceinline__ T ns_scale(T l) {
    if (!(l < T(1))) return T(1);
    const T a = sqrt(T(3) / (T(1) + l + l * l));
    return a < T(kScaleCap) ? a : T(kScaleCap);
}
// the lower end of the interval after the step with factor a
template <typename T>
__device__ __forceinline__ T ns_next_lower(T a, T l) {
    const T x = a * l;
    const T y = T(0.5) * x * (T(3) - x * x);
    return y < T(1) ? y : T(1);
}

// ---------------------------------------------------------------------------
// warp / block reductions
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Deterministic block sum: warp shuffles, then warp 0 sums the warp totals in order.
// All threads of the block must call it; returns the total to every thread.
__device__ __forceinline__ double block_sum(double v, double* scratch /* >= 32 doubles */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nwarps ? scratch[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) scratch[0] = t;
    }
    __syncthreads();
    t = scratch[0];
    __syncthreads();
    return t;
}

}  // namespace smx
