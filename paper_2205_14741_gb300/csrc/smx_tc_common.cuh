// Building blocks of the tcgen05 Newton-Schulz kernels (the single-CTA kernel of k_ns_tc.cu
// and the CTA-pair streamed kernel of k_ns_tc_pair.cu): launch shape, shared-memory layout of
// the stages, shared-memory descriptors, 16-bit packing and the hi/lo split, tensor-memory
// loads and stores.  Each translation unit that includes it gets its own copy (internal
// linkage).
#pragma once

#include "smx_kernels.h"

namespace smx {

namespace {

constexpr int kThreads = 384;
constexpr int kEpiWarps = 8;
// Submatrices with kpad <= kResKpad keep the iterate on chip: X in shared
// memory (both factors of X X, the B factor of Y X) and Y in tensor memory
// (the A factor of Y X); only X' goes through L2.
constexpr int kResKpad = 192;
constexpr uint32_t kABytes = 128 * 128;  // 128 rows x 64 K x 2 B
// On-chip prologue: T_j's rows pass through two staging buffers after the images (at most
// 2 x 72 KB; the second hi image of the double-buffered form is free until iteration 0).
constexpr uint32_t kStageOff = 144u * 1024u;
// On-chip form: the per-warp 32 x 32 transpose buffers (rows 80 bytes apart) after the images
// and the corner operand (for split operands at 192 KB, single ones at 96 KB; free during the
// iterations; the prologue's staging buffers are dead by then)
constexpr uint32_t kXsOff = 96u * 1024u;  // times the operand count NB
constexpr uint32_t kXsWarp = 32 * 80;
// The streamed form's products with K >= kSplitKpad accumulate in two chains (see gemm).
constexpr int kSplitKpad = 2048;
// A step with factor a maps an eigenvalue at 1 to p(a) ~ 1 - 1.5 (a - 1)^2: the last step may
// use a up to 1 + kStopSlack (a shift of at most 1.4e-7, far below the split form's error).
constexpr float kStopSlack = 3e-4f;

template <int PREC>
struct TcCfg {
    static constexpr int kNb = (PREC == 1) ? 2 : 1;        // operand buffers per matrix (hi[, lo])
    static constexpr int kNmax = 256;                      // columns per N tile
    static constexpr uint32_t kBBytes = kNmax * 128;       // 64 K rows x kNmax columns x 2 B
    static constexpr int kStages = (PREC == 1) ? 2 : 4;    // smem ring depth
    static constexpr uint32_t kStage = kNb * (kABytes + kBBytes);
    static constexpr int kFmt = (PREC == 3) ? 1 : 0;       // 0 = FP16, 1 = BF16
    // the streamed form's stages, or the on-chip form's data: for kpad = 192 the hi and lo
    // images (72 KB each), the corner operand Bz (hi and lo, 24 KB each) and 8 KB read past the
    // lo image by the last row tile's MMAs, inside a reserve of three images plus 8 KB
    static constexpr size_t kResSmem = static_cast<size_t>(kNb + 1) * 9 * 8192 + 8192;
    // the streamed form's per-warp transpose buffers (8 epilogue warps, 32 rows of 80 bytes) after its stages
    static constexpr uint32_t kXposeWarp = 32 * 80;
    static constexpr uint32_t kXposeOff = static_cast<uint32_t>(kStages) * kStage;
    static constexpr size_t kStreamSmem = static_cast<size_t>(kXposeOff) + 8 * kXposeWarp;
    static constexpr size_t kDynSmem = 1024 + (kStreamSmem > kResSmem ? kStreamSmem : kResSmem);
    static_assert(kDynSmem <= 227 * 1024, "shared memory per CTA");
    static_assert(static_cast<size_t>(kXsOff) * kNb + 12 * kXsWarp <= kDynSmem - 1024, "on-chip transpose buffers");
    static_assert(kXsOff * kNb >= static_cast<uint32_t>(kNb) * 9 * 8192 + static_cast<uint32_t>(kNb) * 3 * 8192,
                  "transpose buffers after the images and the corner operand");
    // each of the on-chip prologue's two staging buffers: what the allocation leaves after kStageOff
    static constexpr uint32_t kStageBuf = static_cast<uint32_t>((kDynSmem - 1024 - kStageOff) / 2) & ~15u;
    static_assert(kDynSmem - 1024 >= kStageOff + 2 * static_cast<size_t>(kStageBuf) && kStageBuf >= 16u * 1024u,
                  "staging buffers inside the allocation");
};

// Shared-memory descriptor of a B tile in the MN-major 128-byte-swizzled
// layout: 64-column blocks of 64 K rows (8 KB each, LBO) and 8-row K groups
// (1 KB, SBO).
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(8192 >> 4) << 16;  // leading byte offset: next 64-column block
    d |= static_cast<uint64_t>(1024 >> 4) << 32;  // stride byte offset: next 8 K rows
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(2) << 61;
    return d;
}

// two floats -> packed 16-bit pair (hi word = second value)
template <int PREC>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if constexpr (PREC == 3) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <int PREC>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
    if constexpr (PREC == 3) return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w));
    else return __half22float2(*reinterpret_cast<__half2*>(&w));
}
template <int PREC>
__device__ __forceinline__ uint16_t to16(float x) {
    if constexpr (PREC == 3) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    else return __half_as_ushort(__float2half_rn(x));
}
template <int PREC>
__device__ __forceinline__ float from16(uint16_t h) {
    if constexpr (PREC == 3) return __bfloat162float(__ushort_as_bfloat16(h));
    else return __half2float(__ushort_as_half(h));
}


// (a, b) -> hi pair and lo pair with a ~ hi.x + lo.x, b ~ hi.y + lo.y
template <int PREC, int NB>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hw, uint32_t& lw) {
    if constexpr (NB == 2) {
        // hi = (a, b) rounded to the 16-bit format; lo = the FP32 remainder, rounded
        hw = pack2<PREC>(a, b);
        const float2 h = unpack2<PREC>(hw);
        lw = pack2<PREC>(a - h.x, b - h.y);
    } else {
        hw = pack2<PREC>(a, b);
        lw = 0;
    }
}

// 8 consecutive values hi[0..8) + lo[0..8) (16-byte aligned) as FP32
template <int PREC, int NB>
__device__ __forceinline__ void load8(const uint16_t* hi, const uint16_t* lo, float (&v)[8]) {
    const uint4 h = *reinterpret_cast<const uint4*>(hi);
    const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = unpack2<PREC>(hw[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
    if constexpr (NB == 2) {
        const uint4 l = *reinterpret_cast<const uint4*>(lo);
        const uint32_t lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = unpack2<PREC>(lw[i]);
            v[2 * i] += f.x;
            v[2 * i + 1] += f.y;
        }
    }
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 32 consecutive 32-bit TMEM columns of this thread's lane <- r
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// tcgen05.mma kind::f16 with the A operand (M = 128 rows in the 128 lanes, K
// packed two 16-bit values per 32-bit column) in tensor memory
__device__ __forceinline__ void tc_mma_f16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

// MN-major 128-byte-swizzled B descriptor whose 64-column blocks are lbo bytes apart
__device__ __forceinline__ uint64_t sdesc_mn_sw128_lbo(uint32_t saddr, uint32_t lbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(lbo >> 4) << 16;
    d |= static_cast<uint64_t>(1024 >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(2) << 61;
    return d;
}

// Bulk prefetch of [p, p + bytes) into L2 (bytes a multiple of 16, p 16-byte aligned).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// 16-byte asynchronous copy global -> shared (no registers), its group commit and wait.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Byte offset of element (r, c) in a row-major matrix image held as 64 x 64
// boxes in the 128-byte-swizzled layout (what a TMA box load writes), box
// (row block rb, column block cb) at (cb * RB + rb) * 8 KB.
__device__ __forceinline__ uint32_t img_offset(int r, int c, int RB) {
    const int rb = r >> 6, rr = r & 63, cb = c >> 6, cc = c & 63;
    return static_cast<uint32_t>((cb * RB + rb) * 8192 + rr * 128 + ((((cc >> 3) ^ (rr & 7))) << 4) + (cc & 7) * 2);
}

// two TMEM loads (32 columns each), one wait
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
        "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// the same wait, tied to the registers of one load in flight so that no use of them is
// scheduled before it
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                   "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]),
                   "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait_plain(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace

}  // namespace smx
