// Newton-Schulz sign iteration on the tcgen05 tensor cores.
//
// Eq. 13: sign(A) = A (A^2)^(-1/2).  Per submatrix (Fig. 2 step (ii)) the
// iteration X_{k+1} = X_k Y_k, Y_k = 3/2 I - 1/2 X_k^2, X_0 = (T_j - mu I)/b_j
// runs entirely inside one persistent CTA, so each submatrix keeps its own
// iteration count and stopping decision.  The dense contractions are the
// paper's low-precision tensor-unit work (Section 3): FP16 (or BF16) operands,
// FP32 accumulation in tensor memory.  In the split form each operand is held
// as hi + lo (two FP16 numbers, about 22 significant bits) and every product
// is hi*hi + hi*lo + lo*hi, all accumulated in one FP32 TMEM accumulator.
//
// Submatrices are padded to multiples of 32 for the MMA (K steps and N);
// TMA moves 64-wide boxes, whose columns beyond the padded size are never
// multiplied.
//
// Operand layout: both factors of C = A B are read from row-major matrices in
// the CTA's workspace slot.  A (rows of the left factor) is loaded K-major,
// B in its true orientation (MN-major: rows of B are K), so the kernel forms
// the product itself and never the product with a transpose -- with a
// transposed B, the antisymmetric rounding residue of an iterate would double
// at every step.
//
// CTA layout (384 threads).  Streamed form (submatrices larger than 192):
//   warp 0       TMA producer (one lane): 64-wide K chunks of A (128 rows)
//                and B (all columns of the tile, N <= 256) into a ring of
//                shared-memory stages (128-byte swizzle); a row tile spans
//                the whole padded width when n <= 256, so A is read once
//   warp 1       MMA issuer (one lane): tcgen05.mma M=128, K=16 into one of
//                two TMEM accumulator buffers of 256 FP32 columns
//   warps 2..3   help with the per-submatrix prologue and scatter
//   warps 4..11  epilogue: tcgen05.ld, Y = 3/2 I - 1/2 acc (or X' = acc),
//                residual ||X^2 - I||_F^2 in FP32, split to hi/lo, 16-byte
//                stores to the slot (L2-resident)
// On-chip form (up to 192): all 12 warps share the tensor-memory passes; one
// lane of warp 1 issues the MMAs (of warp 10 the next iteration's in two-tile form).
#include "smx_finish.cuh"
#include "smx_kernels.h"
#include "smx_tc_common.cuh"

namespace smx {


template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) k_ns_tc(NsTcArgs a, const __grid_constant__ CUtensorMap tmap) {
    using C = TcCfg<PREC>;
    constexpr int NB = C::kNb, S = C::kStages, NT = C::kNmax;
    extern __shared__ uint8_t smem_raw[];
    if (a.skip && *a.skip) return;  // a skipped step of a device-side bisection (uniform: set before launch)
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

    __shared__ uint64_t full_bar[S], empty_bar[S], tfull[2], tempty[2], drain_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s, job_s, conv_s, bad_s, p_issued_s, m_consumed_s;
    __shared__ int plain_s;  // the scaled schedule is over: plain steps from the next one
    __shared__ float resid_s[kEpiWarps];
    __shared__ uint64_t mma_bar, mma_bar2;
    __shared__ float resid_s2[kThreads / 32];
    __shared__ float red_s[2][kThreads / 32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* const abortp = &abort_s;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], kEpiWarps);
        }
        mbar_init(&drain_bar, 1);
        mbar_init(&mma_bar, 1);
        mbar_init(&mma_bar2, 1);
        abort_s = 0;
        p_issued_s = 0;
        m_consumed_s = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(&tmem_base_s, 512);
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_s;

    auto warp_sum_f = [](float v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    // block-wide maxima of two non-negative values (all threads get the result)
    auto block_max2 = [&](float x, float y) -> float2 {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
            y = fmaxf(y, __shfl_xor_sync(0xffffffffu, y, o));
        }
        if (lane == 0) {
            red_s[0][warp] = x;
            red_s[1][warp] = y;
        }
        __syncthreads();
        float2 m = make_float2(0.0f, 0.0f);
        for (int w = 0; w < kThreads / 32; ++w) {
            m.x = fmaxf(m.x, red_s[0][w]);
            m.y = fmaxf(m.y, red_s[1][w]);
        }
        __syncthreads();
        return m;
    };

    // role-local pipeline positions, continuous over all GEMMs of the CTA
    uint32_t p_it = 0;              // producer: K chunks issued
    uint32_t m_it = 0;              // MMA: K chunks consumed
    // the two TMEM accumulator buffers: tiles alternate between them (the epilogue of one
    // overlaps the products of the next), except in the two-chain mode, where a tile takes both
    uint32_t m_use0 = 0, m_use1 = 0;    // MMA: tiles issued into buffer 0 / 1
    uint32_t m_nb = 0;                  // MMA: the buffer of the next single-chain tile
    uint32_t e_full0 = 0, e_full1 = 0;  // epilogue: tiles drained from buffer 0's / 1's commits
    uint32_t e_nb = 0;                  // epilogue: the buffer of the next single-chain tile
    const int64_t buf = static_cast<int64_t>(a.ld) * a.ld;
    uint16_t* ws = static_cast<uint16_t*>(a.ws);
    const int slot_z = blockIdx.x * 6;
    uint32_t mma_ph = 0, mma_ph2 = 0;  // completed phases of mma_bar, mma_bar2 (uniform over the CTA)
    const uint32_t idesc_b_mn = 1u << 16;  // B operand MN-major

    // C = A * B over K in [0, kpad), written to buffer zo (rows and columns < kpad).  Every
    // product of the iteration is symmetric (X X, and X Y with Y a polynomial in X), so only
    // the tiles on and right of the diagonal 128 x 128 blocks are multiplied: row tile mt
    // covers columns 128 mt .. kpad - 1.  Each epilogue warp owns 32 rows; of a tile's
    // 32 x 32 chunks it writes those right of its diagonal chunk together with their transposes
    // (through a per-warp shared-memory transpose) and the diagonal chunk's upper triangle
    // mirrored into its lower one, so zo holds an exactly symmetric matrix.  (An iterate whose
    // diagonal blocks kept the rounding asymmetry of the products while the rest is mirrored
    // would let that asymmetry grow from step to step.)
    // mode 1: zo = oscale A A + dg I (3/2 I - 1/2 A A for a plain step), residual
    //         ||A A - I||_F^2 accumulated over the chunks written (transposed ones count twice);
    // mode 2: zo = oscale * A B.
    auto gemm = [&](int kpad, int n, int mode, int za, int zb, int zo, float oscale, float dg = 1.5f) {
        const int mtiles = (kpad + 127) / 128, kchunks = (kpad + 63) / 64;
        // Long K: two accumulation chains over the two halves of K in the two TMEM buffers, summed
        // in FP32 by the epilogue (the tensor cores' FP32 accumulation loses accuracy with the
        // length of a chain: at n ~ 2800 one chain puts about 1.2e-5 on D, two about 7.6e-6); a
        // tile then holds both buffers, so its epilogue no longer overlaps the next tile's products.
        const bool split = kpad >= kSplitKpad;
        // row tile mt: N tiles of up to NT columns from column 128 mt
        auto ntiles_of = [&](int mt) { return (kpad - 128 * mt + NT - 1) / NT; };
        if (warp == 0) {
            if (lane == 0) {
                for (int mt = 0; mt < mtiles && !*abortp; ++mt)
                    for (int nt = 0; nt < ntiles_of(mt) && !*abortp; ++nt) {
                        const int n0 = 128 * mt + NT * nt, nn = min(NT, kpad - n0);
                        for (int kc = 0; kc < kchunks; ++kc) {
                            const int stage = p_it % S;
                            const uint32_t round = p_it / S;
                            if (round > 0 && !mbar_wait(&empty_bar[stage], (round - 1) & 1, &abort_s, a.status)) break;
                            uint8_t* st = smem + stage * C::kStage;
                            const int nboxes = (nn + 63) / 64;
                            mbar_arrive_expect_tx(&full_bar[stage], NB * (kABytes + static_cast<uint32_t>(nboxes) * 8192));
                            for (int b = 0; b < NB; ++b) {
                                uint8_t* sa = st + b * kABytes;
                                tma_load_3d(sa, &tmap, kc * 64, 128 * mt, za + b, &full_bar[stage]);
                                tma_load_3d(sa + 8192, &tmap, kc * 64, 128 * mt + 64, za + b, &full_bar[stage]);
                                uint8_t* sb = st + NB * kABytes + b * C::kBBytes;
                                for (int h = 0; h < nboxes; ++h)
                                    tma_load_3d(sb + h * 8192, &tmap, n0 + 64 * h, kc * 64, zb + b, &full_bar[stage]);
                            }
                            ++p_it;
                        }
                    }
                p_issued_s = static_cast<int>(p_it);
            }
            __syncwarp();
        } else if (warp == 1) {
            if (lane == 0) {
                for (int mt = 0; mt < mtiles && !*abortp; ++mt)
                    for (int nt = 0; nt < ntiles_of(mt) && !*abortp; ++nt) {
                        const int nn = min(NT, kpad - 128 * mt - NT * nt);
                        // the buffer(s) of this tile, released by the epilogue of their previous tiles
                        const uint32_t abuf = split ? 0u : m_nb;
                        if (!split) m_nb ^= 1u;
                        bool freed = true;
                        if (abuf == 0 || split) {
                            if (m_use0 > 0 && !mbar_wait(&tempty[0], (m_use0 - 1) & 1, &abort_s, a.status)) freed = false;
                            ++m_use0;
                        }
                        if (abuf == 1 || split) {
                            if (freed && m_use1 > 0 && !mbar_wait(&tempty[1], (m_use1 - 1) & 1, &abort_s, a.status)) freed = false;
                            ++m_use1;
                        }
                        if (!freed) break;
                        tc_fence_after();
                        const int khalf = split ? kchunks / 2 : kchunks;  // the second chain's first K chunk
                        const uint32_t idesc = idesc_f16(128, nn, C::kFmt) | idesc_b_mn;
                        bool ok = true;
                        for (int kc = 0; kc < kchunks; ++kc) {
                            const int stage = m_it % S;
                            const uint32_t round = m_it / S;
                            if (!mbar_wait(&full_bar[stage], round & 1, &abort_s, a.status)) { ok = false; break; }
                            tc_fence_after();
                            const uint32_t base = smem_u32(smem + stage * C::kStage);
                            const uint32_t a_hi = base, a_lo = base + kABytes;
                            const uint32_t b_hi = base + NB * kABytes, b_lo = b_hi + C::kBBytes;
                            // K steps beyond kpad (the tail of the last 64-wide chunk) are not issued
                            const int ksteps = min(4, (kpad - 64 * kc) / 16);
                            const uint32_t d = tmem_base + (kc >= khalf ? 256u : abuf * 256u);
                            for (int kk = 0; kk < ksteps; ++kk) {
                                const uint32_t acc = ((kc == 0 || kc == khalf) && kk == 0) ? 0u : 1u;
                                const uint64_t ah = sdesc_sw128(a_hi + kk * 32), bh = sdesc_mn_sw128(b_hi + kk * 2048);
                                tc_mma_f16(d, ah, bh, idesc, acc);
                                if constexpr (NB == 2) {
                                    tc_mma_f16(d, ah, sdesc_mn_sw128(b_lo + kk * 2048), idesc, 1u);
                                    tc_mma_f16(d, sdesc_sw128(a_lo + kk * 32), bh, idesc, 1u);
                                }
                            }
                            tc_commit(&empty_bar[stage]);
                            ++m_it;
                        }
                        if (!ok) break;
                        tc_commit(&tfull[abuf]);
                    }
                m_consumed_s = static_cast<int>(m_it);
            }
            __syncwarp();
        } else if (warp >= 4) {
            const int q = warp & 3, half = (warp - 4) >> 2;
            const int lrow = q * 32 + lane;
            // this warp's transpose buffer: 32 rows of 32 16-bit values, rows 80 bytes apart
            // (conflict-free 16-byte row writes, 2-byte column reads)
            uint16_t* xs = reinterpret_cast<uint16_t*>(smem + C::kXposeOff + (warp - 4) * C::kXposeWarp);
            float r2 = 0.0f;
            for (int mt = 0; mt < mtiles; ++mt)
                for (int nt = 0; nt < ntiles_of(mt); ++nt) {
                    const int n0 = 128 * mt + NT * nt, nn = min(NT, kpad - n0);
                    const uint32_t abuf = split ? 0u : e_nb;
                    if (!split) e_nb ^= 1u;
                    const uint32_t ph = (abuf ? e_full1++ : e_full0++) & 1u;
                    int ok = 1;
                    if (lane == 0) ok = mbar_wait(&tfull[abuf], ph, &abort_s, a.status) ? 1 : 0;
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) { mt = mtiles; break; }
                    tc_fence_after();
                    const int row = 128 * mt + lrow;
                    uint16_t* zo_hi = ws + static_cast<int64_t>(zo) * buf;
                    uint16_t* out_hi = zo_hi + static_cast<int64_t>(row) * a.ld;
                    uint16_t* out_lo = out_hi + buf;
                    for (int c0 = 32 * half; c0 < nn; c0 += 64) {
                        uint32_t raw[32];
                        tmem_ld32_issue(tmem_base + (static_cast<uint32_t>(q * 32) << 16) + abuf * 256 + c0, raw);
                        if (split) {  // the second chain, added in FP32
                            uint32_t raw1[32];
                            tmem_ld32_issue(tmem_base + (static_cast<uint32_t>(q * 32) << 16) + 256 + c0, raw1);
                            tmem_wait_ld();
#pragma unroll
                            for (int i = 0; i < 32; ++i) raw[i] = __float_as_uint(__uint_as_float(raw[i]) + __uint_as_float(raw1[i]));
                        } else {
                            tmem_wait_ld();
                        }
                        const int r0 = row - lane;  // the warp's first row
                        const int col0 = n0 + c0;
                        // chunks left of the warp's diagonal chunk are not written: the transposes of
                        // the chunks right of it fill them (all warp-uniform; kpad is a multiple of 32)
                        if (r0 < kpad && col0 >= r0) {
                            const bool xp = col0 > r0;  // right of the diagonal chunk: also transposed
                            const bool interior = row < n && col0 + 32 <= n;
                            const int i0 = row - col0;  // position of the diagonal in this chunk, if 0 <= i0 < 32
                            float y[32], rc = 0.0f;
                            if (interior) {
                                if (mode == 1) {
                                    float sq = 0.0f, dv = 0.0f;
#pragma unroll
                                    for (int i = 0; i < 32; ++i) {
                                        const float v = __uint_as_float(raw[i]);
                                        sq = fmaf(v, v, sq);
                                        y[i] = oscale * v;
                                        if (i == i0) { y[i] += dg; dv = v; }
                                    }
                                    // sum (v - delta)^2 = sum v^2 - 2 v_diag + 1 when the diagonal is here
                                    rc = (i0 >= 0 && i0 < 32) ? sq - 2.0f * dv + 1.0f : sq;
                                } else {
#pragma unroll
                                    for (int i = 0; i < 32; ++i) y[i] = oscale * __uint_as_float(raw[i]);
                                }
                            } else {
#pragma unroll
                                for (int i = 0; i < 32; ++i) {
                                    const float v = __uint_as_float(raw[i]);
                                    const bool valid = row < n && col0 + i < n;
                                    if (mode == 1) {
                                        const float dl = (i == i0) ? 1.0f : 0.0f;
                                        const float e = v - dl;
                                        y[i] = valid ? fmaf(oscale, v, dg * dl) : 0.0f;
                                        rc = valid ? fmaf(e, e, rc) : rc;
                                    } else {
                                        y[i] = valid ? oscale * v : 0.0f;
                                    }
                                }
                            }
                            r2 += xp ? 2.0f * rc : rc;
                            uint32_t hw[16], lw[16];
#pragma unroll
                            for (int i = 0; i < 32; i += 2) split2<PREC, NB>(y[i], y[i + 1], hw[i >> 1], lw[i >> 1]);
                            // the warp's 32 x 32 block through shared memory: lane l reads column l,
                            // i.e. element (r0 + k, col0 + l) for k = 0 .. 31
#pragma unroll
                            for (int b = 0; b < NB; ++b) {
                                const uint32_t* w = b == 0 ? hw : lw;
                                uint16_t* dst_row = (b == 0 ? out_hi : out_lo) + col0;
                                if (!xp) {
                                    // the diagonal chunk: its upper triangle (own row from the diagonal
                                    // on), mirrored into the lower one, so the stored iterate is exactly
                                    // symmetric
                                    __syncwarp();
                                    uint4* xr = reinterpret_cast<uint4*>(xs + lane * 40);
#pragma unroll
                                    for (int u = 0; u < 4; ++u) xr[u] = make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
                                    __syncwarp();
                                    uint32_t t[16];
#pragma unroll
                                    for (int k = 0; k < 16; ++k) {
                                        const uint32_t e0 = 2 * k < lane ? static_cast<uint32_t>(xs[(2 * k) * 40 + lane]) : (w[k] & 0xFFFFu);
                                        const uint32_t e1 = 2 * k + 1 < lane ? static_cast<uint32_t>(xs[(2 * k + 1) * 40 + lane]) : (w[k] >> 16);
                                        t[k] = e0 | (e1 << 16);
                                    }
                                    uint4* d = reinterpret_cast<uint4*>(dst_row);
#pragma unroll
                                    for (int u = 0; u < 4; ++u) d[u] = make_uint4(t[4 * u], t[4 * u + 1], t[4 * u + 2], t[4 * u + 3]);
                                } else {
                                    uint4* d = reinterpret_cast<uint4*>(dst_row);
#pragma unroll
                                    for (int u = 0; u < 4; ++u) d[u] = make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
                                    // element (row, col0 + k) -> (col0 + k, row): lane l writes row col0 + l,
                                    // columns r0 .. r0 + 31 (64 contiguous bytes)
                                    __syncwarp();
                                    uint4* xr = reinterpret_cast<uint4*>(xs + lane * 40);
#pragma unroll
                                    for (int u = 0; u < 4; ++u) xr[u] = make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
                                    __syncwarp();
                                    uint32_t t[16];
#pragma unroll
                                    for (int k = 0; k < 16; ++k)
                                        t[k] = static_cast<uint32_t>(xs[(2 * k) * 40 + lane]) |
                                               (static_cast<uint32_t>(xs[(2 * k + 1) * 40 + lane]) << 16);
                                    uint4* dt = reinterpret_cast<uint4*>(zo_hi + b * buf + static_cast<int64_t>(col0 + lane) * a.ld + r0);
#pragma unroll
                                    for (int u = 0; u < 4; ++u) dt[u] = make_uint4(t[4 * u], t[4 * u + 1], t[4 * u + 2], t[4 * u + 3]);
                                }
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(&tempty[abuf]);
                        if (split) mbar_arrive(&tempty[1]);
                    }
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
            if (lane == 0) resid_s[warp - 4] = r2;
            fence_proxy_async_global();
        }
        __syncthreads();
    };

    // Jobs are claimed one ahead: while a submatrix iterates, its successor's staged
    // T_j is prefetched into L2 (the prologue then reads it from there).
    __shared__ int next_s;
    __shared__ float rprev_s;  // the previous step's residual (rounding-floor stop)
    // the job's scalars in FP32: 1 / b_j, the predicted smallest |eigenvalue| of
    // X0 = (T_j - mu I) / b_j (negative when there is no prediction), and b_j / G_j; with b_j
    // itself (FP64), which the job rescales by its a-posteriori factor
    __shared__ float inv_b_s, dhat_s, bg_s;
    __shared__ double b_s;
    __shared__ float next_inv_b_s, next_dhat_s, next_bg_s;
    __shared__ double next_b_s;
    // Claims the successor of the current job: one atomic, its descriptors, a prefetch of its
    // staged T_j into L2, and its scalars (FP32 divisions: FP64 division is slow on this GPU's
    // FP64 pipe).  Run by one thread: thread 0 for the first job, then warp 11's first lane
    // while the job's first product is multiplied, so that no CTA barrier waits for its
    // memory round trips; the loop head takes the results from shared memory.
    auto claim_next = [&]() {
        const int nx = atomicAdd(a.work_counter, 1);
        next_s = nx;
        if (nx < a.n_subs) {
            const int jj = a.order[nx];
            const SubDesc sn = a.subs[jj];
            const double b = a.bound[jj];
            const float pr = a.pred ? a.pred[2 * jj + 1] : -1.0f;
            const float g = static_cast<float>(a.gersh[jj]);
            const uint64_t bytes = static_cast<uint64_t>(sn.n) * sn.ld * sizeof(float);
            const uint32_t len = static_cast<uint32_t>(bytes < (4u << 20) ? bytes : (4u << 20)) & ~15u;
            if (len) prefetch_l2_bulk(a.T + sn.t_off, len);
            const float bf = static_cast<float>(b);
            next_b_s = b;
            next_inv_b_s = 1.0f / bf;
            next_bg_s = bf / g;
            next_dhat_s = a.pred ? pr * (g / bf) : -1.0f;
        }
    };
    if (tid == 0) claim_next();
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            job_s = next_s;
            inv_b_s = next_inv_b_s;
            dhat_s = next_dhat_s;
            bg_s = next_bg_s;
            b_s = next_b_s;
        }
        __syncthreads();
        const int job = job_s;
        if (job >= a.n_subs || *abortp) break;
        const int j = a.order[job];
        const SubDesc s = a.subs[j];
        const int kpad = (s.n + 31) & ~31;  // MMA extent; TMA moves 64-wide boxes
        // learned bound: the predicted smallest |eigenvalue| of X0 = (T_j - mu I) / b_j (read
        // before this job rewrites b_j; negative when there is no prediction)
        const float dhat = dhat_s;
        // lower end of the interval the scaled schedule assumes for the current iterate's
        // |eigenvalues| (1 = plain steps), and the factor a of the current step
        float lsch = 1.0f, acur = 1.0f;

        const int zx0 = slot_z + 0, zx1 = slot_z + 2, zy = slot_z + 4;

        // on-chip form: the image of X (hi boxes, then lo boxes) at the start of the stage area
        const bool resident = kpad <= kResKpad;
        const int RB = (kpad + 63) >> 6;
        const uint32_t img_bytes = static_cast<uint32_t>(RB * RB) * 8192u;
        const uint32_t hi_off = 0u, lo_off = img_bytes;  // hi image, lo image (split form)

        // prologue: X0 = (T_j - mu I) / b_j in FP32, zero-padded to kpad x kpad, split hi/lo,
        // into the shared-memory image (on-chip form) or the slot's X buffer
        if (resident) {
            // rows of T_j through two shared-memory buffers by asynchronous 16-byte copies: the
            // copy of a batch of rows overlaps the split of the batch before
            const float inv_b = inv_b_s;
            const float* t = a.T + s.t_off;
            const int row_chunks = s.ld / 4;  // 16-byte chunks per row of T_j
            const int per = max(1, min(s.n, static_cast<int>(C::kStageBuf / (16u * row_chunks))));  // rows per batch
            const int batches = (s.n + per - 1) / per;
            auto issue = [&](int bi) {  // batch bi into buffer bi & 1 (every thread commits one group)
                if (bi < batches) {
                    const int r0 = bi * per, nr = min(per, s.n - r0);
                    uint8_t* buf_s = smem + kStageOff + (bi & 1) * C::kStageBuf;
                    const float* src = t + static_cast<int64_t>(r0) * s.ld;
                    for (int c = tid; c < nr * row_chunks; c += kThreads) cp_async16(buf_s + 16 * c, src + 4 * c);
                }
                cp_async_commit();
            };
            issue(0);
            issue(1);
            const int per_row = kpad / 8;
            for (int bi = 0; bi < batches; ++bi) {
                cp_async_wait<1>();  // this thread's copies of batch bi are done (bi + 1 may be pending)
                __syncthreads();     // ... and every thread's
                const int r0 = bi * per, r1 = bi + 1 == batches ? kpad : min(s.n, r0 + per);  // the last batch pads to kpad
                const float* buf_s = reinterpret_cast<const float*>(smem + kStageOff + (bi & 1) * C::kStageBuf);
                for (int e = tid; e < (r1 - r0) * per_row; e += kThreads) {
                    const int rr = e / per_row, c0 = (e - rr * per_row) * 8, r = r0 + rr;
                    float x[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = 0.0f;
                    // rows of T are zero in [n, ld); rows n .. kpad - 1 of the image are zero
                    if (r < s.n) {
                        const float4* src = reinterpret_cast<const float4*>(buf_s + static_cast<int64_t>(rr) * s.ld + c0);
                        if (c0 + 4 <= s.ld) {
                            const float4 v = src[0];
                            x[0] = v.x * inv_b; x[1] = v.y * inv_b; x[2] = v.z * inv_b; x[3] = v.w * inv_b;
                        }
                        if (c0 + 8 <= s.ld) {
                            const float4 v = src[1];
                            x[4] = v.x * inv_b; x[5] = v.y * inv_b; x[6] = v.z * inv_b; x[7] = v.w * inv_b;
                        }
                    }
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) split2<PREC, NB>(x[i], x[i + 1], hw[i >> 1], lw[i >> 1]);
                    const uint32_t off = img_offset(r, c0, RB);
                    *reinterpret_cast<uint4*>(smem + hi_off + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    if constexpr (NB == 2)
                        *reinterpret_cast<uint4*>(smem + lo_off + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
                __syncthreads();  // buffer bi & 1 is free again
                issue(bi + 2);
            }
            cp_async_wait<0>();
            fence_proxy_async_smem();
            if (tid == 0) { conv_s = 0; bad_s = 0; plain_s = 0; rprev_s = INFINITY; }
            __syncthreads();
            if (warp == 11 && lane == 0) claim_next();  // while the first product runs
        } else {
            const float inv_b = inv_b_s;
            const float* t = a.T + s.t_off;
            uint16_t* xh = ws + static_cast<int64_t>(zx0) * buf;
            uint16_t* xl = xh + buf;
            const int per_row = kpad / 8, total = kpad * per_row;
            constexpr int kU = 4;  // loads in flight per thread
            for (int e0 = tid; e0 < total; e0 += kU * kThreads) {
                float4 v[kU][2];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int e = e0 + u * kThreads;
                    const int r = e / per_row, c0 = (e - r * per_row) * 8;
                    v[u][0] = v[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    // rows of T are 16-byte aligned (ld is a multiple of 4) and zero in [n, ld)
                    if (e < total && r < s.n) {
                        const float4* src = reinterpret_cast<const float4*>(t + static_cast<int64_t>(r) * s.ld + c0);
                        if (c0 + 4 <= s.ld) v[u][0] = src[0];
                        if (c0 + 8 <= s.ld) v[u][1] = src[1];
                    }
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int e = e0 + u * kThreads;
                    if (e >= total) break;
                    const int r = e / per_row, c0 = (e - r * per_row) * 8;
                    const float x[8] = {v[u][0].x * inv_b, v[u][0].y * inv_b, v[u][0].z * inv_b, v[u][0].w * inv_b,
                                        v[u][1].x * inv_b, v[u][1].y * inv_b, v[u][1].z * inv_b, v[u][1].w * inv_b};
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) split2<PREC, NB>(x[i], x[i + 1], hw[i >> 1], lw[i >> 1]);
                    *reinterpret_cast<uint4*>(xh + static_cast<int64_t>(r) * a.ld + c0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    if constexpr (NB == 2)
                        *reinterpret_cast<uint4*>(xl + static_cast<int64_t>(r) * a.ld + c0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            }
            fence_proxy_async_global();
            if (tid == 0) { conv_s = 0; bad_s = 0; plain_s = 0; rprev_s = INFINITY; }
            __syncthreads();
            if (warp == 11 && lane == 0) claim_next();  // while the first product runs
        }

        // The factor c of the first step X1 = p(c X0), p(x) = x (3 - x^2) / 2, from the guaranteed
        // bound smax >= rho(X0) (every thread gets the same c and lsch).  Without the learned
        // bound X0 = A / G and c = 1.2 / s, then plain steps.  With rho_hat only, the prediction
        // passes the check when s <= 1.7 < sqrt 3 (rho_hat was not an underestimate beyond
        // that) and its scaling is kept, c = max(1, 1.2 / s).  With the predicted gap, the steps
        // follow the scaled schedule from l0 = dhat / s, c = ns_scale(l0) / s; the check is
        // dhat <= s (the gap cannot exceed the spectral radius), and the schedule converges
        // for any l0 in (0, 1].  A failed check falls back to c = 1.2 / s and plain steps (counted).
        auto start_factor = [&](float smax) -> float {
            float c = smax > 0.0f ? 1.2f / smax : 1.0f;
            if (a.use_model && smax > 0.0f) {
                const bool gap = dhat > 0.0f;
                if (gap ? dhat <= smax : smax <= 1.7f) {
                    if (gap) {
                        const float l0 = dhat / smax;
                        const float a0 = ns_scale(l0);
                        c = a0 / smax;
                        lsch = ns_next_lower(a0, l0);
                    } else {
                        c = fmaxf(1.0f, c);
                    }
                } else if (tid == 0) {
                    atomicAdd(a.fallbacks, 1);
                }
            }
            return c;
        };
        // the constants of a later step X' = p(a X) = alpha (Z - shift I) X, Z = X^2:
        // shift = 3 / a^2, alpha = -a^3 / 2 (a = 1: a plain step)
        auto next_step = [&](float& shift, float& alpha) {
            if (plain_s) lsch = 1.0f;
            acur = 1.0f;
            if (lsch < 1.0f) {
                const float f = ns_scale(lsch);
                shift = 3.0f / (f * f);
                alpha = -0.5f * f * f * f;
                lsch = ns_next_lower(f, lsch);
                acur = f;
            }
        };
        // The stopping rule (tid 0, after the residual ||X^2 - I||_F of the current step):
        // stop after this step when the residual is <= tau, unless the step is a scaled one
        // whose factor would move converged eigenvalues off 1 (p(a) = 1 - 1.5 (a - 1)^2 + ...);
        // then the schedule ends and the next steps are plain.
        auto converged = [&]() {
            if (acur - 1.0f <= kStopSlack) conv_s = 1;
            else plain_s = 1;
        };
        // one thread, with the residual r = ||X^2 - I||_F of the current step: the stopping
        // rule, or (single-pass forms) the rounding floor: r below a.stall_level and not half
        // of the previous step's residual.  FP32 throughout: FP64 arithmetic on the thread
        // that decides would hold a warp of the next pass for microseconds.
        auto check_stop = [&](float r) {
            if (!isfinite(r)) bad_s = 1;
            else if (r <= a.tau || (r < a.stall_level && r > 0.5f * rprev_s)) converged();
            rprev_s = r;
        };
        int cur = 0, done = 0;
        if (resident) {
            // ---------------------------------------------------------------
            // On-chip form.  Per iteration, for the 128-row tile 0:
            //   Z_0 <- X_0 X          (A and B from the shared-memory image)
            //   Z_0 <- A-operand form of Z_0 - shift I (hi, lo packed 16-bit, in place)
            //   Q_0 <- (Z_0 - shift I) X   (A from tensor memory, B from the image)
            //   X'_0 = alpha Q_0      into the image once every product of the
            //                         iteration has read it
            // and for the rows past 128 (kpad > 128) only the corner [128 .., 128 ..] of
            // each product, the rest being tile 0's columns transposed (see below).
            // Y X = X Y (Y is a polynomial in X).  Iteration 0 forms Z = X0^2 for
            // every row, bounds rho(Z), and continues with shift = 3/c^2 and
            // alpha = -c^3/2; later iterations use shift = 3, alpha = -1/2.  All 12
            // warps share the tensor-memory passes: warp w serves lanes 32 (w mod 4)
            // and the 32-column chunks c0 = 32 (w / 4) + 96 k; each pass loads its
            // next chunk while the current one is converted.
            // ---------------------------------------------------------------
            const int mtiles = (kpad + 127) >> 7;
            const int ksteps = kpad >> 4;
            const uint32_t idesc = idesc_f16(128, kpad, C::kFmt) | idesc_b_mn;
            const uint32_t smem_base = smem_u32(smem), img_lo = smem_base + lo_off, img_hi = smem_base + hi_off;
            // two row tiles (kpad in (128, 192]): tile 1 holds the wc = kpad - 128 last rows
            const int wc = kpad - 128;
            const uint32_t idesc_w = idesc_f16(128, wc > 0 ? wc : 32, C::kFmt) | idesc_b_mn;
            // Bz = (Z - shift I)[:, 128 ..] as an MN-major B operand (kpad K rows, one 64-column
            // block; hi boxes, then lo boxes) after the images; iteration 0's row-sum scratch at
            // 160 KB is used only before Bz is written
            const uint32_t bz_off = static_cast<uint32_t>(NB) * img_bytes;
            const uint32_t bz_hi = smem_base + bz_off, bz_lo = bz_hi + static_cast<uint32_t>(RB) * 8192u;
            float* rpart_s = reinterpret_cast<float*>(smem + 160 * 1024);  // [3][kResKpad], iteration 0 only
            float* rsum_s = rpart_s + 3 * kResKpad;
            float* rs2_s = rsum_s + kResKpad;
            float* csum_s = rs2_s + kResKpad;  // [4][64]: rows 128 .. over columns 0 .. 127, per lane quadrant
            float* tbsum_s = csum_s + 4 * 64;  // [64]: rows 128 .. over columns 128 .. (the corner)
            const uint32_t lbo = static_cast<uint32_t>(RB) * 8192u;
            const int q = warp & 3, part = warp >> 2;
            const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
            // d <- X_t X[:, col0 ..] (col0 a multiple of 64; N from idn)
            auto issue_xx_cols = [&](int t, uint32_t d, int col0, uint32_t idn) {
                const uint32_t cb = static_cast<uint32_t>(col0 >> 6) * lbo;
                for (int kk = 0; kk < ksteps; ++kk) {
                    const uint32_t aoff = static_cast<uint32_t>(((kk >> 2) * RB + 2 * t) * 8192 + (kk & 3) * 32);
                    const uint32_t boff = static_cast<uint32_t>((kk >> 2) * 8192 + (kk & 3) * 2048) + cb;
                    const uint64_t ah = sdesc_sw128(img_hi + aoff), bh = sdesc_mn_sw128_lbo(img_hi + boff, lbo);
                    tc_mma_f16(d, ah, bh, idn, kk ? 1u : 0u);
                    if constexpr (NB == 2) {
                        tc_mma_f16(d, ah, sdesc_mn_sw128_lbo(img_lo + boff, lbo), idn, 1u);
                        tc_mma_f16(d, sdesc_sw128(img_lo + aoff), bh, idn, 1u);
                    }
                }
            };
            auto issue_xx = [&](int t, uint32_t d) { issue_xx_cols(t, d, 0, idesc); };  // d <- X_t X
            // d <- X_1 Bz: rows 128 .. of X (the image) times (Z - shift I)[:, 128 ..] (N = wc)
            auto issue_cyx = [&](uint32_t d) {
                for (int kk = 0; kk < ksteps; ++kk) {
                    const uint32_t aoff = static_cast<uint32_t>(((kk >> 2) * RB + 2) * 8192 + (kk & 3) * 32);
                    const uint32_t boff = static_cast<uint32_t>((kk >> 2) * 8192 + (kk & 3) * 2048);
                    const uint64_t ah = sdesc_sw128(img_hi + aoff), bh = sdesc_mn_sw128_lbo(bz_hi + boff, lbo);
                    tc_mma_f16(d, ah, bh, idesc_w, kk ? 1u : 0u);
                    if constexpr (NB == 2) {
                        tc_mma_f16(d, ah, sdesc_mn_sw128_lbo(bz_lo + boff, lbo), idesc_w, 1u);
                        tc_mma_f16(d, sdesc_sw128(img_lo + aoff), bh, idesc_w, 1u);
                    }
                }
            };
            // A in tensor memory from column at: per 32 K values, 16 columns hi then 16 lo
            // d <- A X over the K steps [k0, k1) (k0 = 0 starts the accumulator)
            auto issue_yx_k = [&](uint32_t at, uint32_t d, int k0, int k1) {
                for (int kk = k0; kk < k1; ++kk) {
                    const uint32_t boff = static_cast<uint32_t>((kk >> 2) * 8192 + (kk & 3) * 2048);
                    const uint32_t ah = at + 32 * (kk >> 1) + 8 * (kk & 1);
                    const uint64_t bh = sdesc_mn_sw128_lbo(img_hi + boff, lbo);
                    tc_mma_f16_ta(d, ah, bh, idesc, kk ? 1u : 0u);
                    if constexpr (NB == 2) {
                        tc_mma_f16_ta(d, ah, sdesc_mn_sw128_lbo(img_lo + boff, lbo), idesc, 1u);
                        tc_mma_f16_ta(d, ah + 16, bh, idesc, 1u);
                    }
                }
            };
            auto issue_yx = [&](uint32_t at, uint32_t d) { issue_yx_k(at, d, 0, ksteps); };  // d <- A X
            auto mma_wait = [&]() {  // all threads
                mbar_wait(&mma_bar, mma_ph & 1u, &abort_s, a.status);
                ++mma_ph;
                tc_fence_after();
            };
            auto mma_wait2 = [&]() {  // all threads; the second barrier of the pipelined form
                mbar_wait(&mma_bar2, mma_ph2 & 1u, &abort_s, a.status);
                ++mma_ph2;
                tc_fence_after();
            };
            // Tensor-memory passes: thread (warp w, lane) owns row 128 t + 32 (w mod 4) + lane and
            // the 32-column chunks c0 = 32 (w / 4) + 96 k of the tile.
            //
            // convert: accumulator at acc -> A = C - shift I in place, each 32-column chunk becoming
            // 16 columns of packed hi pairs and 16 of lo pairs; with resid, r2 += ||C - I||_F^2 over
            // the thread's entries (rows and columns < n; zero elsewhere)
            // Padding is exact: rows and columns of X in [n, kpad) are zero, so are those of
            // Z = X X, of the A operand and of the second product.  Only the diagonal needs a
            // rule of its own, and rows past kpad (tile 1 of a submatrix with kpad <= 192) are
            // never read back, so their warps skip the passes.
            //
            // convert: accumulator at acc -> A = C - shift I in place, each 32-column chunk becoming
            // 16 columns of packed hi pairs and 16 of lo pairs; with resid, r2 += ||C - I||_F^2 over
            // the thread's entries (the n x n block; the padding contributes nothing)
            // to_bz (two-tile form, tile 0): the chunks at columns >= 128 also go to Bz (rows 0 .. 127),
            // and their residual counts twice (Z is symmetric: the block below the diagonal block)
            // In the two-tile form (to_bz) warp 10 is still issuing the corner product Z_c when
            // this pass starts, so its chunks go to the other two warps of its lane quadrant
            // (warps 2 and 6 take every other chunk).
            auto convert = [&](int t, uint32_t acc, float shift, bool resid, float& r2, bool to_bz = false) {
                const int row0 = 128 * t + 32 * q;  // the warp's first row
                if (row0 >= kpad) return;
                const bool live = row0 + lane < s.n;
                const bool shared2 = to_bz && q == 2;  // quadrant 2 without warp 10
                if (shared2 && part == 2) return;
                const int cstep = shared2 ? 64 : 96;
#pragma unroll 1
                for (int c0 = 32 * part; c0 < kpad; c0 += cstep) {
                    uint32_t raw[32];
                    tmem_ld32_issue(acc + lane_off + c0, raw);
                    tmem_wait_ld_regs(raw);
                    float y[32], sq = 0.0f;
                    if (c0 != row0) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            y[i] = __uint_as_float(raw[i]);
                            sq = fmaf(y[i], y[i], sq);
                        }
                    } else {  // the chunk of the warp's diagonal: element `lane` of each row
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const float v = __uint_as_float(raw[i]);
                            const bool d = (i == lane) && live;
                            const float e = d ? v - 1.0f : v;
                            y[i] = d ? v - shift : v;
                            sq = fmaf(e, e, sq);
                        }
                    }
                    const bool bz = to_bz && c0 >= 128;
                    if (resid) r2 += bz ? 2.0f * sq : sq;
                    uint32_t w[32];
#pragma unroll
                    for (int i = 0; i < 32; i += 2) split2<PREC, NB>(y[i], y[i + 1], w[i >> 1], w[16 + (i >> 1)]);
                    tmem_st32(acc + lane_off + c0, w);
                    if (bz) {
                        const int row = row0 + lane;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const uint32_t off = bz_off + img_offset(row, c0 - 128 + 8 * u, RB);
                            *reinterpret_cast<uint4*>(smem + off) = make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
                            if constexpr (NB == 2)
                                *reinterpret_cast<uint4*>(smem + off + RB * 8192) =
                                    make_uint4(w[16 + 4 * u], w[17 + 4 * u], w[18 + 4 * u], w[19 + 4 * u]);
                        }
                    }
                }
                tmem_wait_st();
            };
            // the corner Z[128 .., 128 ..] (accumulator at acc, wc columns; lanes = rows - 128):
            // (Z - shift I) into Bz rows 128 .. kpad - 1; residual once
            auto convert_corner = [&](uint32_t acc, float shift, bool resid, float& r2) {
                const int crow0 = 32 * q;  // the warp's first corner row
                if (crow0 >= wc) return;
                const int row = 128 + crow0 + lane;
                const bool live = row < s.n;
#pragma unroll 1
                for (int c0 = 32 * part; c0 < wc; c0 += 96) {
                    uint32_t raw[32];
                    tmem_ld32_issue(acc + lane_off + c0, raw);
                    tmem_wait_ld_regs(raw);
                    float y[32], sq = 0.0f;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float v = __uint_as_float(raw[i]);
                        const bool d = (c0 == crow0) && (i == lane) && live;
                        const float e = d ? v - 1.0f : v;
                        y[i] = d ? v - shift : v;
                        sq = fmaf(e, e, sq);
                    }
                    if (resid) r2 += sq;
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int i = 0; i < 32; i += 2) split2<PREC, NB>(y[i], y[i + 1], hw[i >> 1], lw[i >> 1]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t off = bz_off + img_offset(row, c0 + 8 * u, RB);
                        *reinterpret_cast<uint4*>(smem + off) = make_uint4(hw[4 * u], hw[4 * u + 1], hw[4 * u + 2], hw[4 * u + 3]);
                        if constexpr (NB == 2)
                            *reinterpret_cast<uint4*>(smem + off + RB * 8192) =
                                make_uint4(lw[4 * u], lw[4 * u + 1], lw[4 * u + 2], lw[4 * u + 3]);
                    }
                }
            };
            // Mirror of a 32 x 32 chunk of the iterate inside a diagonal block: the warp's rows
            // r0 .. r0 + 31, image columns c0 .. c0 + 31 (hi / lo pairs of the thread's row in
            // hw / lw), through the warp's transpose buffer.  Right of the warp's diagonal chunk
            // (c0 > r0) the chunk is also written transposed, as rows c0 .. c0 + 31 of columns
            // r0 .. r0 + 31; the diagonal chunk (c0 == r0) is written with its lower triangle
            // replaced by the mirror of its upper one.  So the iterate in the image is exactly
            // symmetric there (left as computed, its rounding asymmetry would grow from step to
            // step).  Lane l writes one row of 64 contiguous bytes per hi / lo image.
            // The single-pass forms mirror; the split form keeps the computed diagonal blocks: its
            // rounding (about 1e-7) leaves the asymmetric part far below the error bound over a
            // few steps, and the mirror would cost about 12% of the kernel on water-like inputs.
            constexpr bool kMirror = NB == 1;
            uint16_t* xsw = reinterpret_cast<uint16_t*>(smem + kXsOff * NB + static_cast<uint32_t>(warp) * kXsWarp);
            auto mirror_chunk = [&](const uint32_t (&hw)[16], const uint32_t (&lw)[16], int r0, int c0, bool diag) {
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const uint32_t* w = b == 0 ? hw : lw;
                    __syncwarp();
                    uint4* xr = reinterpret_cast<uint4*>(xsw + lane * 40);
#pragma unroll
                    for (int u = 0; u < 4; ++u) xr[u] = make_uint4(w[4 * u], w[4 * u + 1], w[4 * u + 2], w[4 * u + 3]);
                    __syncwarp();
                    uint32_t t[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const uint32_t x0 = xsw[(2 * k) * 40 + lane], x1 = xsw[(2 * k + 1) * 40 + lane];
                        if (diag) {  // own row from the diagonal on, the mirror left of it
                            t[k] = (2 * k < lane ? x0 : (w[k] & 0xFFFFu)) | ((2 * k + 1 < lane ? x1 : (w[k] >> 16)) << 16);
                        } else {
                            t[k] = x0 | (x1 << 16);
                        }
                    }
                    const uint32_t base = b == 0 ? hi_off : lo_off;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        *reinterpret_cast<uint4*>(smem + base + img_offset(c0 + lane, r0 + 8 * u, RB)) =
                            make_uint4(t[4 * u], t[4 * u + 1], t[4 * u + 2], t[4 * u + 3]);
                }
            };
            // drain: X'_t = alpha C (its padding is zero already) into the image (hi at hi_dst)
            // keep_a: also leave X' in the accumulator columns as the packed A operand (16 columns
            // of hi pairs, then 16 of lo pairs per 32-column chunk) of the next iteration's X X
            // (as computed: the mirror makes only the image exactly symmetric)
            // In the diagonal block (columns < 128) a warp writes the chunks from its diagonal
            // chunk on and mirrors them; the chunks left of it are the mirrors of other warps'.
            auto drain = [&](int t, uint32_t acc, float alpha, uint32_t hi_dst, bool keep_a = false) {
                const int row = 128 * t + 32 * q + lane;
                const int crow0 = 32 * q;  // the warp's first row inside the tile
                if (row - lane >= kpad) return;  // the warp's rows are all padding (kpad is a multiple of 32)
#pragma unroll 1
                for (int c0 = 32 * part; c0 < kpad; c0 += 96) {
                    uint32_t raw[32];
                    tmem_ld32_issue(acc + lane_off + c0, raw);
                    tmem_wait_ld_regs(raw);
                    float y[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) y[i] = alpha * __uint_as_float(raw[i]);
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int i = 0; i < 32; i += 2) split2<PREC, NB>(y[i], y[i + 1], hw[i >> 1], lw[i >> 1]);
                    const bool in_diag = kMirror && c0 < 128;
                    if (!in_diag || c0 > crow0) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const uint32_t off = img_offset(row, c0 + 8 * u, RB);
                            *reinterpret_cast<uint4*>(smem + hi_dst + off) = make_uint4(hw[4 * u], hw[4 * u + 1], hw[4 * u + 2], hw[4 * u + 3]);
                            if constexpr (NB == 2)
                                *reinterpret_cast<uint4*>(smem + lo_off + off) =
                                    make_uint4(lw[4 * u], lw[4 * u + 1], lw[4 * u + 2], lw[4 * u + 3]);
                        }
                    }
                    if (in_diag && c0 >= crow0) mirror_chunk(hw, lw, 128 * t + crow0, c0, c0 == crow0);
                    if (keep_a) {
                        uint32_t w[32];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            w[i] = hw[i];
                            w[16 + i] = lw[i];
                        }
                        tmem_st32(acc + lane_off + c0, w);
                    }
                }
                if (keep_a) tmem_wait_st();
            };
            // two-tile form: the columns 128 .. of tile 0 of X' as rows 128 .. of the image (X' is
            // symmetric), element by element, from the packed operand that drain left at acc.
            // Warps of parts 0 and 1 only (part 2 drains the corner meanwhile): with two chunks
            // (kpad 192) one each, with one (kpad 160) a half (16 columns) each.
            auto drain_t = [&](uint32_t acc) {
                if (part == 2) return;
                const int row = 32 * q + lane;
                const bool halves = wc <= 32;
                const int c0 = 128 + (halves ? 0 : 32 * part);
                if (c0 >= kpad) return;
                const int i0 = halves ? 16 * part : 0;
                uint32_t w[32];
                tmem_ld32_issue(acc + lane_off + c0, w);
                tmem_wait_ld_regs(w);
#pragma unroll
                for (int ii = 0; ii < 32; ++ii) {
                    if (halves && (ii < i0 || ii >= i0 + 16)) continue;  // warp-uniform
                    const int i = ii;
                    const uint32_t off = img_offset(c0 + i, row, RB);  // element (c0 + i, row)
                    const int sh = (i & 1) * 16;                       // pairs hold the even column low
                    *reinterpret_cast<uint16_t*>(smem + hi_off + off) = static_cast<uint16_t>(w[i >> 1] >> sh);
                    if constexpr (NB == 2)
                        *reinterpret_cast<uint16_t*>(smem + lo_off + off) = static_cast<uint16_t>(w[16 + (i >> 1)] >> sh);
                }
            };
            // the corner of X' = alpha C (accumulator at acc, wc columns) into rows and columns
            // 128 .., made exactly symmetric as the diagonal block of tile 0 in drain; by the
            // part-2 warps of the corner's lane quadrants (8, and 9 for wc = 64; never warp 10),
            // all its chunks, while parts 0 and 1 run drain_t
            auto drain_corner = [&](uint32_t acc, float alpha) {
                const int crow0 = 32 * q;
                if (crow0 >= wc || part != 2) return;
                const int row = 128 + crow0 + lane;
#pragma unroll 1
                for (int c0 = 0; c0 < wc; c0 += 32) {
                    if (kMirror && c0 < crow0) continue;  // the mirror of another warp's chunk
                    uint32_t raw[32];
                    tmem_ld32_issue(acc + lane_off + c0, raw);
                    tmem_wait_ld_regs(raw);
                    float y[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) y[i] = alpha * __uint_as_float(raw[i]);
                    uint32_t hw[16], lw[16];
#pragma unroll
                    for (int i = 0; i < 32; i += 2) split2<PREC, NB>(y[i], y[i + 1], hw[i >> 1], lw[i >> 1]);
                    if (!kMirror || c0 > crow0) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const uint32_t off = img_offset(row, 128 + c0 + 8 * u, RB);
                            *reinterpret_cast<uint4*>(smem + hi_off + off) = make_uint4(hw[4 * u], hw[4 * u + 1], hw[4 * u + 2], hw[4 * u + 3]);
                            if constexpr (NB == 2)
                                *reinterpret_cast<uint4*>(smem + lo_off + off) =
                                    make_uint4(lw[4 * u], lw[4 * u + 1], lw[4 * u + 2], lw[4 * u + 3]);
                        }
                    }
                    if (kMirror) mirror_chunk(hw, lw, 128 + crow0, 128 + c0, c0 == crow0);
                }
            };
            // Row sums sum_c |Z_rc| w_c of the first product Z (w = 1 when null), for the bound.
            // Rows 0 .. 127 (tile 0, accumulator acc): each warp adds its columns into
            // rpart_s[part, row].  Rows 128 .. (kpad > 128): Z is symmetric, so their columns
            // 0 .. 127 are tile 0's columns 128 .. summed over the rows (w of the row): the warp
            // holding such a 32-column chunk reduces it over its 32 lanes into csum_s[quadrant]
            // (a transpose-reduce: after five exchange steps lane L holds column L's sum);
            // their columns 128 .. are the corner product (scan_corner).
            auto colsum32 = [&](float (&v)[32]) -> float {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const bool up = lane & 16;
                    const float send = up ? v[i] : v[i + 16], keep = up ? v[i + 16] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const bool up = lane & 8;
                    const float send = up ? v[i] : v[i + 8], keep = up ? v[i + 8] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool up = lane & 4;
                    const float send = up ? v[i] : v[i + 4], keep = up ? v[i + 4] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const bool up = lane & 2;
                    const float send = up ? v[i] : v[i + 2], keep = up ? v[i + 2] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
                }
                const bool up = lane & 1;
                const float send = up ? v[0] : v[1], keep = up ? v[1] : v[0];
                return keep + __shfl_xor_sync(0xffffffffu, send, 1);
            };
            // No masks: the columns of Z past n are exactly zero, rows past n hold zeros (or, past
            // kpad, finite values of an earlier job whose sums are not kept), and w is zero past n.
            auto scan = [&](uint32_t acc, const float* w) {
                const int row = 32 * q + lane;
                const float wr = w ? w[row] : 1.0f;
                float sum = 0.0f;
#pragma unroll 1
                for (int c0 = 32 * part; c0 < kpad; c0 += 96) {
                    uint32_t raw[32];
                    tmem_ld32_issue(acc + c0 + lane_off, raw);
                    tmem_wait_ld();
                    if (w) {
                        const float4* w4 = reinterpret_cast<const float4*>(w + c0);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float4 wv = w4[i];
                            sum = fmaf(fabsf(__uint_as_float(raw[4 * i])), wv.x, sum);
                            sum = fmaf(fabsf(__uint_as_float(raw[4 * i + 1])), wv.y, sum);
                            sum = fmaf(fabsf(__uint_as_float(raw[4 * i + 2])), wv.z, sum);
                            sum = fmaf(fabsf(__uint_as_float(raw[4 * i + 3])), wv.w, sum);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i) sum += fabsf(__uint_as_float(raw[i]));
                    }
                    if (c0 >= 128) {  // warp-uniform
                        float v[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] = fabsf(__uint_as_float(raw[i])) * wr;
                        csum_s[q * 64 + (c0 - 128) + lane] = colsum32(v);
                    }
                }
                if (row < s.n) rpart_s[part * kResKpad + row] = sum;
            };
            // rows 128 + 32 q + lane over the corner's columns 128 .. (warps of part 0, quadrants
            // holding corner rows)
            auto scan_corner = [&](uint32_t acc, const float* w) {
                if (part != 0 || 32 * q >= wc) return;
                const int row = 128 + 32 * q + lane;
                float sum = 0.0f;
#pragma unroll 1
                for (int c0 = 0; c0 < wc; c0 += 32) {  // unmasked, as in scan
                    uint32_t raw[32];
                    tmem_ld32_issue(acc + c0 + lane_off, raw);
                    tmem_wait_ld();
                    if (w) {
                        const float4* w4 = reinterpret_cast<const float4*>(w + 128 + c0);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float4 wv = w4[i];
                            sum = fmaf(fabsf(__uint_as_float(raw[4 * i])), wv.x, sum);
                            sum = fmaf(fabsf(__uint_as_float(raw[4 * i + 1])), wv.y, sum);
                            sum = fmaf(fabsf(__uint_as_float(raw[4 * i + 2])), wv.z, sum);
                            sum = fmaf(fabsf(__uint_as_float(raw[4 * i + 3])), wv.w, sum);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i) sum += fabsf(__uint_as_float(raw[i]));
                    }
                }
                if (row < s.n) tbsum_s[row - 128] = sum;
            };
            // out[r] = the sum of r's parts in a fixed order (after a barrier), and the block's
            // maximum of out[r] (of out[r] / div[r] with div); every thread gets it
            auto gather_max = [&](float* out, const float* div) -> float {
                __syncthreads();
                float mx = 0.0f;
                for (int r = tid; r < s.n; r += kThreads) {
                    float v;
                    if (r < 128) {
                        v = (rpart_s[r] + rpart_s[kResKpad + r]) + rpart_s[2 * kResKpad + r];
                    } else {
                        const int c = r - 128;
                        v = ((csum_s[c] + csum_s[64 + c]) + (csum_s[128 + c] + csum_s[192 + c])) + tbsum_s[c];
                    }
                    out[r] = v;
                    mx = fmaxf(mx, div ? v / div[r] : v);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if (lane == 0) red_s[0][warp] = mx;
                __syncthreads();
                float m = 0.0f;
                for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, red_s[0][w]);
                return m;
            };

            // it = 0: the bound on rho(Z) from the first product's row sums (tile 0 in z0, the
            // corner in zc; after a barrier) and the a-posteriori scaling c = 1.2/s (every thread gets c)
            auto start_scale = [&](uint32_t z0, uint32_t zc) -> float {
                scan(z0, nullptr);
                if (mtiles > 1) scan_corner(zc, nullptr);
                const float rmax = gather_max(rsum_s, nullptr);
                float best = rmax;
                if (a.use_model && rmax > 0.0f) {
                    // one power step: w = the row sums (floored to stay positive), zero past n
                    for (int r = tid; r < kResKpad; r += kThreads) rsum_s[r] = r < s.n ? fmaxf(rsum_s[r], 1e-12f * rmax) : 0.0f;
                    __syncthreads();
                    scan(z0, rsum_s);
                    if (mtiles > 1) scan_corner(zc, rsum_s);
                    best = fminf(best, gather_max(rs2_s, rsum_s));
                }
                const float smax = sqrtf(best * (1.0f + 1e-4f));  // margin for FP32 summation
                const float scale = start_factor(smax);
                if (tid == 0) {  // next-step feature sqrt(rmax) b_j / G_j, and b_j / c
                    a.sq_ratio[j] = sqrtf(rmax * (1.0f + 1e-5f)) * bg_s;
                    a.bound[j] = b_s * static_cast<double>(1.0f / scale);
                }
                return scale;
            };
            // convergence of this step from ||X^2 - I||_F (the residual partials of every warp)
            auto decide = [&]() {
                float rr = 0.0f;
                for (int w = 0; w < kThreads / 32; ++w) rr += resid_s2[w];
                check_stop(sqrtf(rr));
            };

            if (mtiles == 1) {
                // kpad <= 128, one row tile.  Per iteration: Z -> TA; TA -> A operand of
                // Z - shift I; Q = A X -> TB; X' = alpha Q into the image.
                const uint32_t TA = tmem_base, TB = tmem_base + 160;
                for (int it = 0; it < a.max_iter; ++it) {
                    // A = Z - shift I and X' = alpha A X: shift = 3, alpha = -1/2 (Y = 3/2 I - 1/2 Z);
                    // at iteration 0 shift = 3/c^2, alpha = -c^3/2 (the a-posteriori scaling c);
                    // on the scaled schedule 3/a^2 and -a^3/2
                    float alpha = -0.5f, shift = 3.0f;
                    if (it > 0) next_step(shift, alpha);
                    if (warp == 1 && lane == 0) {
                        tc_fence_after();
                        issue_xx(0, TA);
                        tc_commit(&mma_bar);
                    }
                    mma_wait();  // Z
                    if (it == 0) {
                        __syncthreads();
                        if (*abortp) break;
                        const float c = start_scale(TA, 0u);
                        shift = 3.0f / (c * c);
                        alpha = -0.5f * c * c * c;
                    }
                    tc_fence_before();
                    __syncthreads();
                    if (*abortp) break;
                    float r2 = 0.0f;
                    convert(0, TA, shift, it > 0, r2);
                    r2 = warp_sum_f(r2);
                    if (lane == 0) resid_s2[warp] = r2;
                    tc_fence_before();
                    __syncthreads();
                    if (warp == 1 && lane == 0) {
                        tc_fence_after();
                        issue_yx(TA, TB);
                        tc_commit(&mma_bar);
                    }
                    if (tid == 0 && it > 0) decide();
                    mma_wait();
                    __syncthreads();
                    if (*abortp) break;
                    // into the image (the last X too: its owner columns are saved from there)
                    const bool last = conv_s || bad_s || it + 1 == a.max_iter;
                    drain(0, TB, alpha, hi_off);
                    fence_proxy_async_smem();
                    tc_fence_before();
                    __syncthreads();
                    cur ^= 1;
                    done = it + 1;
                    if (last) break;
                }
            } else {
                // kpad in (128, 192]: tile 0 = rows 0 .. 127, tile 1 = the wc = kpad - 128 rows
                // after them.  Z = X X and Q = (Z - shift I) X are symmetric (X commutes with
                // Z), so tile 1's rows are tile 0's columns 128 .. transposed except for the
                // corner [128 .., 128 ..]; only the corners are multiplied for tile 1, with N = wc:
                //   Z_0 = X_0 X -> TA (N = kpad), Z_c = X_1 X[:, 128 ..] -> TB (N = wc);
                //   TA -> A operand of Z_0 - shift I, its columns 128 .. also into Bz (rows
                //   0 .. 127), while Z_c is multiplied; Q_0 = A X -> TC;
                //   Z_c - shift I -> Bz rows 128 .. while Q_0 is multiplied; Q_c = X_1 Bz -> TB;
                //   X' = alpha Q: tile 0 into the image (and, packed, back into TC as the A operand
                //   of the next Z_0, so that after iteration 0 the first product reads A from
                //   tensor memory; the next Z_0 starts over K rows 0 .. 127 as soon as Q_c is
                //   done) while Q_c is multiplied (Q_c reads only
                //   rows 128 .. of the image and Bz; its A tile's rows past kpad, whose results are
                //   dropped, may see the new values), then tile 0's columns 128 .. as rows 128 ..
                //   (transposed) and the corner.
                // Iteration 0's row sums of the bound take rows 128 .. from tile 0's columns by
                // symmetry (no product for tile 1's columns 0 .. 127).  Tensor memory: TA, TB and
                // TC = the last kpad columns.
                const uint32_t TA = tmem_base, TB = tmem_base + kpad, TC = tmem_base + 512 - kpad;
                for (int it = 0; it < a.max_iter; ++it) {
                    float alpha = -0.5f, shift = 3.0f;
                    if (it > 0) next_step(shift, alpha);
                    if (it == 0 && warp == 1 && lane == 0) {  // later iterations: issued at the end of the previous one
                        tc_fence_after();
                        issue_xx(0, TA);
                        tc_commit(&mma_bar);
                        issue_xx_cols(1, TB, 128, idesc_w);
                        tc_commit(&mma_bar2);
                    }
                    mma_wait();  // Z_0
                    if (it == 0) {
                        mma_wait2();  // Z_c
                        __syncthreads();
                        if (*abortp) break;
                        const float c = start_scale(TA, TB);
                        shift = 3.0f / (c * c);
                        alpha = -0.5f * c * c * c;
                        tc_fence_before();
                        __syncthreads();
                        if (*abortp) break;
                    }
                    // later iterations: no barrier here (each thread waited for Z_0 itself; the
                    // abort flag is checked after the next barrier but one), so the conversion
                    // starts while warp 10 is still issuing Z_c
                    float r2 = 0.0f;
                    convert(0, TA, shift, it > 0, r2, true);
                    fence_proxy_async_smem();  // Bz rows 0 .. 127 (read by Q_c's products)
                    tc_fence_before();
                    __syncthreads();
                    if (warp == 1 && lane == 0) {
                        tc_fence_after();
                        issue_yx(TA, TC);
                        tc_commit(&mma_bar);
                    }
                    if (it > 0) mma_wait2();  // Z_c, multiplied while tile 0 was converted
                    convert_corner(TB, shift, it > 0, r2);
                    r2 = warp_sum_f(r2);
                    if (lane == 0) resid_s2[warp] = r2;
                    fence_proxy_async_smem();  // Bz rows 128 ..
                    tc_fence_before();
                    __syncthreads();
                    if (*abortp) break;
                    if (warp == 1 && lane == 0) {
                        tc_fence_after();
                        issue_cyx(TB);
                        tc_commit(&mma_bar2);
                    }
                    if (warp == 8 && lane == 0 && it > 0) decide();  // a warp without corner chunks
                    mma_wait();   // Q_0
                    drain(0, TC, alpha, hi_off, true);
                    fence_proxy_async_smem();  // rows 0 .. 127 of the image (read by the next Z_0)
                    mma_wait2();  // Q_c
                    tc_fence_before();
                    __syncthreads();
                    tc_fence_after();
                    if (*abortp) break;
                    const bool last = conv_s || bad_s || it + 1 == a.max_iter;
                    // the next Z_0 = X_0 X over K rows 0 .. 127 (image rows 0 .. 127 and the packed
                    // X_0 in TC are final) while rows 128 .. are written; issued by warp 10, which
                    // has no rows or chunks in the two passes below, so its wait for the MMA queue
                    // delays no pass
                    if (!last && warp == 10 && lane == 0) issue_yx_k(TC, TA, 0, 8);
                    drain_t(TC);
                    drain_corner(TB, alpha);
                    fence_proxy_async_smem();
                    tc_fence_before();
                    __syncthreads();
                    if (!last && warp == 10 && lane == 0) {
                        tc_fence_after();
                        issue_yx_k(TC, TA, 8, ksteps);  // K rows 128 ..
                        tc_commit(&mma_bar);
                        issue_xx_cols(1, TB, 128, idesc_w);  // the next Z_c, after Z_0 in the queue
                        tc_commit(&mma_bar2);
                    }
                    cur ^= 1;
                    done = it + 1;
                    if (last) break;
                }
            }
        } else {
        for (int it = 0; it < a.max_iter; ++it) {
            const int zx = cur ? zx1 : zx0, zn = cur ? zx0 : zx1;
            if (it == 0) {
                // A-posteriori scaling.  Z = X0^2; every eigenvalue of X0 satisfies
                // |lambda|^2 <= s^2 with s^2 the bound on rho(Z) below, so
                // X0' = c X0 with c = 1.2/s has all |lambda| <= 1.2 < sqrt(3) and the
                // iteration from X0' is guaranteed to converge.  The first step is
                // X1 = X0' (3/2 I - 1/2 X0'^2) = -1/2 c^3 X0 (Z - 3/c^2 I): only the
                // diagonal of Z changes before the second product.
                //
                // Bound on rho(Z) = rho(X0)^2 (Collatz-Wielandt): for any positive
                // vector w, rho(Z) <= rho(|Z|) <= max_r (|Z| w)_r / w_r.  w = 1 gives
                // the Gershgorin bound (the max row sum r, from a pass over the stored Z);
                // one power step (w = r) tightens it (on water-like submatrices from
                // about 1.5 rho to 1.35 rho).
                // The row-sum vector lives in the (still unused) buffer of X1.
                float* wv = reinterpret_cast<float*>(ws + static_cast<int64_t>(zn) * buf);
                gemm(kpad, s.n, 2, zx, zx, zy, 1.0f);  // Z = X0^2 (both triangles)
                {
                    const uint16_t* zh = ws + static_cast<int64_t>(zy) * buf;
                    const uint16_t* zl = zh + buf;
                    // row sums of |Z|, eight rows per warp at a time, 8 columns per lane and load
                    constexpr int kR = 8;
                    for (int r0 = warp * kR; r0 < kpad; r0 += kR * (kThreads / 32)) {
                        float acc[kR];
#pragma unroll
                        for (int u = 0; u < kR; ++u) acc[u] = 0.0f;
                        for (int c = 8 * lane; c < kpad; c += 256) {
#pragma unroll
                            for (int u = 0; u < kR; ++u) {
                                float zr[8];
                                const int r = min(r0 + u, kpad - 1);  // rows past kpad repeat the last (not stored)
                                load8<PREC, NB>(zh + static_cast<int64_t>(r) * a.ld + c, zl + static_cast<int64_t>(r) * a.ld + c, zr);
#pragma unroll
                                for (int i = 0; i < 8; ++i) acc[u] += fabsf(zr[i]);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kR; ++u) {
                            const float v = warp_sum_f(acc[u]);
                            if (lane == 0 && r0 + u < kpad) wv[r0 + u] = v;
                        }
                    }
                }
                __syncthreads();
                float rmax = 0.0f;
                for (int r = tid; r < s.n; r += kThreads) rmax = fmaxf(rmax, wv[r]);
                rmax = block_max2(rmax, 0.0f).x;
                float best = rmax;
                uint16_t* zh = ws + static_cast<int64_t>(zy) * buf;
                uint16_t* zl = zh + buf;
                if (rmax > 0.0f) {  // (a pass over Z is cheap next to the products at these sizes)
                    // w > 0: rows that are zero in Z get a tiny positive weight
                    for (int c = tid; c < s.n; c += kThreads) wv[c] = fmaxf(wv[c], 1e-12f * rmax);
                    __syncthreads();
                    float q = 0.0f;
                    // (|Z| w)_r for eight rows per warp at a time, 8 columns per lane and load
                    constexpr int kR = 8;
                    for (int r0 = warp * kR; r0 < s.n; r0 += kR * (kThreads / 32)) {
                        float acc[kR];
#pragma unroll
                        for (int u = 0; u < kR; ++u) acc[u] = 0.0f;
                        for (int c = 8 * lane; c < kpad; c += 256) {
                            const float4 w0 = *reinterpret_cast<const float4*>(wv + c);
                            const float4 w1 = *reinterpret_cast<const float4*>(wv + c + 4);
                            const float wc[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                            float zr[kR][8];
#pragma unroll
                            for (int u = 0; u < kR; ++u) {
                                const int r = min(r0 + u, s.n - 1);  // rows past n repeat the last (ignored below)
                                load8<PREC, NB>(zh + static_cast<int64_t>(r) * a.ld + c, zl + static_cast<int64_t>(r) * a.ld + c, zr[u]);
                            }
#pragma unroll
                            for (int u = 0; u < kR; ++u)
#pragma unroll
                                for (int i = 0; i < 8; ++i) acc[u] = fmaf(fabsf(zr[u][i]), wc[i], acc[u]);
                        }
#pragma unroll
                        for (int u = 0; u < kR; ++u) {
                            const float v = warp_sum_f(acc[u]);
                            if (r0 + u < s.n) q = fmaxf(q, v / wv[r0 + u]);
                        }
                    }
                    best = fminf(best, block_max2(q, 0.0f).x);
                }
                const float smax = sqrtf(best * (1.0f + 1e-4f));  // margin for FP32 summation
                const float scale = start_factor(smax);
                // Z_rr -= 3 / c^2 (in place, the split re-done)
                const float shift = 3.0f / (scale * scale);
                for (int r = tid; r < s.n; r += kThreads) {
                    const int64_t o = static_cast<int64_t>(r) * a.ld + r;
                    float z = from16<PREC>(zh[o]);
                    if constexpr (NB == 2) z += from16<PREC>(zl[o]);
                    z -= shift;
                    if constexpr (NB == 2) {
                        const uint16_t hi = to16<PREC>(z);
                        zh[o] = hi;
                        zl[o] = to16<PREC>(z - from16<PREC>(hi));
                    } else {
                        zh[o] = to16<PREC>(z);
                    }
                }
                fence_proxy_async_global();
                if (tid == 0) {
                    // feature of the next snapshot: the Gershgorin bound of A^2, over G; and the
                    // effective scaling b_j / c of X0'
                    a.sq_ratio[j] = sqrtf(rmax * (1.0f + 1e-5f)) * bg_s;
                    a.bound[j] = b_s * static_cast<double>(1.0f / scale);
                }
                __syncthreads();
                gemm(kpad, s.n, 2, zx, zy, zn, -0.5f * scale * scale * scale);  // X1 = -c^3/2 X0 (Z - 3/c^2 I)
            } else {
                float shift = 3.0f, alpha = -0.5f;
                next_step(shift, alpha);
                // Y = a (3/2 I - a^2/2 X^2) = alpha X^2 - alpha shift I: the scaled step X' = X Y
                gemm(kpad, s.n, 1, zx, zx, zy, alpha, -alpha * shift);  // Y = 3/2 I - 1/2 X^2 when plain
                if (tid == 0) {
                    float r2 = 0.0f;
                    for (int w = 0; w < kEpiWarps; ++w) r2 += resid_s[w];
                    check_stop(sqrtf(r2));
                }
                gemm(kpad, s.n, 2, zx, zy, zn, 1.0f);  // X' = X Y
            }
            cur ^= 1;
            done = it + 1;
            if (conv_s || bad_s || *abortp) break;
        }
        }  // streamed form
        if (*abortp) break;
        if (tid == 0) {
            a.iters[j] = done;
            atomicAdd(a.work_n3, static_cast<unsigned long long>(s.n) * s.n * s.n * done);
            if (bad_s) atomicCAS(a.status, kOk, kErrNonfinite);
            else if (!conv_s) atomicCAS(a.status, kOk, kErrNoconv);
        }
        // the whole final X for FP64 finishing steps
        if (a.xfull) {
            double* xf = a.xfull + s.t_off;
            for (int e = tid; e < s.n * s.n; e += blockDim.x) {
                const int r = e / s.n, c = e - r * s.n;
                float x;
                if (resident) {
                    const uint32_t off = img_offset(r, c, RB);
                    x = from16<PREC>(*reinterpret_cast<const uint16_t*>(smem + hi_off + off));
                    if constexpr (NB == 2) x += from16<PREC>(*reinterpret_cast<const uint16_t*>(smem + lo_off + off));
                } else {
                    const int64_t o = static_cast<int64_t>(r) * a.ld + c;
                    const uint16_t* fh = ws + static_cast<int64_t>(cur ? zx1 : zx0) * buf;
                    x = from16<PREC>(fh[o]);
                    if constexpr (NB == 2) x += from16<PREC>(fh[buf + o]);
                }
                xf[static_cast<int64_t>(r) * s.ld + c] = static_cast<double>(x);
            }
        }
        // save columns own .. own + b_j of the final X (the method keeps the
        // columns; the iterate is symmetric only up to rounding) for the scatter
        {
            float* dst = a.xown + s.x_off;
            if (resident) {  // the final X is the shared-memory image
                for (int e = tid; e < s.n * s.bown; e += blockDim.x) {
                    const int q = e / s.n, i = e - q * s.n;
                    const uint32_t off = img_offset(i, s.own + q, RB);
                    float x = from16<PREC>(*reinterpret_cast<const uint16_t*>(smem + hi_off + off));
                    if constexpr (NB == 2) x += from16<PREC>(*reinterpret_cast<const uint16_t*>(smem + lo_off + off));
                    dst[e] = x;
                }
            } else {
                const uint16_t* fh = ws + static_cast<int64_t>(cur ? zx1 : zx0) * buf;
                const uint16_t* fl = fh + buf;
                for (int e = tid; e < s.n * s.bown; e += blockDim.x) {
                    const int q = e / s.n, i = e - q * s.n;
                    const int64_t o = static_cast<int64_t>(i) * a.ld + s.own + q;
                    float x = from16<PREC>(fh[o]);
                    if constexpr (NB == 2) x += from16<PREC>(fl[o]);
                    dst[e] = x;
                }
            }
        }
        __syncthreads();
    }

    // teardown: on a timeout, let copies and MMAs in flight finish (bounded) before freeing TMEM
    __syncthreads();
    if (*abortp && tid == 0) {
        for (int it = m_consumed_s; it < p_issued_s; ++it)
            mbar_wait_plain(&full_bar[it % S], (it / S) & 1, 1u << 20);
    }
    if (*abortp && warp == 1 && lane == 0) {
        tc_commit(&drain_bar);
        mbar_wait_plain(&drain_bar, 0, 1u << 20);
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

size_t ns_tc_smem_bytes(int precision) {
    switch (precision) {
        case 1: return TcCfg<1>::kDynSmem;
        case 2: return TcCfg<2>::kDynSmem;
        case 3: return TcCfg<3>::kDynSmem;
        default: return 0;
    }
}

template <int PREC>
static cudaError_t launch_prec(const NsTcArgs& a, const CUtensorMap& tmap, int max_nblk, cudaStream_t st) {
    (void)max_nblk;
    const size_t smem = TcCfg<PREC>::kDynSmem;
    cudaError_t e = cudaFuncSetAttribute(k_ns_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    k_ns_tc<PREC><<<a.n_slots, kThreads, smem, st>>>(a, tmap);
    return cudaGetLastError();
}

cudaError_t launch_ns_tc(const NsTcArgs& a, int precision, const CUtensorMap& tmap, int max_nblk, cudaStream_t st) {
    switch (precision) {
        case 1: return launch_prec<1>(a, tmap, max_nblk, st);
        case 2: return launch_prec<2>(a, tmap, max_nblk, st);
        case 3: return launch_prec<3>(a, tmap, max_nblk, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace smx
