// Newton-Schulz sign iteration on the tcgen05 tensor cores.
//
// Eq. 13: sign(A) = A (A^2)^(-1/2).  Per submatrix (Fig. 2 step (ii)) the
// iteration X_{k+1} = X_k Y_k, Y_k = 3/2 I - 1/2 X_k^2, X_0 = (T_j - mu I)/b_j
// runs entirely inside one persistent CTA, so each submatrix keeps its own
// iteration count and stopping decision.  The dense contractions are the
// paper's low-precision tensor-unit work (Section 3): FP16 (or BF16) operands,
// FP32 accumulation in tensor memory.  In the split form each operand is held
// as hi + lo (two FP16 numbers, about 22 significant bits) and every product
// is hi*hi + hi*lo + lo*hi, all accumulated in FP32.
//
// CTA layout (256 threads):
//   warp 0       TMA producer (one lane): 64-wide K chunks of A (128 rows) and
//                B (up to 256 rows; 128 in the split form) into a ring of
//                shared-memory stages
//   warp 1       MMA issuer (one lane): tcgen05.mma M=128, N<=256, K=16 into
//                one of two TMEM accumulator buffers (128 lanes x 256 FP32
//                columns each)
//   warps 4..7   epilogue: tcgen05.ld, Y = 3/2 I - 1/2 acc (or X' = acc),
//                residual ||X^2 - I||_F^2, split to hi/lo, store to the
//                CTA's workspace slot in global memory (L2-resident)
// Operands and results live in the slot's six 16-bit ld x ld buffers
// (X0 hi/lo, X1 hi/lo, Y hi/lo); X and Y are symmetric, so a K-major B
// operand is just the row-major matrix.
#include "smx_finish.cuh"
#include "smx_kernels.h"

namespace smx {

namespace {

constexpr uint32_t kABytes = 128 * 128;  // 128 rows x 64 K x 2 B

// Split form: N tiles of at most 128 columns, each with two FP32 TMEM
// accumulators -- hi*hi in one, hi*lo + lo*hi in the other -- summed in the
// epilogue.  The tensor core rounds its FP32 accumulator toward zero after
// every instruction; keeping the small cross products out of the main
// accumulator cuts those roundings of the large partial sums by three.
template <int PREC>
struct TcCfg {
    static constexpr int kNb = (PREC == 1) ? 2 : 1;        // operand buffers per matrix (hi[, lo])
    static constexpr int kNmax = (PREC == 1) ? 128 : 256;  // columns per N tile
    static constexpr uint32_t kBBytes = kNmax * 128;       // kNmax rows x 64 K x 2 B
    static constexpr int kStages = (PREC == 1) ? 3 : 4;    // smem ring depth
    static constexpr uint32_t kStage = kNb * (kABytes + kBBytes);
    static constexpr int kFmt = (PREC == 3) ? 1 : 0;       // 0 = FP16, 1 = BF16
    static constexpr size_t kDynSmem = 1024 + static_cast<size_t>(kStages) * kStage;
};

template <int PREC>
__device__ __forceinline__ uint16_t to16(float x) {
    if constexpr (PREC == 3) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    else return __half_as_ushort(__float2half_rn(x));
}
template <int PREC>
__device__ __forceinline__ uint16_t to16d(double x) {
    if constexpr (PREC == 3) return __bfloat16_as_ushort(__double2bfloat16(x));
    else return __half_as_ushort(__double2half(x));
}
template <int PREC>
__device__ __forceinline__ float from16(uint16_t h) {
    if constexpr (PREC == 3) return __bfloat162float(__ushort_as_bfloat16(h));
    else return __half2float(__ushort_as_half(h));
}

__device__ __forceinline__ bool mbar_wait_plain(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace

template <int PREC>
__global__ void __launch_bounds__(256, 1) k_ns_tc(NsTcArgs a, const __grid_constant__ CUtensorMap tmap) {
    using C = TcCfg<PREC>;
    constexpr int NB = C::kNb, S = C::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    int* ls_smem = reinterpret_cast<int*>(smem + static_cast<size_t>(S) * C::kStage);

    __shared__ uint64_t full_bar[S], empty_bar[S], tfull[2], tempty[2], drain_bar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s, job_s, conv_s, bad_s, p_issued_s, m_consumed_s;
    __shared__ double resid_s[4];
    __shared__ double scratch[32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* const abortp = &abort_s;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], 4);
        }
        mbar_init(&drain_bar, 1);
        abort_s = 0;
        p_issued_s = 0;
        m_consumed_s = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(&tmem_base_s, 512);
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_s;

    // role-local pipeline positions, continuous over all GEMMs of the CTA
    uint32_t p_it = 0;                 // producer: K chunks issued
    uint32_t m_it = 0, m_tile = 0;     // MMA: K chunks consumed, tiles issued
    uint32_t e_tile = 0;               // epilogue: tiles drained
    const int64_t buf = static_cast<int64_t>(a.ld) * a.ld;
    uint16_t* ws = static_cast<uint16_t*>(a.ws);
    const int slot_z = blockIdx.x * 6;

    // One product C = A * B^T over the K range [0, kpad) into buffer zo.
    // mode 1: zo = 3/2 I - 1/2 A A (residual accumulated); mode 2: zo = A B.
    auto gemm = [&](int kpad, int n, int mode, int za, int zb, int zo) {
        constexpr int NT = C::kNmax;
        const int mtiles = (kpad + 127) / 128, ntiles = (kpad + NT - 1) / NT, kchunks = kpad / 64;
        if (warp == 0) {
            if (lane == 0) {
                for (int mt = 0; mt < mtiles && !*abortp; ++mt)
                    for (int nt = 0; nt < ntiles && !*abortp; ++nt) {
                        const int nn = min(NT, kpad - NT * nt);
                        if (NT * nt + nn <= 128 * mt) continue;  // strictly below the diagonal
                        for (int kc = 0; kc < kchunks; ++kc) {
                            const int stage = p_it % S;
                            const uint32_t round = p_it / S;
                            if (round > 0 && !mbar_wait(&empty_bar[stage], (round - 1) & 1, &abort_s, a.status)) break;
                            uint8_t* st = smem + stage * C::kStage;
                            mbar_arrive_expect_tx(&full_bar[stage], NB * (kABytes + static_cast<uint32_t>(nn) * 128));
                            for (int b = 0; b < NB; ++b) {
                                uint8_t* sa = st + b * kABytes;
                                tma_load_3d(sa, &tmap, kc * 64, 128 * mt, za + b, &full_bar[stage]);
                                tma_load_3d(sa + 8192, &tmap, kc * 64, 128 * mt + 64, za + b, &full_bar[stage]);
                                uint8_t* sb = st + NB * kABytes + b * C::kBBytes;
                                for (int h = 0; h < nn / 64; ++h)
                                    tma_load_3d(sb + h * 8192, &tmap, kc * 64, NT * nt + 64 * h, zb + b, &full_bar[stage]);
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
                    for (int nt = 0; nt < ntiles && !*abortp; ++nt) {
                        const int nn = min(NT, kpad - NT * nt);
                        if (NT * nt + nn <= 128 * mt) continue;
                        const uint32_t abuf = m_tile & 1, around = m_tile >> 1;
                        if (around > 0 && !mbar_wait(&tempty[abuf], (around - 1) & 1, &abort_s, a.status)) break;
                        tc_fence_after();
                        const uint32_t d = tmem_base + abuf * 256;        // main accumulator
                        const uint32_t dx = d + 128;                      // cross terms (split form)
                        const uint32_t idesc = idesc_f16(128, nn, C::kFmt);
                        bool ok = true;
                        for (int kc = 0; kc < kchunks; ++kc) {
                            const int stage = m_it % S;
                            const uint32_t round = m_it / S;
                            if (!mbar_wait(&full_bar[stage], round & 1, &abort_s, a.status)) { ok = false; break; }
                            tc_fence_after();
                            const uint32_t base = smem_u32(smem + stage * C::kStage);
                            const uint32_t a_hi = base, a_lo = base + kABytes;
                            const uint32_t b_hi = base + NB * kABytes, b_lo = b_hi + C::kBBytes;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint32_t acc = (kc | kk) ? 1u : 0u;
                                tc_mma_f16(d, sdesc_sw128(a_hi + kk * 32), sdesc_sw128(b_hi + kk * 32), idesc, acc);
                                if constexpr (NB == 2) {
                                    tc_mma_f16(dx, sdesc_sw128(a_hi + kk * 32), sdesc_sw128(b_lo + kk * 32), idesc, acc);
                                    tc_mma_f16(dx, sdesc_sw128(a_lo + kk * 32), sdesc_sw128(b_hi + kk * 32), idesc, 1u);
                                }
                            }
                            tc_commit(&empty_bar[stage]);
                            ++m_it;
                        }
                        if (!ok) break;
                        tc_commit(&tfull[abuf]);
                        ++m_tile;
                    }
                m_consumed_s = static_cast<int>(m_it);
            }
            __syncwarp();
        } else if (warp >= 4) {
            const int q = warp & 3;
            const int lrow = q * 32 + lane;
            double r2 = 0.0;
            for (int mt = 0; mt < mtiles; ++mt)
                for (int nt = 0; nt < ntiles; ++nt) {
                    const int nn = min(NT, kpad - NT * nt);
                    if (NT * nt + nn <= 128 * mt) continue;
                    const uint32_t abuf = e_tile & 1, around = e_tile >> 1;
                    int ok = 1;
                    if (lane == 0) ok = mbar_wait(&tfull[abuf], around & 1, &abort_s, a.status) ? 1 : 0;
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) { mt = mtiles; break; }
                    tc_fence_after();
                    const int row = 128 * mt + lrow;
                    uint16_t* out_hi = ws + static_cast<int64_t>(zo) * buf + static_cast<int64_t>(row) * a.ld;
                    uint16_t* out_lo = out_hi + buf;
                    for (int c0 = 0; c0 < nn; c0 += 32) {
                        float v[32];
                        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + abuf * 256 + c0;
                        tmem_ld32(taddr, v);
                        if constexpr (NB == 2) {
                            float vx[32];
                            tmem_ld32(taddr + 128, vx);
#pragma unroll
                            for (int i = 0; i < 32; ++i) v[i] += vx[i];
                        }
                        if (row < kpad) {
                            const int col0 = NT * nt + c0;
                            uint32_t hw[16], lw[16];
#pragma unroll
                            for (int i = 0; i < 32; i += 2) {
                                uint16_t h2[2], l2[2];
#pragma unroll
                                for (int u = 0; u < 2; ++u) {
                                    const int col = col0 + i + u;
                                    const bool valid = row < n && col < n;
                                    float y;
                                    if (mode == 1) {
                                        const float dl = (row == col) ? 1.0f : 0.0f;
                                        y = valid ? (1.5f * dl - 0.5f * v[i + u]) : 0.0f;
                                        if (valid && col >= row) {  // upper triangle, off-diagonal counted twice
                                            const double e = static_cast<double>(v[i + u]) - dl;
                                            r2 += (col == row ? 1.0 : 2.0) * e * e;
                                        }
                                    } else {
                                        y = valid ? v[i + u] : 0.0f;
                                    }
                                    h2[u] = to16<PREC>(y);
                                    l2[u] = (NB == 2) ? to16<PREC>(y - from16<PREC>(h2[u])) : 0;
                                }
                                hw[i >> 1] = static_cast<uint32_t>(h2[0]) | (static_cast<uint32_t>(h2[1]) << 16);
                                lw[i >> 1] = static_cast<uint32_t>(l2[0]) | (static_cast<uint32_t>(l2[1]) << 16);
                            }
                            // The result is symmetric; only its upper triangle (col >= row) is
                            // taken from this tile and mirrored, so the stored matrix is exactly
                            // symmetric.  (A K-major B operand read from rows is the transpose;
                            // any antisymmetric rounding residue would double per iteration.)
                            if (col0 >= row) {
                                uint4* dh = reinterpret_cast<uint4*>(out_hi + col0);
#pragma unroll
                                for (int u = 0; u < 4; ++u) dh[u] = make_uint4(hw[4 * u], hw[4 * u + 1], hw[4 * u + 2], hw[4 * u + 3]);
                                if constexpr (NB == 2) {
                                    uint4* dlo = reinterpret_cast<uint4*>(out_lo + col0);
#pragma unroll
                                    for (int u = 0; u < 4; ++u) dlo[u] = make_uint4(lw[4 * u], lw[4 * u + 1], lw[4 * u + 2], lw[4 * u + 3]);
                                }
                            } else if (col0 + 31 >= row) {
#pragma unroll
                                for (int i = 0; i < 32; ++i)
                                    if (col0 + i >= row) {
                                        out_hi[col0 + i] = static_cast<uint16_t>(hw[i >> 1] >> (16 * (i & 1)));
                                        if constexpr (NB == 2) out_lo[col0 + i] = static_cast<uint16_t>(lw[i >> 1] >> (16 * (i & 1)));
                                    }
                            }
                            if (col0 + 31 > row) {
                                uint16_t* mh = ws + static_cast<int64_t>(zo) * buf + row;
#pragma unroll
                                for (int i = 0; i < 32; ++i)
                                    if (col0 + i > row) {
                                        const int64_t o = static_cast<int64_t>(col0 + i) * a.ld;
                                        mh[o] = static_cast<uint16_t>(hw[i >> 1] >> (16 * (i & 1)));
                                        if constexpr (NB == 2) mh[o + buf] = static_cast<uint16_t>(lw[i >> 1] >> (16 * (i & 1)));
                                    }
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[abuf]);
                    ++e_tile;
                }
            r2 = warp_sum(r2);
            if (lane == 0) resid_s[q] = r2;
            fence_proxy_async_global();
        }
        __syncthreads();
    };

    for (;;) {
        if (tid == 0) job_s = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int job = job_s;
        if (job >= a.n_subs || *abortp) break;
        const int j = a.order[job];
        const SubDesc s = a.subs[j];
        const int kpad = (s.n + 63) & ~63;
        const int zx0 = slot_z + 0, zx1 = slot_z + 2, zy = slot_z + 4;

        // prologue: X0 = (T_j - mu I) / b_j, zero-padded to kpad x kpad, split hi/lo
        {
            const double inv_b = 1.0 / a.bound[j];
            const double* t = a.T + s.t_off;
            uint16_t* xh = ws + static_cast<int64_t>(zx0) * buf;
            uint16_t* xl = xh + buf;
            const int per_row = kpad / 8;
            for (int e = tid; e < kpad * per_row; e += blockDim.x) {
                const int r = e / per_row, c0 = (e - r * per_row) * 8;
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    uint16_t h2[2], l2[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int c = c0 + i + u;
                        const double x = (r < s.n && c < s.n) ? t[static_cast<int64_t>(r) * s.ld + c] * inv_b : 0.0;
                        h2[u] = to16d<PREC>(x);
                        l2[u] = (NB == 2) ? to16d<PREC>(x - static_cast<double>(from16<PREC>(h2[u]))) : 0;
                    }
                    hw[i >> 1] = static_cast<uint32_t>(h2[0]) | (static_cast<uint32_t>(h2[1]) << 16);
                    lw[i >> 1] = static_cast<uint32_t>(l2[0]) | (static_cast<uint32_t>(l2[1]) << 16);
                }
                *reinterpret_cast<uint4*>(xh + static_cast<int64_t>(r) * a.ld + c0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                if constexpr (NB == 2)
                    *reinterpret_cast<uint4*>(xl + static_cast<int64_t>(r) * a.ld + c0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            fence_proxy_async_global();
            if (tid == 0) { conv_s = 0; bad_s = 0; }
            __syncthreads();
        }

        int cur = 0, done = 0;
        for (int it = 0; it < a.max_iter; ++it) {
            const int zx = cur ? zx1 : zx0, zn = cur ? zx0 : zx1;
            gemm(kpad, s.n, 1, zx, zx, zy);  // Y = 3/2 I - 1/2 X^2
            if (tid == 0) {
                const double r2 = resid_s[0] + resid_s[1] + resid_s[2] + resid_s[3];
                if (!isfinite(r2)) bad_s = 1;
                else if (sqrt(r2) <= a.tau) conv_s = 1;
            }
            gemm(kpad, s.n, 2, zx, zy, zn);  // X' = X Y
            cur ^= 1;
            done = it + 1;
            if (conv_s || bad_s || *abortp) break;
        }
        if (*abortp) break;
        if (tid == 0) {
            a.iters[j] = done;
            atomicAdd(a.work_n3, static_cast<unsigned long long>(s.n) * s.n * s.n * done);
            if (bad_s) atomicCAS(a.status, kOk, kErrNonfinite);
            else if (!conv_s) atomicCAS(a.status, kOk, kErrNoconv);
        }
        const uint16_t* fh = ws + static_cast<int64_t>(cur ? zx1 : zx0) * buf;
        const uint16_t* fl = fh + buf;
        const int ld = a.ld;
        auto xrow = [&](int q, int i) -> double {
            const int64_t o = static_cast<int64_t>(s.own + q) * ld + i;
            double x = from16<PREC>(fh[o]);
            if constexpr (NB == 2) x += from16<PREC>(fl[o]);
            return x;
        };
        finish_column(s, a.pv, a.H, a.D, a.partial, xrow, ls_smem, scratch);
        __syncthreads();
    }

    // teardown: on a timeout, let copies and MMAs in flight finish (bounded) before freeing TMEM
    __syncthreads();
    if (abort_s && tid == 0) {
        for (int it = m_consumed_s; it < p_issued_s; ++it)
            mbar_wait_plain(&full_bar[it % S], (it / S) & 1, 1u << 20);
    }
    if (abort_s && warp == 1 && lane == 0) {
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
    const size_t smem = TcCfg<PREC>::kDynSmem + sizeof(int) * (static_cast<size_t>(max_nblk) + 1);
    cudaError_t e = cudaFuncSetAttribute(k_ns_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.work_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_ns_tc<PREC><<<a.n_slots, 256, smem, st>>>(a, tmap);
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
