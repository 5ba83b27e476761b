// Gower interpolation (Eq. (2)) on the tensor cores for byte-valued data of
// any width d (image-like rows of pixels 0..255).
//
// For a tile of 128 new points and every chunk of 256 landmarks:
//   S = Y L^T            (tcgen05.mma into TMEM, K streamed 128 bytes at a time)
//   A^2 = ||y||^2 + ||l||^2 - 2 S, clamped at 0       (epilogue, FP32)
//   X  += A^2 W          (W = -1/2 V Lambda^{-1/2}, r <= 16 columns)
// and finally X += b.  A^2 never leaves the chip.
//
// Two operand encodings, both exact for integers 0..255:
//   kBf16:  y and l as BF16 (8 significant bits hold every byte value);
//           one kind::f16 MMA per 16-element K step.
//   kFp8:   each byte split into nibbles y = 16 h + g (h, g in 0..15), stored
//           as E4M3 values 16h and g (each exactly representable).  Rows of
//           A are [16h | g]; the landmarks are stored twice, B1 = [16h | g]
//           and B2 = [g | 16h], so that A.B1 + A.B2 = 256 hh' + gg' + 16 (hg'
//           + gh') = y . l.  Two kind::f8f6f4 MMAs per 32-element K step.
// The products are exact; the FP32 sums are rounded only once they pass 2^24.
//
// Structure: persistent CTAs (one per SM) walk 128-row tiles.  Warp 0 issues
// TMA loads of 128-byte K slices of the tile and of the landmark chunk into an
// NST-stage ring and bulk copies of the chunk's W rows and norms; one thread
// of warp 1 issues the MMAs into two 256-column TMEM accumulators (alternating
// chunks); warps 2-5 read the accumulators back (tcgen05.ld, one row per
// thread) and do the epilogue.  Every mbarrier wait is bounded and reports a
// timeout through *err.
#include <cuda.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "df.cuh"
#include "tc_common.cuh"

namespace gbmds {
namespace {

using namespace tc;

constexpr int kRowsK = 128;           // points per tile (MMA M)
constexpr int kChunkK = 256;          // landmarks per chunk (MMA N)
constexpr int kThreadsK = 192;        // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint32_t kTmemColsK = 512;  // two accumulators of 256 FP32 columns
constexpr int kMaxRK = 16;
constexpr uint32_t kABytes = kRowsK * 128;    // 16 KB: one 128-byte K slice of the tile
constexpr uint32_t kBBytes = kChunkK * 128;   // 32 KB: one 128-byte K slice of the chunk

template <int MODE>
struct KCfg;
template <>
struct KCfg<kTckBf16> {
    static constexpr int kNB = 1;       // landmark operands per stage
    static constexpr int kStages = 3;
    static constexpr uint32_t kIdesc =  // D F32, A = B = BF16, K-major, M = 128, N = 256
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kChunkK >> 3) << 17) | ((uint32_t)(kRowsK >> 4) << 24);
};
template <>
struct KCfg<kTckFp8> {
    static constexpr int kNB = 2;
    static constexpr int kStages = 2;
    static constexpr uint32_t kIdesc =  // D F32, A = B = E4M3 (format 0), K-major, M = 128, N = 256
        (1u << 4) | ((uint32_t)(kChunkK >> 3) << 17) | ((uint32_t)(kRowsK >> 4) << 24);
};

template <int MODE>
struct KSmem {
    static constexpr int NST = KCfg<MODE>::kStages;
    static constexpr int NB = KCfg<MODE>::kNB;
    uint8_t a[NST][kABytes];          // 1024-byte aligned (offsets are multiples of 16 KB)
    uint8_t b[NST][NB][kBBytes];
    float w[2][kChunkK * kMaxRK];     // W rows of the chunk (width RP)
    float nl[2][kChunkK];             // landmark norms of the chunk
    uint64_t full[NST], empty[NST];
    uint64_t wfull[2], wempty[2];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t mma_done;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

struct TckArgs {
    int64_t m;            // rows of Y
    int nchunks;          // landmark chunks of 256 (W, norms zero-padded to nchunks * 256)
    int nkb;              // 128-byte K slices per row
    int r;
    const float* nrm_y;   // m
    const float* nrm_l;   // nchunks * 256
    const float* W;       // nchunks * 256 x RP
    const double* bias;   // r
    float* X;             // m x r
    int* err;
};

template <int MODE, int RP>
__global__ void __launch_bounds__(kThreadsK, 1)
    k_gower_tck(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b1,
                const __grid_constant__ CUtensorMap tm_b2, TckArgs a) {
    using Cfg = KCfg<MODE>;
    using Smem = KSmem<MODE>;
    constexpr int NST = Cfg::kStages;
    constexpr int NB = Cfg::kNB;
    extern __shared__ __align__(1024) uint8_t tck_smraw[];
    Smem& S = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(tck_smraw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (a.m + kRowsK - 1) / kRowsK;
    volatile int* abort = &S.abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&S.wfull[s], 1);
            mbar_init(&S.wempty[s], 128);
            mbar_init(&S.acc_full[s], 1);
            mbar_init(&S.acc_empty[s], 128);
        }
        mbar_init(&S.mma_done, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(kTmemColsK)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;
    constexpr uint32_t stage_tx = kABytes + NB * kBBytes;
    constexpr int xstep = MODE == kTckBf16 ? 64 : 128;   // elements per 128-byte K slice

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            long long g = 0, kb = 0;   // chunks and K slices issued
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
                for (int c = 0; c < a.nchunks && ok; ++c, ++g) {
                    const int ws = (int)(g & 1);
                    if (g >= 2 && !(ok = mbar_wait(&S.wempty[ws], (uint32_t)(((g >> 1) - 1) & 1), abort, a.err)))
                        break;
                    mbar_expect_tx(&S.wfull[ws], (uint32_t)(kChunkK * RP * 4 + kChunkK * 4));
                    bulk_load(S.w[ws], a.W + (int64_t)c * kChunkK * RP, (uint32_t)(kChunkK * RP * 4), &S.wfull[ws]);
                    bulk_load(S.nl[ws], a.nrm_l + (int64_t)c * kChunkK, (uint32_t)(kChunkK * 4), &S.wfull[ws]);
                    for (int k = 0; k < a.nkb; ++k, ++kb) {
                        const int s = (int)(kb % NST);
                        const long long use = kb / NST;
                        if (use > 0 && !(ok = mbar_wait(&S.empty[s], (uint32_t)((use - 1) & 1), abort, a.err)))
                            break;
                        mbar_expect_tx(&S.full[s], stage_tx);
                        tma_load_2d(S.a[s], &tm_a, k * xstep, (int)(t * kRowsK), &S.full[s]);
                        tma_load_2d(S.b[s][0], &tm_b1, k * xstep, c * kChunkK, &S.full[s]);
                        if (NB == 2) tma_load_2d(S.b[s][NB - 1], &tm_b2, k * xstep, c * kChunkK, &S.full[s]);
                    }
                }
            }
            // drain (bounded): copies this thread issued that may still be in flight
            for (long long q = kb - NST < 0 ? 0 : kb - NST; q < kb; ++q)
                mbar_drain(&S.full[q % NST], (uint32_t)((q / NST) & 1), a.err);
            for (long long q = g - 2 < 0 ? 0 : g - 2; q < g; ++q)
                mbar_drain(&S.wfull[q & 1], (uint32_t)((q >> 1) & 1), a.err);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            long long g = 0, kb = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
                for (int c = 0; c < a.nchunks && ok; ++c, ++g) {
                    const int as = (int)(g & 1);
                    if (g >= 2 && !(ok = mbar_wait(&S.acc_empty[as], (uint32_t)(((g >> 1) - 1) & 1), abort, a.err)))
                        break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t d = tmem + (uint32_t)(as * kChunkK);
                    for (int k = 0; k < a.nkb; ++k, ++kb) {
                        const int s = (int)(kb % NST);
                        if (!(ok = mbar_wait(&S.full[s], (uint32_t)((kb / NST) & 1), abort, a.err))) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {   // 32 bytes of K per MMA
                            const uint64_t ad = umma_desc(smem_u32(S.a[s]) + kk * 32);
                            const uint64_t b1 = umma_desc(smem_u32(S.b[s][0]) + kk * 32);
                            const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
                            if (MODE == kTckBf16) {
                                umma_bf16(d, ad, b1, Cfg::kIdesc, acc);
                            } else {
                                const uint64_t b2 = umma_desc(smem_u32(S.b[s][NB - 1]) + kk * 32);
                                umma_f8(d, ad, b1, Cfg::kIdesc, acc);
                                umma_f8(d, ad, b2, Cfg::kIdesc, 1u);
                            }
                        }
                        umma_commit(&S.empty[s]);    // stage free when these MMAs finish
                    }
                    if (ok) umma_commit(&S.acc_full[as]);
                }
            }
            // every MMA this thread issued has completed before TMEM is released
            umma_commit(&S.mma_done);
            mbar_drain(&S.mma_done, 0, a.err);
        }
    } else {
        // ---------------- epilogue: warps 2-5, one accumulator row per thread
        const int quad = warp & 3;   // TMEM lane quadrant this warp may read
        const int row = quad * 32 + lane;
        long long g = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
            const int64_t gi = t * kRowsK + row;
            const float ny = gi < a.m ? a.nrm_y[gi] : 0.f;
            float x[RP];
#pragma unroll
            for (int o = 0; o < RP; ++o) x[o] = 0.f;
            for (int c = 0; c < a.nchunks; ++c, ++g) {
                const int as = (int)(g & 1);
                const uint32_t par = (uint32_t)((g >> 1) & 1);
                ok = __all_sync(0xffffffffu, mbar_wait(&S.acc_full[as], par, abort, a.err) &&
                                                 mbar_wait(&S.wfull[as], par, abort, a.err));   // warp-uniform
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float* ws = S.w[as];
                const float* ns = S.nl[as];
#pragma unroll 1
                for (int cb = 0; cb < kChunkK; cb += 32) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(as * kChunkK + cb), v);
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const float a2 = fmaxf(fmaf(-2.f, v[e], ny + ns[cb + e]), 0.f);
                        const float4* w4 = reinterpret_cast<const float4*>(ws + (cb + e) * RP);
#pragma unroll
                        for (int q4 = 0; q4 < RP / 4; ++q4) {
                            const float4 w = w4[q4];
                            x[4 * q4 + 0] = fmaf(a2, w.x, x[4 * q4 + 0]);
                            x[4 * q4 + 1] = fmaf(a2, w.y, x[4 * q4 + 1]);
                            x[4 * q4 + 2] = fmaf(a2, w.z, x[4 * q4 + 2]);
                            x[4 * q4 + 3] = fmaf(a2, w.w, x[4 * q4 + 3]);
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&S.acc_empty[as]);
                mbar_arrive(&S.wempty[as]);
            }
            if (ok && gi < a.m) {
#pragma unroll
                for (int o = 0; o < RP; ++o)
                    if (o < a.r) a.X[gi * a.r + o] = x[o] + (float)a.bias[o];
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemColsK)
                     : "memory");
    }
}

// ------------------------------------------------------------ part Gram
//
// Divide-and-conquer (Section 3.2) for byte rows: Delta_j of every part j
// from the same operands.  Part j's members (its c connecting points, then
// its own points) are encoded as rows moff_j .. moff_j + n_j - 1 of one
// operand matrix (moff_j a multiple of 4).  A work unit is (part, 128-row
// tile, 256-column chunk); the accumulator S = Y_tile Y_chunk^T gives
// Delta = ||y_a||^2 + ||y_b||^2 - 2 S (clamped at 0, diagonal 0), stored as
// FP32 at the start of row a's storage in the Q arena (row stride 2 * ldq
// floats), with double-FP32 row sums per 64-column tile into
// rp[tile * n_j + a].  Rows or columns past n_j belong to the next part and
// are masked.

struct GramArgs {
    int units;
    const int4* unit;           // (part, row0, col0, moff)
    const ProbDesc* desc;
    const float* nrm;           // member norms (moff-indexed; zero padding)
    double* qarena;
    double* rparena;
    int nkb;
    int* err;
};

template <int MODE>
__global__ void __launch_bounds__(kThreadsK, 1)
    k_gram_tck(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b1,
               const __grid_constant__ CUtensorMap tm_b2, GramArgs a) {
    using Cfg = KCfg<MODE>;
    using Smem = KSmem<MODE>;
    constexpr int NST = Cfg::kStages;
    constexpr int NB = Cfg::kNB;
    extern __shared__ __align__(1024) uint8_t tck_smraw[];
    Smem& S = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(tck_smraw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abort = &S.abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&S.wfull[s], 1);
            mbar_init(&S.wempty[s], 128);
            mbar_init(&S.acc_full[s], 1);
            mbar_init(&S.acc_empty[s], 128);
        }
        mbar_init(&S.mma_done, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(kTmemColsK)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;
    constexpr uint32_t stage_tx = kABytes + NB * kBBytes;
    constexpr int xstep = MODE == kTckBf16 ? 64 : 128;

    if (warp == 0) {
        // ---------------- TMA producer: operand K slices and the chunk's norms
        if (lane == 0) {
            long long g = 0, kb = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < a.units && ok && !*abort; u += gridDim.x, ++g) {
                const int4 w = a.unit[u];
                const int ws = (int)(g & 1);
                if (g >= 2 && !(ok = mbar_wait(&S.wempty[ws], (uint32_t)(((g >> 1) - 1) & 1), abort, a.err))) break;
                mbar_expect_tx(&S.wfull[ws], (uint32_t)(kChunkK * 4));
                bulk_load(S.nl[ws], a.nrm + w.w + w.z, (uint32_t)(kChunkK * 4), &S.wfull[ws]);
                for (int k = 0; k < a.nkb; ++k, ++kb) {
                    const int s = (int)(kb % NST);
                    const long long use = kb / NST;
                    if (use > 0 && !(ok = mbar_wait(&S.empty[s], (uint32_t)((use - 1) & 1), abort, a.err))) break;
                    mbar_expect_tx(&S.full[s], stage_tx);
                    tma_load_2d(S.a[s], &tm_a, k * xstep, w.w + w.y, &S.full[s]);
                    tma_load_2d(S.b[s][0], &tm_b1, k * xstep, w.w + w.z, &S.full[s]);
                    if (NB == 2) tma_load_2d(S.b[s][NB - 1], &tm_b2, k * xstep, w.w + w.z, &S.full[s]);
                }
            }
            for (long long q = kb - NST < 0 ? 0 : kb - NST; q < kb; ++q)
                mbar_drain(&S.full[q % NST], (uint32_t)((q / NST) & 1), a.err);
            for (long long q = g - 2 < 0 ? 0 : g - 2; q < g; ++q)
                mbar_drain(&S.wfull[q & 1], (uint32_t)((q >> 1) & 1), a.err);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            long long g = 0, kb = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < a.units && ok && !*abort; u += gridDim.x, ++g) {
                const int as = (int)(g & 1);
                if (g >= 2 && !(ok = mbar_wait(&S.acc_empty[as], (uint32_t)(((g >> 1) - 1) & 1), abort, a.err))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(as * kChunkK);
                for (int k = 0; k < a.nkb; ++k, ++kb) {
                    const int s = (int)(kb % NST);
                    if (!(ok = mbar_wait(&S.full[s], (uint32_t)((kb / NST) & 1), abort, a.err))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = umma_desc(smem_u32(S.a[s]) + kk * 32);
                        const uint64_t b1 = umma_desc(smem_u32(S.b[s][0]) + kk * 32);
                        const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
                        if (MODE == kTckBf16) {
                            umma_bf16(d, ad, b1, Cfg::kIdesc, acc);
                        } else {
                            const uint64_t b2 = umma_desc(smem_u32(S.b[s][NB - 1]) + kk * 32);
                            umma_f8(d, ad, b1, Cfg::kIdesc, acc);
                            umma_f8(d, ad, b2, Cfg::kIdesc, 1u);
                        }
                    }
                    umma_commit(&S.empty[s]);
                }
                if (ok) umma_commit(&S.acc_full[as]);
            }
            umma_commit(&S.mma_done);
            mbar_drain(&S.mma_done, 0, a.err);
        }
    } else {
        // ---------------- epilogue: warps 2-5, one tile row per thread
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        long long g = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < a.units && ok && !*abort; u += gridDim.x, ++g) {
            const int4 w = a.unit[u];
            const ProbDesc P = a.desc[w.x];
            const int n = P.n;
            const int ra = w.y + row;                       // part-local row
            const float ny = ra < n ? a.nrm[w.w + ra] : 0.f;
            float* Qrow = reinterpret_cast<float*>(a.qarena + P.q_off) + (int64_t)ra * 2 * P.ldq;
            double* rp = a.rparena + P.rp_off;
            const int as = (int)(g & 1);
            const uint32_t par = (uint32_t)((g >> 1) & 1);
            ok = __all_sync(0xffffffffu, mbar_wait(&S.acc_full[as], par, abort, a.err) &&
                                             mbar_wait(&S.wfull[as], par, abort, a.err));   // warp-uniform
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const float* ns = S.nl[as];
            float rh = 0.f, rl = 0.f;
#pragma unroll 1
            for (int cb = 0; cb < kChunkK; cb += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(as * kChunkK + cb), v);
                const int b0 = w.z + cb;                     // part-local column of v[0]
                if (ra < n && b0 < n) {
                    float dv[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        float dist = fmaxf(fmaf(-2.f, v[e], ny + ns[cb + e]), 0.f);
                        if (b0 + e == ra || b0 + e >= n) dist = 0.f;
                        dv[e] = dist;
                        df_add(rh, rl, dist, 0.f);
                    }
                    if (b0 + 32 <= n) {
#pragma unroll
                        for (int q4 = 0; q4 < 8; ++q4)
                            reinterpret_cast<float4*>(Qrow + b0)[q4] =
                                make_float4(dv[4 * q4], dv[4 * q4 + 1], dv[4 * q4 + 2], dv[4 * q4 + 3]);
                    } else {
                        for (int e = 0; e < n - b0; ++e) Qrow[b0 + e] = dv[e];
                    }
                }
                if ((cb & 63) == 32) {                       // a 64-column tile is complete
                    const int tb = (w.z + cb) >> 6;
                    if (ra < n && tb * 64 < n) rp[(int64_t)tb * n + ra] = (double)rh + (double)rl;
                    rh = rl = 0.f;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&S.acc_empty[as]);
            mbar_arrive(&S.wempty[as]);
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemColsK)
                     : "memory");
    }
}

// ------------------------------------------------------------ operand encodings

__device__ __forceinline__ uint8_t e4m3(float v) {
    return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// E4M3 encodings of 16 h and of g for a nibble h or g (exact: at most four
// significant bits), filled once per block.
__device__ __forceinline__ void fill_nibble_tables(uint8_t* hi16, uint8_t* lo) {
    if (threadIdx.x < 16) {
        hi16[threadIdx.x] = e4m3((float)(threadIdx.x * 16));
        lo[threadIdx.x] = e4m3((float)threadIdx.x);
    }
}

// Rows of byte data -> the kernel's A operand and exact squared norms, one
// warp per row (16 bytes per lane and step when d is a multiple of 16).
// kBf16: n x ldb BF16 (ldb = d rounded up to 8, zero tail).
// kFp8:  n x 2 dh bytes [16 h | g] (dh = d rounded up to 16, zero tails).
template <int MODE>
__global__ void __launch_bounds__(256) k_encode_u8(const uint8_t* __restrict__ Y, int64_t n, int d,
                                                   void* __restrict__ out, float* __restrict__ nrm) {
    __shared__ uint8_t t_hi[16], t_lo[16];
    fill_nibble_tables(t_hi, t_lo);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n) return;
    const uint8_t* y = Y + i * d;
    const bool vec = (d & 15) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    uint32_t ss = 0;
    if (MODE == kTckBf16) {
        const int ld = round_up(d, 8);
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + i * ld;
        if (vec) {
            for (int k = 16 * lane; k < d; k += 512) {
                const uint4 v = *reinterpret_cast<const uint4*>(y + k);
                const uint8_t* b = reinterpret_cast<const uint8_t*>(&v);
                __align__(16) __nv_bfloat16 w[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    ss += (uint32_t)b[u] * b[u];
                    w[u] = __float2bfloat16_rn((float)b[u]);
                }
                reinterpret_cast<uint4*>(o + k)[0] = reinterpret_cast<const uint4*>(w)[0];
                reinterpret_cast<uint4*>(o + k)[1] = reinterpret_cast<const uint4*>(w)[1];
            }
        } else {
            for (int k = lane; k < ld; k += 32) {
                const uint32_t v = k < d ? y[k] : 0u;
                ss += v * v;
                o[k] = __float2bfloat16_rn((float)v);
            }
        }
    } else {
        const int dh = round_up(d, 16);
        uint8_t* o = static_cast<uint8_t*>(out) + i * 2 * dh;
        if (vec) {
            for (int k = 16 * lane; k < d; k += 512) {
                const uint4 v = *reinterpret_cast<const uint4*>(y + k);
                const uint8_t* b = reinterpret_cast<const uint8_t*>(&v);
                __align__(16) uint8_t h[16], g[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    ss += (uint32_t)b[u] * b[u];
                    h[u] = t_hi[b[u] >> 4];
                    g[u] = t_lo[b[u] & 15];
                }
                *reinterpret_cast<uint4*>(o + k) = *reinterpret_cast<const uint4*>(h);
                *reinterpret_cast<uint4*>(o + dh + k) = *reinterpret_cast<const uint4*>(g);
            }
        } else {
            for (int k = lane; k < dh; k += 32) {
                const uint32_t v = k < d ? y[k] : 0u;
                ss += v * v;
                o[k] = t_hi[v >> 4];
                o[dh + k] = t_lo[v & 15];
            }
        }
    }
    // exact: at most d * 65025
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
    if (lane == 0) nrm[i] = (float)ss;
}

// Landmark rows idx[j] of byte data -> B operands (kFp8: B1 = [16h | g] and
// B2 = [g | 16h]; kBf16: BF16 rows) and norms; rows l .. lpad-1 of the norms
// are zero.
template <int MODE>
__global__ void k_encode_landmarks_u8(const uint8_t* __restrict__ Y, int64_t ny, int d,
                                      const int64_t* __restrict__ idx, int l, int lpad, void* __restrict__ B,
                                      float* __restrict__ nrm_l) {
    const int j = blockIdx.x;
    if (j >= lpad) return;
    if (j >= l) {
        if (threadIdx.x == 0) nrm_l[j] = 0.f;
        return;
    }
    int64_t gidx = idx[j];
    gidx = gidx < 0 ? 0 : (gidx >= ny ? ny - 1 : gidx);
    const uint8_t* y = Y + gidx * d;
    uint32_t ss = 0;
    if (MODE == kTckBf16) {
        const int ld = round_up(d, 8);
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(B) + (int64_t)j * ld;
        for (int k = threadIdx.x; k < ld; k += blockDim.x) {
            const uint32_t v = k < d ? y[k] : 0u;
            ss += v * v;
            o[k] = __float2bfloat16_rn((float)v);
        }
    } else {
        const int dh = round_up(d, 16);
        uint8_t* o1 = static_cast<uint8_t*>(B) + (int64_t)j * 2 * dh;
        uint8_t* o2 = static_cast<uint8_t*>(B) + (int64_t)l * 2 * dh + (int64_t)j * 2 * dh;
        for (int k = threadIdx.x; k < dh; k += blockDim.x) {
            const uint32_t v = k < d ? y[k] : 0u;
            ss += v * v;
            const uint8_t h16 = e4m3((float)(v & 0xF0u)), g = e4m3((float)(v & 0x0Fu));
            o1[k] = h16;
            o1[dh + k] = g;
            o2[k] = g;
            o2[dh + k] = h16;
        }
    }
    __shared__ uint32_t red[32];
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        nrm_l[j] = (float)tot;
    }
}

// Members of every part -> operand rows moff_j + a (kFp8: A = [16h | g] and
// B2 = [g | 16h]; kBf16: BF16 rows) and exact norms; one warp per member.
template <int MODE>
__global__ void __launch_bounds__(256) k_encode_parts_u8(const uint8_t* __restrict__ Y, int d,
                                                         const int64_t* __restrict__ anchors,
                                                         const int64_t* __restrict__ own,
                                                         const ProbDesc* __restrict__ desc,
                                                         const int* __restrict__ moff, int p, int64_t total,
                                                         void* __restrict__ A, void* __restrict__ B2,
                                                         float* __restrict__ nrm) {
    __shared__ uint8_t t_hi[16], t_lo[16];
    fill_nibble_tables(t_hi, t_lo);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t m = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);   // member slot (moff space)
    if (m >= total) return;
    // the part whose slots contain m (moff ascending)
    int lo = 0, hi = p - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (moff[mid] <= m) lo = mid;
        else hi = mid - 1;
    }
    const ProbDesc P = desc[lo];
    const int a = (int)(m - moff[lo]);
    const bool real = a < P.n;
    const uint8_t* y = Y + (real ? member_row(P, anchors, own, a) : 0) * d;
    uint32_t ss = 0;
    if (MODE == kTckBf16) {
        const int ld = round_up(d, 8);
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(A) + m * ld;
        for (int k = lane; k < ld; k += 32) {
            const uint32_t v = real && k < d ? y[k] : 0u;
            ss += v * v;
            o[k] = __float2bfloat16_rn((float)v);
        }
    } else {
        const int dh = round_up(d, 16);
        uint8_t* o = static_cast<uint8_t*>(A) + m * 2 * dh;
        uint8_t* o2 = static_cast<uint8_t*>(B2) + m * 2 * dh;
        for (int k = lane; k < dh; k += 32) {
            const uint32_t v = real && k < d ? y[k] : 0u;
            ss += v * v;
            const uint8_t h = t_hi[v >> 4], g = t_lo[v & 15];
            o[k] = h;
            o[dh + k] = g;
            o2[k] = g;
            o2[dh + k] = h;
        }
    }
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
    if (lane == 0) nrm[m] = (float)ss;
}

__global__ void k_pad_w_rows(const float* __restrict__ W, int l, int r, int rp, int lpad, float* __restrict__ Wp) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)lpad * rp) return;
    const int j = (int)(e / rp), o = (int)(e % rp);
    Wp[e] = (j < l && o < r) ? W[(int64_t)j * r + o] : 0.f;
}

bool make_map_k(CUtensorMap* map, CUtensorMapDataType ty, int esize, const void* base, int64_t rows,
                int64_t cols, uint32_t box_rows) {
    const auto encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(cols * esize)};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / esize), box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, ty, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, int RP>
cudaError_t launch_tck_t(const CUtensorMap& ma, const CUtensorMap& mb1, const CUtensorMap& mb2, const TckArgs& a,
                         cudaStream_t st) {
    const size_t smem = sizeof(KSmem<MODE>) + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_gower_tck<MODE, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (a.m + kRowsK - 1) / kRowsK;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    k_gower_tck<MODE, RP><<<grid, kThreadsK, smem, st>>>(ma, mb1, mb2, a);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace

int tck_lpad(int l) { return round_up(l, kChunkK); }

size_t tck_operand_bytes(int mode, int64_t rows, int d) {
    return mode == kTckBf16 ? (size_t)rows * round_up(d, 8) * 2 : (size_t)rows * 2 * round_up(d, 16);
}

size_t tck_landmark_bytes(int mode, int l, int d) {
    return mode == kTckBf16 ? tck_operand_bytes(mode, l, d) : 2 * tck_operand_bytes(mode, l, d);
}

cudaError_t launch_encode_u8(int mode, const uint8_t* Y, int64_t n, int d, void* out, float* nrm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 7) / 8);
    if (mode == kTckBf16) k_encode_u8<kTckBf16><<<blocks, 256, 0, st>>>(Y, n, d, out, nrm);
    else k_encode_u8<kTckFp8><<<blocks, 256, 0, st>>>(Y, n, d, out, nrm);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_encode_landmarks_u8(int mode, const uint8_t* Y, int64_t ny, int d, const int64_t* idx, int l,
                                       void* B, float* nrm_l, cudaStream_t st) {
    const int lpad = tck_lpad(l);
    if (mode == kTckBf16)
        k_encode_landmarks_u8<kTckBf16><<<lpad, 128, 0, st>>>(Y, ny, d, idx, l, lpad, B, nrm_l);
    else
        k_encode_landmarks_u8<kTckFp8><<<lpad, 128, 0, st>>>(Y, ny, d, idx, l, lpad, B, nrm_l);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pad_w_rows(const float* W, int l, int r, float* Wp, cudaStream_t st) {
    const int rp = gower_tc_rp(r), lpad = tck_lpad(l);
    const int64_t total = (int64_t)lpad * rp;
    k_pad_w_rows<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(W, l, r, rp, lpad, Wp);
    note_launch(1);
    return cudaGetLastError();
}

size_t gram_operand_bytes(int mode, int64_t member_slots, int d) {
    return (mode == kTckFp8 ? 2 : 1) * tck_operand_bytes(mode, member_slots, d);
}

cudaError_t launch_encode_parts_u8(int mode, const uint8_t* Y, int d, const int64_t* anchors, const int64_t* own,
                                   const ProbDesc* desc, const int* moff, int p, int64_t slots, void* ops,
                                   float* nrm, cudaStream_t st) {
    if (slots <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((slots + 7) / 8);
    void* b2 = static_cast<uint8_t*>(ops) + tck_operand_bytes(mode, slots, d);
    if (mode == kTckBf16)
        k_encode_parts_u8<kTckBf16><<<blocks, 256, 0, st>>>(Y, d, anchors, own, desc, moff, p, slots, ops, b2, nrm);
    else
        k_encode_parts_u8<kTckFp8><<<blocks, 256, 0, st>>>(Y, d, anchors, own, desc, moff, p, slots, ops, b2, nrm);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_gram_tck(int mode, const void* ops, int64_t slots, int d, const float* nrm, const int4* units,
                            int nunits, const ProbDesc* desc, double* qarena, double* rparena, int* err,
                            cudaStream_t st) {
    if (nunits <= 0) return cudaSuccess;
    CUtensorMap ma, mb1, mb2;
    int64_t cols;
    bool ok;
    if (mode == kTckBf16) {
        cols = round_up(d, 8);
        ok = make_map_k(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ops, slots, cols, kRowsK) &&
             make_map_k(&mb1, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ops, slots, cols, kChunkK);
        mb2 = mb1;
    } else {
        cols = 2 * round_up(d, 16);
        const uint8_t* b2 = static_cast<const uint8_t*>(ops) + (size_t)slots * cols;
        ok = make_map_k(&ma, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, ops, slots, cols, kRowsK) &&
             make_map_k(&mb1, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, ops, slots, cols, kChunkK) &&
             make_map_k(&mb2, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, b2, slots, cols, kChunkK);
    }
    if (!ok) return cudaErrorInvalidValue;
    GramArgs a;
    a.units = nunits;
    a.unit = units;
    a.desc = desc;
    a.nrm = nrm;
    a.qarena = qarena;
    a.rparena = rparena;
    a.nkb = (int)((cols * (mode == kTckBf16 ? 2 : 1) + 127) / 128);
    a.err = err;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nunits < sms ? nunits : sms;
    cudaError_t e;
    if (mode == kTckBf16) {
        const size_t smem = sizeof(KSmem<kTckBf16>) + 1024;
        e = cudaFuncSetAttribute(k_gram_tck<kTckBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gram_tck<kTckBf16><<<grid, kThreadsK, smem, st>>>(ma, mb1, mb2, a);
    } else {
        const size_t smem = sizeof(KSmem<kTckFp8>) + 1024;
        e = cudaFuncSetAttribute(k_gram_tck<kTckFp8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gram_tck<kTckFp8><<<grid, kThreadsK, smem, st>>>(ma, mb1, mb2, a);
    }
    note_launch(1);
    return cudaGetLastError();
}

bool gower_tck_supported(int d, int r) { return d > 0 && d <= 65536 && r > 0 && r <= kMaxRK; }

cudaError_t launch_gower_tck(int mode, const void* A, int64_t m, int d, const float* nrm_y, const void* B, int l,
                             const float* nrm_l, const float* Wp, const double* bias, int r, float* X, int* err,
                             cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    CUtensorMap ma, mb1, mb2;
    int64_t cols;
    bool ok;
    if (mode == kTckBf16) {
        cols = round_up(d, 8);
        ok = make_map_k(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, m, cols, kRowsK) &&
             make_map_k(&mb1, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, l, cols, kChunkK);
        mb2 = mb1;
    } else {
        cols = 2 * round_up(d, 16);
        const uint8_t* b2 = static_cast<const uint8_t*>(B) + (size_t)l * cols;
        ok = make_map_k(&ma, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, A, m, cols, kRowsK) &&
             make_map_k(&mb1, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, B, l, cols, kChunkK) &&
             make_map_k(&mb2, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, b2, l, cols, kChunkK);
    }
    if (!ok) return cudaErrorInvalidValue;
    TckArgs a;
    a.m = m;
    a.nchunks = tck_lpad(l) / kChunkK;
    a.nkb = (int)((cols * (mode == kTckBf16 ? 2 : 1) + 127) / 128);
    a.r = r;
    a.nrm_y = nrm_y;
    a.nrm_l = nrm_l;
    a.W = Wp;
    a.bias = bias;
    a.X = X;
    a.err = err;
    const int rp = gower_tc_rp(r);
#define GB_TCK(MD, R)                                                                 \
    if (rp == R) return launch_tck_t<MD, R>(ma, mb1, mb2, a, st);
    if (mode == kTckBf16) {
        GB_TCK(kTckBf16, 4) GB_TCK(kTckBf16, 8) GB_TCK(kTckBf16, 12) GB_TCK(kTckBf16, 16)
    } else {
        GB_TCK(kTckFp8, 4) GB_TCK(kTckFp8, 8) GB_TCK(kTckFp8, 12) GB_TCK(kTckFp8, 16)
    }
#undef GB_TCK
    return cudaErrorInvalidValue;
}

}  // namespace gbmds
