// Gower interpolation (Eq. (2)) on the 5th-generation tensor cores.
//
// For a tile of 128 new points and every chunk of 128 landmarks:
//   S = Y L^T          (tcgen05.mma, BF16 operands, FP32 accumulation in TMEM)
//   A^2 = ||y||^2 + ||l||^2 - 2 S, clamped at 0       (epilogue, FP32)
//   X  += A^2 W         (W = -1/2 V Lambda^{-1/2}, r <= 16 columns, FP32 FMAs)
// and finally X += b.  A^2 never leaves the chip.
//
// Precision: each value is split into BF16 planes hi = bf16(y), lo = bf16(y - hi)
// and y . l is accumulated from the three products hi.hi + hi.lo + lo.hi
// (about 16 significant bits per operand; the dropped lo.lo term is ~2^-18
// relative).  The norms come from the same split.
//
// Structure: persistent CTAs (one per SM) walk 128-row tiles.  Warp 0 issues
// TMA loads (Y tile once per tile, landmark chunks through a 2-stage ring),
// warp 1 allocates TMEM (2 x 128 FP32 columns) and one thread issues the MMAs
// into alternating accumulators, warps 2-5 read the accumulators back
// (tcgen05.ld, one row per thread) and do the epilogue.  mbarriers order the
// roles; every wait is bounded and reports a timeout through *err instead of
// hanging.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace gbmds {
namespace {

constexpr int kRows = 128;          // points per tile (MMA M)
constexpr int kChunk = 128;         // landmarks per chunk (MMA N)
constexpr int kAtomK = 64;          // BF16 elements per 128-byte swizzle atom
constexpr int kMaxAtoms = 2;        // K up to 128 (d <= 128 padded to 8)
constexpr int kTcMaxR = 16;
constexpr int kThreadsTc = 192;     // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint32_t kTmemCols = 256; // two accumulators of kChunk FP32 columns
constexpr unsigned long long kWaitNs = 2000000000ull;   // give up a wait after 2 s

constexpr uint32_t kPlaneBytes = kRows * 128;                 // one atom of one plane: 16 KB
constexpr uint32_t kTileBytes = 2 * kMaxAtoms * kPlaneBytes;  // hi + lo, all atoms: 64 KB

struct TcSmem {
    // operand tiles first (1024-byte aligned for the 128-byte swizzle)
    uint8_t y[kTileBytes];           // [plane hi/lo][atom][128 rows x 128 B]
    uint8_t l[2][kTileBytes];        // landmark chunk ring
    float w[2][kChunk * kTcMaxR];    // W rows of the chunk (padded width RP)
    float nl[2][kChunk];             // landmark norms of the chunk
    uint64_t y_full, y_empty;
    uint64_t l_full[2], l_empty[2];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t mma_done;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait used while draining: ignores the abort flag, gives up after kWaitNs.
__device__ __forceinline__ void mbar_drain(uint64_t* b, uint32_t parity, int* err) {
    if (mbar_try_wait(b, parity)) return;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(b, parity)) return;
        if (global_ns() - t0 > kWaitNs) break;
    }
    atomicExch(err, MDS_ERR_TIMEOUT);
}

// Bounded wait: false (and *err and the shared abort flag set) after kWaitNs,
// or as soon as another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort, int* err) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(b, parity)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > kWaitNs) break;
    }
    *abort = 1;
    atomicExch(err, MDS_ERR_TIMEOUT);
    return false;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// atoms of 1024 bytes (stride byte offset 1024), version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t u[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
          "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]),
          "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]),
          "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(u[i]);
}

struct TcArgs {
    int64_t m;            // rows of Y
    int l;                // landmarks
    int natoms;           // K atoms (1 or 2)
    int ksteps;           // MMA K-steps of 16 (ceil(d_pad / 16))
    int r;
    const double* nrm_y;  // m
    const float* nrm_l;   // l, zero-padded to a multiple of 4
    const float* W;       // l x RP (columns r..RP-1 zero)
    const double* bias;   // r
    float* X;             // m x r
    int* err;
};

template <int RP>
__global__ void __launch_bounds__(kThreadsTc, 1)
    k_gower_tc(const __grid_constant__ CUtensorMap tm_yhi, const __grid_constant__ CUtensorMap tm_ylo,
               const __grid_constant__ CUtensorMap tm_lhi, const __grid_constant__ CUtensorMap tm_llo,
               TcArgs a) {
    extern __shared__ __align__(1024) uint8_t tc_smraw[];
    // 1024-byte alignment of the operand tiles
    TcSmem& S = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(tc_smraw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (a.m + kRows - 1) / kRows;
    const int nchunks = (a.l + kChunk - 1) / kChunk;
    volatile int* abort = &S.abort;

    if (threadIdx.x == 0) {
        mbar_init(&S.y_full, 1);
        mbar_init(&S.y_empty, 1);
        mbar_init(&S.mma_done, 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&S.l_full[s], 1);
            mbar_init(&S.l_empty[s], 1);
            mbar_init(&S.acc_full[s], 1);
            mbar_init(&S.acc_empty[s], 128);
        }
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;
    const uint32_t tile_tx = 2u * a.natoms * kPlaneBytes;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            long long gc = 0;  // chunks issued
            int ti = 0;        // tiles issued by this CTA
            for (int64_t t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                if (ti > 0 && !mbar_wait(&S.y_empty, (ti - 1) & 1, abort, a.err)) break;
                ++ti;
                mbar_expect_tx(&S.y_full, tile_tx);
                for (int at = 0; at < a.natoms; ++at) {
                    tma_load_2d(S.y + (0 * kMaxAtoms + at) * kPlaneBytes, &tm_yhi, at * kAtomK, (int)(t * kRows), &S.y_full);
                    tma_load_2d(S.y + (1 * kMaxAtoms + at) * kPlaneBytes, &tm_ylo, at * kAtomK, (int)(t * kRows), &S.y_full);
                }
                for (int c = 0; c < nchunks; ++c, ++gc) {
                    const int s = (int)(gc & 1);
                    const long long use = gc >> 1;
                    // stage s is free when the MMAs of its previous chunk are done
                    // (l_empty) and the epilogue has read that chunk's W and norms
                    // (acc_empty of the same use)
                    if (use > 0 && (!mbar_wait(&S.l_empty[s], (uint32_t)((use - 1) & 1), abort, a.err) ||
                                    !mbar_wait(&S.acc_empty[s], (uint32_t)((use - 1) & 1), abort, a.err)))
                        break;
                    const int j0 = c * kChunk;
                    const int nc = min(kChunk, a.l - j0);
                    const uint32_t wbytes = (uint32_t)(nc * RP * 4);
                    const uint32_t nbytes = (uint32_t)(((nc + 3) & ~3) * 4);
                    mbar_expect_tx(&S.l_full[s], tile_tx + wbytes + nbytes);
                    for (int at = 0; at < a.natoms; ++at) {
                        tma_load_2d(S.l[s] + (0 * kMaxAtoms + at) * kPlaneBytes, &tm_lhi, at * kAtomK, j0, &S.l_full[s]);
                        tma_load_2d(S.l[s] + (1 * kMaxAtoms + at) * kPlaneBytes, &tm_llo, at * kAtomK, j0, &S.l_full[s]);
                    }
                    bulk_load(S.w[s], a.W + (int64_t)j0 * RP, wbytes, &S.l_full[s]);
                    bulk_load(S.nl[s], a.nrm_l + j0, nbytes, &S.l_full[s]);
                }
            }
            // drain: wait (bounded) for the copies this thread issued that may
            // still be in flight (the last Y tile and the last two chunk stages)
            if (ti > 0) mbar_drain(&S.y_full, (uint32_t)((ti - 1) & 1), a.err);
            for (long long g = gc - 2 < 0 ? 0 : gc - 2; g < gc; ++g)
                mbar_drain(&S.l_full[g & 1], (uint32_t)((g >> 1) & 1), a.err);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(kRows, kChunk);
            long long gc = 0;
            int ti = 0;
            for (int64_t t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++ti) {
                if (!mbar_wait(&S.y_full, ti & 1, abort, a.err)) break;
                bool ok = true;
                for (int c = 0; c < nchunks && ok; ++c, ++gc) {
                    const int s = (int)(gc & 1);
                    const long long use = gc >> 1;
                    ok = mbar_wait(&S.l_full[s], (uint32_t)(use & 1), abort, a.err);
                    if (ok && use > 0) ok = mbar_wait(&S.acc_empty[s], (uint32_t)((use - 1) & 1), abort, a.err);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t d = tmem + (uint32_t)(s * kChunk);
                    uint32_t acc = 0;
                    for (int k = 0; k < a.ksteps; ++k) {
                        const int at = k / (kAtomK / 16), kk = k % (kAtomK / 16);
                        const uint32_t off = (uint32_t)(at * kPlaneBytes + kk * 32);
                        const uint64_t ahi = umma_desc(smem_u32(S.y) + off);
                        const uint64_t alo = umma_desc(smem_u32(S.y) + kMaxAtoms * kPlaneBytes + off);
                        const uint64_t bhi = umma_desc(smem_u32(S.l[s]) + off);
                        const uint64_t blo = umma_desc(smem_u32(S.l[s]) + kMaxAtoms * kPlaneBytes + off);
                        umma_bf16(d, ahi, bhi, idesc, acc);
                        acc = 1;
                        umma_bf16(d, ahi, blo, idesc, 1);
                        umma_bf16(d, alo, bhi, idesc, 1);
                    }
                    umma_commit(&S.l_empty[s]);    // landmark stage free when these MMAs finish
                    umma_commit(&S.acc_full[s]);   // accumulator ready for the epilogue
                }
                if (!ok) break;
                umma_commit(&S.y_empty);           // Y tile free after the tile's last MMA
            }
            // every MMA this thread issued has completed before TMEM is released
            umma_commit(&S.mma_done);
            mbar_drain(&S.mma_done, 0, a.err);
        }
    } else {
        // ---------------- epilogue: warps 2-5, one accumulator row per thread.
        // The chunk's W rows and norms come from shared memory, loaded with the
        // landmark tiles; the producer refills the stage only after this epilogue
        // has arrived on acc_empty.
        const int quad = warp & 3;                 // TMEM lane quadrant this warp may read
        const int row = quad * 32 + lane;
        const int r = a.r;
        long long gc = 0;
        for (int64_t t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
            const int64_t gi = t * kRows + row;
            const float ny = gi < a.m ? (float)a.nrm_y[gi] : 0.f;
            float x[RP];
#pragma unroll
            for (int o = 0; o < RP; ++o) x[o] = 0.f;
            bool ok = true;
            for (int c = 0; c < nchunks; ++c, ++gc) {
                const int s = (int)(gc & 1);
                ok = mbar_wait(&S.acc_full[s], (uint32_t)((gc >> 1) & 1), abort, a.err);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int nc = min(kChunk, a.l - c * kChunk);
                const float* ws = S.w[s];
                const float* ns = S.nl[s];
#pragma unroll 1
                for (int cb = 0; cb < kChunk; cb += 32) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * kChunk + cb), v);
                    if (cb + 32 <= nc) {
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
                    } else if (cb < nc) {
                        for (int e = 0; e < nc - cb; ++e) {
                            float ve = v[0];
#pragma unroll
                            for (int u = 1; u < 32; ++u) ve = u == e ? v[u] : ve;
                            const float a2 = fmaxf(fmaf(-2.f, ve, ny + ns[cb + e]), 0.f);
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
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&S.acc_empty[s]);
            }
            if (!ok) break;
            if (gi < a.m) {
#pragma unroll
                for (int o = 0; o < RP; ++o)
                    if (o < r) a.X[gi * r + o] = x[o] + (float)a.bias[o];
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

// Landmark rows idx[i] of BF16 split planes (ny x ld each) into split planes
// (l x ld each), and their norms as float.
__global__ void k_gather_split(const __nv_bfloat16* __restrict__ Y, int64_t ny, int ld,
                               const int64_t* __restrict__ idx, int l, __nv_bfloat16* __restrict__ L,
                               const double* __restrict__ nrm, float* __restrict__ nrm_l) {
    const int i = blockIdx.x;
    if (i >= l) return;
    int64_t g = idx[i];
    g = g < 0 ? 0 : (g >= ny ? ny - 1 : g);
    for (int k = threadIdx.x; k < ld; k += blockDim.x) {
        L[(int64_t)i * ld + k] = Y[g * ld + k];
        L[(int64_t)l * ld + (int64_t)i * ld + k] = Y[ny * ld + g * ld + k];
    }
    if (threadIdx.x == 0) nrm_l[i] = (float)nrm[g];
}

// cuTensorMapEncodeTiled is a driver-API call.  It is looked up through the
// runtime at first use rather than linked, so libgbmds.so loads on hosts
// without a GPU driver (where only the argument checks can run).
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        cudaGetLastError();
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

bool make_map(CUtensorMap* map, const void* base, int64_t rows, int cols_pad) {
    const auto encode = encode_tiled();
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols_pad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols_pad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kAtomK, (cuuint32_t)kRows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

__global__ void k_pad_w(const float* __restrict__ W, int l, int r, int rp, float* __restrict__ Wp) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= l * rp) return;
    const int j = e / rp, o = e % rp;
    Wp[e] = o < r ? W[j * r + o] : 0.f;
}

}  // namespace

cudaError_t launch_pad_w(const float* W, int l, int r, float* Wp, cudaStream_t st) {
    const int rp = gower_tc_rp(r);
    k_pad_w<<<(l * rp + 255) / 256, 256, 0, st>>>(W, l, r, rp, Wp);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_split(const void* Ysplit, int64_t ny, int d, const int64_t* idx, int l,
                                void* Lsplit, const double* nrm, float* nrm_l, cudaStream_t st) {
    if (l <= 0) return cudaSuccess;
    k_gather_split<<<l, 128, 0, st>>>((const __nv_bfloat16*)Ysplit, ny, split_ld(d), idx, l,
                                      (__nv_bfloat16*)Lsplit, nrm, nrm_l);
    note_launch(1);
    return cudaGetLastError();
}

bool gower_tc_supported(int d, int r) { return d >= 1 && split_ld(d) <= kMaxAtoms * kAtomK && r >= 1 && r <= kTcMaxR; }

int gower_tc_rp(int r) { return r <= 4 ? 4 : (r <= 8 ? 8 : (r <= 12 ? 12 : 16)); }

template <int RP>
static cudaError_t launch_rp(const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0,
                             const CUtensorMap& b1, const TcArgs& a, int grid, size_t smem,
                             cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_gower_tc<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gower_tc<RP><<<grid, kThreadsTc, smem, st>>>(a0, a1, b0, b1, a);
    return cudaGetLastError();
}

cudaError_t launch_gower_tc(const void* Ysplit, int64_t m, int d, const double* nrm_y,
                            const void* Lsplit, const float* nrm_l, int l, const float* W,
                            const double* bias, int r, float* X, int* err, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (!gower_tc_supported(d, r) || l < 1) return cudaErrorInvalidValue;
    const int ld = split_ld(d);
    const __nv_bfloat16* yh = (const __nv_bfloat16*)Ysplit;
    const __nv_bfloat16* lh = (const __nv_bfloat16*)Lsplit;
    CUtensorMap m_yhi, m_ylo, m_lhi, m_llo;
    if (!make_map(&m_yhi, yh, m, ld) || !make_map(&m_ylo, yh + m * ld, m, ld) ||
        !make_map(&m_lhi, lh, l, ld) || !make_map(&m_llo, lh + (int64_t)l * ld, l, ld))
        return cudaErrorInvalidValue;
    TcArgs a;
    a.m = m;
    a.l = l;
    a.natoms = (ld + kAtomK - 1) / kAtomK;
    a.ksteps = (ld + 15) / 16;
    a.r = r;
    a.nrm_y = nrm_y;
    a.nrm_l = nrm_l;
    a.W = W;
    a.bias = bias;
    a.X = X;
    a.err = err;
    const size_t smem = sizeof(TcSmem) + 1024;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (m + kRows - 1) / kRows;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    note_launch(1);
    switch (gower_tc_rp(r)) {
        case 4: return launch_rp<4>(m_yhi, m_ylo, m_lhi, m_llo, a, grid, smem, st);
        case 8: return launch_rp<8>(m_yhi, m_ylo, m_lhi, m_llo, a, grid, smem, st);
        case 12: return launch_rp<12>(m_yhi, m_ylo, m_lhi, m_llo, a, grid, smem, st);
        default: return launch_rp<16>(m_yhi, m_ylo, m_lhi, m_llo, a, grid, smem, st);
    }
}

}  // namespace gbmds
