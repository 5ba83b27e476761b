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
#include "tc_common.cuh"

namespace gbmds {
namespace {

using namespace tc;

constexpr int kRows = 128;          // points per tile (MMA M)
constexpr int kChunk = 128;         // landmarks per chunk (MMA N)
constexpr int kAtomK = 64;          // BF16 elements per 128-byte swizzle atom
constexpr int kMaxAtoms = 2;        // K up to 128 (d <= 128 padded to 8)
constexpr int kTcMaxR = 16;
constexpr int kThreadsTc = 320;     // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue (two per TMEM lane quadrant)
constexpr uint32_t kTmemCols = 256; // two accumulators of kChunk FP32 columns

constexpr uint32_t kPlaneBytes = kRows * 128;                 // one atom of one plane: 16 KB
constexpr uint32_t kTileBytes = 2 * kMaxAtoms * kPlaneBytes;  // hi + lo, all atoms: 64 KB

struct TcSmem {
    // operand tiles first (1024-byte aligned for the 128-byte swizzle)
    uint8_t y[kTileBytes];           // [plane hi/lo][atom][128 rows x 128 B]
    uint8_t l[2][kTileBytes];        // landmark chunk ring
    float w[2][kChunk * kTcMaxR];    // W rows of the chunk (padded width RP)
    float nl[2][kChunk];             // landmark norms of the chunk
    float xs[kRows][kTcMaxR];        // the second column half's partial projections
    uint64_t y_full, y_empty;
    uint64_t l_full[2], l_empty[2];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t mma_done;
    uint32_t tmem_base;
    int abort;
};

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
            mbar_init(&S.acc_empty[s], 256);
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
                    const uint32_t wbytes = (uint32_t)(kChunk * RP * 4);   // W, norms zero-padded
                    const uint32_t nbytes = (uint32_t)(kChunk * 4);
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
        // ---------------- epilogue: warps 2-9, one accumulator row per thread;
        // warps 2-5 take columns 0-63 of every chunk, warps 6-9 columns 64-127
        // (two warps per TMEM lane quadrant).  The chunk's W rows and norms come
        // from shared memory (zero-padded past l); the producer refills the
        // stage only after all eight warps have arrived on acc_empty.  The r-wide
        // projection runs as packed f32x2 FMAs.
        const int quad = warp & 3;                 // TMEM lane quadrant this warp may read
        const int half = (warp - 2) >> 2;          // column half of the chunk
        const int row = quad * 32 + lane;
        const int r = a.r;
        // Every epilogue warp runs the same tiles and chunks whatever happens
        // (an aborted wait only skips the work), so the eight warps always meet
        // at the named barrier.
        long long gc = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int64_t gi = t * kRows + row;
            const float ny = gi < a.m ? (float)a.nrm_y[gi] : 0.f;
            uint64_t xp[RP / 2];                   // pairs (x[2o], x[2o+1])
#pragma unroll
            for (int o = 0; o < RP / 2; ++o) xp[o] = 0ull;
            for (int c = 0; c < nchunks; ++c, ++gc) {
                const int s = (int)(gc & 1);
                // warp-uniform: tcgen05.ld below is a .sync.aligned warp instruction
                const bool got = __all_sync(0xffffffffu, mbar_wait(&S.acc_full[s], (uint32_t)((gc >> 1) & 1), abort, a.err));
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const float* ws = S.w[s] + half * (kChunk / 2) * RP;
                const float* ns = S.nl[s] + half * (kChunk / 2);
#pragma unroll 1
                for (int cb = 0; cb < (got ? kChunk / 2 : 0); cb += 32) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(s * kChunk + half * (kChunk / 2) + cb), v);
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const float a2 = fmaxf(fmaf(-2.f, v[e], ny + ns[cb + e]), 0.f);
                        uint64_t a2p;
                        asm("mov.b64 %0, {%1, %1};" : "=l"(a2p) : "f"(a2));
                        const uint4* w4 = reinterpret_cast<const uint4*>(ws + (cb + e) * RP);
#pragma unroll
                        for (int q4 = 0; q4 < RP / 4; ++q4) {
                            const uint4 w = w4[q4];
                            uint64_t w01, w23;
                            asm("mov.b64 %0, {%1, %2};" : "=l"(w01) : "r"(w.x), "r"(w.y));
                            asm("mov.b64 %0, {%1, %2};" : "=l"(w23) : "r"(w.z), "r"(w.w));
                            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(xp[2 * q4]) : "l"(a2p), "l"(w01));
                            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(xp[2 * q4 + 1]) : "l"(a2p), "l"(w23));
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&S.acc_empty[s]);
            }
            float x[RP];
#pragma unroll
            for (int o = 0; o < RP / 2; ++o)
                asm("mov.b64 {%0, %1}, %2;" : "=f"(x[2 * o]), "=f"(x[2 * o + 1]) : "l"(xp[o]));
            // the second half hands its partial sums to the first (named barrier of the 8 warps)
            if (half == 1)
#pragma unroll
                for (int o = 0; o < RP; ++o) S.xs[row][o] = x[o];
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (half == 0 && gi < a.m) {
#pragma unroll
                for (int o = 0; o < RP; ++o)
                    if (o < r) a.X[gi * r + o] = x[o] + S.xs[row][o] + (float)a.bias[o];
            }
            asm volatile("bar.sync 1, 256;" ::: "memory");
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

bool make_map(CUtensorMap* map, const void* base, int64_t rows, int cols_pad) {
    const auto encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols_pad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols_pad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kAtomK, (cuuint32_t)kRows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// W (l x r) -> rows padded to a multiple of kChunk, columns to RP, zeros.
__global__ void k_pad_w(const float* __restrict__ W, int l, int r, int rp, int lpad, float* __restrict__ Wp) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= lpad * rp) return;
    const int j = e / rp, o = e % rp;
    Wp[e] = (j < l && o < r) ? W[j * r + o] : 0.f;
}

}  // namespace

// cuTensorMapEncodeTiled is a driver-API call.  It is looked up through the
// runtime at first use rather than linked, so libgbmds.so loads on hosts
// without a GPU driver (where only the argument checks can run).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

int gower_tc_lpad(int l) { return (int)round_up(l, kChunk); }

cudaError_t launch_pad_w(const float* W, int l, int r, float* Wp, cudaStream_t st) {
    const int rp = gower_tc_rp(r);
    const int lpad = gower_tc_lpad(l);
    k_pad_w<<<(lpad * rp + 255) / 256, 256, 0, st>>>(W, l, r, rp, lpad, Wp);
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
