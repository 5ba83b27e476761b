// Gower interpolation (Eq. (2)) on the 5th-generation tensor cores.
//
// For a tile of 128 new points and every chunk of 128 landmarks:
//   S = Y L^T          (tcgen05.mma, BF16 operands, FP32 accumulation in TMEM)
//   A^2 = ||y||^2 + ||l||^2 - 2 S, clamped at 0       (epilogue, FP32)
//   X  += A^2 W         (tcgen05.mma again: A^2 from TMEM, W^T from shared memory)
// and finally X += b.  A^2 never leaves the chip.
//
// Precision: each value is split into BF16 planes hi = bf16(y), lo = bf16(y - hi)
// and y . l is accumulated from the three products hi.hi + hi.lo + lo.hi
// (about 16 significant bits per operand; the dropped lo.lo term is ~2^-18
// relative).  The norms come from the same split.  The projection splits A^2
// and W the same way: A^2_hi [W_hi | W_lo] (one MMA of N = 32, two 16-column
// halves) plus A^2_lo W_hi (N = 16, into the first half), FP32 accumulation in
// TMEM; X is the sum of the two halves.
//
// Structure: persistent CTAs (one per SM) walk 128-row tiles.  Warp 0 issues
// TMA loads (Y tile once per tile, landmark chunks through a 2-stage ring that
// is refilled as soon as the MMAs have read a stage), warp 10 copies each
// chunk's W^T image and landmark norms into a 2-stage ring of its own, warp 1
// allocates TMEM (3 x 128 FP32 accumulator columns plus a 32-column X
// accumulator) and one thread issues the MMAs, warps 2-9 read an accumulator
// back (tcgen05.ld, one row per thread, two warps per lane quadrant, one per
// 64-column half), form A^2 and write it back in place as packed BF16 hi/lo
// pairs (tcgen05.st), which the projection MMA then reads as its A operand.
// mbarriers order the roles; every wait is bounded and reports a timeout
// through *err instead of hanging.
//
// Three accumulators, because tcgen05.commit tracks every MMA the thread has
// issued before it: the commit that frees accumulator g (after chunk g's
// projection, issued behind chunk g + 1's distance MMAs) fires only once chunk
// g + 1's distances are done, so the distance MMAs of chunk g + 2 must not
// need it if the tensor pipe is to stay fed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace gbmds {
namespace {

using namespace tc;

constexpr int kRows = 128;          // points per tile (MMA M)
constexpr int kChunk = 128;         // landmarks per chunk (MMA N, projection K)
constexpr int kAtomK = 64;          // BF16 elements per 128-byte swizzle atom
constexpr int kMaxAtoms = 2;        // K up to 128 (d <= 128 padded to 8)
constexpr int kTcMaxR = 16;         // X columns of the projection (r <= 16, columns r..15 zero)
constexpr int kThreadsTc = 352;     // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue, warp 10 W copies
constexpr int kAcc = 3;             // distance accumulators of kChunk FP32 columns
constexpr uint32_t kTmemCols = 512; // the accumulators + the X accumulator (two 16-column halves)
constexpr uint32_t kXCol = kAcc * kChunk;

constexpr uint32_t kPlaneBytes = kRows * 128;                 // one atom of one plane: 16 KB
constexpr uint32_t kTileBytes = 2 * kMaxAtoms * kPlaneBytes;  // hi + lo, all atoms: 64 KB
constexpr uint32_t kWAtomBytes = 2 * kTcMaxR * 128;           // rows W_hi^T, W_lo^T x 64 landmarks: 4 KB
constexpr uint32_t kWImgBytes = 2 * kWAtomBytes;              // two 64-landmark atoms: 8 KB per chunk

struct TcSmem {
    // operand tiles first (1024-byte aligned for the 128-byte swizzle)
    uint8_t y[kTileBytes];           // [plane hi/lo][atom][128 rows x 128 B]
    uint8_t l[2][kTileBytes];        // landmark chunk ring
    uint8_t w[2][kWImgBytes];        // W^T of the chunk, BF16 hi/lo rows, swizzled
    float nl[2][kChunk];             // landmark norms of the chunk
    uint64_t y_full, y_empty;
    uint64_t l_full[2], l_empty[2];
    uint64_t acc_full[kAcc], acc_empty[kAcc], a2_full[kAcc];
    uint64_t w_full[2], w_empty[2];
    uint64_t x_full, x_empty;
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
    const float* nrm_l;   // l, zero-padded to a multiple of kChunk
    const uint8_t* Wimg;  // W^T images, kWImgBytes per chunk (launch_w_image)
    const double* bias;   // r
    float* X;             // m x r
    int* err;
};

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
        mbar_init(&S.x_full, 1);
        mbar_init(&S.x_empty, 128);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&S.l_full[s], 1);
            mbar_init(&S.l_empty[s], 1);
            mbar_init(&S.w_full[s], 1);
            mbar_init(&S.w_empty[s], 1);
        }
        for (int s = 0; s < kAcc; ++s) {
            mbar_init(&S.acc_full[s], 1);
            mbar_init(&S.acc_empty[s], 1);
            mbar_init(&S.a2_full[s], 256);
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
        // ---------------- TMA producer: Y tiles and landmark operand chunks
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
                    if (use > 0 && !mbar_wait(&S.l_empty[s], (uint32_t)((use - 1) & 1), abort, a.err)) break;
                    const int j0 = c * kChunk;
                    mbar_expect_tx(&S.l_full[s], tile_tx);
                    for (int at = 0; at < a.natoms; ++at) {
                        tma_load_2d(S.l[s] + (0 * kMaxAtoms + at) * kPlaneBytes, &tm_lhi, at * kAtomK, j0, &S.l_full[s]);
                        tma_load_2d(S.l[s] + (1 * kMaxAtoms + at) * kPlaneBytes, &tm_llo, at * kAtomK, j0, &S.l_full[s]);
                    }
                }
            }
            // drain: wait (bounded) for the copies this thread issued that may
            // still be in flight (the last Y tile and the last two chunk stages)
            if (ti > 0) mbar_drain(&S.y_full, (uint32_t)((ti - 1) & 1), a.err);
            for (long long g = gc - 2 < 0 ? 0 : gc - 2; g < gc; ++g)
                mbar_drain(&S.l_full[g & 1], (uint32_t)((g >> 1) & 1), a.err);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer.  Chunk g: the distance MMAs into
        // accumulator g % 3; then, once the epilogue has turned chunk g - 1
        // into A^2, that chunk's projection MMAs into the X accumulator (so the
        // tensor pipe has the next distance tile queued while A^2 is formed).
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(kRows, kChunk);
            const uint32_t idesc_x2 = umma_idesc(kRows, 2 * kTcMaxR);
            const uint32_t idesc_x1 = umma_idesc(kRows, kTcMaxR);
            // Shared-memory descriptors of every operand buffer, built once; a
            // K-step adds its byte offset / 16 to the start-address field (the
            // single issuing thread is on the critical path, so the loops below
            // do no more than that per MMA).
            const uint32_t ybase = smem_u32(S.y);
            const uint64_t dYh = umma_desc(ybase), dYl = umma_desc(ybase + kMaxAtoms * kPlaneBytes);
            const uint64_t dLh0 = umma_desc(smem_u32(S.l[0])), dLl0 = umma_desc(smem_u32(S.l[0]) + kMaxAtoms * kPlaneBytes);
            const uint64_t dLh1 = umma_desc(smem_u32(S.l[1])), dLl1 = umma_desc(smem_u32(S.l[1]) + kMaxAtoms * kPlaneBytes);
            const uint64_t dW0 = umma_desc(smem_u32(S.w[0])), dW1 = umma_desc(smem_u32(S.w[1]));
            const int ksteps = a.ksteps;
            // projection MMAs of chunk g (chunk c of the CTA's tile number tix)
            auto project = [&](long long g, int c, int tix) -> bool {
                const int q = (int)(g % kAcc), s = (int)(g & 1);
                if (!mbar_wait(&S.a2_full[q], (uint32_t)((g / kAcc) & 1), abort, a.err) ||
                    !mbar_wait(&S.w_full[s], (uint32_t)((g >> 1) & 1), abort, a.err))
                    return false;
                // the X accumulator of the previous tile has been read
                if (c == 0 && tix > 0 && !mbar_wait(&S.x_empty, (uint32_t)((tix - 1) & 1), abort, a.err))
                    return false;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a2 = tmem + (uint32_t)(q * kChunk);
                const uint64_t dw = s ? dW1 : dW0;
                const uint32_t first = c > 0 ? 1u : 0u;
#pragma unroll
                for (int k = 0; k < kChunk / 16; ++k) {
                    const int h = k >> 2, kk = k & 3;  // 64-landmark half, K-step within it
                    const uint32_t ahi = a2 + (uint32_t)(h * 64 + kk * 8), alo = ahi + 32;
                    // rows 0-15 of the atom are W_hi^T, rows 16-31 W_lo^T
                    const uint64_t b = dw + (uint64_t)((h * kWAtomBytes + kk * 32) >> 4);
                    umma_bf16_ta(tmem + kXCol, ahi, b, idesc_x2, k > 0 ? 1u : first);
                    umma_bf16_ta(tmem + kXCol, alo, b, idesc_x1, 1);
                }
                umma_commit(&S.acc_empty[q]);              // accumulator and A^2 free
                umma_commit(&S.w_empty[s]);                // W stage free
                if (c == nchunks - 1) umma_commit(&S.x_full);
                return true;
            };
            long long gc = 0, pend = -1;
            int pend_c = 0, pend_t = 0;
            int ti = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x, ++ti) {
                if (!mbar_wait(&S.y_full, ti & 1, abort, a.err)) {
                    ok = false;
                    break;
                }
                for (int c = 0; c < nchunks; ++c, ++gc) {
                    const int s = (int)(gc & 1), q = (int)(gc % kAcc);
                    const long long use = gc >> 1, qu = gc / kAcc;
                    ok = mbar_wait(&S.l_full[s], (uint32_t)(use & 1), abort, a.err);
                    if (ok && qu > 0) ok = mbar_wait(&S.acc_empty[q], (uint32_t)((qu - 1) & 1), abort, a.err);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t d = tmem + (uint32_t)(q * kChunk);
                    const uint64_t dLh = s ? dLh1 : dLh0, dLl = s ? dLl1 : dLl0;
#pragma unroll
                    for (int k = 0; k < kMaxAtoms * kAtomK / 16; ++k) {
                        if (k < ksteps) {
                            const int at = k / (kAtomK / 16), kk = k % (kAtomK / 16);
                            const uint64_t o = (uint64_t)((at * kPlaneBytes + kk * 32) >> 4);
                            umma_bf16(d, dYh + o, dLh + o, idesc, k > 0 ? 1u : 0u);
                            umma_bf16(d, dYh + o, dLl + o, idesc, 1);
                            umma_bf16(d, dYl + o, dLh + o, idesc, 1);
                        }
                    }
                    umma_commit(&S.l_empty[s]);    // landmark stage free when these MMAs finish
                    umma_commit(&S.acc_full[q]);   // accumulator ready for the epilogue
                    if (c == nchunks - 1) umma_commit(&S.y_empty);  // Y tile free after its last MMA
                    if (pend >= 0 && !(ok = project(pend, pend_c, pend_t))) break;
                    pend = gc;
                    pend_c = c;
                    pend_t = ti;
                }
            }
            if (ok && pend >= 0 && !*abort) project(pend, pend_c, pend_t);
            // every MMA this thread issued has completed before TMEM is released
            umma_commit(&S.mma_done);
            mbar_drain(&S.mma_done, 0, a.err);
        }
    } else if (warp == 10) {
        // ---------------- W^T images and landmark norms of each chunk
        if (lane == 0) {
            const uint32_t nbytes = (uint32_t)(kChunk * 4);
            long long gc = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
                for (int c = 0; c < nchunks; ++c, ++gc) {
                    const int s = (int)(gc & 1);
                    const long long use = gc >> 1;
                    // stage s is free when the projection of its previous chunk is done
                    if (use > 0 && !mbar_wait(&S.w_empty[s], (uint32_t)((use - 1) & 1), abort, a.err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&S.w_full[s], kWImgBytes + nbytes);
                    bulk_load(S.w[s], a.Wimg + (int64_t)c * kWImgBytes, kWImgBytes, &S.w_full[s]);
                    bulk_load(S.nl[s], a.nrm_l + c * kChunk, nbytes, &S.w_full[s]);
                }
            }
            for (long long g = gc - 2 < 0 ? 0 : gc - 2; g < gc; ++g)
                mbar_drain(&S.w_full[g & 1], (uint32_t)((g >> 1) & 1), a.err);
        }
    } else {
        // ---------------- epilogue: warps 2-9, one accumulator row per thread;
        // warps 2-5 take columns 0-63 of every chunk, warps 6-9 columns 64-127
        // (two warps per TMEM lane quadrant).  Each thread reads its 64 FP32
        // values, forms A^2 and stores the BF16 hi words over the first 32 of
        // those columns and the lo words over the last 32, the layout the
        // projection MMA reads A from.  Every epilogue warp runs the same tiles
        // and chunks whatever happens (an aborted wait only skips the work).
        const int quad = warp & 3;                 // TMEM lane quadrant this warp may read
        const int half = (warp - 2) >> 2;          // column half of the chunk
        const int row = quad * 32 + lane;
        const uint32_t lanes = (uint32_t)(quad * 32) << 16;
        const int r = a.r;
        long long gc = 0;
        int ti = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++ti) {
            const int64_t gi = t * kRows + row;
            const float ny = gi < a.m ? (float)a.nrm_y[gi] : 0.f;
            for (int c = 0; c < nchunks; ++c, ++gc) {
                const int s = (int)(gc & 1), q = (int)(gc % kAcc);
                // warp-uniform: tcgen05.ld / st are .sync.aligned warp instructions
                const bool got = __all_sync(0xffffffffu,
                                            mbar_wait(&S.acc_full[q], (uint32_t)((gc / kAcc) & 1), abort, a.err) &&
                                                mbar_wait(&S.w_full[s], (uint32_t)((gc >> 1) & 1), abort, a.err));
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (got) {
                    const uint32_t col = tmem + lanes + (uint32_t)(q * kChunk + half * 64);
                    const float* ns = S.nl[s] + half * 64;
                    float v[2][32];
                    tmem_ld32(col, v[0]);
                    tmem_ld32(col + 32, v[1]);
                    uint32_t hi[32], lo[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int e = 2 * i;
                        const float a0 = fmaxf(fmaf(-2.f, v[e >> 5][e & 31], ny + ns[e]), 0.f);
                        const float a1 = fmaxf(fmaf(-2.f, v[(e + 1) >> 5][(e + 1) & 31], ny + ns[e + 1]), 0.f);
                        hi[i] = bf16x2_rn(a0, a1);
                        const float h0 = __uint_as_float(hi[i] << 16), h1 = __uint_as_float(hi[i] & 0xffff0000u);
                        lo[i] = bf16x2_rn(a0 - h0, a1 - h1);
                    }
                    tmem_st32(col, hi);
                    tmem_st32(col + 32, lo);
                    tmem_wait_st();
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&S.a2_full[q]);
            }
            // the tile's X (r <= 16 columns, the sum of the accumulator's two
            // halves) from the X accumulator: warps 2-5
            if (half == 0) {
                const bool got = __all_sync(0xffffffffu, mbar_wait(&S.x_full, (uint32_t)(ti & 1), abort, a.err));
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float x[2 * kTcMaxR];
                if (got) tmem_ld32(tmem + lanes + kXCol, x);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&S.x_empty);
                if (got && gi < a.m) {
#pragma unroll
                    for (int o = 0; o < kTcMaxR; ++o)
                        if (o < r) a.X[gi * r + o] = (x[o] + x[kTcMaxR + o]) + (float)a.bias[o];
                }
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

// W (l x r, float) -> per chunk of kChunk landmarks the shared-memory image
// of W^T that the projection MMAs read as their B operand: [64-landmark
// atom][32 rows: o = 0..15 of hi = bf16(w), then o = 0..15 of lo = bf16(w - hi)]
// [128 bytes], zeros for j >= l or o >= r, each row's 16-byte granules stored
// 128-byte swizzled (granule g of row R at position g ^ (R & 7)).
__global__ void k_w_image(const float* __restrict__ W, int l, int r, int nchunks, uint16_t* __restrict__ img) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nchunks * (kWImgBytes / 2)) return;
    const int k = (int)(e % kAtomK), R = (int)((e / kAtomK) % (2 * kTcMaxR));
    const int at = (int)((e / (kAtomK * 2 * kTcMaxR)) % 2), c = (int)(e / (kWImgBytes / 2));
    const int o = R % kTcMaxR, plane = R / kTcMaxR;
    const int j = c * kChunk + at * kAtomK + k;
    const float w = (j < l && o < r) ? W[(int64_t)j * r + o] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(w);
    const __nv_bfloat16 v = plane == 0 ? h : __float2bfloat16_rn(w - __bfloat162float(h));
    const int64_t byte = (int64_t)c * kWImgBytes + at * (int64_t)kWAtomBytes + R * 128 +
                         (((k >> 3) ^ (R & 7)) << 4) + (k & 7) * 2;
    img[byte / 2] = __bfloat16_as_ushort(v);
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

size_t gower_tc_w_bytes(int l) { return (size_t)(gower_tc_lpad(l) / kChunk) * kWImgBytes; }

cudaError_t launch_w_image(const float* W, int l, int r, void* img, cudaStream_t st) {
    const int nchunks = gower_tc_lpad(l) / kChunk;
    const int64_t total = (int64_t)nchunks * (kWImgBytes / 2);
    k_w_image<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(W, l, r, nchunks, (uint16_t*)img);
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

cudaError_t launch_gower_tc(const void* Ysplit, int64_t m, int64_t ylo_rows, int d, const double* nrm_y,
                            const void* Lsplit, const float* nrm_l, int l, const void* Wimg,
                            const double* bias, int r, float* X, int* err, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (!gower_tc_supported(d, r) || l < 1) return cudaErrorInvalidValue;
    const int ld = split_ld(d);
    const __nv_bfloat16* yh = (const __nv_bfloat16*)Ysplit;
    const __nv_bfloat16* lh = (const __nv_bfloat16*)Lsplit;
    CUtensorMap m_yhi, m_ylo, m_lhi, m_llo;
    if (!make_map(&m_yhi, yh, m, ld) || !make_map(&m_ylo, yh + ylo_rows * ld, m, ld) ||
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
    a.Wimg = (const uint8_t*)Wimg;
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
    cudaError_t e = cudaFuncSetAttribute(k_gower_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gower_tc<<<grid, kThreadsTc, smem, st>>>(m_yhi, m_ylo, m_lhi, m_llo, a);
    return cudaGetLastError();
}

}  // namespace gbmds
