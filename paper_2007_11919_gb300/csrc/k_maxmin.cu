// MaxMin choice of the landmarks of LMDS (Section 3.1): starting from a
// given row, each next landmark is the row whose smallest squared Euclidean
// distance to the landmarks already chosen is largest (ties: lowest row
// index; a chosen row is never chosen again).
//
// The choice is sequential, so each round is one launch that streams every
// row of Y once against the newest landmark, folds the distance into the
// row's running minimum m_i (FP64), and takes the argmax of m over the rows
// not yet chosen (chosen rows hold m_i = -1).  The CTAs publish their best
// (m, i) pair; the last CTA to finish reduces them and records the pick.
//
// Exactness.  The pick is an argmax of FP64 values, taken in FP64 as in the
// FP64 definition (a general round with one warp per row, and a tiled round
// with one thread per row for FP32 and byte rows, below):
//   byte rows   integer differences and sums (exact; the FP64 value too),
//   FP64 rows   the FP64 difference form sum_k (y_k - l_k)^2,
//   FP32 rows   first an FP32 difference form; when it exceeds m_i by more
//               than its rounding bound, (d + 4) 2^-23 relative for d
//               non-negative terms, m_i cannot change and the row is done;
//               otherwise the FP64 difference form decides, as for FP64 rows.
#include <algorithm>

#include "common.cuh"
#include "tc_common.cuh"

namespace gbmds {
namespace {

constexpr int kMmThreads = 256;
constexpr int kMmWarps = kMmThreads / 32;

// (v, i) beats (w, j): larger value, or equal value and lower index.
__device__ __forceinline__ bool beats(double v, int64_t i, double w, int64_t j) {
    return v > w || (v == w && i < j);
}

__device__ __forceinline__ void warp_best(double& v, int64_t& i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t j = __shfl_xor_sync(0xffffffffu, i, o);
        if (beats(w, j, v, i)) {
            v = w;
            i = j;
        }
    }
}

// FP64 difference form of row y against the landmark row held in shared
// memory (as double), lanes over the columns, warp sum.
template <typename T>
__device__ __forceinline__ double dist_f64(const T* __restrict__ y, const double* __restrict__ lm, int d, int lane) {
    double s = 0.0;
    for (int k = lane; k < d; k += 32) {
        const double t = (double)y[k] - lm[k];
        s = fma(t, t, s);
    }
    return warp_sum(s);
}

// One round.  cur[0]: the newest landmark row.  mind: running minima (FP64;
// -1 for chosen rows; +inf before the first round).  The CTAs' best pairs go
// to part_v / part_i; the last CTA writes the pick to idx_out[k] and cur[0],
// marks it chosen, and re-arms the counter.
template <typename T>
__global__ void __launch_bounds__(kMmThreads) k_maxmin_round(const T* __restrict__ Y, int64_t n, int d,
                                                             int64_t* __restrict__ cur, double* __restrict__ mind,
                                                             double* __restrict__ part_v, int64_t* __restrict__ part_i,
                                                             unsigned* __restrict__ counter,
                                                             int64_t* __restrict__ idx_out, int k) {
    extern __shared__ __align__(16) double lm[];              // the landmark row as double, then as T
    T* lmt = reinterpret_cast<T*>(lm + d);
    __shared__ double wv[kMmWarps];
    __shared__ int64_t wi[kMmWarps];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t lrow = cur[0];
    for (int c = threadIdx.x; c < d; c += kMmThreads) {
        const T v = Y[lrow * d + c];
        lm[c] = (double)v;
        lmt[c] = v;
    }
    __syncthreads();

    double bv = -2.0;
    int64_t bi = INT64_MAX;
    const int64_t warps = (int64_t)gridDim.x * kMmWarps;
    for (int64_t i = (int64_t)blockIdx.x * kMmWarps + warp; i < n; i += warps) {
        double m = mind[i];                      // warp-uniform
        if (m >= 0.0) {
            const T* y = Y + i * d;
            double dn;
            if constexpr (sizeof(T) == 1) {
                int s = 0;                       // exact: d * 255^2 < 2^31 for d < 33026
                for (int c = lane; c < d; c += 32) {
                    const int t = (int)y[c] - (int)lmt[c];
                    s += t * t;
                }
                dn = (double)warp_sum(s);
            } else if constexpr (sizeof(T) == 4) {
                float s = 0.f;
                for (int c = lane; c < d; c += 32) {
                    const float t = y[c] - lmt[c];
                    s = fmaf(t, t, s);
                }
                s = warp_sum(s);
                // the FP32 value is within (d + 4) 2^-24 relative of the exact
                // sum of non-negative terms: far enough above m, the FP64
                // value is too and m stays; otherwise FP64 decides
                const double bound = (double)s * (1.0 - (double)(d + 4) * 0x1p-23);
                dn = bound > m ? m : dist_f64(y, lm, d, lane);
            } else {
                dn = dist_f64(y, lm, d, lane);
            }
            if (dn < m) m = dn;
            if (lane == 0) mind[i] = m;
            if (beats(m, i, bv, bi)) {
                bv = m;
                bi = i;
            }
        } else if (beats(m, i, bv, bi)) {        // chosen rows: -1, below every free row
            bv = m;
            bi = i;
        }
    }
    // the CTA's best pair (the lanes agree; lane 0 holds it)
    if (lane == 0) {
        wv[warp] = bv;
        wi[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = wv[0];
        int64_t j = wi[0];
        for (int w = 1; w < kMmWarps; ++w)
            if (beats(wv[w], wi[w], v, j)) {
                v = wv[w];
                j = wi[w];
            }
        part_v[blockIdx.x] = v;
        part_i[blockIdx.x] = j;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last CTA: every other CTA's pair is visible (fence before its arrival)
    __threadfence();
    double v = -2.0;
    int64_t j = INT64_MAX;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kMmThreads) {
        const double pv = __ldcg(part_v + b);
        const int64_t pi = __ldcg(part_i + b);
        if (beats(pv, pi, v, j)) {
            v = pv;
            j = pi;
        }
    }
    warp_best(v, j);
    if (lane == 0) {
        wv[warp] = v;
        wi[warp] = j;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kMmWarps; ++w)
            if (beats(wv[w], wi[w], wv[0], wi[0])) {
                wv[0] = wv[w];
                wi[0] = wi[w];
            }
        const int64_t pick = wi[0];
        idx_out[k] = pick;
        cur[0] = pick;
        mind[pick] = -1.0;
        *counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// Tiled form for FP32 rows (d a multiple of 4) and byte rows (d a multiple of
// 16): thread per row.  Each warp owns tiles of 32 consecutive rows (32 d
// contiguous elements of Y) and brings them into its kMmStages shared-memory
// stages with bulk asynchronous copies (cp.async.bulk, completion counted in
// bytes on one mbarrier per stage), so kMmStages tiles per warp are in flight
// while it computes; the row stride is an odd number of 16-byte groups so
// that 32 lanes reading 32 rows hit distinct banks (the rows' own layout in
// Y when d/4 (d/16 for bytes) is odd: one copy per tile; else one per row).
// The landmark row is broadcast from shared memory.  Lane q owns row q of the
// tile: no warp reductions.
//   byte rows   d^2 = |y|^2 + |l|^2 - 2 y.l in integers (y.l by __dp4a, the
//               row norms computed once): exact.
//   FP32 rows   the bounded FP32 difference form (column pairs with packed
//               sub.rn.f32x2 / fma.rn.f32x2 into two chains of d/2 terms,
//               well inside the bound above), and the FP64 difference form
//               where the running minimum may change, computed for those
//               rows one at a time by the whole warp (lanes over the columns):
//               FP64 issues at 1/64 of FP32, so one lane looping over d
//               columns would hold the warp for d FP64 instructions.
constexpr int kTw = 4;          // warps per CTA of the tiled round
constexpr int kMmStages = 2;    // tiles in flight per warp

union MmPack2 {
    float2 f;
    unsigned long long u;
};

__device__ __forceinline__ float2 mm_sub2(float2 a, float2 b) {
    MmPack2 x, y, z;
    x.f = a;
    y.f = b;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(z.u) : "l"(x.u), "l"(y.u));
    return z.f;
}

__device__ __forceinline__ float2 mm_fma2(float2 a, float2 b, float2 c) {
    MmPack2 x, y, w, z;
    x.f = a;
    y.f = b;
    w.f = c;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(z.u) : "l"(x.u), "l"(y.u), "l"(w.u));
    return z.f;
}

// Bounded wait on a tile's stage; false after ~2 s (the copy source is
// ordinary device memory, so this only guards against a broken launch).
__device__ __forceinline__ bool mm_tile_wait(uint64_t* bar, uint32_t parity) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = tc::global_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (tc::mbar_try_wait(bar, parity)) return true;
        if (tc::global_ns() - t0 > tc::kWaitNs) return false;
    }
}

// The CTA's best (v, i) pair from every thread's, then the round's pick by the
// last CTA to finish (as in k_maxmin_round).
__device__ void mm_pick(double bv, int64_t bi, double* __restrict__ part_v, int64_t* __restrict__ part_i,
                        unsigned* __restrict__ counter, int64_t* __restrict__ cur, double* __restrict__ mind,
                        int64_t* __restrict__ idx_out, int k) {
    __shared__ double wv[32];
    __shared__ int64_t wi[32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_best(bv, bi);
    if (lane == 0) {
        wv[warp] = bv;
        wi[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = wv[0];
        int64_t j = wi[0];
        for (int w = 1; w < nw; ++w)
            if (beats(wv[w], wi[w], v, j)) {
                v = wv[w];
                j = wi[w];
            }
        part_v[blockIdx.x] = v;
        part_i[blockIdx.x] = j;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = -2.0;
    int64_t j = INT64_MAX;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const double pv = __ldcg(part_v + b);
        const int64_t pi = __ldcg(part_i + b);
        if (beats(pv, pi, v, j)) {
            v = pv;
            j = pi;
        }
    }
    warp_best(v, j);
    __syncthreads();
    if (lane == 0) {
        wv[warp] = v;
        wi[warp] = j;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            if (beats(wv[w], wi[w], wv[0], wi[0])) {
                wv[0] = wv[w];
                wi[0] = wi[w];
            }
        const int64_t pick = wi[0];
        idx_out[k] = pick;
        cur[0] = pick;
        mind[pick] = -1.0;
        *counter = 0u;
    }
}

template <bool U8>
__global__ void __launch_bounds__(32 * kTw) k_maxmin_tiles(const void* __restrict__ Yv, int64_t n, int d,
                                                           const int* __restrict__ nrm8, int64_t* __restrict__ cur,
                                                           double* __restrict__ mind, double* __restrict__ part_v,
                                                           int64_t* __restrict__ part_i, unsigned* __restrict__ counter,
                                                           int64_t* __restrict__ idx_out, int k, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char mm_smem[];
    __shared__ int s_lnorm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g16 = U8 ? d >> 4 : d >> 2;       // 16-byte groups per row
    const int s16 = g16 | 1;                    // padded row stride (odd)
    // landmark row: bytes (U8), or floats then doubles (FP32); the stages; their barriers
    uint4* lm16 = reinterpret_cast<uint4*>(mm_smem);
    double* lm64 = reinterpret_cast<double*>(mm_smem + (size_t)g16 * 16);
    uint4* bufs = reinterpret_cast<uint4*>(mm_smem + (size_t)g16 * 16 + (U8 ? 0 : (size_t)d * 8));
    uint4* const ring = bufs + (size_t)warp * kMmStages * 32 * s16;
    uint64_t* const bar = reinterpret_cast<uint64_t*>(bufs + (size_t)kTw * kMmStages * 32 * s16) + warp * kMmStages;
    const int64_t lrow = cur[0];
    const uint4* Y16 = reinterpret_cast<const uint4*>(Yv);
    for (int g = threadIdx.x; g < g16; g += blockDim.x) lm16[g] = Y16[lrow * g16 + g];
    if (threadIdx.x == 0) s_lnorm = 0;
    if (lane == 0) {
        for (int st = 0; st < kMmStages; ++st) tc::mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (U8) {
        unsigned sq = 0;
        for (int g = threadIdx.x; g < g16; g += blockDim.x) {
            const uint4 w = lm16[g];
            sq = __dp4a(w.x, w.x, sq);
            sq = __dp4a(w.y, w.y, sq);
            sq = __dp4a(w.z, w.z, sq);
            sq = __dp4a(w.w, w.w, sq);
        }
        atomicAdd(&s_lnorm, (int)sq);
    } else {
        const float* lf = reinterpret_cast<const float*>(lm16);
        for (int c = threadIdx.x; c < d; c += blockDim.x) lm64[c] = (double)lf[c];
    }
    __syncthreads();
    const int lnorm = s_lnorm;
    const int64_t tiles = (n + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * kTw;
    const int64_t t0 = (int64_t)blockIdx.x * kTw + warp;
    const bool one_copy = s16 == g16;
    // the whole warp calls this with the same tile
    auto issue = [&](int64_t tile, int st) {
        if (tile >= tiles) return;
        const int64_t row0 = tile * 32;
        const int rows = (int)(n - row0 < 32 ? n - row0 : 32);
        uint4* dst = ring + (size_t)st * 32 * s16;
        const uint4* src = Y16 + row0 * g16;
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::mbar_expect_tx(&bar[st], (uint32_t)rows * (uint32_t)g16 * 16u);
        }
        __syncwarp();
        if (one_copy) {
            if (lane == 0) tc::bulk_load(dst, src, (uint32_t)rows * (uint32_t)g16 * 16u, &bar[st]);
        } else if (lane < rows) {
            tc::bulk_load(dst + (size_t)lane * s16, src + (int64_t)lane * g16, (uint32_t)g16 * 16u, &bar[st]);
        }
    };
#pragma unroll
    for (int st = 0; st < kMmStages; ++st) issue(t0 + st * wstride, st);
    double bv = -2.0;
    int64_t bi = INT64_MAX;
    int it = 0;
    for (int64_t t = t0; t < tiles; t += wstride, ++it) {
        const int st = it % kMmStages;
        const int64_t row = t * 32 + lane;
        double m = row < n ? mind[row] : -1.0;   // loaded while the tile lands
        if (!mm_tile_wait(&bar[st], (uint32_t)(it / kMmStages) & 1u)) {
            // give up on this round after the warp's copies in flight have
            // landed; the CTA still takes part in the pick (its barriers)
            if (lane == 0) atomicExch(err, MDS_ERR_TIMEOUT);
            for (int q = 0; q < kMmStages; ++q)
                if (t + (int64_t)q * wstride < tiles)
                    tc::mbar_drain(&bar[(it + q) % kMmStages], (uint32_t)((it + q) / kMmStages) & 1u, err);
            break;
        }
        const uint4* const tile = ring + (size_t)st * 32 * s16;
        bool need64 = false;   // FP32 rows: the FP64 difference form decides
        double dn = m;
        if (row < n && m >= 0.0) {
            const uint4* y = tile + (size_t)lane * s16;
            if (U8) {
                unsigned dot = 0;
                for (int g = 0; g < g16; ++g) {
                    const uint4 a = y[g], b = lm16[g];
                    dot = __dp4a(a.x, b.x, dot);
                    dot = __dp4a(a.y, b.y, dot);
                    dot = __dp4a(a.z, b.z, dot);
                    dot = __dp4a(a.w, b.w, dot);
                }
                dn = (double)((long long)nrm8[row] + lnorm - 2ll * (long long)dot);
            } else {
                const float4* y4 = reinterpret_cast<const float4*>(y);
                const float4* l4 = reinterpret_cast<const float4*>(lm16);
                float2 s2 = make_float2(0.f, 0.f);
#pragma unroll 2
                for (int g = 0; g < g16; ++g) {
                    const float4 a = y4[g], b = l4[g];
                    const float2 t01 = mm_sub2(make_float2(a.x, a.y), make_float2(b.x, b.y));
                    const float2 t23 = mm_sub2(make_float2(a.z, a.w), make_float2(b.z, b.w));
                    s2 = mm_fma2(t01, t01, s2);
                    s2 = mm_fma2(t23, t23, s2);
                }
                const float s = s2.x + s2.y;
                // FP32 value within (d + 4) 2^-24 relative of the exact sum
                const double bound = (double)s * (1.0 - (double)(d + 4) * 0x1p-23);
                need64 = !(bound > m);
            }
        }
        if (!U8) {
            // the rows whose minimum may change: the FP64 difference form.  A
            // few rows (the usual case after the first rounds) one at a time
            // by the whole warp, lanes over the columns and a fixed butterfly
            // sum (every lane holds the same total); many rows each by its
            // own lane, columns in order (one FP64 pass of d columns for the
            // warp, cheaper than ~d/32 + 5 FP64 instructions per row from ~14
            // rows on).
            unsigned pend = __ballot_sync(0xffffffffu, need64);
            if (__popc(pend) > 13) {
                if (need64) {
                    const float* yf = reinterpret_cast<const float*>(tile + (size_t)lane * s16);
                    double s64 = 0.0;
                    for (int c = 0; c < d; ++c) {
                        const double t64 = (double)yf[c] - lm64[c];
                        s64 = fma(t64, t64, s64);
                    }
                    dn = s64;
                }
                pend = 0;
            }
            while (pend) {
                const int q = __ffs(pend) - 1;
                pend &= pend - 1;
                const float* yq = reinterpret_cast<const float*>(tile + (size_t)q * s16);
                double s64 = 0.0;
                for (int c = lane; c < d; c += 32) {
                    const double t64 = (double)yq[c] - lm64[c];
                    s64 = fma(t64, t64, s64);
                }
                s64 = warp_sum(s64);
                if (lane == q) dn = s64;
            }
        }
        if (row < n) {
            if (m >= 0.0 && dn < m) {
                m = dn;
                mind[row] = m;
            }
            if (beats(m, row, bv, bi)) {
                bv = m;
                bi = row;
            }
        }
        __syncwarp();
        issue(t + (int64_t)kMmStages * wstride, st);   // the stage is consumed: the tile kMmStages ahead
    }
    mm_pick(bv, bi, part_v, part_i, counter, cur, mind, idx_out, k);
}

// Squared norms of byte rows (exact, int): one warp per row.
__global__ void k_norms8(const uint8_t* __restrict__ Y, int64_t n, int d, int* __restrict__ nrm) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= n) return;
    int s = 0;
    for (int c = lane; c < d; c += 32) {
        const int v = Y[row * d + c];
        s += v * v;
    }
    s = warp_sum(s);
    if (lane == 0) nrm[row] = s;
}

__global__ void k_maxmin_init(int64_t n, int64_t first, double* __restrict__ mind, int64_t* __restrict__ cur,
                              int64_t* __restrict__ idx_out, unsigned* __restrict__ counter) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mind[i] = i == first ? -1.0 : __longlong_as_double(0x7ff0000000000000ll);   // +inf
    if (i == 0) {
        cur[0] = first;
        idx_out[0] = first;
        *counter = 0u;
    }
}

template <typename T>
cudaError_t maxmin_rounds(const T* Y, int64_t n, int d, int l, int64_t first, MaxminWs ws, int64_t* idx_out,
                          int grid, cudaStream_t st) {
    k_maxmin_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, first, ws.mind, ws.cur, idx_out, ws.counter);
    const size_t smem = (sizeof(double) + sizeof(T)) * (size_t)d;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_maxmin_round<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    for (int k = 1; k < l; ++k)
        k_maxmin_round<T><<<grid, kMmThreads, smem, st>>>(Y, n, d, ws.cur, ws.mind, ws.part_v, ws.part_i,
                                                          ws.counter, idx_out, k);
    note_launch(l);
    return cudaGetLastError();
}

}  // namespace

int maxmin_grid() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g = sms * 8;   // 8 CTAs of 8 warps per SM: 64 rows in flight per SM
    return g < kMaxminGridCap ? g : kMaxminGridCap;
}

// Shared memory of the tiled round (0: the shapes it does not take).
size_t maxmin_tiles_smem(int dt, int d) {
    const size_t bars = (size_t)kTw * kMmStages * 8;
    if (dt == MDS_IN_U8 && d % 16 == 0)
        return (size_t)(d / 16) * 16 + (size_t)kMmStages * kTw * 32 * ((d / 16) | 1) * 16 + bars;
    if (dt == MDS_IN_F32 && d % 4 == 0)
        return (size_t)(d / 4) * 16 + (size_t)d * 8 + (size_t)kMmStages * kTw * 32 * ((d / 4) | 1) * 16 + bars;
    return 0;
}

template <bool U8>
cudaError_t maxmin_tiled(const void* Y, int64_t n, int d, int l, int64_t first, MaxminWs ws, int64_t* idx_out,
                         size_t smem, cudaStream_t st) {
    k_maxmin_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, first, ws.mind, ws.cur, idx_out, ws.counter);
    if (U8) k_norms8<<<(unsigned)((n + 7) / 8), 256, 0, st>>>((const uint8_t*)Y, n, d, ws.nrm8);
    cudaError_t e = cudaFuncSetAttribute(k_maxmin_tiles<U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_maxmin_tiles<U8>, 32 * kTw, smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + 31) / 32;
    int64_t grid = std::min<int64_t>((int64_t)sms * std::max(per, 1), (tiles + kTw - 1) / kTw);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, kMaxminGridCap));
    for (int k = 1; k < l; ++k)
        k_maxmin_tiles<U8><<<(unsigned)grid, 32 * kTw, smem, st>>>(Y, n, d, ws.nrm8, ws.cur, ws.mind, ws.part_v,
                                                                  ws.part_i, ws.counter, idx_out, k, ws.err);
    note_launch(l + (U8 ? 1 : 0));
    return cudaGetLastError();
}

cudaError_t launch_maxmin(const void* Y, int dt, int64_t n, int d, int l, int64_t first, MaxminWs ws,
                          int64_t* idx_out, cudaStream_t st) {
    if (n <= 0 || d <= 0 || l <= 0 || d > kMaxminD) return cudaErrorInvalidValue;
    const size_t tsm = maxmin_tiles_smem(dt, d);
    if (tsm > 0 && tsm <= 200 * 1024 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
        if (dt == MDS_IN_U8) return maxmin_tiled<true>(Y, n, d, l, first, ws, idx_out, tsm, st);
        return maxmin_tiled<false>(Y, n, d, l, first, ws, idx_out, tsm, st);
    }
    const int grid = maxmin_grid();
    if (dt == MDS_IN_F64) return maxmin_rounds((const double*)Y, n, d, l, first, ws, idx_out, grid, st);
    if (dt == MDS_IN_F32) return maxmin_rounds((const float*)Y, n, d, l, first, ws, idx_out, grid, st);
    return maxmin_rounds((const uint8_t*)Y, n, d, l, first, ws, idx_out, grid, st);
}

}  // namespace gbmds
