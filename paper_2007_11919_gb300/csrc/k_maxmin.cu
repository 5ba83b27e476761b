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
// FP64 definition:
//   byte rows   integer differences and sums (exact; the FP64 value too),
//   FP64 rows   the FP64 difference form sum_k (y_k - l_k)^2,
//   FP32 rows   first an FP32 difference form; when it exceeds m_i by more
//               than its rounding bound, (d + 4) 2^-23 relative for d
//               non-negative terms, m_i cannot change and the row is done;
//               otherwise the FP64 difference form decides, as for FP64 rows.
#include "common.cuh"

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

cudaError_t launch_maxmin(const void* Y, int dt, int64_t n, int d, int l, int64_t first, MaxminWs ws,
                          int64_t* idx_out, cudaStream_t st) {
    if (n <= 0 || d <= 0 || l <= 0 || d > kMaxminD) return cudaErrorInvalidValue;
    const int grid = maxmin_grid();
    if (dt == MDS_IN_F64) return maxmin_rounds((const double*)Y, n, d, l, first, ws, idx_out, grid, st);
    if (dt == MDS_IN_F32) return maxmin_rounds((const float*)Y, n, d, l, first, ws, idx_out, grid, st);
    return maxmin_rounds((const uint8_t*)Y, n, d, l, first, ws, idx_out, grid, st);
}

}  // namespace gbmds
