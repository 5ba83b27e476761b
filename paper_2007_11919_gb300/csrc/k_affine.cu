// The affine form of interpolation MDS for rows given by coordinates.
//
// For Euclidean distances the landmarks' Q_1 is the Gram matrix of the
// centred landmark rows, Q_1 = L_c L_c^T (Section 2), so Gower's formula,
// Eq. (2), becomes a projection on the landmarks' principal axes:
//   Xdot = (Y - 1 y_L^T) U_r,   U_r = L_c^T V_r Lambda_r^{-1/2}   (d x r),
// with y_L the landmark mean and V_r, Lambda_r the landmarks' classical-MDS
// eigenpairs.  The landmark rows get X_1 = V_r Lambda_r^{1/2} back.  One pass
// over Y (HBM-bound) instead of n x l distances.
//
// The same two pieces serve pivot MDS (k_pivot.cu): the axes of a set of
// centred rows weighted by eigenvectors, and the projection (Y - 1 c^T) U.
#include <type_traits>

#include "common.cuh"
#include "tc_common.cuh"

namespace gbmds {
namespace {

__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }

constexpr int kAxThreads = 256;

// mean[k] = (1/l) sum_j L[j][k] over the rows of a dense l x d FP64 matrix:
// one CTA per column, the rows split over the threads, a fixed-order tree sum.
__global__ void __launch_bounds__(kAxThreads) k_rows_mean(const double* __restrict__ L, int l, int d,
                                                          double* __restrict__ mean, float* __restrict__ mean_f) {
    __shared__ double red[kAxThreads];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < l; j += kAxThreads) s += L[(int64_t)j * d + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kAxThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = red[0] / l;
        mean[k] = m;
        if (mean_f) mean_f[k] = (float)m;
    }
}

// U[k][i] = scale_i sum_j (L[j][k] - c_k) V[j][i] (d x r, row-major), FP64:
// one CTA per column k, the rows split over the threads, r partial sums per
// thread, a fixed-order tree sum per output.
__global__ void __launch_bounds__(kAxThreads) k_axes(const double* __restrict__ L, int l, int d,
                                                     const double* __restrict__ c, const double* __restrict__ V,
                                                     const double* __restrict__ scale, int r,
                                                     double* __restrict__ U, float* __restrict__ U_f) {
    __shared__ double red[kAxThreads];
    const int k = blockIdx.x;
    const double ck = c[k];
    double acc[kMaxR];
#pragma unroll
    for (int i = 0; i < kMaxR; ++i) acc[i] = 0.0;
    for (int j = threadIdx.x; j < l; j += kAxThreads) {
        const double x = L[(int64_t)j * d + k] - ck;
        const double* v = V + (int64_t)j * r;
#pragma unroll
        for (int i = 0; i < kMaxR; ++i)
            if (i < r) acc[i] = fma(x, v[i], acc[i]);
    }
    for (int i = 0; i < r; ++i) {
        red[threadIdx.x] = acc[i];
        __syncthreads();
        for (int h = kAxThreads / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double u = red[0] * scale[i];
            U[(int64_t)k * r + i] = u;
            if (U_f) U_f[(int64_t)k * r + i] = (float)u;
        }
        __syncthreads();
    }
}

// scale_i = 1 / sqrt(lambda_i): the affine form's U_r = L_c^T V_r Lambda_r^{-1/2}.
__global__ void k_inv_sqrt(const double* __restrict__ lam, int r, double* __restrict__ scale) {
    const int i = threadIdx.x;
    if (i < r) scale[i] = 1.0 / sqrt(lam[i]);
}

// X[row] = (y_row - c) U for FP32 rows with d a multiple of 4, a 16-byte
// aligned base and r <= R (R even).  Thread per row: each warp owns tiles of
// 32 consecutive rows and brings them into its kPbStages shared-memory stages
// with bulk asynchronous copies (cp.async.bulk, completion counted in bytes
// on one mbarrier per stage), so kPbStages tiles per warp are in flight while
// it computes.  A tile's rows sit at a stride of an odd number of 16-byte
// groups, so the 32 lanes reading their 32 rows hit distinct banks: when d/4
// is odd that is the rows' own layout in Y and one copy brings the tile,
// else each row is its own copy.  The arithmetic runs on pairs of columns
// with packed FP32 instructions (sub.rn.f32x2, fma.rn.f32x2): for columns
// (k, k+1), (y_k - c_k, y_{k+1} - c_{k+1}) times (U[k][i], U[k+1][i]) into a
// pair of accumulators per output i, whose halves are added at the end.  U and
// c are staged per column pair as float2 slots (slot 0 the centre pair, slot
// 1 + i the pair of output i) and read as broadcast 16-byte loads.  The r
// outputs of a tile's rows leave through a per-warp buffer as one coalesced
// block of 32 r floats.
constexpr int kPbWarps = 4;
constexpr int kPbStages = 2;

union Pack2 {
    float2 f;
    unsigned long long u;
};

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    Pack2 x, y, z;
    x.f = a;
    y.f = b;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(z.u) : "l"(x.u), "l"(y.u));
    return z.f;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    Pack2 x, y, w, z;
    x.f = a;
    y.f = b;
    w.f = c;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(z.u) : "l"(x.u), "l"(y.u), "l"(w.u));
    return z.f;
}

// One column pair: g points at its R / 2 + 1 groups of 16 bytes.
template <int R>
__device__ __forceinline__ void pair_step(float2 y, const float4* __restrict__ g, float2 (&acc)[R]) {
    const float4 g0 = g[0];
    const float2 yc = sub2(y, make_float2(g0.x, g0.y));
    acc[0] = fma2(yc, make_float2(g0.z, g0.w), acc[0]);
#pragma unroll
    for (int j = 1; j <= R / 2; ++j) {
        const float4 w = g[j];
        acc[2 * j - 1] = fma2(yc, make_float2(w.x, w.y), acc[2 * j - 1]);
        if (2 * j < R) acc[2 * j] = fma2(yc, make_float2(w.z, w.w), acc[2 * j]);
    }
}

// Bounded wait on a tile's stage; false after ~2 s (the copy source is
// ordinary device memory, so this only guards against a broken launch).
__device__ __forceinline__ bool tile_wait(uint64_t* bar, uint32_t parity) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = tc::global_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (tc::mbar_try_wait(bar, parity)) return true;
        if (tc::global_ns() - t0 > tc::kWaitNs) return false;
    }
}

__host__ __device__ inline size_t project_bulk_smem(int d, int R) {
    const int s4 = (d >> 2) | 1;
    return (size_t)(d >> 1) * (R / 2 + 1) * 16 + (size_t)kPbWarps * kPbStages * 32 * s4 * 16 +
           (size_t)kPbWarps * 32 * R * 4 + (size_t)kPbWarps * kPbStages * 8;
}

template <int R>
__global__ void __launch_bounds__(32 * kPbWarps) k_affine_project_bulk(const float* __restrict__ Y, int64_t n, int d,
                                                                       const float* __restrict__ cen,
                                                                       const float* __restrict__ U, int r,
                                                                       float* __restrict__ X, int* __restrict__ err) {
    constexpr int G = R / 2 + 1;   // 16-byte groups per column pair
    extern __shared__ __align__(16) unsigned char pb_smem[];
    const int d2 = d >> 1, d4 = d >> 2, s4 = d4 | 1;
    float4* const Up = reinterpret_cast<float4*>(pb_smem);
    float4* const tiles = Up + (size_t)d2 * G;
    float* const outs = reinterpret_cast<float*>(tiles + (size_t)kPbWarps * kPbStages * 32 * s4);
    uint64_t* const bars = reinterpret_cast<uint64_t*>(outs + (size_t)kPbWarps * 32 * R);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* const ring = tiles + (size_t)warp * kPbStages * 32 * s4;
    float* const out = outs + (size_t)warp * 32 * R;
    uint64_t* const bar = bars + warp * kPbStages;
    // float q of pair p's groups: float2 slot q / 2 of column 2 p + q % 2
    float* const Uf = reinterpret_cast<float*>(Up);
    for (int e = threadIdx.x; e < d2 * 4 * G; e += blockDim.x) {
        const int p = e / (4 * G), q = e - p * 4 * G, slot = q >> 1, k = 2 * p + (q & 1);
        Uf[e] = slot == 0 ? cen[k] : (slot - 1 < r ? U[(int64_t)k * r + slot - 1] : 0.f);
    }
    if (lane == 0) {
        for (int st = 0; st < kPbStages; ++st) tc::mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int64_t ntiles = (n + 31) >> 5;
    const int64_t wstride = (int64_t)gridDim.x * kPbWarps;
    const int64_t t0 = (int64_t)blockIdx.x * kPbWarps + warp;
    const bool one_copy = s4 == d4;
    // the whole warp calls this with the same tile
    auto issue = [&](int64_t tile, int st) {
        if (tile >= ntiles) return;
        const int64_t row0 = tile << 5;
        const int rows = (int)(n - row0 < 32 ? n - row0 : 32);
        float4* dst = ring + (size_t)st * 32 * s4;
        const float* src = Y + row0 * d;
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::mbar_expect_tx(&bar[st], (uint32_t)rows * (uint32_t)d * 4u);
        }
        __syncwarp();
        if (one_copy) {
            if (lane == 0) tc::bulk_load(dst, src, (uint32_t)rows * (uint32_t)d * 4u, &bar[st]);
        } else if (lane < rows) {
            tc::bulk_load(dst + (size_t)lane * s4, src + (int64_t)lane * d, (uint32_t)d * 4u, &bar[st]);
        }
    };
#pragma unroll
    for (int st = 0; st < kPbStages; ++st) issue(t0 + st * wstride, st);
    int it = 0;
    for (int64_t t = t0; t < ntiles; t += wstride, ++it) {
        const int st = it % kPbStages;
        if (!tile_wait(&bar[st], (uint32_t)(it / kPbStages) & 1u)) {
            // leave only after every copy of this warp in flight has landed
            if (lane == 0) atomicExch(err, MDS_ERR_TIMEOUT);
            for (int k = 0; k < kPbStages; ++k)
                if (t + (int64_t)k * wstride < ntiles)
                    tc::mbar_drain(&bar[(it + k) % kPbStages], (uint32_t)((it + k) / kPbStages) & 1u, err);
            return;
        }
        const int64_t row0 = t << 5;
        const int rows = (int)(n - row0 < 32 ? n - row0 : 32);
        if (lane < rows) {
            float2 acc[R];
#pragma unroll
            for (int i = 0; i < R; ++i) acc[i] = make_float2(0.f, 0.f);
            const float4* y4 = ring + (size_t)st * 32 * s4 + (size_t)lane * s4;
            const float4* g = Up;
#pragma unroll 2
            for (int c4 = 0; c4 < d4; ++c4, g += 2 * G) {
                const float4 v = y4[c4];
                pair_step<R>(make_float2(v.x, v.y), g, acc);
                pair_step<R>(make_float2(v.z, v.w), g + G, acc);
            }
#pragma unroll
            for (int i = 0; i < R; ++i)
                if (i < r) out[lane * r + i] = acc[i].x + acc[i].y;
        }
        __syncwarp();
        issue(t + (int64_t)kPbStages * wstride, st);   // the stage is consumed: the tile kPbStages ahead
        for (int e = lane; e < rows * r; e += 32) X[row0 * r + e] = out[e];
        __syncwarp();
    }
}

// General form: any element type and width, arithmetic type A.  U is staged
// transposed in shared memory (Us[i * d + k]) with the centre, so the lanes of
// a warp (one row, lanes over the columns) read consecutive words.
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_affine_project(const T* __restrict__ Y, int64_t n, int d,
                                                        const A* __restrict__ cen, const A* __restrict__ U,
                                                        int r, A* __restrict__ X) {
    extern __shared__ __align__(16) unsigned char asm_raw[];
    A* Us = reinterpret_cast<A*>(asm_raw);
    A* cs = Us + (size_t)r * d;
    for (int e = threadIdx.x; e < r * d; e += blockDim.x) {
        const int i = e / d, k = e % d;
        Us[e] = U[(int64_t)k * r + i];
    }
    for (int k = threadIdx.x; k < d; k += blockDim.x) cs[k] = cen[k];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
        A acc[kMaxR];
#pragma unroll
        for (int i = 0; i < kMaxR; ++i) acc[i] = A(0);
        const T* y = Y + row * d;
        for (int k = lane; k < d; k += 32) {
            const A yc = load_as<A, T>(y + k) - cs[k];
#pragma unroll
            for (int i = 0; i < kMaxR; ++i)
                if (i < r) acc[i] = mad(yc, Us[i * d + k], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < kMaxR; ++i) {
            if (i < r) {
                const A v = warp_sum(acc[i]);
                if (lane == 0) X[row * r + i] = v;
            }
        }
    }
}

unsigned project_grid(int64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 7) / 8;
    return (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
}

template <typename T, typename A>
cudaError_t project_general(const T* Y, int64_t n, int d, const A* cen, const A* U, int r, A* X, cudaStream_t st) {
    const size_t smem = sizeof(A) * ((size_t)r * d + d);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_affine_project<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_affine_project<T, A><<<project_grid(n), 256, smem, st>>>(Y, n, d, cen, U, r, X);
    return cudaSuccess;
}

template <typename T>
cudaError_t project_any(const T* Y, int64_t n, int d, const double* cen, const float* cen_f, const double* U,
                        const float* U_f, int r, int f64, void* X, int* err, cudaStream_t st) {
    cudaError_t e;
    if (f64) {
        e = project_general<T, double>(Y, n, d, cen, U, r, (double*)X, st);
    } else if (std::is_same<T, float>::value && d % 4 == 0 && r <= 16 &&
               project_bulk_smem(d, r + (r & 1)) <= 200 * 1024 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
        const float* Yf = reinterpret_cast<const float*>(Y);
        float* Xf = (float*)X;
        const int R = r + (r & 1);
        const size_t smem = project_bulk_smem(d, R);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t tiles = (n + 31) / 32;
        const int64_t want = (tiles + kPbWarps - 1) / kPbWarps;
        auto go = [&](auto kern) {
            cudaError_t r2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per_sm = 0;
            if (r2 == cudaSuccess)
                r2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kPbWarps, smem);
            if (r2 != cudaSuccess) return r2;
            const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
            const unsigned grid = (unsigned)(want < cap ? want : cap);
            kern<<<grid, 32 * kPbWarps, smem, st>>>(Yf, n, d, cen_f, U_f, r, Xf, err);
            return cudaSuccess;
        };
        switch (R) {
            case 2: e = go(k_affine_project_bulk<2>); break;
            case 4: e = go(k_affine_project_bulk<4>); break;
            case 6: e = go(k_affine_project_bulk<6>); break;
            case 8: e = go(k_affine_project_bulk<8>); break;
            case 10: e = go(k_affine_project_bulk<10>); break;
            case 12: e = go(k_affine_project_bulk<12>); break;
            case 14: e = go(k_affine_project_bulk<14>); break;
            default: e = go(k_affine_project_bulk<16>); break;
        }
    } else {
        e = project_general<T, float>(Y, n, d, cen_f, U_f, r, (float*)X, st);
    }
    if (e != cudaSuccess) return e;
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rows_mean(const double* L, int l, int d, double* mean, float* mean_f, cudaStream_t st) {
    if (l <= 0 || d <= 0) return cudaErrorInvalidValue;
    k_rows_mean<<<d, kAxThreads, 0, st>>>(L, l, d, mean, mean_f);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_axes(const double* L, int l, int d, const double* c, const double* V, const double* scale, int r,
                        double* U, float* U_f, cudaStream_t st) {
    if (l <= 0 || d <= 0 || r <= 0 || r > kMaxR) return cudaErrorInvalidValue;
    k_axes<<<d, kAxThreads, 0, st>>>(L, l, d, c, V, scale, r, U, U_f);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_affine_project(const void* Y, int dt, int64_t n, int d, const double* cen, const float* cen_f,
                                  const double* U, const float* U_f, int r, int f64, void* X, int* err,
                                  cudaStream_t st) {
    if (n <= 0 || d <= 0 || r <= 0 || r > kMaxR || !err) return cudaErrorInvalidValue;
    if (dt == MDS_IN_F64) return project_any((const double*)Y, n, d, cen, cen_f, U, U_f, r, f64, X, err, st);
    if (dt == MDS_IN_F32) return project_any((const float*)Y, n, d, cen, cen_f, U, U_f, r, f64, X, err, st);
    return project_any((const uint8_t*)Y, n, d, cen, cen_f, U, U_f, r, f64, X, err, st);
}

cudaError_t launch_affine_axes(const double* Lg, int l, int d, const double* V, const double* lam, int r,
                               double* scale, double* ybar, float* ybar_f, double* U, float* U_f, cudaStream_t st) {
    if (d <= 0 || l <= 0 || r <= 0 || r > kMaxR) return cudaErrorInvalidValue;
    cudaError_t e = launch_rows_mean(Lg, l, d, ybar, ybar_f, st);
    if (e != cudaSuccess) return e;
    k_inv_sqrt<<<1, 32, 0, st>>>(lam, r, scale);
    note_launch(1);
    return launch_axes(Lg, l, d, ybar, V, scale, r, U, U_f, st);
}

}  // namespace gbmds
