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

// X[row] = (y_row - c) U for FP32 rows with d <= 128 a multiple of 4, r < RB
// and a 16-byte aligned base.  Thread per row: each warp owns tiles of 32
// consecutive rows (32 d contiguous floats in global memory), copied into its
// shared-memory buffer with cp.async (two buffers: the next tile is in flight
// while this one is computed), the row stride padded to an odd number of
// 16-byte groups so that 32 lanes reading 32 rows hit distinct banks.  Lane q
// computes row q of the tile: for each column k, acc_i += (y_k - c_k) U[k][i]
// with the row of U and c_k (stored as Uc[k][0..RB), c_k at RB - 1) read as
// broadcast 16-byte loads.  The r outputs of the 32 rows leave through the
// consumed buffer as one coalesced block of 32 r floats.
constexpr int kPfWarps = 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int RB>
__global__ void __launch_bounds__(32 * kPfWarps) k_affine_project_f4(const float* __restrict__ Y, int64_t n, int d,
                                                                     const float* __restrict__ cen,
                                                                     const float* __restrict__ U, int r,
                                                                     float* __restrict__ X) {
    extern __shared__ __align__(16) float pf_smem[];
    const int d4 = d >> 2, s4 = d4 | 1;                     // row stride in 16-byte groups (odd)
    float* Uc = pf_smem;                                    // d x RB
    float4* bufs = reinterpret_cast<float4*>(pf_smem + (size_t)d * RB);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* const buf0 = bufs + (size_t)(2 * warp) * 32 * s4;
    float4* const buf1 = buf0 + (size_t)32 * s4;
    for (int e = threadIdx.x; e < d * RB; e += blockDim.x) {
        const int k = e / RB, i = e % RB;
        Uc[e] = i < r ? U[(int64_t)k * r + i] : (i == RB - 1 ? cen[k] : 0.f);
    }
    __syncthreads();
    const int64_t tiles = (n + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * kPfWarps;
    int64_t t = (int64_t)blockIdx.x * kPfWarps + warp;
    // the tile's contiguous floats: 16-byte group j = row * d4 + c4 -> buf[row * s4 + c4]
    auto issue = [&](int64_t tile, float4* dst) {
        if (tile < tiles) {
            const int64_t row0 = tile * 32;
            const int rows = (int)(n - row0 < 32 ? n - row0 : 32);
            const float4* src = reinterpret_cast<const float4*>(Y + row0 * d);
            for (int j = lane; j < rows * d4; j += 32) {
                const int row = j / d4, c4 = j - row * d4;
                cp_async16(dst + row * s4 + c4, src + j);
            }
        }
        cp_async_commit();
    };
    issue(t, buf0);
    for (int it = 0; t < tiles; t += wstride, ++it) {
        float4* cur = (it & 1) ? buf1 : buf0;
        issue(t + wstride, (it & 1) ? buf0 : buf1);
        cp_async_wait<1>();
        __syncwarp();
        const int64_t row0 = t * 32;
        const int rows = (int)(n - row0 < 32 ? n - row0 : 32);
        float acc[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) acc[i] = 0.f;
        if (lane < rows) {
            const float4* y4 = cur + lane * s4;
            for (int c4 = 0; c4 < d4; ++c4) {
                const float4 v = y4[c4];
                const float yv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float4* u4 = reinterpret_cast<const float4*>(Uc + (size_t)(4 * c4 + e) * RB);
                    float u[RB];
#pragma unroll
                    for (int g = 0; g < RB / 4; ++g) {
                        const float4 w = u4[g];
                        u[4 * g] = w.x;
                        u[4 * g + 1] = w.y;
                        u[4 * g + 2] = w.z;
                        u[4 * g + 3] = w.w;
                    }
                    const float yc = yv[e] - u[RB - 1];
#pragma unroll
                    for (int i = 0; i < RB - 1; ++i) acc[i] = fmaf(yc, u[i], acc[i]);
                }
            }
        }
        __syncwarp();
        // the outputs of the tile's rows through the consumed buffer, coalesced
        float* o = reinterpret_cast<float*>(cur);
        if (lane < rows) {
#pragma unroll
            for (int i = 0; i < RB - 1; ++i)
                if (i < r) o[lane * r + i] = acc[i];
        }
        __syncwarp();
        for (int e = lane; e < rows * r; e += 32) X[row0 * r + e] = o[e];
        __syncwarp();
    }
    cp_async_wait<0>();
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
                        const float* U_f, int r, int f64, void* X, cudaStream_t st) {
    cudaError_t e;
    if (f64) {
        e = project_general<T, double>(Y, n, d, cen, U, r, (double*)X, st);
    } else if (std::is_same<T, float>::value && d % 4 == 0 && d <= 128 && r <= 15 && r <= 4 * ((d >> 2) | 1) &&
               (reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
        const float* Yf = reinterpret_cast<const float*>(Y);
        float* Xf = (float*)X;
        const int RB = r < 8 ? 8 : (r < 12 ? 12 : 16);
        const size_t smem = sizeof(float) * (size_t)d * RB + (size_t)2 * kPfWarps * 32 * ((d >> 2) | 1) * 16;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t tiles = (n + 31) / 32;
        const int64_t want = (tiles + kPfWarps - 1) / kPfWarps;
        const unsigned grid = (unsigned)(want < (int64_t)sms * 2 ? want : (int64_t)sms * 2);
        auto go = [&](auto kern) {
            cudaError_t r2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (r2 == cudaSuccess) kern<<<grid, 32 * kPfWarps, smem, st>>>(Yf, n, d, cen_f, U_f, r, Xf);
            return r2;
        };
        e = RB == 8 ? go(k_affine_project_f4<8>) : (RB == 12 ? go(k_affine_project_f4<12>) : go(k_affine_project_f4<16>));
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
                                  const double* U, const float* U_f, int r, int f64, void* X, cudaStream_t st) {
    if (n <= 0 || d <= 0 || r <= 0 || r > kMaxR) return cudaErrorInvalidValue;
    if (dt == MDS_IN_F64) return project_any((const double*)Y, n, d, cen, cen_f, U, U_f, r, f64, X, st);
    if (dt == MDS_IN_F32) return project_any((const float*)Y, n, d, cen, cen_f, U, U_f, r, f64, X, st);
    return project_any((const uint8_t*)Y, n, d, cen, cen_f, U, U_f, r, f64, X, st);
}

cudaError_t launch_affine(const void* Y, int dt, int64_t n, int d, const double* Lg, int l, const double* V,
                          const double* lam, int r, int f64, double* scale, double* ybar, float* ybar_f, double* U,
                          float* U_f, void* X, cudaStream_t st) {
    if (n <= 0 || d <= 0 || l <= 0 || r <= 0 || r > kMaxR) return cudaErrorInvalidValue;
    cudaError_t e = launch_rows_mean(Lg, l, d, ybar, ybar_f, st);
    if (e != cudaSuccess) return e;
    k_inv_sqrt<<<1, 32, 0, st>>>(lam, r, scale);
    note_launch(1);
    e = launch_axes(Lg, l, d, ybar, V, scale, r, U, U_f, st);
    if (e != cudaSuccess) return e;
    return launch_affine_project(Y, dt, n, d, ybar, ybar_f, U, U_f, r, f64, X, st);
}

}  // namespace gbmds
