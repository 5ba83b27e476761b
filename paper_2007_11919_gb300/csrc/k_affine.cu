// The affine form of interpolation MDS for rows given by coordinates.
//
// For Euclidean distances the landmarks' Q_1 is the Gram matrix of the
// centred landmark rows, Q_1 = L_c L_c^T (Section 2), so Gower's formula,
// Eq. (2), becomes a projection on the landmarks' principal axes:
//   Xdot = (Y - 1 y_L^T) U_r,   U_r = L_c^T V_r Lambda_r^{-1/2}   (d x r),
// with y_L the landmark mean and V_r, Lambda_r the landmarks' classical-MDS
// eigenpairs.  The landmark rows get X_1 = V_r Lambda_r^{1/2} back.  One pass
// over Y (HBM-bound) instead of n x l distances.
#include "common.cuh"

namespace gbmds {
namespace {

__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }

// Row idx[j] of Y, clamped into [0, ny): a bad index (flagged by the index
// check, which fails the call) never reads outside Y.
__device__ __forceinline__ int64_t clamp_row(int64_t row, int64_t ny) { return row < 0 ? 0 : (row >= ny ? ny - 1 : row); }

// y_L[k] = mean over the landmark rows of y_jk, in FP64 (one thread per column).
template <typename T>
__global__ void __launch_bounds__(256) k_affine_mean(const T* __restrict__ Y, int64_t ny, int d,
                                                     const int64_t* __restrict__ idx, int l,
                                                     double* __restrict__ ybar, float* __restrict__ ybar_f) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d) return;
    double s = 0.0;
    for (int j = 0; j < l; ++j) s += load_as<double, T>(Y + clamp_row(idx[j], ny) * d + k);
    const double m = s / l;
    ybar[k] = m;
    ybar_f[k] = (float)m;
}

// U[k][i] = sum_j (y_jk - y_L[k]) V[j][i] / sqrt(lambda_i), in FP64 (one
// thread per entry of the d x r matrix U, row-major).
template <typename T>
__global__ void __launch_bounds__(256) k_affine_axes(const T* __restrict__ Y, int64_t ny, int d,
                                                     const int64_t* __restrict__ idx, int l,
                                                     const double* __restrict__ ybar,
                                                     const double* __restrict__ V,
                                                     const double* __restrict__ lam, int r,
                                                     double* __restrict__ U, float* __restrict__ U_f) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)d * r) return;
    const int k = (int)(e / r), i = (int)(e % r);
    const double m = ybar[k];
    double s = 0.0;
    for (int j = 0; j < l; ++j)
        s = fma(load_as<double, T>(Y + clamp_row(idx[j], ny) * d + k) - m, V[(int64_t)j * r + i], s);
    const double u = s / sqrt(lam[i]);
    U[e] = u;
    U_f[e] = (float)u;
}

// X[row] = (y_row - y_L) U: one warp per row, lanes over the columns (the
// row's loads coalesce), r accumulators per lane in the arithmetic type A,
// then one warp sum per output column.  U and y_L are small and stay in L1.
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_affine_project(const T* __restrict__ Y, int64_t n, int d,
                                                        const A* __restrict__ ybar, const A* __restrict__ U,
                                                        int r, A* __restrict__ X) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n; row += warps) {
        A acc[kMaxR];
#pragma unroll
        for (int i = 0; i < kMaxR; ++i) acc[i] = A(0);
        const T* y = Y + row * d;
        for (int k = lane; k < d; k += 32) {
            const A yc = load_as<A, T>(y + k) - ybar[k];
            const A* u = U + (int64_t)k * r;
#pragma unroll
            for (int i = 0; i < kMaxR; ++i)
                if (i < r) acc[i] = mad(yc, u[i], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < kMaxR; ++i) {
            if (i < r) {   // r is the same for the whole warp: the shuffles stay convergent
                A v = acc[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) X[row * r + i] = v;
            }
        }
    }
}

template <typename T>
cudaError_t affine_launch(const T* Y, int64_t n, int d, const int64_t* idx, int l, const double* V,
                          const double* lam, int r, int f64, double* ybar, float* ybar_f, double* U,
                          float* U_f, void* X, cudaStream_t st) {
    k_affine_mean<T><<<(unsigned)((d + 255) / 256), 256, 0, st>>>(Y, n, d, idx, l, ybar, ybar_f);
    const int64_t dr = (int64_t)d * r;
    k_affine_axes<T><<<(unsigned)((dr + 255) / 256), 256, 0, st>>>(Y, n, d, idx, l, ybar, V, lam, r, U, U_f);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 7) / 8;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
    if (f64)
        k_affine_project<T, double><<<grid, 256, 0, st>>>(Y, n, d, ybar, U, r, (double*)X);
    else
        k_affine_project<T, float><<<grid, 256, 0, st>>>(Y, n, d, ybar_f, U_f, r, (float*)X);
    note_launch(3);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_affine(const void* Y, int dt, int64_t n, int d, const int64_t* idx, int l, const double* V,
                          const double* lam, int r, int f64, double* ybar, float* ybar_f, double* U, float* U_f,
                          void* X, cudaStream_t st) {
    if (n <= 0 || d <= 0 || l <= 0 || r <= 0 || r > kMaxR) return cudaErrorInvalidValue;
    if (dt == MDS_IN_F64)
        return affine_launch((const double*)Y, n, d, idx, l, V, lam, r, f64, ybar, ybar_f, U, U_f, X, st);
    if (dt == MDS_IN_F32)
        return affine_launch((const float*)Y, n, d, idx, l, V, lam, r, f64, ybar, ybar_f, U, U_f, X, st);
    return affine_launch((const uint8_t*)Y, n, d, idx, l, V, lam, r, f64, ybar, ybar_f, U, U_f, X, st);
}

}  // namespace gbmds
