// Pivot MDS (Section 3.1): C is the n x l block of Q = -1/2 P Delta P (all n
// points) between every point and the l pivots; its SVD C = U Sigma W^T
// approximates the eigendecomposition of Q.
//
// For rows given by coordinates Q is the Gram matrix of the rows centred at
// the mean of all n rows (Section 2), so C = Y_c P_c^T with P_c the centred
// pivot rows, and
//   C^T C = P_c S P_c^T,   S = Y_c^T Y_c  (d x d, the scatter matrix),
// an l x l problem whose top-r eigenpairs (w_i, sigma_i^2) give the left
// singular vectors u_i = C w_i / sigma_i = Y_c (P_c^T w_i / sigma_i).  So the
// whole method is: the column means and S of Y (one pass each), two small
// FP64 products for C^T C, the FP64 eigen-solver, and one more pass over Y
// for X = Y_c M, M = P_c^T W_r Sigma_r^{-1} Lambda_r^{1/2}, with the
// eigenvalue estimates lambda_i = sigma_i sqrt(n / l) (V_P^T V_P ~ (l/n) I for
// random pivots, so C C^T ~ (l/n) Q^2).  This file holds the means, the
// scatter matrix, the FP64 products, the scale factors and the sign
// convention; the projection is k_affine.cu's.
#include <algorithm>

#include "common.cuh"
#include "df.cuh"

namespace gbmds {
namespace {

constexpr int kCT = 64;      // tile edge of the scatter and product kernels
constexpr int kKC = 16;      // rows (or k) staged per step

// ---------------------------------------------------------- column means

// part[c][k] = sum of column k over the rows of chunk c: bytes exactly in
// 64-bit integers, FP32 in double-FP32, FP64 in FP64.
template <typename T>
__global__ void __launch_bounds__(128) k_colsum(const T* __restrict__ Y, int64_t n, int d, int64_t R,
                                                double* __restrict__ part) {
    const int k = blockIdx.x * 128 + threadIdx.x;
    if (k >= d) return;
    const int64_t r0 = (int64_t)blockIdx.y * R, r1 = r0 + R < n ? r0 + R : n;
    double out;
    if constexpr (sizeof(T) == 1) {
        long long s = 0;
        for (int64_t i = r0; i < r1; ++i) s += Y[i * d + k];
        out = (double)s;
    } else if constexpr (sizeof(T) == 4) {
        float h = 0.f, l = 0.f;
        for (int64_t i = r0; i < r1; ++i) df_add(h, l, Y[i * d + k], 0.f);
        out = (double)h + (double)l;
    } else {
        double s = 0.0;
        for (int64_t i = r0; i < r1; ++i) s += Y[i * d + k];
        out = s;
    }
    part[(int64_t)blockIdx.y * d + k] = out;
}

__global__ void k_colmean_final(const double* __restrict__ part, int nch, int d, int64_t n,
                                double* __restrict__ mean, float* __restrict__ mean_f) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d) return;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[(int64_t)c * d + k];
    const double m = s / (double)n;
    mean[k] = m;
    mean_f[k] = (float)m;
}

// ------------------------------------------------------- scatter matrix

// One CTA: the 64 x 64 tile (ta, tb), ta <= tb, of S = sum (y - m)(y - m)^T
// over the rows of chunk blockIdx.y, written to part[chunk][a][b].  FP32
// (float and byte rows): products summed in FP32 over 16 rows, then folded
// into double-FP32 accumulators; FP64 rows: FP64.
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_scatter_tiles(const T* __restrict__ Y, int64_t n, int d,
                                                       const double* __restrict__ mean, int64_t R, int tiles,
                                                       double* __restrict__ part) {
    __shared__ __align__(16) A As[kKC][kCT + 4];
    __shared__ __align__(16) A Bs[kKC][kCT + 4];
    __shared__ A ma[kCT], mb[kCT];
    int t = blockIdx.x;
    int ta = 0;
    while (t >= tiles - ta) {
        t -= tiles - ta;
        ++ta;
    }
    const int tb = ta + t;
    const int a0 = ta * kCT, b0 = tb * kCT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < kCT) ma[tid] = a0 + tid < d ? (A)mean[a0 + tid] : A(0);
    else if (tid < 2 * kCT) mb[tid - kCT] = b0 + tid - kCT < d ? (A)mean[b0 + tid - kCT] : A(0);
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.y * R, r1 = r0 + R < n ? r0 + R : n;
    A acc[4][4];
    float lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j] = A(0);
            lo[i][j] = 0.f;
        }
    for (int64_t rs = r0; rs < r1; rs += kKC) {
        for (int e = tid; e < kKC * kCT; e += 256) {
            const int kk = e / kCT, x = e % kCT;
            const int64_t row = rs + kk;
            const bool ok = row < r1;
            As[kk][x] = (ok && a0 + x < d) ? load_as<A, T>(Y + row * d + a0 + x) - ma[x] : A(0);
            Bs[kk][x] = (ok && b0 + x < d) ? load_as<A, T>(Y + row * d + b0 + x) - mb[x] : A(0);
        }
        __syncthreads();
        A run[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) run[i][j] = A(0);
#pragma unroll
        for (int kk = 0; kk < kKC; ++kk) {
            A av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                av[i] = As[kk][ty * 4 + i];
                bv[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) run[i][j] += av[i] * bv[j];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if constexpr (sizeof(A) == 8) {
                    acc[i][j] += run[i][j];
                } else {
                    float h = acc[i][j], l = lo[i][j];
                    df_add(h, l, run[i][j], 0.f);
                    acc[i][j] = h;
                    lo[i][j] = l;
                }
            }
        __syncthreads();
    }
    double* P = part + (int64_t)blockIdx.y * d * d;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int a = a0 + ty * 4 + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + tx * 4 + j;
            if (a < d && b < d) P[(int64_t)a * d + b] = (double)acc[i][j] + (double)lo[i][j];
        }
    }
}

// S[a][b] = sum over chunks of the tile holding (a, b) or its mirror, fixed order.
__global__ void k_scatter_final(const double* __restrict__ part, int nch, int d, double* __restrict__ S) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)d * d) return;
    int a = (int)(e / d), b = (int)(e % d);
    if (a / kCT > b / kCT) {   // lower tile: read the mirrored upper entry
        const int t = a;
        a = b;
        b = t;
    }
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[(int64_t)c * d * d + (int64_t)a * d + b];
    S[e] = s;
}

// ------------------------------------------------------------ FP64 products

// C[i][j] = sum_k (A[i][k] - ca[k]) (B[j][k] - cb[k]) (ca, cb may be null),
// A m x K (lda), B nb x K (ldb), C m x nb (ldc), FP64, 64 x 64 tiles.
__global__ void __launch_bounds__(256) k_gemm_nt(const double* __restrict__ A, int lda, const double* __restrict__ ca,
                                                 const double* __restrict__ B, int ldb, const double* __restrict__ cb,
                                                 int m, int nb, int K, double* __restrict__ C, int ldc) {
    __shared__ double As[kKC][kCT + 1];
    __shared__ double Bs[kKC][kCT + 1];
    const int i0 = blockIdx.x * kCT, j0 = blockIdx.y * kCT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kKC) {
        for (int e = tid; e < kKC * kCT; e += 256) {
            const int x = e / kKC, kk = e % kKC, k = k0 + kk;
            const int i = i0 + x, j = j0 + x;
            As[kk][x] = (i < m && k < K) ? A[(int64_t)i * lda + k] - (ca ? ca[k] : 0.0) : 0.0;
            Bs[kk][x] = (j < nb && k < K) ? B[(int64_t)j * ldb + k] - (cb ? cb[k] : 0.0) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKC; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                av[q] = As[kk][ty * 4 + q];
                bv[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[q][w] = fma(av[q], bv[w], acc[q][w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty * 4 + q;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int j = j0 + tx * 4 + w;
            if (i < m && j < nb) C[(int64_t)i * ldc + j] = acc[q][w];
        }
    }
}

// sigma_i = sqrt(mu_i) (mu: eigenvalues of C^T C), lambda_i = sigma_i sqrt(n/l),
// scale_i = sqrt(lambda_i) / sigma_i, var_i = lambda_i / n.
__global__ void k_pivot_scale(const double* __restrict__ mu, int r, int64_t n, int l, double* __restrict__ scale,
                              double* __restrict__ var) {
    const int i = threadIdx.x;
    if (i >= r) return;
    const double sg = sqrt(mu[i]);
    const double lam = sg * sqrt((double)n / (double)l);
    scale[i] = sqrt(lam) / sg;
    var[i] = lam / (double)n;
}

// ------------------------------------------------------- sign convention

constexpr int kSgThreads = 256;

// Per column of X (n x r): the entry of largest magnitude (lowest row on a
// tie); the last CTA to finish sets sign[i] = -1 where that entry is
// negative, else +1, and re-arms the counter.
template <typename A>
__global__ void __launch_bounds__(kSgThreads) k_colsign(const A* __restrict__ X, int64_t n, int r,
                                                        double* __restrict__ part_v, int64_t* __restrict__ part_i,
                                                        unsigned* __restrict__ counter, double* __restrict__ sign) {
    __shared__ double sv[kSgThreads];
    __shared__ int64_t si[kSgThreads];
    __shared__ bool last;
    for (int i = 0; i < r; ++i) {
        double bv = -1.0;
        int64_t bi = INT64_MAX;
        for (int64_t row = (int64_t)blockIdx.x * kSgThreads + threadIdx.x; row < n;
             row += (int64_t)gridDim.x * kSgThreads) {
            const double v = fabs((double)X[row * r + i]);
            if (v > bv || (v == bv && row < bi)) {
                bv = v;
                bi = row;
            }
        }
        sv[threadIdx.x] = bv;
        si[threadIdx.x] = bi;
        __syncthreads();
        for (int h = kSgThreads / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) {
                const double w = sv[threadIdx.x + h];
                const int64_t j = si[threadIdx.x + h];
                if (w > sv[threadIdx.x] || (w == sv[threadIdx.x] && j < si[threadIdx.x])) {
                    sv[threadIdx.x] = w;
                    si[threadIdx.x] = j;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part_v[(int64_t)blockIdx.x * r + i] = sv[0];
            part_i[(int64_t)blockIdx.x * r + i] = si[0];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= r) return;
    __threadfence();
    const int i = threadIdx.x;
    double bv = -1.0;
    int64_t bi = INT64_MAX;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        const double w = __ldcg(part_v + (int64_t)b * r + i);
        const int64_t j = __ldcg(part_i + (int64_t)b * r + i);
        if (w > bv || (w == bv && j < bi)) {
            bv = w;
            bi = j;
        }
    }
    sign[i] = (bi < n && X[bi * r + i] < A(0)) ? -1.0 : 1.0;
    if (i == 0) *counter = 0u;
}

template <typename A>
__global__ void k_colscale(A* __restrict__ X, int64_t n, int r, const double* __restrict__ sign) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * r) X[e] = X[e] * (A)sign[e % r];
}

}  // namespace

int64_t colsum_chunk_rows(int64_t n) { return n < 4096 ? (n > 0 ? n : 1) : 4096; }

int64_t scatter_chunk_rows(int64_t n, int d) {
    // at most ~32 MiB of FP64 partial tiles, at least 8192 rows per chunk
    const int64_t maxch = std::max<int64_t>(1, (int64_t)(4u << 20) / ((int64_t)d * d));
    int64_t nch = std::min<int64_t>(maxch, (n + 8191) / 8192);
    nch = std::max<int64_t>(1, nch);
    return (n + nch - 1) / nch;
}

cudaError_t launch_colmean(const void* Y, int dt, int64_t n, int d, double* part, double* mean, float* mean_f,
                           cudaStream_t st) {
    if (n <= 0 || d <= 0) return cudaErrorInvalidValue;
    const int64_t R = colsum_chunk_rows(n);
    const int nch = (int)((n + R - 1) / R);
    const dim3 grid((unsigned)((d + 127) / 128), (unsigned)nch);
    if (dt == MDS_IN_F64) k_colsum<double><<<grid, 128, 0, st>>>((const double*)Y, n, d, R, part);
    else if (dt == MDS_IN_F32) k_colsum<float><<<grid, 128, 0, st>>>((const float*)Y, n, d, R, part);
    else k_colsum<uint8_t><<<grid, 128, 0, st>>>((const uint8_t*)Y, n, d, R, part);
    k_colmean_final<<<(d + 255) / 256, 256, 0, st>>>(part, nch, d, n, mean, mean_f);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const void* Y, int dt, int64_t n, int d, const double* mean, int f64, double* part,
                           double* S, cudaStream_t st) {
    if (n <= 0 || d <= 0) return cudaErrorInvalidValue;
    const int64_t R = scatter_chunk_rows(n, d);
    const int nch = (int)((n + R - 1) / R);
    const int tiles = (d + kCT - 1) / kCT;
    const dim3 grid((unsigned)(tiles * (tiles + 1) / 2), (unsigned)nch);
    if (dt == MDS_IN_F64) {
        if (f64) k_scatter_tiles<double, double><<<grid, 256, 0, st>>>((const double*)Y, n, d, mean, R, tiles, part);
        else k_scatter_tiles<double, float><<<grid, 256, 0, st>>>((const double*)Y, n, d, mean, R, tiles, part);
    } else if (dt == MDS_IN_F32) {
        if (f64) k_scatter_tiles<float, double><<<grid, 256, 0, st>>>((const float*)Y, n, d, mean, R, tiles, part);
        else k_scatter_tiles<float, float><<<grid, 256, 0, st>>>((const float*)Y, n, d, mean, R, tiles, part);
    } else {
        if (f64) k_scatter_tiles<uint8_t, double><<<grid, 256, 0, st>>>((const uint8_t*)Y, n, d, mean, R, tiles, part);
        else k_scatter_tiles<uint8_t, float><<<grid, 256, 0, st>>>((const uint8_t*)Y, n, d, mean, R, tiles, part);
    }
    const int64_t dd = (int64_t)d * d;
    k_scatter_final<<<(unsigned)((dd + 255) / 256), 256, 0, st>>>(part, nch, d, S);
    note_launch(2);
    return cudaGetLastError();
}

size_t scatter_part_doubles(int64_t n, int d) {
    const int64_t R = scatter_chunk_rows(n, d);
    return (size_t)((n + R - 1) / R) * d * d;
}

size_t colmean_part_doubles(int64_t n, int d) {
    const int64_t R = colsum_chunk_rows(n);
    return (size_t)((n + R - 1) / R) * d;
}

cudaError_t launch_gemm_nt(const double* A, int lda, const double* ca, const double* B, int ldb, const double* cb,
                           int m, int nb, int K, double* C, int ldc, cudaStream_t st) {
    if (m <= 0 || nb <= 0 || K <= 0) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((m + kCT - 1) / kCT), (unsigned)((nb + kCT - 1) / kCT));
    k_gemm_nt<<<grid, 256, 0, st>>>(A, lda, ca, B, ldb, cb, m, nb, K, C, ldc);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pivot_scale(const double* mu, int r, int64_t n, int l, double* scale, double* var,
                               cudaStream_t st) {
    k_pivot_scale<<<1, 32, 0, st>>>(mu, r, n, l, scale, var);
    note_launch(1);
    return cudaGetLastError();
}

int colsign_grid(int64_t n) {
    const int64_t g = (n + kSgThreads - 1) / kSgThreads;
    return (int)(g < 1024 ? (g > 0 ? g : 1) : 1024);
}

cudaError_t launch_colsign(void* X, int out_f64, int64_t n, int r, double* part_v, int64_t* part_i, unsigned* counter,
                           double* sign, cudaStream_t st) {
    if (n <= 0 || r <= 0 || r > kMaxR) return cudaErrorInvalidValue;
    const int grid = colsign_grid(n);
    const unsigned g2 = (unsigned)((n * r + 255) / 256);
    if (out_f64) {
        k_colsign<double><<<grid, kSgThreads, 0, st>>>((const double*)X, n, r, part_v, part_i, counter, sign);
        k_colscale<double><<<g2, 256, 0, st>>>((double*)X, n, r, sign);
    } else {
        k_colsign<float><<<grid, kSgThreads, 0, st>>>((const float*)X, n, r, part_v, part_i, counter, sign);
        k_colscale<float><<<g2, 256, 0, st>>>((float*)X, n, r, sign);
    }
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace gbmds
