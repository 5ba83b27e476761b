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
// 64-bit integers, FP32 in double-FP32, FP64 in FP64.  Thread per column,
// eight rows loaded ahead of their sums.
template <typename T>
__global__ void __launch_bounds__(128) k_colsum(const T* __restrict__ Y, int64_t n, int d, int64_t R,
                                                double* __restrict__ part) {
    const int k = blockIdx.x * 128 + threadIdx.x;
    if (k >= d) return;
    const int64_t r0 = (int64_t)blockIdx.y * R, r1 = r0 + R < n ? r0 + R : n;
    constexpr int U = 8;
    double out;
    if constexpr (sizeof(T) == 1) {
        long long s = 0;
        for (int64_t i = r0; i < r1; ++i) s += Y[i * d + k];
        out = (double)s;
    } else if constexpr (sizeof(T) == 4) {
        float h = 0.f, l = 0.f;
        int64_t i = r0;
        for (; i + U <= r1; i += U) {
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = Y[(i + u) * d + k];
#pragma unroll
            for (int u = 0; u < U; ++u) df_add(h, l, v[u], 0.f);
        }
        for (; i < r1; ++i) df_add(h, l, Y[i * d + k], 0.f);
        out = (double)h + (double)l;
    } else {
        double s = 0.0;
        for (int64_t i = r0; i < r1; ++i) s += Y[i * d + k];
        out = s;
    }
    part[(int64_t)blockIdx.y * d + k] = out;
}

// Warp per column: the chunks' sums in a fixed order (lane-strided, then a
// fixed tree).
__global__ void k_colmean_final(const double* __restrict__ part, int nch, int d, int64_t n,
                                double* __restrict__ mean, float* __restrict__ mean_f) {
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= d) return;
    double s = 0.0;
    for (int c = lane; c < nch; c += 32) s += part[(int64_t)c * d + k];
    s = warp_sum(s);
    if (lane == 0) {
        const double m = s / (double)n;
        mean[k] = m;
        mean_f[k] = (float)m;
    }
}

// ------------------------------------------------------- scatter matrix

// S = sum over rows of (y - m)(y - m)^T, upper triangle of 4 x 4 blocks:
// thread-tile t is block (bi, bj), bi <= bj, numbered row by row over the
// nb = ceil(d / 4) block rows, so the products cover the triangle and little
// else.  One CTA: thread-tiles [blockIdx.x * blockDim.x, ...) over the rows
// of chunk blockIdx.y, kc rows at a time: the rows are centred into shared
// memory (each thread's share of the next kc rows is loaded into registers
// while the current ones are multiplied), then each thread takes its two
// 16-byte column groups per row.  FP32 (float and byte rows): products summed
// in FP32 over 32 rows, then folded into double-FP32 accumulators; FP64:
// FP64 sums.  part[chunk][t * 16 + 4 i + j] = block entry (4 bi + i, 4 bj + j).
constexpr int kScPre = 8;   // staged elements per thread and step

template <typename T, typename A>
__global__ void __launch_bounds__(512) k_scatter_tri(const T* __restrict__ Y, int64_t n, int d,
                                                     const double* __restrict__ mean, int64_t R, int nt, int kc,
                                                     double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char sc_raw[];
    A* const Ys = reinterpret_cast<A*>(sc_raw);   // kc x dp centred rows (zero past d and past the chunk)
    const int dp = (d + 3) & ~3, nb = dp >> 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < nt;
    int bi = 0, rem = active ? t : 0;
    while (rem >= nb - bi) {
        rem -= nb - bi;
        ++bi;
    }
    const int bj = bi + rem;
    const int64_t r0 = (int64_t)blockIdx.y * R, r1 = r0 + R < n ? r0 + R : n;
    // this thread's staged elements: e = tid + blockDim * u < kc * dp -> (row e / dp, column e % dp)
    const int ne = kc * dp;
    int erow[kScPre], ecol[kScPre];
#pragma unroll
    for (int u = 0; u < kScPre; ++u) {
        const int e = threadIdx.x + (int)blockDim.x * u;
        erow[u] = e < ne ? e / dp : -1;
        ecol[u] = e < ne ? e - (e / dp) * dp : 0;
    }
    A pre[kScPre];
    auto fetch = [&](int64_t rs) {
#pragma unroll
        for (int u = 0; u < kScPre; ++u) {
            const int64_t row = rs + erow[u];
            pre[u] = (erow[u] >= 0 && row < r1 && ecol[u] < d)
                         ? load_as<A, T>(Y + row * d + ecol[u]) - (A)__ldg(mean + ecol[u])
                         : A(0);
        }
    };
    A acc[4][4], run[4][4];
    float lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j] = A(0);
            run[i][j] = A(0);
            lo[i][j] = 0.f;
        }
    fetch(r0);
    int since = 0;   // rows summed into run since the last fold
    for (int64_t rs = r0; rs < r1; rs += kc) {
#pragma unroll
        for (int u = 0; u < kScPre; ++u)
            if (erow[u] >= 0) Ys[erow[u] * dp + ecol[u]] = pre[u];
        __syncthreads();
        if (rs + kc < r1) fetch(rs + kc);
        if (active) {
            for (int kk = 0; kk < kc; ++kk) {
                A av[4], bv[4];
                const A* row = Ys + kk * dp;
                if constexpr (sizeof(A) == 4) {
                    const float4 a4 = *reinterpret_cast<const float4*>(row + 4 * bi);
                    const float4 b4 = *reinterpret_cast<const float4*>(row + 4 * bj);
                    av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
                    bv[0] = b4.x; bv[1] = b4.y; bv[2] = b4.z; bv[3] = b4.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        av[i] = row[4 * bi + i];
                        bv[i] = row[4 * bj + i];
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) run[i][j] += av[i] * bv[j];
            }
            since += kc;
            if constexpr (sizeof(A) == 4) {
                if (since >= 32 || rs + kc >= r1) {   // fold every 32 rows or so (and at the end)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            float h = acc[i][j], l = lo[i][j];
                            df_add(h, l, run[i][j], 0.f);
                            acc[i][j] = h;
                            lo[i][j] = l;
                            run[i][j] = A(0);
                        }
                    since = 0;
                }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    double* P = part + ((int64_t)blockIdx.y * nt + t) * 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            P[4 * i + j] = sizeof(A) == 8 ? (double)run[i][j] : (double)acc[i][j] + (double)lo[i][j];
}

// The same computation for FP32 rows in FP32 and FP64 rows in FP64 (element
// type = arithmetic type), with the rows staged by cp.async into a ring of
// kScStages steps instead of through registers: the copies of the next two
// steps are in flight while a step is multiplied, and each thread centres its
// own staged elements in place once they have landed (the register form
// waited on its loads at every step).  Same products, same order, same
// results as k_scatter_tri.
constexpr int kScStages = 3;

template <int B>
__device__ __forceinline__ void sc_cp_async(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(B) : "memory");
}

template <typename T>
__global__ void __launch_bounds__(512) k_scatter_tri_async(const T* __restrict__ Y, int64_t n, int d,
                                                           const double* __restrict__ mean, int64_t R, int nt, int kc,
                                                           double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char sc_raw[];
    const int dp = (d + 3) & ~3, nb = dp >> 2, ne = kc * dp;
    T* const ring = reinterpret_cast<T*>(sc_raw);   // kScStages x kc x dp rows, centred in place
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < nt;
    int bi = 0, rem = active ? t : 0;
    while (rem >= nb - bi) {
        rem -= nb - bi;
        ++bi;
    }
    const int bj = bi + rem;
    const int64_t r0 = (int64_t)blockIdx.y * R, r1 = r0 + R < n ? r0 + R : n;
    const int nsteps = (int)((r1 - r0 + kc - 1) / kc);
    int erow[kScPre], ecol[kScPre];
#pragma unroll
    for (int u = 0; u < kScPre; ++u) {
        const int e = threadIdx.x + (int)blockDim.x * u;
        erow[u] = e < ne ? e / dp : -1;
        ecol[u] = e < ne ? e - (e / dp) * dp : 0;
    }
    auto issue = [&](int s) {   // step s's rows into stage s % kScStages (zero past d and past the chunk)
        if (s < nsteps) {
            T* stg = ring + (size_t)(s % kScStages) * ne;
            const int64_t rs = r0 + (int64_t)s * kc;
#pragma unroll
            for (int u = 0; u < kScPre; ++u) {
                if (erow[u] < 0) continue;
                const int64_t row = rs + erow[u];
                T* dst = stg + erow[u] * dp + ecol[u];
                if (row < r1 && ecol[u] < d) sc_cp_async<(int)sizeof(T)>(dst, Y + row * d + ecol[u]);
                else *dst = T(0);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(0);
    issue(1);
    T acc[4][4], run[4][4];
    float lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j] = T(0);
            run[i][j] = T(0);
            lo[i][j] = 0.f;
        }
    int since = 0;
    for (int s = 0; s < nsteps; ++s) {
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // this thread's copies of step s
        T* const stg = ring + (size_t)(s % kScStages) * ne;
        const int64_t rs = r0 + (int64_t)s * kc;
#pragma unroll
        for (int u = 0; u < kScPre; ++u)
            if (erow[u] >= 0 && ecol[u] < d && rs + erow[u] < r1)
                stg[erow[u] * dp + ecol[u]] -= (T)__ldg(mean + ecol[u]);
        __syncthreads();   // step s centred; every thread is past step s - 1
        issue(s + 2);      // its stage was last read at step s - 1
        if (active) {
            for (int kk = 0; kk < kc; ++kk) {
                T av[4], bv[4];
                const T* row = stg + kk * dp;
                if constexpr (sizeof(T) == 4) {
                    const float4 a4 = *reinterpret_cast<const float4*>(row + 4 * bi);
                    const float4 b4 = *reinterpret_cast<const float4*>(row + 4 * bj);
                    av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
                    bv[0] = b4.x; bv[1] = b4.y; bv[2] = b4.z; bv[3] = b4.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        av[i] = row[4 * bi + i];
                        bv[i] = row[4 * bj + i];
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) run[i][j] += av[i] * bv[j];
            }
            since += kc;
            if constexpr (sizeof(T) == 4) {
                if (since >= 32 || rs + kc >= r1) {   // fold every 32 rows or so (and at the end)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            float h = acc[i][j], l = lo[i][j];
                            df_add(h, l, run[i][j], 0.f);
                            acc[i][j] = h;
                            lo[i][j] = l;
                            run[i][j] = T(0);
                        }
                    since = 0;
                }
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!active) return;
    double* P = part + ((int64_t)blockIdx.y * nt + t) * 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            P[4 * i + j] = sizeof(T) == 8 ? (double)run[i][j] : (double)acc[i][j] + (double)lo[i][j];
}

// Warp per entry (a, b), a <= b, of S: the chunks' partials in a fixed order
// (lane-strided, then a fixed tree), written to S[a][b] and S[b][a].
__global__ void k_scatter_final(const double* __restrict__ part, int nch, int nt, int d, double* __restrict__ S) {
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)d * d) return;
    const int a = (int)(w / d), b = (int)(w % d);
    if (a > b) return;
    const int nb = ((d + 3) & ~3) >> 2, bi = a >> 2, bj = b >> 2;
    const int64_t t = (int64_t)bi * nb - (int64_t)bi * (bi - 1) / 2 + (bj - bi);
    const int64_t off = t * 16 + 4 * (a & 3) + (b & 3);
    double s = 0.0;
    for (int c = lane; c < nch; c += 32) s += part[(int64_t)c * nt * 16 + off];
    s = warp_sum(s);
    if (lane == 0) {
        S[(int64_t)a * d + b] = s;
        S[(int64_t)b * d + a] = s;
    }
}

// ------------------------------------------------------------ FP64 products

// C[i][j] = sum_k (A[i][k] - ca[k]) (B[j][k] - cb[k]) (ca, cb may be null),
// A m x K (lda), B nb x K (ldb), C m x nb (ldc), FP64, 64 x 64 tiles.
// With sym the product is known to be symmetric (m == nb): only the tiles
// (ti, tj), ti <= tj, are computed (blockIdx.x numbers them row by row) and
// each is written to both triangles, so C is exactly symmetric.
__global__ void __launch_bounds__(256) k_gemm_nt(const double* __restrict__ A, int lda, const double* __restrict__ ca,
                                                 const double* __restrict__ B, int ldb, const double* __restrict__ cb,
                                                 int m, int nb, int K, double* __restrict__ C, int ldc, int sym) {
    __shared__ double As[kKC][kCT + 1];
    __shared__ double Bs[kKC][kCT + 1];
    int ti = blockIdx.x, tj = blockIdx.y;
    if (sym) {
        const int nt = (m + kCT - 1) / kCT;
        int rem = blockIdx.x;
        ti = 0;
        while (rem >= nt - ti) {
            rem -= nt - ti;
            ++ti;
        }
        tj = ti + rem;
    }
    const int i0 = ti * kCT, j0 = tj * kCT;
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
            if (i < m && j < nb) {
                C[(int64_t)i * ldc + j] = acc[q][w];
                if (sym) C[(int64_t)j * ldc + i] = acc[q][w];
            }
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
// tie), in one coalesced pass over X: element e (row e / r, column e % r) is
// read by thread e mod S of the grid, S = the grid's threads rounded down to
// a multiple of r, so each thread meets one column only and keeps its best;
// thread i < r of each CTA combines the CTA's threads of column i.  The last
// CTA to finish sets sign[i] = -1 where that entry is negative, else +1, and
// re-arms the counter.  The order of the comparisons does not matter: the
// winner is the largest (|x|, -row).
template <typename A>
__global__ void __launch_bounds__(kSgThreads) k_colsign(const A* __restrict__ X, int64_t n, int r,
                                                        double* __restrict__ part_v, int64_t* __restrict__ part_i,
                                                        unsigned* __restrict__ counter, double* __restrict__ sign) {
    __shared__ double sv[kSgThreads];
    __shared__ int64_t si[kSgThreads];
    __shared__ bool last;
    const int64_t q = (int64_t)gridDim.x * kSgThreads / r, S = q * r;
    const int64_t e0 = (int64_t)blockIdx.x * kSgThreads + threadIdx.x;
    double bv = -1.0;
    int64_t bi = INT64_MAX;
    if (e0 < S) {
        int64_t row = e0 / r;
        for (int64_t e = e0; e < n * r; e += S, row += q) {
            const double v = fabs((double)X[e]);
            if (v > bv || (v == bv && row < bi)) {
                bv = v;
                bi = row;
            }
        }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x < r) {
        const int i = threadIdx.x;
        const int t0 = (int)((((int64_t)i - (int64_t)blockIdx.x * kSgThreads) % r + r) % r);
        double cv = -1.0;
        int64_t ci = INT64_MAX;
        for (int t = t0; t < kSgThreads; t += r) {
            const double w = sv[t];
            const int64_t j = si[t];
            if (w > cv || (w == cv && j < ci)) {
                cv = w;
                ci = j;
            }
        }
        part_v[(int64_t)blockIdx.x * r + i] = cv;
        part_i[(int64_t)blockIdx.x * r + i] = ci;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // warp w takes the columns w, w + 8, ...: lanes stride over the CTAs'
    // partials, then a shuffle tree
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < r; i += kSgThreads / 32) {
        double cv = -1.0;
        int64_t ci = INT64_MAX;
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            const double w = __ldcg(part_v + (int64_t)b * r + i);
            const int64_t j = __ldcg(part_i + (int64_t)b * r + i);
            if (w > cv || (w == cv && j < ci)) {
                cv = w;
                ci = j;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, cv, o);
            const int64_t j = __shfl_xor_sync(0xffffffffu, ci, o);
            if (w > cv || (w == cv && j < ci)) {
                cv = w;
                ci = j;
            }
        }
        if (lane == 0) sign[i] = (ci < n && X[ci * r + i] < A(0)) ? -1.0 : 1.0;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

template <typename A>
__global__ void k_colscale(A* __restrict__ X, int64_t n, int r, const double* __restrict__ sign) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * r) X[e] = X[e] * (A)sign[e % r];
}

}  // namespace

int64_t colsum_chunk_rows(int64_t n) { return n < 512 ? (n > 0 ? n : 1) : 512; }

// Geometry of the scatter matrix's triangle kernel: nt thread-tiles in ncta
// CTAs of `threads`, kc rows per step, nch chunks of R rows (about 608 CTAs
// in all, at most 64 MiB of partials, at least 256 rows per chunk).
struct ScatterGeo {
    int nt, ncta, threads, kc, nch;
    int64_t R;
};

static bool scatter_geo(int64_t n, int d, ScatterGeo& g) {
    const int dp = (d + 3) & ~3, nb = dp / 4;
    g.nt = nb * (nb + 1) / 2;
    g.ncta = (g.nt + 511) / 512;
    g.threads = (int)round_up((g.nt + g.ncta - 1) / g.ncta, 32);
    g.kc = std::min(32, kScPre * g.threads / dp);
    if (g.kc < 1) return false;
    const int64_t maxch = std::max<int64_t>(1, (int64_t)(8u << 20) / ((int64_t)g.nt * 16));
    int64_t nch = std::max<int64_t>(1, (608 + g.ncta - 1) / g.ncta);
    nch = std::min<int64_t>(nch, std::min<int64_t>(maxch, (n + 255) / 256));
    nch = std::max<int64_t>(1, nch);
    g.R = (n + nch - 1) / nch;
    g.nch = (int)((n + g.R - 1) / g.R);
    return true;
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
    k_colmean_final<<<(d + 7) / 8, 256, 0, st>>>(part, nch, d, n, mean, mean_f);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const void* Y, int dt, int64_t n, int d, const double* mean, int f64, double* part,
                           double* S, cudaStream_t st) {
    ScatterGeo g;
    if (n <= 0 || d <= 0 || !scatter_geo(n, d, g)) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)g.ncta, (unsigned)g.nch);
    const int dp = (d + 3) & ~3;
    const size_t smem = (size_t)g.kc * dp * (f64 ? 8 : 4);
    if ((dt == MDS_IN_F64 && f64) || (dt == MDS_IN_F32 && !f64)) {
        // element type = arithmetic type: rows staged by cp.async
        const size_t sm = (size_t)kScStages * g.kc * dp * (f64 ? 8 : 4);
        auto go = [&](auto kern, auto* y) {
            cudaError_t e = cudaSuccess;
            if (sm > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e == cudaSuccess) kern<<<grid, g.threads, sm, st>>>(y, n, d, mean, g.R, g.nt, g.kc, part);
            return e;
        };
        const cudaError_t e = f64 ? go(k_scatter_tri_async<double>, (const double*)Y)
                                  : go(k_scatter_tri_async<float>, (const float*)Y);
        if (e != cudaSuccess) return e;
    } else if (dt == MDS_IN_F64) {
        if (f64) k_scatter_tri<double, double><<<grid, g.threads, smem, st>>>((const double*)Y, n, d, mean, g.R, g.nt, g.kc, part);
        else k_scatter_tri<double, float><<<grid, g.threads, smem, st>>>((const double*)Y, n, d, mean, g.R, g.nt, g.kc, part);
    } else if (dt == MDS_IN_F32) {
        if (f64) k_scatter_tri<float, double><<<grid, g.threads, smem, st>>>((const float*)Y, n, d, mean, g.R, g.nt, g.kc, part);
        else k_scatter_tri<float, float><<<grid, g.threads, smem, st>>>((const float*)Y, n, d, mean, g.R, g.nt, g.kc, part);
    } else {
        if (f64) k_scatter_tri<uint8_t, double><<<grid, g.threads, smem, st>>>((const uint8_t*)Y, n, d, mean, g.R, g.nt, g.kc, part);
        else k_scatter_tri<uint8_t, float><<<grid, g.threads, smem, st>>>((const uint8_t*)Y, n, d, mean, g.R, g.nt, g.kc, part);
    }
    const int64_t dd = (int64_t)d * d;
    k_scatter_final<<<(unsigned)((dd + 7) / 8), 256, 0, st>>>(part, g.nch, g.nt, d, S);
    note_launch(2);
    return cudaGetLastError();
}

size_t scatter_part_doubles(int64_t n, int d) {
    ScatterGeo g;
    if (n <= 0 || d <= 0 || !scatter_geo(n, d, g)) return 0;
    return (size_t)g.nch * g.nt * 16;
}

bool scatter_supported(int d) {
    ScatterGeo g;
    return d > 0 && scatter_geo(1, d, g);
}

size_t colmean_part_doubles(int64_t n, int d) {
    const int64_t R = colsum_chunk_rows(n);
    return (size_t)((n + R - 1) / R) * d;
}

cudaError_t launch_gemm_nt(const double* A, int lda, const double* ca, const double* B, int ldb, const double* cb,
                           int m, int nb, int K, double* C, int ldc, int sym, cudaStream_t st) {
    if (m <= 0 || nb <= 0 || K <= 0 || (sym && m != nb)) return cudaErrorInvalidValue;
    const int tm = (m + kCT - 1) / kCT;
    const dim3 grid = sym ? dim3((unsigned)(tm * (tm + 1) / 2), 1u) : dim3((unsigned)tm, (unsigned)((nb + kCT - 1) / kCT));
    k_gemm_nt<<<grid, 256, 0, st>>>(A, lda, ca, B, ldb, cb, m, nb, K, C, ldc, sym);
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
