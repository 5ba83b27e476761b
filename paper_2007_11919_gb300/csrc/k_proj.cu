// Gower's interpolation formula, Eq. (2) of the paper, on CUDA cores.
//
//   Xdot = 1/(2l) (1 q_1^T - A^2) X_1 S_1^{-1},  S_1 = Lambda / l
//        = 1/2 (1 q_1^T - A^2) V Lambda^{-1/2}          (X_1 S_1^{-1} / l = V Lambda^{-1/2})
//        = A^2 W + 1 b^T,  W = -1/2 V Lambda^{-1/2},  b = 1/2 Lambda^{-1/2} V^T q_1.
//
// A^2 is never stored: each CTA computes a 64-point x 64-landmark tile of
// squared distances (norm form, clamped at 0), keeps it in shared memory and
// multiplies it into the CTA's 64 x r output accumulators.
#include <cuda_bf16.h>

#include "common.cuh"

namespace gbmds {

namespace {

__global__ void __launch_bounds__(256) k_interp_model(const double* __restrict__ V,
                                                      const double* __restrict__ lam,
                                                      const double* __restrict__ Q, int ldq,
                                                      int q_f32, int l, int r, double* w64, float* w32,
                                                      double* x1_64, float* x1_32,
                                                      double* __restrict__ bias,
                                                      double* var_out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < l * r; e += 256) {
        const int i = e % r;
        const double li = lam[i];
        const double v = V[e];
        const double w = -0.5 * v / sqrt(li);
        const double x = v * sqrt(li);
        if (w64) w64[e] = w;
        if (w32) w32[e] = (float)w;
        if (x1_64) x1_64[e] = x;
        if (x1_32) x1_32[e] = (float)x;
    }
    for (int i = warp; i < r; i += 8) {
        double s = 0.0;
        for (int a = lane; a < l; a += 32) {
            double qaa;
            if (q_f32) {
                qaa = (double)reinterpret_cast<const float*>(Q)[(int64_t)a * 2 * ldq + a];
            } else {
                qaa = Q[(int64_t)a * ldq + a];
            }
            s += V[(int64_t)a * r + i] * qaa;
        }
        s = warp_sum(s);
        if (lane == 0) {
            bias[i] = 0.5 * s / sqrt(lam[i]);
            if (var_out) var_out[i] = lam[i] / l;
        }
    }
}

// One CTA: 64 rows of Y against all l landmarks.  T: element type of Y,
// A: arithmetic type (float or double).  L is dense l x d in type A.
template <typename Ld, typename A>
__global__ void __launch_bounds__(256) k_gower(Ld Y, int64_t m, int d,
                                               const double* __restrict__ nrm_y,
                                               const A* __restrict__ L,
                                               const double* __restrict__ nrm_l, int l,
                                               const A* __restrict__ W,
                                               const double* __restrict__ bias, int r,
                                               A* __restrict__ X) {
    constexpr int KC = 16;
    constexpr int LD = kTile + 4;
    extern __shared__ __align__(16) unsigned char gsm[];
    A(*Ys)[LD] = reinterpret_cast<A(*)[LD]>(gsm);
    A(*Ls)[LD] = reinterpret_cast<A(*)[LD]>(gsm + sizeof(A) * KC * LD);
    A(*D2)[kTile + 1] = reinterpret_cast<A(*)[kTile + 1]>(gsm + sizeof(A) * 2 * KC * LD);
    A(*Ws)[kMaxR] = reinterpret_cast<A(*)[kMaxR]>(gsm + sizeof(A) * (2 * KC * LD + kTile * (kTile + 1)));

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * kTile;
    // projection mapping: point pp = tid / 4, columns c0, c0+4, ...
    const int pp = tid >> 2, c0 = tid & 3;
    A accx[kMaxR / 4];
#pragma unroll
    for (int u = 0; u < kMaxR / 4; ++u) accx[u] = 0;

    A ny[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gi = i0 + ty * 4 + i;
        ny[i] = gi < m ? (A)nrm_y[gi] : A(0);
    }

    for (int j0 = 0; j0 < l; j0 += kTile) {
        A acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[i][jj] = 0;
        for (int k0 = 0; k0 < d; k0 += KC) {
#pragma unroll
            for (int e = tid; e < kTile * KC; e += 256) {
                const int row = e / KC, kk = e % KC, k = k0 + kk;
                const int64_t gi = i0 + row;
                const int gj = j0 + row;
                Ys[kk][row] = (gi < m && k < d) ? Y.template get<A>(gi, k) : A(0);
                Ls[kk][row] = (gj < l && k < d) ? L[(int64_t)gj * d + k] : A(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                A av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    av[i] = Ys[kk][ty * 4 + i];
                    bv[i] = Ls[kk][tx * 4 + i];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[i][jj] += av[i] * bv[jj];
            }
            __syncthreads();
        }
        // squared distances of the tile -> shared memory; W chunk -> shared memory
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int gj = j0 + tx * 4 + jj;
            const A nl = gj < l ? (A)nrm_l[gj] : A(0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                A v = ny[i] + nl - A(2) * acc[i][jj];
                v = v > A(0) ? v : A(0);
                D2[ty * 4 + i][tx * 4 + jj] = gj < l ? v : A(0);
            }
        }
        for (int e = tid; e < kTile * r; e += 256) {
            const int jl = e / r, c = e % r;
            Ws[jl][c] = (j0 + jl < l) ? W[(int64_t)(j0 + jl) * r + c] : A(0);
        }
        __syncthreads();
        const int jn = min(kTile, l - j0);
        for (int jl = 0; jl < jn; ++jl) {
            const A a2 = D2[pp][jl];
#pragma unroll
            for (int u = 0; u < kMaxR / 4; ++u) {
                const int c = c0 + 4 * u;
                if (c < r) accx[u] += a2 * Ws[jl][c];
            }
        }
        __syncthreads();
    }
    const int64_t gi = i0 + pp;
    if (gi < m) {
#pragma unroll
        for (int u = 0; u < kMaxR / 4; ++u) {
            const int c = c0 + 4 * u;
            if (c < r) X[gi * r + c] = accx[u] + (A)bias[c];
        }
    }
}

template <typename A>
__global__ void k_scatter(const A* __restrict__ X1, const int64_t* __restrict__ idx, int l, int r,
                          int64_t row0, int64_t nx, A* __restrict__ X) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= l * r) return;
    const int i = e / r, c = e % r;
    const int64_t g = idx[i] - row0;
    if (g >= 0 && g < nx) X[g * r + c] = X1[e];
}

template <typename A>
__global__ void k_classical_out(const double* __restrict__ V, const double* __restrict__ lam,
                                int n, int r, A* __restrict__ X, double* lam_out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * r) X[e] = (A)(V[e] * sqrt(lam[e % r]));
    if (e < r && lam_out) lam_out[e] = lam[e];
}

}  // namespace

cudaError_t launch_interp_model(const double* V, const double* lam, const double* Q, int ldq,
                                int q_f32, int l, int r, double* w64, float* w32, double* x1_64,
                                float* x1_32, double* bias, double* var_out, cudaStream_t st) {
    k_interp_model<<<1, 256, 0, st>>>(V, lam, Q, ldq, q_f32, l, r, w64, w32, x1_64, x1_32, bias, var_out);
    note_launch(1);
    return cudaGetLastError();
}

template <typename Ld, typename A>
static cudaError_t gower_launch(Ld Y, int64_t m, int d, const double* nrm_y, const void* L,
                                const double* nrm_l, int l, const void* W, const double* bias,
                                int r, void* X, cudaStream_t st) {
    const dim3 grid((unsigned)((m + kTile - 1) / kTile)), block(256);
    const size_t smem = (2 * 16 * (kTile + 4) + kTile * (kTile + 1) + kTile * kMaxR) * sizeof(A);
    cudaError_t e = cudaFuncSetAttribute(k_gower<Ld, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gower<Ld, A><<<grid, block, smem, st>>>(Y, m, d, nrm_y, (const A*)L, nrm_l, l, (const A*)W, bias, r, (A*)X);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_gower_proj(const void* Y, int dt, int64_t m, int d, const double* nrm_y,
                              const void* L, const double* nrm_l, int l, const void* W,
                              const double* bias, int r, int acc_f64, void* X, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (acc_f64) {
        if (dt == MDS_IN_F64) return gower_launch<RowLoad<double>, double>(RowLoad<double>{(const double*)Y, d}, m, d, nrm_y, L, nrm_l, l, W, bias, r, X, st);
        if (dt == MDS_IN_F32) return gower_launch<RowLoad<float>, double>(RowLoad<float>{(const float*)Y, d}, m, d, nrm_y, L, nrm_l, l, W, bias, r, X, st);
        return gower_launch<RowLoad<uint8_t>, double>(RowLoad<uint8_t>{(const uint8_t*)Y, d}, m, d, nrm_y, L, nrm_l, l, W, bias, r, X, st);
    }
    if (dt == kDtBF16) {
        const int ld = split_ld(d);
        return gower_launch<SplitLoad, float>(SplitLoad{(const __nv_bfloat16*)Y, ld, m * ld}, m, d, nrm_y, L, nrm_l, l, W, bias, r, X, st);
    }
    if (dt == MDS_IN_F64) return gower_launch<RowLoad<double>, float>(RowLoad<double>{(const double*)Y, d}, m, d, nrm_y, L, nrm_l, l, W, bias, r, X, st);
    if (dt == MDS_IN_F32) return gower_launch<RowLoad<float>, float>(RowLoad<float>{(const float*)Y, d}, m, d, nrm_y, L, nrm_l, l, W, bias, r, X, st);
    return gower_launch<RowLoad<uint8_t>, float>(RowLoad<uint8_t>{(const uint8_t*)Y, d}, m, d, nrm_y, L, nrm_l, l, W, bias, r, X, st);
}

cudaError_t launch_scatter_rows(const void* X1, const int64_t* idx, int l, int r, int64_t nx,
                                int out_f64, void* X, cudaStream_t st) {
    const int tot = l * r;
    if (tot <= 0) return cudaSuccess;
    if (out_f64) k_scatter<double><<<(tot + 255) / 256, 256, 0, st>>>((const double*)X1, idx, l, r, 0, nx, (double*)X);
    else k_scatter<float><<<(tot + 255) / 256, 256, 0, st>>>((const float*)X1, idx, l, r, 0, nx, (float*)X);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_scatter_rows_range(const void* X1, const int64_t* idx, int l, int r, int64_t row0,
                                      int64_t rows, int out_f64, void* X, cudaStream_t st) {
    const int tot = l * r;
    if (tot <= 0 || rows <= 0) return cudaSuccess;
    if (out_f64) k_scatter<double><<<(tot + 255) / 256, 256, 0, st>>>((const double*)X1, idx, l, r, row0, rows, (double*)X);
    else k_scatter<float><<<(tot + 255) / 256, 256, 0, st>>>((const float*)X1, idx, l, r, row0, rows, (float*)X);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_classical_out(const double* V, const double* lam, int n, int r, int out_f64,
                                 void* X, double* lam_out, cudaStream_t st) {
    const int tot = n * r;
    if (out_f64) k_classical_out<double><<<(tot + 255) / 256, 256, 0, st>>>(V, lam, n, r, (double*)X, lam_out);
    else k_classical_out<float><<<(tot + 255) / 256, 256, 0, st>>>(V, lam, n, r, (float*)X, lam_out);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace gbmds
