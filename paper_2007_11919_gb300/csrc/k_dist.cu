// Row norms, batched squared-distance tiles and double centering.
//
// Section 2 of the paper: for Euclidean rows y_i, d^2_ij = q_ii + q_jj - 2 q_ij,
// here d^2_ij = ||y_i||^2 + ||y_j||^2 - 2 y_i . y_j (norm form, clamped at 0,
// exact 0 on the diagonal), and Q = -1/2 P Delta P, i.e.
// q_ij = -(d2_ij - d2_i. - d2_.j + d2_..)/2 with row / column / grand means.
#include <cuda_bf16.h>

#include "common.cuh"
#include "df.cuh"

namespace gbmds {

namespace {

// ------------------------------------------------------------------ norms

// Squared norms of rows 0..n-1, or, with idx, of rows idx[0..n-1] (each
// clamped to 0..ny-1) written at their own positions nrm[idx[i]].
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_rownorm(const T* __restrict__ Y, int64_t n, int d,
                                                 double* __restrict__ nrm,
                                                 const int64_t* __restrict__ idx, int64_t ny) {
    const int lane = threadIdx.x & 31;
    int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= n) return;
    if (idx) {
        row = idx[row];
        row = row < 0 ? 0 : (row >= ny ? ny - 1 : row);
    }
    const T* y = Y + row * (int64_t)d;
    A s = 0;
    for (int k = lane; k < d; k += 32) {
        A v = load_as<A, T>(y + k);
        s += v * v;
    }
    s = warp_sum(s);
    if (lane == 0) nrm[row] = (double)s;
}

// ------------------------------------------------------- distance tiles
// One CTA = one 64 x 64 tile (rows a0.., columns b0..) of Delta_j for problem
// blockIdx.y, on or above the diagonal (tb >= ta): Delta is symmetric, so a
// tile off the diagonal is written twice, as itself and as its transpose, from
// the same values.  256 threads, 4 x 4 outputs each; K staged through shared
// memory 16 at a time.  Writes Delta as FP64 (row-major, ld = ldq) or,
// accumulating in FP32, as FP32 at the start of each row's storage (row stride
// 2 * ldq floats), and each tile's row sums into rp[tb * n + a] (the mirrored
// tile's into rp[ta * n + b], from the tile's column sums; all summed later in
// a fixed order).  O64 writes Delta as FP64 whatever the accumulation type
// (FP32 dot products feeding an FP64 eigenproblem).

template <typename T, typename A, bool O64>
__global__ void __launch_bounds__(256) k_sqdist(const T* __restrict__ Y, int d,
                                                const double* __restrict__ nrm,
                                                const int64_t* __restrict__ anchors,
                                                const int64_t* __restrict__ own,
                                                const ProbDesc* __restrict__ desc,
                                                double* __restrict__ qarena,
                                                double* __restrict__ rparena) {
    constexpr int KC = 16;
    constexpr int LD = kTile + 4;
    __shared__ __align__(16) A As[KC][LD];
    __shared__ __align__(16) A Bs[KC][LD];
    __shared__ int64_t rowA[kTile], rowB[kTile];
    // column sums of the tile by row group: [ty][column] (double-FP32 pairs as
    // float2 for FP32 accumulation)
    __shared__ __align__(16) double csum[16][kTile];

    const ProbDesc P = desc[blockIdx.y];
    const int n = P.n;
    int t = blockIdx.x;
    if (t >= P.tiles * (P.tiles + 1) / 2) return;
    int ta = 0;
    while (t >= P.tiles - ta) {   // t -> (ta, tb), tb >= ta, row-major over the upper triangle
        t -= P.tiles - ta;
        ++ta;
    }
    const int tb = ta + t;
    const int a0 = ta * kTile, b0 = tb * kTile;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;

    if (tid < kTile) {
        const int a = a0 + tid;
        rowA[tid] = a < n ? member_row(P, anchors, own, a) : -1;
    } else if (tid < 2 * kTile) {
        const int b = b0 + tid - kTile;
        rowB[tid - kTile] = b < n ? member_row(P, anchors, own, b) : -1;
    }
    __syncthreads();

    A acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = 0;

    // this thread's staged elements of a chunk (fixed): e = tid + 256 u -> row e / KC, column e % KC;
    // the next chunk's are loaded into registers while the current one is multiplied
    constexpr int kPer = kTile * KC / 256;
    A pa[kPer], pb[kPer];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int e = tid + 256 * u, row = e / KC, k = k0 + e % KC;
            const int64_t ga = rowA[row], gb = rowB[row];
            pa[u] = (ga >= 0 && k < d) ? load_as<A, T>(Y + ga * d + k) : A(0);
            pb[u] = (gb >= 0 && k < d) ? load_as<A, T>(Y + gb * d + k) : A(0);
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < d; k0 += KC) {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int e = tid + 256 * u, row = e / KC, kk = e % KC;
            As[kk][row] = pa[u];
            Bs[kk][row] = pb[u];
        }
        __syncthreads();
        if (k0 + KC < d) fetch(k0 + KC);
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            A av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                av[i] = As[kk][ty * 4 + i];
                bv[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] += av[i] * bv[jj];
        }
        __syncthreads();
    }

    double* Q = qarena + P.q_off;
    double* rp = rparena + P.rp_off;
    A nb[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) nb[jj] = b0 + tx * 4 + jj < n ? (A)nrm[rowB[tx * 4 + jj]] : A(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int a = a0 + ty * 4 + i;
        if constexpr (O64) {
            double rs = 0.0;
            if (a < n) {
                const A na = (A)nrm[rowA[ty * 4 + i]];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int b = b0 + tx * 4 + jj;
                    if (b < n) {
                        A dist = na + nb[jj] - A(2) * acc[i][jj];
                        dist = dist > A(0) ? dist : A(0);
                        if (a == b) dist = A(0);
                        Q[(int64_t)a * P.ldq + b] = (double)dist;
                        rs += (double)dist;
                    }
                }
            }
            // sum over the 16 column-threads of this row (same warp, lanes xor 1..8)
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
            if (tx == 0 && a < n) rp[(int64_t)tb * n + a] = rs;
        } else {
            // FP32: Delta as floats at the start of each row's storage (row
            // stride 2 * ldq floats); tile row sums in double-FP32
            float* Qf = reinterpret_cast<float*>(Q);
            float rh = 0.f, rl = 0.f;
            if (a < n) {
                const float na = (float)nrm[rowA[ty * 4 + i]];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int b = b0 + tx * 4 + jj;
                    if (b < n) {
                        float dist = na + nb[jj] - 2.f * acc[i][jj];
                        dist = dist > 0.f ? dist : 0.f;
                        if (a == b) dist = 0.f;
                        Qf[(int64_t)a * 2 * P.ldq + b] = dist;
                        df_add(rh, rl, dist, 0.f);
                    }
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, rh, o);
                const float ol = __shfl_xor_sync(0xffffffffu, rl, o);
                df_add(rh, rl, oh, ol);
            }
            if (tx == 0 && a < n) rp[(int64_t)tb * n + a] = (double)rh + (double)rl;
        }
    }
    if (ta == tb) return;

    // ---- the mirrored tile: Delta[b][a] = Delta[a][b], and the row sums of
    // rows b over this tile's columns a (the tile's column sums: each thread's
    // four rows, then the sixteen row groups in order)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        const int b = b0 + tx * 4 + jj;
        if constexpr (O64) {
            double cs = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int a = a0 + ty * 4 + i;
                if (a < n && b < n) {
                    A dist = (A)nrm[rowA[ty * 4 + i]] + nb[jj] - A(2) * acc[i][jj];
                    dist = dist > A(0) ? dist : A(0);
                    Q[(int64_t)b * P.ldq + a] = (double)dist;
                    cs += (double)dist;
                }
            }
            csum[ty][tx * 4 + jj] = cs;
        } else {
            float* Qf = reinterpret_cast<float*>(Q);
            float ch = 0.f, cl = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int a = a0 + ty * 4 + i;
                if (a < n && b < n) {
                    float dist = (float)nrm[rowA[ty * 4 + i]] + nb[jj] - 2.f * acc[i][jj];
                    dist = dist > 0.f ? dist : 0.f;
                    Qf[(int64_t)b * 2 * P.ldq + a] = dist;
                    df_add(ch, cl, dist, 0.f);
                }
            }
            reinterpret_cast<float2*>(&csum[ty][0])[tx * 4 + jj] = make_float2(ch, cl);
        }
    }
    __syncthreads();
    if (tid < kTile) {
        const int b = b0 + tid;
        if (b < n) {
            if constexpr (O64) {
                double s = 0.0;
                for (int g = 0; g < 16; ++g) s += csum[g][tid];
                rp[(int64_t)ta * n + b] = s;
            } else {
                float sh = 0.f, sl = 0.f;
                for (int g = 0; g < 16; ++g) {
                    const float2 c = reinterpret_cast<const float2*>(&csum[g][0])[tid];
                    df_add(sh, sl, c.x, c.y);
                }
                rp[(int64_t)ta * n + b] = (double)sh + (double)sl;
            }
        }
    }
}

// Copy an external squared-distance matrix into Q's slot with tile row sums.
__global__ void __launch_bounds__(256) k_load_dist(const double* __restrict__ D2,
                                                   const ProbDesc* __restrict__ desc,
                                                   double* __restrict__ qarena,
                                                   double* __restrict__ rparena) {
    const ProbDesc P = desc[0];
    const int n = P.n;
    const int a = blockIdx.x;
    if (a >= n) return;
    __shared__ double red[8];
    double* Q = qarena + P.q_off + (int64_t)a * P.ldq;
    const double* src = D2 + (int64_t)a * n;
    double* rp = rparena + P.rp_off;
    for (int tb = 0; tb < P.tiles; ++tb) {
        const int b = tb * kTile + (threadIdx.x & 63);
        double v = 0.0;
        if (threadIdx.x < kTile && b < n) {
            v = src[b];
            Q[b] = v;
        }
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) rp[(int64_t)tb * n + a] = red[0] + red[1];
        __syncthreads();
    }
}

// ------------------------------------------------------------ centering

// Row means m_a (FP64, from the tile row sums in a fixed order) and the
// grand mean g.  F32: m is stored as double-FP32 pairs for k_center.
template <bool F32>
__global__ void __launch_bounds__(256) k_rowmean(const ProbDesc* __restrict__ desc,
                                                 const double* __restrict__ rparena,
                                                 double* __restrict__ rmarena,
                                                 double* __restrict__ grand) {
    const ProbDesc P = desc[blockIdx.x];
    const int n = P.n;
    const double* rp = rparena + P.rp_off;
    double* rm = rmarena + P.rm_off;
    __shared__ double red[8];
    double loc = 0.0;
    for (int a = threadIdx.x; a < n; a += 256) {
        double s = 0.0;
        for (int tb = 0; tb < P.tiles; ++tb) s += rp[(int64_t)tb * n + a];
        const double m = s / n;
        if (F32) reinterpret_cast<float2*>(rm)[a] = df_of(m);
        else rm[a] = m;
        loc += m;
    }
    loc = warp_sum(loc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        grand[blockIdx.x] = s / n;
    }
}

// Q = -1/2 P Delta P in place, row a of part blockIdx.y.  F32: the row is
// rewritten as n floats at the start of its own storage (zero-padded to a
// multiple of 4), chunk by chunk: a chunk's floats overlap only doubles of
// chunks already read, and the whole chunk is read before any of it is written.
template <bool F32>
__global__ void __launch_bounds__(256) k_center(const ProbDesc* __restrict__ desc,
                                                double* __restrict__ qarena,
                                                const double* __restrict__ rmarena,
                                                const double* __restrict__ grand) {
    const ProbDesc P = desc[blockIdx.y];
    const int a = blockIdx.x;
    if (a >= P.n) return;
    const double* rm = rmarena + P.rm_off;
    const double g = grand[blockIdx.y];
    double* Q = qarena + P.q_off + (int64_t)a * P.ldq;
    if (F32) {
        // Delta (floats, in place) -> Q = -1/2 (Delta - (m_a - g) - m_b) in
        // double-FP32, rounded once to FP32; padding entries set to zero
        float* Qf = reinterpret_cast<float*>(Q);
        const float2* md = reinterpret_cast<const float2*>(rm);
        const float2 ma = md[a];
        const float2 cag = df_sub2(ma, df_of(g));
        const int n4 = (int)round_up(P.n, 4);
        for (int b = threadIdx.x; b < n4; b += 256) {
            float qv = 0.f;
            if (b < P.n) {
                const float2 mb = md[b];
                float ch = cag.x, cl = cag.y;
                df_add(ch, cl, mb.x, mb.y);          // c = m_a - g + m_b
                float dh = Qf[b], dl = 0.f;
                df_add(dh, dl, -ch, -cl);            // Delta - c
                qv = -0.5f * __fadd_rn(dh, dl);
            }
            Qf[b] = qv;
        }
    } else {
        const double ma = rm[a];
        for (int b = threadIdx.x; b < P.n; b += 256) Q[b] = -0.5 * (Q[b] - ma - rm[b] + g);
    }
}

// The FP32 form of k_center with one warp per row and eight rows per CTA
// (a part's rows are short: ~1,000 entries), four entries per lane and step
// with 16-byte loads and stores of the row; the same arithmetic per entry.
__device__ __forceinline__ float center_entry(float d, float2 cag, float2 mb) {
    float ch = cag.x, cl = cag.y;
    df_add(ch, cl, mb.x, mb.y);          // c = m_a - g + m_b
    float dh = d, dl = 0.f;
    df_add(dh, dl, -ch, -cl);            // Delta - c
    return -0.5f * __fadd_rn(dh, dl);
}

__global__ void __launch_bounds__(256) k_center_rows(const ProbDesc* __restrict__ desc,
                                                     double* __restrict__ qarena,
                                                     const double* __restrict__ rmarena,
                                                     const double* __restrict__ grand) {
    const ProbDesc P = desc[blockIdx.y];
    const int a = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (a >= P.n) return;
    const float2* md = reinterpret_cast<const float2*>(rmarena + P.rm_off);
    float4* Q4 = reinterpret_cast<float4*>(qarena + P.q_off + (int64_t)a * P.ldq);
    const float2 cag = df_sub2(md[a], df_of(grand[blockIdx.y]));
    const int n = P.n, n4 = (int)round_up(n, 4) / 4;
    for (int b4 = lane; b4 < n4; b4 += 32) {
        const float4 x = Q4[b4];
        const int b = 4 * b4;
        float4 q;
        q.x = b < n ? center_entry(x.x, cag, md[b]) : 0.f;
        q.y = b + 1 < n ? center_entry(x.y, cag, md[b + 1]) : 0.f;
        q.z = b + 2 < n ? center_entry(x.z, cag, md[b + 2]) : 0.f;
        q.w = b + 3 < n ? center_entry(x.w, cag, md[b + 3]) : 0.f;
        Q4[b4] = q;
    }
}

__global__ void k_check_idx(const int64_t* __restrict__ idx, int64_t count, int64_t ny,
                            int* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count && (idx[i] < 0 || idx[i] >= ny)) atomicOr(flag, 1);
}

__global__ void k_iota(int64_t* __restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i;
}

template <typename T>
__global__ void __launch_bounds__(256) k_quant_bf16(const T* __restrict__ Y, int64_t n, int d,
                                                    __nv_bfloat16* __restrict__ Yq, int64_t row0, int64_t nplane,
                                                    double* __restrict__ nrm) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= n) return;
    const int ld = split_ld(d);
    __nv_bfloat16* hi = Yq + (row0 + row) * ld;
    __nv_bfloat16* lo = hi + nplane * (int64_t)ld;
    float s = 0.f;
    for (int k = lane; k < ld; k += 32) {
        const float y = k < d ? (float)Y[row * d + k] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(y);
        const float hf = __bfloat162float(h);
        const __nv_bfloat16 l = __float2bfloat16_rn(y - hf);
        hi[k] = h;
        lo[k] = l;
        const float lf = __bfloat162float(l);
        s += hf * hf + 2.f * hf * lf;
    }
    s = warp_sum(s);
    if (lane == 0) nrm[row0 + row] = (double)s;
}

// The same split for FP32 rows with d a multiple of 4 and a 16-byte aligned
// base: float4 loads (streamed, the rows are read once), 8-byte stores of four
// BF16 values.  split_ld(d) - d is then 0 or 4, one zero group.
__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__global__ void __launch_bounds__(256) k_quant_bf16_f4(const float* __restrict__ Y, int64_t n, int d,
                                                       __nv_bfloat16* __restrict__ Yq, int64_t row0, int64_t nplane,
                                                       double* __restrict__ nrm) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= n) return;
    const int ld = split_ld(d);
    const float4* y4 = reinterpret_cast<const float4*>(Y + row * d);
    uint2* hi = reinterpret_cast<uint2*>(Yq + (row0 + row) * ld);
    uint2* lo = reinterpret_cast<uint2*>(Yq + nplane * (int64_t)ld + (row0 + row) * ld);
    float s = 0.f;
    for (int k4 = lane; k4 < ld / 4; k4 += 32) {
        const float4 v = k4 < d / 4 ? __ldcs(y4 + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float y[4] = {v.x, v.y, v.z, v.w};
        __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = __float2bfloat16_rn(y[e]);
            const float hf = __bfloat162float(h[e]);
            l[e] = __float2bfloat16_rn(y[e] - hf);
            s += hf * hf + 2.f * hf * __bfloat162float(l[e]);
        }
        hi[k4] = make_uint2(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]));
        lo[k4] = make_uint2(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]));
    }
    s = warp_sum(s);
    if (lane == 0) nrm[row0 + row] = (double)s;
}

template <typename Ld, typename A>
__global__ void __launch_bounds__(256) k_gather(Ld Y, int d,
                                                const int64_t* __restrict__ idx, int l,
                                                int64_t ny, A* __restrict__ out,
                                                const double* __restrict__ nrm_src,
                                                double* __restrict__ nrm_out) {
    const int i = blockIdx.x;
    if (i >= l) return;
    int64_t g = idx[i];
    g = g < 0 ? 0 : (g >= ny ? ny - 1 : g);
    for (int k = threadIdx.x; k < d; k += blockDim.x) out[(int64_t)i * d + k] = Y.template get<A>(g, k);
    if (threadIdx.x == 0 && nrm_out) nrm_out[i] = nrm_src[g];
}

}  // namespace

static cudaError_t rownorm_any(const void* Y, int dt, int64_t n, int d, int acc_f64, double* nrm,
                               const int64_t* idx, int64_t ny, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 7) / 8)), block(256);
    if (acc_f64) {
        if (dt == MDS_IN_F64) k_rownorm<double, double><<<grid, block, 0, st>>>((const double*)Y, n, d, nrm, idx, ny);
        else if (dt == MDS_IN_F32) k_rownorm<float, double><<<grid, block, 0, st>>>((const float*)Y, n, d, nrm, idx, ny);
        else k_rownorm<uint8_t, double><<<grid, block, 0, st>>>((const uint8_t*)Y, n, d, nrm, idx, ny);
    } else {
        if (dt == MDS_IN_F64) k_rownorm<double, float><<<grid, block, 0, st>>>((const double*)Y, n, d, nrm, idx, ny);
        else if (dt == MDS_IN_F32) k_rownorm<float, float><<<grid, block, 0, st>>>((const float*)Y, n, d, nrm, idx, ny);
        else k_rownorm<uint8_t, float><<<grid, block, 0, st>>>((const uint8_t*)Y, n, d, nrm, idx, ny);
    }
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_rownorm(const void* Y, int dt, int64_t n, int d, int acc_f64, double* nrm,
                           cudaStream_t st) {
    return rownorm_any(Y, dt, n, d, acc_f64, nrm, nullptr, n, st);
}

cudaError_t launch_rownorm_idx(const void* Y, int dt, int64_t ny, int d, const int64_t* idx, int64_t count,
                               int acc_f64, double* nrm, cudaStream_t st) {
    return rownorm_any(Y, dt, count, d, acc_f64, nrm, idx, ny, st);
}

template <typename T>
static void sqdist_any(const T* Y, int d, const double* nrm, const int64_t* anchors, const int64_t* own,
                       const ProbDesc* desc, int acc_f64, int out_f64, double* qarena, double* rparena, dim3 grid,
                       cudaStream_t st) {
    if (acc_f64) k_sqdist<T, double, true><<<grid, 256, 0, st>>>(Y, d, nrm, anchors, own, desc, qarena, rparena);
    else if (out_f64) k_sqdist<T, float, true><<<grid, 256, 0, st>>>(Y, d, nrm, anchors, own, desc, qarena, rparena);
    else k_sqdist<T, float, false><<<grid, 256, 0, st>>>(Y, d, nrm, anchors, own, desc, qarena, rparena);
}

cudaError_t launch_sqdist_batched(const void* Y, int dt, int d, const double* nrm,
                                  const int64_t* anchors, const int64_t* own,
                                  const ProbDesc* desc, int p, int max_tiles, int acc_f64, int out_f64,
                                  double* qarena, double* rparena, cudaStream_t st) {
    if (p <= 0) return cudaSuccess;
    const dim3 grid((unsigned)(max_tiles * (max_tiles + 1) / 2), (unsigned)p);
    if (dt == MDS_IN_F64)
        sqdist_any((const double*)Y, d, nrm, anchors, own, desc, acc_f64, out_f64, qarena, rparena, grid, st);
    else if (dt == MDS_IN_F32)
        sqdist_any((const float*)Y, d, nrm, anchors, own, desc, acc_f64, out_f64, qarena, rparena, grid, st);
    else
        sqdist_any((const uint8_t*)Y, d, nrm, anchors, own, desc, acc_f64, out_f64, qarena, rparena, grid, st);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_load_dist(const double* D2, const ProbDesc* desc, double* qarena,
                             double* rparena, int n, int tiles, cudaStream_t st) {
    (void)tiles;
    k_load_dist<<<n, 256, 0, st>>>(D2, desc, qarena, rparena);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_center_batched(const ProbDesc* desc, int p, int max_n, double* qarena,
                                  const double* rparena, double* rmarena, double* grand, int q_f32,
                                  cudaStream_t st) {
    if (p <= 0) return cudaSuccess;
    if (q_f32) k_rowmean<true><<<p, 256, 0, st>>>(desc, rparena, rmarena, grand);
    else k_rowmean<false><<<p, 256, 0, st>>>(desc, rparena, rmarena, grand);
    if (q_f32) k_center_rows<<<dim3((unsigned)((max_n + 7) / 8), (unsigned)p), 256, 0, st>>>(desc, qarena, rmarena, grand);
    else k_center<false><<<dim3((unsigned)max_n, (unsigned)p), 256, 0, st>>>(desc, qarena, rmarena, grand);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const void* Y, int dt, int64_t ny, int d, const int64_t* idx,
                               int l, int acc_f64, void* out, const double* nrm_src,
                               double* nrm_out, cudaStream_t st) {
    if (l <= 0) return cudaSuccess;
    if (acc_f64) {
        double* o = (double*)out;
        if (dt == MDS_IN_F64) k_gather<<<l, 128, 0, st>>>(RowLoad<double>{(const double*)Y, d}, d, idx, l, ny, o, nrm_src, nrm_out);
        else if (dt == MDS_IN_F32) k_gather<<<l, 128, 0, st>>>(RowLoad<float>{(const float*)Y, d}, d, idx, l, ny, o, nrm_src, nrm_out);
        else k_gather<<<l, 128, 0, st>>>(RowLoad<uint8_t>{(const uint8_t*)Y, d}, d, idx, l, ny, o, nrm_src, nrm_out);
    } else {
        float* o = (float*)out;
        if (dt == kDtBF16) {
            const int ld = split_ld(d);
            k_gather<<<l, 128, 0, st>>>(SplitLoad{(const __nv_bfloat16*)Y, ld, ny * ld}, d, idx, l, ny, o, nrm_src, nrm_out);
        } else if (dt == MDS_IN_F64) k_gather<<<l, 128, 0, st>>>(RowLoad<double>{(const double*)Y, d}, d, idx, l, ny, o, nrm_src, nrm_out);
        else if (dt == MDS_IN_F32) k_gather<<<l, 128, 0, st>>>(RowLoad<float>{(const float*)Y, d}, d, idx, l, ny, o, nrm_src, nrm_out);
        else k_gather<<<l, 128, 0, st>>>(RowLoad<uint8_t>{(const uint8_t*)Y, d}, d, idx, l, ny, o, nrm_src, nrm_out);
    }
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_check_idx(const int64_t* idx, int64_t count, int64_t ny, int* flag,
                             cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_check_idx<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(idx, count, ny, flag);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_iota(int64_t* out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_iota<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_quant_bf16_rows(const void* Y, int dt, int64_t rows, int d, void* Yq, int64_t row0,
                                   int64_t nplane, double* nrm, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((rows + 7) / 8));
    __nv_bfloat16* q = (__nv_bfloat16*)Yq;
    if (dt == MDS_IN_F64) k_quant_bf16<double><<<grid, 256, 0, st>>>((const double*)Y, rows, d, q, row0, nplane, nrm);
    else if (dt == MDS_IN_F32 && d % 4 == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0)
        k_quant_bf16_f4<<<grid, 256, 0, st>>>((const float*)Y, rows, d, q, row0, nplane, nrm);
    else if (dt == MDS_IN_F32) k_quant_bf16<float><<<grid, 256, 0, st>>>((const float*)Y, rows, d, q, row0, nplane, nrm);
    else k_quant_bf16<uint8_t><<<grid, 256, 0, st>>>((const uint8_t*)Y, rows, d, q, row0, nplane, nrm);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_quant_bf16(const void* Y, int dt, int64_t n, int d, void* Yq, double* nrm,
                              cudaStream_t st) {
    return launch_quant_bf16_rows(Y, dt, n, d, Yq, 0, n, nrm, st);
}

}  // namespace gbmds
