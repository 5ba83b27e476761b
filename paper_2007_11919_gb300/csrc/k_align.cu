// Divide-and-conquer alignment (Section 3.2 of the paper).
//
// Part j (j >= 1) is mapped onto part 0 by orthogonal Procrustes on the c
// connecting points (rows 0..c-1 of every part): find T_j orthogonal and t_j
// with X_0^c ~ X_j^c T_j + 1 t_j^T.  Centre both point sets,
// C = B_c^T A_c (r x r, B = X_j^c, A = X_0^c), C = U Sigma W^T (one-sided
// Jacobi SVD, FP64), T = U W^T, t = a_bar - T^T b_bar.  Reflections are
// allowed and there is no dilation.  Rows of part j other than the connecting
// points then receive X_j^a T_j + 1 t_j^T; part 0 keeps X_0 whole.  The
// eigenvalue estimate is lambda_bar_i = (1/p) sum_j lambda_i^j / n_j.
#include "common.cuh"

namespace gbmds {
namespace {

// One CTA per part.  The one-sided Jacobi sweeps rotate disjoint column pairs
// concurrently in round-robin order (r - 1 rounds of r / 2 pairs per sweep,
// the circle method).  A pair is a group of r lanes (lane q of the group owns
// row q) and a warp holds floor(32 / r) groups, so a round of r = 10 takes
// two warps instead of five: GB300 issues FP64 at 1/64 of FP32 and every FP64
// warp instruction costs the same however few of its lanes work.  FP64
// throughout.
constexpr int kProcThreads = 512;   // 16 warps: enough for r / 2 <= 16 pairs at one pair per warp

// Sum of v over the r lanes of this lane's group (lane q of group g is lane
// g r + q), returned in every lane of the group: a tree into the group's
// first lane (offsets 16, 8, ... below r, added where q + offset < r), then
// a broadcast.  Every lane of the warp calls it.
__device__ __forceinline__ double group_sum(double v, int q, int r, int leader) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (o < r) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            if (q + o < r) v += w;
        }
    }
    return __shfl_sync(0xffffffffu, v, leader);
}

__device__ __forceinline__ void round_robin_pair(int round, int k, int n, int& p, int& q) {
    int x, y;
    if (k == 0) {
        x = round;
        y = n - 1;
    } else {
        x = (round + k) % (n - 1);
        y = (round - k + (n - 1)) % (n - 1);
    }
    p = x < y ? x : y;
    q = x < y ? y : x;
}

// The orthogonal factor of Procrustes from C = B_c^T A_c (r x r in G, W
// the identity in Wm, both in shared memory): one-sided Jacobi on G until its
// columns are orthogonal, U = G's columns normalised (null directions
// completed by Gram-Schmidt), T = U W^T, t = a_bar - T^T b_bar.  Called by
// every thread of a CTA of kProcThreads; T and t are written by warp 0.
__device__ void procrustes_polar(double (*G)[kMaxR + 1], double (*Wm)[kMaxR + 1], const double* abar,
                                 const double* bbar, int r, double* __restrict__ T, double* __restrict__ t) {
    __shared__ int s_rot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // one-sided Jacobi: rotate column pairs of G (and W) until orthogonal
    const int rr = r + (r & 1);   // column r is a dummy when r is odd
    const int gpw = 32 / r;       // pairs (lane groups) per warp
    const int gi = lane / r, row = lane - gi * r;
    const int pair = warp * gpw + gi;
    const bool in_group = gi < gpw && pair < rr / 2;
    const int leader = gi < gpw ? gi * r : 0;
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int round = 0; round < rr - 1; ++round) {
            if (warp * gpw < rr / 2) {   // warps holding a pair (the same for every lane of the warp)
                int p = 0, q = 0;
                if (in_group) round_robin_pair(round, pair, rr, p, q);
                const bool real = in_group && q < r;
                const double gp = real ? G[row][p] : 0.0;
                const double gq = real ? G[row][q] : 0.0;
                const double al = group_sum(gp * gp, row, r, leader);
                const double be = group_sum(gq * gq, row, r, leader);
                const double ga = group_sum(gp * gq, row, r, leader);
                if (real && fabs(ga) > 1e-15 * sqrt(al * be) && ga != 0.0) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double cs = 1.0 / sqrt(1.0 + tt * tt);
                    const double sn = cs * tt;
                    G[row][p] = cs * gp - sn * gq;
                    G[row][q] = sn * gp + cs * gq;
                    const double wp = Wm[row][p], wq = Wm[row][q];
                    Wm[row][p] = cs * wp - sn * wq;
                    Wm[row][q] = sn * wp + cs * wq;
                    if (row == 0) s_rot = 1;
                }
            }
            __syncthreads();
        }
        const bool again = s_rot != 0;
        __syncthreads();   // every thread has read the flag before it is reset
        if (!again) break;
    }
    if (warp != 0) return;
    // U columns = G columns / sigma; complete null directions by Gram-Schmidt
    double smax = 0.0;
    for (int m = 0; m < r; ++m) {
        const double g = lane < r ? G[lane][m] : 0.0;
        smax = fmax(smax, sqrt(warp_sum(g * g)));
    }
    int unit = 0;
    for (int m = 0; m < r; ++m) {
        const double g = lane < r ? G[lane][m] : 0.0;
        const double sg = sqrt(warp_sum(g * g));
        if (sg > 1e-13 * smax && sg > 0.0) {
            if (lane < r) G[lane][m] = g / sg;
        } else {
            // a unit vector orthogonal to the other (already normalised or later) columns
            for (; unit < r; ++unit) {
                double v = lane == unit ? 1.0 : 0.0;
                for (int o = 0; o < r; ++o) {
                    if (o == m) continue;
                    const double go = lane < r ? G[lane][o] : 0.0;
                    const double no = warp_sum(go * go);
                    if (no == 0.0) continue;
                    v -= warp_sum(go * v) / no * go;
                }
                const double nv = sqrt(warp_sum(v * v));
                if (nv > 1e-6) {
                    if (lane < r) G[lane][m] = v / nv;
                    ++unit;
                    break;
                }
            }
        }
        __syncwarp();
    }
    // T = U W^T ; t = abar - T^T bbar
    if (lane < r) {
        for (int m = 0; m < r; ++m) {
            double s = 0.0;
            for (int k = 0; k < r; ++k) s += G[lane][k] * Wm[m][k];
            T[lane * r + m] = s;
        }
    }
    __syncwarp();
    if (lane < r) {
        double s = 0.0;
        for (int i = 0; i < r; ++i) s += T[i * r + lane] * bbar[i];
        t[lane] = abar[lane] - s;
    }
}

__global__ void __launch_bounds__(kProcThreads) k_procrustes(const ProbDesc* __restrict__ desc,
                                                             const double* __restrict__ varena,
                                                             const double* __restrict__ lam, int r, int c,
                                                             double* __restrict__ Tt) {
    __shared__ double G[kMaxR][kMaxR + 1];
    __shared__ double Wm[kMaxR][kMaxR + 1];
    __shared__ double abar[kMaxR], bbar[kMaxR], sq0[kMaxR], sqj[kMaxR];
    const int j = blockIdx.x;
    const int tid = threadIdx.x;
    double* T = Tt + (size_t)j * (r * r + r);
    double* t = T + r * r;
    if (j == 0) {
        for (int e = tid; e < r * r; e += kProcThreads) T[e] = (e / r == e % r) ? 1.0 : 0.0;
        if (tid < r) t[tid] = 0.0;
        return;
    }
    const double* V0 = varena + desc[0].v_off;
    const double* Vj = varena + desc[j].v_off;
    if (tid < r) {
        sq0[tid] = sqrt(lam[tid]);
        sqj[tid] = sqrt(lam[(size_t)j * r + tid]);
    }
    __syncthreads();
    if (tid < r) {
        double sa = 0.0, sb = 0.0;
        for (int a = 0; a < c; ++a) {
            sa += V0[(int64_t)a * r + tid] * sq0[tid];
            sb += Vj[(int64_t)a * r + tid] * sqj[tid];
        }
        abar[tid] = sa / c;
        bbar[tid] = sb / c;
    }
    __syncthreads();
    // C[i][m] = sum_a (B_ai - bbar_i)(A_am - abar_m), one thread per entry
    for (int e = tid; e < r * r; e += kProcThreads) {
        const int i = e / r, m = e % r;
        double s = 0.0;
        for (int a = 0; a < c; ++a) {
            const double b = Vj[(int64_t)a * r + i] * sqj[i] - bbar[i];
            const double av = V0[(int64_t)a * r + m] * sq0[m] - abar[m];
            s += b * av;
        }
        G[i][m] = s;
        Wm[i][m] = (i == m) ? 1.0 : 0.0;
    }
    __syncthreads();
    procrustes_polar(G, Wm, abar, bbar, r, T, t);
}

// Procrustes of point sets given as matrices: task k aligns B_k onto A_k
// (each c x r row-major at AB + k * 2 c r, A then B), A ~ B T + 1 t^T, into
// Tt + dst[k] * (r r + r).
__global__ void __launch_bounds__(kProcThreads) k_procrustes_sets(const double* __restrict__ AB, int c, int r,
                                                                  const int* __restrict__ dst,
                                                                  double* __restrict__ Tt) {
    __shared__ double G[kMaxR][kMaxR + 1];
    __shared__ double Wm[kMaxR][kMaxR + 1];
    __shared__ double abar[kMaxR], bbar[kMaxR];
    const int tid = threadIdx.x;
    const double* A = AB + (size_t)blockIdx.x * 2 * c * r;
    const double* B = A + (size_t)c * r;
    double* T = Tt + (size_t)dst[blockIdx.x] * (r * r + r);
    double* t = T + r * r;
    if (tid < r) {
        double sa = 0.0, sb = 0.0;
        for (int a = 0; a < c; ++a) {
            sa += A[(int64_t)a * r + tid];
            sb += B[(int64_t)a * r + tid];
        }
        abar[tid] = sa / c;
        bbar[tid] = sb / c;
    }
    __syncthreads();
    for (int e = tid; e < r * r; e += kProcThreads) {
        const int i = e / r, m = e % r;
        double s = 0.0;
        for (int a = 0; a < c; ++a) s += (B[(int64_t)a * r + i] - bbar[i]) * (A[(int64_t)a * r + m] - abar[m]);
        G[i][m] = s;
        Wm[i][m] = (i == m) ? 1.0 : 0.0;
    }
    __syncthreads();
    procrustes_polar(G, Wm, abar, bbar, r, T, t);
}

template <typename A>
__global__ void __launch_bounds__(256) k_align(const ProbDesc* __restrict__ desc,
                                               const double* __restrict__ varena,
                                               const double* __restrict__ lam,
                                               const double* __restrict__ Tt, int r,
                                               const int64_t* __restrict__ anchors,
                                               const int64_t* __restrict__ own,
                                               A* __restrict__ X) {
    const int j = blockIdx.y;
    const ProbDesc P = desc[j];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= P.n) return;
    if (j > 0 && a < P.c) return;  // connecting points come from part 0
    const double* V = varena + P.v_off + (int64_t)a * r;
    const double* T = Tt + (size_t)j * (r * r + r);
    const double* t = T + r * r;
    double x[kMaxR];
#pragma unroll
    for (int m = 0; m < kMaxR; ++m)
        if (m < r) x[m] = V[m] * sqrt(lam[(size_t)j * r + m]);
    const int64_t row = member_row(P, anchors, own, a);
    for (int i = 0; i < r; ++i) {
        double s = t[i];
#pragma unroll
        for (int m = 0; m < kMaxR; ++m)
            if (m < r) s += x[m] * T[m * r + i];
        X[row * r + i] = (A)s;
    }
}

// var_i = (1/p) sum_j lambda^j_i / n_j: warp i, lanes over the problems, a
// fixed butterfly sum (deterministic; the quotients are independent, so a
// batch of thousands of problems is not one long chain of FP64 divisions).
__global__ void k_lambda_bar(const ProbDesc* __restrict__ desc, int p,
                             const double* __restrict__ lam, int r, double* __restrict__ var) {
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (i >= r) return;
    double s = 0.0;
    for (int j = lane; j < p; j += 32) s += lam[(size_t)j * r + i] / desc[j].n;
    s = warp_sum(s);
    if (lane == 0) var[i] = s / p;
}

}  // namespace

cudaError_t launch_dc_procrustes(const ProbDesc* desc, int p, const double* varena,
                                 const double* lam, int r, int c, double* Tt, cudaStream_t st) {
    k_procrustes<<<p, kProcThreads, 0, st>>>(desc, varena, lam, r, c, Tt);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_procrustes_sets(const double* AB, int tasks, int c, int r, const int* dst, double* Tt,
                                   cudaStream_t st) {
    if (tasks <= 0) return cudaSuccess;
    k_procrustes_sets<<<tasks, kProcThreads, 0, st>>>(AB, c, r, dst, Tt);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_dc_align(const ProbDesc* desc, int p, int max_n, const double* varena,
                            const double* lam, const double* Tt, int r, const int64_t* anchors,
                            const int64_t* own, int out_f64, void* X, cudaStream_t st) {
    const dim3 grid((unsigned)((max_n + 255) / 256), (unsigned)p);
    if (out_f64) k_align<double><<<grid, 256, 0, st>>>(desc, varena, lam, Tt, r, anchors, own, (double*)X);
    else k_align<float><<<grid, 256, 0, st>>>(desc, varena, lam, Tt, r, anchors, own, (float*)X);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_dc_lambda_bar(const ProbDesc* desc, int p, const double* lam, int r,
                                 double* var, cudaStream_t st) {
    if (r <= 0 || r > kMaxR) return cudaErrorInvalidValue;
    k_lambda_bar<<<1, 32 * r, 0, st>>>(desc, p, lam, r, var);
    note_launch(1);
    return cudaGetLastError();
}

}  // namespace gbmds
