// Batched top-r symmetric eigen-solver in FP64: Lanczos with full
// re-orthogonalisation, one thread-block cluster per eigenproblem.
//
// The paper computes the classical-MDS eigenpairs of each l x l matrix Q with a
// Lanczos method (Section 2, the svd package's trlan.eigen); steps 2-3 of
// classical MDS keep the r largest eigenvalues and their eigenvectors.  Here:
//
//   Krylov basis v_0, v_1, ... of Q from a fixed pseudo-random start vector;
//   w = Q v_j, two passes of classical Gram-Schmidt against all previous
//   vectors, alpha_j = v_j . Q v_j, beta_j = ||w||, v_{j+1} = w / beta_j.
//   The Rayleigh quotient T_k = V_k^T Q V_k is the tridiagonal of the alphas
//   and betas.  Every few steps the r largest eigenvalues theta_i of T_k are
//   found by Sturm-count multisection, and the Ritz residuals
//   ||Q y_i - theta_i y_i|| = beta_{k-1} |s_{k-1,i}| from the last component of
//   T_k's eigenvector (an O(k) recurrence of the characteristic polynomial and
//   its derivative: s_k^2 = -p_{k-1}(theta) / p_k'(theta)).  The run stops when
//   every residual is below tol * theta_0, at an invariant subspace (beta ~ 0),
//   or at the step cap (status NOCONV).  Eigenvectors s_i of T_k come from
//   inverse iteration (tridiagonal LU with partial pivoting), Ritz vectors
//   are y_i = V_k s_i.
//
// Layout: Q_j row-major FP64 (ld = ldq).  The cluster's CTAs own contiguous
// row slices; each CTA's slice of the current Lanczos vector lives in its
// shared memory and is gathered through distributed shared memory; dot
// products are reduced across the cluster through DSMEM in rank order, so
// every CTA holds bitwise-identical scalars and takes identical decisions.
#include <cooperative_groups.h>
#include <float.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace gbmds {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct Smem {
    double* vfull;   // max_n     : full current Lanczos vector
    double* vloc;    // rmax      : this CTA's slice of v_j
    double* wloc;    // rmax      : this CTA's slice of w
    double* part0;   // mmax + 2  : partial sums published to the cluster
    double* part1;   // mmax + 2
    double* cfull;   // mmax + 2  : reduced coefficients
    double* alpha;   // mmax + 1
    double* beta;    // mmax + 1
    double* beta2;   // mmax + 1
    double* theta;   // kMaxR
    double* resid;   // kMaxR
    double* red;     // 3 * kWarps * ... scratch (64)
    double* sgn;     // 3 * kMaxR : (|max|, row, signed) per eigenvector
};

__host__ __device__ inline size_t smem_doubles(int max_n, int cs, int mmax) {
    const size_t rmax = (size_t)((max_n + cs - 1) / cs);
    return round_up(max_n, 2) + 2 * round_up(rmax, 2) + 3 * (size_t)(mmax + 2) +
           3 * (size_t)(mmax + 1) + 2 * kMaxR + 64 + 3 * kMaxR + 8;
}

__device__ Smem carve(double* base, int max_n, int cs, int mmax) {
    Smem s;
    const int rmax = (max_n + cs - 1) / cs;
    double* p = base;
    s.vfull = p; p += round_up(max_n, 2);
    s.vloc = p; p += round_up(rmax, 2);
    s.wloc = p; p += round_up(rmax, 2);
    s.part0 = p; p += mmax + 2;
    s.part1 = p; p += mmax + 2;
    s.cfull = p; p += mmax + 2;
    s.alpha = p; p += mmax + 1;
    s.beta = p; p += mmax + 1;
    s.beta2 = p; p += mmax + 1;
    s.theta = p; p += kMaxR;
    s.resid = p; p += kMaxR;
    s.red = p; p += 64;
    s.sgn = p; p += 3 * kMaxR;
    return s;
}

// Sum of one value per thread over the CTA, in a fixed order.  Result valid
// in thread 0.  Contains __syncthreads.
__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kWarps; ++i) s += red[i];
    return s;
}

// out[i] = sum over cluster ranks (in rank order) of part[i], i < K.
__device__ void cluster_allreduce(cg::cluster_group& cl, double* part, double* out, int K, int cs) {
    cl.sync();
    for (int i = threadIdx.x; i < K; i += kThreads) {
        double s = 0.0;
        for (int qq = 0; qq < cs; ++qq) s += cl.map_shared_rank(part, qq)[i];
        out[i] = s;
    }
    __syncthreads();
}

// Number of eigenvalues of T (alpha, beta^2) smaller than x.
__device__ int sturm_count(const double* al, const double* b2, int k, double x, double pivmin) {
    int c = 0;
    double dd = al[0] - x;
    if (fabs(dd) < pivmin) dd = -pivmin;
    if (dd < 0.0) ++c;
    for (int t = 1; t < k; ++t) {
        dd = (al[t] - x) - b2[t - 1] / dd;
        if (fabs(dd) < pivmin) dd = -pivmin;
        if (dd < 0.0) ++c;
    }
    return c;
}

// Squared last component of the unit eigenvector of T for eigenvalue x:
// s_k^2 = -p_{k-1}(x) / p_k'(x), through d_t = p_t/p_{t-1} and
// g_t = p_t'/p_{t-1}.
__device__ double last_comp2(const double* al, const double* b2, int k, double x, double pivmin) {
    if (k == 1) return 1.0;
    double d_prev = al[0] - x;   // d_{t-1}
    if (fabs(d_prev) < pivmin) d_prev = -pivmin;
    double g_prev2 = -1.0;                       // g_1
    double g_prev = -1.0 - (al[1] - x) / d_prev;  // g_2
    if (k == 2) return -1.0 / g_prev;
    // advance: compute d_2 then g_3 ... g_k
    for (int t = 3; t <= k; ++t) {
        double d_cur = (al[t - 2] - x) - b2[t - 3] / d_prev;  // d_{t-1}
        if (fabs(d_cur) < pivmin) d_cur = -pivmin;
        const double g = -1.0 + ((al[t - 1] - x) * g_prev - b2[t - 2] * g_prev2 / d_prev) / d_cur;
        d_prev = d_cur;
        g_prev2 = g_prev;
        g_prev = g;
    }
    const double s2 = -1.0 / g_prev;
    return isfinite(s2) ? fmax(0.0, s2) : 0.0;
}

// Warp-cooperative multisection for the i-th largest eigenvalue of T.
__device__ double kth_largest(const double* al, const double* b2, int k, int i, double gl, double gu,
                              double pivmin) {
    const int lane = threadIdx.x & 31;
    const int target = k - 1 - i;  // ascending index
    double lo = gl, hi = gu;
    for (int round = 0; round < 24; ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const int cnt = sturm_count(al, b2, k, x, pivmin);
        const unsigned ball = __ballot_sync(0xffffffffu, cnt > target);
        const int first = ball ? __ffs(ball) - 1 : 32;
        const double xf = __shfl_sync(0xffffffffu, x, first < 32 ? first : 31);
        const double xp = __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0);
        const double nhi = first < 32 ? xf : hi;
        const double nlo = first > 0 ? xp : lo;
        lo = nlo;
        hi = nhi;
        if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin) break;
    }
    return 0.5 * (lo + hi);
}

// Inverse iteration for the eigenvector of T for eigenvalue th (unit 2-norm).
// d, du, dl, du2, x: k doubles each; piv: k doubles (0/1 flags).
__device__ void tri_inverse_iteration(const double* al, const double* be, int k, double th,
                                      double pert, double* d, double* du, double* dl, double* du2,
                                      double* piv, double* x) {
    for (int t = 0; t < k; ++t) {
        d[t] = al[t] - th;
        du2[t] = 0.0;
        if (t < k - 1) {
            du[t] = be[t];
            dl[t] = be[t];
        }
    }
    for (int t = 0; t < k - 1; ++t) {
        if (fabs(d[t]) >= fabs(dl[t])) {
            piv[t] = 0.0;
            if (d[t] == 0.0) d[t] = pert;
            const double f = dl[t] / d[t];
            dl[t] = f;
            d[t + 1] -= f * du[t];
        } else {
            piv[t] = 1.0;
            const double f = d[t] / dl[t];
            d[t] = dl[t];
            dl[t] = f;
            const double tmp = du[t];
            du[t] = d[t + 1];
            d[t + 1] = tmp - f * d[t + 1];
            if (t < k - 2) {
                du2[t] = du[t + 1];
                du[t + 1] = -f * du[t + 1];
            }
        }
    }
    if (d[k - 1] == 0.0) d[k - 1] = pert;
    for (int t = 0; t < k; ++t) x[t] = 1.0 + 0.25 * (double)((t * 7919) % 13) / 13.0;
    for (int it = 0; it < 3; ++it) {
        for (int t = 0; t < k - 1; ++t) {
            if (piv[t] == 0.0) {
                x[t + 1] -= dl[t] * x[t];
            } else {
                const double tmp = x[t];
                x[t] = x[t + 1];
                x[t + 1] = tmp - dl[t] * x[t];
            }
        }
        x[k - 1] /= d[k - 1];
        if (k > 1) x[k - 2] = (x[k - 2] - du[k - 2] * x[k - 1]) / d[k - 2];
        for (int t = k - 3; t >= 0; --t) x[t] = (x[t] - du[t] * x[t + 1] - du2[t] * x[t + 2]) / d[t];
        double mx = 0.0;
        for (int t = 0; t < k; ++t) mx = fmax(mx, fabs(x[t]));
        if (!(mx > 0.0) || !isfinite(mx)) mx = 1.0;
        double ss = 0.0;
        for (int t = 0; t < k; ++t) {
            x[t] /= mx;
            ss += x[t] * x[t];
        }
        const double inv = 1.0 / sqrt(ss);
        for (int t = 0; t < k; ++t) x[t] *= inv;
    }
}

__device__ __forceinline__ double start_entry(int row) {
    // splitmix64 of the row index -> uniform in [-1, 1)
    uint64_t z = (uint64_t)row * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void __launch_bounds__(kThreads, 1) k_lanczos(LanczosArgs A) {
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int pj = blockIdx.x / cs;
    if (pj >= A.p) return;  // the whole cluster shares pj
    const ProbDesc P = A.desc[pj];
    const int n = P.n, ldq = P.ldq, r = A.r;
    const int R = (n + cs - 1) / cs;
    const int r0 = min(n, q * R), r1 = min(n, r0 + R), nr = r1 - r0;
    const double* __restrict__ Q = A.qarena + P.q_off;
    double* __restrict__ B = A.barena + P.b_off;
    const int kmax = min(A.mmax, n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    extern __shared__ __align__(16) double smraw[];
    Smem S = carve(smraw, A.max_n, cs, A.mmax);
    double* part[2] = {S.part0, S.part1};
    int pb = 0;

    // ---- start vector: pseudo-random, unit norm
    double loc = 0.0;
    for (int i = tid; i < nr; i += kThreads) {
        const double v = start_entry(r0 + i);
        S.vloc[i] = v;
        loc += v * v;
    }
    {
        const double s = block_sum(loc, S.red);
        if (tid == 0) part[pb][0] = s;
        cluster_allreduce(cl, part[pb], S.cfull, 1, cs);
        pb ^= 1;
        const double inv = 1.0 / sqrt(S.cfull[0]);
        for (int i = tid; i < nr; i += kThreads) {
            S.vloc[i] *= inv;
            B[r0 + i] = S.vloc[i];
        }
    }

    const int check_every = cs == 1 ? 4 : 8;
    const int kmin = min(kmax, max(2 * r, 8));
    double tnorm = 0.0;
    int k = 0;
    bool converged = false;

    for (int j = 0; j < kmax; ++j) {
        // ---- gather v_j from all ranks
        cl.sync();
        for (int i = tid; i < n; i += kThreads) {
            const int src = i / R;
            S.vfull[i] = cl.map_shared_rank(S.vloc, src)[i - src * R];
        }
        __syncthreads();

        // ---- w = Q v_j on this CTA's rows (one warp per row)
        for (int i = warp; i < nr; i += kWarps) {
            const double* qr = Q + (int64_t)(r0 + i) * ldq;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll 4
            for (int kk = 2 * lane; kk < n; kk += 64) {
                if (kk + 1 < n) {
                    const double2 qv = *reinterpret_cast<const double2*>(qr + kk);
                    const double2 vv = *reinterpret_cast<const double2*>(S.vfull + kk);
                    s0 = fma(qv.x, vv.x, s0);
                    s1 = fma(qv.y, vv.y, s1);
                } else {
                    s0 = fma(qr[kk], S.vfull[kk], s0);
                }
            }
            const double s = warp_sum(s0 + s1);
            if (lane == 0) S.wloc[i] = s;
        }
        __syncthreads();

        // ---- two passes of classical Gram-Schmidt against v_0..v_j
        double alpha_j = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = warp; i <= j; i += kWarps) {
                const double* bi = B + (int64_t)i * ldq + r0;
                double s = 0.0;
                for (int rr = lane; rr < nr; rr += 32) s = fma(bi[rr], S.wloc[rr], s);
                s = warp_sum(s);
                if (lane == 0) part[pb][i] = s;
            }
            __syncthreads();
            cluster_allreduce(cl, part[pb], S.cfull, j + 1, cs);
            pb ^= 1;
            for (int rr = tid; rr < nr; rr += kThreads) {
                double s = 0.0;
                for (int i = 0; i <= j; ++i) s = fma(B[(int64_t)i * ldq + r0 + rr], S.cfull[i], s);
                S.wloc[rr] -= s;
            }
            alpha_j += S.cfull[j];
            __syncthreads();
        }

        // ---- beta_j = ||w||
        loc = 0.0;
        for (int rr = tid; rr < nr; rr += kThreads) loc += S.wloc[rr] * S.wloc[rr];
        {
            const double s = block_sum(loc, S.red);
            if (tid == 0) part[pb][0] = s;
            cluster_allreduce(cl, part[pb], S.cfull, 1, cs);
            pb ^= 1;
        }
        const double beta_j = sqrt(S.cfull[0]);
        if (tid == 0) {
            S.alpha[j] = alpha_j;
            S.beta[j] = beta_j;
            S.beta2[j] = beta_j * beta_j;
        }
        tnorm = fmax(tnorm, fabs(alpha_j) + 2.0 * beta_j);
        k = j + 1;
        __syncthreads();

        const bool breakdown = beta_j <= 1e-12 * tnorm || k == n;
        const bool do_check =
            breakdown || k == kmax || (k >= kmin && ((k - kmin) % check_every) == 0);
        if (do_check && k >= r) {
            // Gershgorin bounds of T_k
            double gl = DBL_MAX, gu = -DBL_MAX, bmax2 = 1.0;
            for (int t = 0; t < k; ++t) {
                const double off = (t > 0 ? S.beta[t - 1] : 0.0) + (t < k - 1 ? S.beta[t] : 0.0);
                gl = fmin(gl, S.alpha[t] - off);
                gu = fmax(gu, S.alpha[t] + off);
                if (t < k - 1) bmax2 = fmax(bmax2, S.beta2[t]);
            }
            const double pad = 2.0 * DBL_EPSILON * fmax(fabs(gl), fabs(gu)) * k + DBL_MIN;
            gl -= pad;
            gu += pad;
            const double pivmin = 1e-290 * bmax2;
            for (int i = warp; i < r; i += kWarps) {
                const double th = kth_largest(S.alpha, S.beta2, k, i, gl, gu, pivmin);
                if (lane == 0) {
                    S.theta[i] = th;
                    S.resid[i] = beta_j * sqrt(last_comp2(S.alpha, S.beta2, k, th, pivmin));
                }
            }
            __syncthreads();
            bool ok = true;
            const double thr = A.tol * fabs(S.theta[0]);
            for (int i = 0; i < r; ++i) ok = ok && (S.resid[i] <= thr || breakdown);
            if (ok) {
                converged = true;
                break;
            }
        }
        if (breakdown) break;  // k < r: fewer Ritz values than wanted

        // ---- v_{j+1} = w / beta_j
        const double inv = 1.0 / beta_j;
        for (int rr = tid; rr < nr; rr += kThreads) {
            const double v = S.wloc[rr] * inv;
            S.vloc[rr] = v;
            B[(int64_t)(j + 1) * ldq + r0 + rr] = v;
        }
        __syncthreads();
    }

    // ---- finish: status, eigenvectors of T_k (rank 0), Ritz vectors (all)
    double* scr = A.scratch + (size_t)pj * lanczos_scratch_per_problem(A.mmax, r);
    double* Sv = scr;  // r x (mmax+1): eigenvectors of T_k
    int status = kDevOk;
    if (k < r) {
        status = kDevRank;
    } else {
        if (!converged) status = kDevNoConv;
        if (!(S.theta[r - 1] > 0.0) || !(S.theta[r - 1] > A.rank_tol * S.theta[0])) status = kDevRank;
    }
    if (q == 0 && k >= r) {
        const double pert = DBL_EPSILON * fmax(tnorm, DBL_MIN);
        for (int i = tid; i < r; i += kThreads) {
            double* base = scr + (size_t)r * (A.mmax + 1) + (size_t)i * 6 * (A.mmax + 1);
            const int L = A.mmax + 1;
            tri_inverse_iteration(S.alpha, S.beta, k, S.theta[i], pert, base, base + L, base + 2 * L,
                                  base + 3 * L, base + 4 * L, base + 5 * L);
            for (int t = 0; t < k; ++t) Sv[(size_t)i * L + t] = base[5 * L + t];
        }
        __syncthreads();
        // modified Gram-Schmidt across the r vectors (warp 0)
        if (warp == 0) {
            const int L = A.mmax + 1;
            for (int i = 0; i < r; ++i) {
                double* xi = Sv + (size_t)i * L;
                for (int m = 0; m < i; ++m) {
                    const double* xm = Sv + (size_t)m * L;
                    double s = 0.0;
                    for (int t = lane; t < k; t += 32) s += xi[t] * xm[t];
                    s = warp_sum(s);
                    for (int t = lane; t < k; t += 32) xi[t] -= s * xm[t];
                    __syncwarp();
                }
                double s = 0.0;
                for (int t = lane; t < k; t += 32) s += xi[t] * xi[t];
                s = warp_sum(s);
                const double inv = 1.0 / sqrt(s);
                for (int t = lane; t < k; t += 32) xi[t] *= inv;
                __syncwarp();
            }
        }
        __threadfence();
    }
    cl.sync();
    if (k < r) {
        if (q == 0 && tid == 0) {
            A.status[pj] = status;
            A.steps[pj] = k;
        }
        return;
    }

    // Ritz vectors y_i = V_k s_i for this CTA's rows; per-column |max| for the sign rule.
    double* V = A.varena + P.v_off;
    const int L = A.mmax + 1;
    for (int rr = tid; rr < nr; rr += kThreads) {
        for (int i = 0; i < r; ++i) {
            const double* si = Sv + (size_t)i * L;
            double s = 0.0;
            for (int t = 0; t < k; ++t) s = fma(B[(int64_t)t * ldq + r0 + rr], __ldcg(si + t), s);
            V[(int64_t)(r0 + rr) * r + i] = s;
        }
    }
    __syncthreads();
    // argmax |y_i| (lowest row on ties): per CTA by warp i, then across the cluster
    for (int i = warp; i < r; i += kWarps) {
        double best = -1.0, bestv = 0.0;
        int brow = INT32_MAX;
        for (int rr = lane; rr < nr; rr += 32) {
            const double v = V[(int64_t)(r0 + rr) * r + i];
            const double a = fabs(v);
            if (a > best || (a == best && r0 + rr < brow)) {
                best = a;
                bestv = v;
                brow = r0 + rr;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const double ov = __shfl_xor_sync(0xffffffffu, bestv, o);
            const int orow = __shfl_xor_sync(0xffffffffu, brow, o);
            if (ob > best || (ob == best && orow < brow)) {
                best = ob;
                bestv = ov;
                brow = orow;
            }
        }
        if (lane == 0) {
            S.sgn[3 * i] = best;
            S.sgn[3 * i + 1] = (double)brow;
            S.sgn[3 * i + 2] = bestv;
        }
    }
    cl.sync();
    __shared__ double flip[kMaxR];
    if (tid < r) {
        double best = -1.0, bestv = 0.0, brow = 1e300;
        for (int qq = 0; qq < cs; ++qq) {
            const double* o = cl.map_shared_rank(S.sgn, qq) + 3 * tid;
            if (o[0] > best || (o[0] == best && o[1] < brow)) {
                best = o[0];
                brow = o[1];
                bestv = o[2];
            }
        }
        flip[tid] = bestv < 0.0 ? -1.0 : 1.0;
    }
    cl.sync();  // peers are done reading S.sgn before any CTA exits
    for (int rr = tid; rr < nr; rr += kThreads)
        for (int i = 0; i < r; ++i) V[(int64_t)(r0 + rr) * r + i] *= flip[i];
    if (q == 0 && tid == 0) {
        for (int i = 0; i < r; ++i) A.lam[(size_t)pj * r + i] = S.theta[i];
        A.status[pj] = status;
        A.steps[pj] = k;
    }
}

}  // namespace

size_t lanczos_smem_bytes(int max_n, int cs, int mmax) {
    return smem_doubles(max_n, cs, mmax) * sizeof(double) + kMaxR * sizeof(double);
}

cudaError_t launch_lanczos(const LanczosArgs& a, int cluster, cudaStream_t st) {
    if (a.p <= 0) return cudaSuccess;
    const int cs = cluster < 1 ? 1 : (cluster > 16 ? 16 : cluster);
    const size_t smem = smem_doubles(a.max_n, cs, a.mmax) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_lanczos, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > 8) {
        e = cudaFuncSetAttribute(k_lanczos, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.p * cs));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launch(1);
    return cudaLaunchKernelEx(&cfg, k_lanczos, a);
}

}  // namespace gbmds
