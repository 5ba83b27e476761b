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
//   found by Sturm-count multisection and their eigenvectors s_i by inverse
//   iteration (tridiagonal LU with partial pivoting); the Ritz residuals are
//   ||Q y_i - theta_i y_i|| = beta_{k-1} |s_i[k-1]|.  The run stops when every
//   residual is below tol * theta_0, at an invariant subspace (beta ~ 0), or
//   at the step cap (status NOCONV).  The s_i of the last check are
//   orthonormalised (modified Gram-Schmidt) and the Ritz vectors are
//   y_i = V_k s_i.
//
// Layout: Q_j row-major FP64 (ld = ldq).  The cluster's CTAs own contiguous
// row slices; each CTA's slice of the current Lanczos vector lives in its
// shared memory and is gathered through distributed shared memory; dot
// products are reduced across the cluster through DSMEM in rank order, so
// every CTA holds bitwise-identical scalars and takes identical decisions.
//
// Streaming: Q is read once per step and does not change, so each warp
// streams its rows of Q through its own ring of shared-memory stages with
// asynchronous bulk copies (cp.async.bulk, completion on an mbarrier per
// stage).  The warp re-issues a stage as soon as it has consumed it, running
// one ring ahead into the next step: the copies for step j+1 are in flight
// while the cluster does step j's Gram-Schmidt passes and reductions.
#include <cooperative_groups.h>
#include <float.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace gbmds {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRing = 3;           // stages per warp
constexpr int kChunkB = 4096;      // bytes per stage (a row segment of Q)
constexpr size_t kRingBytes = (size_t)kWarps * kRing * kChunkB;

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
    double* sgn;     // 4 * kMaxR : (|max|, row, signed) per eigenvector, then sign flips
    double* xv;      // r * (mmax + 1): eigenvectors x_i of T_k, one row of mmax + 1 per i
    double* band;    // ceil(r / cs) * 3 * (mmax + 1): U bands of this CTA's inverse iterations
    uint8_t* ring;   // kWarps * kRing * kChunkB bytes: per-warp Q stages
    uint64_t* full;  // kWarps * kRing mbarriers
};

__host__ __device__ inline int owned_max(int r, int cs) { return (r + cs - 1) / cs; }

__host__ __device__ inline size_t smem_doubles(int max_n, int cs, int mmax, int r) {
    const size_t rmax = (size_t)((max_n + cs - 1) / cs);
    return kRingBytes / 8 + (size_t)kWarps * kRing + round_up(max_n + 1, 2) + 2 * round_up(rmax, 2) +
           3 * (size_t)(mmax + 2) + 3 * (size_t)(mmax + 1) + 2 * kMaxR + 64 + 4 * kMaxR +
           (size_t)r * (mmax + 1) + 3 * (size_t)owned_max(r, cs) * (mmax + 1) + 8;
}

__device__ Smem carve(double* base, int max_n, int cs, int mmax, int r) {
    Smem s;
    const int rmax = (max_n + cs - 1) / cs;
    double* p = base;
    s.ring = reinterpret_cast<uint8_t*>(p); p += kRingBytes / 8;
    s.full = reinterpret_cast<uint64_t*>(p); p += kWarps * kRing;
    s.vfull = p; p += round_up(max_n + 1, 2);
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
    s.sgn = p; p += 4 * kMaxR;
    s.xv = p; p += (size_t)r * (mmax + 1);
    s.band = p;
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

// Number of eigenvalues of T (alpha, beta^2) smaller than x: the sign changes
// of the Sturm sequence p_0 = 1, p_t = det(T_t - x I) =
// (alpha_{t-1} - x) p_{t-1} - beta_{t-2}^2 p_{t-2} (a sign change between
// p_{t-1} and p_t is a negative pivot of T - x I = L D L^T).  No division: the
// pair (p_{t-1}, p_t) is rescaled by exact powers of two to stay in range, and
// an exact zero counts as a sign change (a tiny negative pivot).
__device__ int sturm_count(const double* al, const double* b2, int k, double x) {
    double pm = 1.0, p = al[0] - x;
    if (p == 0.0) p = -1e-300;
    int c = p < 0.0;
    for (int t = 1; t < k; ++t) {
        double pn = fma(al[t] - x, p, -b2[t - 1] * pm);
        if (pn == 0.0) pn = -p * 1e-300;
        c += (pn < 0.0) != (p < 0.0);
        pm = p;
        p = pn;
        const double ap = fabs(p);
        if (ap > 0x1p+500) {
            p *= 0x1p-500;
            pm *= 0x1p-500;
        } else if (ap < 0x1p-500 && fabs(pm) < 0x1p-500) {
            p *= 0x1p+500;
            pm *= 0x1p+500;
        }
    }
    return c;
}

// The i-th largest eigenvalue of T on [lo, hi] (count(lo) <= k-1-i < count(hi))
// by 32-way multisection: each lane of the calling warp counts at its own probe,
// so every FP64 warp instruction (which occupies the SMSP's FP64 unit for the
// whole warp whatever the mask) does 32 useful Sturm steps.  ~11 rounds.
__device__ double kth_largest(const double* al, const double* b2, int k, int i, double lo, double hi) {
    const int lane = threadIdx.x & 31;
    const int target = k - 1 - i;
    for (int round = 0; round < 16; ++round) {
        const double step = (hi - lo) * (1.0 / 33.0);
        const double x = fmin(fma((double)(lane + 1), step, lo), hi);
        const unsigned ball = __ballot_sync(0xffffffffu, sturm_count(al, b2, k, x) > target);
        const int first = ball ? __ffs(ball) - 1 : 32;
        const double xf = __shfl_sync(0xffffffffu, x, first < 32 ? first : 31);
        const double xp = __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0);
        if (first < 32) hi = xf;
        if (first > 0) lo = xp;
        if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi))) break;
    }
    return 0.5 * (lo + hi);
}

// 1/x by Newton-Raphson iteration y <- y (2 - x y) from the FP32 reciprocal:
// 24 -> 48 -> 96 correct bits (limited by FP64), in four FP64 instructions.
__device__ __forceinline__ double rcp_newton(double x) {
    const float xf = (float)x;
    if (!(fabsf(xf) > 1e-30f && fabsf(xf) < 1e30f)) return 1.0 / x;
    double y = (double)__frcp_rn(xf);
    y = y * fma(-x, y, 2.0);
    y = y * fma(-x, y, 2.0);
    return y;
}

// Inverse iteration for the eigenvector of T for eigenvalue th (unit 2-norm),
// all in shared memory.  Each iteration factors T - th I = P L U by Gaussian
// elimination with partial pivoting (U has the bands 1/u0, u1, u2) while it
// applies the same row operations to the right-hand side x, then solves with
// U from the bottom up: one division per row.  Two iterations from a fixed
// positive start vector (th is accurate to a few ulps).
__device__ void tri_inverse_iteration(const double* al, const double* be, int k, double th,
                                      double pert, double* u0i, double* u1, double* u2,
                                      double* x) {
    for (int t = 0; t < k; ++t) x[t] = 1.0 + 0.25 * (double)((t * 7919) % 13) / 13.0;
    for (int it = 0; it < 2; ++it) {
        // working row t: entries (w0, w1) in columns t, t+1 and right-hand side yw
        double w0 = al[0] - th, w1 = k > 1 ? be[0] : 0.0, yw = x[0];
        for (int t = 0; t < k - 1; ++t) {
            const double l0 = be[t];                           // row t+1, column t
            const double l1 = al[t + 1] - th;                  // row t+1, column t+1
            const double l2 = t + 2 < k ? be[t + 1] : 0.0;     // row t+1, column t+2
            const double yl = x[t + 1];
            if (fabs(w0) >= fabs(l0)) {                        // pivot on the working row
                if (w0 == 0.0) w0 = pert;
                const double inv = rcp_newton(w0);
                const double f = l0 * inv;
                u0i[t] = inv;
                u1[t] = w1;
                u2[t] = 0.0;
                x[t] = yw;
                w0 = l1 - f * w1;
                w1 = l2;
                yw = yl - f * yw;
            } else {                                           // pivot on row t+1
                const double inv = rcp_newton(l0);
                const double f = w0 * inv;
                u0i[t] = inv;
                u1[t] = l1;
                u2[t] = l2;
                x[t] = yl;
                w0 = w1 - f * l1;
                w1 = -f * l2;
                yw = yw - f * yl;
            }
        }
        if (w0 == 0.0) w0 = pert;
        u0i[k - 1] = rcp_newton(w0);
        x[k - 1] = yw * u0i[k - 1];
        if (k > 1) x[k - 2] = (x[k - 2] - u1[k - 2] * x[k - 1]) * u0i[k - 2];
        for (int t = k - 3; t >= 0; --t) x[t] = (x[t] - u1[t] * x[t + 1] - u2[t] * x[t + 2]) * u0i[t];
        double mx = 0.0;
        for (int t = 0; t < k; ++t) mx = fmax(mx, fabs(x[t]));
        if (!(mx > 0.0) || !isfinite(mx)) mx = 1.0;
        const double imx = 1.0 / mx;
        double ss = 0.0;
        for (int t = 0; t < k; ++t) {
            x[t] *= imx;
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

// Double-FP32 arithmetic (Dekker 1971; Knuth's TwoSum): a value is an
// unevaluated sum hi + lo of two floats (about 48 significant bits).  The
// products run on the FP32 pipe, whose rate on GB300 is ~57x the FP64 rate.
// __fmul_rn / __fadd_rn / __fsub_rn keep the compiler from contracting the
// error-free transforms into FMAs.
__device__ __forceinline__ void df_madd(float& sh, float& sl, float qh, float ql, float vh,
                                        float vl) {
    const float p = __fmul_rn(qh, vh);
    float e = fmaf(qh, vh, -p);          // exact rounding error of qh * vh
    e = fmaf(qh, vl, e);
    e = fmaf(ql, vh, e);
    const float s = __fadd_rn(sh, p);    // TwoSum(sh, p) = s + t exactly
    const float z = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
    sl = __fadd_rn(sl, __fadd_rn(t, e));
    sh = s;
}

__device__ __forceinline__ void df_add(float& sh, float& sl, float oh, float ol) {
    const float s = __fadd_rn(sh, oh);
    const float z = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(oh, z));
    sl = __fadd_rn(sl, __fadd_rn(t, ol));
    sh = s;
}

// ---------------------------------------------------------------- Q stream
//
// Warp w of a CTA owns rows [wr0, wr1) of the CTA's slice and streams them in
// row segments of at most kChunkB bytes through stages ring[w][0..kRing).
// Chunk g (counted per warp across steps and problems, so the mbarrier phase
// of stage g % kRing is (g / kRing) & 1) is segment u = (g - g0) % per_step of
// the warp's rows, g0 being the problem's first chunk.
struct QStream {
    const uint8_t* q;   // Q of the problem (bytes)
    size_t row_stride;  // ldq * 8
    int rowbytes;       // round_up(n, 2) * 8: what one row's copies cover
    int segs;           // segments per row
    int wr0, wr1;       // this warp's rows
    int per_step;       // (wr1 - wr0) * segs
    long long g0;       // first chunk of the problem
    long long issued;   // chunks issued (valid in lane 0)
    uint8_t* ring;      // this warp's stages
    uint64_t* full;     // this warp's barriers
};

__device__ __forceinline__ void qs_issue(QStream& Qs, long long g) {
    const int u = (int)((g - Qs.g0) % Qs.per_step);
    const int row = Qs.wr0 + u / Qs.segs, seg = u % Qs.segs;
    const int off = seg * kChunkB;
    const int bytes = min(kChunkB, Qs.rowbytes - off);
    const int st = (int)(g % kRing);
    tc::mbar_expect_tx(&Qs.full[st], (uint32_t)bytes);
    tc::bulk_load(Qs.ring + (size_t)st * kChunkB, Qs.q + (size_t)row * Qs.row_stride + off, (uint32_t)bytes,
                  &Qs.full[st]);
}

// Bounded wait on a stage; false after ~2 s (the copy source is ordinary
// device memory, so this only guards against a broken launch).
__device__ __forceinline__ bool qs_wait(uint64_t* bar, uint32_t parity) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = tc::global_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (tc::mbar_try_wait(bar, parity)) return true;
        if (tc::global_ns() - t0 > tc::kWaitNs) return false;
    }
}

// Sets up this warp's stream for a problem and issues its first kRing chunks.
__device__ __forceinline__ void qs_begin(QStream& Qs, const Smem& S, const double* Q, int ldq, int n, int r0,
                                         int nr, long long g) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per_warp = (nr + kWarps - 1) / kWarps;
    Qs.q = reinterpret_cast<const uint8_t*>(Q);
    Qs.row_stride = (size_t)ldq * 8;
    Qs.rowbytes = (int)round_up(n, 2) * 8;
    Qs.segs = (Qs.rowbytes + kChunkB - 1) / kChunkB;
    Qs.wr0 = r0 + min(nr, warp * per_warp);
    Qs.wr1 = r0 + min(nr, (warp + 1) * per_warp);
    Qs.per_step = (Qs.wr1 - Qs.wr0) * Qs.segs;
    Qs.g0 = g;
    Qs.issued = g;
    Qs.ring = S.ring + (size_t)warp * kRing * kChunkB;
    Qs.full = S.full + warp * kRing;
    if (Qs.per_step > 0 && lane == 0)
        for (int i = 0; i < kRing; ++i) qs_issue(Qs, Qs.issued++);
}

// Waits (bounded) for the chunks still in flight at the end of a problem.
__device__ __forceinline__ long long qs_end(QStream& Qs, long long consumed, bool& timeout) {
    if (Qs.per_step > 0) {
        for (long long g = consumed; g < consumed + kRing; ++g)
            if (!qs_wait(&Qs.full[g % kRing], (uint32_t)((g / kRing) & 1))) timeout = true;
    }
    __syncwarp();
    return Qs.per_step > 0 ? consumed + kRing : consumed;
}

// w[row - r0] = Q[row, :] . v for this warp's rows, consuming one step of the
// stream and re-issuing every stage it frees.  DF: Q entries and v are
// (hi, lo) float pairs and the products run in double-FP32; else FP64.
template <bool DF>
__device__ __forceinline__ long long qs_matvec(QStream& Qs, long long g, int n, int r0, const double* vfull,
                                               double* w, bool& timeout) {
    const int lane = threadIdx.x & 31;
    float sh = 0.f, sl = 0.f;
    double acc = 0.0;
    for (int u = 0; u < Qs.per_step; ++u, ++g) {
        const int st = (int)(g % kRing);
        if (!qs_wait(&Qs.full[st], (uint32_t)((g / kRing) & 1))) timeout = true;
        const int row = Qs.wr0 + u / Qs.segs, seg = u % Qs.segs;
        const int col0 = seg * (kChunkB / 8);
        const int bytes = min(kChunkB, Qs.rowbytes - seg * kChunkB);
        const uint8_t* stage = Qs.ring + (size_t)st * kChunkB;
        for (int t = lane; t < bytes / 16; t += 32) {
            const int c = col0 + 2 * t;
            if (DF) {
                const float4 x = reinterpret_cast<const float4*>(stage)[t];
                const float4 vv = reinterpret_cast<const float4*>(vfull)[c >> 1];
                df_madd(sh, sl, x.x, x.y, vv.x, vv.y);
                if (c + 1 < n) df_madd(sh, sl, x.z, x.w, vv.z, vv.w);
            } else {
                const double2 x = reinterpret_cast<const double2*>(stage)[t];
                const double2 vv = reinterpret_cast<const double2*>(vfull)[c >> 1];
                acc = fma(x.x, vv.x, acc);
                if (c + 1 < n) acc = fma(x.y, vv.y, acc);
            }
        }
        __syncwarp();
        if (lane == 0) qs_issue(Qs, Qs.issued++);   // the stage is free: next chunk in the periodic stream
        if (seg == Qs.segs - 1) {
            if (DF) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
                    const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
                    df_add(sh, sl, oh, ol);
                }
                if (lane == 0) w[row - r0] = (double)sh + (double)sl;
                sh = sl = 0.f;
            } else {
                acc = warp_sum(acc);
                if (lane == 0) w[row - r0] = acc;
                acc = 0.0;
            }
        }
    }
    return g;
}

// part[i] = sum over this CTA's rows of B[i][row] * w[row], i <= j (warp per i).
// B is written by this kernel (new Lanczos vectors), so it must never be read
// through the non-coherent read-only path: no __restrict__ on it.
// With with_norm, part[j+1] also receives the partial sum of w[row]^2.
__device__ __forceinline__ void cgs_dots(const double* B, int ldq, int r0, int nr, int j,
                                         const double* w, double* part, bool with_norm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (with_norm && warp == (j + 1) % kWarps) {
        double s0 = 0.0;
        for (int rr = lane; rr < nr; rr += 32) s0 = fma(w[rr], w[rr], s0);
        s0 = warp_sum(s0);
        if (lane == 0) part[j + 1] = s0;
    }
    for (int i = warp; i <= j; i += kWarps) {
        const double* bi = B + (int64_t)i * ldq + r0;
        double s0 = 0.0, s1 = 0.0;
        int rr = lane;
        for (; rr + 32 < nr; rr += 64) {
            s0 = fma(bi[rr], w[rr], s0);
            s1 = fma(bi[rr + 32], w[rr + 32], s1);
        }
        if (rr < nr) s0 = fma(bi[rr], w[rr], s0);
        const double s = warp_sum(s0 + s1);
        if (lane == 0) part[i] = s;
    }
}

// w[row] -= sum_{i <= j} B[i][row] * c[i] (thread per row).
__device__ __forceinline__ void cgs_update(const double* B, int ldq, int r0, int nr, int j,
                                           const double* c, double* w) {
    for (int rr = threadIdx.x; rr < nr; rr += kThreads) {
        const double* b = B + r0 + rr;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int i = 0;
        for (; i + 3 <= j; i += 4) {
            s0 = fma(b[(int64_t)i * ldq], c[i], s0);
            s1 = fma(b[(int64_t)(i + 1) * ldq], c[i + 1], s1);
            s2 = fma(b[(int64_t)(i + 2) * ldq], c[i + 2], s2);
            s3 = fma(b[(int64_t)(i + 3) * ldq], c[i + 3], s3);
        }
        for (; i <= j; ++i) s0 = fma(b[(int64_t)i * ldq], c[i], s0);
        w[rr] -= (s0 + s1) + (s2 + s3);
    }
}

// One eigenproblem (part pj) solved by the calling cluster.  DF: Q is stored
// as double-FP32 pairs and the matrix-vector product runs in double-FP32.
template <bool DF>
__device__ void solve_problem(const LanczosArgs& A, int pj, cg::cluster_group& cl, int cs, int q,
                              double* smraw, int& s_flag, long long& qchunk) {
    const ProbDesc P = A.desc[pj];
    const int n = P.n, ldq = P.ldq, r = A.r;
    const int R = (n + cs - 1) / cs;
    const int r0 = min(n, q * R), r1 = min(n, r0 + R), nr = r1 - r0;
    const double* __restrict__ Q = A.qarena + P.q_off;
    double* B = A.barena + P.b_off;
    const int kmax = min(A.mmax, n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = A.mmax + 1;
    // per-problem global scratch: the final tridiagonal T_k (diagonal, off-diagonal)
    double* scr = A.scratch + (size_t)pj * lanczos_scratch_per_problem(A.mmax, r);

    Smem S = carve(smraw, A.max_n, cs, A.mmax, r);
    double* part[2] = {S.part0, S.part1};
    int pb = 0;
    // start streaming this CTA's rows of Q right away
    QStream Qs;
    qs_begin(Qs, S, Q, ldq, n, r0, nr, qchunk);
    long long g = qchunk;
    bool qtimeout = false;
    if (tid == 0) S.red[40] = 0.0;   // set to 1 by any thread whose stage wait timed out

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

    const int kmin = min(kmax, max(2 * r, 8));
    int next_check = kmin;
    double tnorm = 0.0, prev_worst = -1.0;
    int k = 0, prev_k = 0;
    bool converged = false, have_vectors = false;

    if (tid == 0) S.vfull[n] = 0.0;   // guard entry read by the paired loads when n is odd
    for (int j = 0; j < kmax; ++j) {
        // ---- gather v_j from all ranks
        cl.sync();
        for (int i = tid; i < n; i += kThreads) {
            const int src = i / R;
            const double v = cl.map_shared_rank(S.vloc, src)[i - src * R];
            if (DF) {
                const float h = (float)v;
                reinterpret_cast<float2*>(S.vfull)[i] = make_float2(h, (float)(v - (double)h));
            } else {
                S.vfull[i] = v;
            }
        }
        __syncthreads();

        // ---- w = Q v_j on this CTA's rows (streamed)
        g = qs_matvec<DF>(Qs, g, n, r0, S.vfull, S.wloc, qtimeout);
        __syncthreads();

        // ---- two passes of classical Gram-Schmidt against v_0..v_j; the
        // second pass also reduces ||w_1||^2, and ||w_2||^2 = ||w_1||^2 - ||c_2||^2.
        double alpha_j = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            cgs_dots(B, ldq, r0, nr, j, S.wloc, part[pb], pass == 1);
            __syncthreads();
            cluster_allreduce(cl, part[pb], S.cfull, j + 1 + pass, cs);
            pb ^= 1;
            cgs_update(B, ldq, r0, nr, j, S.cfull, S.wloc);
            alpha_j += S.cfull[j];
            if (pass == 1 && tid == 0) {
                double c2 = 0.0;
                for (int i = 0; i <= j; ++i) c2 = fma(S.cfull[i], S.cfull[i], c2);
                S.red[kWarps] = sqrt(fmax(S.cfull[j + 1] - c2, 0.0));
            }
            __syncthreads();
        }
        const double beta_j = S.red[kWarps];
        if (tid == 0) {
            S.alpha[j] = alpha_j;
            S.beta[j] = beta_j;
            S.beta2[j] = beta_j * beta_j;
        }
        tnorm = fmax(tnorm, fabs(alpha_j) + 2.0 * beta_j);
        k = j + 1;
        __syncthreads();

        const bool breakdown = beta_j <= 1e-12 * tnorm || k == n;
        const bool do_check = breakdown || k == kmax || k >= next_check;
        if (do_check && k >= r) {
            // Ritz values and residuals.  Eigenvalue i belongs to CTA i % cs and,
            // there, to warp m % 4, lane m / 4 (m = i / cs): every FP64 warp
            // instruction occupies an SMSP's FP64 unit for tens of cycles, so the
            // r bisections run on as many SMSPs of the cluster as possible.  Each
            // owner finds theta_i (bisection on Sturm counts, warm-bracketed by the
            // previous check), the eigenvector x_i of T_k (inverse iteration) and
            // the residual beta_j |x_i[k-1]|; all CTAs then read every theta and
            // residual through DSMEM and take the same decision.
            const int mine = (r - q + cs - 1) / cs;  // eigenvalues owned by this CTA
            if (warp < mine) {
                double gl = DBL_MAX, gu = -DBL_MAX;
                for (int t = lane; t < k; t += 32) {
                    const double off = (t > 0 ? S.beta[t - 1] : 0.0) + (t < k - 1 ? S.beta[t] : 0.0);
                    gl = fmin(gl, S.alpha[t] - off);
                    gu = fmax(gu, S.alpha[t] + off);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
                    gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
                }
                const double pad = 2.0 * DBL_EPSILON * fmax(fabs(gl), fabs(gu)) * k + DBL_MIN;
                gl -= pad;
                gu += pad;
                const double pert = DBL_EPSILON * fmax(tnorm, DBL_MIN);
                for (int m = warp; m < mine; m += kWarps) {   // one warp per eigenvalue
                    const int i = q + cs * m;
                    double lo = gl, hi = gu;
                    if (have_vectors) {
                        // lane 0 tests the lower end, lane 1 the upper end of the warm bracket
                        const int target = k - 1 - i;
                        const double t0 = S.theta[i];
                        const double t1 = t0 + 4.0 * S.resid[i] + 64.0 * DBL_EPSILON * fabs(t0);
                        const double xt = lane == 0 ? t0 : t1;
                        const int c = sturm_count(S.alpha, S.beta2, k, xt);
                        const int c0 = __shfl_sync(0xffffffffu, c, 0), c1 = __shfl_sync(0xffffffffu, c, 1);
                        if (t0 > gl && c0 <= target) lo = t0;
                        if (t1 < gu && t1 > lo && c1 > target) hi = t1;
                    }
                    const double th = kth_largest(S.alpha, S.beta2, k, i, lo, hi);
                    if (lane == 0) {
                        double* bd = S.band + (size_t)m * 3 * L;
                        double* x = S.xv + (size_t)i * L;
                        tri_inverse_iteration(S.alpha, S.beta, k, th, pert, bd, bd + L, bd + 2 * L, x);
                        S.theta[i] = th;
                        S.resid[i] = beta_j * fabs(x[k - 1]);
                    }
                    __syncwarp();
                }
            }
            cl.sync();
            for (int i = tid; i < r; i += kThreads) {
                const int owner = i % cs;
                if (owner != q) {
                    S.theta[i] = cl.map_shared_rank(S.theta, owner)[i];
                    S.resid[i] = cl.map_shared_rank(S.resid, owner)[i];
                }
            }
            __syncthreads();
            if (tid == 0) {
                bool ok = true;
                double worst = 0.0;
                const double th0 = fabs(S.theta[0]);
                for (int i = 0; i < r; ++i) {
                    ok = ok && (S.resid[i] <= A.tol * th0 || breakdown);
                    worst = fmax(worst, S.resid[i] / fmax(th0, DBL_MIN));
                }
                S.red[kWarps + 1] = worst;
                s_flag = ok ? 1 : 0;
            }
            cl.sync();  // owners keep theta/resid until every CTA has read them
            have_vectors = true;
            if (s_flag & 1) {
                converged = true;
                break;
            }
            // next check: extrapolate the residual decay seen between checks
            const double worst = S.red[kWarps + 1];
            int gap = 8;
            if (prev_worst > 0.0 && worst > 0.0 && worst < prev_worst) {
                const double rate = (log(prev_worst) - log(worst)) / (double)(k - prev_k);
                const double need = (log(worst) - log(A.tol)) / rate;
                gap = (int)fmin(16.0, fmax(2.0, ceil(need) + 1.0));
            } else if (worst < 1e-6) {
                gap = 4;
            }
            prev_worst = worst;
            prev_k = k;
            next_check = k + gap;
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

    // ---- finish: status, orthonormal eigenvectors of T_k (rank 0), Ritz vectors (all)
    qchunk = qs_end(Qs, g, qtimeout);
    if (qtimeout) S.red[40] = 1.0;
    __syncthreads();
    cl.sync();
    bool any_timeout = false;
    for (int qq = 0; qq < cs; ++qq) any_timeout |= cl.map_shared_rank(S.red, qq)[40] != 0.0;
    cl.sync();   // every CTA has read the flags before S.red is reused
    int status = kDevOk;
    if (k < r || !have_vectors) {
        status = kDevRank;
    } else {
        if (!converged) status = kDevNoConv;
        if (!(S.theta[r - 1] > 0.0) || !(S.theta[r - 1] > A.rank_tol * S.theta[0])) status = kDevRank;
    }
    if (any_timeout) status = kDevTimeout;
    if (q == 0 && status != kDevRank) {
        // rank 0 collects the eigenvectors of T_k computed by the other CTAs
        for (int e = tid; e < r * k; e += kThreads) {
            const int i = e / k, t = e % k;
            if (i % cs != 0) S.xv[(size_t)i * L + t] = cl.map_shared_rank(S.xv, i % cs)[(size_t)i * L + t];
        }
        __syncthreads();
    }
    if (q == 0 && status != kDevRank && warp == 0) {
        // modified Gram-Schmidt across the r inverse-iteration vectors (shared memory)
        for (int i = 0; i < r; ++i) {
            double* xi = S.xv + (size_t)i * L;
            for (int m = 0; m < i; ++m) {
                const double* xm = S.xv + (size_t)m * L;
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
    cl.sync();
    if (status == kDevRank) {
        if (q == 0 && tid == 0) {
            A.status[pj] = status;
            A.steps[pj] = k;
        }
        return;
    }
    // the other CTAs copy the eigenvectors of T_k from rank 0 (DSMEM)
    if (q != 0) {
        const double* src = cl.map_shared_rank(S.xv, 0);
        for (int e = tid; e < r * k; e += kThreads) {
            const int i = e / k, t = e % k;
            S.xv[(size_t)i * L + t] = src[(size_t)i * L + t];
        }
    }
    __syncthreads();

    // Ritz vectors y_i = V_k s_i for this CTA's rows; per-column |max| for the sign rule.
    double* V = A.varena + P.v_off;
    for (int rr = tid; rr < nr; rr += kThreads) {
        for (int i = 0; i < r; ++i) {
            const double* si = S.xv + (size_t)i * L;
            double s = 0.0;
            for (int t = 0; t < k; ++t) s = fma(B[(int64_t)t * ldq + r0 + rr], si[t], s);
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
    double* flip = S.sgn + 3 * kMaxR;  // kMaxR slots after the (|max|, row, value) triples
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
    if (q == 0)
        for (int t = tid; t < k; t += kThreads) {
            scr[t] = S.alpha[t];
            scr[L + t] = S.beta[t];
        }
}

// Persistent batched solver: each cluster takes parts from an atomic queue in
// the host's order (largest first), so uneven part sizes balance across the
// clusters that fit on the GPU at once.
template <bool DF>
__global__ void __launch_bounds__(kThreads, 2) k_lanczos(LanczosArgs A) {
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    extern __shared__ __align__(16) double smraw[];
    __shared__ int s_flag, s_next;
    {
        const Smem S = carve(smraw, A.max_n, cs, A.mmax, A.r);
        if (threadIdx.x == 0) {
            for (int i = 0; i < kWarps * kRing; ++i) tc::mbar_init(&S.full[i], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    long long qchunk = 0;   // Q-stream chunks this warp has consumed (all problems)
    for (;;) {
        if (q == 0 && threadIdx.x == 0) s_next = atomicAdd(A.counter, 1);
        cl.sync();
        const int next = q == 0 ? s_next : *cl.map_shared_rank(&s_next, 0);
        cl.sync();  // every CTA has read the index before rank 0 takes another
        if (next >= A.p) break;
        solve_problem<DF>(A, A.order[next], cl, cs, q, smraw, s_flag, qchunk);
    }
}

}  // namespace

size_t lanczos_smem_bytes(int max_n, int cs, int mmax, int r) {
    return smem_doubles(max_n, cs, mmax, r) * sizeof(double) + kMaxR * sizeof(double);
}

template <bool DF>
static cudaError_t launch_lanczos_t(const LanczosArgs& a, int cs, cudaStream_t st) {
    const size_t smem = smem_doubles(a.max_n, cs, a.mmax, a.r) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_lanczos<DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cs > 8) {
        e = cudaFuncSetAttribute(k_lanczos<DF>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
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
    int resident = 0;
    e = cudaOccupancyMaxActiveClusters(&resident, k_lanczos<DF>, &cfg);
    if (e != cudaSuccess) return e;
    if (resident < 1) return cudaErrorInvalidConfiguration;
    const int clusters = resident < a.p ? resident : a.p;
    cfg.gridDim = dim3((unsigned)(clusters * cs));
    note_launch(1);
    return cudaLaunchKernelEx(&cfg, k_lanczos<DF>, a);
}

cudaError_t launch_lanczos(const LanczosArgs& a, int cluster, cudaStream_t st) {
    if (a.p <= 0) return cudaSuccess;
    const int cs = cluster < 1 ? 1 : (cluster > 16 ? 16 : cluster);
    return a.q_df ? launch_lanczos_t<true>(a, cs, st) : launch_lanczos_t<false>(a, cs, st);
}

}  // namespace gbmds
