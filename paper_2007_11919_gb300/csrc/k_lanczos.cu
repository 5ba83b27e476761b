// Batched top-r symmetric eigen-solver: Lanczos with full
// re-orthogonalisation, one thread-block cluster per eigenproblem.
//
// The paper computes the classical-MDS eigenpairs of each l x l matrix Q with a
// Lanczos method (Section 2, the svd package's trlan.eigen); steps 2-3 of
// classical MDS keep the r largest eigenvalues and their eigenvectors.  Here:
//
//   Krylov basis v_0, v_1, ... of Q from a fixed pseudo-random start vector;
//   w = Q v_j, a local Gram-Schmidt pass against v_{j-1} and v_j (the
//   three-term recurrence, with computed coefficients) and a full classical
//   Gram-Schmidt pass against v_0..v_j, completed after the next step's
//   exchange (see the step loop); alpha_j = v_j . Q v_j, beta_j = ||w||,
//   v_{j+1} = w / beta_j.  The Rayleigh quotient T_k = V_k^T Q V_k is the
//   tridiagonal of the alphas and betas.  Every few steps the r largest
//   eigenvalues theta_i of T_k are found by Sturm-count multisection and their
//   eigenvectors s_i by inverse iteration (tridiagonal LU with partial
//   pivoting); the Ritz residuals are ||Q y_i - theta_i y_i|| =
//   beta_{k-1} |s_i[k-1]|.  The run stops when every residual is below
//   tol * theta_0, at an invariant subspace (beta ~ 0), or at the step cap
//   (status NOCONV).  The s_i of the last check are orthonormalised (modified
//   Gram-Schmidt) and the Ritz vectors are y_i = V_k s_i.
//
// Arithmetic: the scalars (alpha, beta, Gram-Schmidt coefficients) and the
// tridiagonal work are FP64.  For FP64 problems Q and every vector are FP64.
// Otherwise Q (double-centred in FP64 from FP32 distances) is stored in FP32,
// the basis vectors in FP32 and the working vectors in double-FP32 (a value
// is an unevaluated pair of floats, ~48 significant bits), because GB300
// issues FP64 at 1/64 of its FP32 rate; the matvec and the Gram-Schmidt dots
// run as FP32 FMA chains that meet in double-FP32, the updates in
// double-FP32.
//
// Layout: Q_j row-major (ld = ldq).  The cluster's CTAs own contiguous row
// slices; each CTA's slice of the current Lanczos vector lives in its shared
// memory and is gathered through distributed shared memory; dot products are
// reduced across the cluster through DSMEM in rank order, so every CTA holds
// bitwise-identical scalars and takes identical decisions.
//
// Symmetric ranges (FP32 Q, a cluster of cs >= 3 CTAs alone on a problem):
// Q = Q^T, so each entry of an off-diagonal block needs to be read once.  The
// rows are cut into cs blocks of R rows (R a multiple of 4, so every block
// starts on a 16-byte boundary) and CTA q reads, for each of its rows, the
// columns of blocks q, q+1, ..., q+m_q-1 (cyclically): (cs-1)/2 blocks past
// its own, and one more for the first cs/2 CTAs when cs is even.  Every
// unordered pair of blocks then lies in the range of exactly one CTA, which
// uses an entry q_ab of an off-diagonal block twice: in row a's dot and, by
// symmetry, as q_ba x_a towards entry b of the product.  Each row costs
// about (cs+1)/(2cs) of its bytes; the CTAs add the transposed sums of the
// blocks they own through DSMEM after the matvec.
//
// Streaming: Q is read once per step and does not change, so each warp
// streams its rows of Q in row segments of at most 4 KB through its own ring
// of shared-memory stages with asynchronous bulk copies (cp.async.bulk,
// completion on one mbarrier per stage), refilling a stage as soon as it has
// been consumed and running into the next step, so the copies for step j+1
// are in flight during step j's Gram-Schmidt passes.  Before a convergence
// check the rings are drained and their memory holds the check's workspace.
#include <cooperative_groups.h>
#include <float.h>
#include <limits.h>

#include "common.cuh"
#include "df.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace gbmds {

__device__ unsigned long long g_phase_cycles[8];

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Phase timers of the eigen-solver, compiled in only with -DGBMDS_PHASE_TIMERS
// (the build's GBMDS_PHASE_TIMERS=1): per CTA, clock64 cycles spent in each
// phase of the Lanczos steps, added over all CTAs into g_phase_cycles at the
// end of each problem: [0] exchange and completion of the second pass,
// [1] convergence checks, [2] matvec (with the symmetric ranges' collection),
// [3] the pass against v_{j-1}, v_j, [4] publishing w_1, [5] the finish
// (eigenvectors of T, Ritz vectors, signs), [6] CTA-steps.
#ifdef GBMDS_PHASE_TIMERS
#define PHASE_DECL long long ph_t = clock64(), ph[6] = {0, 0, 0, 0, 0, 0}
#define PHASE(i)                           \
    do {                                   \
        const long long ph_n = clock64();  \
        ph[i] += ph_n - ph_t;              \
        ph_t = ph_n;                       \
    } while (0)
#define PHASE_DUMP(steps)                                                                        \
    do {                                                                                         \
        if (threadIdx.x == 0) {                                                                  \
            for (int ph_i = 0; ph_i < 6; ++ph_i)                                                 \
                atomicAdd(&g_phase_cycles[ph_i], (unsigned long long)ph[ph_i]);                  \
            atomicAdd(&g_phase_cycles[6], (unsigned long long)(steps));                          \
        }                                                                                        \
    } while (0)
#else
#define PHASE_DECL
#define PHASE(i)
#define PHASE_DUMP(steps)
#endif
constexpr int kRing = 4;           // stage barriers per warp (stages in use: as many as fit)
constexpr int kChunkB = 4096;      // longest row segment of Q
constexpr int kWarpRingB = 8192;   // stage bytes per warp
constexpr size_t kRingBytes = (size_t)kWarps * kWarpRingB;

struct Smem {
    uint8_t* ring;   // per-warp Q stages while streaming; the check workspace otherwise
    double* xv;      // (in the ring) r x (mmax + 1): eigenvectors x_i of T_k
    double* band;    // (in the ring) per eigenvalue-owning warp 3 x (mmax + 1): U bands
    double* tri;     // (in the ring) 3 x (mmax + 1): scaled alpha, beta, beta^2 as double-FP32
    uint64_t* full;  // kWarps * kRing stage mbarriers
    double* vfull;   // max_n + 4 entries: the full current Lanczos vector
    double* vloc;    // rmax : this CTA's slice of v_j
    double* wloc;    // rmax : this CTA's slice of w
    double* part0;   // mmax + 2 : partial sums published to the cluster
    double* part1;   // mmax + 2
    double* cfull;   // mmax + 2 : reduced coefficients
    double* cdf;     // mmax + 2 : the same as double-FP32 pairs
    double* ecf;     // mmax + 2 : coefficients of the combined update (FP64)
    double* edf;     // mmax + 2 : the same as double-FP32 pairs
    double* alpha;   // mmax + 1
    double* beta;    // mmax + 1
    double* beta2;   // mmax + 1
    double* theta;   // kMaxR
    double* resid;   // kMaxR
    double* red;     // 64 : scratch
    double* sgn;     // 4 * kMaxR : (|max|, row, signed) per eigenvector, then sign flips
    double* ttmp;    // teams only: kMaxTeam x (mmax + 2), the clusters' partial sums
    float2* yoff;    // clusters alone: (cs / 2) x rows_max double-FP32 transposed sums of the range
};

__host__ __device__ inline int owned_max(int r, int cs) { return (r + cs - 1) / cs; }

// Rows of a CTA's slice at most: ceil(max_n / cs), rounded up to a multiple
// of 4 for the symmetric ranges' blocks.
__host__ __device__ inline int rows_max(int max_n, int cs) { return (int)round_up((max_n + cs - 1) / cs, 4); }

// Entries of the transposed sums of a symmetric range: at most cs / 2
// off-diagonal blocks of rows_max columns.
__host__ __device__ inline size_t yoff_entries(int max_n, int cs) {
    return (size_t)round_up((int64_t)(cs / 2) * rows_max(max_n, cs) + 4, 2);
}

// Doubles of the ring region: the Q stages or the check workspace, whichever is larger.
__host__ __device__ inline size_t ring_doubles(int cs, int mmax, int r) {
    const int own = owned_max(r, cs) < kWarps ? owned_max(r, cs) : kWarps;
    const size_t check = (size_t)(r + 3 * own + 3) * (mmax + 1);
    const size_t q = kRingBytes / 8;
    return (size_t)round_up((int64_t)(q > check ? q : check), 16);
}

__host__ __device__ inline size_t smem_doubles(int max_n, int cs, int mmax, int r, bool team = false) {
    const size_t rmax = (size_t)rows_max(max_n, cs);
    return ring_doubles(cs, mmax, r) + (size_t)kWarps * kRing + round_up(max_n + 4, 4) + 2 * rmax +
           6 * (size_t)(mmax + 2) + 3 * (size_t)(mmax + 1) + 2 * kMaxR + 64 + 4 * kMaxR + 8 +
           (team ? (size_t)kMaxTeam * (mmax + 2) : yoff_entries(max_n, cs));
}

__device__ Smem carve(double* base, int max_n, int cs, int mmax, int r, bool team = false) {
    Smem s;
    const int rmax = rows_max(max_n, cs);
    double* p = base;
    s.ring = reinterpret_cast<uint8_t*>(p);
    s.xv = p;
    s.band = p + (size_t)r * (mmax + 1);
    {
        const int own = owned_max(r, cs) < kWarps ? owned_max(r, cs) : kWarps;
        s.tri = s.band + (size_t)3 * own * (mmax + 1);
    }
    p += ring_doubles(cs, mmax, r);
    s.full = reinterpret_cast<uint64_t*>(p); p += kWarps * kRing;
    s.vfull = p; p += round_up(max_n + 4, 4);
    s.vloc = p; p += rmax;
    s.wloc = p; p += rmax;
    s.part0 = p; p += mmax + 2;
    s.part1 = p; p += mmax + 2;
    s.cfull = p; p += mmax + 2;
    s.cdf = p; p += mmax + 2;
    s.ecf = p; p += mmax + 2;
    s.edf = p; p += mmax + 2;
    s.alpha = p; p += mmax + 1;
    s.beta = p; p += mmax + 1;
    s.beta2 = p; p += mmax + 1;
    s.theta = p; p += kMaxR;
    s.resid = p; p += kMaxR;
    s.red = p; p += 64;
    s.sgn = p; p += 4 * kMaxR;
    s.ttmp = team ? p : nullptr;
    s.yoff = team ? nullptr : reinterpret_cast<float2*>(p);
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

// out[i] = sum over cluster ranks (in rank order) of part[i], lo <= i < hi;
// outdf (when not null) receives the sums as double-FP32 pairs.  Each thread
// issues its loads from all ranks before it adds any of them, so the remote
// latencies overlap instead of adding up.
__device__ void cluster_allreduce(cg::cluster_group& cl, double* part, double* out, double* outdf, int lo, int hi,
                                  int cs) {
    cl.sync();
    for (int i = lo + (int)threadIdx.x; i < hi; i += kThreads) {
        double s = 0.0;
        for (int q0 = 0; q0 < cs; q0 += 4) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = q0 + u < cs ? cl.map_shared_rank(part, q0 + u)[i] : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) s += v[u];
        }
        out[i] = s;
        if (outdf) reinterpret_cast<float2*>(outdf)[i] = df_of(s);
    }
    __syncthreads();
}

// put(i, get(i)) for 0 <= i < n, kUnroll independent loads in flight per
// thread before their stores.
constexpr int kUnroll = 4;
template <class G, class P, class T = double>
__device__ __forceinline__ void copy_unrolled(int n, G get, P put) {
    for (int i0 = threadIdx.x; i0 < n; i0 += kUnroll * kThreads) {
        T t[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int i = i0 + u * kThreads;
            t[u] = i < n ? get(i) : T(0);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int i = i0 + u * kThreads;
            if (i < n) put(i, t[u]);
        }
    }
}

template <class T, class G>
__device__ __forceinline__ void gather_unrolled(T* dst, int n, G get) {
    for (int i0 = threadIdx.x; i0 < n; i0 += kUnroll * kThreads) {
        T t[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int i = i0 + u * kThreads;
            t[u] = i < n ? get(i) : T(0);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int i = i0 + u * kThreads;
            if (i < n) dst[i] = t[u];
        }
    }
}

// ------------------------------------------------- tridiagonal eigen-work
//
// The checks work on T_k scaled by an exact power of two to norm ~1 (counts
// and eigenvectors do not change), in double-FP32 arithmetic: every FP64
// warp instruction occupies an SMSP's FP64 unit for tens of cycles on GB300,
// while these recurrences are short dependent chains of FP32 operations.

// Number of eigenvalues of T (a, b2 = beta^2, scaled) smaller than x: the sign
// changes of the Sturm sequence p_0 = 1, p_t = det(T_t - x I) =
// (a_{t-1} - x) p_{t-1} - b2_{t-2} p_{t-2} (a sign change between p_{t-1} and
// p_t is a negative pivot of T - x I = L D L^T).  No division: the pair
// (p_{t-1}, p_t) is rescaled by exact powers of two to stay in range, and an
// exact zero counts as a sign change (a tiny negative pivot).
__device__ int sturm_count_df(const float2* a, const float2* b2, int k, float2 x) {
    float2 pm = make_float2(1.f, 0.f), p = df_sub2(a[0], x);
    if (p.x == 0.f) p = make_float2(-0x1p-100f, 0.f);
    int c = p.x < 0.f;
    for (int t = 1; t < k; ++t) {
        float2 pn = df_sub2(df_mul2(df_sub2(a[t], x), p), df_mul2(b2[t - 1], pm));
        if (pn.x == 0.f) pn = make_float2(-p.x * 0x1p-40f, 0.f);
        c += (pn.x < 0.f) != (p.x < 0.f);
        pm = p;
        p = pn;
        const float ap = fabsf(p.x);
        if (ap > 0x1p+60f) {
            p = df_scale(p, 0x1p-60f);
            pm = df_scale(pm, 0x1p-60f);
        } else if (ap < 0x1p-60f && fabsf(pm.x) < 0x1p-60f) {
            p = df_scale(p, 0x1p+60f);
            pm = df_scale(pm, 0x1p+60f);
        }
    }
    return c;
}

// The i-th largest eigenvalue of T on [lo, hi] (count(lo) <= k-1-i < count(hi))
// by 32-way multisection: each lane of the calling warp counts at its own
// probe.  lo, hi and the result are unscaled FP64; the counts run on the
// scaled arrays at x * scale.  Stops at ~2^-44 relative width.
__device__ double kth_largest_df(const float2* a, const float2* b2, int k, int i, double lo, double hi,
                                 double scale) {
    const int lane = threadIdx.x & 31;
    const int target = k - 1 - i;
    for (int round = 0; round < 16; ++round) {
        const double step = (hi - lo) * (1.0 / 33.0);
        const double x = fmin(fma((double)(lane + 1), step, lo), hi);
        const unsigned ball = __ballot_sync(0xffffffffu, sturm_count_df(a, b2, k, df_of(x * scale)) > target);
        const int first = ball ? __ffs(ball) - 1 : 32;
        const double xf = __shfl_sync(0xffffffffu, x, first < 32 ? first : 31);
        const double xp = __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0);
        if (first < 32) hi = xf;
        if (first > 0) lo = xp;
        if (hi - lo <= 0x1p-44 * fmax(fabs(lo), fabs(hi))) break;
    }
    return 0.5 * (lo + hi);
}

// Inverse iteration for the eigenvector of T (a, b scaled) for eigenvalue th
// (scaled), by lane 0 of a warp, in shared memory: each iteration factors
// T - th I = P L U by Gaussian elimination with partial pivoting (U has the
// bands 1/u0, u1, u2) while it applies the same row operations to the
// right-hand side x, then solves with U from the bottom up.  Two iterations
// from a fixed positive start vector; x leaves with unit 2-norm.
__device__ void tri_inverse_iteration_df(const float2* a, const float2* b, int k, float2 th, float2 pert,
                                         float2* u0i, float2* u1, float2* u2, float2* x) {
    for (int t = 0; t < k; ++t) x[t] = make_float2(1.f + 0.25f * (float)((t * 7919) % 13) / 13.f, 0.f);
    const float2 zero = make_float2(0.f, 0.f);
    for (int it = 0; it < 2; ++it) {
        // working row t: entries (w0, w1) in columns t, t+1 and right-hand side yw
        float2 w0 = df_sub2(a[0], th), w1 = k > 1 ? b[0] : zero, yw = x[0];
        for (int t = 0; t < k - 1; ++t) {
            const float2 l0 = b[t];                            // row t+1, column t
            const float2 l1 = df_sub2(a[t + 1], th);           // row t+1, column t+1
            const float2 l2 = t + 2 < k ? b[t + 1] : zero;     // row t+1, column t+2
            const float2 yl = x[t + 1];
            if (fabsf(w0.x) >= fabsf(l0.x)) {                  // pivot on the working row
                if (w0.x == 0.f) w0 = pert;
                const float2 inv = df_rcp2(w0);
                const float2 f = df_mul2(l0, inv);
                u0i[t] = inv;
                u1[t] = w1;
                u2[t] = zero;
                x[t] = yw;
                w0 = df_sub2(l1, df_mul2(f, w1));
                w1 = l2;
                yw = df_sub2(yl, df_mul2(f, yw));
            } else {                                           // pivot on row t+1
                const float2 inv = df_rcp2(l0);
                const float2 f = df_mul2(w0, inv);
                u0i[t] = inv;
                u1[t] = l1;
                u2[t] = l2;
                x[t] = yl;
                w0 = df_sub2(w1, df_mul2(f, l1));
                w1 = df_mul2(make_float2(-f.x, -f.y), l2);
                yw = df_sub2(yw, df_mul2(f, yl));
            }
        }
        if (w0.x == 0.f) w0 = pert;
        u0i[k - 1] = df_rcp2(w0);
        x[k - 1] = df_mul2(yw, u0i[k - 1]);
        if (k > 1) x[k - 2] = df_mul2(df_sub2(x[k - 2], df_mul2(u1[k - 2], x[k - 1])), u0i[k - 2]);
        for (int t = k - 3; t >= 0; --t)
            x[t] = df_mul2(df_sub2(df_sub2(x[t], df_mul2(u1[t], x[t + 1])), df_mul2(u2[t], x[t + 2])), u0i[t]);
        // scale by a power of two (largest entry ~1), then to unit norm
        float mx = 0.f;
        for (int t = 0; t < k; ++t) mx = fmaxf(mx, fabsf(x[t].x));
        if (!(mx > 0.f) || !isfinite(mx)) mx = 1.f;
        int ex;
        frexpf(mx, &ex);
        const float sc = ldexpf(1.f, -ex);
        float sh = 0.f, sl = 0.f;
        for (int t = 0; t < k; ++t) {
            x[t] = df_scale(x[t], sc);
            df_madd(sh, sl, x[t].x, x[t].y, x[t].x, x[t].y);
        }
        const float2 inv = df_of(1.0 / sqrt((double)sh + (double)sl));
        for (int t = 0; t < k; ++t) x[t] = df_mul2(x[t], inv);
    }
}

// ------------------------------------------------------------------- teams
//
// A problem is solved by a team of G clusters of cs CTAs; G = 1 is the
// cluster alone (every batched problem).  A single large problem (a landmark
// set) uses G > 1 clusters of one cooperative launch: inside a cluster the
// exchanges go through DSMEM as before, across clusters through global memory
// behind a grid barrier (L2-only loads of the exchange buffers, bounded
// waits).  All CTAs of a team take the same decisions from the same sums.
struct Team {
    int G, g, T, qt;    // clusters, this cluster, CTAs in all, this CTA's rank
    double* v;          // n: the current Lanczos vector (G > 1)
    double* part;       // 2 x G x (mmax + 2): cluster partial sums, double-buffered
    double* theta;      // kMaxR
    double* resid;      // kMaxR
    double* xv;         // r x (mmax + 1)
    double* sgn;        // T x kMaxR x 3
    unsigned* bar;      // grid barrier: arrivals, generation
    int* abort;         // set when a barrier wait or a stage wait timed out
    int* sab;           // this CTA's shared copy of the abort word as rank 0 of its cluster saw it
    unsigned long long wait_ns;   // limit of a grid-barrier wait
};

// Grid barrier of the team: a cluster barrier, then thread 0 of each
// cluster's rank 0 arrives on the team counter (the last arrival opens the
// next generation) and waits, then a second cluster barrier releases the
// cluster.  Writes before the barrier are fenced; a wait longer than
// tm.wait_ns sets the team's abort word, after which every barrier returns
// at once.  Returns the abort word as rank 0 of this cluster read it after
// the wait -- the same answer on every CTA of the cluster, so the caller can
// leave the solve on all of them at the same point.
__device__ bool team_sync(cg::cluster_group& cl, const Team& tm) {
    __threadfence();
    cl.sync();
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
        volatile unsigned* gen = tm.bar + 1;
        const unsigned g0 = *gen;
        if (atomicAdd(tm.bar, 1u) == (unsigned)(tm.G - 1)) {
            atomicExch(tm.bar, 0u);
            __threadfence();
            atomicAdd(tm.bar + 1, 1u);
        } else {
            const unsigned long long t0 = tc::global_ns();
            while (*gen == g0) {
                if (*(volatile int*)tm.abort) break;
                if (tc::global_ns() - t0 > tm.wait_ns) {
                    atomicExch(tm.abort, 1);
                    break;
                }
            }
        }
        __threadfence();
        *tm.sab = *(volatile int*)tm.abort;
    }
    cl.sync();
    // every CTA reads rank 0's copy; rank 0 rewrites it only after the first
    // cluster barrier of the next call, which every reader reaches after its read
    return *cl.map_shared_rank(tm.sab, 0) != 0;
}

// Sum over the team of part[i], lo <= i < hi, into out (and outdf as
// double-FP32 pairs): cluster sums through DSMEM, then (G > 1) the clusters'
// sums in cluster order through the team buffers of parity pb.
// tmp: shared scratch of at least G x (hi - lo) doubles (the idle Q-stage ring).
// Returns true (on every CTA of the cluster) when the team barrier aborted;
// out is then not written.
__device__ bool team_allreduce(cg::cluster_group& cl, const Team& tm, int q, int cs, int mmax, int pb, double* part,
                               double* out, double* outdf, int lo, int hi, double* tmp) {
    cluster_allreduce(cl, part, out, tm.G > 1 ? nullptr : outdf, lo, hi, cs);
    if (tm.G == 1) return false;
    const int stride = mmax + 2, K = hi - lo;
    double* gp = tm.part + (size_t)pb * tm.G * stride;
    if (q == 0)
        for (int i = lo + (int)threadIdx.x; i < hi; i += kThreads) gp[(size_t)tm.g * stride + i] = out[i];
    if (team_sync(cl, tm)) return true;
    // every cluster's sums in one pass of independent loads, then the sum in cluster order
    gather_unrolled(tmp, tm.G * K, [&](int e) {
        const int h = e / K, i = e % K;
        return __ldcg(gp + (size_t)h * stride + lo + i);
    });
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += kThreads) {
        double sum = 0.0;
        for (int h = 0; h < tm.G; ++h) sum += tmp[h * K + i];
        out[lo + i] = sum;
        if (outdf) reinterpret_cast<float2*>(outdf)[lo + i] = df_of(sum);
    }
    __syncthreads();
    return false;
}

// The first half of a team reduction whose exchange comes later: partial
// sums part[lo..hi) of this CTA.  In a cluster alone the ranks read part[]
// through DSMEM after the next cluster barrier, so nothing moves now; in a
// team the cluster's sums (in rank order, through DSMEM) go to the team
// buffer of parity pb.  tmp: shared scratch of hi doubles.
__device__ void deferred_publish(cg::cluster_group& cl, const Team& tm, int q, int cs, int mmax, int pb,
                                 double* part, double* tmp, int lo, int hi) {
    if (tm.G == 1) return;
    cluster_allreduce(cl, part, tmp, nullptr, lo, hi, cs);
    double* gp = tm.part + (size_t)pb * tm.G * (mmax + 2);
    if (q == 0)
        for (int i = lo + (int)threadIdx.x; i < hi; i += kThreads) gp[(size_t)tm.g * (mmax + 2) + i] = tmp[i];
}

// The second half, after the exchange: out[lo..hi) (and outdf as double-FP32
// pairs) = the team's sums of the partials published with parity pb, in the
// same order on every CTA.  tmp: shared scratch of G x (hi - lo) doubles.
__device__ void deferred_collect(cg::cluster_group& cl, const Team& tm, int cs, int mmax, int pb, double* part,
                                 double* out, double* outdf, int lo, int hi, double* tmp) {
    if (tm.G == 1) {
        for (int i = lo + (int)threadIdx.x; i < hi; i += kThreads) {
            double s = 0.0;
            for (int q0 = 0; q0 < cs; q0 += 4) {
                double v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = q0 + u < cs ? cl.map_shared_rank(part, q0 + u)[i] : 0.0;
#pragma unroll
                for (int u = 0; u < 4; ++u) s += v[u];
            }
            out[i] = s;
            reinterpret_cast<float2*>(outdf)[i] = df_of(s);
        }
        __syncthreads();
        return;
    }
    const int stride = mmax + 2, K = hi - lo;
    const double* gp = tm.part + (size_t)pb * tm.G * stride;
    gather_unrolled(tmp, tm.G * K, [&](int e) {
        const int h = e / K, i = e % K;
        return __ldcg(gp + (size_t)h * stride + lo + i);
    });
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += kThreads) {
        double sum = 0.0;
        for (int h = 0; h < tm.G; ++h) sum += tmp[h * K + i];
        out[lo + i] = sum;
        reinterpret_cast<float2*>(outdf)[lo + i] = df_of(sum);
    }
    __syncthreads();
}

// Entry `row` of the fixed pseudo-random start vector (splitmix64 of the row
// index, mapped to [-1, 1)).
__device__ __forceinline__ double start_entry(int row) {
    // splitmix64 of the row index -> uniform in [-1, 1)
    uint64_t z = (uint64_t)row * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// ------------------------------------------------------ symmetric ranges
//
// The range of CTA q (see the header): blocks q, ..., q+m_q-1 of R columns,
// cyclically, read as the columns [a0, a0 + la) followed, once it wraps, by
// [0, lb).  The own block comes first: columns [0, wd) of the range.

constexpr int kSymCols = kChunkB / 4;   // longest symmetric range (one stage of FP32)

struct SymPlan {
    bool on;     // the symmetric matvec is in use for this problem
    int R;       // rows per CTA slice
    int a0, la;  // first piece of the range
    int lb;      // second piece (after the wrap), from column 0
    int wd;      // width of the own block
    int len;     // la + lb
};

__host__ __device__ inline int sym_blocks(int q, int cs) { return (cs - 1) / 2 + 1 + ((cs % 2 == 0 && q < cs / 2) ? 1 : 0); }

// Columns of block b (the last one includes the zero padding up to npad).
__host__ __device__ inline int sym_width(int b, int R, int npad) { return R < npad - b * R ? R : npad - b * R; }

// The plan of rank q; identical decisions on every CTA of the cluster.  The
// ranges are used when every CTA has rows and every range fits one stage
// (kSymCols columns, at most 8 float4 per lane).
__host__ __device__ inline SymPlan sym_plan(int n, int cs, int q, bool allowed) {
    SymPlan p;
    p.on = false;
    p.R = (n + cs - 1) / cs;
    p.a0 = p.la = p.lb = p.wd = p.len = 0;
    if (!allowed || cs < 3) return p;
    const int npad = (int)round_up(n, 4);
    const int R = (int)round_up(p.R, 4);
    if ((cs - 1) * R >= n) return p;
    for (int t = 0; t < cs; ++t) {
        int len = 0;
        for (int k = 0; k < sym_blocks(t, cs); ++k) len += sym_width((t + k) % cs, R, npad);
        if (len > kSymCols) return p;
    }
    const int last = q + sym_blocks(q, cs) - 1;   // the range's last block, before the wrap
    p.on = true;
    p.R = R;
    p.a0 = q * R;
    p.la = (last < cs && (last + 1) * R < npad ? (last + 1) * R : npad) - p.a0;
    p.lb = last < cs ? 0 : (last - cs + 1) * R;
    p.wd = sym_width(q, R, npad);
    p.len = p.la + p.lb;
    return p;
}

// ---------------------------------------------------------------- Q stream
//
// Warp w of a CTA owns rows [wr0, wr0 + per_step / nseg) of the CTA's slice
// and streams them as a periodic sequence of row segments (position pos =
// row-offset * nseg + segment) through its kRing stages, in order.  Stage
// indices and mbarrier phases carry over from problem to problem.
struct QStream {
    int nst, stride;    // stages in use and their spacing (bytes) for this problem
    const uint8_t* q;   // Q of the problem
    size_t rstride;     // bytes per row of Q (ldq * 8)
    int rowbytes;       // bytes a row's copies cover: FP32 round_up(n, 4) * 4, FP64 round_up(n, 2) * 8
    int nseg, segb;     // segments per row and bytes per segment (the last may be shorter)
    int aoff;           // symmetric range: byte offset in the row of its first column, else 0
    int abytes;         // symmetric range: bytes of its first piece (the rest is read from column 0), else 0
    int wr0, per_step;  // first row of this warp and segments per step
    uint8_t* ring;      // this warp's stages
    uint64_t* full;     // their mbarriers
    int cpos, ipos;     // stream positions of the next consume and the next issue
    int cst, ist;       // their stages
    int inflight;       // issued and not yet consumed
    int issue_left;     // issues still allowed
    uint32_t phase;     // parity each stage's next completion will have
};

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

// Issues chunks while a stage is free and issues are allowed (the whole warp
// keeps the bookkeeping; lane 0 issues).
__device__ __forceinline__ void qs_fill(QStream& s) {
    while (s.inflight < s.nst && s.issue_left > 0) {
        if ((threadIdx.x & 31) == 0) {
            const int row = s.wr0 + s.ipos / s.nseg, seg = s.ipos % s.nseg;
            const uint8_t* src = s.q + (size_t)row * s.rstride;
            uint8_t* dst = s.ring + (size_t)s.ist * s.stride;
            if (s.abytes == 0) {
                const int off = seg * s.segb;
                const int bytes = min(s.segb, s.rowbytes - off);
                tc::mbar_expect_tx(&s.full[s.ist], (uint32_t)bytes);
                tc::bulk_load(dst, src + off, (uint32_t)bytes, &s.full[s.ist]);
            } else {
                // a symmetric range (one segment): its first piece, then the
                // part past the wrap (from column 0) when there is one
                tc::mbar_expect_tx(&s.full[s.ist], (uint32_t)s.rowbytes);
                tc::bulk_load(dst, src + s.aoff, (uint32_t)s.abytes, &s.full[s.ist]);
                if (s.rowbytes > s.abytes)
                    tc::bulk_load(dst + s.abytes, src, (uint32_t)(s.rowbytes - s.abytes), &s.full[s.ist]);
            }
        }
        s.ipos = s.ipos + 1 == s.per_step ? 0 : s.ipos + 1;
        s.ist = s.ist + 1 == s.nst ? 0 : s.ist + 1;
        ++s.inflight;
        --s.issue_left;
    }
}

__device__ __forceinline__ bool qs_wait_front(QStream& s) {
    const bool ok = qs_wait(&s.full[s.cst], (s.phase >> s.cst) & 1u);
    s.phase ^= 1u << s.cst;
    return ok;
}

__device__ __forceinline__ void qs_pop(QStream& s) {
    s.cpos = s.cpos + 1 == s.per_step ? 0 : s.cpos + 1;
    s.cst = s.cst + 1 == s.nst ? 0 : s.cst + 1;
    --s.inflight;
}

// Waits for the chunks in flight and discards them; they are issued again
// from the same stream position later.  The warp's stages are then free.
__device__ __forceinline__ bool qs_drain(QStream& s) {
    bool ok = true;
    const int keep = s.cpos;
    while (s.inflight > 0) {
        ok = qs_wait_front(s) && ok;
        qs_pop(s);
    }
    s.cpos = s.ipos = keep;
    s.issue_left = 0;
    __syncwarp();
    return ok;
}

// Sets up the warp's stream for a problem and issues its first chunks: whole
// rows, or the symmetric range of sp (FP32 Q) in one segment per row.
template <bool DF>
__device__ __forceinline__ void qs_setup(QStream& s, const double* Q, int ldq, int n, int r0, int nr,
                                         const SymPlan& sp) {
    const int warp = threadIdx.x >> 5;
    const int per_warp = (nr + kWarps - 1) / kWarps;
    const int a = min(nr, warp * per_warp), b = min(nr, (warp + 1) * per_warp);
    s.q = reinterpret_cast<const uint8_t*>(Q);
    s.rstride = (size_t)ldq * 8;
    if (sp.on) {
        s.rowbytes = sp.len * 4;
        s.aoff = sp.a0 * 4;
        s.abytes = sp.la * 4;
        s.nseg = 1;
        s.segb = s.rowbytes;
    } else {
        s.rowbytes = DF ? (int)round_up(n, 4) * 4 : (int)round_up(n, 2) * 8;
        s.aoff = 0;
        s.abytes = 0;
        s.nseg = (s.rowbytes + kChunkB - 1) / kChunkB;
        s.segb = (int)round_up((s.rowbytes + s.nseg - 1) / s.nseg, 16);
    }
    s.wr0 = r0 + a;
    s.per_step = (b - a) * s.nseg;
    s.cpos = s.ipos = 0;
    // as many stages of this problem's segment size as the warp's ring holds
    // (the stream is drained between problems, so the stages restart at 0;
    // each stage's barrier keeps its own phase bit)
    s.stride = (int)round_up(s.segb, 128);
    s.nst = min(kRing, kWarpRingB / s.stride);
    s.cst = s.ist = 0;
    s.issue_left = min(s.nst, s.per_step);
    qs_fill(s);
}

// Re-issues the first chunks of the next step (after a drain).
__device__ __forceinline__ void qs_prime(QStream& s) {
    s.issue_left = min(s.nst, s.per_step);
    qs_fill(s);
}

// One step of the stream: w[row - r0] = Q[row, :] . v for the warp's rows.
// With prefetch the warp keeps issuing into the next step.
template <bool DF>
__device__ __forceinline__ bool qs_matvec(QStream& s, int n, int r0, const double* vfull, double* w,
                                          bool prefetch) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    s.issue_left = s.per_step - s.inflight + (prefetch ? min(s.nst, s.per_step) : 0);
    qs_fill(s);
    // FP32 Q and FP32 v: each lane keeps four FMA chains (one per entry of a
    // float4, ~8 entries per chain and row) that meet in double-FP32 at the
    // end of the row.  Rounding v and the chains' sums to FP32 moves the Ritz
    // values by ~1e-9 relative in a replay of the D&C problem (the FP32
    // storage of Q itself moves them more), for one FMA per entry.
    float sh = 0.f, sl = 0.f, th = 0.f, tl = 0.f;
    double acc = 0.0;
    for (int u = 0; u < s.per_step; ++u) {
        ok = qs_wait_front(s) && ok;
        const int row = s.wr0 + s.cpos / s.nseg, seg = s.cpos % s.nseg;
        const int bytes = min(s.segb, s.rowbytes - seg * s.segb);
        const uint8_t* stage = s.ring + (size_t)s.cst * s.stride;
        if constexpr (DF) {
            // FP32 Q: 4 entries per 16 bytes; the row's padding entries are zero
            // and so are the vector's guard entries
            const int col0 = seg * (s.segb / 4);
            const float4* v4 = reinterpret_cast<const float4*>(vfull) + (col0 >> 2);
            for (int t = lane; t < bytes / 16; t += 32) {
                const float4 x = reinterpret_cast<const float4*>(stage)[t];
                const float4 v = v4[t];
                sh = fmaf(x.x, v.x, sh);
                sl = fmaf(x.y, v.y, sl);
                th = fmaf(x.z, v.z, th);
                tl = fmaf(x.w, v.w, tl);
            }
        } else {
            const int col0 = seg * (s.segb / 8);
            for (int t = lane; t < bytes / 16; t += 32) {
                const int c = col0 + 2 * t;
                const double2 x = reinterpret_cast<const double2*>(stage)[t];
                const double2 vv = reinterpret_cast<const double2*>(vfull)[c >> 1];
                acc = fma(x.x, vv.x, acc);
                if (c + 1 < n) acc = fma(x.y, vv.y, acc);
            }
        }
        __syncwarp();
        qs_pop(s);
        qs_fill(s);   // the stage is free: next chunk of the periodic stream
        if (seg == s.nseg - 1) {
            if constexpr (DF) {
                float h = sh, l = 0.f;
                df_add(h, l, th, 0.f);
                df_add(h, l, sl, 0.f);
                df_add(h, l, tl, 0.f);
                df_warp_sum(h, l);
                if (lane == 0) reinterpret_cast<float2*>(w)[row - r0] = df_norm(h, l);
                sh = sl = th = tl = 0.f;
            } else {
                acc = warp_sum(acc);
                if (lane == 0) w[row - r0] = acc;
                acc = 0.0;
            }
        }
    }
    return ok;
}

// One step of the symmetric-range stream (FP32 Q, one segment per row).
// vv holds u_j over the range (own block first, so u_j[a] = vv[a - r0]).
// For each of the warp's rows a, the dot over the range goes to w[a - r0]
// (double-FP32: four FP32 FMA chains per lane, met at the row's end), and
// q_ab u_j[a] for the off-diagonal columns b gathers in FP32 chains per lane
// over the warp's rows (slot u of a lane holds float4 lane + 32u of the
// range on every row).  The warps then add their chains into yoff
// (double-FP32, entry b - wd of the range) in a fixed order: in round t warp
// w takes slot (w + t) mod 8, so no two warps touch one column in a round.
// One stage per row keeps each copy as large as the range: splitting rows
// into two stages of half the size (four in flight per warp instead of two)
// made this phase 1.5x slower.
constexpr int kSymF4 = 8;   // float4 slots per lane of a range: kSymCols / 128
static_assert(kSymF4 == kWarps && kSymCols == kSymF4 * 128, "one slot per warp and round");

__device__ __forceinline__ bool qs_matvec_sym(QStream& s, const SymPlan& sp, int r0, const float* vv, float2* w,
                                              float2* yoff, bool prefetch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool ok = true;
    s.issue_left = s.per_step - s.inflight + (prefetch ? min(s.nst, s.per_step) : 0);
    qs_fill(s);
    const int nf4 = sp.len >> 2, dg4 = sp.wd >> 2;
    const float4* v4 = reinterpret_cast<const float4*>(vv);
    float4 acc[kSymF4];
#pragma unroll
    for (int u = 0; u < kSymF4; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = 0; it < s.per_step; ++it) {
        ok = qs_wait_front(s) && ok;
        const int row = s.wr0 + s.cpos;
        const float4* st4 = reinterpret_cast<const float4*>(s.ring + (size_t)s.cst * s.stride);
        const float xa = vv[row - r0];
        float sh = 0.f, sl = 0.f, th = 0.f, tl = 0.f;
#pragma unroll
        for (int u = 0; u < kSymF4; ++u) {
            const int g = lane + 32 * u;
            if (g < nf4) {
                const float4 x = st4[g];
                const float4 v = v4[g];
                sh = fmaf(x.x, v.x, sh);
                sl = fmaf(x.y, v.y, sl);
                th = fmaf(x.z, v.z, th);
                tl = fmaf(x.w, v.w, tl);
                if (g >= dg4) {
                    acc[u].x = fmaf(x.x, xa, acc[u].x);
                    acc[u].y = fmaf(x.y, xa, acc[u].y);
                    acc[u].z = fmaf(x.z, xa, acc[u].z);
                    acc[u].w = fmaf(x.w, xa, acc[u].w);
                }
            }
        }
        __syncwarp();
        qs_pop(s);
        qs_fill(s);
        float h = sh, l = 0.f;
        df_add(h, l, th, 0.f);
        df_add(h, l, sl, 0.f);
        df_add(h, l, tl, 0.f);
        df_warp_sum(h, l);
        if (lane == 0) w[row - r0] = df_norm(h, l);
    }
    for (int t = 0; t < kSymF4; ++t) {
        const int u = (warp + t) & (kSymF4 - 1);
        float4 a = acc[0];
#pragma unroll
        for (int k = 1; k < kSymF4; ++k)
            if (k == u) a = acc[k];
        const int g = lane + 32 * u;
        if (g < nf4 && g >= dg4) {
            float2* y = yoff + 4 * (g - dg4);
            if (t == 0) {
                y[0] = make_float2(a.x, 0.f);
                y[1] = make_float2(a.y, 0.f);
                y[2] = make_float2(a.z, 0.f);
                y[3] = make_float2(a.w, 0.f);
            } else {
                const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float2 c = y[e];
                    df_add(c.x, c.y, av[e], 0.f);
                    y[e] = c;
                }
            }
        }
        __syncthreads();
    }
    return ok;
}

// After every CTA's qs_matvec_sym and a cluster barrier: w[rr] (the row dots
// of this CTA's rows) += the transposed sums of the CTAs whose ranges hold
// this CTA's block, in rank order.
__device__ __forceinline__ void sym_collect(cg::cluster_group& cl, const SymPlan& sp, int n, int cs, int q, int nr,
                                            float2* w, float2* yoff) {
    const int npad = (int)round_up(n, 4);
    for (int rr = threadIdx.x; rr < nr; rr += kThreads) {
        float2 t = w[rr];
        for (int p = 0; p < cs; ++p) {
            const int k = (q - p + cs) % cs;
            if (k < 1 || k >= sym_blocks(p, cs)) continue;
            int off = 0;
            for (int kk = 1; kk < k; ++kk) off += sym_width((p + kk) % cs, sp.R, npad);
            const float2 y = cl.map_shared_rank(yoff, p)[off + rr];
            df_add(t.x, t.y, y.x, y.y);
        }
        w[rr] = df_norm(t.x, t.y);
    }
}

// ------------------------------------------------------------ Gram-Schmidt
//
// B is written by this kernel (new Lanczos vectors), so it must never be read
// through the non-coherent read-only path: no __restrict__ on it.

// part[i] = sum over this CTA's rows of B[i][row] * w[row] for ia <= i <= ib
// (one warp per i, two vectors at a time); with_norm also sets part[ib + 1] =
// sum of w[row]^2.
template <bool DF>
__device__ void cgs_dots(const double* B, int ldq, int r0, int nr, int ia, int ib, const double* w, double* part,
                         bool with_norm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (DF) {
        const float2* w2 = reinterpret_cast<const float2*>(w);
        if (with_norm && warp == (ib + 1) % kWarps) {
            float sh = 0.f, sl = 0.f;
            for (int rr = lane; rr < nr; rr += 32) {
                const float2 x = w2[rr];
                df_madd(sh, sl, x.x, x.y, x.x, x.y);
            }
            df_warp_sum(sh, sl);
            if (lane == 0) part[ib + 1] = (double)sh + (double)sl;
        }
        // FP32 basis: per lane FMA chains b * w_hi and b * w_lo, met in double-FP32
        for (int i = ia + warp; i <= ib; i += 2 * kWarps) {
            const int i2 = i + kWarps;
            const bool two = i2 <= ib;
            const float* b1 = reinterpret_cast<const float*>(B) + (int64_t)i * ldq + r0;
            const float* b2 = reinterpret_cast<const float*>(B) + (int64_t)(two ? i2 : i) * ldq + r0;
            float c1h = 0.f, c1l = 0.f, c2h = 0.f, c2l = 0.f;
            for (int rr = lane; rr < nr; rr += 32) {
                const float2 x = w2[rr];
                const float a1 = b1[rr], a2 = b2[rr];
                c1h = fmaf(a1, x.x, c1h);
                c1l = fmaf(a1, x.y, c1l);
                c2h = fmaf(a2, x.x, c2h);
                c2l = fmaf(a2, x.y, c2l);
            }
            float h1 = c1h, l1 = 0.f, h2 = c2h, l2 = 0.f;
            df_add(h1, l1, c1l, 0.f);
            df_add(h2, l2, c2l, 0.f);
            df_warp_sum(h1, l1);
            df_warp_sum(h2, l2);
            if (lane == 0) {
                part[i] = (double)h1 + (double)l1;
                if (two) part[i2] = (double)h2 + (double)l2;
            }
        }
    } else {
        if (with_norm && warp == (ib + 1) % kWarps) {
            double s0 = 0.0;
            for (int rr = lane; rr < nr; rr += 32) s0 = fma(w[rr], w[rr], s0);
            s0 = warp_sum(s0);
            if (lane == 0) part[ib + 1] = s0;
        }
        for (int i = ia + warp; i <= ib; i += kWarps) {
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
}

// w[row] -= sum_{ia <= i <= ib} B[i][row] * c[i] (thread per row); c as FP64
// (cf) and as double-FP32 pairs (cd).
template <bool DF>
__device__ void cgs_update(const double* B, int ldq, int r0, int nr, int ia, int ib, const double* cf,
                           const double* cd, double* w) {
    if constexpr (DF) {
        const float2* c2 = reinterpret_cast<const float2*>(cd);
        float2* w2 = reinterpret_cast<float2*>(w);
        for (int rr = threadIdx.x; rr < nr; rr += kThreads) {
            const float* b = reinterpret_cast<const float*>(B) + r0 + rr;   // FP32 basis
            float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
            int i = ia;
            for (; i + 1 <= ib; i += 2) {
                const float x0 = b[(int64_t)i * ldq], x1 = b[(int64_t)(i + 1) * ldq];
                const float2 k0 = c2[i], k1 = c2[i + 1];
                df_madd1(h0, l0, x0, k0.x, k0.y);
                df_madd1(h1, l1, x1, k1.x, k1.y);
            }
            if (i <= ib) {
                const float x0 = b[(int64_t)i * ldq];
                const float2 k0 = c2[i];
                df_madd1(h0, l0, x0, k0.x, k0.y);
            }
            df_add(h0, l0, h1, l1);
            const float2 wv = w2[rr];
            float sh = wv.x, sl = wv.y;
            df_add(sh, sl, -h0, -l0);
            w2[rr] = df_norm(sh, sl);
        }
    } else {
        for (int rr = threadIdx.x; rr < nr; rr += kThreads) {
            const double* b = B + r0 + rr;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int i = ia;
            for (; i + 3 <= ib; i += 4) {
                s0 = fma(b[(int64_t)i * ldq], cf[i], s0);
                s1 = fma(b[(int64_t)(i + 1) * ldq], cf[i + 1], s1);
                s2 = fma(b[(int64_t)(i + 2) * ldq], cf[i + 2], s2);
                s3 = fma(b[(int64_t)(i + 3) * ldq], cf[i + 3], s3);
            }
            for (; i <= ib; ++i) s0 = fma(b[(int64_t)i * ldq], cf[i], s0);
            w[rr] -= (s0 + s1) + (s2 + s3);
        }
    }
}

// ------------------------------------------------------------ one problem

// One eigenproblem (part pj) solved by the calling cluster.
// Leaving a team solve after an aborted grid barrier: every CTA of the
// cluster gets here at the same point (the barrier's answer is
// cluster-consistent).  The warp's bulk copies still in flight are waited for
// (full limit: their source is ordinary device memory), a cluster barrier
// keeps every CTA's shared memory alive until its peers are done with it, and
// the problem reports MDS_ERR_TIMEOUT.
__device__ void team_abort_exit(const LanczosArgs& A, int pj, cg::cluster_group& cl, QStream& Qs, int qt, int k) {
    qs_drain(Qs);
    __syncthreads();
    cl.sync();
    if (qt == 0 && threadIdx.x == 0) {
        A.status[pj] = kDevTimeout;
        A.steps[pj] = k;
    }
}

template <bool DF>
__device__ void solve_problem(const LanczosArgs& A, int pj, cg::cluster_group& cl, int cs, int q, const Smem& S,
                              int& s_flag, QStream& Qs, const Team& tm) {
    const ProbDesc P = A.desc[pj];
    const int n = P.n, ldq = P.ldq, r = A.r;
    const int T = tm.T, qt = tm.qt;   // CTAs of the team and this CTA's rank (cs, q when G = 1)
    const SymPlan sp = sym_plan(n, cs, q, DF && tm.G == 1 && A.sym != 0);
    const int R = tm.G > 1 ? (n + T - 1) / T : sp.R;
    const int r0 = min(n, qt * R), r1 = min(n, r0 + R), nr = r1 - r0;
    const double* Q = A.qarena + P.q_off;
    double* B = A.barena + P.b_off;
    const int kmax = min(A.mmax, n);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = A.mmax + 1;
    // per-problem global scratch: the final tridiagonal T_k (diagonal, off-diagonal)
    double* scr = A.scratch + (size_t)pj * lanczos_scratch_per_problem(A.mmax, r);
    double* part[2] = {S.part0, S.part1};
    int pb = 0;
    bool qok = true;

    // start streaming this warp's rows of Q right away
    qs_setup<DF>(Qs, Q, ldq, n, r0, nr, sp);

    // ---- start vector: pseudo-random, unit norm
    double loc = 0.0;
    for (int i = tid; i < nr; i += kThreads) {
        const double v = start_entry(r0 + i);
        S.wloc[i] = v;
        loc += v * v;
    }
    {
        const double s = block_sum(loc, S.red);
        if (tid == 0) part[pb][0] = s;
        if (team_allreduce(cl, tm, q, cs, A.mmax, pb, part[pb], S.cfull, nullptr, 0, 1, S.ttmp)) {
            team_abort_exit(A, pj, cl, Qs, qt, 0);
            return;
        }
        pb ^= 1;
        if (tid == 0) S.red[kWarps + 3] = 1.0 / sqrt(S.cfull[0]);
        __syncthreads();
        const double inv = S.red[kWarps + 3];
        for (int i = tid; i < nr; i += kThreads) {
            const double v = S.wloc[i] * inv;
            if constexpr (DF) {
                // the basis holds FP32; the gathered v_0 is that same value
                const float f = (float)v;
                reinterpret_cast<float*>(S.vloc)[i] = f;   // the published vector is FP32
                reinterpret_cast<float*>(B)[r0 + i] = f;
            } else {
                S.vloc[i] = v;
                B[r0 + i] = v;
            }
            if (tm.G > 1) {
                if constexpr (DF) reinterpret_cast<float*>(tm.v)[r0 + i] = reinterpret_cast<const float*>(S.vloc)[i];
                else tm.v[r0 + i] = S.vloc[i];
            }
        }
    }
    if (tid == 0) {
        for (int i = n; i < (int)round_up(n, 4); ++i) {   // guard entries of the padded loads
            if constexpr (DF) reinterpret_cast<float*>(S.vfull)[i] = 0.f;
            else S.vfull[i] = 0.0;
        }
        S.red[40] = 0.0;    // tnorm
    }

    const int kmin = min(kmax, max(2 * r, 8));
    int next_check = kmin;
    PHASE_DECL;
    double prev_worst = -1.0;
    int k = 0, prev_k = 0;
    bool converged = false, have_vectors = false;
    bool aborted = false;   // a team barrier aborted: every CTA of the cluster leaves together

    // Step j orthogonalises w = Q u_j against the two newest vectors (one
    // exchange), giving w_1, and publishes w_1 with its partial dots against
    // v_0..v_j and ||w_1||^2.  The exchange that opens step j+1 carries both,
    // so every CTA completes the second pass on its own rows -- w_2 = w_1 -
    // sum c'_i v_i, beta_j^2 = ||w_1||^2 - ||c'||^2, v_{j+1} = w_2 / beta_j --
    // with no reduction of its own.  The matvec of step j+1 takes u_{j+1} =
    // w_1 / beta_j as gathered; it differs from the stored v_{j+1} by
    // |c'| / beta_j, the rounding-level loss of orthogonality the second pass
    // removes from the basis.
    for (int j = 0;; ++j) {
        // ---- exchange: every rank's published vector and, from step 1 on,
        // its deferred partial sums
        if (tm.G > 1) {
            if (team_sync(cl, tm)) {
                aborted = true;
                break;
            }
            if constexpr (DF)
                gather_unrolled(reinterpret_cast<float*>(S.vfull), n,
                                [&](int i) { return __ldcg(reinterpret_cast<const float*>(tm.v) + i); });
            else
                gather_unrolled(S.vfull, n, [&](int i) { return __ldcg(tm.v + i); });
        } else if (sp.on) {
            // the range's columns, own block first (zero past n)
            cl.sync();
            gather_unrolled(reinterpret_cast<float*>(S.vfull), sp.len, [&](int g) {
                const int c = g < sp.la ? sp.a0 + g : g - sp.la;
                if (c >= n) return 0.f;
                const int src = c / R;
                return reinterpret_cast<const float*>(cl.map_shared_rank(S.vloc, src))[c - src * R];
            });
        } else {
            cl.sync();
            if constexpr (DF)
                gather_unrolled(reinterpret_cast<float*>(S.vfull), n, [&](int i) {
                    const int src = i / R;
                    return reinterpret_cast<const float*>(cl.map_shared_rank(S.vloc, src))[i - src * R];
                });
            else
                gather_unrolled(S.vfull, n, [&](int i) {
                    const int src = i / R;
                    return cl.map_shared_rank(S.vloc, src)[i - src * R];
                });
        }
        if (j > 0) {
            deferred_collect(cl, tm, cs, A.mmax, pb, part[pb], S.cfull, S.cdf, 0, j + 1, S.ttmp);
            pb ^= 1;
            // alpha_{j-1} and beta_{j-1} from the second pass
            if (warp == 0) {
                double c2 = 0.0;
                for (int i = lane; i < j; i += 32) c2 = fma(S.cfull[i], S.cfull[i], c2);
                c2 = warp_sum(c2);
                if (lane == 0) {
                    const double alpha = S.alpha[j - 1] + S.cfull[j - 1];
                    const double beta = sqrt(fmax(S.cfull[j] - c2, 0.0));
                    const double tn = fmax(S.red[40], fabs(alpha) + 2.0 * beta);
                    S.alpha[j - 1] = alpha;
                    S.beta[j - 1] = beta;
                    S.beta2[j - 1] = beta * beta;
                    S.red[40] = tn;
                    S.red[41] = (beta <= 1e-12 * tn || j == n) ? 1.0 : 0.0;
                    S.red[42] = beta > 0.0 ? 1.0 / beta : 0.0;
                    S.red[47] = S.cfull[j - 1];   // d_{j-1}: see alpha_j below
                }
            }
            // the second pass on this CTA's rows: w_2 (in wloc) ...
            cgs_update<DF>(B, ldq, r0, nr, 0, j - 1, S.cfull, S.cdf, S.wloc);
            __syncthreads();
            // ... and what Q (u_j - v_j) = sum_i d_i Q v_i / beta_{j-1} adds to the
            // next matvec along v_m, from the three-term relation
            // Q v_i = beta_{i-1} v_{i-1} + alpha_i v_i + beta_i v_{i+1}:
            // e_m = (d_{m+1} beta_m + d_m alpha_m + d_{m-1} beta_{m-1}) / beta_{j-1}.
            // The update after the next matvec removes it (m <= j-2; the pass
            // against v_{j-1}, v_j measures its own coefficients), so that the
            // one-pass completion never sees components that grow step to step.
            for (int m = tid; m <= j - 2; m += kThreads) {
                double t = S.cfull[m] * S.alpha[m] + S.cfull[m + 1] * S.beta[m];
                if (m >= 1) t += S.cfull[m - 1] * S.beta[m - 1];
                t *= S.red[42];
                S.ecf[m] = t;
                reinterpret_cast<float2*>(S.edf)[m] = df_of(t);
            }
            // ... v_j = w_2 / beta_{j-1} into the basis, and u_j = w_1 / beta_{j-1}
            // (the gathered vector) for the matvec
            if constexpr (DF) {
                const float2 binv = df_of(S.red[42]);
                for (int rr = tid; rr < nr; rr += kThreads) {
                    const float2 v = df_mul(reinterpret_cast<const float2*>(S.wloc)[rr], binv);
                    reinterpret_cast<float*>(B)[(int64_t)j * ldq + r0 + rr] = __fadd_rn(v.x, v.y);
                }
                const float bf = __fadd_rn(binv.x, binv.y);
                const int nv = sp.on ? sp.len : n;
                for (int i = tid; i < nv; i += kThreads) reinterpret_cast<float*>(S.vfull)[i] *= bf;
            } else {
                const double binv = S.red[42];
                for (int rr = tid; rr < nr; rr += kThreads) B[(int64_t)j * ldq + r0 + rr] = S.wloc[rr] * binv;
                for (int i = tid; i < n; i += kThreads) S.vfull[i] *= binv;
            }
        }
        __syncthreads();
        k = j;
        const double beta_j = j > 0 ? S.beta[j - 1] : 0.0;   // beta_{k-1}: the residual coefficient
        const double tnorm = S.red[40];
        const bool breakdown = j > 0 && S.red[41] != 0.0;
        const bool do_check = j > 0 && (breakdown || k == kmax || k >= next_check);
        PHASE(0);
        if (do_check && k >= r) {
            // the stage rings hold the check's workspace from here on
            qok = qs_drain(Qs) && qok;
            __syncthreads();
            // Ritz values and residuals.  Eigenvalue i belongs to CTA i % cs and,
            // there, to warp i / cs: every FP64 warp instruction occupies an
            // SMSP's FP64 unit for tens of cycles, so the r bisections run on as
            // many SMSPs of the cluster as possible.  Each owner finds theta_i
            // (bisection on Sturm counts, warm-bracketed by the previous check),
            // the eigenvector x_i of T_k (inverse iteration) and the residual
            // beta_j |x_i[k-1]|; all CTAs then read every theta and residual
            // through DSMEM and take the same decision.
            const int mine = (r - qt + T - 1) / T;  // eigenvalues owned by this CTA
            // T_k scaled by a power of two to norm ~1, as double-FP32 arrays
            int ex;
            frexp(tnorm, &ex);
            const double scale = ldexp(1.0, -ex);
            float2* adf = reinterpret_cast<float2*>(S.tri);
            float2* bdf = adf + L;
            float2* b2df = bdf + L;
            if (mine > 0)
                for (int t = tid; t < k; t += kThreads) {
                    adf[t] = df_of(S.alpha[t] * scale);
                    bdf[t] = df_of(S.beta[t] * scale);
                    b2df[t] = df_of(S.beta2[t] * (scale * scale));
                }
            __syncthreads();
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
                const float2 pert = df_of(0x1p-44 * fmax(tnorm * scale, 0.5));
                float2* bd = reinterpret_cast<float2*>(S.band + (size_t)warp * 3 * L);
                for (int m = warp; m < mine; m += kWarps) {   // one warp per eigenvalue
                    const int i = qt + T * m;
                    double lo = gl, hi = gu;
                    if (have_vectors) {
                        // lane 0 tests the lower end, lane 1 the upper end of the warm bracket
                        const int target = k - 1 - i;
                        const double t0 = S.theta[i];
                        const double t1 = t0 + 4.0 * S.resid[i] + 0x1p-38 * fabs(t0);   // above the counts' resolution
                        const double xt = lane == 0 ? t0 : t1;
                        const int c = sturm_count_df(adf, b2df, k, df_of(xt * scale));
                        const int c0 = __shfl_sync(0xffffffffu, c, 0), c1 = __shfl_sync(0xffffffffu, c, 1);
                        if (t0 > gl && c0 <= target) lo = t0;
                        if (t1 < gu && t1 > lo && c1 > target) hi = t1;
                    }
                    const double th = kth_largest_df(adf, b2df, k, i, lo, hi, scale);
                    double* x = S.xv + (size_t)i * L;
                    float2* xf = reinterpret_cast<float2*>(x);
                    if (lane == 0) {
                        tri_inverse_iteration_df(adf, bdf, k, df_of(th * scale), pert, bd, bd + L, bd + 2 * L, xf);
                        S.theta[i] = th;
                        S.resid[i] = beta_j * fabs((double)xf[k - 1].x + (double)xf[k - 1].y);
                    }
                    __syncwarp();
                    for (int t = lane; t < k; t += 32) x[t] = (double)xf[t].x + (double)xf[t].y;   // in place
                    __syncwarp();
                }
            }
            if (tm.G > 1) {
                // owners publish theta and residuals; every CTA reads them all
                __syncthreads();
                for (int i = tid; i < r; i += kThreads)
                    if (i % T == qt) {
                        tm.theta[i] = S.theta[i];
                        tm.resid[i] = S.resid[i];
                    }
                if (team_sync(cl, tm)) {
                    aborted = true;
                    break;
                }
                for (int i = tid; i < r; i += kThreads) {
                    S.theta[i] = __ldcg(tm.theta + i);
                    S.resid[i] = __ldcg(tm.resid + i);
                }
            } else {
                cl.sync();
                for (int i = tid; i < r; i += kThreads) {
                    const int owner = i % cs;
                    if (owner != q) {
                        S.theta[i] = cl.map_shared_rank(S.theta, owner)[i];
                        S.resid[i] = cl.map_shared_rank(S.resid, owner)[i];
                    }
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
            if (tm.G > 1) __syncthreads();
            else cl.sync();  // owners keep theta/resid until every CTA has read them
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
                // one problem on the whole GPU: a check costs ~3 steps, so trust
                // the extrapolation further; batched parts overshoot costlier
                gap = (int)fmin(A.p == 1 ? 32.0 : 16.0, fmax(2.0, ceil(need) + 1.0));
            } else if (worst < 1e-6) {
                gap = 4;
            }
            prev_worst = worst;
            prev_k = k;
            next_check = k + gap;
            if (!breakdown) qs_prime(Qs);   // the stages are Q stages again
        }
        PHASE(1);
        if (breakdown || k == kmax) break;  // breakdown with k < r: fewer Ritz values than wanted

        // ---- w = Q u_j on this CTA's rows (streamed); no prefetch into a step
        // that starts with a predicted check
        if (sp.on) {
            qok = qs_matvec_sym(Qs, sp, r0, reinterpret_cast<const float*>(S.vfull), reinterpret_cast<float2*>(S.wloc),
                                S.yoff, j + 1 < next_check && j + 1 < kmax) && qok;
            cl.sync();   // every CTA's row dots and transposed sums are complete
            sym_collect(cl, sp, n, cs, q, nr, reinterpret_cast<float2*>(S.wloc), S.yoff);
        } else {
            qok = qs_matvec<DF>(Qs, n, r0, S.vfull, S.wloc, j + 1 < next_check && j + 1 < kmax) && qok;
        }
        __syncthreads();
        PHASE(2);

        // ---- pass against v_{j-1}, v_j: w_1 = w - c_{j-1} v_{j-1} - c_j v_j
        const int ia = j > 0 ? j - 1 : 0;
        cgs_dots<DF>(B, ldq, r0, nr, ia, j, S.wloc, part[pb], false);
        __syncthreads();
        if (team_allreduce(cl, tm, q, cs, A.mmax, pb, part[pb], S.cfull, S.cdf, ia, j + 1, S.ttmp)) {
            aborted = true;
            break;
        }
        pb ^= 1;
        // alpha_j = v_j . Q v_j; the matvec saw u_j = v_j + sum_i d_i v_i / beta_{j-1},
        // whose extra part adds e_j = v_j . Q v_{j-1} d_{j-1} / beta_{j-1} = d_{j-1}
        // to c_j; the second pass of this step adds its own coefficient later
        if (tid == 0) S.alpha[j] = S.cfull[j] - (j > 0 ? S.red[47] : 0.0);
        if (j >= 2) {
            // one update with e_0..e_{j-2} and the measured c_{j-1}, c_j
            if (tid < 2) {
                S.ecf[j - 1 + tid] = S.cfull[j - 1 + tid];
                S.edf[j - 1 + tid] = S.cdf[j - 1 + tid];
            }
            __syncthreads();
            cgs_update<DF>(B, ldq, r0, nr, 0, j, S.ecf, S.edf, S.wloc);
        } else {
            cgs_update<DF>(B, ldq, r0, nr, ia, j, S.cfull, S.cdf, S.wloc);
        }
        __syncthreads();
        PHASE(3);

        // ---- publish w_1 and its partial dots against v_0..v_j with ||w_1||^2
        cgs_dots<DF>(B, ldq, r0, nr, 0, j, S.wloc, part[pb], true);
        __syncthreads();
        deferred_publish(cl, tm, q, cs, A.mmax, pb, part[pb], S.cfull, 0, j + 2);
        for (int rr = tid; rr < nr; rr += kThreads) {
            if constexpr (DF) {
                // the matvec input is published in FP32 (the basis is FP32 too)
                const float2 w = reinterpret_cast<const float2*>(S.wloc)[rr];
                const float f = __fadd_rn(w.x, w.y);
                reinterpret_cast<float*>(S.vloc)[rr] = f;
                if (tm.G > 1) reinterpret_cast<float*>(tm.v)[r0 + rr] = f;
            } else {
                S.vloc[rr] = S.wloc[rr];
                if (tm.G > 1) tm.v[r0 + rr] = S.wloc[rr];
            }
        }
        PHASE(4);
    }

    // ---- finish: status, orthonormal eigenvectors of T_k (rank 0), Ritz vectors (all)
    if (aborted) {
        team_abort_exit(A, pj, cl, Qs, qt, k);
        return;
    }
    qok = qs_drain(Qs) && qok;
    bool any_timeout = false;
    if (tm.G > 1) {
        if (!qok) atomicExch(tm.abort, 1);
        if (team_sync(cl, tm)) {
            team_abort_exit(A, pj, cl, Qs, qt, k);
            return;
        }
    } else {
        if (!qok) S.red[43] = 1.0;   // zero since the last problem; every writer stores 1
        __syncthreads();
        cl.sync();
        for (int qq = 0; qq < cs; ++qq) any_timeout |= cl.map_shared_rank(S.red, qq)[43] == 1.0;
        cl.sync();   // every CTA has read the flags before S.red is reused
        if (tid == 0) S.red[43] = 0.0;
    }
    int status = kDevOk;
    if (k < r || !have_vectors) {
        status = kDevRank;
    } else {
        if (!converged) status = kDevNoConv;
        if (!(S.theta[r - 1] > 0.0) || !(S.theta[r - 1] > A.rank_tol * S.theta[0])) status = kDevRank;
    }
    if (any_timeout) status = kDevTimeout;
    // rank 0 of the team collects the eigenvectors of T_k from their owners,
    // orthonormalises them (modified Gram-Schmidt, warp 0, shared memory) and
    // every other CTA copies the result
    auto mgs = [&]() {
        for (int i = 0; i < r; ++i) {
            double* xi = S.xv + (size_t)i * L;
            for (int m = 0; m < i; ++m) {
                const double* xm = S.xv + (size_t)m * L;
                double sm = 0.0;
                for (int t = lane; t < k; t += 32) sm += xi[t] * xm[t];
                sm = warp_sum(sm);
                for (int t = lane; t < k; t += 32) xi[t] -= sm * xm[t];
                __syncwarp();
            }
            double sm = 0.0;
            for (int t = lane; t < k; t += 32) sm += xi[t] * xi[t];
            sm = warp_sum(sm);
            const double inv = 1.0 / sqrt(sm);
            for (int t = lane; t < k; t += 32) xi[t] *= inv;
            __syncwarp();
        }
    };
    if (tm.G > 1) {
        if (status != kDevRank)
            for (int e = tid; e < r * k; e += kThreads) {
                const int i = e / k, t = e % k;
                if (i % T == qt) tm.xv[(size_t)i * L + t] = S.xv[(size_t)i * L + t];
            }
        if (team_sync(cl, tm)) {
            team_abort_exit(A, pj, cl, Qs, qt, k);
            return;
        }
        if (qt == 0 && status != kDevRank) {
            copy_unrolled(
                r * k, [&](int e) { return __ldcg(tm.xv + (size_t)(e / k) * L + e % k); },
                [&](int e, double v) { S.xv[(size_t)(e / k) * L + e % k] = v; });
            __syncthreads();
            if (warp == 0) mgs();
            __syncthreads();
            for (int e = tid; e < r * k; e += kThreads) {
                const int i = e / k, t = e % k;
                tm.xv[(size_t)i * L + t] = S.xv[(size_t)i * L + t];
            }
        }
        if (team_sync(cl, tm)) {
            team_abort_exit(A, pj, cl, Qs, qt, k);
            return;
        }
        if (status == kDevRank) {
            if (qt == 0 && tid == 0) {
                A.status[pj] = status;
                A.steps[pj] = k;
            }
            return;
        }
        if (qt != 0)
            copy_unrolled(
                r * k, [&](int e) { return __ldcg(tm.xv + (size_t)(e / k) * L + e % k); },
                [&](int e, double v) { S.xv[(size_t)(e / k) * L + e % k] = v; });
        __syncthreads();
    } else {
        if (q == 0 && status != kDevRank) {
            copy_unrolled(
                r * k,
                [&](int e) {
                    const int i = e / k;
                    const size_t o = (size_t)i * L + e % k;
                    return i % cs != 0 ? cl.map_shared_rank(S.xv, i % cs)[o] : S.xv[o];
                },
                [&](int e, double v) { S.xv[(size_t)(e / k) * L + e % k] = v; });
            __syncthreads();
        }
        if (q == 0 && status != kDevRank && warp == 0) mgs();
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
            copy_unrolled(
                r * k, [&](int e) { return src[(size_t)(e / k) * L + e % k]; },
                [&](int e, double v) { S.xv[(size_t)(e / k) * L + e % k] = v; });
        }
        cl.sync();   // rank 0's vectors have been copied before any CTA rewrites its own
    }
    if constexpr (DF) {
        // s_i as double-FP32 pairs, in place
        for (int e = tid; e < r * k; e += kThreads) {
            const int i = e / k, t = e % k;
            double* p = S.xv + (size_t)i * L + t;
            *reinterpret_cast<float2*>(p) = df_of(*p);
        }
    }
    __syncthreads();

    // Ritz vectors y_i = V_k s_i for this CTA's rows; per-column |max| for the sign rule.
    double* V = A.varena + P.v_off;
    for (int rr = tid; rr < nr; rr += kThreads) {
        if constexpr (DF) {
            const float* b = reinterpret_cast<const float*>(B) + r0 + rr;   // FP32 basis
            for (int ig = 0; ig < r; ig += 8) {
                float h[8], l[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) h[u] = l[u] = 0.f;
                for (int t = 0; t < k; ++t) {
                    const float x = b[(int64_t)t * ldq];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (ig + u < r) {
                            const float2 sv = reinterpret_cast<const float2*>(S.xv + (size_t)(ig + u) * L)[t];
                            df_madd1(h[u], l[u], x, sv.x, sv.y);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (ig + u < r) V[(int64_t)(r0 + rr) * r + ig + u] = (double)h[u] + (double)l[u];
            }
        } else {
            for (int i = 0; i < r; ++i) {
                const double* si = S.xv + (size_t)i * L;
                double s = 0.0;
                for (int t = 0; t < k; ++t) s = fma(B[(int64_t)t * ldq + r0 + rr], si[t], s);
                V[(int64_t)(r0 + rr) * r + i] = s;
            }
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
    double* flip = S.sgn + 3 * kMaxR;  // kMaxR slots after the (|max|, row, value) triples
    if (tm.G > 1) {
        __syncthreads();
        for (int e = tid; e < 3 * r; e += kThreads) tm.sgn[(size_t)qt * 3 * kMaxR + e] = S.sgn[e];
        if (team_sync(cl, tm)) {
            team_abort_exit(A, pj, cl, Qs, qt, k);
            return;
        }
        if (tid < r) {
            double best = -1.0, bestv = 0.0, brow = 1e300;
            for (int qq = 0; qq < T; ++qq) {
                const double* o = tm.sgn + (size_t)qq * 3 * kMaxR + 3 * tid;
                const double o0 = __ldcg(o), o1 = __ldcg(o + 1), o2 = __ldcg(o + 2);
                if (o0 > best || (o0 == best && o1 < brow)) {
                    best = o0;
                    brow = o1;
                    bestv = o2;
                }
            }
            flip[tid] = bestv < 0.0 ? -1.0 : 1.0;
        }
        __syncthreads();
    } else {
        cl.sync();
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
    }
    for (int rr = tid; rr < nr; rr += kThreads)
        for (int i = 0; i < r; ++i) V[(int64_t)(r0 + rr) * r + i] *= flip[i];
    if (qt == 0 && tid == 0) {
        for (int i = 0; i < r; ++i) A.lam[(size_t)pj * r + i] = S.theta[i];
        A.status[pj] = status;
        A.steps[pj] = k;
    }
    if (qt == 0)
        for (int t = tid; t < k; t += kThreads) {
            scr[t] = S.alpha[t];
            scr[L + t] = S.beta[t];
        }
    PHASE(5);
    PHASE_DUMP(k);
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
    __shared__ int s_flag, s_next, s_abort;
    const Smem S = carve(smraw, A.max_n, cs, A.mmax, A.r, A.team > 1);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kWarps * kRing; ++i) tc::mbar_init(&S.full[i], 1);
        S.red[43] = 0.0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    QStream Qs;
    Qs.ring = S.ring + (size_t)(threadIdx.x >> 5) * kWarpRingB;
    Qs.full = S.full + (threadIdx.x >> 5) * kRing;
    Qs.nst = 1;
    Qs.stride = kWarpRingB;
    Qs.cst = Qs.ist = 0;
    Qs.inflight = 0;
    Qs.phase = 0;
    Team tm;
    tm.G = A.team > 1 ? A.team : 1;
    tm.g = (int)blockIdx.x / cs;
    tm.T = tm.G * cs;
    tm.qt = tm.G > 1 ? (int)blockIdx.x : q;
    {
        double* t = A.tscr;
        tm.v = t;
        t += round_up(A.max_n, 4);
        tm.part = t;
        t += (size_t)2 * tm.G * (A.mmax + 2);
        tm.theta = t;
        t += kMaxR;
        tm.resid = t;
        t += kMaxR;
        tm.xv = t;
        t += (size_t)A.r * (A.mmax + 1);
        tm.sgn = t;
        tm.bar = A.tbar;
        tm.abort = reinterpret_cast<int*>(A.tbar + 2);
        tm.sab = &s_abort;
        tm.wait_ns = A.wait_ns ? A.wait_ns : tc::kWaitNs;
    }
    if (tm.G > 1) {   // one problem for the whole team
        solve_problem<DF>(A, A.order[0], cl, cs, q, S, s_flag, Qs, tm);
        return;
    }
    for (;;) {
        if (q == 0 && threadIdx.x == 0) s_next = atomicAdd(A.counter, 1);
        cl.sync();
        const int next = q == 0 ? s_next : *cl.map_shared_rank(&s_next, 0);
        cl.sync();  // every CTA has read the index before rank 0 takes another
        if (next >= A.p) break;
        solve_problem<DF>(A, A.order[next], cl, cs, q, S, s_flag, Qs, tm);
    }
}

thread_local int g_last_team = 0;

}  // namespace

double lanczos_step_bytes(int n, int cs, int q_f32, int sym, int team) {
    if (!q_f32) return (double)n * round_up(n, 2) * 8;
    const SymPlan p0 = sym_plan(n, cs, 0, sym && !team);
    if (!p0.on) return (double)n * round_up(n, 4) * 4;
    double b = 0.0;
    for (int q = 0; q < cs; ++q) {
        const SymPlan p = sym_plan(n, cs, q, true);
        const int r0 = q * p.R < n ? q * p.R : n;
        const int nr = (r0 + p.R < n ? r0 + p.R : n) - r0;
        b += (double)nr * p.len * 4;
    }
    return b;
}

int lanczos_last_team() { return g_last_team; }

int lanczos_phase_cycles(double* out, int reset) {
#ifdef GBMDS_PHASE_TIMERS
    unsigned long long h[8] = {};
    if (reset) return cudaMemcpyToSymbol(g_phase_cycles, h, sizeof(h)) == cudaSuccess ? 0 : MDS_ERR_CUDA;
    if (cudaMemcpyFromSymbol(h, g_phase_cycles, sizeof(h)) != cudaSuccess) return MDS_ERR_CUDA;
    for (int i = 0; i < 7; ++i) out[i] = (double)h[i];
    return 0;
#else
    (void)out;
    (void)reset;
    return MDS_ERR_UNSUPPORTED;
#endif
}

size_t lanczos_smem_bytes(int max_n, int cs, int mmax, int r) {
    return smem_doubles(max_n, cs, mmax, r) * sizeof(double) + kMaxR * sizeof(double);
}

size_t lanczos_team_scratch_doubles(int max_n, int mmax, int r) {
    return (size_t)round_up(max_n, 4) + (size_t)2 * kMaxTeam * (mmax + 2) + 2 * kMaxR + (size_t)r * (mmax + 1) +
           (size_t)kMaxTeam * 8 * 3 * kMaxR;
}

// A single problem spread over G clusters of 8 CTAs (one CTA per SM) in one
// cooperative launch.  Returns cudaErrorNotSupported when the problem is too
// small or the launch form is not available (the caller then uses one cluster).
template <bool DF>
static cudaError_t launch_lanczos_team(LanczosArgs a, cudaStream_t st) {
    constexpr int cs = 8;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // as many clusters as fit, down to 8 rows per CTA: the steps' FP64 dot
    // products and updates spread over more SMs (l = 1,000: 2.85 ms with 7
    // clusters, 2.61 with 12, 2.60 with 15 or 19; l = 2,000: 8.16 ms from 15 on)
    int G = std::min(std::min(sms / cs, kMaxTeam), a.max_n / (cs * 8));
    if (G < 2) return cudaErrorNotSupported;
    const size_t need = smem_doubles(a.max_n, cs, a.mmax, a.r, true) * sizeof(double);
    if (need > kMaxSmem) return cudaErrorNotSupported;
    const size_t smem = need < 120 * 1024 ? 120 * 1024 : need;   // one CTA per SM
    cudaError_t e = cudaFuncSetAttribute(k_lanczos<DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(G * cs));
    int resident = 0;
    e = cudaOccupancyMaxActiveClusters(&resident, k_lanczos<DF>, &cfg);
    if (e != cudaSuccess) return e;
    G = std::min(G, resident);
    if (G < 2) return cudaErrorNotSupported;
    cfg.gridDim = dim3((unsigned)(G * cs));
    cfg.numAttrs = 2;
    a.team = G;
    e = cudaLaunchKernelEx(&cfg, k_lanczos<DF>, a);
    if (e == cudaSuccess) note_launch(1);
    return e;
}

template <bool DF>
static cudaError_t launch_lanczos_t(const LanczosArgs& a, int cs, cudaStream_t st) {
    const size_t need = smem_doubles(a.max_n, cs, a.mmax, a.r) * sizeof(double);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Few CTAs in all (a single landmark problem, say): one CTA per SM, so a
    // cluster spreads over as many SMs as it has CTAs.  Many: two per SM, so
    // one CTA's reductions and checks overlap the other's Q stream.
    const size_t one_per_sm = 120 * 1024;
    const size_t smem = (size_t)a.p * cs <= (size_t)sms && need < one_per_sm ? one_per_sm : need;
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

cudaError_t launch_lanczos(const LanczosArgs& a, int cluster, cudaStream_t st, bool allow_team) {
    if (a.p <= 0) return cudaSuccess;
    g_last_team = 0;
    if (allow_team && a.p == 1 && a.tscr) {
        const cudaError_t e = a.q_f32 ? launch_lanczos_team<true>(a, st) : launch_lanczos_team<false>(a, st);
        if (e == cudaSuccess) {
            g_last_team = 1;
            return e;
        }
        cudaGetLastError();   // not available: one cluster below
    }
    LanczosArgs b = a;
    b.team = 1;
    const int cs = cluster < 1 ? 1 : (cluster > 16 ? 16 : cluster);
    return b.q_f32 ? launch_lanczos_t<true>(b, cs, st) : launch_lanczos_t<false>(b, cs, st);
}

}  // namespace gbmds
