// Fast MDS (Section 3.3): the data are divided at random into p = floor(l/s)
// subsets, recursively while a subset has more than l points; classical MDS
// runs on the leaves; at every inner node the first s points (the sampling
// points) of each subset form the alignment set, whose classical MDS is the
// alignment configuration, and each subset's configuration is mapped onto it
// by Procrustes on its sampling points.
//
// Every classical-MDS problem of the recursion (each leaf, and each inner
// node's alignment set) depends on the data rows only, so all of them run in
// one batched eigen-solver launch.  What remains is a chain of small affine
// maps: the map of node k onto its parent's frame, (T_k, t_k), found bottom
// up one tree level at a time, and the leaves' rows written once through the
// composition of the maps on their path to the root.  This file holds the
// gather of the alignment rows, the preparation of each Procrustes task (the
// alignment rows of the parent, and the child's first s rows in the child's
// own frame), the composition of the maps and the output.
#include "common.cuh"

namespace gbmds {
namespace {

// own_all[g.x + t] = perm[g.y + t], t < s: the sampling points of one subset
// copied into its parent's alignment set.
__global__ void k_fast_gather(const int64_t* __restrict__ perm, const longlong2* __restrict__ copies, int s,
                              int64_t* __restrict__ own_all) {
    const longlong2 g = copies[blockIdx.x];
    for (int t = threadIdx.x; t < s; t += blockDim.x) own_all[g.x + t] = perm[g.y + t];
}

__device__ __forceinline__ void apply_map(double* x, const double* __restrict__ M, int r) {
    double y[kMaxR];
    const double* t = M + r * r;
    for (int i = 0; i < r; ++i) {
        double v = t[i];
        for (int m = 0; m < r; ++m) v += x[m] * M[m * r + i];
        y[i] = v;
    }
    for (int i = 0; i < r; ++i) x[i] = y[i];
}

// Task k: A = rows row0 .. row0 + s - 1 of the alignment problem's
// configuration V Lambda^{1/2}; B = rows 0 .. s - 1 of the leftmost leaf below
// the child, mapped through the maps of the chain chain[off .. off + len)
// (the nodes from that leaf up to, not including, the child).  Written to
// AB + k * 2 s r.
__global__ void __launch_bounds__(128) k_fast_prep(const ProbDesc* __restrict__ desc,
                                                   const double* __restrict__ varena,
                                                   const double* __restrict__ lam, int r, int s,
                                                   const FastTask* __restrict__ tasks, const int* __restrict__ chain,
                                                   const double* __restrict__ maps, double* __restrict__ AB) {
    const FastTask T = tasks[blockIdx.x];
    double* A = AB + (size_t)blockIdx.x * 2 * s * r;
    double* B = A + (size_t)s * r;
    const double* Va = varena + desc[T.align_prob].v_off;
    const double* Vl = varena + desc[T.leaf_prob].v_off;
    const double* la = lam + (size_t)T.align_prob * r;
    const double* ll = lam + (size_t)T.leaf_prob * r;
    for (int a = threadIdx.x; a < s; a += blockDim.x) {
        double x[kMaxR];
        for (int m = 0; m < r; ++m) {
            A[(int64_t)a * r + m] = Va[(int64_t)(T.row0 + a) * r + m] * sqrt(la[m]);
            x[m] = Vl[(int64_t)a * r + m] * sqrt(ll[m]);
        }
        for (int q = 0; q < T.chain_len; ++q) apply_map(x, maps + (size_t)chain[T.chain_off + q] * (r * r + r), r);
        for (int m = 0; m < r; ++m) B[(int64_t)a * r + m] = x[m];
    }
}

// Leaf k's map to the root frame: the composition of the maps of the nodes
// chain[off .. off + len) (leaf first): (T, t) <- (T T_q, t T_q + t_q).
__global__ void k_fast_compose(const int2* __restrict__ leaf_chain, const int* __restrict__ chain,
                               const double* __restrict__ maps, int r, double* __restrict__ lmaps) {
    __shared__ double T[kMaxR * kMaxR + kMaxR], N[kMaxR * kMaxR + kMaxR];
    const int2 lc = leaf_chain[blockIdx.x];
    const int rr = r * r + r;
    for (int e = threadIdx.x; e < rr; e += blockDim.x) T[e] = (e < r * r && e / r == e % r) ? 1.0 : 0.0;
    __syncthreads();
    for (int q = 0; q < lc.y; ++q) {
        const double* M = maps + (size_t)chain[lc.x + q] * rr;
        for (int e = threadIdx.x; e < rr; e += blockDim.x) {
            const int i = e < r * r ? e / r : -1, j = e < r * r ? e % r : e - r * r;
            double v = i >= 0 ? 0.0 : M[r * r + j];
            const double* row = i >= 0 ? T + i * r : T + r * r;   // a row of T, or t
            for (int m = 0; m < r; ++m) v += row[m] * M[m * r + j];
            N[e] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rr; e += blockDim.x) T[e] = N[e];
        __syncthreads();
    }
    for (int e = threadIdx.x; e < rr; e += blockDim.x) lmaps[(size_t)blockIdx.x * rr + e] = T[e];
}

// Row a of leaf problem blockIdx.y: X[own[own_off + a]] = (V_a Lambda^{1/2}) T + t.
template <typename A>
__global__ void __launch_bounds__(256) k_fast_out(const ProbDesc* __restrict__ desc, const double* __restrict__ varena,
                                                  const double* __restrict__ lam, const double* __restrict__ lmaps,
                                                  int r, const int64_t* __restrict__ own, A* __restrict__ X) {
    const int j = blockIdx.y;
    const ProbDesc P = desc[j];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= P.n) return;
    const double* V = varena + P.v_off + (int64_t)a * r;
    const double* M = lmaps + (size_t)j * (r * r + r);
    double x[kMaxR];
    for (int m = 0; m < r; ++m) x[m] = V[m] * sqrt(lam[(size_t)j * r + m]);
    apply_map(x, M, r);
    const int64_t row = member_row(P, nullptr, own, a);
    for (int i = 0; i < r; ++i) X[row * r + i] = (A)x[i];
}

}  // namespace

cudaError_t launch_fast_gather(const int64_t* perm, const longlong2* copies, int ncopies, int s, int64_t* own_all,
                               cudaStream_t st) {
    if (ncopies <= 0) return cudaSuccess;
    k_fast_gather<<<ncopies, 128, 0, st>>>(perm, copies, s, own_all);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_fast_prep(const ProbDesc* desc, const double* varena, const double* lam, int r, int s,
                             const FastTask* tasks, int ntasks, const int* chain, const double* maps, double* AB,
                             cudaStream_t st) {
    if (ntasks <= 0) return cudaSuccess;
    k_fast_prep<<<ntasks, 128, 0, st>>>(desc, varena, lam, r, s, tasks, chain, maps, AB);
    note_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_fast_finish(const ProbDesc* desc, int nleaves, int max_leaf, const double* varena,
                               const double* lam, const int2* leaf_chain, const int* chain, const double* maps, int r,
                               double* lmaps, const int64_t* own, int out_f64, void* X, cudaStream_t st) {
    if (nleaves <= 0) return cudaSuccess;
    k_fast_compose<<<nleaves, 128, 0, st>>>(leaf_chain, chain, maps, r, lmaps);
    const dim3 grid((unsigned)((max_leaf + 255) / 256), (unsigned)nleaves);
    if (out_f64) k_fast_out<double><<<grid, 256, 0, st>>>(desc, varena, lam, lmaps, r, own, (double*)X);
    else k_fast_out<float><<<grid, 256, 0, st>>>(desc, varena, lam, lmaps, r, own, (float*)X);
    note_launch(2);
    return cudaGetLastError();
}

}  // namespace gbmds
