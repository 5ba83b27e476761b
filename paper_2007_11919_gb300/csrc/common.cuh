// Internal declarations shared by the libgbmds translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gbmds.h"

// Device-resident landmark configuration behind an mds_model handle.
struct mds_model_s {
    int l, d, r, prec, device;
    int kind;       // 0: FP64/FP32 rows or BF16 split planes; 1 + kTckBf16 / 1 + kTckFp8:
                    // byte rows encoded for k_gower_tck (norms and W padded to tck_lpad(l))
    void* L;        // landmark rows: l x d double (F64), l x d float (F32), or BF16
                    // split planes hi | lo of l x split_ld(d) each (BF16)
    double* nrm_l;  // l squared norms of the rows as stored in L (F64 / F32 models)
    float* nrm_lf;  // the same as float (BF16 models)
    void* W;        // l x r Gower operator -1/2 V Lambda^{-1/2}
    double* bias;   // r: 1/2 Lambda^{-1/2} V^T q_1
    void* X1;       // l x r landmark configuration
    double* lam;    // r eigenvalues of Q_1
};

namespace gbmds {

constexpr int kMaxR = 32;          // largest supported target dimension r
constexpr int kMaxEigN = 16384;    // largest eigenproblem (points)
constexpr int kTile = 64;          // distance tile edge (points)
constexpr int kDtBF16 = 100;       // internal dtype tag: BF16 hi/lo split planes of the data

// One classical-MDS eigenproblem of a batch (the landmark set of Section 3.1,
// or one part of Section 3.2).  Row a of the problem is data row
//   a <  c : anchors[a]
//   a >= c : own[own_off + a - c]
// All offsets are in elements of the arena they index.
struct ProbDesc {
    int64_t own_off;   // first own row in the own-index array
    int64_t q_off;     // Q_j (n x ldq, row-major FP64) in the Q arena
    int64_t rp_off;    // per-tile row sums (tiles x n FP64) in the row-part arena
    int64_t rm_off;    // row means (n FP64) in the row-mean arena
    int64_t b_off;     // Lanczos basis ((mmax+1) x ldq, column j at j*ldq) in the basis arena
    int64_t v_off;     // top-r eigenvectors (n x r, row-major FP64) in the V arena
    int32_t n;         // points in the problem
    int32_t ldq;       // leading dimension of Q_j and of the basis (n rounded up to 4)
    int32_t c;         // leading anchor rows (0 = none)
    int32_t tiles;     // ceil(n / kTile)
    int64_t ny;        // rows of the data matrix (indices are clamped to [0, ny))
};

// Device-side status codes written per problem (a subset of mds_status).
enum DevStatus : int { kDevOk = 0, kDevRank = MDS_ERR_RANK, kDevNoConv = MDS_ERR_NOCONV, kDevTimeout = MDS_ERR_TIMEOUT };

__host__ __device__ inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Out-of-range caller indices are clamped so that no access leaves Y; the
// host reports them separately (k_check_idx) as MDS_ERR_ARG.
__device__ __forceinline__ int64_t member_row(const ProbDesc& P, const int64_t* anchors,
                                              const int64_t* own, int a) {
    const int64_t g = a < P.c ? anchors[a] : own[P.own_off + (a - P.c)];
    return g < 0 ? 0 : (g >= P.ny ? P.ny - 1 : g);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Loads element k of a row as the accumulation type.
template <typename A, typename T>
__device__ __forceinline__ A load_as(const T* p) { return static_cast<A>(*p); }
template <>
__device__ __forceinline__ float load_as<float, uint8_t>(const uint8_t* p) { return (float)(*p); }
template <>
__device__ __forceinline__ double load_as<double, uint8_t>(const uint8_t* p) { return (double)(*p); }
template <>
__device__ __forceinline__ float load_as<float, __nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}

// Kernel launches made by the current host thread (for mds_last_stats).
void note_launch(int count);

// Row readers for the CUDA-core kernels.  RowLoad: element k of row i of a
// row-major matrix with leading dimension ld.  SplitLoad: BF16 split data,
// value = hi + lo, with the hi plane at p and the lo plane at p + plane.
template <typename T>
struct RowLoad {
    const T* p;
    int64_t ld;
    template <typename A>
    __device__ __forceinline__ A get(int64_t i, int k) const { return load_as<A, T>(p + i * ld + k); }
};
struct SplitLoad {
    const __nv_bfloat16* p;
    int64_t ld, plane;
    template <typename A>
    __device__ __forceinline__ A get(int64_t i, int k) const {
        const __nv_bfloat16* q = p + i * ld + k;
        return (A)__bfloat162float(q[0]) + (A)__bfloat162float(q[plane]);
    }
};

// Padded row length (elements) of the BF16 split planes: 16-byte rows.
__host__ __device__ inline int split_ld(int d) { return (int)round_up(d, 8); }

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `st` and returns cudaGetLastError().

// Squared row norms of an n x d matrix into nrm (length n, FP64 storage),
// accumulated in A (float or double).
cudaError_t launch_rownorm(const void* Y, int dt, int64_t n, int d, int acc_f64, double* nrm,
                           cudaStream_t st);
// The same for rows idx[0..count-1] of an ny x d matrix only, each written at
// nrm[idx[i]] (the other entries of nrm are left as they are).
cudaError_t launch_rownorm_idx(const void* Y, int dt, int64_t ny, int d, const int64_t* idx, int64_t count,
                               int acc_f64, double* nrm, cudaStream_t st);

// Delta_j tiles for every problem of a batch into the Q arena, plus per-tile
// row sums.  acc_f64 selects FP64 (else FP32) dot products; Delta is stored
// as FP64 when acc_f64 or out_f64 is set, else as FP32 rows (row stride
// 2 * ldq floats) for an FP32 Q.
cudaError_t launch_sqdist_batched(const void* Y, int dt, int d, const double* nrm,
                                  const int64_t* anchors, const int64_t* own,
                                  const ProbDesc* desc, int p, int max_tiles, int acc_f64, int out_f64,
                                  double* qarena, double* rparena, cudaStream_t st);

// Copy an external n x n FP64 squared-distance matrix into problem 0's Q slot
// and form its per-tile row sums.
cudaError_t launch_load_dist(const double* D2, const ProbDesc* desc, double* qarena,
                             double* rparena, int n, int tiles, cudaStream_t st);

// Double centering in place: Q = -1/2 (Delta - m 1^T - 1 m^T + g) per problem,
// computed in FP64; stored as FP64, or (q_f32) as FP32 at the start of each
// row's storage (row stride 2 * ldq floats, zero-padded to a multiple of 4).
cudaError_t launch_center_batched(const ProbDesc* desc, int p, int max_n, double* qarena,
                                  const double* rparena, double* rmarena, double* grand, int q_f32,
                                  cudaStream_t st);

struct LanczosArgs {
    const ProbDesc* desc;
    int p;
    const double* qarena;
    double* barena;
    double* varena;
    double* lam;        // p x r
    int* status;        // p
    int* steps;         // p
    double* scratch;    // p x lanczos_scratch_per_problem(mmax, r) doubles
    const int* order;   // p problem indices, the order in which clusters take them
    int q_f32;          // Q stored as FP32 (row stride 2 * ldq floats), vectors in double-FP32
    int* counter;       // queue head, zero before the launch
    int r;
    int mmax;
    double tol;
    double rank_tol;
    int max_n;
    int team;           // clusters sharing one problem (1 = the cluster alone)
    double* tscr;       // team exchange buffers (lanczos_team_scratch_doubles)
    unsigned* tbar;     // team barrier words [arrivals, generation, abort], zero before the launch
    int sym;            // FP32 Q in a cluster alone: read each off-diagonal block of Q once (symmetric ranges)
    unsigned long long wait_ns;   // limit of a team grid-barrier wait (0 = the default 2 s)
};
constexpr int kMaxTeam = 32;   // clusters per team
size_t lanczos_team_scratch_doubles(int max_n, int mmax, int r);
__host__ __device__ inline size_t lanczos_scratch_per_problem(int mmax, int r) {
    return (size_t)(r * 7 + 2) * (mmax + 1) + 8;
}
cudaError_t launch_lanczos(const LanczosArgs& a, int cluster, cudaStream_t st, bool allow_team);
// Bytes of Q one Lanczos step streams for an n x n problem: whole rows, or
// the symmetric ranges of a cluster of cs CTAs (q_f32, sym, not a team).
double lanczos_step_bytes(int n, int cs, int q_f32, int sym, int team);
// 1 when the last launch_lanczos on this thread ran a team of clusters.
int lanczos_last_team();
// The phase-timer build's cycle counters (7 values; reset = 1 zeroes them);
// MDS_ERR_UNSUPPORTED in a build without them.
int lanczos_phase_cycles(double* out, int reset);
// Shared memory one CTA of the eigen-solver needs for a cluster of cs CTAs.
size_t lanczos_smem_bytes(int max_n, int cs, int mmax, int r);
constexpr size_t kMaxSmem = 220 * 1024;

// Interpolation model from the landmark eigenpairs (FP64):
//   X1 = V Lambda^{1/2};  W = -1/2 V Lambda^{-1/2};  b = 1/2 Lambda^{-1/2} V^T q1.
// W and X1 are written in double (w64/x1_64) and float (w32/x1_32) when the
// pointers are not null.
cudaError_t launch_interp_model(const double* V, const double* lam, const double* Qdiag_src,
                                int ldq, int q_f32, int l, int r, double* w64, float* w32,
                                double* x1_64, float* x1_32, double* bias, double* var_out,
                                cudaStream_t st);

// Affine form of Eq. (2) for coordinate rows, from the gathered landmark rows
// Lg (dense l x d FP64): y_L (FP64 and FP32 copies), scale = Lambda^{-1/2} and
// U_r = L_c^T V Lambda^{-1/2} (d x r, both copies); then launch_affine_project
// gives X = (Y - y_L) U_r for all n rows (double X when f64, else float).
cudaError_t launch_affine_axes(const double* Lg, int l, int d, const double* V, const double* lam, int r,
                               double* scale, double* ybar, float* ybar_f, double* U, float* U_f, cudaStream_t st);
// The pieces (k_affine.cu): row mean of a dense l x d FP64 matrix; axes
// U[k][i] = scale_i sum_j (L[j][k] - c_k) V[j][i]; projection X = (Y - 1 c^T) U
// (FP64 when f64, else FP32 with the FP32 copies cen_f, U_f).
cudaError_t launch_rows_mean(const double* L, int l, int d, double* mean, float* mean_f, cudaStream_t st);
cudaError_t launch_axes(const double* L, int l, int d, const double* c, const double* V, const double* scale, int r,
                        double* U, float* U_f, cudaStream_t st);
// err (device, non-null) receives MDS_ERR_TIMEOUT if a bounded wait on a tile
// copy gives up.
cudaError_t launch_affine_project(const void* Y, int dt, int64_t n, int d, const double* cen, const float* cen_f,
                                  const double* U, const float* U_f, int r, int f64, void* X, int* err,
                                  cudaStream_t st);

// Pivot MDS pieces (k_pivot.cu): column means of all n rows (partials of
// colmean_part_doubles(n, d)), the scatter matrix S = Y_c^T Y_c (d x d FP64,
// partials of scatter_part_doubles(n, d); f64 = FP64 products, else FP32
// products in double-FP32 sums), FP64 products C = (A - 1 ca^T)(B - 1 cb^T)^T,
// the scale factors from the eigenvalues of C^T C, and the sign convention on
// the columns of X (partials of colsign_grid(n) x r pairs).
size_t colmean_part_doubles(int64_t n, int d);
size_t scatter_part_doubles(int64_t n, int d);
int colsign_grid(int64_t n);
cudaError_t launch_colmean(const void* Y, int dt, int64_t n, int d, double* part, double* mean, float* mean_f,
                           cudaStream_t st);
cudaError_t launch_scatter(const void* Y, int dt, int64_t n, int d, const double* mean, int f64, double* part,
                           double* S, cudaStream_t st);
// sym: the product is known to be symmetric (m == nb); the upper tiles are
// computed and mirrored.
cudaError_t launch_gemm_nt(const double* A, int lda, const double* ca, const double* B, int ldb, const double* cb,
                           int m, int nb, int K, double* C, int ldc, int sym, cudaStream_t st);
// Whether the scatter matrix kernel takes rows of width d (d <= 4096).
bool scatter_supported(int d);

// Persistent tuning cache (tune.cu): off unless a file is named.  Keys name a
// kernel and every quantity its launch choice depends on.
bool tune_enabled();
bool tune_lookup(const std::string& key, int* value, double* trial_ms, int ntrial);
bool tune_store(const std::string& key, int value, const double* trial_ms, int ntrial);
std::string lanczos_tune_key(int p, int max_n, double sum_n2, int mmax, int r, int q_f32, int sym);
cudaError_t launch_pivot_scale(const double* mu, int r, int64_t n, int l, double* scale, double* var,
                               cudaStream_t st);
cudaError_t launch_colsign(void* X, int out_f64, int64_t n, int r, double* part_v, int64_t* part_i, unsigned* counter,
                           double* sign, cudaStream_t st);

// Gather rows Y[idx[i]] into a dense l x d matrix of the accumulation type.
// For dt == kDtBF16, Y is the split planes of an ny-row matrix.
cudaError_t launch_gather_rows(const void* Y, int dt, int64_t ny, int d, const int64_t* idx,
                               int l, int acc_f64, void* out, const double* nrm_src,
                               double* nrm_out, cudaStream_t st);

// Gower projection, Eq. (2): X_i = sum_j a2_ij W_j + b for m rows of Y
// (FP32 or FP64 SIMT distance tiles).  For dt == kDtBF16, Y is split planes.
cudaError_t launch_gower_proj(const void* Y, int dt, int64_t m, int d, const double* nrm_y,
                              const void* L, const double* nrm_l, int l, const void* W,
                              const double* bias, int r, int acc_f64, void* X, cudaStream_t st);

// flag[0] |= 1 when some idx[i] is outside [0, ny).
cudaError_t launch_check_idx(const int64_t* idx, int64_t count, int64_t ny, int* flag,
                             cudaStream_t st);

// out[i] = i, i < n.
cudaError_t launch_iota(int64_t* out, int64_t n, cudaStream_t st);

// Split an F32/F64/U8 matrix into BF16 planes hi = bf16(y), lo = bf16(y - hi)
// (round to nearest even; rows padded with zeros to split_ld(d)), hi plane
// first, lo plane n * split_ld(d) elements later; nrm = FP32 sum of
// hi^2 + 2 hi lo (the products a split tensor-core dot product forms).
cudaError_t launch_quant_bf16(const void* Y, int dt, int64_t n, int d, void* Yq, double* nrm,
                              cudaStream_t st);
// The same for `rows` rows that are rows row0.. of planes of nplane rows each
// (hi plane at Yq, lo plane nplane * split_ld(d) elements later; norms at nrm[row0..]).
cudaError_t launch_quant_bf16_rows(const void* Y, int dt, int64_t rows, int d, void* Yq, int64_t row0,
                                   int64_t nplane, double* nrm, cudaStream_t st);

// Tensor-core Gower projection for BF16 split data (tcgen05 + TMA): X (m x r,
// float) = A^2 W + b with A^2 from the split planes of Y (m rows) and of the l
// landmarks (norms nrm_l zero-padded to gower_tc_lpad(l)), W as the image
// launch_w_image writes.  The lo plane of Y starts ylo_rows * split_ld(d)
// elements after Ysplit (ylo_rows = m for planes of exactly these rows).
// Requires gower_tc_supported(d, r).  *err receives MDS_ERR_TIMEOUT if a
// bounded wait gives up.
bool gower_tc_supported(int d, int r);
cudaError_t launch_gower_tc(const void* Ysplit, int64_t m, int64_t ylo_rows, int d, const double* nrm_y,
                            const void* Lsplit, const float* nrm_l, int l, const void* Wimg,
                            const double* bias, int r, float* X, int* err, cudaStream_t st);
// Padded width (4, 8, 12 or 16) of W rows for the byte-row kernel.
int gower_tc_rp(int r);
// Landmarks rounded up to whole 128-landmark chunks.
int gower_tc_lpad(int l);
// W (l x r, float, r <= 16) -> the BF16 hi/lo W^T image k_gower_tc's projection
// MMA reads (gower_tc_w_bytes(l) bytes, zero past l and r).
size_t gower_tc_w_bytes(int l);
cudaError_t launch_w_image(const float* W, int l, int r, void* img, cudaStream_t st);
// Landmark rows of split planes into split planes, norms as float.
cudaError_t launch_gather_split(const void* Ysplit, int64_t ny, int d, const int64_t* idx, int l,
                                void* Lsplit, const double* nrm, float* nrm_l, cudaStream_t st);

// X[idx[i]] = X1[i] (landmark rows of interpolation MDS).
cudaError_t launch_scatter_rows(const void* X1, const int64_t* idx, int l, int r, int64_t nx,
                                int out_f64, void* X, cudaStream_t st);
// The same restricted to rows row0 .. row0 + rows - 1, X holding those rows only.
cudaError_t launch_scatter_rows_range(const void* X1, const int64_t* idx, int l, int r, int64_t row0,
                                      int64_t rows, int out_f64, void* X, cudaStream_t st);

// Divide-and-conquer: Procrustes of every part against part 0, then the
// aligned scatter and the averaged eigenvalues.
cudaError_t launch_dc_procrustes(const ProbDesc* desc, int p, const double* varena,
                                 const double* lam, int r, int c, double* Tt, cudaStream_t st);
cudaError_t launch_dc_align(const ProbDesc* desc, int p, int max_n, const double* varena,
                            const double* lam, const double* Tt, int r, const int64_t* anchors,
                            const int64_t* own, int out_f64, void* X, cudaStream_t st);
cudaError_t launch_dc_lambda_bar(const ProbDesc* desc, int p, const double* lam, int r,
                                 double* var, cudaStream_t st);

// Classical MDS output X = V Lambda^{1/2} in row order of problem 0.
cudaError_t launch_classical_out(const double* V, const double* lam, int n, int r, int out_f64,
                                 void* X, double* lam_out, cudaStream_t st);

// Tensor-core Gower projection for byte-valued rows of any width
// (k_gower_tck.cu).  kTckBf16: exact BF16 operands; kTckFp8: exact E4M3
// nibble planes.  Operands come from launch_encode_u8 (rows) and
// launch_encode_landmarks_u8 (landmarks, norms padded to tck_lpad(l)); W is
// padded by launch_pad_w_rows to tck_lpad(l) x gower_tc_rp(r).
constexpr int kTckBf16 = 0;
constexpr int kTckFp8 = 1;
int tck_lpad(int l);
size_t tck_operand_bytes(int mode, int64_t rows, int d);
size_t tck_landmark_bytes(int mode, int l, int d);
bool gower_tck_supported(int d, int r);
cudaError_t launch_encode_u8(int mode, const uint8_t* Y, int64_t n, int d, void* out, float* nrm, cudaStream_t st);
cudaError_t launch_encode_landmarks_u8(int mode, const uint8_t* Y, int64_t ny, int d, const int64_t* idx, int l,
                                       void* B, float* nrm_l, cudaStream_t st);
cudaError_t launch_pad_w_rows(const float* W, int l, int r, float* Wp, cudaStream_t st);
cudaError_t launch_gower_tck(int mode, const void* A, int64_t m, int d, const float* nrm_y, const void* B, int l,
                             const float* nrm_l, const float* Wp, const double* bias, int r, float* X, int* err,
                             cudaStream_t st);

// Divide-and-conquer part Gram of byte rows on the tensor cores
// (k_gower_tck.cu): members of part j encoded at operand rows moff[j] ..
// (moff ascending, multiples of 4, slots = total rows incl. padding); units
// are (part, row0, col0, moff) work items of 128 rows x 256 columns.
size_t gram_operand_bytes(int mode, int64_t member_slots, int d);
cudaError_t launch_encode_parts_u8(int mode, const uint8_t* Y, int d, const int64_t* anchors, const int64_t* own,
                                   const ProbDesc* desc, const int* moff, int p, int64_t slots, void* ops,
                                   float* nrm, cudaStream_t st);
cudaError_t launch_gram_tck(int mode, const void* ops, int64_t slots, int d, const float* nrm, const int4* units,
                            int nunits, const ProbDesc* desc, double* qarena, double* rparena, int* err,
                            cudaStream_t st);

// MaxMin landmark choice (k_maxmin.cu): running minima (n FP64), the newest
// landmark row, per-CTA best pairs (maxmin_grid() entries each) and the
// arrival counter of the last-CTA reduction.  idx_out receives the l picks.
constexpr int kMaxminD = 12288;      // widest rows (the landmark row is staged in shared memory as FP64 and as T)
constexpr int kMaxminGridCap = 4096; // most CTAs of a round (partials sized for this many)
struct MaxminWs {
    double* mind;
    int* nrm8;          // byte rows: exact squared norms (n)
    int64_t* cur;
    double* part_v;
    int64_t* part_i;
    unsigned* counter;
    int* err;           // status word of the tiled rounds' bounded waits
};
int maxmin_grid();
cudaError_t launch_maxmin(const void* Y, int dt, int64_t n, int d, int l, int64_t first, MaxminWs ws,
                          int64_t* idx_out, cudaStream_t st);

// Procrustes of point-set pairs given as matrices (k_align.cu): task k aligns
// B_k onto A_k (c x r each, A then B at AB + k * 2 c r) into Tt + dst[k] * (r r + r).
cudaError_t launch_procrustes_sets(const double* AB, int tasks, int c, int r, const int* dst, double* Tt,
                                   cudaStream_t st);

// Fast MDS (k_fast.cu).  A Procrustes task maps a subset (a child) onto its
// parent's alignment configuration: rows row0 .. row0 + s - 1 of problem
// align_prob against rows 0 .. s - 1 of problem leaf_prob (the leftmost leaf
// below the child) carried through the maps of chain[chain_off ..
// chain_off + chain_len).
struct FastTask {
    int align_prob, row0, leaf_prob, chain_off, chain_len;
};
cudaError_t launch_fast_gather(const int64_t* perm, const longlong2* copies, int ncopies, int s, int64_t* own_all,
                               cudaStream_t st);
cudaError_t launch_fast_prep(const ProbDesc* desc, const double* varena, const double* lam, int r, int s,
                             const FastTask* tasks, int ntasks, const int* chain, const double* maps, double* AB,
                             cudaStream_t st);
// Leaves are problems 0 .. nleaves - 1; leaf_chain[k] = (offset, length) of
// the nodes from leaf k up to, not including, the root.
cudaError_t launch_fast_finish(const ProbDesc* desc, int nleaves, int max_leaf, const double* varena,
                               const double* lam, const int2* leaf_chain, const int* chain, const double* maps, int r,
                               double* lmaps, const int64_t* own, int out_f64, void* X, cudaStream_t st);

// Failure injection (api.cu): the team grid-barrier wait limit for the next
// eigen-solver launches (0 = default), and device allocations of model, plan
// and server creation that are made to fail (dev_malloc consumes the count).
unsigned long long wait_limit_ns();
cudaError_t dev_malloc(void** p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) { return dev_malloc(reinterpret_cast<void**>(p), bytes); }

// Host side (api.cu): queue an embedding against a model without waiting.
int embed_enqueue(mds_model m, const void* Ynew, int dt, int64_t rows, char* ws, cudaStream_t st, void* X,
                  int** kerr_out);

}  // namespace gbmds
