/*
 * gbmds.h -- C ABI of libgbmds.so: interpolation MDS and divide-and-conquer MDS
 * on one NVIDIA GB300 (sm_103a).
 *
 * Method: Delicado & Pachon-Garcia, "Multidimensional scaling for big data"
 * (arXiv 2007.11919).  Classical MDS (Section 2), interpolation MDS with
 * Gower's formula (Section 3.1, Eq. (2)) and divide-and-conquer MDS with
 * orthogonal Procrustes alignment (Section 3.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Data Y is row-major n x d (rows are individuals), element type given by
 *    an mds_dtype.  Distances are squared Euclidean distances between rows.
 *  - Unless stated otherwise every array argument is a DEVICE pointer owned by
 *    the caller; the library never frees it and writes only the outputs.
 *  - Configurations X are row-major n x r: double when opts->prec is
 *    MDS_PREC_F64, float otherwise.  Eigenvalue / variance outputs are double.
 *  - Scratch memory: the caller passes opts->workspace (device memory of at
 *    least the matching *_workspace_size() bytes, 256-byte aligned).  The
 *    library allocates device memory only inside mds_model handles.
 *  - Work is queued on opts->stream.  Each call synchronises that stream
 *    before it returns, to read the device status words (eigen-solver
 *    convergence, rank); outputs are complete when it returns MDS_OK.
 *  - Errors never abort the process.  On any status other than MDS_OK the
 *    outputs are unspecified.
 *  - Randomness of the method (the random landmark subset of Section 3.1, the
 *    random connecting points and parts of Section 3.2) is drawn by the
 *    caller; index arrays are inputs.
 *  - Eigenvector sign: each eigenvector is flipped so that its entry of
 *    largest magnitude is positive (lowest row index wins a tie).
 *  - r <= 32.  Eigenproblems (landmark sets, parts, classical MDS) have at
 *    most 16384 points.
 */
#ifndef GBMDS_H
#define GBMDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MDS_OK = 0,
    MDS_ERR_ARG = 1,          /* invalid argument (null pointer, size, index) */
    MDS_ERR_NOMEM = 2,        /* device allocation inside a model handle failed */
    MDS_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    MDS_ERR_RANK = 4,         /* fewer than r eigenvalues > rank_tol * lambda_1 */
    MDS_ERR_NOCONV = 5,       /* eigen-solver hit max_steps before tolerance */
    MDS_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    MDS_ERR_UNSUPPORTED = 7,  /* precision / dtype combination not built */
    MDS_ERR_WORKSPACE = 8,    /* opts->workspace missing, misaligned or too small */
    MDS_ERR_IO = 9            /* model file could not be read or written */
} mds_status;

typedef enum { MDS_IN_F64 = 0, MDS_IN_F32 = 1, MDS_IN_U8 = 2 } mds_dtype;

/* Arithmetic of the distance contractions.  For every precision the
 * centering means, the Procrustes SVDs and the scalars of the eigen-solver
 * (Lanczos coefficients, Ritz values, convergence tests) are FP64, and the
 * landmark eigenproblem of interpolation MDS (Section 3.1, one l x l problem)
 * is solved entirely in FP64 (Q, Lanczos vectors and products), from FP32
 * distances of the unrounded rows unless the precision is MDS_PREC_F64.
 * Eigenproblems of the other calls (classical MDS, the parts of
 * divide-and-conquer MDS) follow the precision: FP64 for MDS_PREC_F64;
 * otherwise Q is double-centred in FP64 from the FP32 (or tensor-core)
 * distances and stored in FP32, the Lanczos basis is FP32, and the
 * products and working vectors run in double-FP32 (about 48 significand
 * bits) with FP64 scalars. */
typedef enum {
    MDS_PREC_F64 = 0,   /* FP64 throughout */
    MDS_PREC_F32 = 1,   /* FP32 distances (CUDA cores) */
    MDS_PREC_BF16 = 2,  /* BF16 tensor-core distances, FP32 accumulate */
    MDS_PREC_FP8 = 3    /* E4M3 tensor-core distances (uint8 data), FP32 accumulate */
} mds_precision;

typedef struct {
    int32_t prec;            /* mds_precision */
    int32_t max_steps;       /* Lanczos step cap per eigenproblem; 0 = 256 */
    double eig_tol;          /* stop when every wanted Ritz residual
                                <= eig_tol * lambda_1; 0 = 1e-10 for
                                MDS_PREC_F64 / F32, 1e-8 for BF16 / FP8 */
    double rank_tol;         /* MDS_ERR_RANK unless lambda_r > rank_tol * lambda_1;
                                0 = 1e-12 */
    void* stream;            /* cudaStream_t; NULL = the legacy default stream */
    void* workspace;         /* device scratch (see *_workspace_size) */
    size_t workspace_bytes;
    int32_t cluster;         /* CTAs per eigenproblem (1..16); 0 = automatic */
    int32_t flags;           /* 0 or MDS_FLAG_FULL_MATVEC */
} mds_opts;

/* Flag of mds_opts.flags.  MDS_FLAG_FULL_MATVEC: the eigen-solver streams
 * every row of Q whole.  Without it, an FP32 Q solved by one cluster of 3 or
 * more CTAs is read in symmetric ranges: each off-diagonal block once, used
 * for both triangles (Q = -1/2 P Delta P is symmetric, Section 2).  The two
 * forms differ only in rounding. */
#define MDS_FLAG_FULL_MATVEC 1

/* Opaque device-resident landmark configuration of interpolation MDS: the l
 * landmark rows, their classical-MDS eigenpairs and the Gower projection
 * operator derived from them (Section 3.1). */
typedef struct mds_model_s* mds_model;

/* Human-readable name of a status code (static string, never NULL). */
const char* mds_status_str(int status);

/* Library ABI version (currently 1). */
int mds_version(void);

/* ------------------------------------------------------------------ */
/* Classical MDS of n points (Section 2, steps 1-4).
 *   Delta = squared distances between the rows of Y (n x d, dtype dt),
 *   Q = -1/2 P Delta P, top-r eigenpairs (lambda_i, v_i) of Q,
 *   X = V_r Lambda_r^{1/2}  (n x r), lambda (r, descending).
 * Fails with MDS_ERR_RANK if lambda_r <= rank_tol * lambda_1. */
size_t mds_classical_workspace_size(int64_t n, int d, int r, int prec);
int mds_classical(const void* Y, int dt, int64_t n, int d, int r, const mds_opts* opts,
                  void* X, double* lambda);

/* Classical MDS of a given n x n squared-distance matrix D2 (row-major,
 * double, symmetric, zero diagonal; need not be Euclidean) (Section 2). */
size_t mds_classical_dist_workspace_size(int64_t n, int r);
int mds_classical_dist(const double* D2, int64_t n, int r, const mds_opts* opts,
                       double* X, double* lambda);

/* ------------------------------------------------------------------ */
/* Interpolation MDS (Section 3.1).
 *   landmark_idx (device, l distinct int64 rows of Y) is the first subset;
 *   classical MDS of the landmarks gives X_1 = V Lambda^{1/2};
 *   every other row i is placed by Gower's formula, Eq. (2):
 *     Xdot_i = 1/(2l) (q_1 - a2_i)^T X_1 S_1^{-1},  S_1 = Lambda / l,
 *   a2_i = squared distances from row i to the landmarks, q_1 = diag(Q_1).
 *   Landmark rows receive X_1.  X is n x r in the original row order;
 *   var (r) = lambda / l, the column-variance estimates.
 *   If out_model is not NULL a device-resident model (mds_model) is created
 *   for mds_embed_new; release it with mds_model_free. */
size_t mds_interpolate_workspace_size(int64_t n, int d, int l, int r, int prec);
int mds_interpolate(const void* Y, int dt, int64_t n, int d, const int64_t* landmark_idx, int l,
                    int r, const mds_opts* opts, void* X, double* var, mds_model* out_model);

/* Interpolation MDS (Section 3.1) of rows that live in host memory: the same
 * result as mds_interpolate on a device copy of Y (bitwise), computed while Y
 * crosses the link.  Y (n x d, dtype dt), landmark_idx (l int64), X (n x r:
 * float, or double for MDS_PREC_F64) and var (r) are HOST pointers; the
 * caller keeps them alive until the call returns.  The landmark rows are
 * gathered on the host and their eigenproblem starts at once; meanwhile the
 * rows are copied in chunks of chunk_rows (0 = about 96 MiB of rows) on a second stream,
 * each chunk is turned into the projection operands as it lands, projected
 * once the model is ready, and its rows of X are copied back on a third
 * stream.  Y and X should be page-locked (pinned) for the copies to overlap
 * the computation; pageable memory works but serialises them.  The
 * workspace (opts->workspace, mds_interpolate_host_workspace_size bytes)
 * holds a device copy of Y and X besides mds_interpolate's workspace.
 * Errors: MDS_ERR_ARG also for a landmark index outside [0, n) (checked on
 * the host before any work); statuses as mds_interpolate. */
size_t mds_interpolate_host_workspace_size(int64_t n, int d, int l, int r, int prec, int dt);
int mds_interpolate_host(const void* Y, int dt, int64_t n, int d, const int64_t* landmark_idx, int l,
                         int r, int64_t chunk_rows, const mds_opts* opts, void* X, double* var,
                         mds_model* out_model);

/* Interpolation MDS (Section 3.1) in its affine form, for rows given by
 * Euclidean coordinates: with squared Euclidean distances Q_1 = L_c L_c^T
 * (Section 2, L_c the landmark rows minus their mean y_L), so Eq. (2) is
 *   Xdot = (Y - 1 y_L^T) U_r,  U_r = L_c^T V_r Lambda_r^{-1/2}  (d x r),
 * one pass over Y instead of n x l distances.  The landmark eigenproblem is
 * that of mds_interpolate; every row, landmarks included, gets (y - y_L) U_r
 * (for the landmarks this is X_1 up to rounding).  Arguments as for
 * mds_interpolate (device pointers; X float, or double for MDS_PREC_F64);
 * opts->prec must be MDS_PREC_F64 or MDS_PREC_F32 (else
 * MDS_ERR_UNSUPPORTED); no model is made.  The result equals
 * mds_interpolate's for Euclidean input, up to rounding. */
size_t mds_interpolate_affine_workspace_size(int64_t n, int d, int l, int r, int prec);
int mds_interpolate_affine(const void* Y, int dt, int64_t n, int d, const int64_t* landmark_idx, int l,
                           int r, const mds_opts* opts, void* X, double* var);

/* MaxMin choice of l landmarks (Section 3.1, the LMDS variant of the first
 * subset): starting from row `first`, each next landmark is the row of Y
 * whose smallest squared Euclidean distance to the landmarks already chosen
 * is largest; ties go to the lowest row index; a chosen row is never chosen
 * again (a duplicate of a chosen row can be).  idx_out (device, l int64)
 * receives the rows in the order chosen; pass them to mds_interpolate as
 * landmark_idx.  The argmax is taken on FP64 distances: exact integer sums
 * for MDS_IN_U8 rows, the FP64 difference form sum_k (y_k - l_k)^2 for FP64
 * rows, and for FP32 rows an FP32 difference form whose rounding bound
 * proves the running minimum unchanged, else the FP64 difference form.
 * opts->prec is ignored; opts->workspace holds
 * mds_landmarks_maxmin_workspace_size(n, d) bytes (n FP64 running minima).
 * Errors: MDS_ERR_ARG for l outside [1, n] or first outside [0, n);
 * MDS_ERR_UNSUPPORTED for d > 12288. */
size_t mds_landmarks_maxmin_workspace_size(int64_t n, int d);
int mds_landmarks_maxmin(const void* Y, int dt, int64_t n, int d, int l, int64_t first, const mds_opts* opts,
                         int64_t* idx_out);

/* Pivot MDS (Section 3.1): with C the n x l block of Q = -1/2 P Delta P
 * (all n points) between every point and the l pivots pivot_idx (device, l
 * int64 rows), the SVD C = U Sigma W^T approximates the eigendecomposition of
 * Q: X = U_r diag(lambda_r)^{1/2} (n x r: double for MDS_PREC_F64, else
 * float), lambda_i = sigma_i sqrt(n / l) (random pivots give
 * V_P^T V_P ~ (l/n) I, so C C^T ~ (l/n) Q^2), var (r) = lambda / n.  Rows
 * are Euclidean coordinates, so C = Y_c P_c^T (Y_c the rows centred at their
 * mean, P_c the centred pivot rows) and C^T C = P_c S P_c^T with
 * S = Y_c^T Y_c: the call computes the column means and S of Y, the l x l
 * matrix C^T C and its top-r eigenpairs in FP64, and one pass
 * X = Y_c M, M = P_c^T W_r Sigma_r^{-1} Lambda_r^{1/2} (d x r).  Each column
 * of X has its entry of largest magnitude positive (lowest row on a tie).
 * opts->prec: MDS_PREC_F64 (FP64 throughout) or MDS_PREC_F32 (the scatter
 * matrix from FP32 products summed in double-FP32, the projection in FP32;
 * the means, C^T C and the eigen-solve in FP64); else MDS_ERR_UNSUPPORTED,
 * which d > 4096 also returns (the workspace size is then 0).
 * Requires 1 <= r <= min(l, d, 32); MDS_ERR_RANK if sigma_r^2 <=
 * rank_tol * sigma_1^2. */
size_t mds_pivot_workspace_size(int64_t n, int d, int l, int r, int prec);
int mds_pivot(const void* Y, int dt, int64_t n, int d, const int64_t* pivot_idx, int l, int r, const mds_opts* opts,
              void* X, double* var);

/* Gower's formula, Eq. (2), for m new rows Ynew (m x d, dtype dt) against a
 * stored model; X is m x r.  opts->prec must equal the model's precision.
 * Equal inputs give bitwise-equal outputs regardless of what else is batched
 * with them: rows are computed independently. */
size_t mds_embed_new_workspace_size(mds_model model, int64_t m);
int mds_embed_new(mds_model model, const void* Ynew, int dt, int64_t m, const mds_opts* opts,
                  void* X);

/* Allocation-free variant of mds_embed_new.  The paper has no counterpart:
 * this exists for callers that must not allocate device memory when they
 * embed points -- for example a serving process whose device memory is all
 * reserved up front by another allocator (a new cudaMalloc would fail), or a
 * plugin / real-time loop that forbids allocation after start-up (an
 * allocation can stall on device-wide synchronisation).
 *   - Scratch is a 16 MiB array inside the library (mds_embed_new_static_capacity()
 *     bytes), present on every GPU that loads libgbmds.so until the process
 *     exits.  opts->workspace must be NULL and opts->workspace_bytes 0.
 *   - Sizes: a call fits when mds_embed_new_workspace_size(model, m) is at most
 *     the capacity (about 2 million rows for FP32/FP64 models; fewer for BF16
 *     models, which also stage a rounded copy of the rows); larger m returns
 *     MDS_ERR_WORKSPACE without doing any work.  Split large batches.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make that
 *     first call before any stream capture on that device.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind.  Nothing in it needs to start at zero (each call writes every
 *     scratch byte it reads).  Calls whose work overlaps on the GPU (other
 *     streams, other host threads) race on the array: serialise them.
 *   - Calls no cudaMalloc/cudaFree and no allocating library routine.
 *   Results are the same as mds_embed_new's. */
size_t mds_embed_new_static_capacity(void);
int mds_embed_new_static(mds_model model, const void* Ynew, int dt, int64_t m,
                         const mds_opts* opts, void* X);

/* Model inspection / persistence.  lambda may be NULL. */
int mds_model_info(mds_model model, int* l, int* d, int* r, int* prec, double* lambda);
int mds_model_save(mds_model model, const char* path);
int mds_model_load(const char* path, mds_model* out_model);
void mds_model_free(mds_model model);

/* ------------------------------------------------------------------ */
/* Divide-and-conquer MDS (Section 3.2).
 *   anchors   device, c int64 rows: the connecting points shared by all parts.
 *   part_ptr  HOST, p+1 int64 offsets into part_own (part_ptr[0] = 0).
 *   part_own  device, part_ptr[p] int64 rows: part j owns
 *             part_own[part_ptr[j] .. part_ptr[j+1]).
 *   Part j's points are the c anchors followed by its own rows, n_j = c + own_j.
 *   Classical MDS of every part gives X_j, lambda^j (all parts in one batched
 *   launch); each X_j, j >= 1, is aligned to part 0 by orthogonal Procrustes
 *   on the connecting points, X_0^c ~ X_j^c T_j + 1 t_j^T (T_j orthogonal,
 *   reflections allowed, no scaling); rows of part j other than the anchors
 *   receive X_j^a T_j + 1 t_j^T; part 0's rows (anchors included) receive X_0.
 *   X (n x r) is written only at rows that appear in the parts, in original
 *   row order.  var (r) = (1/p) sum_j lambda^j / n_j.
 *   Requires c >= r + 1 and r < n_j for every part. */
size_t mds_divide_conquer_workspace_size(int64_t n, int d, int p, const int64_t* part_ptr, int c,
                                         int r, int prec);
int mds_divide_conquer(const void* Y, int dt, int64_t n, int d, int p, const int64_t* part_ptr,
                       const int64_t* part_own, const int64_t* anchors, int c, int r,
                       const mds_opts* opts, void* X, double* var);

/* ------------------------------------------------------------------ */
/* Fast MDS (Section 3.3).  The random recursive division is an input:
 *   perm         device, n int64: the rows in the order of the division
 *                (every node's points are a contiguous range of perm);
 *   node_range   HOST, 2 * nnodes int64: [begin, end) of node k in perm;
 *   node_parent  HOST, nnodes int32: the parent of node k (-1 for node 0, the
 *                root, whose range is [0, n)).
 * The children of a node are the nodes whose parent it is, ordered by begin;
 * they must tile the parent's range (at least two of them), each holding at
 * least s points.  A node without children is a leaf: classical MDS
 * (Section 2) gives its configuration.  At an inner node the first s points
 * of each child (its sampling points) form the alignment set; its
 * classical MDS is the alignment configuration X_align, and child j's
 * configuration X_j is mapped onto rows j s .. j s + s - 1 of it by
 * Procrustes on its first s rows, X_align,j^s ~ X_j^s T_j + 1 t_j^T (T_j
 * orthogonal, reflections allowed); the node's configuration is the
 * children's mapped configurations in order.  X (n x r, double for
 * MDS_PREC_F64, else float) is the root's configuration in original row
 * order; var (r) = mean over the leaves of lambda^j / n_j.
 * All classical problems (leaves and alignment sets, each at most 16384 and
 * more than r points) run in one batched eigen-solver launch; the maps are
 * found one tree level at a time.  opts->prec: MDS_PREC_F64 or MDS_PREC_F32
 * (distances and eigen-solve as for mds_divide_conquer); s >= r + 1.
 * Errors: MDS_ERR_ARG for a malformed tree or sizes, or a perm entry
 * outside [0, n). */
size_t mds_fast_workspace_size(int64_t n, int d, int nnodes, const int64_t* node_range, const int32_t* node_parent,
                               int s, int r, int prec);
int mds_fast(const void* Y, int dt, int64_t n, int d, const int64_t* perm, int nnodes, const int64_t* node_range,
             const int32_t* node_parent, int s, int r, const mds_opts* opts, void* X, double* var);

/* ------------------------------------------------------------------ */
/* Divide-and-conquer plans (Section 3.2 repeated on new data of fixed shape).
 * A plan fixes n, d, dtype, the part layout (part_ptr, c), r and the
 * precision; it allocates its own workspace once (opts->workspace must be
 * NULL), keeps the part descriptors on the device, and on execute runs the
 * whole launch sequence of mds_divide_conquer -- every part in one persistent
 * eigen-solver launch -- as one CUDA graph, captured at the first execute and
 * again whenever a buffer pointer or the stream changes.
 *   tune  nonzero (and opts->cluster 0): the first execute is an autotuner:
 *         it runs the complete computation once per eligible cluster size
 *         (CTAs per eigenproblem, 1..16, shared memory permitting), times each
 *         with CUDA events on these buffers, and keeps the fastest; those
 *         runs write valid outputs.  Otherwise the cluster size is
 *         opts->cluster or the library's heuristic.
 *   execute: buffers as for mds_divide_conquer (Y, part_own, anchors, X, var
 *         device pointers).  The graph runs on a stream the plan owns (stream
 *         capture needs one), ordered after the work already queued on
 *         `stream` (NULL = opts->stream); execute waits for it and returns
 *         the status of the run.
 *   info: cluster size in use, nodes of the captured graph, and per cluster
 *         size 0..16 the autotuner's time in ms (0 = not tried).
 * With a tuning cache (mds_set_tune_cache) the autotuner first looks its
 * batch shape up there and, on a hit, takes the stored cluster size and
 * trial times without timing anything; after timing it stores its choice. */
typedef struct mds_dc_plan_s* mds_dc_plan;
int mds_dc_plan_create(int64_t n, int d, int dt, int p, const int64_t* part_ptr, int c, int r,
                       const mds_opts* opts, int tune, mds_dc_plan* out);
int mds_dc_plan_execute(mds_dc_plan plan, const void* Y, const int64_t* part_own, const int64_t* anchors,
                        void* X, double* var, void* stream);
/* Execute on data in HOST memory (Section 3.2, the same computation as
 * mds_dc_plan_execute, bitwise the same result): Y (n x d), part_own,
 * anchors, X (n x r: double for MDS_PREC_F64, else float) and var (r) are
 * host pointers.  The plan copies the inputs into device buffers it owns
 * (allocated at the first call: n x d input elements, the indices, n x r
 * outputs; MDS_ERR_NOMEM if that fails), replays its graph on them, copies
 * X and var back, and returns when they are in host memory.  Rows of X
 * outside every part are zero.  Page-locked host buffers make the copies
 * asynchronous DMA; pageable ones work too. */
int mds_dc_plan_execute_host(mds_dc_plan plan, const void* Y, const int64_t* part_own, const int64_t* anchors,
                             void* X, double* var, void* stream);
int mds_dc_plan_info(mds_dc_plan plan, int* cluster, int64_t* graph_nodes, double* trial_ms);
void mds_dc_plan_destroy(mds_dc_plan plan);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of embed requests (Section 3.1, Eq. (2),
 * applied to points that arrive after the landmark configurations were built;
 * the paper embeds its new points in fixed blocks and has no request loop).
 *
 * A server owns `slots` CUDA streams, each with its own device arena of
 * slot_bytes bytes, and one host scheduler thread.  Requests name one of the
 * server's resident models.  Whenever a slot is free the scheduler fills it
 * with a batch: rows of waiting requests for the model of the oldest waiting
 * request, in arrival order, as many as the slot's arena holds (staged input
 * rows, scratch and results); a request too large for one slot is split
 * across batches.  The batch is copied in, embedded by one launch of the
 * model's projection kernel and copied out on the slot's stream, so batches
 * on different slots (copies and kernels) overlap on the device, and requests
 * that arrive while others are on the GPU join the next free slot.  Every row
 * is computed from its own input and the model only: a result is bitwise the
 * same whether its request ran alone or in a mix.
 *
 *   models     the resident configurations (mds_interpolate / mds_model_load),
 *              all on the calling thread's current device; the server keeps
 *              the handles (the caller frees them after mds_server_destroy).
 *   slots      concurrent batches, 1..16 (0: 4).
 *   slot_bytes device bytes per slot (0: 64 MiB); allocated at creation.
 *   max_batch_rows  cap on rows per batch (0: whatever fits).
 *   flags      must be 0.
 * Submit: Y is a HOST pointer to m x d rows of the model's d (dtype dt); X a
 * HOST pointer to m x r outputs (double for MDS_PREC_F64 models, float
 * otherwise).  Both must stay valid until mds_server_wait returns for the
 * ticket; page-locked (cudaHostAlloc / pinned) buffers let copies overlap,
 * pageable ones serialise the scheduler on each copy.  Submit only queues the
 * request and returns at once.
 * Wait: blocks until the request is complete or timeout_s passes (returns
 * MDS_ERR_TIMEOUT, request still pending; wait again).  On completion *status
 * is the request's status and *latency_ms the time from submit to the end of
 * its last batch on the device; the ticket is then released.
 * Destroy: drains all queued work, then frees the slots. */
typedef struct mds_server_s* mds_server;

typedef struct {
    int32_t slots;
    int32_t flags;
    size_t slot_bytes;
    int64_t max_batch_rows;
} mds_server_opts;

typedef struct {
    int64_t requests;       /* completed */
    int64_t rows;           /* rows embedded */
    int64_t batches;        /* batches launched */
    int32_t max_in_flight;  /* most slots busy at once */
    int32_t slots;
} mds_server_stats;

int mds_server_create(const mds_model* models, int nmodels, const mds_server_opts* opts, mds_server* out);
int mds_server_submit(mds_server srv, int model, const void* Y, int dt, int64_t m, void* X,
                      uint64_t* ticket);
int mds_server_wait(mds_server srv, uint64_t ticket, double timeout_s, int* status, double* latency_ms);
int mds_server_get_stats(mds_server srv, mds_server_stats* out);
int mds_server_destroy(mds_server srv);

/* ------------------------------------------------------------------ */
/* Instrumentation (the paper has no counterpart; used by the benchmark).
 * mds_set_timing(1) makes subsequent calls on the calling host thread record
 * CUDA events on opts->stream between pipeline stages; mds_last_stats then
 * returns the stage durations of the last completed call on that thread:
 *   stage_ms[0] data preparation (norms, BF16 rounding)
 *   stage_ms[1] squared-distance tiles (Delta_j, Section 2)
 *   stage_ms[2] double centering (Q_j = -1/2 P Delta_j P)
 *   stage_ms[3] batched Lanczos eigen-solve (top-r eigenpairs)
 *   stage_ms[4] Gower projection / Procrustes alignment and output
 * eig_flops / eig_qbytes: algorithmic FP64 flops of the eigen-solve
 * (2 n^2 per matrix-vector product, 8 n for the local Gram-Schmidt pass and
 * 4 n (j+1) for the full one at step j, 2 n k r for the Ritz vectors) and bytes of Q read per step (8 n^2
 * for FP64 problems, 4 n^2 otherwise, where Q is stored in FP32),
 * summed over the problems of the call with their actual step counts. */
typedef struct {
    double stage_ms[5];
    int64_t launches;      /* kernels launched by the call */
    int64_t eig_steps;     /* Lanczos steps summed over problems */
    double eig_flops;
    double eig_qbytes;
    int32_t problems;      /* eigenproblems in the call */
    int32_t cluster;       /* CTAs per eigenproblem used */
    double eig_qread;      /* bytes of Q the eigen-solver streamed: eig_qbytes, or
                              less where it read symmetric ranges (each
                              off-diagonal block of Q once) */
} mds_stats;

void mds_set_timing(int on);
int mds_last_stats(mds_stats* out);

/* Eigen-solver phase timers, compiled in only when the library is built with
 * GBMDS_PHASE_TIMERS=1 (otherwise MDS_ERR_UNSUPPORTED).  out[0..6]: clock
 * cycles summed over all CTAs of every launch since the last reset, spent in
 * [0] the exchange and completion of the second Gram-Schmidt pass, [1] the
 * convergence checks, [2] the matrix-vector product, [3] the pass against the
 * two newest vectors, [4] publishing the new vector, [5] the finish (Ritz
 * vectors, signs); out[6] the CTA-steps.  reset = 1 zeroes the counters
 * (out may then be NULL).  Process-wide; the cycles are SM clocks. */
int mds_lanczos_phase_cycles(double* out, int reset);

/* ------------------------------------------------------------------ */
/* Failure injection (testing the error paths; the paper has no
 * counterpart).  Neither faults the GPU: each makes an ordinary, bounded
 * error path run.
 * mds_set_wait_limit_ns(ns): from the next call on, a grid-barrier wait of
 *   the eigen-solver that solves one problem with a team of clusters (the
 *   landmark problem of interpolation MDS, classical MDS) gives up after ns
 *   nanoseconds instead of 2 s; the team then leaves the solve together,
 *   waits for its copies in flight, and the call returns MDS_ERR_TIMEOUT.
 *   0 restores the default.  Process-wide.
 * mds_inject_alloc_failures(count): the next `count` device allocations made
 *   by model, plan or server creation fail as if the device were out of
 *   memory (the calls return MDS_ERR_NOMEM and free what they had).  The
 *   environment variable GBMDS_FAULT=alloc:N sets the same count when the
 *   library loads. */
void mds_set_wait_limit_ns(unsigned long long ns);
void mds_inject_alloc_failures(int count);

/* ------------------------------------------------------------------ */
/* Tuning cache (the autotuner's memory across processes; the paper has no
 * counterpart).  A JSON file, one entry per line:
 *   {"key": "<kernel and the quantities its choice depends on>", "value": V,
 *    "trial_ms": [...]}
 * Today it holds the eigen-solver's cluster size (CTAs per eigenproblem,
 * 1..16) per batch shape: problem count, largest problem, sum of squared
 * sizes, step cap, r, Q precision, symmetric ranges allowed, SM count and
 * compute capability.  D&C plans created with tune store what they measured
 * and reuse a stored value; every call whose opts->cluster is 0 uses a stored
 * value for its batch shape instead of the heuristic.  Updates replace the
 * file through a temporary file and a rename; concurrent writers can lose an
 * update, never corrupt the file.
 * mds_set_tune_cache(path): the cache file (NULL or "" turns the cache off).
 *   Without a call, the environment variable GBMDS_TUNE_CACHE names it at
 *   first use; otherwise the cache is off.  Process-wide.  Returns MDS_OK.
 * mds_tune_cache_lookup(key, &value): value = the stored value, or 0 when the
 *   key is absent or the cache is off; MDS_ERR_ARG for a null or malformed
 *   key (empty, longer than 1,024 bytes, or holding a quote, a backslash or
 *   a line break).
 * mds_tune_cache_store(key, value): adds or replaces an entry; MDS_ERR_ARG
 *   for a malformed key, a cache that is off or a file that cannot be
 *   written. */
int mds_set_tune_cache(const char* path);
int mds_tune_cache_lookup(const char* key, int* value);
int mds_tune_cache_store(const char* key, int value);

#ifdef __cplusplus
}
#endif
#endif /* GBMDS_H */
