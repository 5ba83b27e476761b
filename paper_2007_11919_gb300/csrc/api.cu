// Host side of libgbmds: argument checks, workspace carving and the stream-
// ordered launch sequences behind the C ABI declared in include/gbmds.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

using namespace gbmds;

namespace gbmds {
thread_local int64_t g_launches = 0;
void note_launch(int count) { g_launches += count; }

// Failure injection.  The team grid-barrier wait limit of the next
// eigen-solver launches (0 = the kernel's default), and a count of device
// allocations (model, plan and server creation) that fail on purpose -- set
// by mds_inject_alloc_failures or, at load, by GBMDS_FAULT=alloc:N.
std::atomic<unsigned long long> g_wait_ns{0};
std::atomic<int> g_fail_allocs{0};
static const int g_fault_env = [] {
    const char* e = getenv("GBMDS_FAULT");
    if (e && strncmp(e, "alloc:", 6) == 0) g_fail_allocs.store(atoi(e + 6));
    return 0;
}();

unsigned long long wait_limit_ns() { return g_wait_ns.load(); }

cudaError_t dev_malloc(void** p, size_t bytes) {
    int c = g_fail_allocs.load();
    while (c > 0)
        if (g_fail_allocs.compare_exchange_weak(c, c - 1)) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    return cudaMalloc(p, bytes);
}
}  // namespace gbmds

namespace {

constexpr int kDefaultSteps = 256;

// Model kinds: how the landmark rows are stored and which kernel projects.
constexpr int kKindRows = 0;               // FP64 / FP32 rows (k_gower) or BF16 split planes (k_gower_tc)
constexpr int kKindU8Bf16 = 1 + kTckBf16;  // byte rows as exact BF16 (k_gower_tck)
constexpr int kKindU8Fp8 = 1 + kTckFp8;    // byte rows as exact E4M3 nibble planes (k_gower_tck)

// Kind for a precision and input dtype; -1 when the pair is not built.
int model_kind(int prec, int dt, int d, int r) {
    if (prec == MDS_PREC_FP8) return dt == MDS_IN_U8 && gower_tck_supported(d, r) ? kKindU8Fp8 : -1;
    if (prec == MDS_PREC_BF16) {
        if (dt == MDS_IN_U8) return gower_tck_supported(d, r) ? kKindU8Bf16 : -1;
        return gower_tc_supported(d, r) ? kKindRows : -1;
    }
    return kKindRows;
}

// Tensor-core models keep W in the form their kernel reads: padded to the
// kernel's width and tck_lpad(l) rows for byte-row kinds, the BF16 W^T image
// for BF16 split rows.
size_t model_W_bytes(int kind, int prec, int l, int r) {
    if (kind != kKindRows) return (size_t)tck_lpad(l) * gower_tc_rp(r) * 4;
    if (prec == MDS_PREC_BF16) return gower_tc_w_bytes(l);
    return (size_t)l * r * (prec == MDS_PREC_F64 ? 8 : 4);
}

size_t model_L_bytes(int kind, int prec, int l, int d) {
    if (kind != kKindRows) return tck_landmark_bytes(kind - 1, l, d);
    if (prec == MDS_PREC_BF16) return (size_t)2 * l * split_ld(d) * sizeof(uint16_t);
    return (size_t)l * d * (prec == MDS_PREC_F64 ? 8 : 4);
}

size_t model_nlf_count(int kind, int l) {
    return kind != kKindRows ? (size_t)tck_lpad(l) : (size_t)gower_tc_lpad(l);
}

// ---- per-thread instrumentation (mds_set_timing / mds_last_stats)
bool g_timing = false;
thread_local mds_stats g_last = {};
thread_local cudaEvent_t g_ev[6] = {};
thread_local bool g_ev_made = false;
thread_local int g_cluster = 0;

// While a plan captures its launch sequence, stage marks go to the plan's
// events as event-record nodes of the graph.
thread_local cudaEvent_t* g_capture_ev = nullptr;

// NVTX ranges for profilers (nvtx3, header-only; inert unless a tool is
// attached): one range per call, named for its entry point, and inside it one
// per pipeline stage (the stages of mds_stats), on the host thread that issues
// the call's launches.  A range left open by an early error return is closed
// by the next call on the thread.
thread_local nvtxRangeId_t g_nvtx_call = 0, g_nvtx_stage = 0;
const char* const kStageNames[5] = {"gbmds prep", "gbmds dist", "gbmds center", "gbmds eig", "gbmds post"};

// Closes the open stage range and opens stage `next` (none when next > 4).
void nvtx_stage(int next) {
    if (g_nvtx_stage) nvtxRangeEnd(g_nvtx_stage);
    g_nvtx_stage = 0;
    if (next >= 0 && next <= 4) g_nvtx_stage = nvtxRangeStartA(kStageNames[next]);
}

void nvtx_end_call() {
    nvtx_stage(5);
    if (g_nvtx_call) nvtxRangeEnd(g_nvtx_call);
    g_nvtx_call = 0;
}

void record_mark(int stage, cudaStream_t st) {
    if (g_capture_ev) {
        cudaEventRecordWithFlags(g_capture_ev[stage + 1], st, cudaEventRecordExternal);
        return;
    }
    if (!g_timing) return;
    if (!g_ev_made) {
        for (auto& e : g_ev) cudaEventCreate(&e);
        g_ev_made = true;
    }
    cudaEventRecord(g_ev[stage + 1], st);
}

// Marks the start (stage = -1) or the end of a pipeline stage on the stream.
void tmark(int stage, cudaStream_t st) {
    record_mark(stage, st);
    nvtx_stage(stage + 1);
}

void begin_call(cudaStream_t st, const char* what) {
    nvtx_end_call();
    g_nvtx_call = nvtxRangeStartA(what);
    g_launches = 0;
    g_cluster = 0;
    g_last = mds_stats{};
    if (g_timing || g_capture_ev)
        for (int i = 0; i <= 5; ++i) record_mark(i - 1, st);  // all stages empty by default
    nvtx_stage(0);
}

struct Arena {
    char* base;
    size_t off;
    template <class T>
    T* take(size_t count) {
        off = (size_t)round_up((int64_t)off, 256);
        T* p = reinterpret_cast<T*>(base + off);
        off += count * sizeof(T);
        return p;
    }
};

struct Opts {
    int prec;
    int mmax;
    double tol;
    double rank_tol;
    cudaStream_t st;
    char* ws;
    size_t wsb;
    int cluster;
    int flags;
};

int read_opts(const mds_opts* o, Opts* out) {
    if (!o) return MDS_ERR_ARG;
    if (o->prec < MDS_PREC_F64 || o->prec > MDS_PREC_FP8) return MDS_ERR_ARG;
    if (o->max_steps < 0 || o->eig_tol < 0 || o->rank_tol < 0 || o->cluster < 0 ||
        o->cluster > 16 || (o->flags & ~MDS_FLAG_FULL_MATVEC) != 0)
        return MDS_ERR_ARG;
    out->prec = o->prec;
    out->mmax = o->max_steps ? o->max_steps : kDefaultSteps;
    // BF16 / FP8 distances carry ~2^-16 relative rounding, far above what a
    // 1e-8 residual leaves in the eigenpairs; the FP32 / FP64 paths keep 1e-10
    out->tol = o->eig_tol > 0 ? o->eig_tol
                              : (o->prec == MDS_PREC_BF16 || o->prec == MDS_PREC_FP8 ? 1e-8 : 1e-10);
    out->rank_tol = o->rank_tol > 0 ? o->rank_tol : 1e-12;
    out->st = (cudaStream_t)o->stream;
    out->ws = (char*)o->workspace;
    out->wsb = o->workspace_bytes;
    out->cluster = o->cluster;
    out->flags = o->flags;
    if (out->mmax < 2) return MDS_ERR_ARG;
    return MDS_OK;
}

int check_ws(const Opts& o, size_t need) {
    if (need == 0) return MDS_OK;
    if (!o.ws || ((uintptr_t)o.ws & 255) != 0 || o.wsb < need) return MDS_ERR_WORKSPACE;
    return MDS_OK;
}

// ----------------------------------------------------------- eigen batches

struct Batch {
    std::vector<ProbDesc> desc;
    int p = 0, max_n = 0, max_tiles = 0, mmax = 0, r = 0;
    int q_bytes = 8;                   // bytes per entry of Q as the eigen-solver reads it
    int sym = 1;                       // symmetric ranges allowed (mds_opts flags)
    int team = 0;                      // the eigen-solver ran as a team of clusters
    size_t q_el = 0, rp_el = 0, rm_el = 0, b_el = 0, v_el = 0;
    ProbDesc* d_desc = nullptr;
    double *q = nullptr, *rp = nullptr, *rm = nullptr, *grand = nullptr, *b = nullptr,
           *v = nullptr, *lam = nullptr, *scr = nullptr;
    int *status = nullptr, *steps = nullptr;
    std::vector<int> order;            // problems, largest first (eigen-solver queue order)
    int *d_order = nullptr, *counter = nullptr;
    double* tscr = nullptr;            // single-problem team exchange buffers
    unsigned* tbar = nullptr;          // team barrier words
};

void plan_batch(Batch& B, const std::vector<int>& sizes, const std::vector<int64_t>& own_off,
                int c, int r, int mmax, int64_t ny) {
    B = Batch();
    B.p = (int)sizes.size();
    B.r = r;
    B.mmax = mmax;
    for (int j = 0; j < B.p; ++j) {
        const int n = sizes[j];
        ProbDesc P;
        P.own_off = own_off[j];
        P.n = n;
        P.ldq = (int)round_up(n, 4);
        P.c = c;
        P.tiles = (n + kTile - 1) / kTile;
        P.ny = ny;
        const int kcap = std::min(mmax, n);
        P.q_off = (int64_t)B.q_el;
        P.rp_off = (int64_t)B.rp_el;
        P.rm_off = (int64_t)B.rm_el;
        P.b_off = (int64_t)B.b_el;
        P.v_off = (int64_t)B.v_el;
        B.q_el += (size_t)n * P.ldq;
        B.rp_el += (size_t)round_up((int64_t)P.tiles * n, 4);
        B.rm_el += (size_t)round_up(n, 4);
        B.b_el += (size_t)(kcap + 1) * P.ldq;
        B.v_el += (size_t)round_up((int64_t)n * r, 4);
        B.max_n = std::max(B.max_n, n);
        B.max_tiles = std::max(B.max_tiles, P.tiles);
        B.desc.push_back(P);
    }
    B.order.resize(B.p);
    for (int j = 0; j < B.p; ++j) B.order[j] = j;
    std::stable_sort(B.order.begin(), B.order.end(),
                     [&](int x, int y) { return B.desc[x].n > B.desc[y].n; });
}

void carve_batch(Batch& B, Arena& A) {
    B.d_desc = A.take<ProbDesc>(B.p);
    B.q = A.take<double>(B.q_el);
    B.rp = A.take<double>(B.rp_el);
    B.rm = A.take<double>(B.rm_el);
    B.grand = A.take<double>(B.p);
    B.b = A.take<double>(B.b_el);
    B.v = A.take<double>(B.v_el);
    B.lam = A.take<double>((size_t)B.p * B.r);
    B.scr = A.take<double>((size_t)B.p * lanczos_scratch_per_problem(B.mmax, B.r));
    B.status = A.take<int>(B.p);
    B.steps = A.take<int>(B.p);
    B.d_order = A.take<int>(B.p);
    B.counter = A.take<int>(1);
    if (B.p == 1) {
        B.tscr = A.take<double>(lanczos_team_scratch_doubles(B.max_n, B.mmax, B.r));
        B.tbar = A.take<unsigned>(4);
    }
}

// Tuning-cache key of a batch's eigen-solve (the batch shape, Q precision,
// whether symmetric ranges are allowed, the device).
std::string batch_tune_key(const Batch& B, int q_f32, int sym) {
    double sum_n2 = 0.0;
    for (const ProbDesc& P : B.desc) sum_n2 += (double)P.n * P.n;
    return lanczos_tune_key(B.p, B.max_n, sum_n2, B.mmax, B.r, q_f32, sym);
}

// CTAs per eigenproblem when the call does not fix it (and no tuned value is
// cached).  Two CTAs per SM are resident, so `slots / cs` problems run at a
// time.  Many small problems (enough to fill every slot): the smallest
// cs <= 4 whose concurrently active Q matrices fit in ~112 MB of L2 (they are re-read every Lanczos step; fast
// MDS's 400-point leaves: 35 ms at cs = 2 against 47 ms at 1 and 46 ms at 4).
// Otherwise about 1.5 problems per cluster slot, so that largest-first
// scheduling evens out uneven sizes, and at least one CTA per ~400 rows
// (D&C parts of 1,000 points: cs = 5; of 2,050 points: cs = 5, 211 ms
// against 283 ms at cs = 1).
int pick_cluster(int requested, int p, int max_n, int mmax, int r, double sum_n2, int q_bytes) {
    if (requested > 0) return std::min(requested, 16);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int slots = 2 * sms;
    int cs = 0;
    if (p == 1) {
        cs = 16;
    } else {
        const double mean_q = sum_n2 / p * q_bytes;
        for (int c = 1; c <= 4 && cs == 0; ++c)
            if ((int64_t)p * c >= slots && (slots / c) * mean_q <= 112.0 * (1 << 20) &&
                lanczos_smem_bytes(max_n, c, mmax, r) <= kMaxSmem)
                cs = c;
        if (cs == 0) {
            cs = std::max(1, std::min(8, (int)std::lround(2.0 * sms * 1.5 / p)));
            cs = std::max(cs, std::min(16, (int)std::lround(max_n / 400.0)));
        }
    }
    cs = std::min(cs, std::max(1, max_n / 64));
    while (cs < 16 && lanczos_smem_bytes(max_n, cs, mmax, r) > kMaxSmem) ++cs;
    return cs;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return MDS_ERR_CUDA; \
    } while (0)

// Tensor-core part Gram of byte rows (divide-and-conquer with BF16 or FP8
// distances): the encoded member rows, their norms and the work units.
struct GramOp {
    int mode = -1;                 // kTckBf16 / kTckFp8, or -1: SIMT distance tiles
    int64_t slots = 0;             // operand rows (parts at 4-aligned offsets)
    std::vector<int> h_moff;       // per part: first operand row
    std::vector<int4> h_units;     // (part, row0, col0, moff)
    int* moff = nullptr;
    int4* units = nullptr;
    void* ops = nullptr;
    float* nrm = nullptr;
    int* kerr = nullptr;
};

// Uploads descriptors, forms Q_j for every problem (squared distances +
// double centering) and runs the batched eigen-solver.  acc_f64: FP64 dot
// products for the distances.  eig_f64: Q, the Lanczos vectors and the
// products in IEEE FP64; otherwise Q is stored in FP32 and the products and
// vector work run in double-FP32 (with FP64 scalars).
int run_eig_batch(Batch& B, const void* Y, int dt, int d, const double* nrm,
                  const int64_t* anchors, const int64_t* own, int acc_f64, int eig_f64, const Opts& o,
                  bool upload = true, const GramOp* gram = nullptr, bool center = true, bool mark_dist = true) {
    if (upload) {
        CK(cudaMemcpyAsync(B.d_desc, B.desc.data(), sizeof(ProbDesc) * B.p, cudaMemcpyHostToDevice, o.st));
        CK(cudaMemcpyAsync(B.d_order, B.order.data(), sizeof(int) * B.p, cudaMemcpyHostToDevice, o.st));
        if (gram && gram->mode >= 0) {
            CK(cudaMemcpyAsync(gram->moff, gram->h_moff.data(), sizeof(int) * B.p, cudaMemcpyHostToDevice, o.st));
            CK(cudaMemcpyAsync(gram->units, gram->h_units.data(), sizeof(int4) * gram->h_units.size(),
                               cudaMemcpyHostToDevice, o.st));
        }
    }
    CK(cudaMemsetAsync(B.counter, 0, sizeof(int), o.st));
    if (gram && gram->mode >= 0) {
        CK(cudaMemsetAsync(gram->kerr, 0, sizeof(int), o.st));
        CK(launch_encode_parts_u8(gram->mode, (const uint8_t*)Y, d, anchors, own, B.d_desc, gram->moff, B.p,
                                  gram->slots, gram->ops, gram->nrm, o.st));
        CK(launch_gram_tck(gram->mode, gram->ops, gram->slots, d, gram->nrm, gram->units,
                           (int)gram->h_units.size(), B.d_desc, B.q, B.rp, gram->kerr, o.st));
    } else if (Y) {
        CK(launch_sqdist_batched(Y, dt, d, nrm, anchors, own, B.d_desc, B.p, B.max_tiles, acc_f64, eig_f64,
                                 B.q, B.rp, o.st));
    }
    if (mark_dist) tmark(1, o.st);   // else the caller marked the end of its distance stage
    // An FP64 eigenproblem keeps Q and the products in IEEE FP64.  The
    // divide-and-conquer parts of the other precisions, whose Q carries
    // FP32-level distance rounding anyway, store Q in FP32 and run the
    // products and vector work in double-FP32.
    const int q_f32 = !eig_f64;
    B.q_bytes = q_f32 ? 4 : 8;
    // (center = false: Q is already in the arena, FP64, e.g. pivot MDS's C^T C)
    if (center) CK(launch_center_batched(B.d_desc, B.p, B.max_n, B.q, B.rp, B.rm, B.grand, q_f32, o.st));
    LanczosArgs a;
    a.desc = B.d_desc;
    a.p = B.p;
    a.qarena = B.q;
    a.barena = B.b;
    a.varena = B.v;
    a.lam = B.lam;
    a.status = B.status;
    a.steps = B.steps;
    a.scratch = B.scr;
    a.order = B.d_order;
    a.q_f32 = q_f32;
    a.counter = B.counter;
    a.r = B.r;
    a.mmax = B.mmax;
    a.tol = o.tol;
    a.rank_tol = o.rank_tol;
    a.max_n = B.max_n;
    a.team = 1;
    a.tscr = B.tscr;
    a.tbar = B.tbar;
    a.sym = (o.flags & MDS_FLAG_FULL_MATVEC) == 0;
    a.wait_ns = wait_limit_ns();
    B.sym = a.sym;
    if (B.tbar) CK(cudaMemsetAsync(B.tbar, 0, 4 * sizeof(unsigned), o.st));
    tmark(2, o.st);
    double sum_n2 = 0.0;
    for (const ProbDesc& P : B.desc) sum_n2 += (double)P.n * P.n;
    g_cluster = pick_cluster(o.cluster, B.p, B.max_n, B.mmax, B.r, sum_n2, q_f32 ? 4 : 8);
    if (o.cluster == 0 && tune_enabled()) {
        // a cluster size an autotuner measured for this batch shape
        int v = 0;
        if (tune_lookup(batch_tune_key(B, q_f32, a.sym), &v, nullptr, 0) && v >= 1 && v <= 16 &&
            lanczos_smem_bytes(B.max_n, v, B.mmax, B.r) <= kMaxSmem)
            g_cluster = v;
    }
    CK(launch_lanczos(a, g_cluster, o.st, o.cluster == 0));
    B.team = lanczos_last_team();
    tmark(3, o.st);
    return MDS_OK;
}

// Waits for the stream and folds the device status words into one code.
int batch_status(const Batch& B, const int* hs, const int* steps, int flag, int kerr);

int finish(const Batch* B, const int* d_flag, const Opts& o, const int* d_kerr = nullptr) {
    tmark(4, o.st);
    std::vector<int> hs(B ? B->p : 0), steps(B ? B->p : 0);
    int flag = 0, kerr = 0;
    unsigned team_abort = 0;
    if (d_kerr) CK(cudaMemcpyAsync(&kerr, d_kerr, sizeof(int), cudaMemcpyDeviceToHost, o.st));
    // a team solve that aborted a grid barrier reports it here even where a
    // cluster finished its own part (the word is read after the launch ends)
    if (B && B->team && B->tbar)
        CK(cudaMemcpyAsync(&team_abort, B->tbar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, o.st));
    if (B && B->p) {
        CK(cudaMemcpyAsync(hs.data(), B->status, sizeof(int) * B->p, cudaMemcpyDeviceToHost, o.st));
        CK(cudaMemcpyAsync(steps.data(), B->steps, sizeof(int) * B->p, cudaMemcpyDeviceToHost, o.st));
    }
    if (d_flag) CK(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, o.st));
    CK(cudaStreamSynchronize(o.st));
    CK(cudaGetLastError());
    if (g_timing)
        for (int i = 0; i < 5; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, g_ev[i], g_ev[i + 1]);
            g_last.stage_ms[i] = ms;
        }
    nvtx_end_call();
    if (B) return batch_status(*B, hs.data(), steps.data(), flag, kerr ? kerr : (team_abort ? MDS_ERR_TIMEOUT : 0));
    g_last.launches = g_launches;
    g_last.cluster = g_cluster;
    if (flag) return MDS_ERR_ARG;
    return kerr;
}

bool valid_dt(int dt) { return dt == MDS_IN_F64 || dt == MDS_IN_F32 || dt == MDS_IN_U8; }

// --------------------------------------------------------------- layouts

struct ClassicalWs {
    int* flag;
    double* nrm;
    int64_t* iota;
    Batch B;
};

size_t classical_layout(ClassicalWs& W, char* base, int64_t n, int r, int mmax) {
    Arena A{base, 0};
    W.flag = A.take<int>(1);
    W.nrm = A.take<double>(n);
    W.iota = A.take<int64_t>(n);
    plan_batch(W.B, {(int)n}, {0}, 0, r, mmax, n);
    carve_batch(W.B, A);
    return A.off;
}

struct InterpWs {
    int* flag;
    int* kerr;        // device error word of the tensor-core kernel
    float* nrm_lf;    // tensor-core paths: landmark norms as float (zero-padded)
    float* Wpad;      // tensor-core paths: W padded to gower_tc_rp(r) columns
    double* nrm;
    double* nrm_raw;  // BF16 path: FP32 norms of the unrounded rows (landmark problem)
    float* nrm_f;     // byte-row paths: exact norms of the rows as float
    void* Yq;
    Batch B;
    void* L;
    double* nrm_l;
    void* W;
    double* bias;
    void* X1;
};

size_t interp_layout(InterpWs& W, char* base, int64_t n, int d, int l, int r, int prec, int kind, int mmax) {
    Arena A{base, 0};
    const size_t es = prec == MDS_PREC_F64 ? 8 : 4;
    const bool split = prec == MDS_PREC_BF16 && kind == kKindRows;
    W.flag = A.take<int>(1);
    W.kerr = A.take<int>(1);
    W.nrm_lf = A.take<float>(model_nlf_count(kind, l));
    W.Wpad = A.take<float>(model_W_bytes(kind, prec, l, r) / 4 + 16 * (size_t)l);
    W.nrm = A.take<double>(n);
    W.nrm_raw = (split || kind != kKindRows) ? A.take<double>(n) : nullptr;
    W.nrm_f = kind != kKindRows ? A.take<float>(n) : nullptr;
    W.Yq = split ? (void*)A.take<uint16_t>((size_t)2 * n * split_ld(d))
                 : (kind != kKindRows ? (void*)A.take<char>(tck_operand_bytes(kind - 1, n, d)) : nullptr);
    plan_batch(W.B, {l}, {0}, 0, r, mmax, n);
    carve_batch(W.B, A);
    W.L = A.take<char>(model_L_bytes(kind, prec, l, d));
    W.nrm_l = A.take<double>(l);
    W.W = A.take<char>((size_t)l * r * es);
    W.bias = A.take<double>(r);
    W.X1 = A.take<char>((size_t)l * r * es);
    return A.off;
}

struct DcWs {
    int* flag;
    double* nrm;
    void* Yq;
    Batch B;
    double* Tt;
    GramOp G;
};

size_t dc_layout(DcWs& W, char* base, int64_t n, int d, int p, const int64_t* part_ptr, int c,
                 int r, int prec, int mmax) {
    Arena A{base, 0};
    W.flag = A.take<int>(1);
    W.nrm = A.take<double>(n);
    W.Yq = nullptr;
    std::vector<int> sizes(p);
    std::vector<int64_t> offs(p);
    for (int j = 0; j < p; ++j) {
        sizes[j] = (int)(part_ptr[j + 1] - part_ptr[j]) + c;
        offs[j] = part_ptr[j];
    }
    plan_batch(W.B, sizes, offs, c, r, mmax, n);
    carve_batch(W.B, A);
    W.Tt = A.take<double>((size_t)p * (r * r + r));
    // BF16 / FP8 (byte rows): tensor-core part Gram
    W.G = GramOp();
    if (prec == MDS_PREC_BF16 || prec == MDS_PREC_FP8) {
        GramOp& G = W.G;
        G.mode = prec == MDS_PREC_FP8 ? kTckFp8 : kTckBf16;
        G.h_moff.resize(p);
        int64_t slots = 0;
        for (int j = 0; j < p; ++j) {
            G.h_moff[j] = (int)slots;
            const int nj = sizes[j];
            slots += round_up(nj, 4);
            for (int r0 = 0; r0 < nj; r0 += 128)
                for (int c0 = 0; c0 < nj; c0 += 256) G.h_units.push_back(make_int4(j, r0, c0, G.h_moff[j]));
        }
        G.slots = slots;
        G.kerr = A.take<int>(1);
        G.moff = A.take<int>(p);
        G.units = A.take<int4>(G.h_units.size());
        G.nrm = A.take<float>((size_t)slots + 256);
        G.ops = A.take<char>(gram_operand_bytes(G.mode, slots, d));
    }
    return A.off;
}

// Norms (and the BF16-rounded copy) of the data; returns the dtype tag and
// pointer the distance kernels read.
int prep_data(const void* Y, int dt, int64_t n, int d, int prec, double* nrm, void* Yq,
              const Opts& o, const void** Yeff, int* dteff) {
    if (prec == MDS_PREC_BF16) {
        CK(launch_quant_bf16(Y, dt, n, d, Yq, nrm, o.st));
        *Yeff = Yq;
        *dteff = kDtBF16;
    } else {
        CK(launch_rownorm(Y, dt, n, d, prec == MDS_PREC_F64, nrm, o.st));
        *Yeff = Y;
        *dteff = dt;
    }
    return MDS_OK;
}

// The whole divide-and-conquer launch sequence on o.st, without waiting:
// index checks, norms, every part's distance tiles, centering and eigenpairs
// (one persistent launch), Procrustes, alignment and lambda-bar.  The
// workspace W is carved; upload = false when its part descriptors are
// already on the device.
int dc_enqueue(DcWs& W, const void* Y, int dt, int64_t n, int d, int p, const int64_t* part_ptr,
               const int64_t* part_own, const int64_t* anchors, int c, int r, const Opts& o, void* X,
               double* var, bool upload) {
    const int f64 = o.prec == MDS_PREC_F64;
    CK(cudaMemsetAsync(W.flag, 0, sizeof(int), o.st));
    CK(launch_check_idx(anchors, c, n, W.flag, o.st));
    CK(launch_check_idx(part_own, part_ptr[p], n, W.flag, o.st));
    const void* Ye = Y;
    int dte = dt;
    int s = MDS_OK;
    if (W.G.mode < 0 && (s = prep_data(Y, dt, n, d, o.prec, W.nrm, W.Yq, o, &Ye, &dte))) return s;
    tmark(0, o.st);
    if ((s = run_eig_batch(W.B, Ye, dte, d, W.nrm, anchors, part_own, f64, f64, o, upload, &W.G))) return s;
    CK(launch_dc_procrustes(W.B.d_desc, p, W.B.v, W.B.lam, r, c, W.Tt, o.st));
    CK(launch_dc_align(W.B.d_desc, p, W.B.max_n, W.B.v, W.B.lam, W.Tt, r, anchors, part_own, f64, X, o.st));
    CK(launch_dc_lambda_bar(W.B.d_desc, p, W.B.lam, r, var, o.st));
    tmark(4, o.st);
    return MDS_OK;
}

// Stats of a finished batch from host copies of its status words.
int batch_status(const Batch& B, const int* hs, const int* steps, int flag, int kerr) {
    g_last.launches = g_launches;
    g_last.cluster = g_cluster;
    g_last.problems = B.p;
    for (int j = 0; j < B.p; ++j) {
        const double n = B.desc[j].n, k = steps[j];
        g_last.eig_steps += steps[j];
        g_last.eig_flops += 2.0 * n * n * k + 8.0 * n * k + 2.0 * n * k * (k + 1) + 2.0 * n * k * B.r;
        g_last.eig_qbytes += (double)B.q_bytes * n * n * k;
        g_last.eig_qread += lanczos_step_bytes(B.desc[j].n, g_cluster, B.q_bytes == 4, B.sym, B.team) * k;
    }
    if (flag) return MDS_ERR_ARG;
    if (kerr) return kerr;
    int worst = MDS_OK;
    for (int j = 0; j < B.p; ++j) {
        if (hs[j] == MDS_ERR_RANK) return MDS_ERR_RANK;
        if (hs[j] != MDS_OK) worst = hs[j];
    }
    return worst;
}

}  // namespace

// Queues the embedding of `rows` new points on `st` without waiting: norms
// (and the BF16 split for BF16 models), then the fused distance + Gower
// projection kernel.  `ws` holds at least mds_embed_new_workspace_size() - 256
// bytes, 256-byte aligned; *kerr receives the device status word (zero when
// the kernel succeeded), which lives at the start of ws.
int gbmds::embed_enqueue(mds_model m, const void* Ynew, int dt, int64_t rows, char* ws, cudaStream_t st,
                         void* X, int** kerr_out) {
    Opts o{};
    o.prec = m->prec;
    o.st = st;
    o.ws = ws;
    Arena A{ws, 0};
    int* kerr = A.take<int>(1);
    double* nrm = A.take<double>(rows);
    *kerr_out = kerr;
    if (m->kind != kKindRows) {
        // byte-row models project byte rows only (the operands are exact)
        if (dt != MDS_IN_U8) return MDS_ERR_ARG;
        void* Yk = A.take<char>(tck_operand_bytes(m->kind - 1, rows, m->d));
        float* nf = reinterpret_cast<float*>(nrm);
        CK(cudaMemsetAsync(kerr, 0, sizeof(int), st));
        CK(launch_encode_u8(m->kind - 1, (const uint8_t*)Ynew, rows, m->d, Yk, nf, st));
        for (int i = 0; i < 4; ++i) tmark(i, st);
        CK(launch_gower_tck(m->kind - 1, Yk, rows, m->d, nf, m->L, m->l, m->nrm_lf, (const float*)m->W, m->bias,
                            m->r, (float*)X, kerr, st));
        return MDS_OK;
    }
    void* Yq = m->prec == MDS_PREC_BF16 ? (void*)A.take<uint16_t>((size_t)2 * rows * split_ld(m->d)) : nullptr;
    CK(cudaMemsetAsync(kerr, 0, sizeof(int), st));
    const void* Ye;
    int dte;
    int s = prep_data(Ynew, dt, rows, m->d, m->prec, nrm, Yq, o, &Ye, &dte);
    if (s) return s;
    for (int i = 0; i < 4; ++i) tmark(i, st);   // stage 0 = preparation, stage 4 = projection
    if (m->prec == MDS_PREC_BF16) {
        CK(launch_gower_tc(Ye, rows, rows, m->d, nrm, m->L, m->nrm_lf, m->l, m->W, m->bias,
                           m->r, (float*)X, kerr, st));
        return MDS_OK;
    }
    CK(launch_gower_proj(Ye, dte, rows, m->d, nrm, m->L, m->nrm_l, m->l, m->W, m->bias, m->r,
                         m->prec == MDS_PREC_F64, X, st));
    return MDS_OK;
}

// =================================================================== C ABI

extern "C" {

const char* mds_status_str(int s) {
    switch (s) {
        case MDS_OK: return "ok";
        case MDS_ERR_ARG: return "invalid argument";
        case MDS_ERR_NOMEM: return "device allocation failed";
        case MDS_ERR_CUDA: return "CUDA error";
        case MDS_ERR_RANK: return "fewer than r positive eigenvalues";
        case MDS_ERR_NOCONV: return "eigen-solver did not converge";
        case MDS_ERR_TIMEOUT: return "device wait timed out";
        case MDS_ERR_UNSUPPORTED: return "unsupported precision or dtype";
        case MDS_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case MDS_ERR_IO: return "model file error";
        default: return "unknown status";
    }
}

int mds_version(void) { return 1; }

void mds_set_timing(int on) { g_timing = on != 0; }

int mds_lanczos_phase_cycles(double* out, int reset) {
    if (!out && !reset) return MDS_ERR_ARG;
    return lanczos_phase_cycles(out, reset);
}

void mds_set_wait_limit_ns(unsigned long long ns) { g_wait_ns.store(ns); }

void mds_inject_alloc_failures(int count) { g_fail_allocs.store(count > 0 ? count : 0); }

int mds_last_stats(mds_stats* out) {
    if (!out) return MDS_ERR_ARG;
    *out = g_last;
    return MDS_OK;
}

// ------------------------------------------------------ MaxMin landmarks

static size_t maxmin_layout(MaxminWs& M, char* base, int64_t n) {
    Arena A{base, 0};
    M.mind = A.take<double>(n);
    M.nrm8 = A.take<int>(n);
    M.cur = A.take<int64_t>(1);
    M.part_v = A.take<double>(kMaxminGridCap);
    M.part_i = A.take<int64_t>(kMaxminGridCap);
    M.counter = A.take<unsigned>(1);
    M.err = A.take<int>(1);
    return A.off;
}

size_t mds_landmarks_maxmin_workspace_size(int64_t n, int d) {
    if (n <= 0 || d <= 0) return 0;
    MaxminWs M;
    return maxmin_layout(M, nullptr, n) + 256;
}

int mds_landmarks_maxmin(const void* Y, int dt, int64_t n, int d, int l, int64_t first, const mds_opts* opts,
                         int64_t* idx_out) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (!Y || !idx_out || !valid_dt(dt) || n < 1 || d <= 0 || l < 1 || l > n || first < 0 || first >= n)
        return MDS_ERR_ARG;
    if (d > kMaxminD) return MDS_ERR_UNSUPPORTED;
    MaxminWs M;
    const size_t need = maxmin_layout(M, nullptr, n);
    if ((s = check_ws(o, need))) return s;
    maxmin_layout(M, o.ws, n);
    begin_call(o.st, __func__);
    CK(cudaMemsetAsync(M.err, 0, sizeof(int), o.st));
    tmark(0, o.st);
    CK(launch_maxmin(Y, dt, n, d, l, first, M, idx_out, o.st));
    tmark(1, o.st);   // stage "dist": the l - 1 distance passes and picks
    tmark(2, o.st);
    tmark(3, o.st);
    return finish(nullptr, nullptr, o, M.err);
}

// ------------------------------------------------------------- classical

size_t mds_classical_workspace_size(int64_t n, int d, int r, int prec) {
    (void)d;
    (void)prec;
    if (n <= 0 || n > kMaxEigN || r <= 0) return 0;
    ClassicalWs W;
    return classical_layout(W, nullptr, n, r, kDefaultSteps) + 256;
}

int mds_classical(const void* Y, int dt, int64_t n, int d, int r, const mds_opts* opts, void* X,
                  double* lambda) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (!Y || !X || !lambda || !valid_dt(dt) || n < 2 || n > kMaxEigN || d <= 0 || r <= 0 ||
        r > kMaxR || r >= n)
        return MDS_ERR_ARG;
    if (o.prec != MDS_PREC_F64 && o.prec != MDS_PREC_F32) return MDS_ERR_UNSUPPORTED;
    ClassicalWs W;
    const size_t need = classical_layout(W, nullptr, n, r, o.mmax);
    if ((s = check_ws(o, need))) return s;
    if (classical_layout(W, o.ws, n, r, o.mmax) != need) return MDS_ERR_WORKSPACE;
    begin_call(o.st, __func__);
    CK(cudaMemsetAsync(W.flag, 0, sizeof(int), o.st));
    CK(launch_iota(W.iota, n, o.st));
    const int f64 = o.prec == MDS_PREC_F64;
    CK(launch_rownorm(Y, dt, n, d, f64, W.nrm, o.st));
    tmark(0, o.st);
    if ((s = run_eig_batch(W.B, Y, dt, d, W.nrm, nullptr, W.iota, f64, f64, o))) return s;
    CK(launch_classical_out(W.B.v, W.B.lam, (int)n, r, f64, X, lambda, o.st));
    return finish(&W.B, W.flag, o);
}

size_t mds_classical_dist_workspace_size(int64_t n, int r) {
    if (n <= 0 || n > kMaxEigN || r <= 0) return 0;
    ClassicalWs W;
    return classical_layout(W, nullptr, n, r, kDefaultSteps) + 256;
}

int mds_classical_dist(const double* D2, int64_t n, int r, const mds_opts* opts, double* X,
                       double* lambda) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (!D2 || !X || !lambda || n < 2 || n > kMaxEigN || r <= 0 || r > kMaxR || r >= n)
        return MDS_ERR_ARG;
    ClassicalWs W;
    const size_t need = classical_layout(W, nullptr, n, r, o.mmax);
    if ((s = check_ws(o, need))) return s;
    if (classical_layout(W, o.ws, n, r, o.mmax) != need) return MDS_ERR_WORKSPACE;
    begin_call(o.st, __func__);
    CK(cudaMemcpyAsync(W.B.d_desc, W.B.desc.data(), sizeof(ProbDesc), cudaMemcpyHostToDevice, o.st));
    tmark(0, o.st);
    CK(launch_load_dist(D2, W.B.d_desc, W.B.q, W.B.rp, (int)n, W.B.max_tiles, o.st));
    if ((s = run_eig_batch(W.B, nullptr, 0, 0, nullptr, nullptr, nullptr, 1, 1, o))) return s;
    CK(launch_classical_out(W.B.v, W.B.lam, (int)n, r, 1, X, lambda, o.st));
    return finish(&W.B, nullptr, o);
}

// ---------------------------------------------------------- interpolation

size_t mds_interpolate_workspace_size(int64_t n, int d, int l, int r, int prec) {
    if (n <= 0 || d <= 0 || l <= 0 || l > kMaxEigN || r <= 0) return 0;
    // the precision alone does not fix the kind (BF16 of byte rows differs from
    // BF16 of float rows): size for the larger of the kinds it may take
    InterpWs W;
    size_t need = 0;
    const int kinds[3] = {kKindRows, kKindU8Bf16, kKindU8Fp8};
    for (int k : kinds) {
        if (k == kKindRows && prec == MDS_PREC_FP8) continue;
        if (k != kKindRows && (k == kKindU8Fp8) != (prec == MDS_PREC_FP8)) continue;
        if (k == kKindU8Bf16 && prec != MDS_PREC_BF16) continue;
        need = std::max(need, interp_layout(W, nullptr, n, d, l, r, prec, k, kDefaultSteps));
    }
    return need + 256;
}

// Copies the interpolation model of a finished call out of its workspace into
// a device-resident handle for mds_embed_new.
static int make_model(InterpWs& W, int kind, const Opts& o, int l, int d, int r, mds_model* out_model) {
    const int f64 = o.prec == MDS_PREC_F64;
    // device-resident model for mds_embed_new
    mds_model m = new (std::nothrow) mds_model_s();
    if (!m) return MDS_ERR_NOMEM;
    const size_t es = f64 ? 8 : 4;
    m->l = l;
    m->d = d;
    m->r = r;
    m->prec = o.prec;
    m->kind = kind;
    cudaGetDevice(&m->device);
    const size_t szL = model_L_bytes(kind, o.prec, l, d);
    const size_t szW = model_W_bytes(kind, o.prec, l, r);
    const size_t nlf = model_nlf_count(kind, l);
    bool ok = dev_malloc(&m->L, szL) == cudaSuccess &&
              dev_malloc((void**)&m->nrm_l, sizeof(double) * l) == cudaSuccess &&
              dev_malloc((void**)&m->nrm_lf, sizeof(float) * nlf) == cudaSuccess &&
              dev_malloc(&m->W, szW) == cudaSuccess &&
              dev_malloc((void**)&m->bias, sizeof(double) * r) == cudaSuccess &&
              dev_malloc(&m->X1, (size_t)l * r * es) == cudaSuccess &&
              dev_malloc((void**)&m->lam, sizeof(double) * r) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mds_model_free(m);
        return MDS_ERR_NOMEM;
    }
    ok = cudaMemcpyAsync(m->L, W.L, szL, cudaMemcpyDeviceToDevice, o.st) == cudaSuccess &&
         cudaMemcpyAsync(m->nrm_l, W.nrm_l, sizeof(double) * l, cudaMemcpyDeviceToDevice, o.st) == cudaSuccess &&
         cudaMemcpyAsync(m->nrm_lf, W.nrm_lf, sizeof(float) * nlf, cudaMemcpyDeviceToDevice, o.st) == cudaSuccess &&
         cudaMemcpyAsync(m->W, (kind != kKindRows || o.prec == MDS_PREC_BF16) ? (void*)W.Wpad : W.W, szW,
                         cudaMemcpyDeviceToDevice, o.st) == cudaSuccess &&
         cudaMemcpyAsync(m->bias, W.bias, sizeof(double) * r, cudaMemcpyDeviceToDevice, o.st) == cudaSuccess &&
         cudaMemcpyAsync(m->X1, W.X1, (size_t)l * r * es, cudaMemcpyDeviceToDevice, o.st) == cudaSuccess &&
         cudaMemcpyAsync(m->lam, W.B.lam, sizeof(double) * r, cudaMemcpyDeviceToDevice, o.st) == cudaSuccess &&
         cudaStreamSynchronize(o.st) == cudaSuccess;
    if (!ok) {
        mds_model_free(m);
        return MDS_ERR_CUDA;
    }
    *out_model = m;
    return MDS_OK;
}

// ------------------------------------------------ affine interpolation

struct AffineWs {
    int* flag;
    int* kerr;        // status word of the pass over Y
    double* Lg;       // l x d: the landmark rows, gathered as FP64
    int64_t* iota;    // l
    double* nrm;      // l: their squared norms (the landmark problem indexes Lg through iota)
    Batch B;
    double* ybar;     // d
    float* ybar_f;
    double* scale;    // r: Lambda^{-1/2}
    double* U;        // d x r
    float* U_f;
    double* bias;     // r: the Gower bias (written with the variances; not used by the affine form)
};

static size_t affine_layout(AffineWs& W, char* base, int d, int l, int r, int mmax) {
    Arena A{base, 0};
    W.flag = A.take<int>(1);
    W.kerr = A.take<int>(1);
    W.Lg = A.take<double>((size_t)l * d);
    W.iota = A.take<int64_t>(l);
    W.nrm = A.take<double>(l);
    plan_batch(W.B, {l}, {0}, 0, r, mmax, l);
    carve_batch(W.B, A);
    W.ybar = A.take<double>(d);
    W.ybar_f = A.take<float>(d);
    W.scale = A.take<double>(r);
    W.U = A.take<double>((size_t)d * r);
    W.U_f = A.take<float>((size_t)d * r);
    W.bias = A.take<double>(r);
    return A.off;
}

size_t mds_interpolate_affine_workspace_size(int64_t n, int d, int l, int r, int prec) {
    if (n <= 0 || d <= 0 || l <= 0 || l > kMaxEigN || r <= 0 || r > kMaxR) return 0;
    if (prec != MDS_PREC_F64 && prec != MDS_PREC_F32) return 0;
    AffineWs W;
    return affine_layout(W, nullptr, d, l, r, kDefaultSteps) + 256;
}

int mds_interpolate_affine(const void* Y, int dt, int64_t n, int d, const int64_t* landmark_idx, int l, int r,
                           const mds_opts* opts, void* X, double* var) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (!Y || !X || !var || !landmark_idx || !valid_dt(dt) || n < 2 || d <= 0 || l < 2 || l > n ||
        l > kMaxEigN || r <= 0 || r > kMaxR || r >= l)
        return MDS_ERR_ARG;
    if (o.prec != MDS_PREC_F64 && o.prec != MDS_PREC_F32) return MDS_ERR_UNSUPPORTED;
    AffineWs W;
    const size_t need = affine_layout(W, nullptr, d, l, r, o.mmax);
    if ((s = check_ws(o, need))) return s;
    if (affine_layout(W, o.ws, d, l, r, o.mmax) != need) return MDS_ERR_WORKSPACE;
    begin_call(o.st, __func__);
    const int f64 = o.prec == MDS_PREC_F64;
    CK(cudaMemsetAsync(W.flag, 0, sizeof(int), o.st));
    CK(cudaMemsetAsync(W.kerr, 0, sizeof(int), o.st));
    CK(launch_check_idx(landmark_idx, l, n, W.flag, o.st));
    // the landmark problem of mds_interpolate on the gathered landmark rows
    // (FP64 copies of the inputs: the same distances in the same arithmetic)
    CK(launch_gather_rows(Y, dt, n, d, landmark_idx, l, 1, W.Lg, nullptr, nullptr, o.st));
    CK(launch_iota(W.iota, l, o.st));
    CK(launch_rownorm(W.Lg, MDS_IN_F64, l, d, f64, W.nrm, o.st));
    tmark(0, o.st);
    if ((s = run_eig_batch(W.B, W.Lg, MDS_IN_F64, d, W.nrm, nullptr, W.iota, f64, 1, o))) return s;
    CK(launch_interp_model(W.B.v, W.B.lam, W.B.q, W.B.desc[0].ldq, 0, l, r, nullptr, nullptr, nullptr,
                           nullptr, W.bias, var, o.st));
    CK(launch_affine_axes(W.Lg, l, d, W.B.v, W.B.lam, r, W.scale, W.ybar, W.ybar_f, W.U, W.U_f, o.st));
    tmark(3, o.st);   // the stage "post" is the one pass over Y
    CK(launch_affine_project(Y, dt, n, d, W.ybar, W.ybar_f, W.U, W.U_f, r, f64, X, W.kerr, o.st));
    return finish(&W.B, W.flag, o, W.kerr);
}

// ---------------------------------------------------------------- pivot MDS

struct PivotWs {
    int* flag;
    int* kerr;        // status word of the pass over Y
    double* cpart;    // column-sum partials
    double* mean;     // d: mean of all n rows
    float* mean_f;
    double* spart;    // scatter partials
    double* S;        // d x d
    double* Lg;       // l x d: the pivot rows (FP64)
    double* T;        // l x d: (Lg - mean) S
    Batch B;          // the l x l problem C^T C
    double* scale;    // r
    double* U;        // d x r
    float* U_f;
    double* sg_v;     // sign-convention partials
    int64_t* sg_i;
    unsigned* sg_cnt;
    double* sign;     // r
};

static size_t pivot_layout(PivotWs& W, char* base, int64_t n, int d, int l, int r, int mmax) {
    Arena A{base, 0};
    W.flag = A.take<int>(1);
    W.kerr = A.take<int>(1);
    W.cpart = A.take<double>(colmean_part_doubles(n, d));
    W.mean = A.take<double>(d);
    W.mean_f = A.take<float>(d);
    W.spart = A.take<double>(scatter_part_doubles(n, d));
    W.S = A.take<double>((size_t)d * d);
    W.Lg = A.take<double>((size_t)l * d);
    W.T = A.take<double>((size_t)l * d);
    plan_batch(W.B, {l}, {0}, 0, r, mmax, l);
    carve_batch(W.B, A);
    W.scale = A.take<double>(r);
    W.U = A.take<double>((size_t)d * r);
    W.U_f = A.take<float>((size_t)d * r);
    const int g = colsign_grid(n);
    W.sg_v = A.take<double>((size_t)g * r);
    W.sg_i = A.take<int64_t>((size_t)g * r);
    W.sg_cnt = A.take<unsigned>(1);
    W.sign = A.take<double>(r);
    return A.off;
}

size_t mds_pivot_workspace_size(int64_t n, int d, int l, int r, int prec) {
    if (n <= 0 || d <= 0 || l <= 0 || l > kMaxEigN || r <= 0 || r > kMaxR || !scatter_supported(d)) return 0;
    if (prec != MDS_PREC_F64 && prec != MDS_PREC_F32) return 0;
    PivotWs W;
    return pivot_layout(W, nullptr, n, d, l, r, kDefaultSteps) + 256;
}

int mds_pivot(const void* Y, int dt, int64_t n, int d, const int64_t* pivot_idx, int l, int r, const mds_opts* opts,
              void* X, double* var) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (!Y || !X || !var || !pivot_idx || !valid_dt(dt) || n < 2 || d <= 0 || l < 1 || l > n || l > kMaxEigN ||
        r <= 0 || r > kMaxR || r > l || r > d)
        return MDS_ERR_ARG;
    if ((o.prec != MDS_PREC_F64 && o.prec != MDS_PREC_F32) || !scatter_supported(d)) return MDS_ERR_UNSUPPORTED;
    PivotWs W;
    const size_t need = pivot_layout(W, nullptr, n, d, l, r, o.mmax);
    if ((s = check_ws(o, need))) return s;
    if (pivot_layout(W, o.ws, n, d, l, r, o.mmax) != need) return MDS_ERR_WORKSPACE;
    begin_call(o.st, __func__);
    const int f64 = o.prec == MDS_PREC_F64;
    CK(cudaMemsetAsync(W.flag, 0, sizeof(int), o.st));
    CK(cudaMemsetAsync(W.kerr, 0, sizeof(int), o.st));
    CK(cudaMemsetAsync(W.sg_cnt, 0, sizeof(unsigned), o.st));
    CK(launch_check_idx(pivot_idx, l, n, W.flag, o.st));
    // the centre and the scatter matrix of all n rows, the pivot rows
    CK(launch_colmean(Y, dt, n, d, W.cpart, W.mean, W.mean_f, o.st));
    CK(launch_gather_rows(Y, dt, n, d, pivot_idx, l, 1, W.Lg, nullptr, nullptr, o.st));
    tmark(0, o.st);
    CK(launch_scatter(Y, dt, n, d, W.mean, f64, W.spart, W.S, o.st));
    tmark(1, o.st);   // the stage "dist" is the scatter matrix; "center" forms C^T C
    // C^T C = P_c S P_c^T into the eigen-solver's Q slot (FP64)
    CK(launch_gemm_nt(W.Lg, d, W.mean, W.S, d, nullptr, l, d, d, W.T, d, 0, o.st));
    const ProbDesc& P0 = W.B.desc[0];
    CK(launch_gemm_nt(W.T, d, nullptr, W.Lg, d, W.mean, l, l, d, W.B.q + P0.q_off, P0.ldq, 1, o.st));
    if ((s = run_eig_batch(W.B, nullptr, 0, 0, nullptr, nullptr, nullptr, 1, 1, o, true, nullptr, false, false)))
        return s;
    // M = P_c^T W_r Sigma_r^{-1} Lambda_r^{1/2}; X = Y_c M; the sign convention
    CK(launch_pivot_scale(W.B.lam, r, n, l, W.scale, var, o.st));
    CK(launch_axes(W.Lg, l, d, W.mean, W.B.v, W.scale, r, W.U, W.U_f, o.st));
    tmark(3, o.st);   // the stage "post": the pass over Y for X and the sign convention
    CK(launch_affine_project(Y, dt, n, d, W.mean, W.mean_f, W.U, W.U_f, r, f64, X, W.kerr, o.st));
    CK(launch_colsign(X, f64, n, r, W.sg_v, W.sg_i, W.sg_cnt, W.sign, o.st));
    return finish(&W.B, W.flag, o, W.kerr);
}

int mds_interpolate(const void* Y, int dt, int64_t n, int d, const int64_t* landmark_idx, int l,
                    int r, const mds_opts* opts, void* X, double* var, mds_model* out_model) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (out_model) *out_model = nullptr;
    if (!Y || !X || !var || !landmark_idx || !valid_dt(dt) || n < 2 || d <= 0 || l < 2 ||
        l > n || l > kMaxEigN || r <= 0 || r > kMaxR || r >= l)
        return MDS_ERR_ARG;
    const int kind = model_kind(o.prec, dt, d, r);
    if (kind < 0) return MDS_ERR_UNSUPPORTED;
    InterpWs W;
    const size_t need = interp_layout(W, nullptr, n, d, l, r, o.prec, kind, o.mmax);
    if ((s = check_ws(o, need))) return s;
    if (interp_layout(W, o.ws, n, d, l, r, o.prec, kind, o.mmax) != need) return MDS_ERR_WORKSPACE;
    begin_call(o.st, __func__);
    const int f64 = o.prec == MDS_PREC_F64;
    CK(cudaMemsetAsync(W.flag, 0, sizeof(int), o.st));
    CK(cudaMemsetAsync(W.kerr, 0, sizeof(int), o.st));
    CK(launch_check_idx(landmark_idx, l, n, W.flag, o.st));
    const void* Ye = nullptr;
    int dte = dt;
    if (kind == kKindRows) {
        if ((s = prep_data(Y, dt, n, d, o.prec, W.nrm, W.Yq, o, &Ye, &dte))) return s;
    } else {
        // byte rows: exact tensor-core operands and exact norms
        CK(launch_encode_u8(kind - 1, (const uint8_t*)Y, n, d, W.Yq, W.nrm_f, o.st));
    }
    // The landmark problem is small: its distances come from the unrounded data
    // in FP32 even on the BF16 / FP8 paths, which use the tensor cores only for
    // the bulk of Eq. (2).
    const void* Yl = Ye;
    int dtl = dte;
    const double* nrml = W.nrm;
    if (o.prec == MDS_PREC_BF16 || o.prec == MDS_PREC_FP8) {
        CK(launch_rownorm_idx(Y, dt, n, d, landmark_idx, l, 0, W.nrm_raw, o.st));
        Yl = Y;
        dtl = dt;
        nrml = W.nrm_raw;
    }
    tmark(0, o.st);
    // classical MDS of the landmarks (first subset of Section 3.1): one small
    // l x l problem, solved in FP64 whatever the precision of the projection
    if ((s = run_eig_batch(W.B, Yl, dtl, d, nrml, nullptr, landmark_idx, f64, 1, o))) return s;
    // Gower operator, landmark rows, projection of every row, landmark rows <- X_1
    CK(launch_interp_model(W.B.v, W.B.lam, W.B.q, W.B.desc[0].ldq, 0, l, r,
                           f64 ? (double*)W.W : nullptr, f64 ? nullptr : (float*)W.W,
                           f64 ? (double*)W.X1 : nullptr, f64 ? nullptr : (float*)W.X1, W.bias,
                           var, o.st));
    if (kind != kKindRows) {
        // tensor-core distance tiles of byte rows fused with the Gower projection
        CK(launch_encode_landmarks_u8(kind - 1, (const uint8_t*)Y, n, d, landmark_idx, l, W.L, W.nrm_lf, o.st));
        CK(launch_pad_w_rows((const float*)W.W, l, r, W.Wpad, o.st));
        CK(launch_gower_tck(kind - 1, W.Yq, n, d, W.nrm_f, W.L, l, W.nrm_lf, W.Wpad, W.bias, r, (float*)X, W.kerr,
                            o.st));
    } else if (o.prec == MDS_PREC_BF16) {
        // tensor-core distance tiles fused with the Gower projection
        CK(cudaMemsetAsync(W.nrm_lf, 0, sizeof(float) * model_nlf_count(kind, l), o.st));
        CK(launch_gather_split(Ye, n, d, landmark_idx, l, W.L, W.nrm, W.nrm_lf, o.st));
        CK(launch_w_image((const float*)W.W, l, r, W.Wpad, o.st));
        CK(launch_gower_tc(Ye, n, n, d, W.nrm, W.L, W.nrm_lf, l, W.Wpad, W.bias, r, (float*)X,
                           W.kerr, o.st));
    } else {
        CK(launch_gather_rows(Ye, dte, n, d, landmark_idx, l, f64, W.L, W.nrm, W.nrm_l, o.st));
        CK(launch_gower_proj(Ye, dte, n, d, W.nrm, W.L, W.nrm_l, l, W.W, W.bias, r, f64, X, o.st));
    }
    CK(launch_scatter_rows(W.X1, landmark_idx, l, r, n, f64, X, o.st));
    s = finish(&W.B, W.flag, o, W.kerr);
    if (s != MDS_OK || !out_model) return s;
    return make_model(W, kind, o, l, d, r, out_model);
}

// ------------------------------------------ interpolation from host memory

struct InterpHostWs {
    InterpWs W;
    void* Yd;          // n x d of the input type: the rows as they arrive
    void* Xd;          // n x r (float, or double for FP64)
    void* Ylm;         // l x d: the landmark rows
    int64_t* idx;      // l: landmark indices (for the landmark rows of X)
    int64_t* iota;     // l
    double* nrm_lm;    // l: norms of the landmark rows for the landmark problem
    double* nrm_lms;   // l: BF16 split norms of the landmark rows
    void* Yq_lm;       // BF16 split planes of the landmark rows
    double* var;       // r
};

static size_t in_size(int dt) { return dt == MDS_IN_F64 ? 8 : (dt == MDS_IN_F32 ? 4 : 1); }

static size_t interp_host_layout(InterpHostWs& H, char* base, int64_t n, int d, int l, int r, int prec, int kind,
                          int dt, int mmax) {
    Arena A{base, interp_layout(H.W, base, n, d, l, r, prec, kind, mmax)};
    const size_t es = in_size(dt), ex = prec == MDS_PREC_F64 ? 8 : 4;
    H.Yd = A.take<char>((size_t)n * d * es);
    H.Xd = A.take<char>((size_t)n * r * ex);
    H.Ylm = A.take<char>((size_t)l * d * es);
    H.idx = A.take<int64_t>(l);
    H.iota = A.take<int64_t>(l);
    H.nrm_lm = A.take<double>(l);
    H.nrm_lms = A.take<double>(l);
    H.Yq_lm = A.take<uint16_t>((size_t)2 * l * split_ld(d));
    H.var = A.take<double>(r);
    return A.off;
}

// Default chunk: ~96 MiB of input rows (fewer, larger copies and launches
// measured faster than 64k-row chunks: 1M x 100 FP32 rows in 3.9 vs 4.2 ms),
// at least 16k rows.
static int64_t host_chunk_rows(int64_t n, int d, size_t es) {
    const int64_t rows = (int64_t)((96ull << 20) / ((size_t)d * es));
    return std::max<int64_t>(16384, std::min<int64_t>(rows, n));
}

// Streams and events of one host-input call, released on every return path.
struct HostPipe {
    cudaStream_t h2d = nullptr, d2h = nullptr;
    std::vector<cudaEvent_t> ev;
    ~HostPipe() {
        if (h2d) cudaStreamSynchronize(h2d);
        if (d2h) cudaStreamSynchronize(d2h);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (h2d) cudaStreamDestroy(h2d);
        if (d2h) cudaStreamDestroy(d2h);
    }
    cudaError_t make(int nev) {
        cudaError_t e = cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking);
        for (int i = 0; i < nev && e == cudaSuccess; ++i) {
            cudaEvent_t x;
            e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
            if (e == cudaSuccess) ev.push_back(x);
        }
        return e;
    }
};

size_t mds_interpolate_host_workspace_size(int64_t n, int d, int l, int r, int prec, int dt) {
    if (n <= 0 || d <= 0 || l <= 0 || l > kMaxEigN || r <= 0 || !valid_dt(dt)) return 0;
    const int kind = model_kind(prec, dt, d, r);
    if (kind < 0) return 0;
    InterpHostWs H;
    return interp_host_layout(H, nullptr, n, d, l, r, prec, kind, dt, kDefaultSteps) + 256;
}

int mds_interpolate_host(const void* Y, int dt, int64_t n, int d, const int64_t* landmark_idx, int l, int r,
                         int64_t chunk_rows, const mds_opts* opts, void* X, double* var, mds_model* out_model) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (out_model) *out_model = nullptr;
    if (!Y || !X || !var || !landmark_idx || !valid_dt(dt) || n < 2 || d <= 0 || l < 2 || l > n ||
        l > kMaxEigN || r <= 0 || r > kMaxR || r >= l || chunk_rows < 0)
        return MDS_ERR_ARG;
    for (int i = 0; i < l; ++i)
        if (landmark_idx[i] < 0 || landmark_idx[i] >= n) return MDS_ERR_ARG;
    const int kind = model_kind(o.prec, dt, d, r);
    if (kind < 0) return MDS_ERR_UNSUPPORTED;
    InterpHostWs H;
    const size_t need = interp_host_layout(H, nullptr, n, d, l, r, o.prec, kind, dt, o.mmax);
    if ((s = check_ws(o, need))) return s;
    if (interp_host_layout(H, o.ws, n, d, l, r, o.prec, kind, dt, o.mmax) != need) return MDS_ERR_WORKSPACE;
    InterpWs& W = H.W;
    const int f64 = o.prec == MDS_PREC_F64;
    const size_t es = in_size(dt), ex = f64 ? 8 : 4;
    const int64_t chunk = chunk_rows > 0 ? chunk_rows : host_chunk_rows(n, d, es);
    const int nch = (int)((n + chunk - 1) / chunk);
    const char* Yh = static_cast<const char*>(Y);
    char* Xh = static_cast<char*>(X);
    char* Yd = static_cast<char*>(H.Yd);
    char* Xd = static_cast<char*>(H.Xd);

    // the landmark rows, gathered on the host so that the landmark problem can
    // start before the bulk of the rows has crossed the link
    std::vector<char> lm((size_t)l * d * es);
    for (int i = 0; i < l; ++i) memcpy(lm.data() + (size_t)i * d * es, Yh + (size_t)landmark_idx[i] * d * es, d * es);

    HostPipe P;
    CK(P.make(2 * nch + 1));
    begin_call(o.st, __func__);
    CK(cudaMemsetAsync(W.flag, 0, sizeof(int), o.st));
    CK(cudaMemsetAsync(W.kerr, 0, sizeof(int), o.st));
    CK(cudaMemcpyAsync(H.Ylm, lm.data(), lm.size(), cudaMemcpyHostToDevice, o.st));
    CK(cudaMemcpyAsync(H.idx, landmark_idx, sizeof(int64_t) * l, cudaMemcpyHostToDevice, o.st));
    CK(launch_iota(H.iota, l, o.st));

    // rows stream in on their own stream while the landmark problem runs: each
    // chunk is copied and turned into the projection kernel's operands
    for (int c = 0; c < nch; ++c) {
        const int64_t row0 = (int64_t)c * chunk, rows = std::min(chunk, n - row0);
        char* Yc = Yd + (size_t)row0 * d * es;
        CK(cudaMemcpyAsync(Yc, Yh + (size_t)row0 * d * es, (size_t)rows * d * es, cudaMemcpyHostToDevice, P.h2d));
        if (kind != kKindRows)
            CK(launch_encode_u8(kind - 1, (const uint8_t*)Yc, rows, d,
                                static_cast<char*>(W.Yq) + tck_operand_bytes(kind - 1, row0, d), W.nrm_f + row0,
                                P.h2d));
        else if (o.prec == MDS_PREC_BF16)
            CK(launch_quant_bf16_rows(Yc, dt, rows, d, W.Yq, row0, n, W.nrm, P.h2d));
        else
            CK(launch_rownorm(Yc, dt, rows, d, f64, W.nrm + row0, P.h2d));
        CK(cudaEventRecord(P.ev[2 * c], P.h2d));
    }

    // classical MDS of the landmarks (first subset of Section 3.1) from the
    // unrounded landmark rows, then the Gower operator and its operands
    CK(launch_rownorm(H.Ylm, dt, l, d, f64, H.nrm_lm, o.st));
    tmark(0, o.st);
    if ((s = run_eig_batch(W.B, H.Ylm, dt, d, H.nrm_lm, nullptr, H.iota, f64, 1, o))) return s;
    CK(launch_interp_model(W.B.v, W.B.lam, W.B.q, W.B.desc[0].ldq, 0, l, r,
                           f64 ? (double*)W.W : nullptr, f64 ? nullptr : (float*)W.W,
                           f64 ? (double*)W.X1 : nullptr, f64 ? nullptr : (float*)W.X1, W.bias,
                           H.var, o.st));
    if (kind != kKindRows) {
        CK(launch_encode_landmarks_u8(kind - 1, (const uint8_t*)H.Ylm, l, d, H.iota, l, W.L, W.nrm_lf, o.st));
        CK(launch_pad_w_rows((const float*)W.W, l, r, W.Wpad, o.st));
    } else if (o.prec == MDS_PREC_BF16) {
        CK(cudaMemsetAsync(W.nrm_lf, 0, sizeof(float) * model_nlf_count(kind, l), o.st));
        CK(launch_quant_bf16(H.Ylm, dt, l, d, H.Yq_lm, H.nrm_lms, o.st));
        CK(launch_gather_split(H.Yq_lm, l, d, H.iota, l, W.L, H.nrm_lms, W.nrm_lf, o.st));
        CK(launch_w_image((const float*)W.W, l, r, W.Wpad, o.st));
    } else {
        CK(launch_gather_rows(H.Ylm, dt, l, d, H.iota, l, f64, W.L, H.nrm_lm, W.nrm_l, o.st));
    }

    // each chunk is projected once it has arrived, its landmark rows set to
    // X_1, and its X copied out on a third stream
    for (int c = 0; c < nch; ++c) {
        const int64_t row0 = (int64_t)c * chunk, rows = std::min(chunk, n - row0);
        char* Xc = Xd + (size_t)row0 * r * ex;
        CK(cudaStreamWaitEvent(o.st, P.ev[2 * c], 0));
        if (kind != kKindRows)
            CK(launch_gower_tck(kind - 1, static_cast<char*>(W.Yq) + tck_operand_bytes(kind - 1, row0, d), rows, d,
                                W.nrm_f + row0, W.L, l, W.nrm_lf, W.Wpad, W.bias, r, (float*)Xc, W.kerr, o.st));
        else if (o.prec == MDS_PREC_BF16)
            CK(launch_gower_tc(static_cast<uint16_t*>(W.Yq) + (size_t)row0 * split_ld(d), rows, n, d, W.nrm + row0,
                               W.L, W.nrm_lf, l, W.Wpad, W.bias, r, (float*)Xc, W.kerr, o.st));
        else
            CK(launch_gower_proj(Yd + (size_t)row0 * d * es, dt, rows, d, W.nrm + row0, W.L, W.nrm_l, l, W.W,
                                 W.bias, r, f64, Xc, o.st));
        CK(launch_scatter_rows_range(W.X1, H.idx, l, r, row0, rows, f64, Xc, o.st));
        CK(cudaEventRecord(P.ev[2 * c + 1], o.st));
        CK(cudaStreamWaitEvent(P.d2h, P.ev[2 * c + 1], 0));
        CK(cudaMemcpyAsync(Xh + (size_t)row0 * r * ex, Xc, (size_t)rows * r * ex, cudaMemcpyDeviceToHost, P.d2h));
    }
    CK(cudaMemcpyAsync(var, H.var, sizeof(double) * r, cudaMemcpyDeviceToHost, P.d2h));
    CK(cudaEventRecord(P.ev[2 * nch], P.d2h));
    CK(cudaStreamWaitEvent(o.st, P.ev[2 * nch], 0));
    s = finish(&W.B, W.flag, o, W.kerr);
    if (s != MDS_OK || !out_model) return s;
    return make_model(W, kind, o, l, d, r, out_model);
}

size_t mds_embed_new_workspace_size(mds_model m, int64_t rows) {
    if (!m || rows <= 0) return 0;
    Arena A{nullptr, 0};
    A.take<int>(1);
    A.take<double>(rows);
    if (m->kind != kKindRows) A.take<char>(tck_operand_bytes(m->kind - 1, rows, m->d));
    else if (m->prec == MDS_PREC_BF16) A.take<uint16_t>((size_t)2 * rows * split_ld(m->d));
    return A.off + 256;
}

int mds_embed_new(mds_model m, const void* Ynew, int dt, int64_t rows, const mds_opts* opts,
                  void* X) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (!m || !Ynew || !X || !valid_dt(dt) || rows <= 0) return MDS_ERR_ARG;
    if (o.prec != m->prec) return MDS_ERR_ARG;
    if ((s = check_ws(o, mds_embed_new_workspace_size(m, rows) - 256))) return s;
    begin_call(o.st, __func__);
    int* kerr = nullptr;
    if ((s = gbmds::embed_enqueue(m, Ynew, dt, rows, o.ws, o.st, X, &kerr))) return s;
    return finish(nullptr, nullptr, o, kerr);
}

int mds_model_info(mds_model m, int* l, int* d, int* r, int* prec, double* lambda) {
    if (!m) return MDS_ERR_ARG;
    if (l) *l = m->l;
    if (d) *d = m->d;
    if (r) *r = m->r;
    if (prec) *prec = m->prec;
    if (lambda && cudaMemcpy(lambda, m->lam, sizeof(double) * m->r, cudaMemcpyDeviceToHost) != cudaSuccess)
        return MDS_ERR_CUDA;
    return MDS_OK;
}

void mds_model_free(mds_model m) {
    if (!m) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m->device);
    cudaFree(m->L);
    cudaFree(m->nrm_l);
    cudaFree(m->nrm_lf);
    cudaFree(m->W);
    cudaFree(m->bias);
    cudaFree(m->X1);
    cudaFree(m->lam);
    cudaSetDevice(cur);
    delete m;
}

static const char kMagic[8] = {'G', 'B', 'M', 'D', 'S', 'M', '0', '5'};

int mds_model_save(mds_model m, const char* path) {
    if (!m || !path) return MDS_ERR_ARG;
    const size_t es = m->prec == MDS_PREC_F64 ? 8 : 4;
    const size_t szL = model_L_bytes(m->kind, m->prec, m->l, m->d), szW = model_W_bytes(m->kind, m->prec, m->l, m->r);
    const size_t szX = (size_t)m->l * m->r * es, nlf = model_nlf_count(m->kind, m->l);
    std::vector<char> L(szL), W(szW), X1(szX);
    std::vector<double> nrm(m->l), bias(m->r), lam(m->r);
    std::vector<float> nrmf(nlf);
    if (cudaMemcpy(L.data(), m->L, szL, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(nrmf.data(), m->nrm_lf, 4 * nlf, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(W.data(), m->W, szW, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(X1.data(), m->X1, szX, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(nrm.data(), m->nrm_l, 8 * m->l, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(bias.data(), m->bias, 8 * m->r, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(lam.data(), m->lam, 8 * m->r, cudaMemcpyDeviceToHost) != cudaSuccess)
        return MDS_ERR_CUDA;
    FILE* f = fopen(path, "wb");
    if (!f) return MDS_ERR_IO;
    const int32_t hdr[5] = {m->l, m->d, m->r, m->prec, m->kind};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, 4, 5, f) == 5 &&
              fwrite(L.data(), 1, szL, f) == szL && fwrite(nrm.data(), 8, m->l, f) == (size_t)m->l &&
              fwrite(W.data(), 1, szW, f) == szW && fwrite(bias.data(), 8, m->r, f) == (size_t)m->r &&
              fwrite(X1.data(), 1, szX, f) == szX && fwrite(lam.data(), 8, m->r, f) == (size_t)m->r &&
              fwrite(nrmf.data(), 4, nlf, f) == nlf;
    ok = (fclose(f) == 0) && ok;
    return ok ? MDS_OK : MDS_ERR_IO;
}

int mds_model_load(const char* path, mds_model* out) {
    if (!path || !out) return MDS_ERR_ARG;
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return MDS_ERR_IO;
    char magic[8];
    int32_t hdr[5];
    if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kMagic, 8) != 0 || fread(hdr, 4, 5, f) != 5 ||
        hdr[0] < 2 || hdr[0] > kMaxEigN || hdr[1] <= 0 || hdr[2] <= 0 || hdr[2] > kMaxR ||
        hdr[3] < MDS_PREC_F64 || hdr[3] > MDS_PREC_FP8 || hdr[4] < kKindRows || hdr[4] > kKindU8Fp8 ||
        model_kind(hdr[3], hdr[4] == kKindRows ? MDS_IN_F32 : MDS_IN_U8, hdr[1], hdr[2]) != hdr[4]) {
        fclose(f);
        return MDS_ERR_IO;
    }
    mds_model m = new (std::nothrow) mds_model_s();
    if (!m) {
        fclose(f);
        return MDS_ERR_NOMEM;
    }
    m->l = hdr[0];
    m->d = hdr[1];
    m->r = hdr[2];
    m->prec = hdr[3];
    m->kind = hdr[4];
    cudaGetDevice(&m->device);
    const size_t es = m->prec == MDS_PREC_F64 ? 8 : 4;
    const size_t szL = model_L_bytes(m->kind, m->prec, m->l, m->d), szW = model_W_bytes(m->kind, m->prec, m->l, m->r);
    const size_t szX = (size_t)m->l * m->r * es, nlf = model_nlf_count(m->kind, m->l);
    std::vector<char> L(szL), W(szW), X1(szX);
    std::vector<double> nrm(m->l), bias(m->r), lam(m->r);
    std::vector<float> nrmf(nlf);
    bool ok = fread(L.data(), 1, szL, f) == szL && fread(nrm.data(), 8, m->l, f) == (size_t)m->l &&
              fread(W.data(), 1, szW, f) == szW && fread(bias.data(), 8, m->r, f) == (size_t)m->r &&
              fread(X1.data(), 1, szX, f) == szX && fread(lam.data(), 8, m->r, f) == (size_t)m->r &&
              fread(nrmf.data(), 4, nlf, f) == nlf;
    fclose(f);
    if (!ok) {
        delete m;
        return MDS_ERR_IO;
    }
    ok = dev_malloc(&m->L, szL) == cudaSuccess && dev_malloc((void**)&m->nrm_l, 8 * m->l) == cudaSuccess &&
         dev_malloc((void**)&m->nrm_lf, 4 * nlf) == cudaSuccess &&
         dev_malloc(&m->W, szW) == cudaSuccess && dev_malloc((void**)&m->bias, 8 * m->r) == cudaSuccess &&
         dev_malloc(&m->X1, szX) == cudaSuccess && dev_malloc((void**)&m->lam, 8 * m->r) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mds_model_free(m);
        return MDS_ERR_NOMEM;
    }
    ok = cudaMemcpy(m->L, L.data(), szL, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->nrm_l, nrm.data(), 8 * m->l, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->nrm_lf, nrmf.data(), 4 * nlf, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->W, W.data(), szW, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->bias, bias.data(), 8 * m->r, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->X1, X1.data(), szX, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->lam, lam.data(), 8 * m->r, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        mds_model_free(m);
        return MDS_ERR_CUDA;
    }
    *out = m;
    return MDS_OK;
}

// -------------------------------------------------------- divide-and-conquer

size_t mds_divide_conquer_workspace_size(int64_t n, int d, int p, const int64_t* part_ptr, int c,
                                         int r, int prec) {
    if (n <= 0 || d <= 0 || p <= 0 || !part_ptr || c <= 0 || r <= 0) return 0;
    for (int j = 0; j < p; ++j)
        if (part_ptr[j + 1] < part_ptr[j] || part_ptr[j + 1] - part_ptr[j] + c > kMaxEigN) return 0;
    DcWs W;
    return dc_layout(W, nullptr, n, d, p, part_ptr, c, r, prec, kDefaultSteps) + 256;
}

int mds_divide_conquer(const void* Y, int dt, int64_t n, int d, int p, const int64_t* part_ptr,
                       const int64_t* part_own, const int64_t* anchors, int c, int r,
                       const mds_opts* opts, void* X, double* var) {
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (!Y || !X || !var || !part_ptr || !anchors || !valid_dt(dt) || n < 2 || d <= 0 || p <= 0 ||
        r <= 0 || r > kMaxR || c < r + 1 || c > n || part_ptr[0] != 0)
        return MDS_ERR_ARG;
    for (int j = 0; j < p; ++j) {
        const int64_t own = part_ptr[j + 1] - part_ptr[j];
        if (own < 0 || own + c > kMaxEigN || own + c <= r) return MDS_ERR_ARG;
    }
    if (part_ptr[p] > 0 && !part_own) return MDS_ERR_ARG;
    if ((o.prec == MDS_PREC_FP8 || o.prec == MDS_PREC_BF16) && dt != MDS_IN_U8) return MDS_ERR_UNSUPPORTED;
    DcWs W;
    const size_t need = dc_layout(W, nullptr, n, d, p, part_ptr, c, r, o.prec, o.mmax);
    if ((s = check_ws(o, need))) return s;
    if (dc_layout(W, o.ws, n, d, p, part_ptr, c, r, o.prec, o.mmax) != need) return MDS_ERR_WORKSPACE;
    begin_call(o.st, __func__);
    if ((s = dc_enqueue(W, Y, dt, n, d, p, part_ptr, part_own, anchors, c, r, o, X, var, true))) return s;
    return finish(&W.B, W.flag, o, W.G.mode >= 0 ? W.G.kerr : nullptr);
}


// ------------------------------------------------------------ fast MDS

}  // extern "C"

namespace {

// The division tree of fast MDS as the host sees it, validated, with the
// batch of classical problems (leaves first, then each inner node's
// alignment set) and the Procrustes tasks grouped by tree level.
struct FastPlan {
    int nnodes = 0, nleaves = 0, s = 0, r = 0, max_leaf = 0;
    std::vector<std::vector<int>> kids;
    std::vector<int> leaf_prob, align_prob, depth, leftmost_leaf;
    std::vector<int> sizes;               // problem sizes
    std::vector<int64_t> own_off;         // problem offsets into own_all
    std::vector<longlong2> copies;        // alignment-row copies (dst in own_all, src in perm)
    std::vector<std::vector<FastTask>> level_tasks;   // deepest level first
    std::vector<std::vector<int>> level_dst;          // child node of each task
    std::vector<int> chain;
    std::vector<int2> leaf_chain;
    int64_t own_total = 0;
    int max_tasks = 0;
};

int fast_plan(FastPlan& F, int64_t n, int nnodes, const int64_t* range, const int32_t* parent, int s, int r) {
    if (nnodes < 1 || !range || !parent || s < r + 1 || r < 1 || r > kMaxR) return MDS_ERR_ARG;
    if (parent[0] != -1 || range[0] != 0 || range[1] != n) return MDS_ERR_ARG;
    F = FastPlan();
    F.nnodes = nnodes;
    F.s = s;
    F.r = r;
    F.kids.assign(nnodes, {});
    for (int k = 1; k < nnodes; ++k) {
        const int q = parent[k];
        if (q < 0 || q >= nnodes || q == k || range[2 * k] < range[2 * q] || range[2 * k + 1] > range[2 * q + 1] ||
            range[2 * k] >= range[2 * k + 1])
            return MDS_ERR_ARG;
        F.kids[q].push_back(k);
    }
    // children in order, tiling their parent's range; every node reached once from the root
    F.depth.assign(nnodes, -1);
    std::vector<int> order{0};
    F.depth[0] = 0;
    for (size_t h = 0; h < order.size(); ++h) {
        const int k = order[h];
        auto& ch = F.kids[k];
        std::sort(ch.begin(), ch.end(), [&](int a, int b) { return range[2 * a] < range[2 * b]; });
        if (ch.size() == 1) return MDS_ERR_ARG;
        int64_t at = range[2 * k];
        for (int c : ch) {
            if (range[2 * c] != at || F.depth[c] != -1) return MDS_ERR_ARG;
            at = range[2 * c + 1];
            F.depth[c] = F.depth[k] + 1;
            order.push_back(c);
        }
        if (!ch.empty() && at != range[2 * k + 1]) return MDS_ERR_ARG;
    }
    if ((int)order.size() != nnodes) return MDS_ERR_ARG;
    // problems: leaves, then alignment sets
    F.leaf_prob.assign(nnodes, -1);
    F.align_prob.assign(nnodes, -1);
    for (int k = 0; k < nnodes; ++k)
        if (F.kids[k].empty()) {
            const int64_t m = range[2 * k + 1] - range[2 * k];
            if (m > kMaxEigN || m <= r) return MDS_ERR_ARG;
            F.leaf_prob[k] = F.nleaves++;
            F.sizes.push_back((int)m);
            F.own_off.push_back(range[2 * k]);
            F.max_leaf = std::max(F.max_leaf, (int)m);
        }
    int64_t at = n;
    for (int k = 0; k < nnodes; ++k) {
        if (F.kids[k].empty()) continue;
        const int64_t m = (int64_t)F.kids[k].size() * s;
        if (m > kMaxEigN || m <= r) return MDS_ERR_ARG;
        F.align_prob[k] = (int)F.sizes.size();
        F.sizes.push_back((int)m);
        F.own_off.push_back(at);
        for (size_t j = 0; j < F.kids[k].size(); ++j) {
            const int c = F.kids[k][j];
            if (range[2 * c + 1] - range[2 * c] < s) return MDS_ERR_ARG;
            F.copies.push_back(make_longlong2(at + (int64_t)j * s, range[2 * c]));
        }
        at += m;
    }
    F.own_total = at;
    // leftmost leaf of every node (children come after their parent in `order`)
    F.leftmost_leaf.assign(nnodes, -1);
    for (int h = nnodes - 1; h >= 0; --h) {
        const int k = order[h];
        F.leftmost_leaf[k] = F.kids[k].empty() ? k : F.leftmost_leaf[F.kids[k][0]];
    }
    // nodes on the path from node a up to, not including, node top
    auto path = [&](int a, int top) {
        std::vector<int> p;
        for (int x = a; x != top; x = parent[x]) p.push_back(x);
        return p;
    };
    int maxd = 0;
    for (int k = 0; k < nnodes; ++k) maxd = std::max(maxd, F.depth[k]);
    for (int lev = maxd - 1; lev >= 0; --lev) {
        std::vector<FastTask> tasks;
        std::vector<int> dst;
        for (int k = 0; k < nnodes; ++k) {
            if (F.depth[k] != lev || F.kids[k].empty()) continue;
            for (size_t j = 0; j < F.kids[k].size(); ++j) {
                const int c = F.kids[k][j];
                const std::vector<int> p = path(F.leftmost_leaf[c], c);
                FastTask t{F.align_prob[k], (int)(j * s), F.leaf_prob[F.leftmost_leaf[c]], (int)F.chain.size(),
                           (int)p.size()};
                F.chain.insert(F.chain.end(), p.begin(), p.end());
                tasks.push_back(t);
                dst.push_back(c);
            }
        }
        F.max_tasks = std::max(F.max_tasks, (int)tasks.size());
        F.level_tasks.push_back(tasks);
        F.level_dst.push_back(dst);
    }
    for (int k = 0; k < nnodes; ++k) {
        if (!F.kids[k].empty()) continue;
        const std::vector<int> p = path(k, 0);
        F.leaf_chain.push_back(make_int2((int)F.chain.size(), (int)p.size()));
        F.chain.insert(F.chain.end(), p.begin(), p.end());
    }
    return MDS_OK;
}

struct FastWs {
    int* flag;
    double* nrm;
    int64_t* own_all;
    Batch B;
    longlong2* copies;
    FastTask* tasks;      // all levels, concatenated
    int* dst;
    int* chain;
    int2* leaf_chain;
    double* maps;         // nnodes x (r r + r)
    double* lmaps;        // nleaves x (r r + r)
    double* AB;           // max_tasks x 2 s r
};

size_t fast_layout(FastWs& W, const FastPlan& F, char* base, int64_t n, int mmax) {
    Arena A{base, 0};
    W.flag = A.take<int>(1);
    W.nrm = A.take<double>(n);
    W.own_all = A.take<int64_t>(F.own_total);
    plan_batch(W.B, F.sizes, F.own_off, 0, F.r, mmax, n);
    carve_batch(W.B, A);
    size_t ntasks = 0;
    for (const auto& t : F.level_tasks) ntasks += t.size();
    W.copies = A.take<longlong2>(std::max<size_t>(1, F.copies.size()));
    W.tasks = A.take<FastTask>(std::max<size_t>(1, ntasks));
    W.dst = A.take<int>(std::max<size_t>(1, ntasks));
    W.chain = A.take<int>(std::max<size_t>(1, F.chain.size()));
    W.leaf_chain = A.take<int2>(std::max(1, F.nleaves));
    const size_t rr = (size_t)F.r * F.r + F.r;
    W.maps = A.take<double>((size_t)F.nnodes * rr);
    W.lmaps = A.take<double>((size_t)std::max(1, F.nleaves) * rr);
    W.AB = A.take<double>((size_t)std::max(1, F.max_tasks) * 2 * F.s * F.r);
    return A.off;
}

}  // namespace

extern "C" {

size_t mds_fast_workspace_size(int64_t n, int d, int nnodes, const int64_t* node_range, const int32_t* node_parent,
                               int s, int r, int prec) {
    (void)prec;
    if (n <= 0 || d <= 0) return 0;
    FastPlan F;
    if (fast_plan(F, n, nnodes, node_range, node_parent, s, r) != MDS_OK) return 0;
    FastWs W;
    return fast_layout(W, F, nullptr, n, kDefaultSteps) + 256;
}

int mds_fast(const void* Y, int dt, int64_t n, int d, const int64_t* perm, int nnodes, const int64_t* node_range,
             const int32_t* node_parent, int s, int r, const mds_opts* opts, void* X, double* var) {
    Opts o;
    int st = read_opts(opts, &o);
    if (st) return st;
    if (!Y || !X || !var || !perm || !valid_dt(dt) || n < 2 || d <= 0) return MDS_ERR_ARG;
    if (o.prec != MDS_PREC_F64 && o.prec != MDS_PREC_F32) return MDS_ERR_UNSUPPORTED;
    FastPlan F;
    if ((st = fast_plan(F, n, nnodes, node_range, node_parent, s, r))) return st;
    FastWs W;
    const size_t need = fast_layout(W, F, nullptr, n, o.mmax);
    if ((st = check_ws(o, need))) return st;
    if (fast_layout(W, F, o.ws, n, o.mmax) != need) return MDS_ERR_WORKSPACE;
    begin_call(o.st, __func__);
    const int f64 = o.prec == MDS_PREC_F64;
    std::vector<FastTask> all_tasks;
    std::vector<int> all_dst;
    for (size_t v = 0; v < F.level_tasks.size(); ++v) {
        all_tasks.insert(all_tasks.end(), F.level_tasks[v].begin(), F.level_tasks[v].end());
        all_dst.insert(all_dst.end(), F.level_dst[v].begin(), F.level_dst[v].end());
    }
    CK(cudaMemsetAsync(W.flag, 0, sizeof(int), o.st));
    CK(launch_check_idx(perm, n, n, W.flag, o.st));
    // the rows of every problem: perm for the leaves, the gathered sampling
    // points for the alignment sets; the tables of tasks and chains
    CK(cudaMemcpyAsync(W.own_all, perm, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, o.st));
    if (!F.copies.empty()) {
        CK(cudaMemcpyAsync(W.copies, F.copies.data(), sizeof(longlong2) * F.copies.size(), cudaMemcpyHostToDevice, o.st));
        CK(launch_fast_gather(perm, W.copies, (int)F.copies.size(), s, W.own_all, o.st));
    }
    if (!all_tasks.empty()) {
        CK(cudaMemcpyAsync(W.tasks, all_tasks.data(), sizeof(FastTask) * all_tasks.size(), cudaMemcpyHostToDevice,
                           o.st));
        CK(cudaMemcpyAsync(W.dst, all_dst.data(), sizeof(int) * all_dst.size(), cudaMemcpyHostToDevice, o.st));
    }
    if (!F.chain.empty())
        CK(cudaMemcpyAsync(W.chain, F.chain.data(), sizeof(int) * F.chain.size(), cudaMemcpyHostToDevice, o.st));
    CK(cudaMemcpyAsync(W.leaf_chain, F.leaf_chain.data(), sizeof(int2) * F.leaf_chain.size(), cudaMemcpyHostToDevice,
                       o.st));
    const void* Ye = Y;
    int dte = dt;
    if ((st = prep_data(Y, dt, n, d, o.prec, W.nrm, nullptr, o, &Ye, &dte))) return st;
    tmark(0, o.st);
    // every classical problem of the recursion in one batched eigen-solver launch
    if ((st = run_eig_batch(W.B, Ye, dte, d, W.nrm, nullptr, W.own_all, f64, f64, o))) return st;
    // maps of the subsets onto their parents' alignment configurations, deepest level first
    size_t off = 0;
    for (size_t v = 0; v < F.level_tasks.size(); ++v) {
        const int nt = (int)F.level_tasks[v].size();
        CK(launch_fast_prep(W.B.d_desc, W.B.v, W.B.lam, r, s, W.tasks + off, nt, W.chain, W.maps, W.AB, o.st));
        CK(launch_procrustes_sets(W.AB, nt, s, r, W.dst + off, W.maps, o.st));
        off += nt;
    }
    // each leaf's rows through the composition of its maps; lambda-bar over the leaves
    CK(launch_fast_finish(W.B.d_desc, F.nleaves, F.max_leaf, W.B.v, W.B.lam, W.leaf_chain, W.chain, W.maps, r,
                          W.lmaps, W.own_all, f64, X, o.st));
    CK(launch_dc_lambda_bar(W.B.d_desc, F.nleaves, W.B.lam, r, var, o.st));
    return finish(&W.B, W.flag, o);
}

// ------------------------------------------------- divide-and-conquer plans

}  // extern "C"

struct mds_dc_plan_s {
    int device = 0;
    int64_t n = 0;
    int d = 0, dt = 0, p = 0, c = 0, r = 0;
    std::vector<int64_t> ptr;
    Opts o{};
    void* ws = nullptr;
    DcWs W;
    bool tune = false, tuned = false;
    int cs = 0;
    double trial_ms[17] = {};   // autotuner: call time per cluster size (0 = not tried)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
    int64_t launches = 0;
    const void* cY = nullptr;   // buffers the graph was captured with
    const int64_t* cown = nullptr;
    const int64_t* canc = nullptr;
    void* cX = nullptr;
    double* cvar = nullptr;
    cudaStream_t pst = nullptr; // the plan's own stream (stream capture needs one)
    cudaEvent_t join = nullptr; // orders it after the caller's stream
    int* hbuf = nullptr;        // page-locked: status[p], steps[p], flag
    cudaEvent_t ev[6] = {};
    // device buffers of mds_dc_plan_execute_host (allocated at its first call)
    void* dY = nullptr;
    int64_t* down = nullptr;
    int64_t* danc = nullptr;
    void* dX = nullptr;
    double* dvar = nullptr;
};

namespace {

void plan_drop_graph(mds_dc_plan P) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    P->exec = nullptr;
    P->graph = nullptr;
}

// One direct (uncaptured) run with cluster size cs, timed on the stream.
int plan_trial(mds_dc_plan P, int cs, const void* Y, const int64_t* own, const int64_t* anc, void* X,
               double* var, cudaStream_t st, double* ms) {
    Opts o = P->o;
    o.st = st;
    o.cluster = cs;
    begin_call(st, __func__);
    CK(cudaEventRecord(P->ev[0], st));
    int s = dc_enqueue(P->W, Y, P->dt, P->n, P->d, P->p, P->ptr.data(), own, anc, P->c, P->r, o, X, var, false);
    if (s) return s;
    CK(cudaEventRecord(P->ev[5], st));
    const int p = P->p;
    CK(cudaMemcpyAsync(P->hbuf, P->W.B.status, sizeof(int) * p, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(P->hbuf + p, P->W.B.steps, sizeof(int) * p, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(P->hbuf + 2 * p, P->W.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    P->hbuf[2 * p + 1] = 0;
    if (P->W.G.mode >= 0)
        CK(cudaMemcpyAsync(P->hbuf + 2 * p + 1, P->W.G.kerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    float f = 0.f;
    cudaEventElapsedTime(&f, P->ev[0], P->ev[5]);
    *ms = f;
    return batch_status(P->W.B, P->hbuf, P->hbuf + p, P->hbuf[2 * p], P->hbuf[2 * p + 1]);
}

}  // namespace

extern "C" {

int mds_dc_plan_create(int64_t n, int d, int dt, int p, const int64_t* part_ptr, int c, int r,
                       const mds_opts* opts, int tune, mds_dc_plan* out) {
    if (!out) return MDS_ERR_ARG;
    *out = nullptr;
    Opts o;
    int s = read_opts(opts, &o);
    if (s) return s;
    if (opts->workspace || opts->workspace_bytes) return MDS_ERR_ARG;   // the plan owns its workspace
    if (!part_ptr || !valid_dt(dt) || n < 2 || d <= 0 || p <= 0 || r <= 0 || r > kMaxR || c < r + 1 || c > n ||
        part_ptr[0] != 0)
        return MDS_ERR_ARG;
    for (int j = 0; j < p; ++j) {
        const int64_t own = part_ptr[j + 1] - part_ptr[j];
        if (own < 0 || own + c > kMaxEigN || own + c <= r) return MDS_ERR_ARG;
    }
    if ((o.prec == MDS_PREC_FP8 || o.prec == MDS_PREC_BF16) && dt != MDS_IN_U8) return MDS_ERR_UNSUPPORTED;
    mds_dc_plan P = new (std::nothrow) mds_dc_plan_s();
    if (!P) return MDS_ERR_NOMEM;
    P->n = n;
    P->d = d;
    P->dt = dt;
    P->p = p;
    P->c = c;
    P->r = r;
    P->ptr.assign(part_ptr, part_ptr + p + 1);
    P->tune = tune != 0 && o.cluster == 0;
    P->cs = o.cluster;
    cudaGetDevice(&P->device);
    const size_t need = dc_layout(P->W, nullptr, n, d, p, part_ptr, c, r, o.prec, o.mmax);
    bool ok = dev_malloc(&P->ws, need) == cudaSuccess &&
              cudaHostAlloc((void**)&P->hbuf, sizeof(int) * (2 * p + 2), cudaHostAllocDefault) == cudaSuccess;
    for (auto& e : P->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&P->join, cudaEventDisableTiming) == cudaSuccess &&
         cudaStreamCreateWithFlags(&P->pst, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mds_dc_plan_destroy(P);
        return MDS_ERR_NOMEM;
    }
    dc_layout(P->W, (char*)P->ws, n, d, p, part_ptr, c, r, o.prec, o.mmax);
    o.ws = (char*)P->ws;
    o.wsb = need;
    P->o = o;
    // part descriptors and queue order stay on the device for the plan's life
    const GramOp& G = P->W.G;
    if (cudaMemcpy(P->W.B.d_desc, P->W.B.desc.data(), sizeof(ProbDesc) * p, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->W.B.d_order, P->W.B.order.data(), sizeof(int) * p, cudaMemcpyHostToDevice) != cudaSuccess ||
        (G.mode >= 0 &&
         (cudaMemcpy(G.moff, G.h_moff.data(), sizeof(int) * p, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(G.units, G.h_units.data(), sizeof(int4) * G.h_units.size(), cudaMemcpyHostToDevice) !=
              cudaSuccess))) {
        cudaGetLastError();
        mds_dc_plan_destroy(P);
        return MDS_ERR_CUDA;
    }
    *out = P;
    return MDS_OK;
}

int mds_dc_plan_execute(mds_dc_plan P, const void* Y, const int64_t* part_own, const int64_t* anchors, void* X,
                        double* var, void* stream) {
    if (!P || !Y || !X || !var || !anchors || (P->ptr[P->p] > 0 && !part_own)) return MDS_ERR_ARG;
    // work runs on the plan's stream, after what the caller queued on theirs
    const cudaStream_t ust = stream ? (cudaStream_t)stream : P->o.st;
    const cudaStream_t st = P->pst;
    CK(cudaEventRecord(P->join, ust));
    CK(cudaStreamWaitEvent(st, P->join, 0));
    const Batch& B = P->W.B;
    const std::string tkey =
        batch_tune_key(B, P->o.prec != MDS_PREC_F64, (P->o.flags & MDS_FLAG_FULL_MATVEC) == 0);
    if (P->cs == 0 && P->tune && tune_enabled()) {
        // a cluster size measured before for this batch shape on this kind of GPU
        int v = 0;
        double tms[17] = {};
        if (tune_lookup(tkey, &v, tms, 17) && v >= 1 && v <= 16 &&
            lanczos_smem_bytes(B.max_n, v, B.mmax, B.r) <= kMaxSmem) {
            P->cs = v;
            P->tuned = true;
            for (int i = 0; i < 17; ++i) P->trial_ms[i] = tms[i];
        }
    }
    if (P->cs == 0 && P->tune) {
        // autotuner: every cluster size that fits, timed on these buffers
        // (each trial is a complete, correct run); the fastest one is kept
        double best = 0.0;
        for (int cs = 1; cs <= 16; ++cs) {
            if (lanczos_smem_bytes(B.max_n, cs, B.mmax, B.r) > kMaxSmem || cs > std::max(1, B.max_n / 64)) continue;
            double ms = 0.0;
            int s = plan_trial(P, cs, Y, part_own, anchors, X, var, st, &ms);
            if (s == MDS_OK && P->trial_ms[0] == 0.0) {   // the first run also warms the device up
                P->trial_ms[0] = ms;
                s = plan_trial(P, cs, Y, part_own, anchors, X, var, st, &ms);
            }
            if (s != MDS_OK) {
                if (s == MDS_ERR_ARG || s == MDS_ERR_RANK) return s;   // the data, not the cluster size
                continue;
            }
            P->trial_ms[cs] = ms;
            if (P->cs == 0 || ms < best) {
                best = ms;
                P->cs = cs;
            }
        }
        P->tuned = true;
        P->trial_ms[0] = 0.0;
        if (P->cs == 0) return MDS_ERR_CUDA;
        tune_store(tkey, P->cs, P->trial_ms, 17);
    }
    if (P->cs == 0) {
        double sum_n2 = 0.0;
        for (const ProbDesc& D : B.desc) sum_n2 += (double)D.n * D.n;
        P->cs = pick_cluster(0, B.p, B.max_n, B.mmax, B.r, sum_n2, P->o.prec == MDS_PREC_F64 ? 8 : 4);
    }
    if (!P->exec || Y != P->cY || part_own != P->cown || anchors != P->canc || X != P->cX || var != P->cvar) {
        plan_drop_graph(P);
        Opts o = P->o;
        o.st = st;
        o.cluster = P->cs;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MDS_ERR_CUDA;
        g_capture_ev = P->ev;
        begin_call(st, __func__);
        int s = dc_enqueue(P->W, Y, P->dt, P->n, P->d, P->p, P->ptr.data(), part_own, anchors, P->c, P->r, o, X,
                           var, false);
        const int p = P->p;
        if (s == MDS_OK &&
            (cudaMemcpyAsync(P->hbuf, B.status, sizeof(int) * p, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaMemcpyAsync(P->hbuf + p, B.steps, sizeof(int) * p, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaMemcpyAsync(P->hbuf + 2 * p, P->W.flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             (P->W.G.mode >= 0 && cudaMemcpyAsync(P->hbuf + 2 * p + 1, P->W.G.kerr, sizeof(int),
                                                  cudaMemcpyDeviceToHost, st) != cudaSuccess)))
            s = MDS_ERR_CUDA;
        g_capture_ev = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(st, &P->graph);
        if (s == MDS_OK && ce != cudaSuccess) s = MDS_ERR_CUDA;
        if (s == MDS_OK && cudaGraphInstantiate(&P->exec, P->graph, 0) != cudaSuccess) s = MDS_ERR_CUDA;
        if (s != MDS_OK) {
            cudaGetLastError();
            plan_drop_graph(P);
            return s;
        }
        cudaGraphGetNodes(P->graph, nullptr, &P->nodes);
        P->launches = g_launches;
        P->cY = Y;
        P->cown = part_own;
        P->canc = anchors;
        P->cX = X;
        P->cvar = var;
    }
    g_last = mds_stats{};
    nvtx_end_call();
    g_nvtx_call = nvtxRangeStartA("mds_dc_plan_execute (graph)");
    CK(cudaGraphLaunch(P->exec, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    nvtx_end_call();
    g_launches = P->launches;
    g_cluster = P->cs;
    if (g_timing)
        for (int i = 0; i < 5; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, P->ev[i], P->ev[i + 1]);
            g_last.stage_ms[i] = ms;
        }
    return batch_status(B, P->hbuf, P->hbuf + P->p, P->hbuf[2 * P->p], P->W.G.mode >= 0 ? P->hbuf[2 * P->p + 1] : 0);
}

int mds_dc_plan_execute_host(mds_dc_plan P, const void* Y, const int64_t* part_own, const int64_t* anchors, void* X,
                             double* var, void* stream) {
    if (!P || !Y || !X || !var || !anchors || (P->ptr[P->p] > 0 && !part_own)) return MDS_ERR_ARG;
    const size_t es = P->dt == MDS_IN_F64 ? 8 : (P->dt == MDS_IN_F32 ? 4 : 1);
    const size_t ex = P->o.prec == MDS_PREC_F64 ? 8 : 4;
    const size_t yb = (size_t)P->n * P->d * es, xb = (size_t)P->n * P->r * ex;
    const size_t ob = sizeof(int64_t) * (size_t)P->ptr[P->p], ab = sizeof(int64_t) * P->c;
    if (!P->dY) {
        // the plan's own device copies of the inputs and outputs; X starts at
        // zero (rows outside every part are never written)
        bool ok = dev_malloc(&P->dY, yb) == cudaSuccess && dev_malloc((void**)&P->down, ob + 8) == cudaSuccess &&
                  dev_malloc((void**)&P->danc, ab) == cudaSuccess && dev_malloc(&P->dX, xb) == cudaSuccess &&
                  dev_malloc((void**)&P->dvar, sizeof(double) * P->r) == cudaSuccess &&
                  cudaMemset(P->dX, 0, xb) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            cudaFree(P->dY);
            cudaFree(P->down);
            cudaFree(P->danc);
            cudaFree(P->dX);
            cudaFree(P->dvar);
            P->dY = P->dX = nullptr;
            P->down = P->danc = nullptr;
            P->dvar = nullptr;
            return MDS_ERR_NOMEM;
        }
    }
    const cudaStream_t ust = stream ? (cudaStream_t)stream : P->o.st;
    const cudaStream_t st = P->pst;
    CK(cudaEventRecord(P->join, ust));
    CK(cudaStreamWaitEvent(st, P->join, 0));
    CK(cudaMemcpyAsync(P->dY, Y, yb, cudaMemcpyHostToDevice, st));
    if (ob) CK(cudaMemcpyAsync(P->down, part_own, ob, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(P->danc, anchors, ab, cudaMemcpyHostToDevice, st));
    int s = mds_dc_plan_execute(P, P->dY, P->down, P->danc, P->dX, P->dvar, st);
    if (s != MDS_OK) return s;
    CK(cudaMemcpyAsync(X, P->dX, xb, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(var, P->dvar, sizeof(double) * P->r, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return MDS_OK;
}

int mds_dc_plan_info(mds_dc_plan P, int* cluster, int64_t* graph_nodes, double* trial_ms) {
    if (!P) return MDS_ERR_ARG;
    if (cluster) *cluster = P->cs;
    if (graph_nodes) *graph_nodes = (int64_t)P->nodes;
    if (trial_ms)
        for (int i = 0; i <= 16; ++i) trial_ms[i] = P->trial_ms[i];
    return MDS_OK;
}

void mds_dc_plan_destroy(mds_dc_plan P) {
    if (!P) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(P->device);
    if (P->pst) cudaStreamSynchronize(P->pst);
    plan_drop_graph(P);
    if (P->pst) cudaStreamDestroy(P->pst);
    if (P->join) cudaEventDestroy(P->join);
    if (P->ws) cudaFree(P->ws);
    if (P->hbuf) cudaFreeHost(P->hbuf);
    if (P->dY) cudaFree(P->dY);
    if (P->down) cudaFree(P->down);
    if (P->danc) cudaFree(P->danc);
    if (P->dX) cudaFree(P->dX);
    if (P->dvar) cudaFree(P->dvar);
    for (auto& e : P->ev)
        if (e) cudaEventDestroy(e);
    cudaGetLastError();
    cudaSetDevice(cur);
    delete P;
}

}  // extern "C"
