// Serving loop: continuous batching of embed requests onto resident models.
//
// Gower's formula (Section 3.1, Eq. (2)) embeds each new point from its own
// squared distances to the landmarks, so rows of different requests for the
// same model can share one kernel launch without changing any row's result.
// The server keeps `slots` CUDA streams, each with a fixed device arena.  A
// host scheduler thread fills every free slot with a batch: rows of waiting
// requests for the model (and input dtype) of the oldest waiting request, in
// arrival order, as many as the arena holds; larger requests are split across
// batches.  A batch is copied in, embedded by one projection launch and
// copied out on its slot's stream; a host callback on that stream marks the
// slot complete, so batches on different slots overlap on the device and
// requests that arrive meanwhile wait only for the next free slot.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxSlots = 16;
constexpr size_t kDefaultSlotBytes = 64u << 20;

struct Request {
    int model = 0, dt = 0;
    const char* Y = nullptr;   // host rows
    char* X = nullptr;         // host results
    int64_t m = 0;
    int64_t dispatched = 0;    // rows handed to batches
    int64_t finished = 0;      // rows whose batch has completed
    int status = MDS_OK;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

struct Chunk {
    std::shared_ptr<Request> req;
    int64_t row0, rows, off;   // request rows [row0, row0 + rows) at batch row `off`
};

struct Slot;

}  // namespace

struct mds_server_s {
    int device = 0;
    std::vector<mds_model> models;
    std::vector<std::unique_ptr<Slot>> slots;
    size_t slot_bytes = 0;
    int64_t max_rows = 0;
    std::mutex mu;
    std::condition_variable wake;   // scheduler: new request, slot complete, shutdown
    std::condition_variable done;   // waiters: a request completed
    std::deque<std::shared_ptr<Request>> pending;   // not yet fully dispatched, arrival order
    std::unordered_map<uint64_t, std::shared_ptr<Request>> live;
    uint64_t next_ticket = 1;
    bool stop = false;
    int busy = 0;
    mds_server_stats stats{};
    std::thread thread;
};

namespace {

struct Slot {
    mds_server_s* srv = nullptr;
    cudaStream_t st = nullptr;
    char* arena = nullptr;
    int* kerr_host = nullptr;   // page-locked copy of the batch's device status word
    std::vector<Chunk> chunks;
    bool busy = false;
    bool complete = false;
    int launch_status = MDS_OK;
    Clock::time_point t_complete;
};

size_t dt_size(int dt) { return dt == MDS_IN_F64 ? 8 : dt == MDS_IN_F32 ? 4 : 1; }
size_t x_row_bytes(const mds_model_s* m) { return (size_t)m->r * (m->prec == MDS_PREC_F64 ? 8 : 4); }
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Arena layout of a batch of R rows: [embed scratch | staged input | results].
struct BatchLayout {
    size_t ws, y, x, total;
};
BatchLayout layout(const mds_model_s* m, int dt, int64_t R) {
    BatchLayout L;
    L.ws = align256(mds_embed_new_workspace_size(const_cast<mds_model>(m), R));
    L.y = L.ws;
    L.x = L.y + align256((size_t)R * m->d * dt_size(dt));
    L.total = L.x + align256((size_t)R * x_row_bytes(m));
    return L;
}

// Largest R whose layout fits the slot arena (0 if not even one row does).
int64_t rows_that_fit(const mds_model_s* m, int dt, size_t bytes, int64_t cap) {
    int64_t lo = 0, hi = cap > 0 ? cap : (int64_t)(bytes / std::max<size_t>(1, m->d * dt_size(dt))) + 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (layout(m, dt, mid).total <= bytes) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

void CUDART_CB on_slot_done(void* p) {
    Slot* s = static_cast<Slot*>(p);
    {
        std::lock_guard<std::mutex> g(s->srv->mu);
        s->complete = true;
        s->t_complete = Clock::now();
    }
    s->srv->wake.notify_all();
}

// Under the lock: credit a completed batch to its requests.
void retire(mds_server_s* S, Slot& sl) {
    const int ks = sl.launch_status != MDS_OK ? sl.launch_status : *sl.kerr_host;
    for (auto& c : sl.chunks) {
        Request& q = *c.req;
        q.finished += c.rows;
        if (ks != MDS_OK && q.status == MDS_OK) q.status = ks;
        S->stats.rows += c.rows;
        if (q.finished == q.m) {
            q.done = true;
            q.t_done = sl.t_complete;
            S->stats.requests += 1;
        }
    }
    sl.chunks.clear();
    sl.busy = false;
    sl.complete = false;
    S->busy -= 1;
    S->done.notify_all();
}

// Under the lock: pick the next batch for a free slot; false if nothing waits.
bool form_batch(mds_server_s* S, Slot& sl) {
    while (!S->pending.empty()) {
        const Request& head = *S->pending.front();
        const mds_model_s* m = S->models[head.model];
        const int64_t cap = rows_that_fit(m, head.dt, S->slot_bytes, S->max_rows);
        if (cap < 1) {   // the model's rows cannot fit a slot at all
            auto q = S->pending.front();
            S->pending.pop_front();
            q->status = MDS_ERR_WORKSPACE;
            q->done = true;
            q->t_done = Clock::now();
            S->stats.requests += 1;
            S->done.notify_all();
            continue;
        }
        const int model = head.model, dt = head.dt;
        int64_t total = 0;
        for (auto& q : S->pending) {
            if (total == cap) break;
            if (q->model != model || q->dt != dt) continue;
            const int64_t take = std::min(q->m - q->dispatched, cap - total);
            sl.chunks.push_back({q, q->dispatched, take, total});
            q->dispatched += take;
            total += take;
        }
        S->pending.erase(std::remove_if(S->pending.begin(), S->pending.end(),
                                        [](const std::shared_ptr<Request>& q) { return q->dispatched == q->m; }),
                         S->pending.end());
        return true;
    }
    return false;
}

// Without the lock: queue copies in, one projection launch, copies out and the
// completion callback on the slot's stream.  Returns false when the callback
// could not be queued (the slot is then complete at once).
bool launch_batch(mds_server_s* S, Slot& sl) {
    const Request& first = *sl.chunks.front().req;
    mds_model_s* m = S->models[first.model];
    const int dt = first.dt;
    int64_t R = 0;
    for (auto& c : sl.chunks) R = std::max(R, c.off + c.rows);
    const BatchLayout L = layout(m, dt, R);
    const size_t yrow = (size_t)m->d * dt_size(dt), xrow = x_row_bytes(m);
    int st = MDS_OK;
    for (auto& c : sl.chunks)
        if (st == MDS_OK && cudaMemcpyAsync(sl.arena + L.y + c.off * yrow, c.req->Y + c.row0 * yrow, c.rows * yrow,
                                            cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
            st = MDS_ERR_CUDA;
    int* kerr = nullptr;
    if (st == MDS_OK) st = gbmds::embed_enqueue(m, sl.arena + L.y, dt, R, sl.arena, sl.st, sl.arena + L.x, &kerr);
    for (auto& c : sl.chunks)
        if (st == MDS_OK && cudaMemcpyAsync(c.req->X + c.row0 * xrow, sl.arena + L.x + c.off * xrow, c.rows * xrow,
                                            cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
            st = MDS_ERR_CUDA;
    if (st == MDS_OK &&
        cudaMemcpyAsync(sl.kerr_host, kerr, sizeof(int), cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
        st = MDS_ERR_CUDA;
    if (st != MDS_OK) cudaGetLastError();
    sl.launch_status = st;
    if (cudaLaunchHostFunc(sl.st, on_slot_done, &sl) != cudaSuccess) {
        cudaGetLastError();
        if (sl.launch_status == MDS_OK) sl.launch_status = MDS_ERR_CUDA;
        return false;
    }
    return true;
}

void scheduler(mds_server_s* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        for (auto& sl : S->slots)
            if (sl->busy && sl->complete) retire(S, *sl);
        bool progressed = false;
        for (auto& slp : S->slots) {
            Slot& sl = *slp;
            if (sl.busy) continue;
            if (!form_batch(S, sl)) break;
            sl.busy = true;
            sl.complete = false;
            S->busy += 1;
            S->stats.batches += 1;
            S->stats.max_in_flight = std::max(S->stats.max_in_flight, S->busy);
            lk.unlock();
            const bool queued = launch_batch(S, sl);
            lk.lock();
            if (!queued) {
                sl.complete = true;
                sl.t_complete = Clock::now();
            }
            progressed = true;
        }
        if (S->stop && S->pending.empty() && S->busy == 0) break;
        if (progressed) continue;
        bool ready = false;
        for (auto& sl : S->slots) ready |= sl->busy && sl->complete;
        if (!ready) S->wake.wait(lk);
    }
}

void free_slots(mds_server_s* S) {
    for (auto& sl : S->slots) {
        if (sl->st) {
            cudaStreamSynchronize(sl->st);
            cudaStreamDestroy(sl->st);
        }
        if (sl->arena) cudaFree(sl->arena);
        if (sl->kerr_host) cudaFreeHost(sl->kerr_host);
    }
    S->slots.clear();
    cudaGetLastError();
}

}  // namespace

extern "C" {

int mds_server_create(const mds_model* models, int nmodels, const mds_server_opts* opts, mds_server* out) {
    if (!models || nmodels <= 0 || !opts || !out || opts->flags != 0 || opts->slots < 0 ||
        opts->slots > kMaxSlots || opts->max_batch_rows < 0)
        return MDS_ERR_ARG;
    for (int i = 0; i < nmodels; ++i)
        if (!models[i]) return MDS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MDS_ERR_CUDA;
    for (int i = 0; i < nmodels; ++i)
        if (models[i]->device != dev) return MDS_ERR_ARG;
    auto S = std::make_unique<mds_server_s>();
    S->device = dev;
    S->models.assign(models, models + nmodels);
    S->slot_bytes = opts->slot_bytes ? opts->slot_bytes : kDefaultSlotBytes;
    S->max_rows = opts->max_batch_rows;
    S->stats.slots = opts->slots ? opts->slots : 4;
    for (int i = 0; i < S->stats.slots; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->srv = S.get();
        const bool ok = cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking) == cudaSuccess &&
                        gbmds::dev_malloc(&sl->arena, S->slot_bytes) == cudaSuccess &&
                        cudaHostAlloc(&sl->kerr_host, sizeof(int), cudaHostAllocDefault) == cudaSuccess;
        S->slots.push_back(std::move(sl));
        if (!ok) {
            free_slots(S.get());
            return MDS_ERR_NOMEM;
        }
        *S->slots.back()->kerr_host = 0;
    }
    S->thread = std::thread(scheduler, S.get());
    *out = S.release();
    return MDS_OK;
}

int mds_server_submit(mds_server S, int model, const void* Y, int dt, int64_t m, void* X, uint64_t* ticket) {
    if (!S || !Y || !X || !ticket || m <= 0 || model < 0 || model >= (int)S->models.size() ||
        (dt != MDS_IN_F64 && dt != MDS_IN_F32 && dt != MDS_IN_U8))
        return MDS_ERR_ARG;
    auto q = std::make_shared<Request>();
    q->model = model;
    q->dt = dt;
    q->Y = static_cast<const char*>(Y);
    q->X = static_cast<char*>(X);
    q->m = m;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) return MDS_ERR_ARG;
        q->t_submit = Clock::now();
        *ticket = S->next_ticket++;
        S->live.emplace(*ticket, q);
        S->pending.push_back(q);
    }
    S->wake.notify_all();
    return MDS_OK;
}

int mds_server_wait(mds_server S, uint64_t ticket, double timeout_s, int* status, double* latency_ms) {
    if (!S || !status || timeout_s < 0) return MDS_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->live.find(ticket);
    if (it == S->live.end()) return MDS_ERR_ARG;
    auto q = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::min(timeout_s, 1e6)));
    if (!S->done.wait_until(lk, deadline, [&] { return q->done; })) return MDS_ERR_TIMEOUT;
    *status = q->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    S->live.erase(ticket);
    return MDS_OK;
}

int mds_server_get_stats(mds_server S, mds_server_stats* out) {
    if (!S || !out) return MDS_ERR_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    *out = S->stats;
    return MDS_OK;
}

int mds_server_destroy(mds_server S) {
    if (!S) return MDS_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->wake.notify_all();
    if (S->thread.joinable()) S->thread.join();
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(S->device);
    free_slots(S);
    cudaSetDevice(dev);
    delete S;
    return MDS_OK;
}

}  // extern "C"
