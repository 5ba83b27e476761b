// mds_embed_new_static: Gower projection of new rows against a stored model
// without any device allocation by anyone.
//
// Who needs it: callers that cannot call cudaMalloc (or ask another allocator
// such as PyTorch's for device memory) at the moment they embed new points.
// Examples are a serving process whose device memory is fully reserved up
// front by a different allocator, so a fresh allocation would fail with
// out-of-memory, and a host program that embeds this library inside a plugin
// or real-time loop that forbids allocation after start-up, because an
// allocation can block on device-wide synchronisation and stall the loop.
//
// How: the scratch that mds_embed_new needs (the rows' squared norms, and the
// BF16-rounded copy of the rows for BF16 models) lives in one file-scope
// __device__ array of kStaticScratchBytes bytes.  Every GPU that loads
// libgbmds.so holds that array until the process exits.  Host code cannot
// use the array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current)
// and caches it; later calls on that device reuse it.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;   // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_embed_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_embed_scratch on the current device (looked up once).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MDS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_embed_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MDS_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MDS_OK;
}

}  // namespace

extern "C" {

size_t mds_embed_new_static_capacity(void) { return kStaticScratchBytes; }

int mds_embed_new_static(mds_model model, const void* Ynew, int dt, int64_t m,
                         const mds_opts* opts, void* X) {
    if (!opts || !model || !Ynew || !X || m <= 0) return MDS_ERR_ARG;
    if (opts->workspace || opts->workspace_bytes) return MDS_ERR_ARG;   // scratch is built in
    const size_t need = mds_embed_new_workspace_size(model, m);
    if (need == 0) return MDS_ERR_ARG;
    if (need > kStaticScratchBytes) return MDS_ERR_WORKSPACE;           // too many rows for the array
    void* scratch = nullptr;
    const int s = scratch_address(&scratch);
    if (s != MDS_OK) return s;
    mds_opts o = *opts;
    o.workspace = scratch;
    o.workspace_bytes = kStaticScratchBytes;
    return mds_embed_new(model, Ynew, dt, m, &o, X);
}

}  // extern "C"
