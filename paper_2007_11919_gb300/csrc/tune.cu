// Persistent tuning cache: the launch choices an autotuner measured, kept in a
// JSON file so that a later process (or plan) with the same problem shape on
// the same kind of GPU reuses them instead of timing every candidate again.
//
// The file is named by mds_set_tune_cache() or, at first use, by the
// environment variable GBMDS_TUNE_CACHE; without either the cache is off.  It
// holds one entry per line:
//
//   {"gbmds_tune_cache": 1, "entries": [
//   {"key": "k_lanczos p=418 ...", "value": 5, "trial_ms": [0, 191.2, ...]},
//   ...
//   ]}
//
// A key names the kernel and every quantity its choice depends on (problem
// sizes, precision, SM count and compute capability).  Updates read the file,
// replace or add the entry and write the result to a temporary file that is
// renamed over the old one, so a reader never sees a half-written file; two
// processes updating at once can lose one of the two updates (the cache then
// only misses, it is never wrong).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <unistd.h>

#include "common.cuh"

namespace gbmds {
namespace {

std::mutex g_tune_mu;
std::string g_tune_path;
bool g_tune_init = false;

struct TuneEntry {
    std::string key;
    int value = 0;
    std::vector<double> trial;
};

void tune_init_locked() {
    if (g_tune_init) return;
    g_tune_init = true;
    const char* env = std::getenv("GBMDS_TUNE_CACHE");
    if (env && *env) g_tune_path = env;
}

bool key_ok(const char* key) {
    if (!key || !*key || std::strlen(key) > 1024) return false;
    for (const char* c = key; *c; ++c)
        if (*c == '"' || *c == '\\' || *c == '\n' || *c == '\r') return false;
    return true;
}

// Parses the entries this file writes (one per line); other lines are skipped.
std::vector<TuneEntry> read_entries(const std::string& path) {
    std::vector<TuneEntry> out;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return out;
    std::string line;
    char buf[4096];
    while (std::fgets(buf, sizeof buf, f)) {
        line = buf;
        const size_t k = line.find("\"key\": \"");
        if (k == std::string::npos) continue;
        const size_t k0 = k + 8, k1 = line.find('"', k0);
        if (k1 == std::string::npos) continue;
        const size_t v = line.find("\"value\": ", k1);
        if (v == std::string::npos) continue;
        TuneEntry e;
        e.key = line.substr(k0, k1 - k0);
        char* end = nullptr;
        e.value = (int)std::strtol(line.c_str() + v + 9, &end, 10);
        if (end == line.c_str() + v + 9) continue;
        const size_t t = line.find("\"trial_ms\": [", v);
        if (t != std::string::npos) {
            const char* p = line.c_str() + t + 13;
            while (*p && *p != ']') {
                char* q = nullptr;
                const double x = std::strtod(p, &q);
                if (q == p) break;
                e.trial.push_back(x);
                p = q;
                while (*p == ',' || *p == ' ') ++p;
            }
        }
        out.push_back(std::move(e));
    }
    std::fclose(f);
    return out;
}

bool write_entries(const std::string& path, const std::vector<TuneEntry>& es) {
    const std::string tmp = path + ".tmp." + std::to_string((long long)getpid());
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\"gbmds_tune_cache\": 1, \"entries\": [\n");
    for (size_t i = 0; i < es.size(); ++i) {
        std::fprintf(f, "{\"key\": \"%s\", \"value\": %d, \"trial_ms\": [", es[i].key.c_str(), es[i].value);
        for (size_t j = 0; j < es[i].trial.size(); ++j) std::fprintf(f, "%s%.6g", j ? ", " : "", es[i].trial[j]);
        std::fprintf(f, "]}%s\n", i + 1 < es.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    const bool ok = std::fclose(f) == 0;
    if (!ok || std::rename(tmp.c_str(), path.c_str()) != 0) {
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

}  // namespace

bool tune_enabled() {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_init_locked();
    return !g_tune_path.empty();
}

bool tune_lookup(const std::string& key, int* value, double* trial_ms, int ntrial) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_init_locked();
    if (g_tune_path.empty() || !key_ok(key.c_str())) return false;
    for (const TuneEntry& e : read_entries(g_tune_path)) {
        if (e.key != key) continue;
        *value = e.value;
        if (trial_ms)
            for (int j = 0; j < ntrial; ++j) trial_ms[j] = j < (int)e.trial.size() ? e.trial[j] : 0.0;
        return true;
    }
    return false;
}

bool tune_store(const std::string& key, int value, const double* trial_ms, int ntrial) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_init_locked();
    if (g_tune_path.empty() || !key_ok(key.c_str())) return false;
    std::vector<TuneEntry> es = read_entries(g_tune_path);
    TuneEntry* hit = nullptr;
    for (TuneEntry& e : es)
        if (e.key == key) hit = &e;
    if (!hit) {
        es.emplace_back();
        hit = &es.back();
        hit->key = key;
    }
    hit->value = value;
    hit->trial.assign(trial_ms ? trial_ms : nullptr, trial_ms ? trial_ms + ntrial : nullptr);
    return write_entries(g_tune_path, es);
}

// The eigen-solver's key: the batch's shape (problem count, largest problem,
// sum of squared sizes, step cap, r, Q precision, symmetric ranges allowed)
// and the device (SM count, compute capability).
std::string lanczos_tune_key(int p, int max_n, double sum_n2, int mmax, int r, int q_f32, int sym) {
    int dev = 0, sms = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    char buf[256];
    std::snprintf(buf, sizeof buf, "k_lanczos cluster p=%d max_n=%d sum_n2=%.0f mmax=%d r=%d q=%s sym=%d sms=%d sm=%d%d",
                  p, max_n, sum_n2, mmax, r, q_f32 ? "f32" : "f64", sym, sms, major, minor);
    return buf;
}

}  // namespace gbmds

extern "C" {

int mds_set_tune_cache(const char* path) {
    std::lock_guard<std::mutex> g(gbmds::g_tune_mu);
    gbmds::g_tune_init = true;
    gbmds::g_tune_path = path ? path : "";
    return MDS_OK;
}

int mds_tune_cache_lookup(const char* key, int* value) {
    if (!key || !value || !gbmds::key_ok(key)) return MDS_ERR_ARG;
    if (!gbmds::tune_lookup(key, value, nullptr, 0)) *value = 0;
    return MDS_OK;
}

int mds_tune_cache_store(const char* key, int value) {
    if (!key || !gbmds::key_ok(key)) return MDS_ERR_ARG;
    return gbmds::tune_store(key, value, nullptr, 0) ? MDS_OK : MDS_ERR_ARG;
}

}  // extern "C"
