// Autotuner of the strided HBM passes: the schedule of the generic
// multi-pass plans (rows too long for one tile: a first pass over row
// segments, then strided passes over the high bits), the GPU counterpart of
// the forest cut of Sec. V.B (how much of each transform one work unit owns).
//
// ptdr_autotune times candidate schedules -- first-pass tile bytes, masks per
// first-pass tile, strided-pass tile bytes (hence bits per pass), threads per
// CTA -- with CUDA events on the caller's buffers and keeps the fastest.  The
// choice is cached in memory and, when PTDR_TUNE_CACHE names a file, in that
// file as JSON, one entry per key
//     "<GPU name>|<op>|n=<n>|<input type>|<output type>|<precision>"
// loaded lazily the first time a plan is looked up.  Every later call with a
// matching key runs the cached schedule; other keys keep the default.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "plan.h"

namespace ptdr {

namespace {

struct Entry {
    TuneParams p;
    double ms;
};

std::mutex g_mu;
bool g_loaded = false;
std::string g_loaded_from;
std::map<std::string, Entry> g_cache;
std::string g_dev_name[128];

const char* dtype_name(ptdr_dtype t)
{
    switch (t) {
    case PTDR_C64: return "c64";
    case PTDR_C128: return "c128";
    case PTDR_F32: return "f32";
    case PTDR_F64: return "f64";
    }
    return "?";
}

const char* prec_name(ptdr_precision p)
{
    switch (p) {
    case PTDR_PREC_FP64: return "fp64";
    case PTDR_PREC_FP32: return "fp32";
    case PTDR_PREC_SPLIT_BF16_TC: return "bf16x3";
    case PTDR_PREC_FIXED_I128: return "fixed";
    }
    return "?";
}

std::string make_key(const char* gpu, bool compose, int n, ptdr_dtype in_t, ptdr_dtype out_t, ptdr_precision prec)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|%s|n=%d|%s|%s|%s", gpu, compose ? "compose" : "decompose", n, dtype_name(in_t),
                  dtype_name(out_t), prec_name(prec));
    return buf;
}

std::string cache_path()
{
    const char* p = std::getenv("PTDR_TUNE_CACHE");
    return p ? p : "";
}

// Reads entries of the form  "key": {"tile_log2": a, "masks_log2": b,
// "pass_tile_log2": c, "threads": d, "ms": e}  (one per line; the file this
// module writes).  Lines that do not parse are skipped.
void load_locked()
{
    const std::string path = cache_path();
    if (g_loaded && path == g_loaded_from) return;
    g_loaded = true;
    g_loaded_from = path;
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
        const char* q0 = std::strchr(line, '"');
        if (!q0) continue;
        const char* q1 = std::strstr(q0 + 1, "\": {");
        if (!q1) continue;
        Entry e{};
        if (std::sscanf(q1, "\": {\"tile_log2\": %d, \"masks_log2\": %d, \"pass_tile_log2\": %d, \"threads\": %d, \"ms\": %lf",
                        &e.p.tile_log2, &e.p.masks_log2, &e.p.pass_tile_log2, &e.p.threads, &e.ms) != 5)
            continue;
        g_cache[std::string(q0 + 1, q1)] = e;
    }
    std::fclose(f);
}

// Rewrites the whole cache file (written to a temporary name, then renamed).
bool save_locked()
{
    const std::string path = cache_path();
    if (path.empty()) return true;
    const std::string tmp = path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (const auto& kv : g_cache) {
        const Entry& e = kv.second;
        std::fprintf(f, "  \"%s\": {\"tile_log2\": %d, \"masks_log2\": %d, \"pass_tile_log2\": %d, \"threads\": %d, \"ms\": %.6f}%s\n",
                     kv.first.c_str(), e.p.tile_log2, e.p.masks_log2, e.p.pass_tile_log2, e.p.threads, e.ms,
                     ++i < g_cache.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    const bool ok = std::fclose(f) == 0;
    return ok && std::rename(tmp.c_str(), path.c_str()) == 0;
}

bool device_name(int dev, std::string* out)
{
    if (dev < 0 || dev >= 128) return false;
    if (g_dev_name[dev].empty()) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        g_dev_name[dev] = prop.name;
    }
    *out = g_dev_name[dev];
    return true;
}

} // namespace

bool tuned_params_for(int dev, const DensePlan& p, TuneParams* out)
{
    if (!multipass_tunable(p)) return false;
    std::lock_guard<std::mutex> lk(g_mu);
    std::string name;
    if (!device_name(dev, &name)) return false;
    load_locked();
    const auto it = g_cache.find(make_key(name.c_str(), p.compose, p.n, p.in_t, p.out_t, p.prec));
    if (it == g_cache.end()) return false;
    *out = it->second.p;
    return true;
}

} // namespace ptdr

using namespace ptdr;

extern "C" {

ptdr_status ptdr_tune_lookup(const char* gpu_name, ptdr_op op, int n, ptdr_dtype in_type, ptdr_dtype out_type,
                             ptdr_precision prec, ptdr_tune_params* out)
{
    if (!gpu_name || !out || (op != PTDR_OP_DECOMPOSE && op != PTDR_OP_COMPOSE)) return PTDR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    const auto it = g_cache.find(make_key(gpu_name, op == PTDR_OP_COMPOSE, n, in_type, out_type, prec));
    if (it == g_cache.end()) return PTDR_ERR_UNSUPPORTED;
    out->tile_log2 = it->second.p.tile_log2;
    out->masks_log2 = it->second.p.masks_log2;
    out->pass_tile_log2 = it->second.p.pass_tile_log2;
    out->threads = it->second.p.threads;
    out->ms = it->second.ms;
    return PTDR_OK;
}

ptdr_status ptdr_tune_store(const char* gpu_name, ptdr_op op, int n, ptdr_dtype in_type, ptdr_dtype out_type,
                            ptdr_precision prec, const ptdr_tune_params* params)
{
    if (!gpu_name || !params || (op != PTDR_OP_DECOMPOSE && op != PTDR_OP_COMPOSE) || n < 1 || n > kMaxDenseN)
        return PTDR_ERR_INVALID_ARG;
    if (std::strchr(gpu_name, '"') || std::strchr(gpu_name, '\n')) return PTDR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    Entry e{{params->tile_log2, params->masks_log2, params->pass_tile_log2, params->threads}, params->ms};
    g_cache[make_key(gpu_name, op == PTDR_OP_COMPOSE, n, in_type, out_type, prec)] = e;
    return save_locked() ? PTDR_OK : PTDR_ERR_INVALID_ARG;
}

} // extern "C"
