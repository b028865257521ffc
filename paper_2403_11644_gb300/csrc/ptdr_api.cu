// C ABI of libptdr: argument validation, launch planning and dispatch.
// Every compute entry point validates its arguments before touching the
// device, returns PTDR_ERR_NO_DEVICE when no CUDA device is usable (there is
// no CPU fallback) and enqueues its kernels on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "plan.h"
#include "ptdr_internal.h"

namespace ptdr {

// The device status word (one per device, see common.cuh).
__device__ unsigned int g_status_word;

static std::mutex g_mu;
static unsigned int* g_status_ptr[128];

ptdr_status device_ready(int* dev)
{
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
        cudaGetLastError();
        return PTDR_ERR_NO_DEVICE;
    }
    if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= 128) {
        cudaGetLastError();
        return PTDR_ERR_NO_DEVICE;
    }
    return PTDR_OK;
}

ptdr_status status_word(int dev, unsigned int** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) {
            cudaGetLastError();
            return PTDR_ERR_CUDA;
        }
        g_status_ptr[dev] = (unsigned int*)p;
    }
    *out = g_status_ptr[dev];
    return PTDR_OK;
}

// Rejects pointers the device cannot address as ordinary device memory.
ptdr_status check_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return PTDR_ERR_INVALID_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return PTDR_ERR_INVALID_ARG;
    return PTDR_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb)
{
    const char* pa = (const char*)a;
    const char* pb = (const char*)b;
    return pa < pb + nb && pb < pa + na;
}

bool fault_injected(const char* what)
{
    const char* f = std::getenv("PTDR_FAULT");
    return f && std::strcmp(f, what) == 0;
}

unsigned long long wait_limit_ns()
{
    const char* v = std::getenv("PTDR_WAIT_NS");
    if (!v || !*v) return 1000000000ull;
    char* end = nullptr;
    const unsigned long long ns = std::strtoull(v, &end, 10);
    if (end == v || ns == 0) return 1000000000ull;
    return std::min<unsigned long long>(ns, 60000000000ull);
}

} // namespace ptdr

using namespace ptdr;

namespace {

bool valid_dtype(int t) { return t >= PTDR_C64 && t <= PTDR_F64; }
bool valid_prec(int p) { return p >= PTDR_PREC_FP64 && p <= PTDR_PREC_FIXED_I128; }

ptdr_status validate_dense(const void* in, ptdr_dtype in_t, const void* out, ptdr_dtype out_t,
                           int n, ptdr_precision prec, bool compose)
{
    if (!in || !out) return PTDR_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxDenseN) return PTDR_ERR_INVALID_ARG;
    if (!valid_dtype(in_t) || !valid_dtype(out_t) || !valid_prec(prec)) return PTDR_ERR_INVALID_ARG;
    // decompose: real or complex A; a real C stores Re c (all of c for Hermitian A, Thm 2).
    // compose: real coefficients describe a Hermitian A, which is complex.
    if (compose && !dtype_complex(out_t)) return PTDR_ERR_UNSUPPORTED;
    if (prec == PTDR_PREC_SPLIT_BF16_TC) {
        if (compose) return PTDR_ERR_UNSUPPORTED;
        if (in_t != PTDR_C64 || (out_t != PTDR_C64 && out_t != PTDR_F32)) return PTDR_ERR_UNSUPPORTED;
    }
    const size_t elems = (size_t)1 << (2 * n);
    if ((uintptr_t)in % dtype_bytes(in_t) || (uintptr_t)out % dtype_bytes(out_t))
        return PTDR_ERR_INVALID_ARG;
    if (overlaps(in, elems * dtype_bytes(in_t), out, elems * dtype_bytes(out_t)))
        return PTDR_ERR_INVALID_ARG;
    return PTDR_OK;
}

ptdr_status run_dense(bool compose, const void* in, ptdr_dtype in_t, void* out, ptdr_dtype out_t,
                      int n, double scale, ptdr_precision prec, void* ws, size_t ws_bytes,
                      void* stream)
{
    ptdr_status v = validate_dense(in, in_t, out, out_t, n, prec, compose);
    if (v != PTDR_OK) return v;
    DensePlan plan;
    v = make_dense_plan(compose, n, in_t, out_t, prec, &plan);
    if (v != PTDR_OK) return v;
    if (plan.ws_bytes > 0 && (!ws || ws_bytes < plan.ws_bytes)) return PTDR_ERR_WORKSPACE;
    if (fault_injected("plan")) return PTDR_ERR_INTERNAL;
    int dev = 0;
    v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(in) != PTDR_OK || check_device_ptr(out) != PTDR_OK)
        return PTDR_ERR_INVALID_ARG;
    if (plan.ws_bytes > 0 && check_device_ptr(ws) != PTDR_OK) return PTDR_ERR_INVALID_ARG;
    unsigned int* st = nullptr;
    v = status_word(dev, &st);
    if (v != PTDR_OK) return v;
    if (fault_injected("launch")) return PTDR_ERR_CUDA;
    TuneParams tp;
    if (tuned_params_for(dev, plan, &tp)) apply_multipass_tuning(&plan, tp); // schedule from the autotuner's cache
    return execute_dense(plan, in, out, ws, scale, st, (cudaStream_t)stream);
}

} // namespace

extern "C" {

ptdr_status ptdr_decompose(const void* A, ptdr_dtype a_type, void* C, ptdr_dtype c_type, int n,
                           ptdr_precision prec, void* workspace, size_t workspace_bytes,
                           void* stream)
{
    PTDR_TRACE();
    return run_dense(false, A, a_type, C, c_type, n, std::ldexp(1.0, -n), prec, workspace,
                     workspace_bytes, stream);
}

ptdr_status ptdr_compose(const void* C, ptdr_dtype c_type, void* A, ptdr_dtype a_type, int n,
                         double scale, ptdr_precision prec, void* workspace,
                         size_t workspace_bytes, void* stream)
{
    PTDR_TRACE();
    if (!std::isfinite(scale)) return PTDR_ERR_INVALID_ARG;
    return run_dense(true, C, c_type, A, a_type, n, scale, prec, workspace, workspace_bytes,
                     stream);
}

ptdr_status ptdr_autotune(ptdr_op op, int n, ptdr_dtype in_type, ptdr_dtype out_type, ptdr_precision prec,
                          const void* in, void* out, void* workspace, size_t workspace_bytes, void* stream,
                          ptdr_tune_params* best)
{
    PTDR_TRACE();
    if (!best || (op != PTDR_OP_DECOMPOSE && op != PTDR_OP_COMPOSE)) return PTDR_ERR_INVALID_ARG;
    const bool compose = op == PTDR_OP_COMPOSE;
    ptdr_status v = validate_dense(in, in_type, out, out_type, n, prec, compose);
    if (v != PTDR_OK) return v;
    DensePlan plan;
    v = make_dense_plan(compose, n, in_type, out_type, prec, &plan);
    if (v != PTDR_OK) return v;
    if (plan.ws_bytes > 0 && (!workspace || workspace_bytes < plan.ws_bytes)) return PTDR_ERR_WORKSPACE;
    if (!multipass_tunable(plan)) return PTDR_ERR_UNSUPPORTED; // no strided passes to schedule
    int dev = 0;
    v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(in) != PTDR_OK || check_device_ptr(out) != PTDR_OK ||
        (plan.ws_bytes > 0 && check_device_ptr(workspace) != PTDR_OK))
        return PTDR_ERR_INVALID_ARG;
    unsigned int* st = nullptr;
    v = status_word(dev, &st);
    if (v != PTDR_OK) return v;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return PTDR_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const double scale = compose ? 1.0 : std::ldexp(1.0, -n);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PTDR_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PTDR_ERR_CUDA;
    }
    ptdr_status result = PTDR_ERR_UNSUPPORTED;
    double best_ms = 1e300;
    TuneParams best_p{};
    for (int tl = 15; tl <= 17; ++tl)
        for (int ml = 0; ml <= (compose ? 0 : 3); ++ml)
            for (int pl = 15; pl <= 17; ++pl)
                for (int th = 256; th <= 512; th *= 2) {
                    DensePlan q = plan;
                    const TuneParams t{tl, ml, pl, th};
                    if (!apply_multipass_tuning(&q, t)) continue;
                    // one warm-up launch, then the mean of two timed ones
                    if (execute_dense(q, in, out, workspace, scale, st, s) != PTDR_OK) continue;
                    cudaEventRecord(e0, s);
                    bool ok = true;
                    for (int r = 0; r < 2 && ok; ++r) ok = execute_dense(q, in, out, workspace, scale, st, s) == PTDR_OK;
                    cudaEventRecord(e1, s);
                    float ms = 0.f;
                    if (!ok || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        cudaGetLastError();
                        continue;
                    }
                    if (ms / 2 < best_ms) {
                        best_ms = ms / 2;
                        best_p = t;
                        result = PTDR_OK;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != PTDR_OK) return PTDR_ERR_CUDA;
    best->tile_log2 = best_p.tile_log2;
    best->masks_log2 = best_p.masks_log2;
    best->pass_tile_log2 = best_p.pass_tile_log2;
    best->threads = best_p.threads;
    best->ms = best_ms;
    return ptdr_tune_store(prop.name, op, n, in_type, out_type, prec, best);
}

ptdr_status ptdr_workspace_size(ptdr_op op, int n, ptdr_dtype a_type, ptdr_dtype c_type,
                                ptdr_precision prec, size_t* bytes)
{
    if (!bytes) return PTDR_ERR_INVALID_ARG;
    if (op != PTDR_OP_DECOMPOSE && op != PTDR_OP_COMPOSE) return PTDR_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxDenseN) return PTDR_ERR_INVALID_ARG;
    if (!valid_dtype(a_type) || !valid_dtype(c_type) || !valid_prec(prec)) return PTDR_ERR_INVALID_ARG;
    const bool compose = op == PTDR_OP_COMPOSE;
    // decompose reads A (a_type) and writes C (c_type); compose the reverse
    DensePlan plan;
    ptdr_status v = compose ? make_dense_plan(true, n, c_type, a_type, prec, &plan)
                            : make_dense_plan(false, n, a_type, c_type, prec, &plan);
    if (v != PTDR_OK) return v;
    *bytes = plan.ws_bytes;
    return PTDR_OK;
}

ptdr_status ptdr_last_device_status(void* stream)
{
    int dev = 0;
    ptdr_status v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    unsigned int* st = nullptr;
    v = status_word(dev, &st);
    if (v != PTDR_OK) return v;
    unsigned int word = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&word, st, sizeof(word), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(st, 0, sizeof(word), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return PTDR_ERR_CUDA;
    }
    return (ptdr_status)word;
}

const char* ptdr_status_string(ptdr_status s)
{
    switch (s) {
    case PTDR_OK: return "PTDR_OK";
    case PTDR_ERR_INVALID_ARG: return "PTDR_ERR_INVALID_ARG";
    case PTDR_ERR_UNSUPPORTED: return "PTDR_ERR_UNSUPPORTED";
    case PTDR_ERR_NO_DEVICE: return "PTDR_ERR_NO_DEVICE";
    case PTDR_ERR_CUDA: return "PTDR_ERR_CUDA";
    case PTDR_ERR_WORKSPACE: return "PTDR_ERR_WORKSPACE";
    case PTDR_ERR_TIMEOUT: return "PTDR_ERR_TIMEOUT";
    case PTDR_ERR_INTERNAL: return "PTDR_ERR_INTERNAL";
    }
    return "PTDR_ERR_UNKNOWN";
}

int ptdr_version(void) { return 100; }

} // extern "C"
