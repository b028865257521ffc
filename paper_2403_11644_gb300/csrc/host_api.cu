// Host-buffer entry point: decomposes matrices that live in host memory.
//
// The matrices pass through two device buffers each for A and C (the
// caller's scratch), so that the upload of matrix i + 1, the decomposition of
// matrix i and the download of matrix i - 1 run at the same time: on GB300 the
// host link carries both directions at once (about 170 GB/s each way), so a
// stream of matrices costs one transfer time per matrix instead of two plus
// the kernel.  Uploads and downloads run on two library streams per device;
// every step is ordered by events, and the caller's stream completes after
// the last download.
#include <cmath>
#include <mutex>

#include "plan.h"

using namespace ptdr;

namespace {

struct HostPipe {
    bool ready = false;
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t start = nullptr, loaded[2] = {}, done[2] = {}, drained[2] = {};
};

std::mutex g_pipe_mu; // also serialises the enqueue of concurrent calls
HostPipe g_pipe[128];

ptdr_status pipe_for(int dev, HostPipe** out)
{
    HostPipe& p = g_pipe[dev];
    if (!p.ready) {
        bool ok = cudaStreamCreateWithFlags(&p.up, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&p.down, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming) == cudaSuccess;
        for (int b = 0; b < 2 && ok; ++b)
            ok = cudaEventCreateWithFlags(&p.loaded[b], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&p.done[b], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&p.drained[b], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return PTDR_ERR_CUDA;
        }
        p.ready = true;
    }
    *out = &p;
    return PTDR_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct HostLayout {
    size_t a_bytes, c_bytes, ws_bytes, total;
};

ptdr_status host_layout(int n, ptdr_dtype a_t, ptdr_dtype c_t, ptdr_precision prec, DensePlan* plan,
                        HostLayout* lay)
{
    if (n < 1 || n > kMaxDenseN) return PTDR_ERR_INVALID_ARG;
    if ((int)a_t < PTDR_C64 || (int)a_t > PTDR_F64 || (int)c_t < PTDR_C64 || (int)c_t > PTDR_F64)
        return PTDR_ERR_INVALID_ARG;
    if ((int)prec < PTDR_PREC_FP64 || (int)prec > PTDR_PREC_FIXED_I128) return PTDR_ERR_INVALID_ARG;
    if (prec == PTDR_PREC_SPLIT_BF16_TC && (a_t != PTDR_C64 || (c_t != PTDR_C64 && c_t != PTDR_F32)))
        return PTDR_ERR_UNSUPPORTED;
    ptdr_status v = make_dense_plan(false, n, a_t, c_t, prec, plan);
    if (v != PTDR_OK) return v;
    const size_t elems = (size_t)1 << (2 * n);
    lay->a_bytes = elems * dtype_bytes(a_t);
    lay->c_bytes = elems * dtype_bytes(c_t);
    lay->ws_bytes = plan->ws_bytes;
    lay->total = 2 * align256(lay->a_bytes) + 2 * align256(lay->c_bytes) + align256(lay->ws_bytes);
    return PTDR_OK;
}

} // namespace

extern "C" {

ptdr_status ptdr_decompose_host_scratch_size(int n, ptdr_dtype a_type, ptdr_dtype c_type, ptdr_precision prec,
                                             size_t* bytes)
{
    if (!bytes) return PTDR_ERR_INVALID_ARG;
    DensePlan plan;
    HostLayout lay;
    ptdr_status v = host_layout(n, a_type, c_type, prec, &plan, &lay);
    if (v != PTDR_OK) return v;
    *bytes = lay.total;
    return PTDR_OK;
}

ptdr_status ptdr_decompose_host(const void* const* h_A, void* const* h_C, int count, ptdr_dtype a_type,
                                ptdr_dtype c_type, int n, ptdr_precision prec, void* d_scratch,
                                size_t d_scratch_bytes, void* stream)
{
    PTDR_TRACE();
    if (!h_A || !h_C || count < 1) return PTDR_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!h_A[i] || !h_C[i]) return PTDR_ERR_INVALID_ARG;
    DensePlan plan;
    HostLayout lay;
    ptdr_status v = host_layout(n, a_type, c_type, prec, &plan, &lay);
    if (v != PTDR_OK) return v;
    for (int i = 0; i < count; ++i)
        if ((uintptr_t)h_A[i] % dtype_bytes(a_type) || (uintptr_t)h_C[i] % dtype_bytes(c_type) ||
            overlaps(h_A[i], lay.a_bytes, h_C[i], lay.c_bytes))
            return PTDR_ERR_INVALID_ARG;
    if (!d_scratch || d_scratch_bytes < lay.total) return PTDR_ERR_WORKSPACE;
    if ((uintptr_t)d_scratch % 256) return PTDR_ERR_INVALID_ARG;
    if (fault_injected("plan")) return PTDR_ERR_INTERNAL;
    int dev = 0;
    v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(d_scratch) != PTDR_OK) return PTDR_ERR_INVALID_ARG;
    unsigned int* st = nullptr;
    v = status_word(dev, &st);
    if (v != PTDR_OK) return v;
    if (fault_injected("launch")) return PTDR_ERR_CUDA;

    char* base = (char*)d_scratch;
    void* dA[2] = {base, base + align256(lay.a_bytes)};
    char* cbase = base + 2 * align256(lay.a_bytes);
    void* dC[2] = {cbase, cbase + align256(lay.c_bytes)};
    void* ws = lay.ws_bytes ? cbase + 2 * align256(lay.c_bytes) : nullptr;
    const double scale = std::ldexp(1.0, -n);

    std::lock_guard<std::mutex> lk(g_pipe_mu);
    HostPipe* p = nullptr;
    v = pipe_for(dev, &p);
    if (v != PTDR_OK) return v;
    cudaStream_t s = (cudaStream_t)stream;
    bool ok = true;
    auto chk = [&](cudaError_t e) {
        if (e != cudaSuccess) ok = false;
    };
    // the copies follow whatever the caller enqueued on its stream before
    chk(cudaEventRecord(p->start, s));
    chk(cudaStreamWaitEvent(p->up, p->start, 0));
    chk(cudaStreamWaitEvent(p->down, p->start, 0));
    for (int i = 0; i < count && ok; ++i) {
        const int b = i & 1;
        // buffer b was read by the decomposition of matrix i - 2
        if (i >= 2) chk(cudaStreamWaitEvent(p->up, p->done[b], 0));
        chk(cudaMemcpyAsync(dA[b], h_A[i], lay.a_bytes, cudaMemcpyHostToDevice, p->up));
        chk(cudaEventRecord(p->loaded[b], p->up));
        chk(cudaStreamWaitEvent(s, p->loaded[b], 0));
        // C buffer b was copied out for matrix i - 2
        if (i >= 2) chk(cudaStreamWaitEvent(s, p->drained[b], 0));
        if (!ok) break;
        v = execute_dense(plan, dA[b], dC[b], ws, scale, st, s);
        if (v != PTDR_OK) return v;
        chk(cudaEventRecord(p->done[b], s));
        chk(cudaStreamWaitEvent(p->down, p->done[b], 0));
        chk(cudaMemcpyAsync(h_C[i], dC[b], lay.c_bytes, cudaMemcpyDeviceToHost, p->down));
        chk(cudaEventRecord(p->drained[b], p->down));
    }
    // the caller's stream completes after the last downloads
    if (ok) chk(cudaStreamWaitEvent(s, p->drained[(count - 1) & 1], 0));
    if (ok && count >= 2) chk(cudaStreamWaitEvent(s, p->drained[count & 1], 0));
    if (!ok) {
        cudaGetLastError();
        return PTDR_ERR_CUDA;
    }
    return PTDR_OK;
}

} // extern "C"
