// ptdr_decompose_batched: validation, workspace layout and launch.
#include <cstdint>

#include "batched.h"
#include "plan.h"

using namespace ptdr;

namespace {

int tile_log_for(ptdr_precision prec) { return prec == PTDR_PREC_FP64 ? 12 : 13; }

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

ptdr_status validate_batched(const int* h_n, int count, ptdr_dtype a_t, ptdr_dtype c_t,
                             ptdr_precision prec, size_t* ws, long long* items, int* max_n)
{
    if (!h_n || count < 1 || count > (1 << 20)) return PTDR_ERR_INVALID_ARG;
    if ((int)a_t < PTDR_C64 || (int)a_t > PTDR_F64 || (int)c_t < PTDR_C64 || (int)c_t > PTDR_F64)
        return PTDR_ERR_INVALID_ARG;
    if ((int)prec < PTDR_PREC_FP64 || (int)prec > PTDR_PREC_FIXED_I128) return PTDR_ERR_INVALID_ARG;
    if (!dtype_complex(a_t) || !dtype_complex(c_t)) return PTDR_ERR_UNSUPPORTED;
    if (prec != PTDR_PREC_FP64 && prec != PTDR_PREC_FP32) return PTDR_ERR_UNSUPPORTED;
    long long total = 0;
    int mx = 0;
    for (int i = 0; i < count; ++i) {
        if (h_n[i] < 1 || h_n[i] > kBatchMaxN) return PTDR_ERR_INVALID_ARG;
        total += batched_items(h_n[i], tile_log_for(prec));
        mx = h_n[i] > mx ? h_n[i] : mx;
    }
    if (total > INT32_MAX) return PTDR_ERR_INVALID_ARG;
    *items = total;
    *max_n = mx;
    *ws = 16 + align16((size_t)count * 4) * 2;
    return PTDR_OK;
}

} // namespace

extern "C" {

ptdr_status ptdr_batched_workspace_size(const int* h_n, int count, ptdr_dtype a_type,
                                        ptdr_dtype c_type, ptdr_precision prec, size_t* bytes)
{
    if (!bytes) return PTDR_ERR_INVALID_ARG;
    long long items = 0;
    int mx = 0;
    return validate_batched(h_n, count, a_type, c_type, prec, bytes, &items, &mx);
}

ptdr_status ptdr_decompose_batched(const void* const* d_A, void* const* d_C, const int* d_n,
                                   const int* h_n, int count, ptdr_dtype a_type,
                                   ptdr_dtype c_type, ptdr_precision prec, void* workspace,
                                   size_t workspace_bytes, void* stream)
{
    PTDR_TRACE();
    if (!d_A || !d_C || !d_n) return PTDR_ERR_INVALID_ARG;
    size_t need = 0;
    long long items = 0;
    int max_n = 0;
    ptdr_status v = validate_batched(h_n, count, a_type, c_type, prec, &need, &items, &max_n);
    if (v != PTDR_OK) return v;
    if (!workspace || workspace_bytes < need) return PTDR_ERR_WORKSPACE;
    if ((uintptr_t)workspace % 16) return PTDR_ERR_INVALID_ARG;
    if (fault_injected("plan")) return PTDR_ERR_INTERNAL;
    int dev = 0;
    v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(d_A) != PTDR_OK || check_device_ptr(d_C) != PTDR_OK ||
        check_device_ptr(d_n) != PTDR_OK || check_device_ptr(workspace) != PTDR_OK)
        return PTDR_ERR_INVALID_ARG;
    unsigned int* st = nullptr;
    v = status_word(dev, &st);
    if (v != PTDR_OK) return v;
    if (fault_injected("launch")) return PTDR_ERR_CUDA;

    char* w = (char*)workspace;
    BatchTables tab;
    tab.hdr = (int*)w;
    tab.order = (int*)(w + 16);
    tab.start = (int*)(w + 16 + align16((size_t)count * 4));
    tab.max_items = (int)items;
    BatchLaunch p;
    p.d_A = d_A;
    p.d_C = d_C;
    p.d_n = d_n;
    p.count = count;
    p.a_t = a_type;
    p.c_t = c_type;
    p.calc = prec == PTDR_PREC_FP64 ? Calc::F64 : Calc::F32;
    p.tile_log = tile_log_for(prec);
    p.max_n = max_n;
    return launch_batched(p, tab, st, (cudaStream_t)stream) == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

} // extern "C"
