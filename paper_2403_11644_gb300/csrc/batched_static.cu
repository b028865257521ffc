// ptdr_decompose_batched_static: the batched decomposition without a
// caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they want to
// decompose: a host application whose device memory is entirely owned by its
// own pool or allocator, code on a latency-critical stream where an
// allocation would add a device-wide synchronisation, or a runtime that forbids dynamic allocation after start-up.
// This entry point lets them run the batched decomposition with nothing but
// their inputs and outputs: its only scratch (the planner's tables and the
// work-queue counter) lives in a fixed array in the library's device image,
// which every GPU that loads the library keeps until the process exits.
#include <mutex>

#include "batched.h"
#include "plan.h"

namespace {

constexpr int kStaticMaxMatrices = 4096;
constexpr size_t kTableBytes = ((size_t)kStaticMaxMatrices * 4 + 15) & ~(size_t)15;
constexpr size_t kStaticScratchBytes = 16 + 2 * kTableBytes; // 32,784 bytes

// The scratch: header (queue head, item count, ranked matrices), then the
// rank -> matrix table, then the rank -> first item table.
static __device__ __align__(256) unsigned char g_batched_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];

// Device address of the scratch array on device `dev` (which must be
// current).  In host code the array's name is only a host-side stand-in, so
// the address is looked up once per device and cached for the life of the
// process (a cudaDeviceReset reloads the module, so the library must not be
// used across one).
ptdr_status scratch_address(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return PTDR_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_batched_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PTDR_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PTDR_OK;
}

} // namespace

using namespace ptdr;

extern "C" {

ptdr_status ptdr_decompose_batched_static(const void* const* d_A, void* const* d_C,
                                          const int* d_n, const int* h_n, int count,
                                          ptdr_dtype a_type, ptdr_dtype c_type,
                                          ptdr_precision prec, void* stream)
{
    PTDR_TRACE();
    if (!d_A || !d_C || !d_n) return PTDR_ERR_INVALID_ARG;
    // Same argument rules as ptdr_decompose_batched; the table size it reports
    // must fit the static array.
    size_t need = 0;
    ptdr_status v = ptdr_batched_workspace_size(h_n, count, a_type, c_type, prec, &need);
    if (v != PTDR_OK) return v;
    if (count > kStaticMaxMatrices || need > kStaticScratchBytes) return PTDR_ERR_WORKSPACE;
    if (fault_injected("plan")) return PTDR_ERR_INTERNAL;
    long long items = 0;
    int max_n = 0;
    for (int i = 0; i < count; ++i) {
        items += batched_items(h_n[i], prec == PTDR_PREC_FP64 ? 12 : 13);
        max_n = h_n[i] > max_n ? h_n[i] : max_n;
    }
    int dev = 0;
    v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(d_A) != PTDR_OK || check_device_ptr(d_C) != PTDR_OK ||
        check_device_ptr(d_n) != PTDR_OK)
        return PTDR_ERR_INVALID_ARG;
    unsigned int* st = nullptr;
    v = status_word(dev, &st);
    if (v != PTDR_OK) return v;
    void* scratch = nullptr;
    v = scratch_address(dev, &scratch);
    if (v != PTDR_OK) return v;
    if (fault_injected("launch")) return PTDR_ERR_CUDA;

    // Every table entry the kernels read is rewritten by the planner kernel at
    // the start of each call, and the planner also resets the queue head to
    // zero, so the previous call's contents never leak into this one.
    char* w = (char*)scratch;
    BatchTables tab;
    tab.hdr = (int*)w;
    tab.order = (int*)(w + 16);
    tab.start = (int*)(w + 16 + kTableBytes);
    tab.max_items = (int)items;
    BatchLaunch p;
    p.d_A = d_A;
    p.d_C = d_C;
    p.d_n = d_n;
    p.count = count;
    p.a_t = a_type;
    p.c_t = c_type;
    p.calc = prec == PTDR_PREC_FP64 ? Calc::F64 : Calc::F32;
    p.tile_log = prec == PTDR_PREC_FP64 ? 12 : 13;
    p.max_n = max_n;
    return launch_batched(p, tab, st, (cudaStream_t)stream) == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

} // extern "C"
