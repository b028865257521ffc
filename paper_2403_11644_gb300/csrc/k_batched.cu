// Batched decomposition of many independent matrices of uneven size in one
// persistent launch.  The paper splits its Pauli tree into a forest of
// independent subtrees, one per thread (Sec. V.B); here the independent work
// items are (matrix, block of masks) pairs taken from an atomic queue in
// longest-first order, so a single grid of resident CTAs balances matrices
// of n = 1..13 without a launch per matrix.  Items of complex64 matrices of
// n = 9 .. 12 computed in FP32 run the register-round items of rr_items.cuh;
// every other item runs the generic tile path (gather, shared-memory passes,
// phased write-out).
#include <algorithm>
#include <type_traits>

#include "batched.h"
#include "rr_items.cuh"
#include "tile_ops.cuh"

namespace ptdr {

// Masks per work item: whole rows of 2^n values, up to 16 rows and within the
// tile budget (the same rule as the single-matrix planner).
__host__ __device__ __forceinline__ int batch_log_r(int n, int tile_log)
{
    int lr = 0;
    while (lr < 4 && lr < n && n + lr + 1 <= (tile_log > n ? tile_log : n)) ++lr;
    return lr;
}

// Planner: counting sort of the matrices by descending n, and the first work
// item of each.  One thread; the table is a few entries per matrix.
__global__ void k_batch_plan(const int* d_n, int count, BatchTables tab, int tile_log,
                             unsigned int* st)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int cls[kBatchMaxN + 2];
    for (int i = 0; i <= kBatchMaxN + 1; ++i) cls[i] = 0;
    bool bad = false;
    for (int i = 0; i < count; ++i) {
        const int n = d_n[i];
        if (n < 1 || n > kBatchMaxN) {
            bad = true;
            continue;
        }
        ++cls[n];
    }
    // class start ranks, largest n first
    int pos[kBatchMaxN + 2];
    int r = 0;
    for (int n = kBatchMaxN; n >= 1; --n) {
        pos[n] = r;
        r += cls[n];
    }
    for (int i = 0; i < count; ++i) {
        const int n = d_n[i];
        if (n < 1 || n > kBatchMaxN) continue;
        tab.order[pos[n]++] = i;
    }
    long long items = 0;
    for (int k = 0; k < r; ++k) {
        const int n = d_n[tab.order[k]];
        tab.start[k] = (int)items;
        items += 1ll << (n - batch_log_r(n, tile_log));
    }
    if (bad || items > tab.max_items) {
        report_status(st, PTDR_ERR_INVALID_ARG);
        items = 0;
        r = 0;
    }
    tab.hdr[0] = 0;            // queue head
    tab.hdr[1] = (int)items;   // total items
    tab.hdr[2] = r;            // ranked matrices
}

template <typename T, typename InT, typename OutT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_batched(BatchLaunch p, BatchTables tab, unsigned int* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using T2 = cplx_t<T>;
    T2* s = reinterpret_cast<T2*>(smem_raw);
    __shared__ int s_item;
    const int total = tab.hdr[1];
    const int ranked = tab.hdr[2];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&tab.hdr[0], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        // rank = last k with start[k] <= item
        int lo = 0, hi = ranked - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab.start[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const int m = tab.order[lo];
        const int n = p.d_n[m];
        const int log_r = batch_log_r(n, p.tile_log);
        const uint64_t x0 = (uint64_t)(item - tab.start[lo]) << log_r;
        const InT* A = (const InT*)p.d_A[m];
        OutT* C = (OutT*)p.d_C[m];
        if constexpr (std::is_same<T, float>::value && std::is_same<InT, float2>::value &&
                      std::is_same<OutT, float2>::value) {
            if (n >= 9 && n <= 12 && log_r == 13 - n && !(((uintptr_t)A | (uintptr_t)C) & 15)) {
                const float sc = ldexpf(1.0f, -n);
                if (n == 9) rr_item<9>(A, C, (uint32_t)x0, s, sc, st);
                else if (n == 10) rr_item<10>(A, C, (uint32_t)x0, s, sc, st);
                else if (n == 11) rr_item<11>(A, C, (uint32_t)x0, s, sc, st);
                else rr_item<12>(A, C, (uint32_t)x0, s, sc, st);
                __syncthreads(); // s and s_item are reused by the next item
                continue;
            }
        }
        const Smem sm = make_smem(n);
        const uint64_t elems = 1ull << (2 * n);
        load_gather<T>(s, sm, A, n, x0, log_r, 0, n, elems, st);
        __syncthreads();
        wht_bits(s, sm, log_r + n, 0, n);
        store_row_phase<T>(C, s, sm, n, x0, log_r, 0, n, 0, (T)ldexp(1.0, -n), elems, st);
        __syncthreads(); // s and s_item are reused by the next item
    }
}

template <typename T, typename InT, typename OutT>
static cudaError_t run_batched(const BatchLaunch& p, const BatchTables& tab, unsigned int* st,
                               cudaStream_t s)
{
    auto kern = k_batched<T, InT, OutT>;
    size_t need = 0;
    for (int n = 1; n <= p.max_n; ++n) {
        const size_t b = smem_elems((size_t)1 << batch_log_r(n, p.tile_log), n) * sizeof(cplx_t<T>);
        need = b > need ? b : need;
    }
    if (std::is_same<T, float>::value && std::is_same<InT, float2>::value && std::is_same<OutT, float2>::value &&
        p.max_n >= 9)
        need = std::max(need, (size_t)kRrElems * sizeof(float2));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, need)) != cudaSuccess)
        return e;
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    k_batch_plan<<<1, 32, 0, s>>>(p.d_n, p.count, tab, p.tile_log, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kern<<<grid, 256, need, s>>>(p, tab, st);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t batched_by_types(const BatchLaunch& p, const BatchTables& tab, unsigned int* st,
                                    cudaStream_t s)
{
    if (p.a_t == PTDR_C64 && p.c_t == PTDR_C64) return run_batched<T, float2, float2>(p, tab, st, s);
    if (p.a_t == PTDR_C64 && p.c_t == PTDR_C128) return run_batched<T, float2, double2>(p, tab, st, s);
    if (p.a_t == PTDR_C128 && p.c_t == PTDR_C64) return run_batched<T, double2, float2>(p, tab, st, s);
    if (p.a_t == PTDR_C128 && p.c_t == PTDR_C128)
        return run_batched<T, double2, double2>(p, tab, st, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_batched(const BatchLaunch& p, const BatchTables& tab, unsigned int* st,
                           cudaStream_t s)
{
    return p.calc == Calc::F32 ? batched_by_types<float>(p, tab, st, s)
                               : batched_by_types<double>(p, tab, st, s);
}

int batched_items(int n, int tile_log) { return 1 << (n - batch_log_r(n, tile_log)); }

} // namespace ptdr
