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

// Planner: stable counting sort of the matrices by descending n, and the
// first work item of each rank.  One CTA of kPlanThreads threads:
//   1. a class histogram of the sizes (shared atomics);
//   2. per class (largest n first) its first rank and its first work item:
//      every matrix of size n has the same number of items, so the first item
//      of rank k in class n is that class's first item plus (k - pos[n])
//      times the class's items per matrix -- no sequential scan;
//   3. the ranks, chunk by chunk in index order: a matrix's rank is its class's
//      first rank, plus the matrices of its class in earlier chunks, plus those
//      in earlier warps of the chunk (per-warp class counts), plus those in
//      earlier lanes of its warp (__match_any_sync), so the order inside a
//      class is the index order.
constexpr int kPlanThreads = 1024;
constexpr int kPlanWarps = kPlanThreads / 32;
constexpr int kClasses = kBatchMaxN + 1; // n = 1 .. kBatchMaxN (entry 0 unused)

__global__ void __launch_bounds__(kPlanThreads) k_batch_plan(const int* d_n, int count, BatchTables tab, int tile_log,
                                                             unsigned int* st)
{
    __shared__ int s_cls[kClasses], s_pos[kClasses], s_run[kClasses], s_chunk[kClasses], s_wcnt[kPlanWarps][kClasses];
    __shared__ long long s_base[kClasses];
    __shared__ int s_bad, s_ranked;
    __shared__ long long s_items;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t < kClasses) {
        s_cls[t] = 0;
        s_run[t] = 0;
    }
    if (t == 0) s_bad = 0;
    __syncthreads();
    for (int i = t; i < count; i += kPlanThreads) {
        const int n = d_n[i];
        if (n < 1 || n > kBatchMaxN) s_bad = 1;
        else atomicAdd(&s_cls[n], 1);
    }
    __syncthreads();
    if (t == 0) {
        int r = 0;
        long long items = 0;
        for (int n = kBatchMaxN; n >= 1; --n) {
            s_pos[n] = r;
            s_base[n] = items;
            r += s_cls[n];
            items += (long long)s_cls[n] << (n - batch_log_r(n, tile_log));
        }
        s_ranked = r;
        s_items = items;
        if (s_bad || items > tab.max_items) {
            report_status(st, PTDR_ERR_INVALID_ARG);
            s_ranked = 0;
            s_items = 0;
        }
        tab.hdr[0] = 0;                 // queue head
        tab.hdr[1] = (int)s_items;      // total items
        tab.hdr[2] = s_ranked;          // ranked matrices
    }
    __syncthreads();
    if (s_ranked == 0) return;
    const unsigned lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < count; c0 += kPlanThreads) {
        const int i = c0 + t;
        const int n = i < count ? d_n[i] : 0; // 0: no matrix (sizes are valid here)
        const unsigned same = __match_any_sync(0xffffffffu, n);
        const int before = __popc(same & lt);
        for (int k = t; k < kPlanWarps * kClasses; k += kPlanThreads) s_wcnt[k / kClasses][k % kClasses] = 0;
        __syncthreads();
        if (n > 0 && before == 0) s_wcnt[warp][n] = __popc(same);
        __syncthreads();
        // exclusive prefix over the warps, per class; the chunk's totals go to s_run
        if (t < kClasses && t > 0) {
            int acc = 0;
            for (int w = 0; w < kPlanWarps; ++w) {
                const int v = s_wcnt[w][t];
                s_wcnt[w][t] = acc;
                acc += v;
            }
            s_chunk[t] = acc;
        }
        __syncthreads();
        if (n > 0) tab.order[s_pos[n] + s_run[n] + s_wcnt[warp][n] + before] = i;
        __syncthreads();
        if (t < kClasses && t > 0) s_run[t] += s_chunk[t];
        __syncthreads();
    }
    // first work item of every rank
    for (int k = t; k < s_ranked; k += kPlanThreads) {
        int n = kBatchMaxN;
        while (n > 1 && k >= s_pos[n] + s_run[n]) --n; // s_run[n] = class size by now
        tab.start[k] = (int)(s_base[n] + ((long long)(k - s_pos[n]) << (n - batch_log_r(n, tile_log))));
    }
}

// One work item as the loop needs it: its queue index (>= total: no item),
// matrix and first mask, and whether it runs the register rounds.
struct BatchItem {
    int item;
    int n, log_r, rr;
    uint64_t x0;
    const void* A;
    void* C;
};

// Warp 0's view of the queue, kept in shared memory (nothing of it stays in
// registers across an item): the rank of the last resolved item (a CTA's
// items only increase, so the rank never decreases), that rank's matrix, and
// the queue index taken ahead of time (its atomic's latency overlaps an item).
struct BatchCursor {
    int rank, m, n, start, ahead;
    const void* A;
    void* C;
};

// Warp-collective (all 32 lanes of warp 0): resolves queue index `item`
// against the cursor c; lane 0 updates c and returns the item.
template <bool kRr>
__device__ BatchItem resolve_item(BatchCursor* c, int item, const BatchLaunch& p, const BatchTables& tab, int total,
                                  int ranked, int lane)
{
    BatchItem it{};
    it.item = item;
    if (item >= total) return it;
    // rank = last r with start[r] <= item: probe the next 32 ranks at once
    // (starts increase, so those <= item are a prefix), else binary search
    int rank = c->rank;
    const int r = rank + 1 + lane;
    const int v = r < ranked ? tab.start[r] : 0x7fffffff;
    const unsigned le = __ballot_sync(0xffffffffu, v <= item);
    if (le != 0xffffffffu) {
        rank += __popc(le);
    } else {
        int lo = rank + 32, hi = ranked - 1;
        if (lane == 0)
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tab.start[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
        rank = __shfl_sync(0xffffffffu, lo, 0);
    }
    if (lane == 0) {
        const int m = tab.order[rank];
        if (m != c->m) {
            c->m = m;
            c->start = tab.start[rank];
            c->n = p.d_n[m];
            c->A = p.d_A[m];
            c->C = p.d_C[m];
        }
        c->rank = rank;
        it.n = c->n;
        it.log_r = batch_log_r(it.n, p.tile_log);
        it.x0 = (uint64_t)(item - c->start) << it.log_r;
        it.A = c->A;
        it.C = c->C;
        it.rr = kRr && it.n >= 9 && it.n <= 12 && it.log_r == 13 - it.n && !(((uintptr_t)it.A | (uintptr_t)it.C) & 15);
    }
    __syncwarp();
    return it;
}

__device__ __forceinline__ void rr_issue_n(int n, const void* A, uint64_t x0, float2* s, unsigned int* st)
{
    const float2* a = (const float2*)A;
    if (n == 9) rr_issue<9>(a, (uint32_t)x0, s, st);
    else if (n == 10) rr_issue<10>(a, (uint32_t)x0, s, st);
    else if (n == 11) rr_issue<11>(a, (uint32_t)x0, s, st);
    else rr_issue<12>(a, (uint32_t)x0, s, st);
}

// The persistent loop.  Items pass through a ring of three shared slots: while
// item i runs, item i + 1 is already resolved (its copies are issued by item
// i's hook) and warp 0 resolves item i + 2 after item i's first round, so
// that its dependent table loads overlap the other warps' second round
// instead of holding every warp at a barrier.
template <typename T, typename InT, typename OutT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_batched(BatchLaunch p, BatchTables tab, unsigned int* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using T2 = cplx_t<T>;
    T2* s = reinterpret_cast<T2*>(smem_raw);
    __shared__ BatchItem s_it[3];
    __shared__ BatchCursor s_cur;
    constexpr bool kRr = std::is_same<T, float>::value && std::is_same<InT, float2>::value &&
                         std::is_same<OutT, float2>::value;
    const int total = tab.hdr[1];
    const int ranked = tab.hdr[2];
    const int t = threadIdx.x, lane = t & 31;
    // warp 0: resolves the queue index taken ahead into slot `to` and takes the next one
    auto advance = [&](int to) {
        const int q = s_cur.ahead;
        int q2 = total;
        if (lane == 0 && q < total) q2 = atomicAdd(&tab.hdr[0], 1);
        const BatchItem nx = resolve_item<kRr>(&s_cur, q, p, tab, total, ranked, lane);
        if (lane == 0) {
            s_it[to] = nx;
            s_cur.ahead = q2;
        }
        __syncwarp();
    };
    if (t < 32) {
        if (lane == 0) {
            s_cur.rank = 0;
            s_cur.m = -1;
            s_cur.ahead = atomicAdd(&tab.hdr[0], 1);
        }
        __syncwarp();
        advance(0);
        advance(1);
    }
    __syncthreads();
    int slot = 0;
    bool issued = false; // the current item's piece copies are in flight
    if constexpr (kRr) {
        const BatchItem it = s_it[0];
        if (it.item < total && it.rr) {
            rr_issue_n(it.n, it.A, it.x0, reinterpret_cast<float2*>(s), st);
            issued = true;
        }
    }
    for (;;) {
        const BatchItem it = s_it[slot];
        if (it.item >= total) break;
        const int s1 = slot == 2 ? 0 : slot + 1, s2 = s1 == 2 ? 0 : s1 + 1;
        if constexpr (kRr) {
            if (it.rr) {
                float2* sf = reinterpret_cast<float2*>(s);
                bool next_issued = false;
                // after round 1 (warp 0): resolve the item after next; once the last
                // round has read the tile: the next item's copies
                auto mid = [&]() {
                    if (t < 32) advance(s2);
                };
                auto hook = [&]() {
                    __syncthreads();
                    const BatchItem nx = s_it[s1];
                    if (nx.item < total && nx.rr) {
                        rr_issue_n(nx.n, nx.A, nx.x0, sf, st);
                        next_issued = true;
                    }
                };
                const float2* A = (const float2*)it.A;
                float2* C = (float2*)it.C;
                const float sc = ldexpf(1.0f, -it.n);
                if (it.n == 9) rr_item<9>(A, C, (uint32_t)it.x0, sf, sc, st, issued, hook, mid);
                else if (it.n == 10) rr_item<10>(A, C, (uint32_t)it.x0, sf, sc, st, issued, hook, mid);
                else if (it.n == 11) rr_item<11>(A, C, (uint32_t)it.x0, sf, sc, st, issued, hook, mid);
                else rr_item<12>(A, C, (uint32_t)it.x0, sf, sc, st, issued, hook, mid);
                __syncthreads(); // s_it[s2] is complete; s is rewritten next
                issued = next_issued;
                slot = s1;
                continue;
            }
        }
        if (t < 32) advance(s2);
        const Smem sm = make_smem(it.n);
        const uint64_t elems = 1ull << (2 * it.n);
        load_gather<T>(s, sm, (const InT*)it.A, it.n, it.x0, it.log_r, 0, it.n, elems, st);
        __syncthreads();
        wht_bits(s, sm, it.log_r + it.n, 0, it.n);
        store_row_phase<T>((OutT*)it.C, s, sm, it.n, it.x0, it.log_r, 0, it.n, 0, (T)ldexp(1.0, -it.n), elems, st);
        __syncthreads(); // s is reused next
        issued = false;
        slot = s1;
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
    k_batch_plan<<<1, kPlanThreads, 0, s>>>(p.d_n, p.count, tab, p.tile_log, st);
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
