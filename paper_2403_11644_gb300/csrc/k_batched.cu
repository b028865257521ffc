// Batched decomposition of many independent matrices of uneven size in one
// persistent launch.  The paper splits its Pauli tree into a forest of
// independent subtrees, one per thread (Sec. V.B); here the independent work
// items are (matrix, block of masks) pairs taken from an atomic queue in
// longest-first order, so a single grid of resident CTAs balances matrices
// of n = 1..13 without a launch per matrix.  Items of complex64 matrices of
// n = 9, 10, 11 computed in FP32 run a register-round path (below); every
// other item runs the generic tile path (gather, shared-memory passes,
// phased write-out).
#include <algorithm>
#include <type_traits>

#include "batched.h"
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

// ---------------------------------------------------------------------------
// Register-round items for complex64 matrices of n = 9, 10, 11 computed in
// FP32 (nearly all the work of a batch of mixed sizes: 4^n grows fastest).
// An item is the R = 2^(13-n) masks x0 .. x0 + R - 1 (x0 a multiple of R), a
// tile of 8192 values.  Its gather d_x[k] = A[k ^ x][k] is, row by row of A,
// the R columns (r ^ x0) & ~(R - 1) .. + R - 1 of row r: the item copies these
// pieces (32, 64 or 128 bytes) into shared memory as they are, 16 bytes per
// cp.async, and reads the XOR permutation out of that "piece tile": with
// k = kh R + kl, value (xl, k) sits at ((kh ^ X0) << 2 lr) + ((kl ^ xl) << lr)
// + kl, X0 = x0 / R.  The length-2^n transform then runs in register rounds
// of up to 5 bits (kh bits 0-4; then the rest), each thread holding 32
// values, with transposes through a padded "round tile" of rows (xl, w) where
// w is the transformed kh bits 0-4.  Row stride 2^(n-5) + 1 and mask stride
// 32 rows + 8 place every warp access on distinct bank pairs (two wavefronts
// per 8-byte warp access, the minimum) and make every address a register
// plus a constant.  The first round reads its 32 values at kh bits 0-4 equal
// to (slot ^ X0 bits 0-4), so that its output slot w carries the sign
// (-1)^{|w & X0 bits 0-4|}; w is the lane in the last round, where the sign
// joins the phase.  The last round writes C rows with 16-byte stores.  A's
// pieces are shared by the neighbouring items (x0 +- R ...), which run at the
// same time, so each line of A is read from HBM once.

template <int NQ>
struct RrShape {
    static constexpr int LR = 13 - NQ;    // log2 of the masks per item
    static constexpr int R = 1 << LR;
    static constexpr int W = NQ - 5;      // log2 of a round-tile row (xl, w)
    static constexpr int S = (1 << W) + 1; // padded row stride
    static constexpr int XS = 32 * S + 8; // stride between masks
    static constexpr int SIZE = R * XS;   // elements of the round tile
    static_assert(SIZE >= 8192, "the round tile holds the piece tile");
};
constexpr int kRrElems = RrShape<9>::SIZE; // the largest of n = 9, 10, 11
static_assert(RrShape<10>::SIZE <= kRrElems && RrShape<11>::SIZE <= kRrElems, "tile size");

// Radix-2 butterflies over 2^NB of the registers: v[OFF + STEP i], i < 2^NB.
template <int NB, int OFF, int STEP, int M>
__device__ __forceinline__ void wht_sub(float2 (&v)[M])
{
#pragma unroll
    for (int h = 1; h < (1 << NB); h <<= 1)
#pragma unroll
        for (int i = 0; i < (1 << NB); ++i)
            if (!(i & h)) {
                const float2 a = v[OFF + STEP * i], b = v[OFF + STEP * (i + h)];
                v[OFF + STEP * i] = make_float2(a.x + b.x, a.y + b.y);
                v[OFF + STEP * (i + h)] = make_float2(a.x - b.x, a.y - b.y);
            }
}

// C[x][z], C[x][z + 1] = scale (-i)^{|x&z| + sg} a, ... (z even): one 16-byte store.
__device__ __forceinline__ void rr_put(float2* C, uint32_t x, uint32_t z, int sg, float2 a, float2 b,
                                       float scale)
{
    const float2 pa = phase_neg_i(a, __popc(x & z) + sg, scale);
    const float2 pb = phase_neg_i(b, __popc(x & (z + 1)) + sg, scale);
    *reinterpret_cast<float4*>(C + z) = make_float4(pa.x, pa.y, pb.x, pb.y);
}

template <int NQ>
__device__ __forceinline__ void rr_item(const float2* __restrict__ A, float2* __restrict__ C, uint32_t x0,
                                        float2* s, float scale, unsigned int* st)
{
    using Sh = RrShape<NQ>;
    constexpr int LR = Sh::LR, R = Sh::R;
    constexpr uint64_t kElems = 1ull << (2 * NQ);
    const int t = threadIdx.x;
    // the piece tile: row r of A, columns ((r ^ x0) & ~(R - 1)) + [0, R), at s[r R]
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(s);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t q = t + 256 * i; // 16-byte piece: row q >> (lr - 1)
        const uint32_t r = q >> (LR - 1), h = q & ((R >> 1) - 1);
        const uint64_t gi = ((uint64_t)r << NQ) + ((r ^ x0) & ~(uint32_t)(R - 1)) + 2 * h;
        if (in_bounds(st, gi + 1, kElems))
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + 16u * q), "l"(A + gi) : "memory");
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const uint32_t X0 = x0 >> LR;
    const int X0h = (int)(X0 >> 5), X0l = (int)(X0 & 31);
    float2 v[32];
    {
        // round 1: thread (kl, xl, kh bits 5+), 32 values over kh bits 0-4
        const int kl = t & (R - 1), xl = (t >> LR) & (R - 1), khh = t >> (2 * LR);
        const float2* p = s + (((khh ^ X0h) << (5 + 2 * LR)) + ((kl ^ xl) << LR) + kl);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = p[j << (2 * LR)];
        wht_sub<5, 0, 1>(v);
        __syncthreads();
        float2* q = s + (xl * Sh::XS + ((khh << LR) | kl));
#pragma unroll
        for (int w = 0; w < 32; ++w) q[w * Sh::S] = v[w];
        __syncthreads();
    }
    const int warp = t >> 5, w = t & 31;
    const int sg = 2 * (__popc(w & X0l) & 1);
    if constexpr (NQ == 10) {
        // round 2: thread (xl = warp, w = lane), 32 values over (kh bits 5-6, kl)
        const float2* p = s + (warp * Sh::XS + w * Sh::S);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = p[j];
        wht_sub<5, 0, 1>(v);
        const uint32_t x = x0 + warp;
        float2* row = C + ((uint64_t)x << NQ);
        if (in_bounds(st, ((uint64_t)x << NQ) + (1u << NQ) - 1, kElems))
#pragma unroll
            for (int zk = 0; zk < 4; ++zk)
#pragma unroll
                for (int zl = 0; zl < 8; zl += 2)
                    rr_put(row, x, (zk << 8) | (w << 3) | zl, sg, v[zk * 8 + zl], v[zk * 8 + zl + 1], scale);
    } else if constexpr (NQ == 9) {
        // round 2: thread (xl bits 0-2 = warp, w = lane), 2 x 16 values over kl
#pragma unroll
        for (int xh = 0; xh < 2; ++xh) {
            const float2* p = s + ((warp | (xh << 3)) * Sh::XS + w * Sh::S);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[xh * 16 + j] = p[j];
        }
        wht_sub<4, 0, 1>(v);
        wht_sub<4, 16, 1>(v);
#pragma unroll
        for (int xh = 0; xh < 2; ++xh) {
            const uint32_t x = x0 + (warp | (xh << 3));
            float2* row = C + ((uint64_t)x << NQ);
            if (in_bounds(st, ((uint64_t)x << NQ) + (1u << NQ) - 1, kElems))
#pragma unroll
                for (int zl = 0; zl < 16; zl += 2)
                    rr_put(row, x, (w << 4) | zl, sg, v[xh * 16 + zl], v[xh * 16 + zl + 1], scale);
        }
    } else {
        static_assert(NQ == 11, "register-round items cover n = 9, 10, 11");
        // round 2: thread (kl bit 1, xl = warp, w = lane), 2 x 16 values over kh bits 5-8,
        // rewritten in place (each thread rewrites the slots it read)
        {
            float2* p = s + ((warp >> 1) * Sh::XS + w * Sh::S + ((warp & 1) << 1));
#pragma unroll
            for (int kl0 = 0; kl0 < 2; ++kl0)
#pragma unroll
                for (int khh = 0; khh < 16; ++khh) v[kl0 * 16 + khh] = p[(khh << 2) | kl0];
            wht_sub<4, 0, 1>(v);
            wht_sub<4, 16, 1>(v);
#pragma unroll
            for (int kl0 = 0; kl0 < 2; ++kl0)
#pragma unroll
                for (int zk = 0; zk < 16; ++zk) p[(zk << 2) | kl0] = v[kl0 * 16 + zk];
        }
        __syncthreads();
        // round 3: thread (z kh bit 8, xl = warp, w = lane), 8 x 4 values over kl
        const int xl = warp >> 1;
        const float2* p = s + (xl * Sh::XS + w * Sh::S + ((warp & 1) << 5));
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = p[j];
#pragma unroll
        for (int zk = 0; zk < 8; ++zk) {
            // a 4-point transform of registers 4 zk .. 4 zk + 3
            const float2 a0 = v[4 * zk], a1 = v[4 * zk + 1], a2 = v[4 * zk + 2], a3 = v[4 * zk + 3];
            const float2 b0 = make_float2(a0.x + a1.x, a0.y + a1.y), b1 = make_float2(a0.x - a1.x, a0.y - a1.y);
            const float2 b2 = make_float2(a2.x + a3.x, a2.y + a3.y), b3 = make_float2(a2.x - a3.x, a2.y - a3.y);
            v[4 * zk] = make_float2(b0.x + b2.x, b0.y + b2.y);
            v[4 * zk + 1] = make_float2(b1.x + b3.x, b1.y + b3.y);
            v[4 * zk + 2] = make_float2(b0.x - b2.x, b0.y - b2.y);
            v[4 * zk + 3] = make_float2(b1.x - b3.x, b1.y - b3.y);
        }
        const uint32_t x = x0 + xl;
        float2* row = C + ((uint64_t)x << NQ);
        if (in_bounds(st, ((uint64_t)x << NQ) + (1u << NQ) - 1, kElems))
#pragma unroll
            for (int zk = 0; zk < 8; ++zk) {
                const uint32_t z = ((uint32_t)(((warp & 1) << 3) | zk) << 7) | (w << 2);
                rr_put(row, x, z, sg, v[4 * zk], v[4 * zk + 1], scale);
                rr_put(row, x, z + 2, sg, v[4 * zk + 2], v[4 * zk + 3], scale);
            }
    }
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
            if (n >= 9 && n <= 11 && log_r == 13 - n && !(((uintptr_t)A | (uintptr_t)C) & 15)) {
                const float sc = ldexpf(1.0f, -n);
                if (n == 9) rr_item<9>(A, C, (uint32_t)x0, s, sc, st);
                else if (n == 10) rr_item<10>(A, C, (uint32_t)x0, s, sc, st);
                else rr_item<11>(A, C, (uint32_t)x0, s, sc, st);
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
