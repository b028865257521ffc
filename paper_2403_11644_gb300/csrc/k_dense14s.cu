// Dense n = 14 and n = 15 decompositions, complex64 -> complex64, FP32
// arithmetic, as two passes over an L2-resident staging buffer with
// contiguous HBM traffic.  (Written out below for n = 14; at n = 15 the
// transform across column blocks has 8 bits, as a 5-bit and a 3-bit register
// round, row items cover 32 of a mask's 128 z_lo values, and three staging
// slots of 32 MiB replace four of 16 MiB.)
//
// The XOR shear d_x[k] = A[k ^ x][k] maps 128 x 128 tiles onto 128 x 128
// tiles: with x = 128 xt + xl and k = 128 cb + cl, the entries of masks
// x in x-tile xt and columns k in column block cb are A[128 (cb ^ xt) + (cl ^ xl)]
// [128 cb + cl], all inside the one tile (R = cb ^ xt, cb) of A, permuted by
// cl ^ xl.  The length-2^14 transform over k splits into 7 bits inside the
// column block (cl) and 7 bits across blocks (cb):
//   pass 1 (tile item):  load the A tile with contiguous 1 KiB rows, transform
//            over cl for its 128 masks, write D'[xl][128 cb + zl] to the
//            staging slot of x-tile xt (16 MiB, stays in L2);
//   pass 2 (row item):   read the staging row of one mask x (128 KiB from L2),
//            transform over cb, apply (-i)^{|x&z|} and 2^-14, write C[x][.]
//            with contiguous stores, and discard the staging lines so the
//            dead intermediate is never written back to HBM.
// HBM sees A read once and C written once, both in whole 1 KiB rows, instead
// of 32-byte pieces from rows 128 KiB apart.  A is loaded with an L2
// evict-first policy so that its lines, read once, leave L2 before the live
// staging does (at n = 15 the staging fills 96 MiB of L2).
//
// Work items are halves (64 KiB each) so that two CTAs share an SM and one
// CTA's loads overlap the other's arithmetic: a half-tile item covers 64 of
// the tile's 128 masks, a half-row item 64 of a row's 128 z_lo values.  An
// item that has read the shared buffer for the last time issues the next
// item's A copies into it (if that item is a tile item) before finishing from
// registers.
//
// One persistent kernel runs both passes from an atomic work queue.  The
// queue order is x-tile major with one tile of look-ahead: round r holds the
// 256 half-tile items of x-tile r, then the 256 half-row items of x-tile r-1.
// A half-row item waits (bounded) until its x-tile's 256 half-tile items are
// done; a half-tile item of x-tile c waits (bounded) before writing until
// x-tile c - kSlots has been read out of the same staging slot.  Every item waited
// on was dequeued earlier by a running CTA, so the waits always end.
#include <mutex>

#include "common.cuh"
#include "pair_ops.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kT = 128;                     // tile edge / masks per x-tile
constexpr int kH = 64;                      // half tile: masks per tile item
constexpr int kThreads = 256;
constexpr int kYaStride = 129;              // pass 1 transpose: 64 rows x 128, padded (float2)
constexpr int kSmemElems = 8448;            // float2: >= 64 x 129 and every row item's 2^RB x (ZL + 1)
constexpr int kSmemBytes = kSmemElems * 8 + 128;

// Sizes for n = LOG (14 or 15).  Row items cover ZL of the 128 z_lo values of
// one mask over all 2^(LOG-7) column blocks (8192 values, 64 KiB, at both n);
// the transform over the column-block bits runs as a 5-bit register round and
// an RB-bit one.
template <int LOG> struct Geo {
    static constexpr int kN = 1 << LOG;
    static constexpr int kTiles = kN / kT;          // x-tiles = column blocks
    static constexpr int kCbBits = LOG - 7;         // transform bits across column blocks
    static constexpr int kRb = kCbBits - 5;         // second-round bits (2 or 3)
    static constexpr int kZl = 8192 >> kCbBits;     // z_lo values per row item (64 or 32)
    static constexpr int kYb = kZl + 1;             // padded row-item transpose stride
    static constexpr int kTileItems = 2 * kTiles;   // half tiles per x-tile
    static constexpr int kRowItems = kT * (kT / kZl);
    static constexpr int kPerRound = kTileItems + kRowItems;
    static constexpr int kItems = (kTiles + 1) * kPerRound;
    static constexpr int kSlots = LOG == 14 ? 4 : 3; // staging slots: 64 MiB (n = 14), 96 MiB (n = 15) of L2
    static_assert((1 << kCbBits) * kYb <= kSmemElems, "row item fits the shared buffer");
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int NB>
__device__ __forceinline__ void wht_regs(float2 (&v)[1 << NB])
{
#pragma unroll
    for (int h = 1; h < (1 << NB); h <<= 1)
#pragma unroll
        for (int i = 0; i < (1 << NB); ++i)
            if (!(i & h)) bfly2(v[i], v[i + h]);
}

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait by thread 0 for *p >= target; records a timeout and gives up
// (the item then runs on whatever the slot holds: no hang, and the status word
// reports the result as invalid).
__device__ __forceinline__ void wait_count(const int* p, int target, unsigned long long limit_ns, unsigned int* st)
{
    const unsigned long long t0 = now_ns();
    while (ld_acquire(p) < target) {
        if (now_ns() - t0 > limit_ns) {
            report_status(st, PTDR_ERR_TIMEOUT);
            return;
        }
        __nanosleep(64);
    }
}

} // namespace

// Issues (one commit group, not waited for) the 16-byte copies of half-tile
// item (xt, cb, h) of the A tile (R = cb ^ xt, cb) into the buffer at buf_a:
// row rl of the tile contributes columns cl with cl bit 6 = (rl bit 6) ^ h,
// one contiguous 512-byte run per row.
template <int LOG>
__device__ __forceinline__ void issue_half_tile(const float2* __restrict__ A, int xt, int cb, int h, uint32_t buf_a,
                                                uint64_t pol_a, unsigned int* st)
{
    constexpr int kN = 1 << LOG;
    const int R = cb ^ xt;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int qc = threadIdx.x + kThreads * i; // 16-byte chunk: row qc >> 5, pair qc & 31
        const int rl = qc >> 5;
        const int b = ((rl >> 6) ^ h) & 1;
        const uint64_t gi = ((uint64_t)(kT * R + rl) << LOG) + (uint64_t)(kT * cb + kH * b) + 2u * (qc & 31);
        const float2* src = A + (in_bounds(st, gi + 1, (uint64_t)kN * kN) ? gi : 0);
        asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(buf_a + (uint32_t)qc * 16u),
                     "l"(src), "l"(pol_a)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

struct StagedTables {
    int* head;  // work-queue counter
    int* done1; // tile items finished per x-tile
    int* done2; // row items finished per x-tile
    float2* stage; // kSlots x 128 rows x 2^14
    unsigned long long wait_ns; // bound of every wait for another CTA
};

template <int LOG>
__global__ void __launch_bounds__(kThreads, 2)
    k_dense_staged(const float2* __restrict__ A, float2* __restrict__ C, StagedTables tab, unsigned int* st)
{
    using G = Geo<LOG>;
    constexpr int kN = G::kN, kTiles = G::kTiles, kPerRound = G::kPerRound, kItems = G::kItems,
                  kSlots = G::kSlots, kZl = G::kZl, kYb = G::kYb, kRb = G::kRb;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_item, s_next;
    const uint32_t raw_a = su32(smem_raw);
    const uint32_t buf_a = (raw_a + 127u) & ~127u;
    float2* buf = reinterpret_cast<float2*>(smem_raw + (buf_a - raw_a));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float scale = 1.0f / (float)kN;
    uint64_t pol_a; // A is read once: its lines go first, ahead of live staging
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_a));

    // thread 0 keeps the next item in hand so the queue's atomic latency
    // overlaps the current item (a held item is always later in the queue
    // than the one being processed, so the dependency waits still end)
    int next = 0;
    if (t == 0) next = atomicAdd(tab.head, 1);
    bool issued = false; // this item's A copies were issued by the previous item
    // once an item has read the shared buffer for the last time, the next item's
    // A copies (if it is a tile item) go into it while this item finishes from
    // registers; every thread calls it at the same point
    auto prefetch_next = [&]() {
        if (t == 0) s_next = next;
        __syncthreads();
        const int nx = s_next;
        bool go = false;
        if (nx < kItems) {
            const int nr = nx / kPerRound, nj = nx % kPerRound;
            if (nj < G::kTileItems && nr < kTiles) {
                issue_half_tile<LOG>(A, nr, nj >> 1, nj & 1, buf_a, pol_a, st);
                go = true;
            }
        }
        return go;
    };
    for (;;) {
        if (t == 0) {
            s_item = next;
            if (next < kItems) next = atomicAdd(tab.head, 1);
        }
        __syncthreads();
        const int item = s_item;
        if (item >= kItems) break;
        const int r = item / kPerRound, j = item % kPerRound;

        if (j < G::kTileItems) {
            // ------------------------------------------------ half-tile item
            // masks xl in [64 h, 64 h + 64) of x-tile xt, column block cb.
            // Row rl of the A tile contributes columns cl with cl bit 6 =
            // (rl bit 6) ^ h: one contiguous 512-byte run per row.
            const int xt = r, cb = j >> 1, h = j & 1;
            if (xt >= kTiles) { __syncthreads(); continue; }
            if (!issued) issue_half_tile<LOG>(A, xt, cb, h, buf_a, pol_a, st);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            // round a: cl bits 0-4.  Lane l of warp w handles mask xl = 64 h + 32 (w & 1) + l
            // and column group g = w >> 1; at step s it reads cl = 32 g + (s ^ l), so all
            // lanes read the same tile row at distinct columns; the register transform
            // then carries the sign (-1)^{|z & l|}.
            const int xloc = 32 * (warp & 1) + lane, xl = kH * h + xloc, g = warp >> 1;
            float2 v[32];
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const int cl = 32 * g + (s ^ lane);
                v[s] = buf[(cl ^ xl) * kH + (cl & (kH - 1))];
            }
            wht_regs<5>(v);
#pragma unroll
            for (int z = 0; z < 32; ++z)
                if (__popc(z & lane) & 1) v[z] = make_float2(-v[z].x, -v[z].y);
            __syncthreads();
#pragma unroll
            for (int z = 0; z < 32; ++z) buf[xloc * kYaStride + 32 * g + z] = v[z];
            __syncthreads();
            // round b: cl bits 5-6; lane = z5, rows 8 w + i of the half tile
            if (t == 0 && xt >= kSlots) wait_count(tab.done2 + (xt - kSlots), G::kRowItems, tab.wait_ns, st);
            __syncthreads();
            float2* stage = tab.stage + ((size_t)(xt % kSlots) * kT + kH * h) * kN;
            float2 e[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int gg = 0; gg < 4; ++gg) e[i][gg] = buf[(8 * warp + i) * kYaStride + 32 * gg + lane];
            issued = prefetch_next();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int row = 8 * warp + i;
                wht_regs<2>(e[i]);
#pragma unroll
                for (int gg = 0; gg < 4; ++gg)
                    __stcg(stage + (size_t)row * kN + kT * cb + 32 * gg + lane, e[i][gg]);
            }
            __syncthreads();
            if (t == 0) {
                __threadfence();
                atomicAdd(tab.done1 + xt, 1);
            }
        } else {
            // ------------------------------------------------ row item
            // mask xl of x-tile xt, output columns z_lo in [ZL h, ZL h + ZL) over all
            // 2^(LOG-7) column blocks
            const int jj = j - G::kTileItems;
            const int xt = r - 1, xl = jj / (kT / kZl), h = jj % (kT / kZl);
            if (xt < 0) { __syncthreads(); continue; }
            if (t == 0) wait_count(tab.done1 + xt, G::kTileItems, tab.wait_ns, st);
            __syncthreads();
            const uint64_t x = (uint64_t)(kT * xt + xl);
            const float2* srow = tab.stage + ((size_t)(xt % kSlots) * kT + xl) * kN + kZl * h;
            // round a: cb bits 0-4; lanes take consecutive z_lo (coalesced L2 reads)
            const int zloc = t % kZl, q = t / kZl;
            float2 v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = __ldcg(srow + (size_t)(32 * q + i) * kT + zloc);
            wht_regs<5>(v);
#pragma unroll
            for (int i = 0; i < 32; ++i) buf[(32 * q + i) * kYb + zloc] = v[i];
            __syncthreads();
            // this item's part of the staging row is consumed: drop its lines from
            // L2 without write-back (kZl * 8 / 128 lines of 128 bytes per column block)
            {
                constexpr int kLinesPerCb = kZl / 16, kLines = kTiles * kLinesPerCb;
#pragma unroll
                for (int i = 0; i < kLines / kThreads; ++i) {
                    const int ln = t + kThreads * i;
                    const float2* p = srow + (size_t)(ln / kLinesPerCb) * kT + 16 * (ln % kLinesPerCb);
                    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
                }
            }
            // round b: cb bits 5 .. LOG-8, then phase, scale and contiguous stores
            constexpr int kPb = kZl / 8; // (c5, z_lo) pairs per thread: 32 kZl / 256
            float2* out = C + (x << LOG) + kZl * h;
            float2 eb[kPb][1 << kRb];
#pragma unroll
            for (int i = 0; i < kPb; ++i)
#pragma unroll
                for (int gg = 0; gg < (1 << kRb); ++gg) eb[i][gg] = buf[(32 * gg + kPb * q + i) * kYb + zloc];
            issued = prefetch_next();
#pragma unroll
            for (int i = 0; i < kPb; ++i) {
                const int c5 = kPb * q + i;
                float2 (&e)[1 << kRb] = eb[i];
                wht_regs<kRb>(e);
#pragma unroll
                for (int gg = 0; gg < (1 << kRb); ++gg) {
                    const uint64_t zoff = (uint64_t)(kT * (32 * gg + c5) + zloc);
                    const uint64_t z = zoff + (uint64_t)(kZl * h);
                    const float2 w = e[gg];
                    const float2 o = phase_neg_i(w, (int)(__popcll(x & z) & 3), scale);
                    if (in_bounds(st, (x << LOG) + z, (uint64_t)kN * kN)) __stcs(out + zoff, o);
                }
            }
            __syncthreads();
            if (t == 0) {
                __threadfence();
                atomicAdd(tab.done2 + xt, 1);
            }
        }
    }
}

// ------------------------------------------------------------------ host

size_t dense_staged_workspace(int n)
{
    // counters (head, done1[x-tiles], done2[x-tiles]) padded to 4 KiB, then the slots:
    // 4 x 16 MiB at n = 14, 3 x 32 MiB at n = 15
    return n == 14 ? 4096 + (size_t)Geo<14>::kSlots * kT * Geo<14>::kN * sizeof(float2)
                   : 4096 + (size_t)Geo<15>::kSlots * kT * Geo<15>::kN * sizeof(float2);
}

template <int LOG>
static cudaError_t run_staged(const void* A, void* C, void* ws, unsigned int* st, cudaStream_t s)
{
    static std::mutex mu;
    static int grid_for[128];
    auto kern = k_dense_staged<LOG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        grid = grid_for[dev & 127];
    }
    if (grid == 0) {
        int sms = 0, per = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, kSmemBytes)) != cudaSuccess)
            return e;
        grid = sms * (per > 0 ? per : 1);
        std::lock_guard<std::mutex> lk(mu);
        grid_for[dev & 127] = grid;
    }
    char* w = (char*)ws;
    StagedTables tab;
    tab.head = (int*)w;
    tab.done1 = (int*)(w + 64);
    tab.done2 = (int*)(w + 64 + 4 * Geo<LOG>::kTiles);
    tab.stage = (float2*)(w + 4096);
    tab.wait_ns = wait_limit_ns();
    if ((e = cudaMemsetAsync(ws, 0, 4096, s)) != cudaSuccess) return e;
    kern<<<grid, kThreads, kSmemBytes, s>>>((const float2*)A, (float2*)C, tab, st);
    return cudaGetLastError();
}

cudaError_t launch_dense_staged(int n, const void* A, void* C, void* ws, unsigned int* st, cudaStream_t s)
{
    if (n == 14) return run_staged<14>(A, C, ws, st, s);
    if (n == 15) return run_staged<15>(A, C, ws, st, s);
    return cudaErrorInvalidValue;
}

} // namespace ptdr
