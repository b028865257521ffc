// Dense n = 14 compose (the inverse map A = scale * sum_P c_P P), complex64 ->
// complex64, FP32 arithmetic, as two passes over an L2-resident staging
// buffer: the mirror of the staged decompose.
//
// Per mask x the inverse is f_x[k] = scale * sum_z (-1)^{|z&k|} i^{|x&z|} C[x][z]
// and A[k ^ x][k] = f_x[k].  With x = 128 xt + xl, z = 128 zb + zl and
// k = 128 cb + cl the length-2^14 transform splits into the 7 bits across
// blocks (zb -> cb) and the 7 bits inside a block (zl -> cl):
//   pass 1 (half-row item: mask x, zl in [64 h, 64 h + 64)): read C[x][128 zb + zl]
//            for every zb (512-byte runs), apply scale * i^{|x&z|}, transform over zb,
//            write S[xl][128 cb + zl] to the staging slot of x-tile xt (16 MiB,
//            stays in L2);
//   pass 2 (half-tile item: x-tile xt, column block cb, masks xl in [64 h, 64 h + 64)):
//            read S[xl][128 cb + .] (1 KiB rows), transform over zl, and write
//            A[128 (cb ^ xt) + (cl ^ xl)][128 cb + cl]: for each of the 128 rows r of
//            the A tile, the 64 columns cl whose bit 6 is (r bit 6) ^ h (512-byte
//            runs).  The consumed staging lines are discarded from L2.
// HBM sees C read once and A written once, in whole 512-byte runs.
//
// One persistent kernel (3 CTAs of 256 threads per SM) takes items from an
// atomic queue in x-tile-major rounds: round r holds the 256 half-row items of
// x-tile r, then the 256 half-tile items of x-tile r - 1.  A half-tile item
// waits (bounded) until its x-tile's 256 half-row items are done; a half-row
// item of x-tile c waits (bounded) before writing until x-tile c - kSlots has
// been read out of the same staging slot.  Every item waited on was dequeued
// earlier by a running CTA, so the waits end.
#include <mutex>

#include "common.cuh"
#include "pair_ops.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kLog = 14;
constexpr int kN = 1 << kLog;
constexpr int kT = 128;                    // block edge / masks per x-tile
constexpr int kH = 64;                     // half: zl values (pass 1) or masks (pass 2) per item
constexpr int kTiles = kN / kT;            // 128 x-tiles, 128 column blocks
constexpr int kThreads = 256;
constexpr int kSlots = 4;                  // staging slots (x-tiles in flight)
constexpr int kRowStride = 65;             // pass 1 buffer: 128 zb x 64 zl, padded (float2)
constexpr int kTileStride = 129;           // pass 2 buffer: 64 masks x 128 zl, padded (float2)
constexpr int kSmemElems = kT * kRowStride; // 8320 float2 >= 64 x 129 and the 128 x 64 A tile
constexpr int kSmemBytes = kSmemElems * 8 + 128;
constexpr int kPerRound = 4 * kT;          // 256 half-row items + 256 half-tile items
constexpr int kItems = (kTiles + 1) * kPerRound;
constexpr int kDone = 2 * kT;              // items per x-tile and pass

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

// Bounded wait by one thread for *p >= target; records a timeout and gives up.
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

struct ComposeTables {
    int* head;     // work-queue counter
    int* done1;    // half-row items finished per x-tile
    int* done2;    // half-tile items finished per x-tile
    float2* stage; // kSlots x 128 rows x 2^14
    unsigned long long wait_ns; // bound of every wait for another CTA
};

__global__ void __launch_bounds__(kThreads, 3)
    k_compose14_staged(const float2* __restrict__ C, float2* __restrict__ A, float scale, ComposeTables tab,
                       unsigned int* st)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_item;
    float2* buf = reinterpret_cast<float2*>(smem_raw + ((128u - ((uintptr_t)smem_raw & 127u)) & 127u));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint64_t lim = (uint64_t)kN * kN;

    int next = 0;
    if (t == 0) next = atomicAdd(tab.head, 1);
    for (;;) {
        if (t == 0) {
            s_item = next;
            if (next < kItems) next = atomicAdd(tab.head, 1);
        }
        __syncthreads();
        const int item = s_item;
        if (item >= kItems) break;
        const int r = item / kPerRound, j = item % kPerRound;

        if (j < 2 * kT) {
            // ------------------------------------------------ half-row item
            // mask xl of x-tile xt, zl in [64 h, 64 h + 64)
            const int xt = r, xl = j >> 1, h = j & 1;
            if (xt >= kTiles) { __syncthreads(); continue; }
            const uint64_t x = (uint64_t)(kT * xt + xl);
            // C[x][128 zb + 64 h + .] for every zb -> buf[zb][64] (dense 512-byte rows), by
            // 16-byte asynchronous copies: 16 per thread in flight
            const float2* crow = C + (x << kLog) + kH * h;
            const uint32_t buf_a = (uint32_t)__cvta_generic_to_shared(buf);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int qc = t + kThreads * i; // 4096 pieces: row qc >> 5, pair qc & 31
                const uint64_t gi = (x << kLog) + (uint64_t)(kT * (qc >> 5) + kH * h + 2 * (qc & 31));
                const float2* src = crow + (size_t)kT * (qc >> 5) + 2 * (qc & 31);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(buf_a + 16u * (uint32_t)qc),
                             "l"(in_bounds(st, gi + 1, lim) ? src : C)
                             : "memory");
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            // round a: zb bits 0-4 in registers; lanes take consecutive zl
            const int zloc = 32 * (warp & 1) + lane, q = warp >> 1;
            float2 v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const uint64_t z = (uint64_t)kT * (32 * q + i) + (uint64_t)(kH * h + zloc);
                // i^p = (-i)^{(4 - p) mod 4}
                v[i] = phase_neg_i(buf[(32 * q + i) * kH + zloc], (int)((4u - (__popcll(x & z) & 3u)) & 3u), scale);
            }
            wht_regs<5>(v);
            __syncthreads(); // every row of buf has been read: round a's results go back padded
#pragma unroll
            for (int i = 0; i < 32; ++i) buf[(32 * q + i) * kRowStride + zloc] = v[i];
            // the staging slot is free once x-tile xt - kSlots has been read from it
            if (t == 0 && xt >= kSlots) wait_count(tab.done2 + (xt - kSlots), kDone, tab.wait_ns, st);
            __syncthreads();
            // round b: zb bits 5-6, then contiguous staging stores S[xl][128 cb + zl]
            float2* srow = tab.stage + ((size_t)(xt % kSlots) * kT + xl) * kN + kH * h + zloc;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c5 = 8 * q + i;
                float2 e[4];
#pragma unroll
                for (int gg = 0; gg < 4; ++gg) e[gg] = buf[(32 * gg + c5) * kRowStride + zloc];
                wht_regs<2>(e);
#pragma unroll
                for (int gg = 0; gg < 4; ++gg) __stcg(srow + (size_t)kT * (32 * gg + c5), e[gg]);
            }
            __syncthreads();
            if (t == 0) {
                __threadfence();
                atomicAdd(tab.done1 + xt, 1);
            }
        } else {
            // ------------------------------------------------ half-tile item
            // x-tile xt, column block cb, masks xl in [64 h, 64 h + 64)
            const int jj = j - 2 * kT;
            const int xt = r - 1, cb = jj >> 1, h = jj & 1;
            if (xt < 0) { __syncthreads(); continue; }
            if (t == 0) wait_count(tab.done1 + xt, kDone, tab.wait_ns, st);
            __syncthreads();
            const int R = cb ^ xt;
            // staging rows xl = 64 h + row, columns 128 cb .. 128 cb + 127, straight into
            // registers (coalesced 256-byte L2 reads, 32 in flight per thread): thread =
            // (row 8 w + i, zl bits 0-4 = lane); zl bits 5-6 transformed there, then buf[row][zl]
            const float2* sblk = tab.stage + ((size_t)(xt % kSlots) * kT + kH * h) * kN + (size_t)kT * cb;
            {
                float2 e[8][4];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int gg = 0; gg < 4; ++gg)
                        e[i][gg] = __ldcg(sblk + (size_t)(8 * warp + i) * kN + 32 * gg + lane);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    wht_regs<2>(e[i]);
#pragma unroll
                    for (int gg = 0; gg < 4; ++gg) buf[(8 * warp + i) * kTileStride + 32 * gg + lane] = e[i][gg];
                }
            }
            __syncthreads();
            // the 64 staging rows of this block are consumed: drop their lines from L2
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int ln = t + kThreads * i; // 512 lines of 128 bytes
                const float2* p = sblk + (size_t)(ln >> 3) * kN + 16 * (ln & 7);
                asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
            }
            // zl bits 0-4 in registers: thread = (mask xloc = 32 (w & 1) + l, group g = w >> 1).
            // Multiplying input s by (-1)^{|l & s|} before the transform leaves register c
            // holding output cl = 32 g + (c ^ l), so that for each c the 32 lanes of the warp
            // write one row (cl ^ xl has low bits c) of the A tile at 32 distinct columns.
            const int xloc = 32 * (warp & 1) + lane, g = warp >> 1;
            float2 v[32];
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const float2 w = buf[xloc * kTileStride + 32 * g + s];
                const uint32_t sg = (uint32_t)(__popc(lane & s) & 1) << 31;
                v[s] = make_float2(__uint_as_float(__float_as_uint(w.x) ^ sg), __uint_as_float(__float_as_uint(w.y) ^ sg));
            }
            wht_regs<5>(v);
            __syncthreads();
            // A tile half in shared memory: row rr (0..127), column c6 = cl & 63 (dense rows)
            const int xl = kH * h + xloc;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int cl = 32 * g + (c ^ lane);
                buf[((cl ^ xl) & (kT - 1)) * kH + (cl & (kH - 1))] = v[c];
            }
            __syncthreads();
            // contiguous 16-byte stores: row rr holds columns cl with bit 6 = (rr bit 6) ^ h
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int e = t + kThreads * i; // 4096 pairs: row e >> 5, pair e & 31
                const int rr = e >> 5, pr = e & 31;
                const int b = ((rr >> 6) ^ h) & 1;
                const uint64_t gi = ((uint64_t)(kT * R + rr) << kLog) + (uint64_t)(kT * cb + kH * b + 2 * pr);
                const float4 val = *reinterpret_cast<const float4*>(buf + rr * kH + 2 * pr);
                if (in_bounds(st, gi + 1, lim)) __stcs(reinterpret_cast<float4*>(A + gi), val);
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

size_t compose14_staged_workspace()
{
    // counters (head, done1[128], done2[128]) padded to 4 KiB, then the slots
    return 4096 + (size_t)kSlots * kT * kN * sizeof(float2);
}

cudaError_t launch_compose14_staged(const void* C, void* A, double scale, void* ws, unsigned int* st, cudaStream_t s)
{
    static std::mutex mu;
    static int grid_for[128];
    cudaError_t e = cudaFuncSetAttribute(k_compose14_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
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
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_compose14_staged, kThreads, kSmemBytes)) !=
            cudaSuccess)
            return e;
        grid = sms * (per > 0 ? per : 1);
        std::lock_guard<std::mutex> lk(mu);
        grid_for[dev & 127] = grid;
    }
    char* w = (char*)ws;
    ComposeTables tab;
    tab.head = (int*)w;
    tab.done1 = (int*)(w + 64);
    tab.done2 = (int*)(w + 64 + 4 * kTiles);
    tab.stage = (float2*)(w + 4096);
    tab.wait_ns = wait_limit_ns();
    if ((e = cudaMemsetAsync(ws, 0, 4096, s)) != cudaSuccess) return e;
    k_compose14_staged<<<grid, kThreads, kSmemBytes, s>>>((const float2*)C, (float2*)A, (float)scale, tab, st);
    return cudaGetLastError();
}

} // namespace ptdr
