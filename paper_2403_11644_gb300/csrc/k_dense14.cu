// Dense n = 14 decomposition, complex64 -> complex64, FP32 arithmetic:
// clusters of 4 CTAs, sector-wide asynchronous tile gathers, register radix
// rounds, and an exchange of the last two bits through a small L2-resident
// scratch that lets the next gather overlap the current exchange.
//
// Work unit: an x-block of 4 masks x = 4 xb + x_lo (xb = 0..4095).  For a
// block of 4 rows R and 4 columns kb with R ^ kb = xb, the 4x4 tile of A holds
// d_x[k] for all 4 masks and the 4 columns k = 4 kb + t: element (r, t) is
// d_{4 xb + (r ^ t)}[4 kb + t].  Each row of the tile is one 32-byte sector,
// so the whole x-block reads A's 32-byte sectors exactly once: two 16-byte
// cp.async copies per tile row, 16 rows per warp instruction.  (One TMA box
// per tile would also work, but 16.8M boxes of 128 bytes run far below the
// copy engine's byte rate; the load/store units sustain the row rate.)
//
// CTA j of the cluster gathers the 1024 tiles with kb in [1024 j, 1024 j + 1024),
// i.e. k in a slice of 4096 values for all 4 masks (128 KiB), and transforms
// 10 of the 12 slice-local bits of k in two register rounds of 5 bits.  Round
// 2 leaves the values in registers, so the shared buffer is free and the next
// x-block's gather is issued at that point.  The values then go out: the
// quarter of mask 4 xb + j stays in shared memory, the other three quarters
// go to the cluster's scratch in global memory (L2-resident, double-buffered
// by x-block parity).  After a cluster barrier (release/acquire), CTA j reads
// its mask's quarters from the other three CTAs, runs the last 4 bits (2
// local + 2 across the cluster), applies (-i)^{|x&z|} and 2^-14 and writes the
// output row with coalesced streaming stores.  (Distributed shared memory
// would carry the same exchange, but it holds the buffer until every peer
// has read it, which serialises gather and exchange; it also measured at
// about a quarter of the L2 read rate per SM.)
//
// Persistent: one cluster per 4 SMs stays resident and walks x-blocks.
#include <mutex>

#include "common.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kLog = 14;
constexpr int kN = 1 << kLog;
constexpr int kThreads = 512;
constexpr int kXBlocks = kN / 4;
constexpr int kMaxClusters = 64;            // scratch is sized for this many resident clusters
constexpr int kS1 = 4228;                  // mask row stride of the round-1 layout (float2)
constexpr int kMainElems = 4 * kS1;        // float2: tiles, then the round-1 layout
constexpr int kBufBytes = (kMainElems + 4096) * 8 + 128; // + own quarter + alignment slack

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int pad32(int k) { return k + (k >> 5); }
// layout after round 1: [mask][k_loc], one pad element per 32 and a mask row
// stride that keeps round 1's stores and round 2's loads at two wavefronts
__device__ __forceinline__ int w1(int m, int kloc) { return m * kS1 + pad32(kloc); }

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_index()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int NB>
__device__ __forceinline__ void wht_regs(float2 (&v)[1 << NB])
{
#pragma unroll
    for (int h = 1; h < (1 << NB); h <<= 1)
#pragma unroll
        for (int i = 0; i < (1 << NB); ++i)
            if (!(i & h)) {
                float2 a = v[i], b = v[i + h];
                v[i] = make_float2(a.x + b.x, a.y + b.y);
                v[i + h] = make_float2(a.x - b.x, a.y - b.y);
            }
}

} // namespace

__device__ __forceinline__ void gather_slice(const float2* __restrict__ A, uint32_t buf_a, uint32_t rank,
                                             uint32_t xb, int t, unsigned int* st)
{
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int qc = t + kThreads * i; // 16-byte chunk of the slice
        const uint32_t tl = (uint32_t)qc >> 3, r = ((uint32_t)qc >> 1) & 3u, hf = (uint32_t)qc & 1u;
        const uint32_t kb = rank * 1024u + tl;
        const uint64_t row = 4ull * (kb ^ xb) + r;
        const uint64_t gi = (row << kLog) + 4ull * kb + 2ull * hf; // complex index
        const float2* src = A + (in_bounds(st, gi + 1, (uint64_t)kN * kN) ? gi : 0);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(buf_a + (uint32_t)qc * 16u), "l"(src)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    k_dense14_x4(const float2* __restrict__ A, float2* __restrict__ C, float2* __restrict__ scratch,
                 int nclusters, unsigned int* st)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t raw_a = su32(smem_raw);
    const uint32_t buf_a = (raw_a + 127u) & ~127u; // 16-byte copies land 128-byte aligned
    float2* buf = reinterpret_cast<float2*>(smem_raw + (buf_a - raw_a));
    float2* loc = buf + kMainElems; // this CTA's own mask quarter after round 2
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t rank = cluster_rank();
    const uint32_t cid = cluster_index();
    const float scale = 1.0f / (float)kN;
    // scratch[cluster][parity][source rank][mask][4096]
    float2* my_scratch = scratch + (size_t)cid * (2u * 16u * 4096u);

    uint32_t xb = cid;
    if (xb < (uint32_t)kXBlocks) gather_slice(A, buf_a, rank, xb, t, st);
    for (uint32_t it = 0; xb < (uint32_t)kXBlocks; xb += (uint32_t)nclusters, ++it) {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();

        // ---- round 1: k_loc bits 0-4; lane (m, q) reads element i = s ^ (q & 3)
        // of its group so that the 32 lanes hit 16 distinct (row, col) slots of
        // the tiles; the register transform then carries the sign (-1)^{|z & c|}.
        const int m = lane & 3;
        float2 v[32];
        {
            const int q = lane >> 2, g = warp * 8 + q, c = q & 3;
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const int i = s ^ c;
                const int tt = i & 3;
                v[s] = buf[(8 * g + (i >> 2)) * 16 + (m ^ tt) * 4 + tt];
            }
            wht_regs<5>(v);
#pragma unroll
            for (int z = 0; z < 32; ++z)
                if (__popc(z & c) & 1) v[z] = make_float2(-v[z].x, -v[z].y);
            __syncthreads();
#pragma unroll
            for (int z = 0; z < 32; ++z) buf[w1(m, 32 * g + z)] = v[z];
        }
        __syncthreads();

        // ---- round 2: k_loc bits 5-9, one mask per warp.  Once every thread
        // holds its values the buffer is free and the next x-block's gather
        // starts underneath.
        const int m2 = warp & 3;
        const int kbase = lane | ((warp >> 2) << 10);
#pragma unroll
        for (int s = 0; s < 32; ++s) v[s] = buf[w1(m2, kbase | (s << 5))];
        __syncthreads();
        if (xb + (uint32_t)nclusters < (uint32_t)kXBlocks)
            gather_slice(A, buf_a, rank, xb + (uint32_t)nclusters, t, st);
        wht_regs<5>(v);
        if ((uint32_t)m2 == rank) {
#pragma unroll
            for (int s = 0; s < 32; ++s) loc[kbase | (s << 5)] = v[s];
        } else {
            float2* out_q = my_scratch + ((size_t)((it & 1u) * 4u + rank) * 4u + (uint32_t)m2) * 4096u;
#pragma unroll
            for (int s = 0; s < 32; ++s) __stcg(out_q + (kbase | (s << 5)), v[s]);
        }
        cluster_sync(); // release this slice's quarters; acquire the others'

        // ---- final: k_loc bits 10-11 and the 2 cluster bits, then write out
        const uint64_t x = 4ull * xb + rank;
        float2* row = C + (x << kLog);
        const float2* in_base = my_scratch + (size_t)((it & 1u) * 16u + rank) * 4096u; // [src = 0][mask = rank]
        float2 e[2][16];
#pragma unroll
        for (int half = 0; half < 2; ++half)
#pragma unroll
            for (int src = 0; src < 4; ++src)
#pragma unroll
                for (int c2 = 0; c2 < 4; ++c2) {
                    const int kl = (c2 << 10) | (t + 512 * half);
                    e[half][c2 | (src << 2)] =
                        ((uint32_t)src == rank) ? loc[kl] : __ldcg(in_base + src * 4 * 4096 + kl);
                }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int zp = t + 512 * half;
            wht_regs<4>(e[half]);
#pragma unroll
            for (int f = 0; f < 16; ++f) {
                const uint64_t z = (uint64_t)(zp | (f << 10));
                const float2 w = e[half][f];
                float2 o;
                switch (__popcll(x & z) & 3) {
                case 0: o = make_float2(w.x, w.y); break;
                case 1: o = make_float2(w.y, -w.x); break;
                case 2: o = make_float2(-w.x, -w.y); break;
                default: o = make_float2(-w.y, w.x); break;
                }
                o.x *= scale;
                o.y *= scale;
                if (in_bounds(st, (x << kLog) + z, (uint64_t)kN * kN)) __stcs(row + z, o);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ------------------------------------------------------------------ host

namespace {

std::mutex g_mu;
int g_clusters[128];

} // namespace

bool dense14_x4_supported(const void* A, ptdr_dtype a_t, ptdr_dtype c_t)
{
    return a_t == PTDR_C64 && c_t == PTDR_C64 && ((uintptr_t)A % 16) == 0;
}

size_t dense14_x4_workspace() { return (size_t)kMaxClusters * 2u * 16u * 4096u * sizeof(float2); }

cudaError_t launch_dense14_x4(const void* A, void* C, void* ws, unsigned int* st, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_dense14_x4, cudaFuncAttributeMaxDynamicSharedMemorySize, kBufBytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 4;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kBufBytes;
    cfg.stream = s;
    int ncl = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        ncl = g_clusters[dev & 127];
    }
    if (ncl == 0) {
        cfg.gridDim = dim3(4);
        if ((e = cudaOccupancyMaxActiveClusters(&ncl, k_dense14_x4, &cfg)) != cudaSuccess) return e;
        if (ncl < 1) return cudaErrorNotSupported;
        ncl = ncl > kMaxClusters ? kMaxClusters : ncl;
        std::lock_guard<std::mutex> lk(g_mu);
        g_clusters[dev & 127] = ncl;
    }
    cfg.gridDim = dim3(4 * ncl);
    e = cudaLaunchKernelEx(&cfg, k_dense14_x4, (const float2*)A, (float2*)C, (float2*)ws, ncl, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

} // namespace ptdr
