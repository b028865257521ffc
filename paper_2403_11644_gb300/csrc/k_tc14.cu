// Dense n = 14 decomposition on the tensor cores: complex64 -> complex64 with
// the Hadamard stage of 7 bits run as a dense H_128 (+-1) tcgen05 MMA on bf16
// hi/mid/lo splits of float32 data, accumulated in float32 in tensor memory.
//
// The +-1 matrix is exact in bf16, and x = hi + mid + lo (each bf16, taken
// by successive rounding of the remainder) carries the 24 bits of a float32,
// so H (hi + mid + lo) accumulated in float32 differs from the float32
// transform only by the accumulation rounding.
//
// Same work split as the CUDA-core kernel (clusters of 4 CTAs, an x-block of
// 4 masks, CTA j holding the k-slice j of 4096 values for the 4 masks):
//   gather   2 x 16-byte cp.async per 32-byte tile row (4x4 tiles of A);
//   round 1  k_loc bits 0-4 in registers (lane-XORed reads, sign fix-up);
//   split    each value -> bf16 hi/mid/lo, written as the MMA's B operand
//            B[k7][n] (K = k_loc bits 5-11, N = (mask, z bits 0-4, re/im) = 256,
//            MN-major core matrices of 8 N-contiguous values x 8 K rows);
//   MMA      D[z7][n] += H128[z7][k7] * B_s[k7][n] for s = hi, mid, lo:
//            24 instructions of M=128, N=256, K=16 issued by one thread, D in
//            256 columns of tensor memory;
//   unload   tcgen05.ld D rows (lane = z7) into the exchange layout;
//   final    the 2 cluster bits across the 4 CTAs through distributed shared
//            memory, phase (-i)^{|x&z|}, scale 2^-14, coalesced stores.
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kLog = 14;
constexpr int kN = 1 << kLog;
constexpr int kThreads = 512;
constexpr int kXBlocks = kN / 4;
constexpr int kS2 = 4232;                    // mask row stride of the exchange layout (float2)
constexpr uint32_t kMainBytes = 3u * 65536u; // B operand: 3 splits x 128 x 256 bf16
constexpr uint32_t kHBytes = 32768u;         // H_128 in bf16
constexpr uint32_t kSmemBytes = kMainBytes + kHBytes + 128u; // + alignment slack
constexpr uint32_t kTmemCols = 256;
constexpr int kWaitSpins = 1 << 22;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int pad32(int k) { return k + (k >> 5); }
__device__ __forceinline__ int w2(int m, int kloc) { return m * kS2 + pad32(kloc); }

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
__device__ __forceinline__ float2 ld_cluster(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < kWaitSpins; ++i) {
        uint32_t done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// Shared-memory matrix descriptor (no swizzle): start, leading and stride
// byte offsets in 16-byte units, version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
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

// x = hi + mid + lo, each a bf16 (round to nearest at every step).
__device__ __forceinline__ void split3(float x, uint16_t& hi, uint16_t& mid, uint16_t& lo)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    const __nv_bfloat16 l = __float2bfloat16_rn(r2);
    hi = __bfloat16_as_ushort(h);
    mid = __bfloat16_as_ushort(m);
    lo = __bfloat16_as_ushort(l);
}

#define TC_LD64(r, addr)                                                                              \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 "                                            \
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22," \
                 "%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43," \
                 "%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];" \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),    \
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), \
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),           \
                   "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),           \
                   "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),           \
                   "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]),           \
                   "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]),           \
                   "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),           \
                   "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),           \
                   "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]),           \
                   "=r"(r[62]), "=r"(r[63])                                                                \
                 : "r"(addr))

} // namespace

__global__ void __launch_bounds__(kThreads, 1)
    k_tc14(const float2* __restrict__ A, float2* __restrict__ C, int nclusters, unsigned int* st)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t tmem_slot;
    const uint32_t raw_a = su32(smem_raw);
    const uint32_t main_a = (raw_a + 127u) & ~127u;
    unsigned char* mainp = smem_raw + (main_a - raw_a);
    float2* buf = reinterpret_cast<float2*>(mainp); // tiles, then the exchange layout
    const uint32_t h_a = main_a + kMainBytes;
    uint16_t* hmat = reinterpret_cast<uint16_t*>(mainp + kMainBytes);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t rank = cluster_rank();
    const uint32_t cid = cluster_index();
    const uint32_t bar_a = su32(&bar);

    // H_128 in the K-major core-matrix layout: element (z, k) = (-1)^{|z & k|}.
    for (int e = t; e < 128 * 128; e += kThreads) {
        const int z = e >> 7, k = e & 127;
        hmat[((z >> 3) * 16 + (k >> 3)) * 64 + (z & 7) * 8 + (k & 7)] = (__popc(z & k) & 1) ? 0xBF80u : 0x3F80u;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    uint32_t remote[4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote[s]) : "r"(main_a), "r"(s));

    // M = 128, N = 256, A = bf16 K-major, B = bf16 MN-major, D = f32
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((256u >> 3) << 17) |
                           ((128u >> 4) << 24);
    uint32_t parity = 0;
    bool pending = false;
    const float scale = 1.0f / (float)kN;

    for (uint32_t xb = cid; xb < (uint32_t)kXBlocks; xb += (uint32_t)nclusters) {
        // ---- gather the slice's 1024 tiles (4 rows x 32 bytes each)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int qc = t + kThreads * i;
            const uint32_t tl = (uint32_t)qc >> 3, r = ((uint32_t)qc >> 1) & 3u, hf = (uint32_t)qc & 1u;
            const uint32_t kb = rank * 1024u + tl;
            const uint64_t row = 4ull * (kb ^ xb) + r;
            const uint64_t gi = (row << kLog) + 4ull * kb + 2ull * hf;
            const float2* src = A + (in_bounds(st, gi + 1, (uint64_t)kN * kN) ? gi : 0);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(main_a + (uint32_t)qc * 16u), "l"(src)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncthreads();

        // ---- round 1: k_loc bits 0-4 (see the CUDA-core kernel for the lane XOR)
        const int m = lane & 3, q = lane >> 2, g = warp * 8 + q, c = q & 3;
        float2 v[32];
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
        __syncthreads(); // tiles consumed: the region becomes the B operand

        // ---- split into bf16 hi/mid/lo, B[k7 = g][n = 64 m + 2 z5 + ri]
        {
            const uint32_t row_off = (uint32_t)((g >> 3) * 32) * 128u + (uint32_t)(g & 7) * 16u;
#pragma unroll
            for (int ng = 0; ng < 8; ++ng) { // 4 z5 values x (re, im) per 16-byte row piece
                uint16_t hi[8], mid[8], lo[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    split3(v[4 * ng + u].x, hi[2 * u], mid[2 * u], lo[2 * u]);
                    split3(v[4 * ng + u].y, hi[2 * u + 1], mid[2 * u + 1], lo[2 * u + 1]);
                }
                const uint32_t off = row_off + (uint32_t)(8 * m + ng) * 128u;
                uint4 ph, pm, pl;
                ph.x = hi[0] | ((uint32_t)hi[1] << 16); ph.y = hi[2] | ((uint32_t)hi[3] << 16);
                ph.z = hi[4] | ((uint32_t)hi[5] << 16); ph.w = hi[6] | ((uint32_t)hi[7] << 16);
                pm.x = mid[0] | ((uint32_t)mid[1] << 16); pm.y = mid[2] | ((uint32_t)mid[3] << 16);
                pm.z = mid[4] | ((uint32_t)mid[5] << 16); pm.w = mid[6] | ((uint32_t)mid[7] << 16);
                pl.x = lo[0] | ((uint32_t)lo[1] << 16); pl.y = lo[2] | ((uint32_t)lo[3] << 16);
                pl.z = lo[4] | ((uint32_t)lo[5] << 16); pl.w = lo[6] | ((uint32_t)lo[7] << 16);
                *reinterpret_cast<uint4*>(mainp + off) = ph;
                *reinterpret_cast<uint4*>(mainp + 65536u + off) = pm;
                *reinterpret_cast<uint4*>(mainp + 131072u + off) = pl;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

        // ---- MMA: D = sum over splits and K steps of H128 x B_s
        if (t == 0) {
#pragma unroll 1
            for (int s = 0; s < 3; ++s)
#pragma unroll 1
                for (int kk = 0; kk < 8; ++kk) {
                    const uint64_t da = sdesc(h_a + (uint32_t)kk * 256u, 128u, 2048u);
                    const uint64_t db = sdesc(main_a + (uint32_t)s * 65536u + (uint32_t)kk * 8192u, 4096u, 128u);
                    const uint32_t acc = (s | kk) ? 1u : 0u;
                    asm volatile("{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
                                 ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc)
                                 : "memory");
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                         : "memory");
        }
        if (!mbar_wait(bar_a, parity)) {
            report_status(st, PTDR_ERR_TIMEOUT);
            pending = true;
        }
        parity ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

        // ---- unload D: warp (lane quarter qd, mask mm) -> exchange layout
        {
            const int qd = warp & 3, mm = warp >> 2;
            const int z7 = 32 * qd + lane;
            uint32_t r[64];
            TC_LD64(r, tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(64 * mm));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int z5 = 0; z5 < 32; ++z5)
                buf[w2(mm, z5 | (z7 << 5))] = make_float2(__uint_as_float(r[2 * z5]), __uint_as_float(r[2 * z5 + 1]));
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        cluster_sync();

        // ---- final: the 2 cluster bits, phase, scale, store
        const uint64_t x = 4ull * xb + rank;
        float2* out = C + (x << kLog);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int zl = t + kThreads * i;
            float2 e[4];
#pragma unroll
            for (int src = 0; src < 4; ++src) e[src] = ld_cluster(remote[src] + 8u * (uint32_t)w2((int)rank, zl));
            wht_regs<2>(e);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const uint64_t z = (uint64_t)(zl | (f << 12));
                float2 o;
                switch (__popcll(x & z) & 3) {
                case 0: o = make_float2(e[f].x, e[f].y); break;
                case 1: o = make_float2(e[f].y, -e[f].x); break;
                case 2: o = make_float2(-e[f].x, -e[f].y); break;
                default: o = make_float2(-e[f].y, e[f].x); break;
                }
                o.x *= scale;
                o.y *= scale;
                if (in_bounds(st, (x << kLog) + z, (uint64_t)kN * kN)) __stcs(out + z, o);
            }
        }
        cluster_sync();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // an MMA whose completion was not observed may still be writing tensor memory
    if (pending) mbar_wait(bar_a, parity ^ 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ------------------------------------------------------------------ host

namespace {
std::mutex g_mu;
int g_clusters[128];
} // namespace

bool tc14_supported(const void* A, ptdr_dtype a_t, ptdr_dtype c_t)
{
    return a_t == PTDR_C64 && c_t == PTDR_C64 && ((uintptr_t)A % 16) == 0;
}

cudaError_t launch_tc14(const void* A, void* C, unsigned int* st, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_tc14, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
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
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = s;
    int ncl = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        ncl = g_clusters[dev & 127];
    }
    if (ncl == 0) {
        cfg.gridDim = dim3(4);
        if ((e = cudaOccupancyMaxActiveClusters(&ncl, k_tc14, &cfg)) != cudaSuccess) return e;
        if (ncl < 1) return cudaErrorNotSupported;
        std::lock_guard<std::mutex> lk(g_mu);
        g_clusters[dev & 127] = ncl;
    }
    cfg.gridDim = dim3(4 * ncl);
    e = cudaLaunchKernelEx(&cfg, k_tc14, (const float2*)A, (float2*)C, ncl, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

} // namespace ptdr
