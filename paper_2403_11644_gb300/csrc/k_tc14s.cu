// Dense n = 14 decomposition with the Hadamard stage over the column blocks
// on the tensor cores (split-bf16 path): complex64 -> complex64.
//
// Same two passes over an L2-resident staging buffer as the CUDA-core kernel
// (the XOR shear maps 128 x 128 tiles of A onto tiles; k = 128 cb + cl):
//   pass 1 (tile item, CUDA cores): load the A tile with contiguous 1 KiB
//            rows, transform over cl (7 bits) for its 128 masks in registers
//            (the XOR-permuted gather needs a per-lane register order that an
//            MMA operand cannot express), write D'[xl][128 cb + zl] to staging;
//   pass 2 (row item, tensor cores): the staging row of mask x, read as
//            B[cb][2 zl + ri] (K = cb, N = 256 real columns, MN-major core
//            matrices), split into bf16 hi/mid/lo; one thread issues
//            D[zb][n] = sum_s H128[zb][cb] B_s[cb][n] as 24 tcgen05.mma of
//            M = 128, N = 256, K = 16 with D (float32) in tensor memory; the
//            epilogue unloads D through shared memory into contiguous stores
//            of C[x][128 zb + zl] with the phase (-i)^{|x&z|} and 2^-14.
// The +-1 matrix is exact in bf16 and hi + mid + lo carries the 24 bits of a
// float32, so the tensor-core stage differs from float32 arithmetic only by
// the accumulation rounding.  Staging lines are discarded once read.
//
// One persistent CTA per SM (the pass-2 operands fill shared memory), work
// from the same ordered atomic queue with bounded dependency waits.
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kLog = 14;
constexpr int kN = 1 << kLog;
constexpr int kT = 128;
constexpr int kTiles = kN / kT;
constexpr int kThreads = 512;
constexpr int kSlots = 4;
constexpr int kY = 129;                        // padded row stride of the transposes (float2)
constexpr uint32_t kOpBytes = 3u * 65536u;     // B operand: 3 splits x 128 x 256 bf16
constexpr uint32_t kHBytes = 32768u;           // H_128 in bf16
constexpr uint32_t kSmemBytes = kOpBytes + kHBytes + 128u;
constexpr uint32_t kTmemCols = 256;
constexpr long long kSpinLimit = 1ll << 24;
constexpr int kWaitSpins = 1 << 22;
constexpr int kPerRound = 2 * kT;
constexpr int kItems = (kTiles + 1) * kPerRound;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void wait_count(const int* p, int target, unsigned int* st)
{
    long long spins = 0;
    while (ld_acquire(p) < target) {
        if (++spins > kSpinLimit) {
            report_status(st, PTDR_ERR_TIMEOUT);
            return;
        }
        __nanosleep(64);
    }
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

// Shared-memory matrix descriptor without swizzle (version 1).  K-major:
// lbo = K-direction core-matrix stride, sbo = M/N-direction stride.
// MN-major: lbo = K-direction stride, sbo = M/N-direction stride as well
// (both checked against a CPU product on the GPU before use).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) { return (uint32_t)a | ((uint32_t)b << 16); }

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

struct TcStagedTables {
    int* head;
    int* done1;
    int* done2;
    float2* stage; // kSlots x 128 rows x 2^14
};

__global__ void __launch_bounds__(kThreads, 1)
    k_tc14_staged(const float2* __restrict__ A, float2* __restrict__ C, TcStagedTables tab, unsigned int* st)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_item;
    const uint32_t raw_a = su32(smem_raw);
    const uint32_t op_a = (raw_a + 127u) & ~127u;
    unsigned char* opp = smem_raw + (op_a - raw_a);
    float2* buf = reinterpret_cast<float2*>(opp); // pass-1 tile / transposes / epilogue staging
    const uint32_t h_a = op_a + kOpBytes;
    uint16_t* hmat = reinterpret_cast<uint16_t*>(opp + kOpBytes);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t bar_a = su32(&bar);
    const float scale = 1.0f / (float)kN;

    // H_128, K-major core matrices: element (zb, cb) = (-1)^{|zb & cb|}
    for (int e = t; e < kT * kT; e += kThreads) {
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
    // M = 128, N = 256, A = bf16 K-major, B = bf16 MN-major, D = f32
    const uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
    uint32_t parity = 0;
    bool pending = false;

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

        if (j < kT) {
            // ------------------------------------------------ tile item (CUDA cores)
            const int xt = r, cb = j;
            if (xt >= kTiles) { __syncthreads(); continue; }
            const int R = cb ^ xt;
            const uint32_t buf_a = op_a;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int qc = t + kThreads * i;
                const uint64_t gi = ((uint64_t)(kT * R + (qc >> 6)) << kLog) + (uint64_t)(kT * cb) + 2u * (qc & 63);
                const float2* src = A + (in_bounds(st, gi + 1, (uint64_t)kN * kN) ? gi : 0);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(buf_a + (uint32_t)qc * 16u), "l"(src)
                             : "memory");
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            const int xl = 32 * (warp & 3) + lane, g = warp >> 2;
            float2 v[32];
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const int cl = 32 * g + (s ^ lane);
                v[s] = buf[(cl ^ xl) * kT + cl];
            }
            wht_regs<5>(v);
#pragma unroll
            for (int z = 0; z < 32; ++z)
                if (__popc(z & lane) & 1) v[z] = make_float2(-v[z].x, -v[z].y);
            __syncthreads();
#pragma unroll
            for (int z = 0; z < 32; ++z) buf[xl * kY + 32 * g + z] = v[z];
            __syncthreads();
            if (t == 0 && xt >= kSlots) wait_count(tab.done2 + (xt - kSlots), kT, st);
            __syncthreads();
            float2* stage = tab.stage + (size_t)(xt % kSlots) * kT * kN;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int row = 8 * warp + i;
                float2 e[4];
#pragma unroll
                for (int gg = 0; gg < 4; ++gg) e[gg] = buf[row * kY + 32 * gg + lane];
                wht_regs<2>(e);
#pragma unroll
                for (int gg = 0; gg < 4; ++gg) __stcg(stage + (size_t)row * kN + kT * cb + 32 * gg + lane, e[gg]);
            }
            __syncthreads();
            if (t == 0) {
                __threadfence();
                atomicAdd(tab.done1 + xt, 1);
            }
        } else {
            // ------------------------------------------------ row item (tensor cores)
            const int xt = r - 1, xl = j - kT;
            if (xt < 0) { __syncthreads(); continue; }
            if (t == 0) wait_count(tab.done1 + xt, kT, st);
            __syncthreads();
            const uint64_t x = (uint64_t)(kT * xt + xl);
            const float2* srow = tab.stage + ((size_t)(xt % kSlots) * kT + xl) * kN;
            // B[cb][n = 2 zl + ri]: lane (cb & 7, zq & 3) takes 4 complex (32 bytes),
            // so a warp reads 8 rows x 128 bytes and writes 32 distinct 16-byte
            // slots of 4 core matrices per split.  All 16 loads are issued first;
            // each split is stored and handed to the tensor core as soon as it is
            // complete, so the next split's stores overlap the previous MMAs.
            float4 a[16];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int task = t + kThreads * i; // 4096 tasks = 128 cb x 32 zq
                const int rest = task >> 5;
                const int zq = ((task >> 3) & 3) + 4 * (rest & 7);
                const int cbv = (task & 7) + 8 * (rest >> 3);
                const float4* p = reinterpret_cast<const float4*>(srow + (size_t)cbv * kT + 4 * zq);
                a[2 * i] = __ldcg(p);
                a[2 * i + 1] = __ldcg(p + 1);
            }
#pragma unroll 1
            for (int sp = 0; sp < 3; ++sp) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int task = t + kThreads * i;
                    const int rest = task >> 5;
                    const int zq = ((task >> 3) & 3) + 4 * (rest & 7);
                    const int cbv = (task & 7) + 8 * (rest >> 3);
                    float f[8] = {a[2 * i].x, a[2 * i].y, a[2 * i].z, a[2 * i].w,
                                  a[2 * i + 1].x, a[2 * i + 1].y, a[2 * i + 1].z, a[2 * i + 1].w};
                    uint16_t q[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        // peel split sp off the remainder: q = bf16(f), f -= q
                        const __nv_bfloat16 b = __float2bfloat16_rn(f[u]);
                        q[u] = __bfloat16_as_ushort(b);
                        f[u] -= __bfloat162float(b);
                    }
                    a[2 * i] = make_float4(f[0], f[1], f[2], f[3]);
                    a[2 * i + 1] = make_float4(f[4], f[5], f[6], f[7]);
                    const uint32_t off = (uint32_t)((cbv >> 3) * 32 + zq) * 128u + (uint32_t)(cbv & 7) * 16u;
                    *reinterpret_cast<uint4*>(opp + (uint32_t)sp * 65536u + off) =
                        make_uint4(pack2(q[0], q[1]), pack2(q[2], q[3]), pack2(q[4], q[5]), pack2(q[6], q[7]));
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (t == 0) {
#pragma unroll 1
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint64_t da = sdesc(h_a + (uint32_t)kk * 256u, 128u, 2048u);
                        const uint64_t db = sdesc(op_a + (uint32_t)sp * 65536u + (uint32_t)kk * 8192u, 4096u, 128u);
                        const uint32_t acc = (sp | kk) ? 1u : 0u;
                        asm volatile(
                            "{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                                tmem),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                    if (sp == 2)
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                         bar_a)
                                     : "memory");
                }
            }
            // the staging row is in shared memory now: drop its L2 lines
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float2* pl = srow + (size_t)(t + kThreads * i) * 16;
                asm volatile("discard.global.L2 [%0], 128;" ::"l"(pl) : "memory");
            }
            if (!mbar_wait(bar_a, parity)) {
                report_status(st, PTDR_ERR_TIMEOUT);
                pending = true;
            }
            parity ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // unload D[zb][2 zl + ri] into buf[zb][zl] (padded), 4 lane quarters x 4 column chunks
            {
                const int qd = warp & 3, cc = warp >> 2;
                const int zb = 32 * qd + lane;
                uint32_t rr[64];
                TC_LD64(rr, tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(64 * cc));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int u = 0; u < 32; ++u)
                    buf[zb * kY + 32 * cc + u] = make_float2(__uint_as_float(rr[2 * u]), __uint_as_float(rr[2 * u + 1]));
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            // contiguous stores of C[x][128 zb + zl] with the phase and scale
            {
                const int zl = 32 * (warp & 3) + lane, zg = warp >> 2;
                float2* out = C + (x << kLog);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int zb = 32 * zg + i;
                    const uint64_t z = (uint64_t)(kT * zb + zl);
                    const float2 o = phase_neg_i(buf[zb * kY + zl], (int)(__popcll(x & z) & 3), scale);
                    if (in_bounds(st, (x << kLog) + z, (uint64_t)kN * kN)) __stcs(out + z, o);
                }
            }
            __syncthreads();
            if (t == 0) {
                __threadfence();
                atomicAdd(tab.done2 + xt, 1);
            }
        }
    }
    if (pending) mbar_wait(bar_a, parity ^ 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ------------------------------------------------------------------ host

size_t tc14_staged_workspace() { return 4096 + (size_t)kSlots * kT * kN * sizeof(float2); }

cudaError_t launch_tc14_staged(const void* A, void* C, void* ws, unsigned int* st, cudaStream_t s)
{
    static std::mutex mu;
    static int grid_for[128];
    cudaError_t e = cudaFuncSetAttribute(k_tc14_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        grid = grid_for[dev & 127];
    }
    if (grid == 0) {
        int sms = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        grid = sms; // one CTA per SM: the operands fill shared memory and 256 TMEM columns are held
        std::lock_guard<std::mutex> lk(mu);
        grid_for[dev & 127] = grid;
    }
    char* w = (char*)ws;
    TcStagedTables tab;
    tab.head = (int*)w;
    tab.done1 = (int*)(w + 64);
    tab.done2 = (int*)(w + 64 + 4 * kTiles);
    tab.stage = (float2*)(w + 4096);
    if ((e = cudaMemsetAsync(ws, 0, 4096, s)) != cudaSuccess) return e;
    k_tc14_staged<<<grid, kThreads, kSmemBytes, s>>>((const float2*)A, (float2*)C, tab, st);
    return cudaGetLastError();
}

} // namespace ptdr
