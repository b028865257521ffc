// Dense n = 14 decomposition with both Hadamard stages on the tensor cores
// (split-bf16 path): complex64 -> complex64.
//
// With x = 128 xt + xl and k = 128 cb + cl the XOR-diagonal entries
// d_x[k] = A[k ^ x][k] of the 128 masks of x-tile xt and the 128 columns of
// block cb all lie in the tile T = A[128 R + .][128 cb + .], R = cb ^ xt:
// d_x[128 cb + cl] = T[cl ^ xl][cl].  The length-2^14 transform over k splits
// into 7 bits inside a block (cl) and 7 bits across blocks (cb), and both
// halves become products with the 128 x 128 Hadamard matrix
// H[a][b] = (-1)^{|a & b|}:
//
//   tile job (xt, cb):  with U[m][xl] = T[m][m ^ xl] (row m of the tile
//     permuted by XOR with m) and (-1)^{|zl & (m ^ xl)|} =
//     (-1)^{|zl & m|} (-1)^{|zl & xl|},
//       D'[xl][zl] = sum_cl (-1)^{|zl & cl|} T[cl ^ xl][cl]
//                  = (-1)^{|zl & xl|} (H U)[zl][xl],
//     written to an L2-resident staging row S[xl][128 cb + zl];
//   row job (x):  c_x[128 zb + zl] = 2^-14 (-i)^{|x & z|} (H B)[zb][zl]
//     with B[cb][zl] = S[xl][128 cb + zl].
//
// Each job is one tcgen05 product D = H_128 * B (M = 128, K = 128, N = 256
// real columns: n = 2 * column + re/im) accumulated in float32 in tensor
// memory.  The float32 operand is split exactly into three bf16 parts by
// truncation (hi = top 16 bits of x, mid = top 16 bits of x - hi, lo =
// x - hi - mid, which has at most 8 significant bits), so the only rounding
// of the tensor-core stage is the float32 accumulation; H is exact in bf16.
//
// One persistent CTA per SM, warp-specialised:
//   warps 0-7   loaders: 32-byte loads of 8 rows x 128 bytes per warp
//               instruction (tile rows from HBM, staging rows from L2), the
//               XOR permutation (tile jobs), the split, and 16-byte stores
//               into MN-major core matrices of a 4-deep ring of K chunks
//               (32 rows of K each);
//   warp 12     one lane issues 6 MMAs per chunk and commits each chunk back
//               to the ring and each job to one of two tensor-memory
//               accumulators (2 x 256 columns);
//   warps 8-11  epilogue: tcgen05.ld of the accumulator, sign or phase and
//               scale, coalesced stores (staging rows, or 32-byte pieces of
//               C rows).
// So the loads of one job, the MMAs of the previous one and the epilogue of
// the one before overlap on each SM.
//
// Jobs come from one atomic queue in x-tile-major rounds: round r holds the
// 128 tile jobs of x-tile r, then the 128 row jobs of x-tile r-1.  A row job
// waits (bounded) until its x-tile's tile jobs are done; a tile job waits
// (bounded) before writing its staging slot until the row jobs of the x-tile
// that used the slot before are done.  Within a CTA every stage waits only
// on older jobs, so the earliest unfinished job can always proceed.  Every
// wait is bounded: on time-out the kernel records PTDR_ERR_TIMEOUT, each
// role leaves its loop, in-flight MMAs are awaited (bounded) and the tensor
// memory is released.
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
constexpr int kLoadWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = kLoadWarps + kEpiWarps;
constexpr int kThreads = (kMmaWarp + 1) * 32; // 416
constexpr int kLoadThreads = kLoadWarps * 32;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kChunks = 4;                        // K chunks of 32 rows per job
constexpr uint32_t kSplitBytes = 32u * 256u * 2u; // one split of a chunk: 32 K x 256 N bf16
constexpr uint32_t kChunkSmem = 3u * kSplitBytes;
constexpr uint32_t kRingBytes = kChunks * kChunkSmem;
constexpr uint32_t kHBytes = kT * kT * 2u;
constexpr uint32_t kSmemBytes = kRingBytes + kHBytes + 1024u; // + alignment slack
constexpr uint32_t kTmemCols = 512;                           // two 128 x 256 float32 accumulators
constexpr int kSlots = 4;                                     // staging slots (x-tiles in flight)
constexpr int kPerRound = 2 * kT;
constexpr int kItems = (kTiles + 1) * kPerRound;
constexpr unsigned long long kWaitNs = 1000000000ull; // bound of every wait: 1 s

enum : int { kBarLoad = 1, kBarEpi = 2 };

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// Named barrier that also returns the OR of v over the participating threads.
__device__ __forceinline__ bool named_sync_or(int id, int n, bool v)
{
    uint32_t r;
    asm volatile("{ .reg .pred p, q; setp.ne.u32 q, %1, 0; bar.red.or.pred p, %2, %3, q; selp.u32 %0, 1, 0, p; }"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id), "r"(n)
                 : "memory");
    return r != 0;
}

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait for *p >= target (one thread).  False on time-out or abort.
__device__ __forceinline__ bool wait_count(const int* p, int target, const volatile int* abort_flag)
{
    const unsigned long long t0 = now_ns();
    while (ld_acquire(p) < target) {
        if (*abort_flag || now_ns() - t0 > kWaitNs) return false;
        __nanosleep(128);
    }
    return true;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity to complete (one thread).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag || now_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(bar) : "memory");
}

// Shared-memory matrix descriptor without swizzle (version 1).  K-major:
// lbo = K-direction core-matrix stride, sbo = M/N-direction stride.
// MN-major: lbo = K-direction stride, sbo = M/N-direction stride.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void ld8(const float* p, float (&f)[8])
{
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(f[0]), "=f"(f[1]), "=f"(f[2]), "=f"(f[3]), "=f"(f[4]), "=f"(f[5]), "=f"(f[6]), "=f"(f[7])
                 : "l"(p));
}

__device__ __forceinline__ void st8_cs(float* p, const float (&f)[8])
{
    asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(f[0]), "f"(f[1]), "f"(f[2]),
                 "f"(f[3]), "f"(f[4]), "f"(f[5]), "f"(f[6]), "f"(f[7])
                 : "memory");
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// Upper 16 bits of a and b as one bf16x2 word (element 0 in the low half).
__device__ __forceinline__ uint32_t hi16x2(float a, float b)
{
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

__device__ __forceinline__ float trunc_bf16(float a) { return __uint_as_float(__float_as_uint(a) & 0xFFFF0000u); }

// Exact three-way split of 8 floats into bf16 parts, written as three 16-byte
// core-matrix rows (hi at a, mid at a + kSplitBytes, lo at a + 2 kSplitBytes).
__device__ __forceinline__ void split_store(const float (&f)[8], uint32_t a)
{
    float r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = f[k] - trunc_bf16(f[k]);
    sts128(a, hi16x2(f[0], f[1]), hi16x2(f[2], f[3]), hi16x2(f[4], f[5]), hi16x2(f[6], f[7]));
    sts128(a + kSplitBytes, hi16x2(r[0], r[1]), hi16x2(r[2], r[3]), hi16x2(r[4], r[5]), hi16x2(r[6], r[7]));
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = r[k] - trunc_bf16(r[k]);
    sts128(a + 2u * kSplitBytes, hi16x2(r[0], r[1]), hi16x2(r[2], r[3]), hi16x2(r[4], r[5]), hi16x2(r[6], r[7]));
}

// v <- (v[j ^ p]) for the four complex values j = 0..3 held as 8 floats.
__device__ __forceinline__ void xor_permute(float (&f)[8], int p)
{
    float g[8];
    const bool s1 = (p & 1) != 0, s2 = (p & 2) != 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        g[2 * j] = s1 ? f[2 * (j ^ 1)] : f[2 * j];
        g[2 * j + 1] = s1 ? f[2 * (j ^ 1) + 1] : f[2 * j + 1];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        f[2 * j] = s2 ? g[2 * (j ^ 2)] : g[2 * j];
        f[2 * j + 1] = s2 ? g[2 * (j ^ 2) + 1] : g[2 * j + 1];
    }
}

#define TC_LD32(r, addr)                                                                              \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "                                            \
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22," \
                 "%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                       \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),    \
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), \
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),           \
                   "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),           \
                   "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])            \
                 : "r"(addr))

} // namespace

struct TcPipeTables {
    int* head;     // work-queue counter
    int* done1;    // tile jobs finished per x-tile
    int* done2;    // row jobs finished per x-tile
    float2* stage; // kSlots x 128 rows x 2^14
};

__global__ void __launch_bounds__(kThreads, 1)
    k_tc14_pipe(const float2* __restrict__ A, float2* __restrict__ C, TcPipeTables tab, unsigned int* st)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar_full[kChunks], bar_empty[kChunks], bar_tfull[2], bar_tempty[2],
        bar_exit;
    __shared__ int s_jobq[8];
    __shared__ int s_load_job[2];
    __shared__ int s_epi_job;
    __shared__ volatile int s_abort;
    __shared__ uint32_t s_tmem;

    const uint32_t raw_a = su32(smem_raw);
    const uint32_t ring_a = (raw_a + 1023u) & ~1023u;
    const uint32_t h_a = ring_a + kRingBytes;
    uint16_t* hmat = reinterpret_cast<uint16_t*>(smem_raw + (h_a - raw_a));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    // H_128 as the K-major A operand: element (zb, cb) = (-1)^{|zb & cb|}
    for (int e = t; e < kT * kT; e += kThreads) {
        const int z = e >> 7, k = e & 127;
        hmat[((z >> 3) * 16 + (k >> 3)) * 64 + (z & 7) * 8 + (k & 7)] = (__popc(z & k) & 1) ? 0xBF80u : 0x3F80u;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        for (int i = 0; i < kChunks; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar_full[i])), "r"(kLoadThreads));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_empty[i])));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_tfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar_tempty[i])), "r"(kEpiThreads));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_exit)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint64_t lim = (uint64_t)kN * kN;

    if (warp < kLoadWarps) {
        // ============================================================ loaders
        // warp w: k-group g = w >> 1 of each chunk, N groups a = 4 i' + (lane >> 3)
        // with i' in [4 (w & 1), 4 (w & 1) + 4); row m&7 = lane & 7.  A warp
        // instruction covers 8 rows x 4 N groups: full 32-byte sectors in
        // global memory and 4 conflict-free wavefronts in shared memory.
        const int g = warp >> 1, ib = 4 * (warp & 1), r7 = lane & 7, ag = lane >> 3;
        int next = 0;
        if (t == 0) next = atomicAdd(tab.head, 1);
        uint32_t L = 0;
        for (uint32_t it = 0;; ++it) {
            if (t == 0) {
                s_load_job[it & 1] = next;
                if (next < kItems) next = atomicAdd(tab.head, 1);
            }
            named_sync(kBarLoad, kLoadThreads);
            const int job = s_load_job[it & 1];
            bool tile = false;
            int xt = 0, cb = 0, xl = 0;
            if (job < kItems) {
                const int r = job / kPerRound, j = job % kPerRound;
                tile = j < kT;
                if (tile) {
                    xt = r;
                    cb = j;
                    if (xt >= kTiles) continue; // empty slot of the last round
                } else {
                    xt = r - 1;
                    xl = j - kT;
                    if (xt < 0) continue; // empty slot of the first round
                }
            }
            bool fail = false;
            if (t == 0) {
                if (job < kItems && !tile && !wait_count(tab.done1 + xt, kT, &s_abort)) {
                    report_status(st, PTDR_ERR_TIMEOUT);
                    s_abort = 1;
                    fail = true;
                }
                s_jobq[L & 7] = (job < kItems && !fail) ? job : -1;
            }
            fail = named_sync_or(kBarLoad, kLoadThreads, fail);
            const bool stop = job >= kItems || fail;

            // row sources: tile rows of A, or the staging row of mask x
            const float* src0;
            if (tile)
                src0 = reinterpret_cast<const float*>(A + ((uint64_t)(kT * (cb ^ xt)) << kLog) + (uint64_t)(kT * cb));
            else
                src0 = reinterpret_cast<const float*>(tab.stage + ((size_t)(xt % kSlots) * kT + xl) * kN);

            float f[2][4][8];
            auto issue = [&](int c, float (&buf)[4][8]) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int m = 32 * c + 8 * g + r7;
                    const int a = 4 * (ib + i) + ag;
                    const int as = tile ? (a ^ (m >> 2)) : a;
                    const uint64_t off = ((uint64_t)m << (tile ? kLog : 7)) + 4u * (uint32_t)as; // complex units
                    const bool okb =
                        !tile || in_bounds(st, ((uint64_t)(kT * (cb ^ xt) + m) << kLog) + (uint64_t)(kT * cb + 4 * as + 3), lim);
                    if (okb) {
                        ld8(src0 + 2 * off, buf[i]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; ++k) buf[i][k] = 0.f;
                    }
                }
            };
            if (!stop) {
                issue(0, f[0]);
                issue(1, f[1]);
            }
            bool broke = false;
#pragma unroll
            for (int c = 0; c < kChunks; ++c) {
                // the ring slot of chunk c was last read by the previous job's MMAs
                bool wfail = false;
                if (t == 0 && L > 0 && !mbar_wait(su32(&bar_empty[c]), (L - 1) & 1, &s_abort)) {
                    report_status(st, PTDR_ERR_TIMEOUT);
                    s_abort = 1;
                    wfail = true;
                }
                if (named_sync_or(kBarLoad, kLoadThreads, wfail)) {
                    broke = true;
                    break;
                }
                if (!stop) {
                    const uint32_t slot = ring_a + (uint32_t)c * kChunkSmem;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int m = 32 * c + 8 * g + r7;
                        const int a = 4 * (ib + i) + ag;
                        if (tile) xor_permute(f[c & 1][i], m & 3);
                        split_store(f[c & 1][i], slot + (uint32_t)g * 4096u + (uint32_t)a * 128u + (uint32_t)r7 * 16u);
                        if (!tile && ag == 0) {
                            // the 128-byte staging line (row m, groups 4 i'..4 i'+3) is in
                            // registers: drop it from L2 without write-back
                            const float* pl = src0 + 2 * (((uint64_t)m << 7) + 16u * (uint32_t)(ib + i));
                            asm volatile("discard.global.L2 [%0], 128;" ::"l"(pl) : "memory");
                        }
                    }
                    if (c + 2 < kChunks) issue(c + 2, f[c & 1]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(su32(&bar_full[c]));
                if (stop) break; // the end marker travels with chunk 0
            }
            if (stop || broke) break;
            ++L;
        }
    } else if (warp < kMmaWarp) {
        // ============================================================ epilogue
        const int q = warp & 3, et = t - kLoadThreads;
        const float scale = 1.0f / (float)kN;
        for (uint32_t L = 0;; ++L) {
            const uint32_t b = L & 1;
            if (et == 0) {
                const bool ok = mbar_wait(su32(&bar_tfull[b]), (L >> 1) & 1, &s_abort);
                int job = ok ? s_jobq[L & 7] : -1;
                if (!ok) {
                    report_status(st, PTDR_ERR_TIMEOUT);
                    s_abort = 1;
                }
                if (job >= 0) {
                    const int r = job / kPerRound, j = job % kPerRound;
                    // a tile job may overwrite its staging slot once the row jobs
                    // of the x-tile that used it before have read it
                    if (j < kT && r >= kSlots && !wait_count(tab.done2 + (r - kSlots), kT, &s_abort)) {
                        report_status(st, PTDR_ERR_TIMEOUT);
                        s_abort = 1;
                        job = -1;
                    }
                }
                s_epi_job = job;
            }
            named_sync(kBarEpi, kEpiThreads);
            const int job = s_epi_job;
            if (job < 0) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int r = job / kPerRound, j = job % kPerRound;
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + 256u * b;
            if (j < kT) {
                // tile job: lane = zl, columns n = 2 xl + ri
                const int xt = r, cb = j, zl = 32 * q + lane;
                float2* stage = tab.stage + (size_t)(xt % kSlots) * kT * kN + (size_t)(kT * cb + zl);
#pragma unroll 1
                for (int cc = 0; cc < 8; ++cc) {
                    uint32_t v[32];
                    TC_LD32(v, tbase + 32u * cc);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int xl = 16 * cc + u;
                        const float sg = (__popc(zl & xl) & 1) ? -1.0f : 1.0f;
                        __stcg(stage + (size_t)xl * kN, make_float2(sg * __uint_as_float(v[2 * u]), sg * __uint_as_float(v[2 * u + 1])));
                    }
                }
            } else {
                // row job: lane = zb, columns n = 2 zl + ri
                const int xt = r - 1, xl = j - kT, zb = 32 * q + lane;
                const int x = kT * xt + xl;
                float* out = reinterpret_cast<float*>(C + ((uint64_t)x << kLog) + (uint64_t)(kT * zb));
#pragma unroll 1
                for (int cc = 0; cc < 8; ++cc) {
                    uint32_t v[32];
                    TC_LD32(v, tbase + 32u * cc);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        float o[8];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int zl = 16 * cc + 4 * h + u;
                            const float2 w = make_float2(__uint_as_float(v[8 * h + 2 * u]), __uint_as_float(v[8 * h + 2 * u + 1]));
                            const float2 c2 = phase_neg_i(w, __popc(x & (kT * zb + zl)) & 3, scale);
                            o[2 * u] = c2.x;
                            o[2 * u + 1] = c2.y;
                        }
                        const int zl0 = 16 * cc + 4 * h;
                        if (in_bounds(st, ((uint64_t)x << kLog) + (uint64_t)(kT * zb + zl0 + 3), lim))
                            st8_cs(out + 2 * zl0, o);
                    }
                }
            }
            // the accumulator is in registers and stored: hand it back to the MMA warp
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(su32(&bar_tempty[b]));
            named_sync(kBarEpi, kEpiThreads);
            if (et == 0) {
                __threadfence();
                atomicAdd((j < kT ? tab.done1 + r : tab.done2 + (r - 1)), 1);
            }
        }
    } else {
        // ============================================================ MMA issue
        // M = 128, N = 256, A = bf16 K-major (H), B = bf16 MN-major, D = f32
        const uint32_t idesc =
            (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
        bool issued = false;
        for (uint32_t L = 0;; ++L) {
            const uint32_t b = L & 1;
            bool quit = false;
            for (int c = 0; c < kChunks && !quit; ++c) {
                int go = 1;
                if (lane == 0) {
                    bool ok = mbar_wait(su32(&bar_full[c]), L & 1, &s_abort);
                    if (ok && c == 0) {
                        if (s_jobq[L & 7] < 0) {
                            go = 0; // end of work: pass the marker on to the epilogue
                            mbar_arrive(su32(&bar_tfull[b]));
                        } else if (L >= 2) {
                            ok = mbar_wait(su32(&bar_tempty[b]), ((L >> 1) - 1) & 1, &s_abort);
                        }
                    }
                    if (!ok) {
                        report_status(st, PTDR_ERR_TIMEOUT);
                        s_abort = 1;
                        go = 0;
                    }
                }
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) {
                    quit = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (lane == 0) {
                    const uint32_t slot = ring_a + (uint32_t)c * kChunkSmem;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t da = sdesc(h_a + (uint32_t)(2 * c + kk) * 256u, 128u, 2048u);
#pragma unroll
                        for (int s = 0; s < 3; ++s) {
                            const uint64_t db = sdesc(slot + (uint32_t)s * kSplitBytes + (uint32_t)kk * 8192u, 4096u, 128u);
                            const uint32_t acc = (c | kk | s) ? 1u : 0u;
                            asm volatile(
                                "{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                                    tmem + 256u * b),
                                "l"(da), "l"(db), "r"(idesc), "r"(acc)
                                : "memory");
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     su32(&bar_empty[c]))
                                 : "memory");
                    if (c == kChunks - 1)
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                         su32(&bar_tfull[b]))
                                     : "memory");
                    issued = true;
                }
                __syncwarp();
            }
            if (quit) break;
        }
        // every MMA this warp issued has completed before the memory is released
        if (lane == 0 && issued) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&bar_exit))
                         : "memory");
            if (!mbar_wait(su32(&bar_exit), 0, &s_abort)) {
                // s_abort may be set: wait again without it, still bounded
                const unsigned long long t0 = now_ns();
                while (!mbar_try(su32(&bar_exit), 0) && now_ns() - t0 < kWaitNs) {
                }
            }
        }
        __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ------------------------------------------------------------------ host

size_t tc14_pipe_workspace() { return 4096 + (size_t)kSlots * kT * kN * sizeof(float2); }

cudaError_t launch_tc14_pipe(const void* A, void* C, void* ws, unsigned int* st, cudaStream_t s)
{
    static std::mutex mu;
    static int grid_for[128];
    cudaError_t e = cudaFuncSetAttribute(k_tc14_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
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
        grid = sms; // one CTA per SM: the ring fills shared memory and all 512 TMEM columns are held
        std::lock_guard<std::mutex> lk(mu);
        grid_for[dev & 127] = grid;
    }
    char* w = (char*)ws;
    TcPipeTables tab;
    tab.head = (int*)w;
    tab.done1 = (int*)(w + 64);
    tab.done2 = (int*)(w + 64 + 4 * kTiles);
    tab.stage = (float2*)(w + 4096);
    if ((e = cudaMemsetAsync(ws, 0, 4096, s)) != cudaSuccess) return e;
    k_tc14_pipe<<<grid, kThreads, kSmemBytes, s>>>((const float2*)A, (float2*)C, tab, st);
    return cudaGetLastError();
}

} // namespace ptdr
