// Dense n = 14 decomposition with both Hadamard stages on the tensor cores
// (split-bf16 path): complex64 -> complex64.
//
// With x = 128 xt + xl and k = 128 cb + cl the XOR-diagonal entries
// d_x[k] = A[k ^ x][k] of the 128 masks of x-tile xt and the 128 columns of
// block cb all lie in the tile T = A[128 R + .][128 cb + .], R = cb ^ xt:
// d_x[128 cb + cl] = T[cl ^ xl][cl].  The length-2^14 transform over k splits
// into 7 bits inside a block (cl) and 7 bits across blocks (cb), and both
// halves become products with the 128 x 128 Hadamard matrix
// H[a][b] = (-1)^{|a & b|}, stored scaled by 2^-7 (exact in bf16) so that
// the two stages together apply the 2^-14 of the definition:
//
//   tile job (xt, cb):  with U[m][xl] = T[m][m ^ xl] (row m of the tile
//     permuted by XOR with m) and (-1)^{|zl & (m ^ xl)|} =
//     (-1)^{|zl & m|} (-1)^{|zl & xl|},
//       sum_cl (-1)^{|zl & cl|} T[cl ^ xl][cl] = (-1)^{|zl & xl|} (H U)[zl][xl];
//     the staging row receives S[xl][128 cb + zl] = (H U)[zl][xl];
//   row job (x):  c_x[128 zb + zl] = (-i)^{|xt & zb|} i^{|xl & zl|} (H B)[zb][zl],
//     B[cb][zl] = S[xl][128 cb + zl].
// The phase of the definition, (-i)^{|x & z|} with |x & z| = |xt & zb| +
// |xl & zl|, times the sign (-1)^{|zl & xl|} of the tile stage is
// (-i)^{|xt & zb|} i^{|xl & zl|}.  Both factors are applied once, after the
// row stage (which is linear over cb, so a factor of zl commutes with it): in
// the row epilogue each thread holds one zl, so i^{|xl & zl|} is a constant
// added to the 2-bit exponent of the zb factor, which is the same for a whole
// warp's run of zb.  The tile epilogue stores the products as they are.
//
// Each job is one tcgen05 product accumulated in float32 in tensor memory
// (K = 128, taken in 4 chunks of 32).  Tile jobs: D = H U, M = zl, N = 256
// real columns n = 2 xl + re/im, so a warp's lanes are consecutive zl and each
// staging store covers 256 contiguous bytes.  Row jobs: the transposed
// product D^T = B^T H in two halves of M = 128 (the real parts of the 128 zl,
// then the imaginary parts), N = zb, so a thread holds the real and the
// imaginary part of the same output and a warp's lanes are 32 consecutive
// outputs of one row of C.  The float32 operand is split exactly into three
// bf16 parts by truncation (hi = top 16 bits of x, mid = top 16 bits of
// x - hi, lo = x - hi - mid, which has at most 8 significant bits), so the
// only rounding of the tensor-core stage is the float32 accumulation; H is
// exact in bf16.
//
// One persistent CTA per SM, warp-specialised, every hand-off an mbarrier:
//   warp 25     producer: takes jobs from the queue and copies each K chunk
//               (32 rows of 1 KiB: tile rows from HBM, staging rows from L2)
//               into a 3-deep raw ring with eight tensor-map copies of
//               32 rows x 128 bytes (128-byte swizzle), which the copy engine
//               serves at over twice the rate of 1 KiB row copies;
//   warps 0-15  loaders: one raw row per lane (tile jobs read each complex
//               value at its XOR-permuted column; the swizzle keeps the eight
//               rows of a read phase on distinct banks), the split, and
//               16-byte stores into the MN-major core matrices of a 2-deep
//               operand ring;
//   warp 24     one lane issues the MMAs of each chunk and commits the chunk
//               back to the ring and each job to one of two tensor-memory
//               accumulators (2 x 256 columns);
//   warps 16-23 epilogue: tcgen05.ld of the accumulator, phase, coalesced
//               stores.
// So the copies of one job, the split of the next chunk, the MMAs and the
// epilogue of the job before overlap on each SM.
//
// Jobs come from one atomic queue in x-tile-major rounds: round r holds the
// 128 tile jobs of x-tile r, then the 128 row jobs of x-tile r - 2 (two
// rounds of slack, so that a row job rarely finds its x-tile unfinished).  A
// row job waits (bounded) until its x-tile's tile jobs are done; a tile job
// waits (bounded) before writing its staging slot until the row jobs of the
// x-tile that used the slot before are done.  A publisher warp (warp 26)
// counts each finished job once, after one fence, so that the epilogue warps
// never wait for their own stores to drain.  Within a CTA
// every stage waits only on older jobs, so the earliest unfinished job can
// always proceed.  Every wait is bounded: on time-out the kernel records
// PTDR_ERR_TIMEOUT, each role leaves its loop, in-flight MMAs are awaited
// (bounded) and the tensor memory is released.
#include <cuda.h>
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
constexpr int kLoadWarps = 16;
constexpr int kGroupsPerWarp = 32 / kLoadWarps; // tile jobs: groups of 4 complex per loader thread and chunk
constexpr int kUnitsPerWarp = 16 / kLoadWarps;  // row jobs: units of 8 zl per loader thread and chunk
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = kLoadWarps + kEpiWarps; // 24
constexpr int kProdWarp = kMmaWarp + 1;          // 25
constexpr int kPubWarp = kProdWarp + 1;          // 26
constexpr int kThreads = (kPubWarp + 1) * 32;    // 864
constexpr int kChunks = 4;                        // K chunks of 32 rows per job
constexpr uint32_t kSplitBytes = 32u * 256u * 2u; // one split of a chunk: 32 K x 256 M/N bf16
constexpr uint32_t kChunkSmem = 3u * kSplitBytes; // 48 KiB operand chunk
constexpr int kOpSlots = 2;
constexpr int kRawSlots = 3;
constexpr uint32_t kRawSlotBytes = 32u * 1024u;  // 8 swizzled boxes of 32 rows x 128 bytes
constexpr uint32_t kRawOff = kOpSlots * kChunkSmem;
constexpr uint32_t kHOff = kRawOff + kRawSlots * kRawSlotBytes;
constexpr uint32_t kHBytes = kT * kT * 2u;
constexpr uint32_t kSmemBytes = kHOff + kHBytes + 1024u; // + alignment slack (swizzled boxes: 1 KiB)
constexpr uint32_t kTmemCols = 512;                     // two 128 x 256 float32 accumulators
constexpr int kSlots = 4;                               // staging slots (x-tiles in flight)
constexpr int kLag = 2;                                 // row jobs of x-tile r run in round r + kLag
constexpr int kPerRound = 2 * kT;
constexpr int kItems = (kTiles + kLag) * kPerRound;
constexpr int kDoneTarget = kT; // jobs per finished x-tile pass
// Bound of the final wait for this CTA's own tensor-map copies still in flight
// after an abort (they land in microseconds; the CTA must not exit before).
constexpr unsigned long long kDrainNs = 100000000ull; // 100 ms
constexpr uint16_t kHPos = 0x3C00u, kHNeg = 0xBC00u;  // +2^-7, -2^-7 in bf16

static_assert(kSlots >= kLag + 2, "a staging slot is rewritten only after its row jobs were dequeued");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Per-CTA control block in shared memory: the abort flag every role polls and
// the bound of every wait for another role or another CTA (a launch parameter).
struct Ctl {
    volatile int abort;
    unsigned long long wait_ns;
};

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait for *p >= target (one thread).  False on time-out or abort.
__device__ __forceinline__ bool wait_count(const int* p, int target, Ctl* ctl)
{
    const unsigned long long t0 = now_ns();
    while (ld_acquire(p) < target) {
        if (ctl->abort || now_ns() - t0 > ctl->wait_ns) return false;
        __nanosleep(128);
    }
    return true;
}

// One test of an mbarrier phase (a potentially blocking try_wait with the
// system's default time limit: a longer suspend hint delays the wake-up of
// the operand-ring hand-offs).
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, Ctl* ctl)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (ctl->abort || now_ns() - t0 > ctl->wait_ns) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Tensor-map copy of one 2-D box global -> shared with an L2 eviction policy
// (A is read once: its lines go first, so that the staging stays in L2).
__device__ __forceinline__ void tma_2d_hint(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar, uint64_t pol)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(
                     dst),
                 "l"(map), "r"(x), "r"(y), "r"(bar), "l"(pol)
                 : "memory");
}

// Tensor-map copy of one 2-D box global -> shared (coordinates: x = float
// column, y = row), completion counted on an mbarrier.
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                     dst),
                 "l"(map), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void lds128(uint32_t addr, float& a, float& b, float& c, float& d)
{
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(a), "=f"(b), "=f"(c), "=f"(d) : "r"(addr));
}

// Lane 0 of the warp runs a bounded mbarrier wait; every lane gets the result.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, Ctl* ctl, int lane,
                                          unsigned int* st)
{
    int ok = 1;
    if (lane == 0 && !mbar_wait(bar, parity, ctl)) {
        report_status(st, PTDR_ERR_TIMEOUT);
        ctl->abort = 1;
        ok = 0;
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Shared-memory matrix descriptor without swizzle (version 1).  K-major:
// lbo = K-direction core-matrix stride, sbo = M/N-direction stride.
// MN-major: lbo = K-direction stride, sbo = M/N-direction stride.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint64_t pack64(uint32_t lo, uint32_t hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}

// One tcgen05 product D (+)= A B with both operands in shared memory.
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ void lds64(uint32_t addr, float& a, float& b)
{
    asm volatile("ld.shared.v2.f32 {%0,%1}, [%2];" : "=f"(a), "=f"(b) : "r"(addr));
}

__device__ __forceinline__ float trunc_bf16(float a) { return __uint_as_float(__float_as_uint(a) & 0xFFFF0000u); }

// (a, b) - (c, d) as one packed float32 pair operation.
__device__ __forceinline__ void sub2(float a, float b, float c, float d, float& r0, float& r1)
{
    uint64_t x, y, r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(x) : "f"(a), "f"(b));
    asm("mov.b64 %0, {%1,%2};" : "=l"(y) : "f"(c), "f"(d));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    asm("mov.b64 {%0,%1}, %2;" : "=f"(r0), "=f"(r1) : "l"(r));
}

// Exact three-way split of the pair (a, b) into bf16x2 words (a in the low
// half): hi = top 16 bits, mid = top 16 bits of the remainder, lo = the rest.
// Each remainder x - trunc(x) is exact in float32 (same sign and exponent).
__device__ __forceinline__ void split3(float a, float b, uint32_t& hi, uint32_t& mid, uint32_t& lo)
{
    hi = __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
    float ra, rb, la, lb;
    sub2(a, b, trunc_bf16(a), trunc_bf16(b), ra, rb);
    mid = __byte_perm(__float_as_uint(ra), __float_as_uint(rb), 0x7632);
    sub2(ra, rb, trunc_bf16(ra), trunc_bf16(rb), la, lb);
    lo = __byte_perm(__float_as_uint(la), __float_as_uint(lb), 0x7632);
}

// Job number -> kind, x-tile and column block (tile job) or mask (row job).
// Round r holds the tile jobs of x-tile r, then the row jobs of x-tile
// r - kLag; slots past either end of the x-tile range are empty (false).
__device__ __forceinline__ bool decode(int job, bool& tile, int& xt, int& idx)
{
    const int r = job / kPerRound, j = job % kPerRound;
    tile = j < kT;
    xt = tile ? r : r - kLag;
    idx = tile ? j : j - kT;
    return xt >= 0 && xt < kTiles;
}

// Sign bit of bit k of a mask, moved to bit 31.
__device__ __forceinline__ uint32_t sgn(uint32_t mask, int k) { return (mask << (31 - k)) & 0x80000000u; }

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
    int* done1;    // tile jobs finished per x-tile (x 8 epilogue warps)
    int* done2;    // row jobs finished per x-tile (x 8 epilogue warps)
    float2* stage; // kSlots x 128 rows x 2^14
    unsigned long long wait_ns; // bound of every wait for another role or CTA
};

// kRealOut: C holds float32 real parts only (the Hermitian real-output mode:
// for Hermitian A every coefficient is real, Thm 2), half the write bytes.
template <bool kRealOut>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc14_pipe(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmS, void* __restrict__ Cv,
                TcPipeTables tab, unsigned int* st)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long raw_full[kRawSlots], raw_empty[kRawSlots], op_full[kOpSlots],
        op_empty[kOpSlots], t_full[2], t_empty[2], e_done[2], p_done[2], bar_exit;
    __shared__ int s_jobq[8], s_pubq[4];
    __shared__ Ctl s_ctl;
    __shared__ int s_q_issued, s_q_seen; // raw chunks copied / observed landed (drain at exit)
    __shared__ uint32_t s_tmem;

    const uint32_t raw_a = su32(smem_raw);
    const uint32_t base = (raw_a + 1023u) & ~1023u;
    const uint32_t op_a = base, rawb_a = base + kRawOff, h_a = base + kHOff;
    uint16_t* hmat = reinterpret_cast<uint16_t*>(smem_raw + (h_a - raw_a));
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    // 2^-7 H_128 in K-major core matrices (A operand of tile jobs, B operand
    // of row jobs; H is symmetric): element (r, k) = 2^-7 (-1)^{|r & k|}
    for (int e = t; e < kT * kT; e += kThreads) {
        const int z = e >> 7, k = e & 127;
        hmat[((z >> 3) * 16 + (k >> 3)) * 64 + (z & 7) * 8 + (k & 7)] = (__popc(z & k) & 1) ? kHNeg : kHPos;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        for (int i = 0; i < kRawSlots; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&raw_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&raw_empty[i])), "r"(kLoadWarps));
        }
        for (int i = 0; i < kOpSlots; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&op_full[i])), "r"(kLoadWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&op_empty[i])));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&t_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&t_empty[i])), "r"(kEpiWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&e_done[i])), "r"(kEpiWarps));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&p_done[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_exit)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ctl.abort = 0;
        s_ctl.wait_ns = tab.wait_ns;
        s_q_issued = 0;
        s_q_seen = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint64_t lim = (uint64_t)kN * kN;

    if (warp == kProdWarp) {
        // ============================================================ producer
        int next = 0;
        if (lane == 0) next = atomicAdd(tab.head, 1);
        uint64_t evict_first;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(evict_first));
        uint32_t Q = 0, J = 0;
        for (;;) {
            int job = 0;
            if (lane == 0) {
                job = next;
                if (next < kItems) next = atomicAdd(tab.head, 1);
            }
            job = __shfl_sync(0xffffffffu, job, 0);
            bool tile = false;
            int xt = 0, idx = 0;
            if (job < kItems && !decode(job, tile, xt, idx)) continue; // empty slot of the first or last rounds
            int ok = 1;
            if (lane == 0 && job < kItems && !tile && !wait_count(tab.done1 + xt, kDoneTarget, &s_ctl)) {
                report_status(st, PTDR_ERR_TIMEOUT);
                s_ctl.abort = 1;
                ok = 0;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (job >= kItems || !ok) {
                // end marker: travels with the next raw chunk
                if (lane == 0) {
                    s_jobq[J & 7] = -1;
                    const uint32_t sl = Q % kRawSlots;
                    if (Q < (uint32_t)kRawSlots ||
                        mbar_wait(su32(&raw_empty[sl]), (Q / kRawSlots - 1) & 1, &s_ctl))
                        mbar_arrive(su32(&raw_full[sl]));
                }
                break;
            }
            if (!tile) {
                // the staging rows were written through the generic proxy by other
                // CTAs: acquire their counter, then order the bulk copies after it
                (void)ld_acquire(tab.done1 + xt);
                asm volatile("fence.proxy.async;" ::: "memory");
            }
            if (lane == 0) s_jobq[J & 7] = job;
            const int cb = idx, xl = idx;
            // tile job: rows 128 (cb ^ xt) + k of A, float columns 256 cb + 32 b + .;
            // row job: staging rows (slot, xl, k) of 256 floats (k = K row of the job)
            const int x0 = tile ? 256 * cb : 0;
            const int y0 = tile ? kT * (cb ^ xt) : ((xt % kSlots) * kT + xl) * kT;
            bool quit = false;
            for (int c = 0; c < kChunks; ++c, ++Q) {
                const uint32_t sl = Q % kRawSlots;
                int go = 1;
                if (lane == 0) {
                    if (Q >= (uint32_t)kRawSlots &&
                        !mbar_wait(su32(&raw_empty[sl]), (Q / kRawSlots - 1) & 1, &s_ctl)) {
                        report_status(st, PTDR_ERR_TIMEOUT);
                        s_ctl.abort = 1;
                        go = 0;
                    } else {
                        mbar_arrive_tx(su32(&raw_full[sl]), 32u * 1024u);
                    }
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    quit = true;
                    break;
                }
                if (lane < 8) {
                    const int x = x0 + 32 * lane, y = y0 + 32 * c;
                    const bool okb = in_bounds(st, (uint64_t)(y + 31), tile ? (uint64_t)kN : (uint64_t)kSlots * kT * kT) &&
                                     in_bounds(st, (uint64_t)(x + 31), tile ? 2ull * kN : 256ull);
                    const uint32_t dst = rawb_a + sl * kRawSlotBytes + 4096u * (uint32_t)lane;
                    if (tile)
                        tma_2d_hint(dst, &tmA, okb ? x : 0, okb ? y : 0, su32(&raw_full[sl]), evict_first);
                    else
                        tma_2d(dst, &tmS, okb ? x : 0, okb ? y : 0, su32(&raw_full[sl]));
                }
            }
            if (quit) break;
            ++J;
        }
        if (lane == 0) s_q_issued = (int)Q; // chunks whose copies were issued
    } else if (warp < kLoadWarps) {
        // ============================================================ loaders
        // Lane l takes K row l of each chunk (m = 32 c + l), which sits in row l of
        // each 4 KiB box of the raw slot with its 16-byte pieces swizzled by l & 7.
        // Tile job (B operand, N = 2 xl + re/im): N groups a = 4 w + i, i = 0..3; group
        //   a is xl = 4a .. 4a + 3, whose values in tile row m sit at complex columns
        //   m ^ xl = 4 A + ((m & 3) ^ j), A = a ^ (m >> 2).
        // Row job (A operand, M = real parts of zl = 0..127, then imaginary parts):
        //   units v = 2 w + u, u = 0, 1; unit v is zl = 8v .. 8v + 7 (64 raw bytes),
        //   stored as M group v (real parts) and M group 16 + v (imaginary parts).
        // The 8 lanes of a read phase hold 8 consecutive rows (distinct swizzles), and
        // the 8 lanes of a store phase fill one 128-byte core matrix: no bank conflicts.
        const int ml = lane;
        const uint32_t sw = (uint32_t)(ml & 7);
        const uint32_t pj = (uint32_t)(ml & 3); // m & 3 for every row this thread reads
        // byte offset of complex j of a tile group inside its 32-byte piece pair:
        // piece (2 (A & 3) + (q >> 1)) ^ sw, half q & 1, q = pj ^ j
        const uint32_t e0 = ((((pj >> 1) ^ sw) & 1u) << 4) + 8u * (pj & 1u);
        uint32_t Q = 0;
        for (uint32_t J = 0;; ++J) {
            int job = -1;
            bool quit = false;
            for (int c = 0; c < kChunks; ++c, ++Q) {
                const uint32_t rs = Q % kRawSlots, os = Q % kOpSlots;
                if (!warp_wait(su32(&raw_full[rs]), (Q / kRawSlots) & 1, &s_ctl, lane, st)) {
                    quit = true;
                    break;
                }
                if (c == 0) job = s_jobq[J & 7];
                const bool stop = job < 0;
                bool tile = false;
                int xt = 0, xl = 0;
                if (!stop) (void)decode(job, tile, xt, xl);
                const uint32_t rrow = rawb_a + rs * kRawSlotBytes + 128u * (uint32_t)ml;
                uint32_t w[12 * kGroupsPerWarp];
                // all shared loads of the chunk first, then the splits
                float f[8 * kGroupsPerWarp];
                if (!stop && tile) {
                    const int mh = (32 * c + ml) >> 2;
#pragma unroll
                    for (int i = 0; i < kGroupsPerWarp; ++i) {
                        const uint32_t A = (uint32_t)((kGroupsPerWarp * warp + i) ^ mh);
                        const uint32_t gb = rrow + 4096u * (A >> 2) + (((2u * (A & 3u)) ^ (sw & 6u)) << 4);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            lds64(gb + (e0 ^ (uint32_t)(((j >> 1) << 4) | ((j & 1) << 3))), f[8 * i + 2 * j], f[8 * i + 2 * j + 1]);
                    }
#pragma unroll
                    for (int i = 0; i < kGroupsPerWarp; ++i)
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            split3(f[8 * i + 2 * k], f[8 * i + 2 * k + 1], w[12 * i + k], w[12 * i + 4 + k], w[12 * i + 8 + k]);
                } else if (!stop) {
#pragma unroll
                    for (int u = 0; u < kUnitsPerWarp; ++u) {
                        const uint32_t v = (uint32_t)(kUnitsPerWarp * warp + u);
                        const uint32_t vb = rrow + 4096u * (v >> 1);
#pragma unroll
                        for (int k = 0; k < 4; ++k) // re0, im0, re1, im1, ...
                            lds128(vb + (((4u * (v & 1u) + (uint32_t)k) ^ sw) << 4), f[16 * u + 4 * k], f[16 * u + 4 * k + 1],
                                   f[16 * u + 4 * k + 2], f[16 * u + 4 * k + 3]);
                    }
#pragma unroll
                    for (int u = 0; u < kUnitsPerWarp; ++u)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            split3(f[16 * u + 4 * k], f[16 * u + 4 * k + 2], w[24 * u + k], w[24 * u + 4 + k], w[24 * u + 8 + k]);
                            split3(f[16 * u + 4 * k + 1], f[16 * u + 4 * k + 3], w[24 * u + 12 + k], w[24 * u + 16 + k],
                                   w[24 * u + 20 + k]);
                        }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(su32(&raw_empty[rs]));
                // the operand slot was last read by the MMAs of chunk Q - 2
                if (Q >= (uint32_t)kOpSlots &&
                    !warp_wait(su32(&op_empty[os]), (Q / kOpSlots - 1) & 1, &s_ctl, lane, st)) {
                    quit = true;
                    break;
                }
                const uint32_t slot = op_a + os * kChunkSmem + (uint32_t)(ml >> 3) * 4096u + (uint32_t)(ml & 7) * 16u;
                if (!stop && tile) {
#pragma unroll
                    for (int i = 0; i < kGroupsPerWarp; ++i) {
                        const uint32_t at = slot + (uint32_t)(kGroupsPerWarp * warp + i) * 128u;
#pragma unroll
                        for (int s = 0; s < 3; ++s)
                            sts128(at + (uint32_t)s * kSplitBytes, w[12 * i + 4 * s], w[12 * i + 4 * s + 1],
                                   w[12 * i + 4 * s + 2], w[12 * i + 4 * s + 3]);
                    }
                } else if (!stop) {
#pragma unroll
                    for (int u = 0; u < kUnitsPerWarp; ++u) {
                        const uint32_t at = slot + (uint32_t)(kUnitsPerWarp * warp + u) * 128u;
#pragma unroll
                        for (int s = 0; s < 3; ++s) {
                            sts128(at + (uint32_t)s * kSplitBytes, w[24 * u + 4 * s], w[24 * u + 4 * s + 1],
                                   w[24 * u + 4 * s + 2], w[24 * u + 4 * s + 3]);
                            sts128(at + 2048u + (uint32_t)s * kSplitBytes, w[24 * u + 12 + 4 * s],
                                   w[24 * u + 13 + 4 * s], w[24 * u + 14 + 4 * s], w[24 * u + 15 + 4 * s]);
                        }
                    }
                    // the chunk's 32 staging rows are consumed: drop their 256 lines
                    // from L2 without write-back (one per loader thread of the first 256)
                    const int ln = 32 * warp + lane;
                    const float2* pl =
                        tab.stage + ((size_t)(xt % kSlots) * kT + xl) * kN + (size_t)(32 * c + (ln >> 3)) * kT + 16 * (ln & 7);
                    if (ln < 256) asm volatile("discard.global.L2 [%0], 128;" ::"l"(pl) : "memory");
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(su32(&op_full[os]));
                if (stop) {
                    quit = true; // the end marker has been passed on with chunk 0
                    break;
                }
            }
            if (quit) break;
        }
        if (lane == 0) atomicMax(&s_q_seen, (int)Q); // chunks seen landed by this warp
    } else if (warp < kMmaWarp) {
        // ============================================================ epilogue
        // warp e = warp - 8 reads TMEM lanes 32 q .. 32 q + 31 (q = warp & 3, the
        // lanes its warp slot may access) and accumulator columns of half h = e >> 2.
        const int q = warp & 3, hcol = (warp - kLoadWarps) >> 2;
        const int zl = 32 * q + lane;
        for (uint32_t J = 0;; ++J) {
            const uint32_t b = J & 1;
            int job = -1;
            if (lane == 0) {
                if (mbar_wait(su32(&t_full[b]), (J >> 1) & 1, &s_ctl)) {
                    job = s_jobq[J & 7];
                    bool tl = false;
                    int xt = 0, ix = 0;
                    // a tile job may overwrite its staging slot once the row jobs
                    // of the x-tile that used it before have read it
                    if (job >= 0 && decode(job, tl, xt, ix) && tl && xt >= kSlots &&
                        !wait_count(tab.done2 + (xt - kSlots), kDoneTarget, &s_ctl)) {
                        report_status(st, PTDR_ERR_TIMEOUT);
                        s_ctl.abort = 1;
                        job = -1;
                    }
                } else {
                    report_status(st, PTDR_ERR_TIMEOUT);
                    s_ctl.abort = 1;
                }
            }
            job = __shfl_sync(0xffffffffu, job, 0);
            if (warp == kLoadWarps && lane == 0) s_pubq[J & 3] = job;
            // hand job J to the publisher warp, which must have taken job J - 2 off
            // this barrier pair first (so that no phase of it is skipped)
            auto hand_off = [&]() {
                if (lane == 0) {
                    if (J >= 2 && !mbar_wait(su32(&p_done[b]), ((J >> 1) - 1) & 1, &s_ctl)) {
                        report_status(st, PTDR_ERR_TIMEOUT);
                        s_ctl.abort = 1;
                    }
                    mbar_arrive(su32(&e_done[b]));
                }
            };
            if (job < 0) {
                hand_off(); // pass the end (or abort) on to the publisher
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            bool tile = false;
            int xt = 0, idx = 0;
            (void)decode(job, tile, xt, idx);
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + 256u * b;
            if (tile) {
                // columns n = 2 xl + re/im, xl = 64 h + 16 cc + u; row S[xl] of the slot
                const int cb = idx;
                float2* stage = tab.stage + (size_t)(xt % kSlots) * kT * kN + (size_t)(64 * hcol) * kN +
                                (size_t)(kT * cb + zl);
#pragma unroll 1
                for (int cc = 0; cc < 4; ++cc) {
                    uint32_t v[32];
                    TC_LD32(v, tbase + 128u * hcol + 32u * cc);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (cc == 3) {
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(su32(&t_empty[b]));
                    }
                    // the product as it is: the phase is applied after the row stage
                    float2* srow = stage + (size_t)(16 * cc) * kN;
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        __stcg(srow + (size_t)u * kN, make_float2(__uint_as_float(v[2 * u]), __uint_as_float(v[2 * u + 1])));
                }
            } else {
                // real parts of zl in columns zb, imaginary parts in 128 + zb;
                // this warp writes zb = 64 h + 32 cc + u of row x
                const int xl = idx, x = kT * xt + xl;
                // (-i)^{|xt & zb|}: bits u of the two low bits of popc((xt & 31) & u),
                // accumulated over the set bits of xt & 31 (adding 1 to a 2-bit value
                // flips bit 0 and carries bit 0 into bit 1)
                const uint32_t m5 = (uint32_t)xt & 31u;
                uint32_t w1 = 0u, w2 = 0u;
                const uint32_t pat[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
#pragma unroll
                for (int bb = 0; bb < 5; ++bb) {
                    const uint32_t pb = ((m5 >> bb) & 1u) ? pat[bb] : 0u;
                    w2 ^= w1 & pb;
                    w1 ^= pb;
                }
                const uint64_t o0 = ((uint64_t)x << kLog) + (uint64_t)(kT * 64 * hcol) + (uint64_t)zl;
                float2* out = (float2*)Cv + o0;
                float* outr = (float*)Cv + o0;
#pragma unroll
                // the tile stage's factor i^{|xl & zl|} = (-i)^{3 |xl & zl|} is constant for
                // this thread's zl (the row stage is linear over cb, so it commutes)
                const uint32_t c_l = (3u * (uint32_t)__popc(xl & zl)) & 3u;
                for (int cc = 0; cc < 2; ++cc) {
                    const uint32_t bs = ((uint32_t)__popc(xt & (64 * hcol + 32 * cc)) + c_l) & 3u;
                    const uint32_t odd = w1 ^ ((bs & 1u) ? 0xFFFFFFFFu : 0u);
                    const uint32_t two = w2 ^ ((bs & 2u) ? 0xFFFFFFFFu : 0u) ^ ((bs & 1u) ? w1 : 0u);
                    const uint32_t sx = two, sy = odd ^ two;
                    uint32_t vr[32], vi[32];
                    TC_LD32(vr, tbase + 64u * hcol + 32u * cc);
                    TC_LD32(vi, tbase + 128u + 64u * hcol + 32u * cc);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (cc == 1) {
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(su32(&t_empty[b]));
                    }
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const bool o = ((odd >> u) & 1u) != 0;
                        const uint32_t ox = (o ? vi[u] : vr[u]) ^ sgn(sx, u);
                        const uint32_t oy = (o ? vr[u] : vi[u]) ^ sgn(sy, u);
                        if (in_bounds(st, ((uint64_t)x << kLog) + (uint64_t)(kT * (64 * hcol + 32 * cc + u) + zl), lim)) {
                            if constexpr (kRealOut)
                                __stcs(outr + (size_t)(kT * (32 * cc + u)), __uint_as_float(ox));
                            else
                                __stcs(out + (size_t)(kT * (32 * cc + u)), make_float2(__uint_as_float(ox), __uint_as_float(oy)));
                        }
                    }
                }
            }
            __syncwarp();
            hand_off(); // the publisher fences and counts the job's stores
        }
    } else if (warp == kMmaWarp) {
        // ============================================================ MMA issue
        // tile jobs: M = 128 (zl), N = 256, A = H (K-major), B = operand (MN-major)
        const uint32_t idesc_tile =
            (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
        // row jobs: M = 128 (one half of the 256 operand rows), N = 128 (zb),
        // A = operand (MN-major), B = H (K-major)
        const uint32_t idesc_row =
            (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
        const uint64_t dop = sdesc(op_a, 4096u, 128u), dhh = sdesc(h_a, 128u, 2048u);
        const uint32_t op_lo = (uint32_t)dop, op_hi = (uint32_t)(dop >> 32);
        const uint32_t h_lo = (uint32_t)dhh, h_hi = (uint32_t)(dhh >> 32);
        bool issued = false;
        uint32_t Q = 0;
        for (uint32_t J = 0;; ++J) {
            const uint32_t b = J & 1;
            bool quit = false, tile = true;
            for (int c = 0; c < kChunks; ++c, ++Q) {
                const uint32_t os = Q % kOpSlots;
                int go = 1, tl = 1;
                if (lane == 0) {
                    bool ok = mbar_wait(su32(&op_full[os]), (Q / kOpSlots) & 1, &s_ctl);
                    if (ok && c == 0) {
                        const int job = s_jobq[J & 7];
                        if (job < 0) {
                            go = 0; // end of work: pass the marker on to the epilogue
                            mbar_arrive(su32(&t_full[b]));
                        } else {
                            tl = (job % kPerRound) < kT;
                            if (J >= 2) ok = mbar_wait(su32(&t_empty[b]), ((J >> 1) - 1) & 1, &s_ctl);
                        }
                    }
                    if (!ok) {
                        report_status(st, PTDR_ERR_TIMEOUT);
                        s_ctl.abort = 1;
                        go = 0;
                    }
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    quit = true;
                    break;
                }
                if (c == 0) tile = __shfl_sync(0xffffffffu, tl, 0) != 0;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (lane == 0) {
                    // descriptors of one layout differ only in the address field (bits 0-13
                    // of the low word): each product adds a constant to a base word
                    const uint32_t slo = op_lo + ((os * kChunkSmem) >> 4);
                    const uint32_t hlo = h_lo + ((uint32_t)(2 * c) * 256u >> 4);
                    const uint32_t dt = tmem + 256u * b;
                    const uint32_t first = c ? 1u : 0u; // accumulate into the job's earlier chunks
                    if (tile) {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                            for (int s = 0; s < 3; ++s)
                                mma_ss(dt, pack64(hlo + 16u * kk, h_hi),
                                       pack64(slo + ((uint32_t)s * kSplitBytes + (uint32_t)kk * 8192u) / 16u, op_hi), idesc_tile,
                                       (kk | s) ? 1u : first);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                            for (int s = 0; s < 3; ++s)
#pragma unroll
                                for (int h = 0; h < 2; ++h)
                                    mma_ss(dt + 128u * h,
                                           pack64(slo + ((uint32_t)s * kSplitBytes + (uint32_t)kk * 8192u + 2048u * h) / 16u, op_hi),
                                           pack64(hlo + 16u * kk, h_hi), idesc_row, (kk | s) ? 1u : first);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     su32(&op_empty[os]))
                                 : "memory");
                    if (c == kChunks - 1)
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                         su32(&t_full[b]))
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
            const unsigned long long t0 = now_ns();
            while (!mbar_try(su32(&bar_exit), 0) && now_ns() - t0 < kDrainNs) {
            }
        }
        __syncwarp();
    } else if (warp == kPubWarp) {
        // ============================================================ publisher
        // Once the 8 epilogue warps have stored job J (their mbarrier arrivals
        // release the stores to this thread), one fence makes them visible at GPU
        // scope before the job is counted for the CTAs that wait on its x-tile.
        for (uint32_t J = 0;; ++J) {
            const uint32_t b = J & 1;
            int job = -1;
            if (lane == 0) {
                if (mbar_wait(su32(&e_done[b]), (J >> 1) & 1, &s_ctl)) {
                    job = s_pubq[J & 3];
                } else {
                    report_status(st, PTDR_ERR_TIMEOUT);
                    s_ctl.abort = 1;
                }
                bool tl = false;
                int xt = 0, ix = 0;
                if (job >= 0 && decode(job, tl, xt, ix)) {
                    __threadfence();
                    atomicAdd((tl ? tab.done1 : tab.done2) + xt, 1);
                }
                mbar_arrive(su32(&p_done[b]));
            }
            job = __shfl_sync(0xffffffffu, job, 0);
            if (job < 0) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    // After an abort the loaders may have left chunks whose tensor-map copies are
    // still landing in this CTA's shared memory: wait (bounded) for each of them
    // before the CTA exits.  Each such chunk is the last fill of its ring slot (a
    // slot is refilled only after the loaders release it), so its phase parity
    // identifies it.  Without an abort every chunk was seen landed: no wait.
    if (t == 0) {
        const int q0 = max(s_q_seen, s_q_issued - kRawSlots);
        for (int q = q0; q < s_q_issued; ++q) {
            const uint32_t bar = su32(&raw_full[q % kRawSlots]), par = (uint32_t)(q / kRawSlots) & 1u;
            const unsigned long long t0 = now_ns();
            while (!mbar_try(bar, par) && now_ns() - t0 < kDrainNs) {
            }
        }
    }
}

// ------------------------------------------------------------------ host

size_t tc14_pipe_workspace() { return 4096 + (size_t)kSlots * kT * kN * sizeof(float2); }

namespace {

using encode_fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                               const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
encode_fn tensor_map_encoder()
{
    static std::once_flag once;
    static encode_fn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<encode_fn>(p);
    });
    return fn;
}

// A float32 matrix of `rows` x `cols` (row pitch `cols` floats) read in
// 32 x 32 boxes with the 128-byte swizzle.
bool encode_boxes(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols)
{
    encode_fn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 4};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

} // namespace

cudaError_t launch_tc14_pipe(const void* A, void* C, bool real_out, void* ws, unsigned int* st, cudaStream_t s)
{
    static std::mutex mu;
    static int grid_for[128];
    auto kern = real_out ? k_tc14_pipe<true> : k_tc14_pipe<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
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
        grid = sms; // one CTA per SM: the rings fill shared memory and all 512 TMEM columns are held
        std::lock_guard<std::mutex> lk(mu);
        grid_for[dev & 127] = grid;
    }
    char* w = (char*)ws;
    TcPipeTables tab;
    tab.head = (int*)w;
    tab.done1 = (int*)(w + 64);
    tab.done2 = (int*)(w + 64 + 4 * kTiles);
    tab.stage = (float2*)(w + 4096);
    tab.wait_ns = wait_limit_ns();
    CUtensorMap tmA, tmS;
    if (!encode_boxes(&tmA, A, kN, 2 * kN) || !encode_boxes(&tmS, tab.stage, (uint64_t)kSlots * kT * kT, 2 * kT))
        return cudaErrorInvalidValue;
    if ((e = cudaMemsetAsync(ws, 0, 4096, s)) != cudaSuccess) return e;
    kern<<<grid, kThreads, kSmemBytes, s>>>(tmA, tmS, C, tab, st);
    return cudaGetLastError();
}

} // namespace ptdr
