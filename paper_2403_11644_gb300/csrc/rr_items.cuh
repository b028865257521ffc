// Register-round items: the decomposition of R = 2^(13-n) masks of one
// complex64 matrix of n = 9 .. 12, computed in FP32 by one CTA of 256 threads
// through one shared tile of 8192 values.  Used by the batched kernel and by
// the dense single-matrix launch.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace ptdr {

// An item is the R = 2^(13-n) masks x0 .. x0 + R - 1 (x0 a multiple of R), a
// tile of 8192 values.  Its gather d_x[k] = A[k ^ x][k] is, row by row of A,
// the R columns (r ^ x0) & ~(R - 1) .. + R - 1 of row r: the item copies these
// pieces into shared memory as they are (16-byte cp.async copies), and reads
// the XOR permutation out of that "piece tile": with
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
//
// n = 12 (R = 2): a piece-tile bank pair is fixed by kh bits 0-1, kl and xl,
// so those stay with the lanes and round 1 transforms kh bits 2-6 instead
// (its sign is (-1)^{|w & X0 bits 2-6|}); round 2 transforms kh bits 7-10
// and round 3 (kl, kh bits 0-1), the lowest three bits of z, so that the
// last round again stores 64-byte runs of a C row with lanes over w.

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
constexpr int kRrElems = RrShape<9>::SIZE; // the largest of n = 9 .. 12
static_assert(RrShape<10>::SIZE <= kRrElems && RrShape<11>::SIZE <= kRrElems && RrShape<12>::SIZE <= kRrElems,
              "tile size");

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
    __stcs(reinterpret_cast<float4*>(C + z), make_float4(pa.x, pa.y, pb.x, pb.y));
}

// Issues (one commit group, not waited for) the 16-byte copies of item x0's
// piece tile: row r of A, columns ((r ^ x0) & ~(R - 1)) + [0, R), at s[r R].
// 4096 value pairs, 16 per thread: pair q is row q >> (lr - 1), columns
// ((r ^ x0) & ~(R - 1)) + 2 (q & (R / 2 - 1)) + {0, 1}, tile values 2q, 2q + 1.
template <int NQ>
__device__ __forceinline__ void rr_issue(const float2* __restrict__ A, uint32_t x0, float2* s, unsigned int* st)
{
    using Sh = RrShape<NQ>;
    constexpr int LR = Sh::LR, R = Sh::R;
    constexpr uint64_t kElems = 1ull << (2 * NQ);
    const int t = threadIdx.x;
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(s);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t q = t + 256 * i;
        const uint32_t r = q >> (LR - 1), h = q & ((R >> 1) - 1);
        const uint64_t gi = ((uint64_t)r << NQ) + ((r ^ x0) & ~(uint32_t)(R - 1)) + 2 * h;
        if (in_bounds(st, gi + 1, kElems))
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sb + 16u * q), "l"(A + gi) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Hooks of a persistent caller, called by every thread of the CTA at the
// same point.  `mid` runs after round 1's barrier, when no transform values
// are held in registers (a caller's bookkeeping there overlaps the other
// warps' round 2); `hook` runs once the last round has read the shared tile
// into registers (the rest of the item works from registers and writes C), so
// that the next item's piece copies, issued there, fly during this item's
// last transform and stores.  The single-item launch has nothing to do.
struct RrNoHook {
    __device__ __forceinline__ void operator()() const {}
};

// One item.  `issued`: its piece copies were already issued (by the previous
// item's hook) into s.
template <int NQ, typename Hook = RrNoHook, typename Mid = RrNoHook>
__device__ __forceinline__ void rr_item(const float2* __restrict__ A, float2* __restrict__ C, uint32_t x0,
                                        float2* s, float scale, unsigned int* st, bool issued = false,
                                        Hook hook = Hook(), Mid mid = Mid())
{
    using Sh = RrShape<NQ>;
    constexpr int LR = Sh::LR, R = Sh::R;
    constexpr uint64_t kElems = 1ull << (2 * NQ);
    const int t = threadIdx.x;
    if (!issued) rr_issue<NQ>(A, x0, s, st);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const uint32_t X0 = x0 >> LR;
    float2 v[32];
    if constexpr (NQ == 12) {
        // round 1: thread (kl, xl, kh bits 0-1, kh bits 7-10), 32 values over kh bits 2-6
        const int kl = t & 1, xl = (t >> 1) & 1, kh01 = (t >> 2) & 3, khh = t >> 4;
        const float2* p = s + (((((khh ^ (int)(X0 >> 7)) << 7) | (kh01 ^ (int)(X0 & 3))) << 2) + ((kl ^ xl) << 1) + kl);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = p[j << 4];
        wht_sub<5, 0, 1>(v);
        __syncthreads();
        float2* q = s + (xl * Sh::XS + ((khh << 3) | (kh01 << 1) | kl));
#pragma unroll
        for (int w = 0; w < 32; ++w) q[w * Sh::S] = v[w];
        __syncthreads();
        mid();
        const int warp = t >> 5, w = t & 31;
        const int sg = 2 * (__popc(w & (int)((X0 >> 2) & 31)) & 1);
        // round 2: thread (xl, kh bits 0-1) = warp, w = lane; 2 x 16 values over kh bits 7-10,
        // rewritten in place
        {
            float2* p2 = s + ((warp & 1) * Sh::XS + w * Sh::S + ((warp >> 1) << 1));
#pragma unroll
            for (int k0 = 0; k0 < 2; ++k0)
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) v[k0 * 16 + kk] = p2[(kk << 3) | k0];
            wht_sub<4, 0, 1>(v);
            wht_sub<4, 16, 1>(v);
#pragma unroll
            for (int k0 = 0; k0 < 2; ++k0)
#pragma unroll
                for (int zk = 0; zk < 16; ++zk) p2[(zk << 3) | k0] = v[k0 * 16 + zk];
        }
        __syncthreads();
        // round 3: thread (xl, z kh bits 9-10) = warp, w = lane; 4 x 8 values over (kl, kh bits 0-1)
        const int xl3 = warp & 1, zk23 = warp >> 1;
        const float2* p3 = s + (xl3 * Sh::XS + w * Sh::S + (zk23 << 5));
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = p3[j];
        hook();
        wht_sub<3, 0, 1>(v);
        wht_sub<3, 8, 1>(v);
        wht_sub<3, 16, 1>(v);
        wht_sub<3, 24, 1>(v);
        const uint32_t x = x0 + xl3;
        float2* row = C + ((uint64_t)x << NQ);
        if (in_bounds(st, ((uint64_t)x << NQ) + (1u << NQ) - 1, kElems))
#pragma unroll
            for (int g = 0; g < 4; ++g)
#pragma unroll
                for (int zl = 0; zl < 8; zl += 2) {
                    const uint32_t z = ((uint32_t)((zk23 << 2) | g) << 8) | (w << 3) | zl;
                    rr_put(row, x, z, sg, v[8 * g + zl], v[8 * g + zl + 1], scale);
                }
    } else {
    const int X0h = (int)(X0 >> 5), X0l = (int)(X0 & 31);
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
    mid();
    const int warp = t >> 5, w = t & 31;
    const int sg = 2 * (__popc(w & X0l) & 1);
    if constexpr (NQ == 10) {
        // round 2: thread (xl = warp, w = lane), 32 values over (kh bits 5-6, kl)
        const float2* p = s + (warp * Sh::XS + w * Sh::S);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = p[j];
        hook();
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
        hook();
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
        static_assert(NQ == 11, "register-round items cover n = 9 .. 12");
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
        hook();
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
    } // n = 9, 10, 11
}

} // namespace ptdr
