// Device building blocks shared by the tile kernels: the padded shared-memory
// layout, in-register and in-shared-memory Walsh-Hadamard butterflies, and the
// tile loads/stores of the decompose (gather, phased write-out) and compose
// (phased load, XOR-scatter) paths.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace ptdr {

// ------------------------------------------------------------ smem layout

// Tile viewed as rows of 2^log_ls elements; one pad element every 16 and
// one per row keep the strided and XOR-permuted accesses conflict-free.
struct Smem {
    int log_ls;
    int rs; // row stride in elements
    __device__ __forceinline__ int idx(int f) const
    {
        int row = f >> log_ls;
        int col = f & ((1 << log_ls) - 1);
        return row * rs + col + (col >> 4);
    }
};

__device__ __forceinline__ Smem make_smem(int log_ls)
{
    Smem s;
    s.log_ls = log_ls;
    int ls = 1 << log_ls;
    s.rs = ls + ls / 16 + 1;
    return s;
}

// --------------------------------------------------------- register WHT

// In-register Walsh-Hadamard transform of 2^NB values: radix-2 butterflies
// (u + v, u - v) over each of the NB index bits.
template <int NB, typename T2>
__device__ __forceinline__ void wht_reg(T2 (&v)[1 << NB])
{
#pragma unroll
    for (int h = 1; h < (1 << NB); h <<= 1)
#pragma unroll
        for (int i = 0; i < (1 << NB); ++i)
            if (!(i & h)) {
                T2 a = v[i], b = v[i + h];
                v[i] = cadd(a, b);
                v[i + h] = csub(a, b);
            }
}

// Transform bits [b, b + NB) of the flat tile index (tile of 2^log_e values).
template <int NB, typename T2>
__device__ __forceinline__ void wht_pass(T2* s, const Smem& sm, int log_e, int b)
{
    const int groups = 1 << (log_e - NB);
    const int lowmask = (1 << b) - 1;
    for (int q = threadIdx.x; q < groups; q += blockDim.x) {
        const int base = (q & lowmask) | ((q >> b) << (b + NB));
        T2 v[1 << NB];
#pragma unroll
        for (int j = 0; j < (1 << NB); ++j) v[j] = s[sm.idx(base + (j << b))];
        wht_reg<NB>(v);
#pragma unroll
        for (int j = 0; j < (1 << NB); ++j) s[sm.idx(base + (j << b))] = v[j];
    }
}

// Transform flat-index bits [b0, b1), up to MaxNB (4 or 3) at a time, barrier
// after each pass (wide value types take 3 bits per pass: 8 values in registers).
template <int MaxNB = 4, typename T2>
__device__ void wht_bits(T2* s, const Smem& sm, int log_e, int b0, int b1)
{
    static_assert(MaxNB == 3 || MaxNB == 4, "radix-8 or radix-16 passes");
    for (int b = b0; b < b1; b += MaxNB) {
        const int nb = min(MaxNB, b1 - b);
        if constexpr (MaxNB == 4) { // not instantiated for radix-8 types
            if (nb == 4) {
                wht_pass<4>(s, sm, log_e, b);
                __syncthreads();
                continue;
            }
        }
        switch (nb) {
        case 3: wht_pass<3>(s, sm, log_e, b); break;
        case 2: wht_pass<2>(s, sm, log_e, b); break;
        default: wht_pass<1>(s, sm, log_e, b); break;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- loads

// Loads issued per thread before their values are stored to shared memory:
// independent loads in flight hide the memory latency of the gathers.
constexpr int kLoadBatch = 8;

// d_x[k] = A[k ^ x][k] for the tile's masks x in [x0, x0 + 2^log_r) and
// k in [k0, k0 + 2^log_l) (log_r <= log_l, both aligned).  With a row_mask the
// source holds only the rows r & row_mask of a sheared tile set (the
// matrix-free input): S[i][k] = A[((k >> a) ^ xt) 2^a + i][k].  Walked in the row
// view: row r of A supplies the aligned block of 2^log_r columns r ^ x, so
// consecutive threads read consecutive addresses.  Tile row = mask.
template <typename T, typename InT>
__device__ void load_gather(cplx_t<T>* s, const Smem& sm, const InT* A, int n, uint64_t x0,
                            int log_r, uint64_t k0, int log_l, uint64_t lim, unsigned int* st,
                            uint64_t row_mask = ~0ull)
{
    const uint64_t N = 1ull << n;
    const uint64_t R = 1ull << log_r, L = 1ull << log_l;
    const uint64_t rb = (k0 ^ x0) & ~(L - 1);
    const int E = 1 << (log_r + log_l);
    if constexpr (sizeof(InT) == sizeof(cplx_t<T>) && std::is_same<InT, cplx_t<T>>::value) {
        // same type in HBM and in the tile: asynchronous copies straight into shared
        // memory, all of a thread's elements in flight at once (no registers held)
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            const uint64_t r = rb + ((uint64_t)e >> log_r);
            const uint64_t c = ((r ^ x0) & ~(R - 1)) + ((uint64_t)e & (R - 1));
            const int xl = (int)((r ^ c) - x0);
            const int kl = (int)(c - k0);
            const uint64_t gi = (r & row_mask) * N + c;
            cplx_t<T>* d = s + sm.idx((xl << log_l) + kl);
            if (in_bounds(st, gi, lim)) {
                const uint32_t da = (uint32_t)__cvta_generic_to_shared(d);
                if constexpr (sizeof(InT) == 16)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(da), "l"(A + gi) : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(da), "l"(A + gi) : "memory");
            } else {
                *d = mk<T>(0, 0);
            }
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    } else {
        for (int e0 = threadIdx.x; e0 < E; e0 += kLoadBatch * blockDim.x) {
            cplx_t<T> v[kLoadBatch];
            int dst[kLoadBatch];
#pragma unroll
            for (int u = 0; u < kLoadBatch; ++u) {
                const int e = e0 + u * blockDim.x;
                dst[u] = -1;
                v[u] = mk<T>(0, 0);
                if (e < E) {
                    const uint64_t r = rb + ((uint64_t)e >> log_r);
                    const uint64_t c = ((r ^ x0) & ~(R - 1)) + ((uint64_t)e & (R - 1));
                    const int xl = (int)((r ^ c) - x0);
                    const int kl = (int)(c - k0);
                    const uint64_t gi = (r & row_mask) * N + c;
                    dst[u] = sm.idx((xl << log_l) + kl);
                    if (in_bounds(st, gi, lim)) v[u] = io<InT>::template ld<T>(A + gi);
                }
            }
#pragma unroll
            for (int u = 0; u < kLoadBatch; ++u)
                if (dst[u] >= 0) s[dst[u]] = v[u];
        }
    }
}

// Compose input: e_x[z] = scale * i^{|x&z|} * C[x][z] for the tile's masks and
// z in [k0, k0 + 2^log_l).  Contiguous rows.
template <typename T, typename InT>
__device__ void load_row_phase(cplx_t<T>* s, const Smem& sm, const InT* C, int n, uint64_t x0,
                               int log_r, uint64_t k0, int log_l, uint64_t row0, T scale,
                               uint64_t lim, unsigned int* st)
{
    const uint64_t N = 1ull << n;
    const int E = 1 << (log_r + log_l);
    for (int e0 = threadIdx.x; e0 < E; e0 += kLoadBatch * blockDim.x) {
        cplx_t<T> v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = mk<T>(0, 0);
            if (e < E) {
                const uint64_t x = x0 + (uint64_t)(e >> log_l);
                const uint64_t z = k0 + (uint64_t)(e & ((1 << log_l) - 1));
                const uint64_t gi = (x - row0) * N + z;
                if (in_bounds(st, gi, lim)) v[u] = io<InT>::template ld<T>(C + gi);
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < E) {
                const uint64_t x = x0 + (uint64_t)(e >> log_l);
                const uint64_t z = k0 + (uint64_t)(e & ((1 << log_l) - 1));
                // i^p = (-i)^(4 - p)
                s[sm.idx(e)] = phase_neg_i(v[u], 4 - (__popcll(x & z) & 3), scale);
            }
        }
    }
}

template <typename T>
__device__ void load_row_buf(cplx_t<T>* s, const Smem& sm, const cplx_t<T>* B, int n,
                             uint64_t x0, int log_r, uint64_t k0, int log_l, uint64_t row0,
                             uint64_t lim, unsigned int* st)
{
    const uint64_t N = 1ull << n;
    const int E = 1 << (log_r + log_l);
    for (int e0 = threadIdx.x; e0 < E; e0 += kLoadBatch * blockDim.x) {
        cplx_t<T> v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = mk<T>(0, 0);
            if (e < E) {
                const uint64_t x = x0 + (uint64_t)(e >> log_l);
                const uint64_t gi = (x - row0) * N + k0 + (uint64_t)(e & ((1 << log_l) - 1));
                if (in_bounds(st, gi, lim)) v[u] = B[gi];
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < E) s[sm.idx(e)] = v[u];
        }
    }
}

// --------------------------------------------------------------- stores

// Final decompose write-out: c_{x,z} = scale * (-i)^{|x&z|} * w_x[z].
template <typename T, typename OutT>
__device__ void store_row_phase(OutT* C, const cplx_t<T>* s, const Smem& sm, int n, uint64_t x0,
                                int log_r, uint64_t k0, int log_l, uint64_t row0, T scale,
                                uint64_t lim, unsigned int* st)
{
    const uint64_t N = 1ull << n;
    const int E = 1 << (log_r + log_l);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint64_t x = x0 + (uint64_t)(e >> log_l);
        const uint64_t z = k0 + (uint64_t)(e & ((1 << log_l) - 1));
        const uint64_t gi = (x - row0) * N + z;
        cplx_t<T> v = phase_neg_i(s[sm.idx(e)], __popcll(x & z), scale);
        if (in_bounds(st, gi, lim)) io<OutT>::st(C + gi, v);
    }
}

template <typename T>
__device__ void store_row_buf(cplx_t<T>* B, const cplx_t<T>* s, const Smem& sm, int n,
                              uint64_t x0, int log_r, uint64_t k0, int log_l, uint64_t row0,
                              uint64_t lim, unsigned int* st)
{
    const uint64_t N = 1ull << n;
    const int E = 1 << (log_r + log_l);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint64_t x = x0 + (uint64_t)(e >> log_l);
        const uint64_t gi = (x - row0) * N + k0 + (uint64_t)(e & ((1 << log_l) - 1));
        if (in_bounds(st, gi, lim)) B[gi] = s[sm.idx(e)];
    }
}

// Final compose write-out: A[k ^ x][k] = f_x[k]; the mirror of load_gather.
template <typename T, typename OutT>
__device__ void store_scatter(OutT* A, const cplx_t<T>* s, const Smem& sm, int n, uint64_t x0,
                              int log_r, uint64_t k0, int log_l, uint64_t lim, unsigned int* st)
{
    const uint64_t N = 1ull << n;
    const uint64_t R = 1ull << log_r, L = 1ull << log_l;
    const uint64_t rb = (k0 ^ x0) & ~(L - 1);
    const int E = 1 << (log_r + log_l);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint64_t r = rb + ((uint64_t)e >> log_r);
        const uint64_t c = ((r ^ x0) & ~(R - 1)) + ((uint64_t)e & (R - 1));
        const int xl = (int)((r ^ c) - x0);
        const int kl = (int)(c - k0);
        const uint64_t gi = r * N + c;
        if (in_bounds(st, gi, lim)) io<OutT>::st(A + gi, s[sm.idx((xl << log_l) + kl)]);
    }
}

} // namespace ptdr
