// Band-diagonal matrices (Sec. IV.A of the paper): only the masks a band of
// half-width s can reach are transformed, and within a mask only the entries
// inside the band.
//
// For a mask x, entry k of the XOR-diagonal d_x[k] = A[k^x][k] lies at
// row - column = x - 2 (k & x), so it is inside the band only for the few
// t = k & x in T_x = { t subset of x : |x - 2t| <= s }.  Writing k = t | u'
// with u' a subset of the free bits F = ~x,
//     WHT(d_x)[z] = sum_{t in T_x} (-1)^{|z & t|} V_t[compress_F(z)],
//     V_t = WHT over the |F| free bits of g_t[u] = band_{x-2t}[t | expand_F(u)],
// so each mask costs |T_x| transforms of length 2^{n-|x|} plus one
// expansion pass, instead of a full length-2^n transform (the pruned X/Y
// subtrees of Sec. IV.A; for the tridiagonal masks 2^m - 1, |T_x| = 2).
// For a real band the rows g_t and V_t are real, so their transforms run in
// real arithmetic (half the adds and half the bytes of complex rows); the
// phase is applied once, in the expansion.
#include "tile_ops.cuh"
#include "structured.h"

namespace ptdr {

// Spreads the low bits of u over the free (zero) bits of x: the zeros of x
// below bit h1 = msb(x) + 1 take the low zc bits of u in order, every bit at
// or above h1 is free and takes the rest of u as a plain shift.
__device__ __forceinline__ uint64_t expand_free(uint64_t u, uint64_t x, int h1, int zc)
{
    uint64_t out = (u >> zc) << h1;
    uint64_t zeros = ~x & ((1ull << h1) - 1);
    uint64_t lo = u;
    while (zeros) {
        const int b = __ffsll((long long)zeros) - 1;
        zeros &= zeros - 1;
        out |= (lo & 1ull) << b;
        lo >>= 1;
    }
    return out;
}

// Inverse of expand_free on the free bits: the bits of z at the zeros of x
// below h1, packed, then the bits of z at and above h1.
__device__ __forceinline__ uint64_t compress_free(uint64_t z, uint64_t x, int h1, int zc)
{
    uint64_t out = (z >> h1) << zc;
    uint64_t zeros = ~x & ((1ull << h1) - 1);
    int j = 0;
    while (zeros) {
        const int b = __ffsll((long long)zeros) - 1;
        zeros &= zeros - 1;
        out |= ((z >> b) & 1ull) << j;
        ++j;
    }
    return out;
}

// A band value as a row value: complex rows take complex or real bands,
// real rows take real bands.
template <typename V, typename T, typename BandT> struct band_val {
    __device__ static __forceinline__ V ld(const BandT* p) { return io<BandT>::template ld<T>(p); }
};
template <typename T> struct band_val<T, T, float> {
    __device__ static __forceinline__ T ld(const float* p) { return (T)__ldg(p); }
};
template <typename T> struct band_val<T, T, double> {
    __device__ static __forceinline__ T ld(const double* p) { return (T)__ldg(p); }
};

// Sign flips as integer operations on the sign bit: the FP64 pipe (0.5 T
// operations/s on this part) is kept for the adds of the transforms.
__device__ __forceinline__ float neg_if(float a, bool c)
{
    return __uint_as_float(__float_as_uint(a) ^ (c ? 0x80000000u : 0u));
}
__device__ __forceinline__ double neg_if(double a, bool c)
{
    return __hiloint2double(__double2hiint(a) ^ (c ? (int)0x80000000u : 0), __double2loint(a));
}
__device__ __forceinline__ float2 neg_if(float2 a, bool c) { return make_float2(neg_if(a.x, c), neg_if(a.y, c)); }
__device__ __forceinline__ double2 neg_if(double2 a, bool c) { return make_double2(neg_if(a.x, c), neg_if(a.y, c)); }

// (-i)^p v for a complex v, by a swap and sign flips (no multiplies).
template <typename T2>
__device__ __forceinline__ T2 phase_flip(T2 v, int p)
{
    const bool odd = (p & 1) != 0;
    T2 r;
    r.x = neg_if(odd ? v.y : v.x, (p & 2) != 0);
    r.y = neg_if(odd ? v.x : v.y, ((p ^ (p >> 1)) & 1) != 0);
    return r;
}

__device__ __forceinline__ float scale_by(float v, float s) { return v * s; }
__device__ __forceinline__ double scale_by(double v, double s) { return v * s; }
__device__ __forceinline__ float2 scale_by(float2 v, float s) { return make_float2(v.x * s, v.y * s); }
__device__ __forceinline__ double2 scale_by(double2 v, double s) { return make_double2(v.x * s, v.y * s); }

__device__ __forceinline__ float2 as_cplx(float v) { return make_float2(v, 0.f); }
__device__ __forceinline__ double2 as_cplx(double v) { return make_double2(v, 0.0); }
__device__ __forceinline__ float2 as_cplx(float2 v) { return v; }
__device__ __forceinline__ double2 as_cplx(double2 v) { return v; }

// First pass: one CTA per (pair j, segment of 2^log_l values of u).  V is the
// row value type (complex, or T for a real band).  The 2^-n of the definition
// is applied here, once per band value (exact: a power of two), instead of
// once per coefficient in the expansion.
template <typename T, typename BandT, typename V>
__global__ void __launch_bounds__(512) k_band_first(BandMaskLaunch p, unsigned int* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s = reinterpret_cast<V*>(smem_raw);
    const Smem sm = make_smem(p.log_l);
    const int segs_log = p.f - p.log_l;
    const int j = blockIdx.x >> segs_log;
    const uint64_t seg = (uint64_t)blockIdx.x & ((1ull << segs_log) - 1);
    const uint64_t N = 1ull << p.n;
    const uint64_t t = p.t[j];
    const int64_t d = p.d[j];
    const BandT* band = (const BandT*)p.bands + (uint64_t)(d + p.s) * N;
    const int L = 1 << p.log_l;
    const uint64_t bands_elems = (uint64_t)(2 * p.s + 1) * N;
    const T scale = (T)p.scale;
    for (int e0 = threadIdx.x; e0 < L; e0 += kLoadBatch * blockDim.x) {
        V v[kLoadBatch];
#pragma unroll
        for (int b = 0; b < kLoadBatch; ++b) {
            const int e = e0 + b * blockDim.x;
            v[b] = V{};
            if (e < L) {
                const uint64_t u = (seg << p.log_l) + (uint64_t)e;
                const uint64_t k = t | expand_free(u, p.x, p.h1, p.zc);
                const uint64_t gi = (uint64_t)(d + p.s) * N + k;
                if (in_bounds(st, gi, bands_elems)) v[b] = scale_by(band_val<V, T, BandT>::ld(band + k), scale);
            }
        }
#pragma unroll
        for (int b = 0; b < kLoadBatch; ++b) {
            const int e = e0 + b * blockDim.x;
            if (e < L) s[sm.idx(e)] = v[b];
        }
    }
    __syncthreads();
    wht_bits(s, sm, p.log_l, 0, p.log_l);
    V* out = (V*)p.ws;
    const uint64_t row = (uint64_t)j << p.f;
    for (int e = threadIdx.x; e < L; e += blockDim.x) {
        const uint64_t gi = row + (seg << p.log_l) + (uint64_t)e;
        if (in_bounds(st, gi, p.ws_elems)) out[gi] = s[sm.idx(e)];
    }
}

// Expansion: C[row][z] = (-i)^{|x&z|} sum_j (-1)^{|z & t_j|} V_j[compress_F(z)]
// (V already carries the 2^-n).  The sum starts from the signed first term, so
// a mask of |T_x| pairs costs |T_x| - 1 adds per coefficient; signs and the
// phase are sign-bit flips and a swap.
template <typename T, typename OutT, typename RowV>
__global__ void __launch_bounds__(256) k_band_expand(BandMaskLaunch p, unsigned int* st)
{
    const uint64_t N = 1ull << p.n;
    const RowV* V = (const RowV*)p.ws;
    for (uint64_t z = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; z < N;
         z += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = compress_free(z, p.x, p.h1, p.zc);
        RowV acc{};
        for (int j = 0; j < p.npairs; ++j) {
            const uint64_t gi = ((uint64_t)j << p.f) + v;
            RowV w{};
            if (in_bounds(st, gi, p.ws_elems)) w = V[gi];
            const bool neg = (__popcll(z & p.t[j]) & 1) != 0;
            if (j == 0) acc = neg_if(w, neg);
            else acc = neg ? csub(acc, w) : cadd(acc, w);
        }
        // band: (-i)^{|x&z|}; anti-band, A = B J with J = X..X: the coefficient of
        // the anti-band mask x_A = x ^ (2^n - 1) is (-1)^{|z|} (-i)^{|x_A & z|} times the
        // same transform value, i.e. the exponent |x_A & z| + 2 |z|
        const int ph = p.anti ? __popcll(p.anti_x & z) + 2 * __popcll(z) : __popcll(p.x & z);
        const cplx_t<T> c = phase_flip(as_cplx(acc), ph);
        const uint64_t gi = p.out_row * N + z;
        if (in_bounds(st, gi, p.out_elems)) io<OutT>::st((OutT*)p.out + gi, c);
    }
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, typename BandT, typename V>
static cudaError_t run_first(const BandMaskLaunch& p, unsigned int* st, cudaStream_t s)
{
    auto kern = k_band_first<T, BandT, V>;
    const size_t bytes = smem_elems(1, p.log_l) * sizeof(V);
    cudaError_t e = set_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)p.npairs << (p.f - p.log_l);
    kern<<<blocks, p.threads, bytes, s>>>(p, st);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t first_by_band(const BandMaskLaunch& p, unsigned int* st, cudaStream_t s)
{
    switch (p.b_t) {
    case PTDR_F32: return p.real ? run_first<T, float, T>(p, st, s) : run_first<T, float, cplx_t<T>>(p, st, s);
    case PTDR_F64: return p.real ? run_first<T, double, T>(p, st, s) : run_first<T, double, cplx_t<T>>(p, st, s);
    case PTDR_C64: return run_first<T, float2, cplx_t<T>>(p, st, s);
    case PTDR_C128: return run_first<T, double2, cplx_t<T>>(p, st, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_band_first(const BandMaskLaunch& p, unsigned int* st, cudaStream_t s)
{
    return p.calc == Calc::F32 ? first_by_band<float>(p, st, s) : first_by_band<double>(p, st, s);
}

template <typename T, typename OutT>
static cudaError_t run_expand(const BandMaskLaunch& p, unsigned int* st, cudaStream_t s)
{
    const uint64_t N = 1ull << p.n;
    const uint64_t want = (N + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152ull * 16 ? want : 152ull * 16);
    if (p.real)
        k_band_expand<T, OutT, T><<<blocks, 256, 0, s>>>(p, st);
    else
        k_band_expand<T, OutT, cplx_t<T>><<<blocks, 256, 0, s>>>(p, st);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t expand_by_out(const BandMaskLaunch& p, unsigned int* st, cudaStream_t s)
{
    switch (p.c_t) {
    case PTDR_F32: return run_expand<T, float>(p, st, s);
    case PTDR_F64: return run_expand<T, double>(p, st, s);
    case PTDR_C64: return run_expand<T, float2>(p, st, s);
    case PTDR_C128: return run_expand<T, double2>(p, st, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_band_expand(const BandMaskLaunch& p, unsigned int* st, cudaStream_t s)
{
    return p.calc == Calc::F32 ? expand_by_out<float>(p, st, s) : expand_by_out<double>(p, st, s);
}

} // namespace ptdr
