// Exact fixed-point path (PTDR_PREC_FIXED_I128): the FP64-accuracy mode that
// does not use the FP64 pipe.
//
// The Walsh-Hadamard transform of Sec. II.A's sparse trace (per mask x,
// c_{x,z} = 2^-n (-i)^{|x&z|} sum_k (-1)^{|z&k|} A[k^x][k]) and of the inverse
// map is a sum of +-1 multiples of the inputs, so in two's-complement fixed
// point it is exact.  With E the binary exponent bound of the input
// (every |Re|, |Im| < 2^E, from a max pre-pass over the whole input) each
// real input v becomes the 128-bit integer X = round(v 2^S), S = 124 - n - E:
// |X| < 2^(124-n), and a sum of 2^n such values stays below 2^124, inside
// 127 bits.  The transform is then integer adds (no rounding at all), and
// each result is rounded once to the output type.  The only error is the
// input rounding below 2^-(124-n) of the largest input and the final
// rounding.
//
// GB300's FP64 pipe is slow (about 0.5 T adds/s, the bound of the FP64
// path); nothing here uses it: inputs are decoded from their IEEE bit fields
// and outputs encoded the same way, with integer shifts and round-to-nearest-
// even done on the integers.  Only a compose scale that is not a power of two
// costs one FP64 multiply per output value.
//
// Kernels: a pre-pass (maximum exponent field of the input), the tile kernel
// (gather or phased row load, radix-8 transform passes in shared memory,
// phased write-out / intermediate rows / XOR-scatter) and the strided pass
// over the high bits, which reads and writes 32-byte fixed-point complex
// values of an intermediate in the workspace (chunks of masks small enough to
// stay in L2).
#include <algorithm>
#include <cmath>

#include "fixed_point.cuh"
#include "plan.h"
#include "tile_ops.cuh"

namespace ptdr {

using fxp::i128;
using fxp::fixed_of;
using fxp::f32_bits;
using fxp::f64_bits;

// A complex value in 128-bit fixed point (real, imaginary).
struct __align__(16) fx2 {
    i128 x, y;
};

__device__ __forceinline__ fx2 cadd(fx2 a, fx2 b)
{
    a.x += b.x;
    a.y += b.y;
    return a;
}
__device__ __forceinline__ fx2 csub(fx2 a, fx2 b)
{
    a.x -= b.x;
    a.y -= b.y;
    return a;
}

// The shared tile as two planes of 16-byte integers (real parts, then
// imaginary parts) under the padded index of tile_ops.cuh, which keeps warp
// accesses to 16-byte elements at the minimum number of wavefronts; whole
// 32-byte values at that index put eight lanes on each bank group.
struct FxTile {
    i128* re;
    i128* im;
    __device__ __forceinline__ fx2 get(int i) const { return fx2{re[i], im[i]}; }
    __device__ __forceinline__ void put(int i, const fx2& v) const
    {
        re[i] = v.x;
        im[i] = v.y;
    }
};

// The planes of a tile of rows x 2^log_ls values (each plane padded as
// smem_elems counts it; the launch reserves two planes of 16 bytes).
__device__ __forceinline__ FxTile fx_tile(void* smem, int rows, int log_ls)
{
    const int ls = 1 << log_ls;
    i128* b = reinterpret_cast<i128*>(smem);
    return FxTile{b, b + rows * (ls + ls / 16 + 1)};
}

// Radix-2^NB butterflies over bits [b, b + NB) of the flat tile index.
template <int NB>
__device__ __forceinline__ void fx_pass(const FxTile& s, const Smem& sm, int log_e, int b)
{
    const int groups = 1 << (log_e - NB);
    const int lowmask = (1 << b) - 1;
    for (int q = threadIdx.x; q < groups; q += blockDim.x) {
        const int base = (q & lowmask) | ((q >> b) << (b + NB));
        fx2 v[1 << NB];
#pragma unroll
        for (int j = 0; j < (1 << NB); ++j) v[j] = s.get(sm.idx(base + (j << b)));
#pragma unroll
        for (int h = 1; h < (1 << NB); h <<= 1)
#pragma unroll
            for (int i = 0; i < (1 << NB); ++i)
                if (!(i & h)) {
                    const fx2 a = v[i], c = v[i + h];
                    v[i] = cadd(a, c);
                    v[i + h] = csub(a, c);
                }
#pragma unroll
        for (int j = 0; j < (1 << NB); ++j) s.put(sm.idx(base + (j << b)), v[j]);
    }
}

// Flat-index bits [b0, b1) in radix-8 passes, a barrier after each.
__device__ __forceinline__ void fx_bits(const FxTile& s, const Smem& sm, int log_e, int b0, int b1)
{
    for (int b = b0; b < b1; b += 3) {
        const int nb = min(3, b1 - b);
        if (nb == 3) fx_pass<3>(s, sm, log_e, b);
        else if (nb == 2) fx_pass<2>(s, sm, log_e, b);
        else fx_pass<1>(s, sm, log_e, b);
        __syncthreads();
    }
}

namespace {

template <typename InT> struct in_of;
template <> struct in_of<float2> {
    __device__ static __forceinline__ fx2 cvt(float2 v, int S) { return fx2{fixed_of(v.x, S), fixed_of(v.y, S)}; }
};
template <> struct in_of<double2> {
    __device__ static __forceinline__ fx2 cvt(double2 v, int S) { return fx2{fixed_of(v.x, S), fixed_of(v.y, S)}; }
};
// real inputs (a real matrix, or real coefficients of a Hermitian matrix)
template <> struct in_of<float> {
    __device__ static __forceinline__ fx2 cvt(float v, int S) { return fx2{fixed_of(v, S), 0}; }
};
template <> struct in_of<double> {
    __device__ static __forceinline__ fx2 cvt(double v, int S) { return fx2{fixed_of(v, S), 0}; }
};

// How the fixed-point results become output values: value = X 2^(q_pow - S),
// times `mul` when the scale is not a power of two.
struct FxOut {
    int q;
    double mul;
    bool use_mul;
};

// Output value (-i)^p * X 2^q (* mul): an odd p swaps the parts, the real part
// changes sign for p = 2, 3 and the imaginary part for p = 1, 2 (sign bits).
template <typename OutT> struct out_of;
template <> struct out_of<double2> {
    __device__ static __forceinline__ double2 cvt(fx2 v, int p, const FxOut& o)
    {
        const bool odd = (p & 1) != 0;
        uint64_t re = f64_bits(odd ? v.y : v.x, o.q), im = f64_bits(odd ? v.x : v.y, o.q);
        re ^= (uint64_t)((p >> 1) & 1) << 63;
        im ^= (uint64_t)((p ^ (p >> 1)) & 1) << 63;
        double2 r = make_double2(__longlong_as_double((long long)re), __longlong_as_double((long long)im));
        if (o.use_mul) {
            r.x *= o.mul;
            r.y *= o.mul;
        }
        return r;
    }
};
template <> struct out_of<float2> {
    __device__ static __forceinline__ float2 cvt(fx2 v, int p, const FxOut& o)
    {
        const bool odd = (p & 1) != 0;
        if (o.use_mul) { // round once to double, scale, round to float
            const double2 d = out_of<double2>::cvt(v, p, o);
            return make_float2((float)d.x, (float)d.y);
        }
        uint32_t re = f32_bits(odd ? v.y : v.x, o.q), im = f32_bits(odd ? v.x : v.y, o.q);
        re ^= (uint32_t)((p >> 1) & 1) << 31;
        im ^= (uint32_t)((p ^ (p >> 1)) & 1) << 31;
        return make_float2(__uint_as_float(re), __uint_as_float(im));
    }
};

// Real outputs store the real part of (-i)^p X 2^q (Hermitian A: all of c, Thm 2):
// Re for even p, Im for odd p, negated for p = 2, 3.
template <> struct out_of<double> {
    __device__ static __forceinline__ double cvt(fx2 v, int p, const FxOut& o)
    {
        uint64_t re = f64_bits((p & 1) ? v.y : v.x, o.q) ^ ((uint64_t)((p >> 1) & 1) << 63);
        double r = __longlong_as_double((long long)re);
        return o.use_mul ? r * o.mul : r;
    }
};
template <> struct out_of<float> {
    __device__ static __forceinline__ float cvt(fx2 v, int p, const FxOut& o)
    {
        if (o.use_mul) return (float)out_of<double>::cvt(v, p, o);
        const uint32_t re = f32_bits((p & 1) ? v.y : v.x, o.q) ^ ((uint32_t)((p >> 1) & 1) << 31);
        return __uint_as_float(re);
    }
};

// i^p times a fixed-point value (exact: swaps and negations).
__device__ __forceinline__ fx2 times_i_pow(fx2 v, int p)
{
    // i^p = (-i)^m with m = 4 - p (mod 4); (-i)^m: an odd m swaps the parts,
    // the real part changes sign for m = 2, 3 and the imaginary part for m = 1, 2
    const int m = (4 - (p & 3)) & 3;
    const bool odd = (m & 1) != 0;
    const i128 u = odd ? v.y : v.x, w = odd ? v.x : v.y;
    return fx2{(m & 2) ? -u : u, ((m ^ (m >> 1)) & 1) ? -w : w};
}

} // namespace

// Threads per CTA of the tile and strided kernels: two CTAs of 256 threads
// share an SM (64 KiB tiles, up to 128 registers a thread without spills);
// two small CTAs wait at their barriers independently, where one CTA of 512
// threads stalls as a whole.
constexpr int kFxThreads = 256;

struct FxLaunch {
    const void* src;
    void* dst;
    Load load;
    Store store;
    int n;
    int log_r, log_l;    // tile kernel: masks x segment
    int b0, b1, log_w;   // strided kernel: bits [b0, b1), 2^log_w columns
    uint64_t x_begin, x_count, dst_row0, src_row0, src_elems, dst_elems;
    const int* emax;     // largest exponent field of the original input (pre-pass)
    int bias;            // exponent bias of the original input's type
    int q_pow;           // output value = X 2^(q_pow - S) (* mul)
    double mul;
    bool use_mul;
};

namespace {

// Exponent bound E of the original input (every |value| < 2^E) and the shift S.
__device__ __forceinline__ int fx_shift(const FxLaunch& p)
{
    const int f = *p.emax;
    const int E = f ? f - p.bias + 1 : 1 - p.bias;
    return 124 - p.n - E;
}

__device__ __forceinline__ FxOut fx_out(const FxLaunch& p, int S) { return FxOut{p.q_pow - S, p.mul, p.use_mul}; }

// ----------------------------------------------------------------- pre-pass

// Largest exponent field over `words` machine words of real values (32-bit
// words for float data, 64-bit for double); a non-finite value is an argument
// error recorded in the status word.
template <typename W>
__global__ void __launch_bounds__(256) k_fx_maxexp(const W* __restrict__ v, uint64_t words, int* emax, unsigned int* st)
{
    constexpr int kShift = sizeof(W) == 4 ? 23 : 52;
    constexpr uint32_t kMask = sizeof(W) == 4 ? 0xFFu : 0x7FFu;
    uint32_t best = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    constexpr int kU = 8;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (kU - 1) * stride < words; i += kU * stride) {
        W w[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) w[u] = __ldcs(v + i + u * stride);
#pragma unroll
        for (int u = 0; u < kU; ++u) best = max(best, (uint32_t)(w[u] >> kShift) & kMask);
    }
    for (; i < words; i += stride) best = max(best, (uint32_t)(__ldcs(v + i) >> kShift) & kMask);
#pragma unroll
    for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best) {
        if (best == kMask) report_status(st, PTDR_ERR_INVALID_ARG);
        atomicMax(emax, (int)best);
    }
}

// ------------------------------------------------------------- tile kernel

template <typename InT, Load LD>
__device__ void fx_load(const FxTile& s, const Smem& sm, const FxLaunch& p, uint64_t x0, uint64_t k0, int S, unsigned int* st)
{
    const uint64_t N = 1ull << p.n;
    const int log_r = p.log_r, log_l = p.log_l;
    const uint64_t R = 1ull << log_r, L = 1ull << log_l;
    const int E = 1 << (log_r + log_l);
    for (int e0 = threadIdx.x; e0 < E; e0 += kLoadBatch * blockDim.x) {
        InT v[kLoadBatch];
        fx2 f[kLoadBatch];
        int dst[kLoadBatch];
        int ph[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            dst[u] = -1;
            ph[u] = 0;
            if (e >= E) continue;
            if constexpr (LD == Load::GatherA) {
                // row r of A supplies the aligned block of 2^log_r columns r ^ x
                const uint64_t rb = (k0 ^ x0) & ~(L - 1);
                const uint64_t r = rb + ((uint64_t)e >> log_r);
                const uint64_t c = ((r ^ x0) & ~(R - 1)) + ((uint64_t)e & (R - 1));
                const uint64_t gi = r * N + c;
                dst[u] = sm.idx((int)(((r ^ c) - x0) << log_l) + (int)(c - k0));
                if (in_bounds(st, gi, p.src_elems)) v[u] = __ldg((const InT*)p.src + gi);
                else dst[u] = -2;
            } else {
                const uint64_t x = x0 + (uint64_t)(e >> log_l);
                const uint64_t z = k0 + (uint64_t)(e & ((1 << log_l) - 1));
                const uint64_t gi = (x - p.src_row0) * N + z;
                dst[u] = sm.idx(e);
                ph[u] = __popcll(x & z);
                if (!in_bounds(st, gi, p.src_elems)) dst[u] = -2;
                else if constexpr (LD == Load::RowBuf) f[u] = ((const fx2*)p.src)[gi];
                else v[u] = __ldg((const InT*)p.src + gi);
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            if (dst[u] == -1) continue;
            const int d = dst[u] == -2 ? -1 : dst[u];
            fx2 w;
            if constexpr (LD == Load::RowBuf)
                w = f[u];
            else if constexpr (LD == Load::RowPhaseC)
                w = times_i_pow(in_of<InT>::cvt(v[u], S), ph[u]);
            else
                w = in_of<InT>::cvt(v[u], S);
            if (d >= 0) s.put(d, w);
        }
    }
}

template <typename OutT, Store ST>
__device__ void fx_store(const FxTile& s, const Smem& sm, const FxLaunch& p, uint64_t x0, uint64_t k0, int S,
                         unsigned int* st)
{
    const uint64_t N = 1ull << p.n;
    const int log_r = p.log_r, log_l = p.log_l;
    const uint64_t R = 1ull << log_r, L = 1ull << log_l;
    const int E = 1 << (log_r + log_l);
    const FxOut o = fx_out(p, S);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        if constexpr (ST == Store::ScatterA) {
            const uint64_t rb = (k0 ^ x0) & ~(L - 1);
            const uint64_t r = rb + ((uint64_t)e >> log_r);
            const uint64_t c = ((r ^ x0) & ~(R - 1)) + ((uint64_t)e & (R - 1));
            const uint64_t gi = r * N + c;
            const fx2 v = s.get(sm.idx((int)(((r ^ c) - x0) << log_l) + (int)(c - k0)));
            if (in_bounds(st, gi, p.dst_elems)) ((OutT*)p.dst)[gi] = out_of<OutT>::cvt(v, 0, o);
        } else {
            const uint64_t x = x0 + (uint64_t)(e >> log_l);
            const uint64_t z = k0 + (uint64_t)(e & ((1 << log_l) - 1));
            const uint64_t gi = (x - p.dst_row0) * N + z;
            const fx2 v = s.get(sm.idx(e));
            if (!in_bounds(st, gi, p.dst_elems)) continue;
            if constexpr (ST == Store::RowBuf)
                ((fx2*)p.dst)[gi] = v;
            else
                ((OutT*)p.dst)[gi] = out_of<OutT>::cvt(v, __popcll(x & z) & 3, o);
        }
    }
}

template <typename InT, typename OutT, Load LD, Store ST>
__global__ void __launch_bounds__(kFxThreads, 2) k_fx_tile(FxLaunch p, unsigned int* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FxTile s = fx_tile(smem_raw, 1 << p.log_r, p.log_l);
    const Smem sm = make_smem(p.log_l);
    const int segs_log = p.n - p.log_l;
    const uint64_t blk = (uint64_t)blockIdx.x >> segs_log;
    const uint64_t seg = (uint64_t)blockIdx.x & ((1ull << segs_log) - 1);
    const uint64_t x0 = p.x_begin + (blk << p.log_r);
    const uint64_t k0 = seg << p.log_l;
    const int S = fx_shift(p);
    fx_load<InT, LD>(s, sm, p, x0, k0, S, st);
    __syncthreads();
    fx_bits(s, sm, p.log_r + p.log_l, 0, p.log_l);
    fx_store<OutT, ST>(s, sm, p, x0, k0, S, st);
}

// One CTA per (mask, group of bits >= b1, chunk of 2^log_w low columns) of an
// intermediate of fixed-point rows; transform over bits [b0, b1).
template <typename OutT, Store ST>
__global__ void __launch_bounds__(kFxThreads, 2) k_fx_strided(FxLaunch p, unsigned int* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = p.b1 - p.b0;
    const FxTile s = fx_tile(smem_raw, 1 << nb, p.log_w);
    const Smem sm = make_smem(p.log_w);
    const uint64_t N = 1ull << p.n;
    const int chunks_log = p.b0 - p.log_w;
    const int groups_log = p.n - p.b1;
    uint64_t id = blockIdx.x;
    const uint64_t chunk = id & ((1ull << chunks_log) - 1);
    id >>= chunks_log;
    const uint64_t g = id & ((1ull << groups_log) - 1);
    id >>= groups_log;
    const uint64_t x = p.x_begin + id;
    const uint64_t kbase = (g << p.b1) + (chunk << p.log_w);
    const fx2* src = (const fx2*)p.src + (x - p.src_row0) * N;
    const int E = 1 << (nb + p.log_w);
    const int wmask = (1 << p.log_w) - 1;
    for (int e0 = threadIdx.x; e0 < E; e0 += kLoadBatch * blockDim.x) {
        fx2 v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = fx2{0, 0};
            if (e < E) {
                const uint64_t k = kbase + ((uint64_t)(e >> p.log_w) << p.b0) + (uint64_t)(e & wmask);
                if (in_bounds(st, (x - p.src_row0) * N + k, p.src_elems)) v[u] = src[k];
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < E) s.put(sm.idx(e), v[u]);
        }
    }
    __syncthreads();
    fx_bits(s, sm, nb + p.log_w, p.log_w, nb + p.log_w);
    const int S = fx_shift(p);
    const FxOut o = fx_out(p, S);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint64_t k = kbase + ((uint64_t)(e >> p.log_w) << p.b0) + (uint64_t)(e & wmask);
        const fx2 v = s.get(sm.idx(e));
        if constexpr (ST == Store::RowPhaseOut) {
            const uint64_t gi = (x - p.dst_row0) * N + k;
            if (in_bounds(st, gi, p.dst_elems))
                ((OutT*)p.dst)[gi] = out_of<OutT>::cvt(v, __popcll(x & k) & 3, o);
        } else if constexpr (ST == Store::RowBuf) {
            const uint64_t gi = (x - p.dst_row0) * N + k;
            if (in_bounds(st, gi, p.dst_elems)) ((fx2*)p.dst)[gi] = v;
        } else {
            const uint64_t gi = (k ^ x) * N + k;
            if (in_bounds(st, gi, p.dst_elems)) ((OutT*)p.dst)[gi] = out_of<OutT>::cvt(v, 0, o);
        }
    }
}

// ------------------------------------- compile-time shapes (n = 13 .. 15)
//
// The multi-pass decompose plans of n = 13, 14, 15 (first pass: 4 masks x
// 512 values per tile; one strided pass over the remaining n - 9 bits) with
// every shape a constant: the index arithmetic folds to shifts and masks of
// 32-bit integers (n <= 15: every element index is below 2^30) and each
// thread takes a fixed number of values.  Same arithmetic and layout as the
// generic kernels above.

// Tile layouts: the padded index of a row length 2^LS with one pad value
// every 2^PS values and row stride RS.  FxLay<LS> is the layout of make_smem
// (a pad every 16, stride 2^LS + 2^LS/16 + 1).  FxLayGather is the first-pass
// tile of 4 rows x 512: a pad every 8 and stride 580 put every warp access of
// that kernel -- the gather's stores to four XOR-permuted rows, the radix-8
// passes, the row reads -- at the minimum of four wavefronts of 16-byte
// elements (checked on a model of all its access patterns), where the
// make_smem layout took 12 for the gather and 8 for the first pass.
template <int LS, int PS, int RS>
struct FxLayout {
    static constexpr int kRs = RS;
    __device__ static __forceinline__ int idx(int f)
    {
        const int col = f & ((1 << LS) - 1);
        return (f >> LS) * RS + col + (col >> PS);
    }
};
template <int LS>
using FxLay = FxLayout<LS, 4, (1 << LS) + (1 << LS) / 16 + 1>;
using FxLayGather = FxLayout<9, 3, 580>;

// Radix-2^NB butterflies over bits [B, B + NB) of a tile of 2^LOGE values.
template <int NB, int B, int LOGE, typename Lay>
__device__ __forceinline__ void fx_pass_c(const FxTile& s)
{
    constexpr int kGroups = 1 << (LOGE - NB);
    static_assert(kGroups % kFxThreads == 0, "whole groups per thread");
#pragma unroll 1
    for (int q = threadIdx.x; q < kGroups; q += kFxThreads) {
        const int base = (q & ((1 << B) - 1)) | ((q >> B) << (B + NB));
        fx2 v[1 << NB];
#pragma unroll
        for (int j = 0; j < (1 << NB); ++j) v[j] = s.get(Lay::idx(base + (j << B)));
#pragma unroll
        for (int h = 1; h < (1 << NB); h <<= 1)
#pragma unroll
            for (int i = 0; i < (1 << NB); ++i)
                if (!(i & h)) {
                    const fx2 a = v[i], c = v[i + h];
                    v[i] = cadd(a, c);
                    v[i + h] = csub(a, c);
                }
#pragma unroll
        for (int j = 0; j < (1 << NB); ++j) s.put(Lay::idx(base + (j << B)), v[j]);
    }
}

// Bits [B0, B1) in radix-8 passes (the last one narrower), a barrier after each.
template <int B0, int B1, int LOGE, typename Lay>
__device__ __forceinline__ void fx_bits_c(const FxTile& s)
{
    if constexpr (B0 < B1) {
        constexpr int NB = B1 - B0 < 3 ? B1 - B0 : 3;
        fx_pass_c<NB, B0, LOGE, Lay>(s);
        __syncthreads();
        fx_bits_c<B0 + NB, B1, LOGE, Lay>(s);
    }
}

// First pass of a chunk: 2^LR masks x 2^LL values gathered from A (row view,
// as load_gather), transformed over the LL low bits, stored as fixed-point
// rows of the intermediate.
template <typename InT, int LR, int LL>
__global__ void __launch_bounds__(kFxThreads, 2) k_fx_tile_c(FxLaunch p, unsigned int* st)
{
    constexpr int kE = 1 << (LR + LL), kPer = kE / kFxThreads, kR = 1 << LR, kL = 1 << LL;
    static_assert(LR == 2 && LL == 9, "the gather layout is laid out for 4 x 512 tiles");
    using Lay = FxLayGather;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    i128* const plane = reinterpret_cast<i128*>(smem_raw);
    const FxTile s{plane, plane + kR * Lay::kRs};
    const int n = p.n, t = threadIdx.x;
    const int segs_log = n - LL;
    const uint32_t blk = blockIdx.x >> segs_log, seg = blockIdx.x & ((1u << segs_log) - 1);
    const uint32_t x0 = (uint32_t)p.x_begin + (blk << LR), k0 = seg << LL;
    const uint32_t rb = (k0 ^ x0) & ~(uint32_t)(kL - 1);
    const int S = fx_shift(p);
    const InT* A = (const InT*)p.src;
    InT v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        // row r of A supplies the aligned block of 2^LR columns r ^ x
        const int e = t + u * kFxThreads;
        const uint32_t r = rb + (uint32_t)(e >> LR);
        const uint32_t c = ((r ^ x0) & ~(uint32_t)(kR - 1)) + (uint32_t)(e & (kR - 1));
        const uint32_t gi = (r << n) + c;
        v[u] = __ldg(A + (in_bounds(st, gi, p.src_elems) ? gi : 0));
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = t + u * kFxThreads;
        const uint32_t r = rb + (uint32_t)(e >> LR);
        const uint32_t c = ((r ^ x0) & ~(uint32_t)(kR - 1)) + (uint32_t)(e & (kR - 1));
        s.put(Lay::idx((int)(((r ^ c) - x0) << LL) + (int)(c - k0)), in_of<InT>::cvt(v[u], S));
    }
    __syncthreads();
    fx_bits_c<0, LL, LR + LL, Lay>(s);
    fx2* dst = (fx2*)p.dst;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = t + u * kFxThreads;
        const uint32_t x = x0 + (uint32_t)(e >> LL), z = k0 + (uint32_t)(e & (kL - 1));
        const uint32_t gi = ((x - (uint32_t)p.dst_row0) << n) + z;
        if (in_bounds(st, gi, p.dst_elems)) dst[gi] = s.get(Lay::idx(e));
    }
}

// The strided pass that finishes a chunk: per mask and chunk of 2^LW low
// columns, bits [b0, b0 + NB) = [n - NB, n), then the phase, the scale and the
// rounding to the output type.
template <typename OutT, int NB, int LW>
__global__ void __launch_bounds__(kFxThreads, 2) k_fx_strided_c(FxLaunch p, unsigned int* st)
{
    constexpr int kE = 1 << (NB + LW), kPer = kE / kFxThreads, kW = 1 << LW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FxTile s = fx_tile(smem_raw, 1 << NB, LW);
    const int n = p.n, b0 = n - NB, t = threadIdx.x;
    const int chunks_log = b0 - LW;
    const uint32_t chunk = blockIdx.x & ((1u << chunks_log) - 1);
    const uint32_t x = (uint32_t)p.x_begin + (blockIdx.x >> chunks_log);
    const uint32_t kbase = chunk << LW;
    const fx2* src = (const fx2*)p.src + ((size_t)(x - (uint32_t)p.src_row0) << n);
    fx2 v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = t + u * kFxThreads;
        const uint32_t k = kbase + ((uint32_t)(e >> LW) << b0) + (uint32_t)(e & (kW - 1));
        v[u] = src[in_bounds(st, ((uint64_t)(x - (uint32_t)p.src_row0) << n) + k, p.src_elems) ? k : 0];
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) s.put(FxLay<LW>::idx(t + u * kFxThreads), v[u]);
    __syncthreads();
    fx_bits_c<LW, LW + NB, NB + LW, FxLay<LW>>(s);
    const int S = fx_shift(p);
    const FxOut o = fx_out(p, S);
    OutT* dst = (OutT*)p.dst;
#pragma unroll 2
    for (int u = 0; u < kPer; ++u) {
        const int e = t + u * kFxThreads;
        const uint32_t k = kbase + ((uint32_t)(e >> LW) << b0) + (uint32_t)(e & (kW - 1));
        const uint32_t gi = ((x - (uint32_t)p.dst_row0) << n) + k;
        if (in_bounds(st, gi, p.dst_elems)) dst[gi] = out_of<OutT>::cvt(s.get(FxLay<LW>::idx(e)), __popc(x & k) & 3, o);
    }
}

// ------------------------------------------------------------------ launch

template <typename K>
cudaError_t fx_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename InT, typename OutT, Load LD, Store ST>
cudaError_t run_fx_tile(const FxLaunch& p, unsigned int* st, cudaStream_t s)
{
    auto kern = k_fx_tile<InT, OutT, LD, ST>;
    const size_t bytes = smem_elems((size_t)1 << p.log_r, p.log_l) * sizeof(fx2);
    cudaError_t e = fx_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (p.x_count >> p.log_r) << (p.n - p.log_l);
    kern<<<(unsigned)blocks, kFxThreads, bytes, s>>>(p, st);
    return cudaGetLastError();
}

template <typename OutT, Store ST>
cudaError_t run_fx_strided(const FxLaunch& p, unsigned int* st, cudaStream_t s)
{
    auto kern = k_fx_strided<OutT, ST>;
    const size_t bytes = smem_elems((size_t)1 << (p.b1 - p.b0), p.log_w) * sizeof(fx2);
    cudaError_t e = fx_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = p.x_count << ((p.n - p.b1) + (p.b0 - p.log_w));
    kern<<<(unsigned)blocks, kFxThreads, bytes, s>>>(p, st);
    return cudaGetLastError();
}

// Dispatch on (input type, output type) for a given load/store pair.  The
// intermediate rows (Store::RowBuf) ignore the output type.
template <typename InT, Load LD, Store ST>
cudaError_t fx_tile_out(const FxLaunch& p, ptdr_dtype out_t, unsigned int* st, cudaStream_t s)
{
    if (ST == Store::RowBuf) return run_fx_tile<InT, float2, LD, ST>(p, st, s);
    switch (out_t) {
    case PTDR_C64: return run_fx_tile<InT, float2, LD, ST>(p, st, s);
    case PTDR_C128: return run_fx_tile<InT, double2, LD, ST>(p, st, s);
    case PTDR_F32:
        if constexpr (ST == Store::RowPhaseOut) return run_fx_tile<InT, float, LD, ST>(p, st, s);
        break;
    case PTDR_F64:
        if constexpr (ST == Store::RowPhaseOut) return run_fx_tile<InT, double, LD, ST>(p, st, s);
        break;
    }
    return cudaErrorInvalidValue;
}

template <Load LD, Store ST>
cudaError_t fx_tile_types(const FxLaunch& p, ptdr_dtype in_t, ptdr_dtype out_t, unsigned int* st, cudaStream_t s)
{
    switch (in_t) {
    case PTDR_C64: return fx_tile_out<float2, LD, ST>(p, out_t, st, s);
    case PTDR_C128: return fx_tile_out<double2, LD, ST>(p, out_t, st, s);
    case PTDR_F32: return fx_tile_out<float, LD, ST>(p, out_t, st, s);
    case PTDR_F64: return fx_tile_out<double, LD, ST>(p, out_t, st, s);
    }
    return cudaErrorInvalidValue;
}

template <Store ST>
cudaError_t fx_strided_types(const FxLaunch& p, ptdr_dtype out_t, unsigned int* st, cudaStream_t s)
{
    if (ST == Store::RowBuf) return run_fx_strided<float2, ST>(p, st, s);
    switch (out_t) {
    case PTDR_C64: return run_fx_strided<float2, ST>(p, st, s);
    case PTDR_C128: return run_fx_strided<double2, ST>(p, st, s);
    case PTDR_F32:
        if constexpr (ST == Store::RowPhaseOut) return run_fx_strided<float, ST>(p, st, s);
        break;
    case PTDR_F64:
        if constexpr (ST == Store::RowPhaseOut) return run_fx_strided<double, ST>(p, st, s);
        break;
    }
    return cudaErrorInvalidValue;
}

template <typename InT>
cudaError_t run_fx_tile_c(const FxLaunch& p, unsigned int* st, cudaStream_t s)
{
    auto kern = k_fx_tile_c<InT, 2, 9>;
    const size_t bytes = (size_t)4 * FxLayGather::kRs * sizeof(fx2); // two planes of 4 rows
    cudaError_t e = fx_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (p.x_count >> 2) << (p.n - 9);
    kern<<<(unsigned)blocks, kFxThreads, bytes, s>>>(p, st);
    return cudaGetLastError();
}

template <typename OutT, int NB, int LW>
cudaError_t run_fx_strided_c(const FxLaunch& p, unsigned int* st, cudaStream_t s)
{
    auto kern = k_fx_strided_c<OutT, NB, LW>;
    const size_t bytes = smem_elems((size_t)1 << NB, LW) * sizeof(fx2);
    cudaError_t e = fx_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = p.x_count << (p.n - NB - LW);
    kern<<<(unsigned)blocks, kFxThreads, bytes, s>>>(p, st);
    return cudaGetLastError();
}

template <typename OutT>
cudaError_t fx_strided_c_shape(const FxLaunch& p, unsigned int* st, cudaStream_t s)
{
    const int nb = p.b1 - p.b0;
    if (nb == 4 && p.log_w == 7) return run_fx_strided_c<OutT, 4, 7>(p, st, s);
    if (nb == 5 && p.log_w == 6) return run_fx_strided_c<OutT, 5, 6>(p, st, s);
    if (nb == 6 && p.log_w == 5) return run_fx_strided_c<OutT, 6, 5>(p, st, s);
    return cudaErrorInvalidValue;
}

cudaError_t fx_strided_c_types(const FxLaunch& p, ptdr_dtype out_t, unsigned int* st, cudaStream_t s)
{
    switch (out_t) {
    case PTDR_C64: return fx_strided_c_shape<float2>(p, st, s);
    case PTDR_C128: return fx_strided_c_shape<double2>(p, st, s);
    case PTDR_F32: return fx_strided_c_shape<float>(p, st, s);
    case PTDR_F64: return fx_strided_c_shape<double>(p, st, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t fx_tile_c_types(const FxLaunch& p, ptdr_dtype in_t, unsigned int* st, cudaStream_t s)
{
    switch (in_t) {
    case PTDR_C64: return run_fx_tile_c<float2>(p, st, s);
    case PTDR_C128: return run_fx_tile_c<double2>(p, st, s);
    case PTDR_F32: return run_fx_tile_c<float>(p, st, s);
    case PTDR_F64: return run_fx_tile_c<double>(p, st, s);
    }
    return cudaErrorInvalidValue;
}

// The decompose plans the compile-time kernels cover: 4 masks x 512 values
// in the first pass, then one strided pass over the remaining bits with the
// (bits, columns) shapes of n = 13, 14, 15.
bool fx_shapes_c(const DensePlan& plan)
{
    if (plan.compose || plan.single || plan.log_r != 2 || plan.log_l != 9 || plan.passes.size() != 1) return false;
    const StridedPass& q = plan.passes[0];
    const int nb = q.b1 - q.b0;
    return q.b0 == 9 && q.b1 == plan.n &&
           ((nb == 4 && q.log_w == 7) || (nb == 5 && q.log_w == 6) || (nb == 6 && q.log_w == 5));
}

} // namespace

size_t fixed_ws_header() { return 256; }

// The whole fixed-point decompose / compose of one matrix: the exponent
// pre-pass over the input, then single tile passes (rows that fit) or, per
// chunk of masks, a first pass into the intermediate and strided passes.
cudaError_t launch_fixed(const DensePlan& plan, const void* in, void* out, void* ws, double scale, unsigned int* st,
                         cudaStream_t s)
{
    const uint64_t N = 1ull << plan.n;
    int* emax = (int*)ws;
    cudaError_t e = cudaMemsetAsync(ws, 0, fixed_ws_header(), s);
    if (e != cudaSuccess) return e;
    const bool in64 = plan.in_t == PTDR_C128 || plan.in_t == PTDR_F64;
    {
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        const uint64_t words = (dtype_complex(plan.in_t) ? 2 : 1) * N * N;
        const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)sms * 8, std::max<uint64_t>(1, words / 256));
        if (in64)
            k_fx_maxexp<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)in, words, emax, st);
        else
            k_fx_maxexp<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)in, words, emax, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    FxLaunch p{};
    p.n = plan.n;
    p.emax = emax;
    p.bias = in64 ? 1023 : 127;
    // output value = X 2^-S times 2^-n (decompose) or times the compose scale
    if (!plan.compose) {
        p.q_pow = -plan.n;
    } else {
        int ex = 0;
        const double m = std::frexp(scale, &ex);
        if (m == 0.5 || m == -0.5) {
            p.q_pow = ex - 1;
            p.use_mul = m < 0;
            p.mul = -1.0;
        } else {
            p.q_pow = 0;
            p.use_mul = true;
            p.mul = scale;
        }
    }
    const Load ld = plan.compose ? Load::RowPhaseC : Load::GatherA;
    if (plan.single) {
        p.src = in;
        p.dst = out;
        p.log_r = plan.log_r;
        p.log_l = plan.log_l;
        p.x_begin = 0;
        p.x_count = N;
        p.src_elems = p.dst_elems = N * N;
        if (plan.compose) return fx_tile_types<Load::RowPhaseC, Store::ScatterA>(p, plan.in_t, plan.out_t, st, s);
        return fx_tile_types<Load::GatherA, Store::RowPhaseOut>(p, plan.in_t, plan.out_t, st, s);
    }
    fx2* buf = (fx2*)((char*)ws + fixed_ws_header());
    for (uint64_t x0 = 0; x0 < N && e == cudaSuccess; x0 += plan.chunk) {
        FxLaunch t = p;
        t.src = in;
        t.dst = buf;
        t.load = ld;
        t.store = Store::RowBuf;
        t.log_r = plan.log_r;
        t.log_l = plan.log_l;
        t.x_begin = x0;
        t.x_count = plan.chunk;
        t.dst_row0 = x0;
        t.src_row0 = 0;
        t.src_elems = N * N;
        t.dst_elems = plan.chunk * N;
        const bool shaped = fx_shapes_c(plan);
        e = plan.compose ? fx_tile_types<Load::RowPhaseC, Store::RowBuf>(t, plan.in_t, plan.out_t, st, s)
            : shaped     ? fx_tile_c_types(t, plan.in_t, st, s)
                         : fx_tile_types<Load::GatherA, Store::RowBuf>(t, plan.in_t, plan.out_t, st, s);
        for (size_t i = 0; i < plan.passes.size() && e == cudaSuccess; ++i) {
            const bool last = i + 1 == plan.passes.size();
            FxLaunch q = p;
            q.src = buf;
            q.b0 = plan.passes[i].b0;
            q.b1 = plan.passes[i].b1;
            q.log_w = plan.passes[i].log_w;
            q.x_begin = x0;
            q.x_count = plan.chunk;
            q.src_row0 = x0;
            q.src_elems = plan.chunk * N;
            if (!last) {
                q.dst = buf;
                q.dst_row0 = x0;
                q.dst_elems = plan.chunk * N;
                e = fx_strided_types<Store::RowBuf>(q, plan.out_t, st, s);
            } else {
                q.dst = out;
                q.dst_row0 = 0;
                q.dst_elems = N * N;
                e = plan.compose ? fx_strided_types<Store::ScatterA>(q, plan.out_t, st, s)
                    : shaped     ? fx_strided_c_types(q, plan.out_t, st, s)
                                 : fx_strided_types<Store::RowPhaseOut>(q, plan.out_t, st, s);
            }
        }
    }
    return e;
}

} // namespace ptdr
