// Conversions between IEEE binary32/binary64 values and 128-bit two's-
// complement fixed point, done on the integer bit fields (no floating-point
// arithmetic), for the exact fixed-point transform path.  Host and device
// code share them so that a host program can check them exhaustively on the
// edge cases (ties, subnormals, carries into the exponent).
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define PTDR_HD __host__ __device__ __forceinline__
#else
#define PTDR_HD inline
#endif

namespace ptdr {
namespace fxp {

using i128 = __int128;
using u128 = unsigned __int128;

PTDR_HD uint32_t bits_of(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
#endif
}

PTDR_HD uint64_t bits_of(double d)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    memcpy(&b, &d, 8);
    return b;
#endif
}

PTDR_HD int clz64(uint64_t v)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// Two's-complement negation of the 128-bit value (hi, lo) in place.
PTDR_HD void neg128(uint64_t& hi, uint64_t& lo)
{
    lo = ~lo + 1;
    hi = ~hi + (lo == 0 ? 1 : 0);
}

// X = round(m 2^(p + S)) with the given sign, m < 2^53 (ties away from zero on
// the magnitude; only digits below the fixed-point resolution are rounded).
// Built from 64-bit words: m 2^sh spans at most two of them.
PTDR_HD i128 fixed_of(uint64_t m, int p, bool neg, int S)
{
    const int sh = p + S;
    uint64_t hi = 0, lo = 0;
    if (m == 0 || sh <= -64 || sh >= 128) { // sh >= 128 would need |X| >= 2^128: only m = 0
    } else if (sh < 0) {
        lo = (m + (1ull << (-sh - 1))) >> (-sh);
    } else if (sh < 64) {
        lo = m << sh;
        hi = sh ? m >> (64 - sh) : 0;
    } else {
        hi = m << (sh - 64);
    }
    if (neg) neg128(hi, lo);
    return (i128)(((u128)hi << 64) | lo);
}

// round(v 2^S) for a binary32 value: significand m (implicit bit added for
// normal numbers) and exponent p with v = m 2^p.
PTDR_HD i128 fixed_of(float f, int S)
{
    const uint32_t b = bits_of(f);
    const uint32_t ef = (b >> 23) & 0xFFu, fr = b & 0x7FFFFFu;
    return fixed_of(ef ? (uint64_t)(fr | 0x800000u) : (uint64_t)fr, ef ? (int)ef - 150 : -149, (b >> 31) != 0, S);
}

// round(v 2^S) for a binary64 value.
PTDR_HD i128 fixed_of(double d, int S)
{
    const uint64_t b = bits_of(d);
    const uint32_t ef = (uint32_t)(b >> 52) & 0x7FFu;
    const uint64_t fr = b & 0xFFFFFFFFFFFFFull;
    return fixed_of(ef ? (fr | (1ull << 52)) : fr, ef ? (int)ef - 1075 : -1074, (b >> 63) != 0, S);
}

// IEEE bits (sign included) of X 2^q rounded to nearest even, for a format
// with MB significand bits (implicit bit included), exponent bias BIAS and
// all-ones exponent field EFMAX.  The magnitude is first normalised into a
// 64-bit window (leading one at bit 63) plus a sticky flag for any one below
// the window, so that the rounding works on 64-bit words.  Subnormal results
// keep fewer significand bits; an exponent above the range gives infinity.
// Adding the significand (implicit bit included) to (field - 1) << (MB - 1)
// lets a rounding carry move into the exponent field.
template <int MB, int BIAS, int EFMAX, int SIGN>
PTDR_HD uint64_t ieee_of(i128 X, int q)
{
    uint64_t hi = (uint64_t)((u128)X >> 64), lo = (uint64_t)X;
    const bool neg = (int64_t)hi < 0;
    if (neg) neg128(hi, lo);
    int msb;
    uint64_t top;
    bool sticky;
    if (hi) {
        const int l = clz64(hi);
        msb = 127 - l;
        top = l ? (hi << l) | (lo >> (64 - l)) : hi;
        sticky = (l ? lo << l : lo) != 0;
    } else if (lo) {
        const int l = clz64(lo);
        msb = 63 - l;
        top = lo << l;
        sticky = false;
    } else {
        return 0;
    }
    int ef = msb + q + BIAS;  // biased exponent of the leading bit
    int drop = 64 - MB;       // window bits below the significand
    if (ef < 1) {             // subnormal: the significand loses 1 - ef bits
        drop += 1 - ef;
        ef = 0;
    }
    uint64_t mant;
    if (drop >= 64) { // the whole window is below the last place: 0, or 1 above one half
        mant = (drop == 64 && (top > (1ull << 63) || (top == (1ull << 63) && sticky))) ? 1 : 0;
    } else {
        mant = top >> drop;
        const uint64_t rem = top & ((1ull << drop) - 1), half = 1ull << (drop - 1);
        if (rem > half || (rem == half && (sticky || (mant & 1)))) ++mant;
    }
    uint64_t bits = ef >= 1 ? ((uint64_t)(ef - 1) << (MB - 1)) + mant : mant;
    const uint64_t inf = (uint64_t)EFMAX << (MB - 1);
    if (ef >= EFMAX || bits > inf) bits = inf;
    return bits | ((uint64_t)neg << SIGN);
}

PTDR_HD uint64_t f64_bits(i128 X, int q) { return ieee_of<53, 1023, 2047, 63>(X, q); }
PTDR_HD uint32_t f32_bits(i128 X, int q) { return (uint32_t)ieee_of<24, 127, 255, 31>(X, q); }

} // namespace fxp
} // namespace ptdr
