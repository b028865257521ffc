// Host check of the IEEE <-> 128-bit fixed-point conversions of the exact
// fixed-point path (paper_2403_11644_gb300/csrc/fixed_point.cuh), built with
// g++ by tests/test_fixed_point_host.py.  References come from other routes:
// the compiler's own correctly rounded __int128 -> double/float conversion
// with ldexp for normal results, plain integer rounding for subnormal ones,
// and exact integer arithmetic for the float -> fixed direction.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../paper_2403_11644_gb300/csrc/fixed_point.cuh"

using ptdr::fxp::i128;
using ptdr::fxp::u128;

static int failures = 0;

static void fail(const char* what, double a, double b)
{
    if (++failures <= 10) std::printf("FAIL %s: got %.17g want %.17g\n", what, a, b);
}

static double as_double(uint64_t b)
{
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}

static float as_float(uint32_t b)
{
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

// round-half-even of |X| / 2^shift (shift >= 1), sign restored
static i128 round_shift_even(i128 X, int shift)
{
    const bool neg = X < 0;
    u128 u = neg ? (u128)(-X) : (u128)X;
    if (shift >= 128) return 0;
    u128 q = u >> shift, r = u - (q << shift), h = (u128)1 << (shift - 1);
    if (r > h || (r == h && (q & 1))) ++q;
    return neg ? -(i128)q : (i128)q;
}

int main()
{
    std::mt19937_64 rng(12345);
    // 1. exact round trips: IEEE -> fixed -> IEEE with no bits below the resolution
    for (int t = 0; t < 200000; ++t) {
        const int e = (int)(rng() % 200) - 100;
        const double v = std::ldexp((double)(rng() >> 11) / 9007199254740992.0, e) * ((rng() & 1) ? -1 : 1);
        const int S = 120 - (e + 1); // |v| < 2^(e+1): |X| < 2^120, every significand bit kept
        const i128 X = ptdr::fxp::fixed_of(v, S);
        if (ptdr::fxp::f64_bits(X, -S) != ptdr::fxp::bits_of(v)) fail("double round trip", as_double(ptdr::fxp::f64_bits(X, -S)), v);
        const float f = (float)v;
        const i128 Y = ptdr::fxp::fixed_of(f, S);
        if (ptdr::fxp::f32_bits(Y, -S) != ptdr::fxp::bits_of(f)) fail("float round trip", as_float(ptdr::fxp::f32_bits(Y, -S)), f);
    }
    // subnormal and zero inputs
    for (double v : {0.0, -0.0, 4.9406564584124654e-324, -2.2250738585072009e-308, 1e-310}) {
        const int S = 1100;
        const i128 X = ptdr::fxp::fixed_of(v, S);
        if (ptdr::fxp::f64_bits(X, -S) != (ptdr::fxp::bits_of(v) & (v == 0 ? 0 : ~0ull))) fail("subnormal round trip", as_double(ptdr::fxp::f64_bits(X, -S)), v);
    }
    // 2. fixed -> double against the compiler's correctly rounded conversion
    for (int t = 0; t < 400000; ++t) {
        const int bits = 1 + (int)(rng() % 126);
        i128 X = (i128)(((u128)rng() << 64) | rng());
        X &= (((i128)1) << bits) - 1;
        if (rng() & 1) X = -X;
        if (t % 7 == 0) X = (X >> 20) << 20; // exact ties and short values
        const int q = (int)(rng() % 400) - 200;
        const double want = std::ldexp((double)X, q);
        const double got = as_double(ptdr::fxp::f64_bits(X, q));
        if (!(got == want && std::signbit(got) == std::signbit(want)) && !(X == 0 && got == 0)) fail("f64_bits", got, want);
        const float wantf = std::ldexp((float)X, q);
        if (std::isfinite(wantf) && std::fabs(wantf) >= 1.1754944e-38f) {
            const float gotf = as_float(ptdr::fxp::f32_bits(X, q));
            if (gotf != wantf) fail("f32_bits", gotf, wantf);
        }
    }
    // rounding carries into the exponent, overflow to infinity
    if (as_double(ptdr::fxp::f64_bits(((i128)1 << 54) - 1, 0)) != 18014398509481984.0) fail("carry", 0, 0);
    if (!std::isinf(as_double(ptdr::fxp::f64_bits(1, 1024)))) fail("overflow", 0, 0);
    if (as_double(ptdr::fxp::f64_bits(((i128)1 << 53) + 1, 0)) != 9007199254740992.0) fail("tie to even", 0, 0);
    if (as_double(ptdr::fxp::f64_bits(((i128)1 << 53) + 3, 0)) != 9007199254740996.0) fail("tie to even up", 0, 0);
    // half of the smallest subnormal: ties to even (zero), anything above rounds up,
    // also when the excess lies below the 64-bit window (sticky bit)
    if (ptdr::fxp::f64_bits(1, -1075) != 0) fail("half-min tie", 0, 0);
    if (ptdr::fxp::f64_bits(3, -1076) != 1) fail("above half-min", 0, 0);
    if (ptdr::fxp::f64_bits(((i128)1 << 70) + 1, -1145) != 1) fail("sticky above half-min", 0, 0);
    if (ptdr::fxp::f64_bits((i128)1 << 70, -1145) != 0) fail("exact half-min", 0, 0);
    if (ptdr::fxp::f64_bits(-(((i128)1 << 70) + 1), -1145) != (1ull | (1ull << 63))) fail("negative sticky", 0, 0);
    // 3. subnormal results: round-half-even of X 2^(q + 1074) in integers
    for (int t = 0; t < 100000; ++t) {
        const i128 X = (i128)(rng() >> (rng() % 60)) * ((rng() & 1) ? -1 : 1);
        const int q = -1074 - (int)(rng() % 70) - 1;
        const i128 R = round_shift_even(X, -(q + 1074)); // in units of 2^-1074
        const u128 mag = R < 0 ? (u128)(-R) : (u128)R;
        if (mag >= ((u128)1 << 52)) continue; // normal after rounding
        const uint64_t want = (uint64_t)mag | ((uint64_t)(X < 0) << 63);
        const uint64_t got = ptdr::fxp::f64_bits(X, q);
        if (got != want && !(mag == 0 && (got & ~(1ull << 63)) == 0)) fail("subnormal result", as_double(got), as_double(want));
    }
    // 4. IEEE -> fixed with bits below the resolution: nearest integer, ties away from zero
    for (int t = 0; t < 200000; ++t) {
        const double v = std::ldexp((double)(rng() >> 11), -(int)(rng() % 60)) * ((rng() & 1) ? -1 : 1);
        const int S = (int)(rng() % 40);
        // v 2^S = m 2^k exactly; round |m 2^k| to an integer in exact arithmetic
        const i128 X = ptdr::fxp::fixed_of(v, S);
        int ex;
        const double fr = std::frexp(std::fabs(v), &ex); // |v| = fr 2^ex, fr in [0.5, 1)
        const u128 m = (u128)std::ldexp(fr, 53);         // |v| = m 2^(ex - 53)
        const int k = ex - 53 + S;
        u128 want = k >= 0 ? (m << k) : (k <= -128 ? 0 : ((m + ((u128)1 << (-k - 1))) >> (-k)));
        const i128 w = v < 0 ? -(i128)want : (i128)want;
        if (v != 0 && X != w) fail("fixed_of rounding", (double)X, (double)w);
    }
    std::printf(failures ? "failures: %d\n" : "ok\n", failures);
    return failures ? 1 : 0;
}
