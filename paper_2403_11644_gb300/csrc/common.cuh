// Shared device-side helpers for the libptdr kernels (sm_103a).
//
// Notation (Sec. II.B of the paper, PauliComposer): operator P_{x,z} with
// x_l = d(sigma_l) and z_l = 1 for Y/Z; qubit l <-> index bit l.  On the GPU
// each mask x is handled as
//     d_x[k]   = A[k XOR x][k]                       (XOR-diagonal gather)
//     w_x      = WHT(d_x)        (length-2^n Walsh-Hadamard transform over k)
//     c_{x,z}  = 2^-n (-i)^{|x&z|} w_x[z]
// which is the O(2^n) sparse trace of Sec. II.A with the nonzero of row j
// of P at column j XOR x and value i^{|x&z|} (-1)^{|z&(j XOR x)|}; substituting
// k = j and taking (-1)^{|z&x|} out of the sign leaves the transform above.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ptdr_internal.h"

namespace ptdr {

// ---------------------------------------------------------------- complex

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx_of<T>::type;

template <typename T> __device__ __forceinline__ cplx_t<T> mk(T re, T im)
{
    cplx_t<T> v;
    v.x = re;
    v.y = im;
    return v;
}

template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b)
{
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b)
{
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
// Real rows (transforms of real data): plain scalar butterflies.
__device__ __forceinline__ float cadd(float a, float b) { return a + b; }
__device__ __forceinline__ float csub(float a, float b) { return a - b; }
__device__ __forceinline__ double cadd(double a, double b) { return a + b; }
__device__ __forceinline__ double csub(double a, double b) { return a - b; }

// Multiply by (-i)^p (p taken mod 4) and by a real scale without a complex
// multiply or a branch: an odd p swaps the real and imaginary parts, the real
// part changes sign for p = 2, 3 and the imaginary part for p = 1, 2.  (Lanes
// of a warp hold different p, so a switch here would diverge four ways.)
template <typename T2, typename T>
__device__ __forceinline__ T2 phase_neg_i(T2 v, int p, T s)
{
    const bool odd = (p & 1) != 0;
    const T u = odd ? v.y : v.x;
    const T w = odd ? v.x : v.y;
    const T sr = (p & 2) ? -s : s;
    const T si = ((p ^ (p >> 1)) & 1) ? -s : s;
    T2 r;
    r.x = u * sr;
    r.y = w * si;
    return r;
}

// ------------------------------------------------------------ I/O element

// Element types as stored in HBM.  Complex values are 8 or 16 bytes; real
// band inputs are promoted to complex with a zero imaginary part.
template <typename E> struct io;
template <> struct io<float2> {
    template <typename T> __device__ static __forceinline__ cplx_t<T> ld(const float2* p)
    {
        float2 v = __ldg(p);
        return mk<T>((T)v.x, (T)v.y);
    }
    template <typename T2> __device__ static __forceinline__ void st(float2* p, T2 v)
    {
        *p = make_float2((float)v.x, (float)v.y);
    }
};
template <> struct io<double2> {
    template <typename T> __device__ static __forceinline__ cplx_t<T> ld(const double2* p)
    {
        double2 v = __ldg(p);
        return mk<T>((T)v.x, (T)v.y);
    }
    template <typename T2> __device__ static __forceinline__ void st(double2* p, T2 v)
    {
        *p = make_double2((double)v.x, (double)v.y);
    }
};
template <> struct io<float> {
    template <typename T> __device__ static __forceinline__ cplx_t<T> ld(const float* p)
    {
        return mk<T>((T)__ldg(p), (T)0);
    }
    template <typename T2> __device__ static __forceinline__ void st(float* p, T2 v)
    {
        *p = (float)v.x;
    }
};
template <> struct io<double> {
    template <typename T> __device__ static __forceinline__ cplx_t<T> ld(const double* p)
    {
        return mk<T>((T)__ldg(p), (T)0);
    }
    template <typename T2> __device__ static __forceinline__ void st(double* p, T2 v)
    {
        *p = (double)v.x;
    }
};

// ------------------------------------------------------------ status word

// One 32-bit word per device (defined in the API translation unit, its
// address passed to every kernel), written by kernels that detect an error:
// a bounded wait that ran out, a failed index check in a checked build.
// The first error wins; the host reads and clears it.
__device__ __forceinline__ void report_status(unsigned int* status, unsigned int s)
{
    atomicCAS(status, 0u, s);
}

// In a checked build (-DPTDR_CHECKED) every computed global index is
// range-checked before use: an index out of range records PTDR_ERR_INTERNAL
// and the access is skipped (no early return, so barriers stay balanced).
__device__ __forceinline__ bool in_bounds(unsigned int* status, unsigned long long idx,
                                          unsigned long long limit)
{
#ifdef PTDR_CHECKED
    if (idx >= limit) {
        report_status(status, PTDR_ERR_INTERNAL);
        return false;
    }
#else
    (void)status;
    (void)idx;
    (void)limit;
#endif
    return true;
}

} // namespace ptdr
