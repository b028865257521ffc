// Fast path for one whole transform row per CTA: n = 14 (2^14 complex
// values, 128 KiB in float32), one CTA per mask x, 512 threads.
//
// The XOR-diagonal gather d_x[k] = A[k^x][k] takes one 8-byte element from
// each of the 2^14 rows of A.  The 32-byte sector that holds it also holds
// the elements of the three sibling masks x^1, x^2, x^3, which the
// neighbouring CTAs (consecutive blockIdx, resident at the same time) read
// moments later, so L2 serves them and HBM sees A read about once.
//
// The length-2^14 Walsh-Hadamard transform runs as three register rounds of
// 5, 5 and 4 bits with two shared-memory exchanges between them:
//   A: thread t gathers k = 32t + j (j < 32) straight into registers (32
//      independent loads in flight per thread) and transforms bits 0-4;
//   B: bits 5-9 (stride 32);
//   C: bits 10-13 (stride 1024), then the phase (-i)^{|x&z|}, the exact
//      2^-14 scale and the store of z = q + 1024 j, contiguous across the warp.
// Shared-memory index k + (k >> 5) (one pad element per 32) keeps every
// round's accesses at the minimum number of wavefronts.
#include "common.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kLog = 14;
constexpr int kN = 1 << kLog;
constexpr int kThreads = 512;
constexpr int kSmemElems = kN + kN / 32;

__device__ __forceinline__ int pad32(int k) { return k + (k >> 5); }

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

template <typename InT>
__device__ __forceinline__ float2 ld_in(const InT* p);
template <> __device__ __forceinline__ float2 ld_in<float2>(const float2* p) { return __ldg(p); }
template <> __device__ __forceinline__ float2 ld_in<double2>(const double2* p)
{
    double2 v = __ldg(p);
    return make_float2((float)v.x, (float)v.y);
}
// a real matrix enters with a zero imaginary part
template <> __device__ __forceinline__ float2 ld_in<float>(const float* p) { return make_float2(__ldg(p), 0.f); }
template <> __device__ __forceinline__ float2 ld_in<double>(const double* p) { return make_float2((float)__ldg(p), 0.f); }

template <typename OutT>
__device__ __forceinline__ void st_out(OutT* p, float2 v);
template <> __device__ __forceinline__ void st_out<float2>(float2* p, float2 v) { __stcs(p, v); }
template <> __device__ __forceinline__ void st_out<double2>(double2* p, float2 v)
{
    __stcs(p, make_double2((double)v.x, (double)v.y));
}
// real outputs store the real part (Hermitian A: all of c, Thm 2)
template <> __device__ __forceinline__ void st_out<float>(float* p, float2 v) { __stcs(p, v.x); }
template <> __device__ __forceinline__ void st_out<double>(double* p, float2 v) { __stcs(p, (double)v.x); }

} // namespace

template <typename InT, typename OutT>
__global__ void __launch_bounds__(kThreads, 1)
    k_row14(const InT* __restrict__ A, OutT* __restrict__ C, uint64_t x_begin, unsigned int* st)
{
    extern __shared__ __align__(16) float2 s[];
    const int t = threadIdx.x;
    const uint64_t x = x_begin + blockIdx.x;
    const uint64_t lim = (uint64_t)kN * kN;

    // Round A: gather 32 consecutive k into registers, transform bits 0-4.
    float2 v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint64_t k = (uint64_t)(32 * t + j);
        const uint64_t gi = ((k ^ x) << kLog) + k;
        v[j] = in_bounds(st, gi, lim) ? ld_in(A + gi) : make_float2(0.f, 0.f);
    }
    wht_regs<5>(v);
#pragma unroll
    for (int j = 0; j < 32; ++j) s[pad32(32 * t + j)] = v[j];
    __syncthreads();

    // Round B: bits 5-9.
    {
        const int base = (t & 31) | ((t >> 5) << 10);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = s[pad32(base + 32 * j)];
        wht_regs<5>(v);
#pragma unroll
        for (int j = 0; j < 32; ++j) s[pad32(base + 32 * j)] = v[j];
    }
    __syncthreads();

    // Round C: bits 10-13 for groups q = t and q = t + 512, then write out.
    const float scale = 1.0f / (float)kN;
    OutT* row = C + (x << kLog);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int q = t + g * kThreads;
        float2 w[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) w[j] = s[pad32(q + 1024 * j)];
        wht_regs<4>(w);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint64_t z = (uint64_t)(q + 1024 * j);
            const float2 c = phase_neg_i(w[j], (int)(__popcll(x & z) & 3), scale);
            if (in_bounds(st, (x << kLog) + z, lim)) st_out(row + z, c);
        }
    }
}

template <typename InT, typename OutT>
static cudaError_t run_row14(const void* A, void* C, unsigned int* st, cudaStream_t s)
{
    auto kern = k_row14<InT, OutT>;
    const int bytes = kSmemElems * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    kern<<<kN, kThreads, bytes, s>>>((const InT*)A, (OutT*)C, 0, st);
    return cudaGetLastError();
}

cudaError_t launch_row14(const void* A, ptdr_dtype a_t, void* C, ptdr_dtype c_t, unsigned int* st,
                         cudaStream_t s)
{
    auto by_out = [&](auto in_tag) -> cudaError_t {
        using InT = decltype(in_tag);
        switch (c_t) {
        case PTDR_C64: return run_row14<InT, float2>(A, C, st, s);
        case PTDR_C128: return run_row14<InT, double2>(A, C, st, s);
        case PTDR_F32: return run_row14<InT, float>(A, C, st, s);
        case PTDR_F64: return run_row14<InT, double>(A, C, st, s);
        }
        return cudaErrorInvalidValue;
    };
    switch (a_t) {
    case PTDR_C64: return by_out(float2{});
    case PTDR_C128: return by_out(double2{});
    case PTDR_F32: return by_out(float{});
    case PTDR_F64: return by_out(double{});
    }
    return cudaErrorInvalidValue;
}

} // namespace ptdr
