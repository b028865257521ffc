// Dense decomposition of one complex64 matrix of n = 9 .. 12 into complex64
// coefficients, computed in FP32: one CTA per register-round item (R =
// 2^(13-n) masks), 3 CTAs of 256 threads per SM.  A and C 16-byte aligned
// (checked by the planner).
#include "plan.h"
#include "rr_items.cuh"

namespace ptdr {

template <int NQ>
__global__ void __launch_bounds__(256, 3) k_rr_dense(const float2* __restrict__ A, float2* __restrict__ C,
                                                     float scale, unsigned int* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s = reinterpret_cast<float2*>(smem_raw);
    rr_item<NQ>(A, C, (uint32_t)blockIdx.x << RrShape<NQ>::LR, s, scale, st);
}

template <int NQ>
static cudaError_t run_rr(const void* A, void* C, double scale, unsigned int* st, cudaStream_t s)
{
    auto kern = k_rr_dense<NQ>;
    const int bytes = kRrElems * (int)sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    const unsigned items = 1u << (2 * NQ - 13); // 2^n masks, R per item
    kern<<<items, 256, bytes, s>>>((const float2*)A, (float2*)C, (float)scale, st);
    return cudaGetLastError();
}

cudaError_t launch_rr_dense(int n, const void* A, void* C, double scale, unsigned int* st, cudaStream_t s)
{
    switch (n) {
    case 9: return run_rr<9>(A, C, scale, st, s);
    case 10: return run_rr<10>(A, C, scale, st, s);
    case 11: return run_rr<11>(A, C, scale, st, s);
    case 12: return run_rr<12>(A, C, scale, st, s);
    }
    return cudaErrorInvalidValue;
}

} // namespace ptdr
