// Measurement helper: the FP64 add throughput of the device.  The FP64
// transforms of the library (the FP64 precision path, the band paths) are
// bound by the FP64 pipe; the benchmark measures that bound in the same run
// with this add chain instead of quoting a constant.
#include "common.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kChains = 8; // independent dependency chains per thread

// Each thread runs kChains independent chains of `iters` dependent adds; the
// increments differ per chain and thread, so nothing folds at compile time.
__global__ void k_fp64_add_chain(double* sink, int iters, double inc)
{
    double v[kChains];
    const double d = inc * (1.0 + 1e-9 * (double)threadIdx.x);
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (double)c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] += d;
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == -1.0) sink[blockIdx.x] = s; // never true; keeps the chains live
}

} // namespace

} // namespace ptdr

extern "C" ptdr_status ptdr_probe_fp64_adds(void* d_sink, int blocks, int threads, int iters, double* adds,
                                            void* stream)
{
    if (!d_sink || !adds || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1)
        return PTDR_ERR_INVALID_ARG;
    int dev = 0;
    ptdr_status v = ptdr::device_ready(&dev);
    if (v != PTDR_OK) return v;
    ptdr::k_fp64_add_chain<<<blocks, threads, 0, (cudaStream_t)stream>>>((double*)d_sink, iters, 1e-3);
    if (cudaGetLastError() != cudaSuccess) return PTDR_ERR_CUDA;
    *adds = (double)blocks * threads * (double)iters * ptdr::kChains;
    return PTDR_OK;
}
