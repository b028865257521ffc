// Decomposition algebra on coefficient arrays (Sec. IV.B, "Combinations of
// matrices"): the decomposition of a matrix built from others, computed from
// their decompositions without decomposing it again.
//
//   linear combination (Sec. IV.B.3):  c(mu A + B) = mu c(A) + c(B)
//   block-diagonal (Sec. IV.B.1-2):    diag(A_0, ..., A_{2^m-1}) = sum_i |i><i| (x) A_i
//       with |i><i| = 2^-m sum_t (-1)^{|t & i|} Z^t on the m top qubits, so
//       c[x][z + 2^n t] = 2^-m sum_i (-1)^{|t & i|} c(A_i)[x][z]  (x < 2^n),
//       0 for every mask x >= 2^n; m = 1 is the direct sum
//       A (+) B = I (x) (A + B)/2 + Z (x) (A - B)/2
//   Hermitian augmentation (Sec. IV.B.5): [[0, A^H], [A, 0]] =
//       X (x) sum Re(alpha_j) P_j + Y (x) sum Im(alpha_j) P_j
//
// All are streaming passes over HBM: one read of each input coefficient and
// one write of each output coefficient (the zero rows of the outputs are
// written by a separate 16-byte-store fill kernel), grids of a few CTAs per SM.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kMaxBlockLog = 4;

// Real / complex element access in the compute type (complex64 and float32
// data in float32, the double types in float64).
template <typename E> struct el;
template <> struct el<float2> {
    using T = float;
    __device__ static float2 ld(const float2* p, uint64_t i) { return __ldcs(p + i); }
    __device__ static void st(float2* p, uint64_t i, float re, float im) { __stcs(p + i, make_float2(re, im)); }
};
template <> struct el<double2> {
    using T = double;
    __device__ static double2 ld(const double2* p, uint64_t i) { return __ldcs(p + i); }
    __device__ static void st(double2* p, uint64_t i, double re, double im) { __stcs(p + i, make_double2(re, im)); }
};
template <> struct el<float> {
    using T = float;
    __device__ static float2 ld(const float* p, uint64_t i) { return make_float2(__ldcs(p + i), 0.f); }
    __device__ static void st(float* p, uint64_t i, float re, float) { __stcs(p + i, re); }
};
template <> struct el<double> {
    using T = double;
    __device__ static double2 ld(const double* p, uint64_t i) { return make_double2(__ldcs(p + i), 0.0); }
    __device__ static void st(double* p, uint64_t i, double re, double) { __stcs(p + i, re); }
};

unsigned grid_for(uint64_t work, int per_cta)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    const uint64_t want = (work + per_cta - 1) / per_cta;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 8));
}

// out = mu a + b (b may be absent), elementwise.
template <typename E>
__global__ void __launch_bounds__(256) k_lincomb(const E* __restrict__ a, const E* b, E* out, uint64_t count,
                                                 double mr, double mi)
{
    using T = typename el<E>::T;
    const T r = (T)mr, m = (T)mi;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const auto va = el<E>::ld(a, i);
        T re = r * va.x - m * va.y, im = r * va.y + m * va.x;
        if (b) {
            const auto vb = el<E>::ld(b, i);
            re += vb.x;
            im += vb.y;
        }
        el<E>::st(out, i, re, im);
    }
}

struct Blocks {
    const void* p[1 << kMaxBlockLog];
};

// Rows x < 2^n of the block-diagonal's coefficients: per (x, z) a length-2^m
// Walsh-Hadamard transform across the blocks, scaled by 2^-m (exact).
template <typename E, int M>
__global__ void __launch_bounds__(256) k_block_diag(Blocks blk, E* __restrict__ out, int n)
{
    using T = typename el<E>::T;
    constexpr int B = 1 << M;
    const uint64_t N = 1ull << n, count = N * N, W = N << M; // W = output row length
    const T sc = (T)1 / (T)B;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        T re[B], im[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const auto v = el<E>::ld((const E*)blk.p[j], i);
            re[j] = v.x;
            im[j] = v.y;
        }
#pragma unroll
        for (int h = 1; h < B; h <<= 1)
#pragma unroll
            for (int j = 0; j < B; ++j)
                if (!(j & h)) {
                    const T ar = re[j], ai = im[j];
                    re[j] = ar + re[j + h];
                    im[j] = ai + im[j + h];
                    re[j + h] = ar - re[j + h];
                    im[j + h] = ai - im[j + h];
                }
        const uint64_t x = i >> n, z = i & (N - 1);
#pragma unroll
        for (int t = 0; t < B; ++t) el<E>::st(out, x * W + (z | ((uint64_t)t << n)), re[t] * sc, im[t] * sc);
    }
}

// Rows 2^n .. 2^(n+1) - 1 of the augmented matrix's coefficients: the real
// parts under top-qubit X (z < 2^n), the imaginary parts under Y (z >= 2^n).
template <typename EA, typename E>
__global__ void __launch_bounds__(256) k_herm_aug(const EA* __restrict__ a, E* __restrict__ out, int n)
{
    const uint64_t N = 1ull << n, count = N * N, W = 2 * N;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const auto v = el<EA>::ld(a, i);
        const uint64_t x = i >> n, z = i & (N - 1);
        const uint64_t row = (x + N) * W;
        el<E>::st(out, row + z, (typename el<E>::T)v.x, 0);
        el<E>::st(out, row + z + N, (typename el<E>::T)v.y, 0);
    }
}

// Zero fill with 16-byte stores (the byte count is a multiple of 16).
__global__ void __launch_bounds__(256) k_zero16(uint4* p, uint64_t count)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        __stcs(p + i, make_uint4(0, 0, 0, 0));
}

cudaError_t zero_bytes(void* p, uint64_t bytes, cudaStream_t s)
{
    if (bytes == 0) return cudaSuccess;
    k_zero16<<<grid_for(bytes / 16, 256 * 8), 256, 0, s>>>((uint4*)p, bytes / 16);
    return cudaGetLastError();
}

template <typename E>
cudaError_t run_block_diag(const Blocks& blk, void* out, int n, int m, cudaStream_t s)
{
    const uint64_t count = 1ull << (2 * n);
    const unsigned g = grid_for(count, 256 * 4);
    switch (m) {
    case 1: k_block_diag<E, 1><<<g, 256, 0, s>>>(blk, (E*)out, n); break;
    case 2: k_block_diag<E, 2><<<g, 256, 0, s>>>(blk, (E*)out, n); break;
    case 3: k_block_diag<E, 3><<<g, 256, 0, s>>>(blk, (E*)out, n); break;
    default: k_block_diag<E, 4><<<g, 256, 0, s>>>(blk, (E*)out, n); break;
    }
    return cudaGetLastError();
}

template <typename EA>
cudaError_t run_herm_aug(const void* a, void* out, ptdr_dtype out_t, int n, cudaStream_t s)
{
    const uint64_t count = 1ull << (2 * n);
    const unsigned g = grid_for(count, 256 * 4);
    switch (out_t) {
    case PTDR_C64: k_herm_aug<EA, float2><<<g, 256, 0, s>>>((const EA*)a, (float2*)out, n); break;
    case PTDR_C128: k_herm_aug<EA, double2><<<g, 256, 0, s>>>((const EA*)a, (double2*)out, n); break;
    case PTDR_F32: k_herm_aug<EA, float><<<g, 256, 0, s>>>((const EA*)a, (float*)out, n); break;
    default: k_herm_aug<EA, double><<<g, 256, 0, s>>>((const EA*)a, (double*)out, n); break;
    }
    return cudaGetLastError();
}

bool valid_dtype(int t) { return t >= PTDR_C64 && t <= PTDR_F64; }

ptdr_status prepare(int* dev, unsigned int** st)
{
    ptdr_status v = device_ready(dev);
    if (v != PTDR_OK) return v;
    return status_word(*dev, st);
}

} // namespace

} // namespace ptdr

using namespace ptdr;

extern "C" {

ptdr_status ptdr_coeff_lincomb(int n, double mu_re, double mu_im, const void* CA, const void* CB, void* C_out,
                               ptdr_dtype c_type, void* stream)
{
    PTDR_TRACE();
    if (n < 1 || n > kMaxDenseN || !CA || !C_out || !valid_dtype(c_type)) return PTDR_ERR_INVALID_ARG;
    if (!std::isfinite(mu_re) || !std::isfinite(mu_im)) return PTDR_ERR_INVALID_ARG;
    if (!dtype_complex(c_type) && mu_im != 0.0) return PTDR_ERR_UNSUPPORTED; // real arrays stay real
    const uint64_t count = 1ull << (2 * n);
    const size_t bytes = count * dtype_bytes(c_type);
    if ((uintptr_t)CA % dtype_bytes(c_type) || (uintptr_t)C_out % dtype_bytes(c_type) ||
        (CB && (uintptr_t)CB % dtype_bytes(c_type)))
        return PTDR_ERR_INVALID_ARG;
    // the output may be B itself (in place), never a shifted copy of A or B
    if ((overlaps(CA, bytes, C_out, bytes) && CA != C_out) || (CB && overlaps(CB, bytes, C_out, bytes) && CB != C_out))
        return PTDR_ERR_INVALID_ARG;
    int dev = 0;
    unsigned int* st = nullptr;
    ptdr_status v = prepare(&dev, &st);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(CA) != PTDR_OK || check_device_ptr(C_out) != PTDR_OK || (CB && check_device_ptr(CB) != PTDR_OK))
        return PTDR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned g = grid_for(count, 256 * 4);
    switch (c_type) {
    case PTDR_C64: k_lincomb<float2><<<g, 256, 0, s>>>((const float2*)CA, (const float2*)CB, (float2*)C_out, count, mu_re, mu_im); break;
    case PTDR_C128: k_lincomb<double2><<<g, 256, 0, s>>>((const double2*)CA, (const double2*)CB, (double2*)C_out, count, mu_re, mu_im); break;
    case PTDR_F32: k_lincomb<float><<<g, 256, 0, s>>>((const float*)CA, (const float*)CB, (float*)C_out, count, mu_re, 0.0); break;
    case PTDR_F64: k_lincomb<double><<<g, 256, 0, s>>>((const double*)CA, (const double*)CB, (double*)C_out, count, mu_re, 0.0); break;
    }
    return cudaGetLastError() == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

ptdr_status ptdr_coeff_block_diag(int n, int m, const void* const* h_blocks, void* C_out, ptdr_dtype c_type,
                                  void* stream)
{
    PTDR_TRACE();
    if (n < 1 || m < 1 || m > kMaxBlockLog || n + m > kMaxDenseN || !h_blocks || !C_out || !valid_dtype(c_type))
        return PTDR_ERR_INVALID_ARG;
    const uint64_t in_bytes = (1ull << (2 * n)) * dtype_bytes(c_type);
    const uint64_t out_bytes = (1ull << (2 * (n + m))) * dtype_bytes(c_type);
    Blocks blk{};
    for (int i = 0; i < (1 << m); ++i) {
        if (!h_blocks[i] || (uintptr_t)h_blocks[i] % dtype_bytes(c_type)) return PTDR_ERR_INVALID_ARG;
        if (overlaps(h_blocks[i], in_bytes, C_out, out_bytes)) return PTDR_ERR_INVALID_ARG;
        blk.p[i] = h_blocks[i];
    }
    if ((uintptr_t)C_out % 16) return PTDR_ERR_INVALID_ARG; // 16-byte zero fill
    int dev = 0;
    unsigned int* st = nullptr;
    ptdr_status v = prepare(&dev, &st);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(C_out) != PTDR_OK) return PTDR_ERR_INVALID_ARG;
    for (int i = 0; i < (1 << m); ++i)
        if (check_device_ptr(h_blocks[i]) != PTDR_OK) return PTDR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // rows x >= 2^n (masks with X or Y on a top qubit) are all zero
    const uint64_t row_bytes = (1ull << (n + m)) * dtype_bytes(c_type);
    cudaError_t e = zero_bytes((char*)C_out + (row_bytes << n), out_bytes - (row_bytes << n), s);
    if (e == cudaSuccess) {
        switch (c_type) {
        case PTDR_C64: e = run_block_diag<float2>(blk, C_out, n, m, s); break;
        case PTDR_C128: e = run_block_diag<double2>(blk, C_out, n, m, s); break;
        case PTDR_F32: e = run_block_diag<float>(blk, C_out, n, m, s); break;
        case PTDR_F64: e = run_block_diag<double>(blk, C_out, n, m, s); break;
        }
    }
    return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

ptdr_status ptdr_coeff_hermitian_augment(int n, const void* CA, ptdr_dtype a_type, void* C_out, ptdr_dtype out_type,
                                         void* stream)
{
    PTDR_TRACE();
    if (n < 1 || n + 1 > kMaxDenseN || !CA || !C_out || !valid_dtype(a_type) || !valid_dtype(out_type))
        return PTDR_ERR_INVALID_ARG;
    const uint64_t in_bytes = (1ull << (2 * n)) * dtype_bytes(a_type);
    const uint64_t out_bytes = (1ull << (2 * (n + 1))) * dtype_bytes(out_type);
    if ((uintptr_t)CA % dtype_bytes(a_type) || (uintptr_t)C_out % 16 || overlaps(CA, in_bytes, C_out, out_bytes))
        return PTDR_ERR_INVALID_ARG;
    int dev = 0;
    unsigned int* st = nullptr;
    ptdr_status v = prepare(&dev, &st);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(CA) != PTDR_OK || check_device_ptr(C_out) != PTDR_OK) return PTDR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // rows x < 2^n (top qubit I or Z) are all zero
    cudaError_t e = zero_bytes(C_out, out_bytes / 2, s);
    if (e == cudaSuccess) {
        switch (a_type) {
        case PTDR_C64: e = run_herm_aug<float2>(CA, C_out, out_type, n, s); break;
        case PTDR_C128: e = run_herm_aug<double2>(CA, C_out, out_type, n, s); break;
        case PTDR_F32: e = run_herm_aug<float>(CA, C_out, out_type, n, s); break;
        case PTDR_F64: e = run_herm_aug<double>(CA, C_out, out_type, n, s); break;
        }
    }
    return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

} // extern "C"
