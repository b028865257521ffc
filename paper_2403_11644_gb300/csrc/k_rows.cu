// Generic tile kernels: XOR-diagonal gather, shared-memory Walsh-Hadamard
// transform, phased write-out (decompose) and the mirror path (compose).
//
// These cover every n and both FP32 and FP64 arithmetic.  A row of the
// transform (one mask x, 2^n values) is handled in one tile when it fits in
// shared memory, otherwise as a first pass over contiguous segments followed
// by strided passes over the remaining high bits through an intermediate
// buffer in HBM (the "top bits" passes).
#include "tile_ops.cuh"

namespace ptdr {

// ---------------------------------------------------------------- kernels

// One CTA per (mask block, segment).  blockIdx.x = block * segs + seg.
template <typename T, typename InT, typename OutT, Load LD, Store ST>
__global__ void __launch_bounds__(512) k_tile(TileLaunch p, unsigned int* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using T2 = cplx_t<T>;
    T2* s = reinterpret_cast<T2*>(smem_raw);
    const Smem sm = make_smem(p.log_l);
    const int segs_log = p.n - p.log_l;
    const uint64_t blk = (uint64_t)blockIdx.x >> segs_log;
    const uint64_t seg = (uint64_t)blockIdx.x & ((1ull << segs_log) - 1);
    const uint64_t x0 = p.x_begin + (blk << p.log_r);
    const uint64_t k0 = seg << p.log_l;
    const T scale = (T)p.scale;

    if (LD == Load::GatherA)
        load_gather<T>(s, sm, (const InT*)p.src, p.n, x0, p.log_r, k0, p.log_l, p.src_elems, st,
                       p.src_row_mask ? p.src_row_mask : ~0ull);
    else if (LD == Load::RowPhaseC)
        load_row_phase<T>(s, sm, (const InT*)p.src, p.n, x0, p.log_r, k0, p.log_l, p.src_row0,
                          scale, p.src_elems, st);
    else
        load_row_buf<T>(s, sm, (const T2*)p.src, p.n, x0, p.log_r, k0, p.log_l, p.src_row0,
                        p.src_elems, st);
    __syncthreads();

    wht_bits(s, sm, p.log_r + p.log_l, 0, p.log_l);

    if (ST == Store::RowPhaseOut)
        store_row_phase<T>((OutT*)p.dst, s, sm, p.n, x0, p.log_r, k0, p.log_l, p.dst_row0, scale,
                           p.dst_elems, st);
    else if (ST == Store::RowBuf)
        store_row_buf<T>((T2*)p.dst, s, sm, p.n, x0, p.log_r, k0, p.log_l, p.dst_row0,
                         p.dst_elems, st);
    else
        store_scatter<T>((OutT*)p.dst, s, sm, p.n, x0, p.log_r, k0, p.log_l, p.dst_elems, st);
}

// One CTA per (mask, group of bits >= b1, chunk of 2^log_w low columns).
// Tile element (j, w) <-> k = g 2^b1 + j 2^b0 + c0 + w; transform over j.
// V is the row value type: complex (cplx_t<T>), or T for rows of real values
// (transforms of real band data), which only pass through buffers.
template <typename T, typename V, typename OutT, Store ST>
__global__ void __launch_bounds__(512) k_strided(StridedLaunch p, unsigned int* st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* s = reinterpret_cast<V*>(smem_raw);
    const int nb = p.b1 - p.b0;
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
    const V* src = (const V*)p.src + (x - p.src_row0) * N;
    const int E = 1 << (nb + p.log_w);
    const int wmask = (1 << p.log_w) - 1;
    for (int e0 = threadIdx.x; e0 < E; e0 += kLoadBatch * blockDim.x) {
        V v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            v[u] = V{};
            if (e < E) {
                const uint64_t k = kbase + ((uint64_t)(e >> p.log_w) << p.b0) + (uint64_t)(e & wmask);
                if (in_bounds(st, (x - p.src_row0) * N + k, p.src_elems)) v[u] = src[k];
            }
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < E) s[sm.idx(e)] = v[u];
        }
    }
    __syncthreads();

    wht_bits(s, sm, nb + p.log_w, p.log_w, nb + p.log_w);

    const T scale = (T)p.scale;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const uint64_t k = kbase + ((uint64_t)(e >> p.log_w) << p.b0) + (uint64_t)(e & wmask);
        const V v = s[sm.idx(e)];
        if constexpr (ST == Store::RowPhaseOut) {
            const uint64_t gi = (x - p.dst_row0) * N + k;
            if (in_bounds(st, gi, p.dst_elems))
                io<OutT>::st((OutT*)p.dst + gi, phase_neg_i(v, __popcll(x & k), scale));
        } else if constexpr (ST == Store::RowBuf) {
            const uint64_t gi = (x - p.dst_row0) * N + k;
            if (in_bounds(st, gi, p.dst_elems)) ((V*)p.dst)[gi] = v;
        } else {
            const uint64_t gi = (k ^ x) * N + k;
            if (in_bounds(st, gi, p.dst_elems)) io<OutT>::st((OutT*)p.dst + gi, v);
        }
    }
}

// ---------------------------------------------------------------- launch

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, typename InT, typename OutT, Load LD, Store ST>
static cudaError_t run_tile(const TileLaunch& p, unsigned int* st, cudaStream_t s)
{
    auto kern = k_tile<T, InT, OutT, LD, ST>;
    const size_t bytes = smem_elems((size_t)1 << p.log_r, p.log_l) * sizeof(cplx_t<T>);
    cudaError_t e = set_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (p.x_count >> p.log_r) << (p.n - p.log_l);
    kern<<<(unsigned)blocks, p.threads, bytes, s>>>(p, st);
    return cudaGetLastError();
}

template <typename T, typename OutT, Store ST, typename V = cplx_t<T>>
static cudaError_t run_strided(const StridedLaunch& p, unsigned int* st, cudaStream_t s)
{
    auto kern = k_strided<T, V, OutT, ST>;
    const size_t bytes = smem_elems((size_t)1 << (p.b1 - p.b0), p.log_w) * sizeof(V);
    cudaError_t e = set_smem(kern, bytes);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = p.x_count << ((p.n - p.b1) + (p.b0 - p.log_w));
    kern<<<(unsigned)blocks, p.threads, bytes, s>>>(p, st);
    return cudaGetLastError();
}

template <typename T, typename InT, Load LD>
static cudaError_t tile_by_store(const TileLaunch& p, unsigned int* st, cudaStream_t s)
{
    using T2 = cplx_t<T>;
    switch (p.store) {
    case Store::RowBuf: return run_tile<T, InT, T2, LD, Store::RowBuf>(p, st, s);
    case Store::RowPhaseOut: // a real output type stores the real part (Hermitian A: all of c, Thm 2)
        if (p.dst_t == PTDR_C64) return run_tile<T, InT, float2, LD, Store::RowPhaseOut>(p, st, s);
        if (p.dst_t == PTDR_C128) return run_tile<T, InT, double2, LD, Store::RowPhaseOut>(p, st, s);
        if (p.dst_t == PTDR_F32) return run_tile<T, InT, float, LD, Store::RowPhaseOut>(p, st, s);
        if (p.dst_t == PTDR_F64) return run_tile<T, InT, double, LD, Store::RowPhaseOut>(p, st, s);
        break;
    case Store::ScatterA:
        if (p.dst_t == PTDR_C64) return run_tile<T, InT, float2, LD, Store::ScatterA>(p, st, s);
        if (p.dst_t == PTDR_C128) return run_tile<T, InT, double2, LD, Store::ScatterA>(p, st, s);
        break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t tile_by_load(const TileLaunch& p, unsigned int* st, cudaStream_t s)
{
    using T2 = cplx_t<T>;
    switch (p.load) {
    case Load::RowBuf: return tile_by_store<T, T2, Load::RowBuf>(p, st, s);
    case Load::GatherA: // real matrices enter with a zero imaginary part
        if (p.src_t == PTDR_C64) return tile_by_store<T, float2, Load::GatherA>(p, st, s);
        if (p.src_t == PTDR_C128) return tile_by_store<T, double2, Load::GatherA>(p, st, s);
        if (p.src_t == PTDR_F32) return tile_by_store<T, float, Load::GatherA>(p, st, s);
        if (p.src_t == PTDR_F64) return tile_by_store<T, double, Load::GatherA>(p, st, s);
        break;
    case Load::RowPhaseC: // real coefficients: a Hermitian matrix (Thm 2)
        if (p.src_t == PTDR_C64) return tile_by_store<T, float2, Load::RowPhaseC>(p, st, s);
        if (p.src_t == PTDR_C128) return tile_by_store<T, double2, Load::RowPhaseC>(p, st, s);
        if (p.src_t == PTDR_F32) return tile_by_store<T, float, Load::RowPhaseC>(p, st, s);
        if (p.src_t == PTDR_F64) return tile_by_store<T, double, Load::RowPhaseC>(p, st, s);
        break;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tile(const TileLaunch& p, unsigned int* st, cudaStream_t s)
{
    return p.calc == Calc::F32 ? tile_by_load<float>(p, st, s) : tile_by_load<double>(p, st, s);
}

template <typename T>
static cudaError_t strided_by_store(const StridedLaunch& p, unsigned int* st, cudaStream_t s)
{
    using T2 = cplx_t<T>;
    if (p.real) return p.store == Store::RowBuf ? run_strided<T, T, Store::RowBuf, T>(p, st, s) : cudaErrorInvalidValue;
    switch (p.store) {
    case Store::RowBuf: return run_strided<T, T2, Store::RowBuf>(p, st, s);
    case Store::RowPhaseOut:
        if (p.dst_t == PTDR_C64) return run_strided<T, float2, Store::RowPhaseOut>(p, st, s);
        if (p.dst_t == PTDR_C128) return run_strided<T, double2, Store::RowPhaseOut>(p, st, s);
        if (p.dst_t == PTDR_F32) return run_strided<T, float, Store::RowPhaseOut>(p, st, s);
        if (p.dst_t == PTDR_F64) return run_strided<T, double, Store::RowPhaseOut>(p, st, s);
        break;
    case Store::ScatterA:
        if (p.dst_t == PTDR_C64) return run_strided<T, float2, Store::ScatterA>(p, st, s);
        if (p.dst_t == PTDR_C128) return run_strided<T, double2, Store::ScatterA>(p, st, s);
        break;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_strided(const StridedLaunch& p, unsigned int* st, cudaStream_t s)
{
    return p.calc == Calc::F32 ? strided_by_store<float>(p, st, s)
                               : strided_by_store<double>(p, st, s);
}

} // namespace ptdr
