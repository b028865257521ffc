// Sparse output of a decomposition for block-encoding (Sec. VI): the terms a
// linear combination of unitaries keeps, their coefficients, and the
// normaliser sum_i |alpha_i| of the ancilla state it prepares.
//
// Every coefficient gets an order key from its magnitude: the float32 bits of
// |c| for complex64 (computed as max(|re|,|im|) sqrt(1 + r^2), which neither
// underflows nor overflows), the float64 bits of |c|^2 for complex128, the
// bits of |c| for real arrays.  Non-negative IEEE values order like their bit
// patterns, so the keys are compared as unsigned integers.
//   threshold:  keep key > key(threshold);
//   top-k:      a radix select (8-bit digits, most significant first) finds
//               the key T of the k-th largest kept coefficient and how many
//               coefficients equal to T still fit; one compaction pass then
//               keeps every key > T and the first of those equal to T in index
//               order.
// The compaction is in index order (per-CTA counts, one scan, per-CTA writes
// in order), so the output is deterministic: indices x 2^n + z ascending.
// The normaliser is summed in float64 in a fixed order (per thread, per CTA
// tree, then the CTA partials in order).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "plan.h"

namespace ptdr {

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;                     // consecutive elements per thread per tile
constexpr int kTile = kThreads * kPerThread;      // elements per CTA tile
constexpr int kBins = 256;

// Order key and magnitude of one coefficient.
template <typename E> struct mag;
template <> struct mag<float2> {
    using K = uint32_t;
    __device__ static K key(const float2* p, uint64_t i, double& m)
    {
        const float2 v = p[i];
        const float a = fabsf(v.x), b = fabsf(v.y);
        const float hi = fmaxf(a, b), lo = fminf(a, b);
        const float r = hi > 0.f ? lo / hi : 0.f;
        const float mg = hi * sqrtf(1.f + r * r);
        m = (double)mg;
        return __float_as_uint(mg);
    }
    static K thr_key(double t)
    {
        const float f = (float)t;
        uint32_t k;
        memcpy(&k, &f, 4);
        return k;
    }
};
template <> struct mag<double2> {
    using K = unsigned long long;
    __device__ static K key(const double2* p, uint64_t i, double& m)
    {
        const double2 v = p[i];
        const double q = v.x * v.x + v.y * v.y;
        m = q; // the square root is taken only for kept terms
        return (K)__double_as_longlong(q);
    }
    static K thr_key(double t)
    {
        const double q = t * t;
        unsigned long long k;
        memcpy(&k, &q, 8);
        return k;
    }
};
template <> struct mag<float> {
    using K = uint32_t;
    __device__ static K key(const float* p, uint64_t i, double& m)
    {
        const float a = fabsf(p[i]);
        m = (double)a;
        return __float_as_uint(a);
    }
    static K thr_key(double t) { return mag<float2>::thr_key(t); }
};
template <> struct mag<double> {
    using K = unsigned long long;
    __device__ static K key(const double* p, uint64_t i, double& m)
    {
        const double a = fabs(p[i]);
        m = a;
        return (K)__double_as_longlong(a);
    }
    static K thr_key(double t)
    {
        const double a = fabs(t);
        unsigned long long k;
        memcpy(&k, &a, 8);
        return k;
    }
};
template <typename E> __device__ __forceinline__ double l1_of(double m) { return m; }
template <> __device__ __forceinline__ double l1_of<double2>(double m) { return sqrt(m); }

// Device state of one selection (in the workspace).
struct SelState {
    unsigned long long prefix;   // key bits fixed so far (top-k)
    unsigned long long kleft;    // how many of the keys matching the prefix are still to take
    unsigned long long total;    // keys above the threshold
    unsigned long long eq_take;  // keys equal to T that are kept (top-k)
    unsigned long long count;    // number kept
    int use_topk;                // 0: threshold only, or fewer than k above it
    int pad;
    double l1;
    unsigned int hist[kBins];
};

// Histogram of digit `shift` of the keys above the threshold that match the
// prefix on the digits above (all keys above the threshold at the first pass,
// which also counts them).
template <typename E>
__global__ void __launch_bounds__(kThreads) k_sel_hist(const E* __restrict__ c, uint64_t count,
                                                       typename mag<E>::K thr, int shift, SelState* s, int first)
{
    using K = typename mag<E>::K;
    __shared__ unsigned int h[kBins];
    __shared__ unsigned long long above;
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
    if (threadIdx.x == 0) above = 0;
    __syncthreads();
    const int width = (int)sizeof(K) * 8;
    const K hi_mask = shift + 8 >= width ? (K)0 : (K)(~(K)0 << (shift + 8));
    const K prefix = (K)s->prefix;
    unsigned long long mine = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        double m;
        const K k = mag<E>::key(c, i, m);
        if (k <= thr || (k & hi_mask) != (prefix & hi_mask)) continue;
        ++mine;
        atomicAdd(&h[(k >> shift) & (kBins - 1)], 1u);
    }
    if (first && mine) atomicAdd(&above, mine);
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&s->hist[i], h[i]);
    if (first && threadIdx.x == 0 && above) atomicAdd(&s->total, above);
}

// One thread: pick the bin that holds the kleft-th largest key, fix that digit
// of the prefix, clear the histogram.  The first pass decides whether a
// selection is needed at all (more than k keys above the threshold).
__global__ void k_sel_pick(SelState* s, int shift, unsigned long long k, int first)
{
    if (first) {
        s->use_topk = k > 0 && s->total > k;
        s->kleft = k;
    }
    if (s->use_topk) {
        unsigned long long need = s->kleft, seen = 0;
        int b = kBins - 1;
        for (; b > 0; --b) {
            if (seen + s->hist[b] >= need) break;
            seen += s->hist[b];
        }
        s->prefix |= (unsigned long long)b << shift;
        s->kleft = need - seen;
    }
    for (int i = 0; i < kBins; ++i) s->hist[i] = 0;
}

__device__ __forceinline__ bool kept(unsigned long long k, unsigned long long thr, unsigned long long T, int topk,
                                     bool& eq)
{
    eq = false;
    if (k <= thr) return false;
    if (!topk) return true;
    if (k > T) return true;
    eq = k == T;
    return eq;
}

// Per-CTA counts over its contiguous range: keys kept for sure (gt) and keys equal to T.
template <typename E>
__global__ void __launch_bounds__(kThreads) k_sel_count(const E* __restrict__ c, uint64_t count, uint64_t per_cta,
                                                        typename mag<E>::K thr, const SelState* s,
                                                        unsigned long long* gt, unsigned long long* eqc)
{
    using K = typename mag<E>::K;
    __shared__ unsigned long long sg, se;
    if (threadIdx.x == 0) sg = se = 0;
    __syncthreads();
    const uint64_t b0 = (uint64_t)blockIdx.x * per_cta, b1 = min(count, b0 + per_cta);
    const int topk = s->use_topk;
    const K T = (K)s->prefix;
    unsigned long long g = 0, e = 0;
    for (uint64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        double m;
        bool eq;
        const K k = mag<E>::key(c, i, m);
        if (kept(k, thr, T, topk, eq)) {
            if (eq) ++e;
            else ++g;
        }
    }
    atomicAdd(&sg, g);
    atomicAdd(&se, e);
    __syncthreads();
    if (threadIdx.x == 0) {
        gt[blockIdx.x] = sg;
        eqc[blockIdx.x] = se;
    }
}

// One CTA: exclusive scan of the per-CTA counts in CTA order; CTA b may keep
// eq_take - (equal keys before it) of its equal keys.  Output offsets go to gt[],
// per-CTA equal-key budgets to eqc[].
__global__ void k_sel_scan(SelState* s, int ctas, unsigned long long* gt, unsigned long long* eqc)
{
    if (threadIdx.x != 0) return;
    const unsigned long long take = s->use_topk ? s->kleft : 0;
    unsigned long long off = 0, eq_before = 0;
    for (int b = 0; b < ctas; ++b) {
        const unsigned long long g = gt[b], e = eqc[b];
        const unsigned long long budget = s->use_topk ? (eq_before >= take ? 0 : min(e, take - eq_before)) : 0;
        gt[b] = off;
        eqc[b] = budget;
        off += g + budget;
        eq_before += e;
    }
    s->count = off;
    s->eq_take = take;
}

// Writes the kept terms of each CTA's range in index order, and the CTA's
// partial normaliser.
template <typename E>
__global__ void __launch_bounds__(kThreads) k_sel_write(const E* __restrict__ c, uint64_t count, uint64_t per_cta,
                                                        typename mag<E>::K thr, const SelState* s,
                                                        const unsigned long long* off, const unsigned long long* budget,
                                                        uint64_t* idx_out, E* val_out, uint64_t cap, double* l1_part)
{
    using K = typename mag<E>::K;
    __shared__ unsigned int wk[kThreads / 32], we[kThreads / 32];
    __shared__ double red[kThreads];
    const uint64_t b0 = (uint64_t)blockIdx.x * per_cta, b1 = min(count, b0 + per_cta);
    const int topk = s->use_topk;
    const K T = (K)s->prefix;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long pos = off[blockIdx.x], eq_left = budget[blockIdx.x];
    double l1 = 0.0;
    for (uint64_t t0 = b0; t0 < b1; t0 += kTile) {
        // thread t looks at elements t0 + kPerThread t + j, j < kPerThread (index order = thread order)
        K kk[kPerThread];
        double mm[kPerThread];
        unsigned int keepm = 0, eqm = 0;
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const uint64_t i = t0 + (uint64_t)kPerThread * threadIdx.x + j;
            kk[j] = 0;
            mm[j] = 0.0;
            if (i < b1) {
                bool eq;
                kk[j] = mag<E>::key(c, i, mm[j]);
                if (kept(kk[j], thr, T, topk, eq)) {
                    keepm |= 1u << j;
                    if (eq) eqm |= 1u << j;
                }
            }
        }
        // exclusive prefix over threads of (kept not equal, equal) counts
        const unsigned int nk = __popc(keepm & ~eqm), ne = __popc(eqm);
        unsigned int pk = nk, pe = ne;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int a = __shfl_up_sync(0xffffffffu, pk, o), b = __shfl_up_sync(0xffffffffu, pe, o);
            if (lane >= o) {
                pk += a;
                pe += b;
            }
        }
        if (lane == 31) {
            wk[warp] = pk;
            we[warp] = pe;
        }
        __syncthreads();
        unsigned int base_k = 0, base_e = 0, tot_k = 0, tot_e = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            if (w < warp) {
                base_k += wk[w];
                base_e += we[w];
            }
            tot_k += wk[w];
            tot_e += we[w];
        }
        pk += base_k - nk; // exclusive
        pe += base_e - ne;
        // walk this thread's elements in order: equal keys consume the CTA's budget in index order
        unsigned long long rank_eq = pe, written_before = pk + min((unsigned long long)pe, eq_left);
        unsigned long long w = pos + written_before;
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            if (!((keepm >> j) & 1u)) continue;
            if ((eqm >> j) & 1u) {
                if (rank_eq >= eq_left) continue;
                ++rank_eq;
            }
            const uint64_t i = t0 + (uint64_t)kPerThread * threadIdx.x + j;
            if (w < cap) {
                idx_out[w] = i;
                val_out[w] = c[i];
            }
            ++w;
            l1 += l1_of<E>(mm[j]);
        }
        const unsigned long long used_eq = min((unsigned long long)tot_e, eq_left);
        pos += tot_k + used_eq;
        eq_left -= used_eq;
        __syncthreads();
    }
    red[threadIdx.x] = l1;
    __syncthreads();
    for (int o = kThreads / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) l1_part[blockIdx.x] = red[0];
}

// One thread: the normaliser as the in-order sum of the CTA partials, and the count.
__global__ void k_sel_finish(SelState* s, int ctas, const double* l1_part, unsigned long long* d_count, double* d_l1)
{
    if (threadIdx.x != 0) return;
    double l1 = 0.0;
    for (int b = 0; b < ctas; ++b) l1 += l1_part[b];
    s->l1 = l1;
    *d_count = s->count;
    *d_l1 = l1;
}

int select_ctas()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, sms) * 4;
}

size_t state_bytes() { return (sizeof(SelState) + 255) & ~(size_t)255; }

template <typename E>
cudaError_t run_select(const void* C, uint64_t count, double threshold, unsigned long long k, void* ws,
                       uint64_t* idx, void* val, uint64_t cap, unsigned long long* d_count, double* d_l1, cudaStream_t st)
{
    using K = typename mag<E>::K;
    const int ctas = select_ctas();
    SelState* s = (SelState*)ws;
    unsigned long long* gt = (unsigned long long*)((char*)ws + state_bytes());
    unsigned long long* eqc = gt + ctas;
    double* l1p = (double*)(eqc + ctas);
    cudaError_t e = cudaMemsetAsync(ws, 0, state_bytes(), st);
    if (e != cudaSuccess) return e;
    const K thr = mag<E>::thr_key(threshold);
    const E* c = (const E*)C;
    const int width = (int)sizeof(K) * 8;
    const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)ctas, std::max<uint64_t>(1, count / kThreads));
    // radix select (a threshold-only call still takes the first pass: it counts)
    for (int shift = width - 8, first = 1; shift >= 0; shift -= 8, first = 0) {
        k_sel_hist<E><<<grid, kThreads, 0, st>>>(c, count, thr, shift, s, first);
        k_sel_pick<<<1, 1, 0, st>>>(s, shift, k, first);
        if (k == 0) break;
    }
    const uint64_t per_cta = ((count + ctas - 1) / ctas + kTile - 1) / kTile * kTile;
    k_sel_count<E><<<ctas, kThreads, 0, st>>>(c, count, per_cta, thr, s, gt, eqc);
    k_sel_scan<<<1, 32, 0, st>>>(s, ctas, gt, eqc);
    k_sel_write<E><<<ctas, kThreads, 0, st>>>(c, count, per_cta, thr, s, gt, eqc, idx, (E*)val, cap, l1p);
    k_sel_finish<<<1, 32, 0, st>>>(s, ctas, l1p, d_count, d_l1);
    return cudaGetLastError();
}

bool valid_dtype(int t) { return t >= PTDR_C64 && t <= PTDR_F64; }

} // namespace

} // namespace ptdr

using namespace ptdr;

extern "C" {

ptdr_status ptdr_select_workspace_size(size_t* bytes)
{
    if (!bytes) return PTDR_ERR_INVALID_ARG;
    // the CTA count depends on the device; size for the largest GPU this library targets
    *bytes = state_bytes() + (size_t)4096 * 3 * 8;
    return PTDR_OK;
}

ptdr_status ptdr_coeff_select(int n, const void* C, ptdr_dtype c_type, double threshold, unsigned long long k,
                              uint64_t* d_idx, void* d_val, size_t cap, unsigned long long* d_count, double* d_l1,
                              void* workspace, size_t workspace_bytes, void* stream)
{
    PTDR_TRACE();
    if (n < 1 || n > kMaxDenseN || !C || !valid_dtype(c_type) || !d_count || !d_l1) return PTDR_ERR_INVALID_ARG;
    if (!(threshold >= 0.0) || !std::isfinite(threshold)) return PTDR_ERR_INVALID_ARG;
    if (cap > 0 && (!d_idx || !d_val)) return PTDR_ERR_INVALID_ARG;
    if ((uintptr_t)C % dtype_bytes(c_type) || (d_val && (uintptr_t)d_val % dtype_bytes(c_type)) ||
        (d_idx && (uintptr_t)d_idx % 8) || (uintptr_t)d_count % 8 || (uintptr_t)d_l1 % 8)
        return PTDR_ERR_INVALID_ARG;
    size_t need = 0;
    ptdr_select_workspace_size(&need);
    if (!workspace || workspace_bytes < need || (uintptr_t)workspace % 256) return PTDR_ERR_WORKSPACE;
    int dev = 0;
    ptdr_status v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    if (select_ctas() * 3 * 8 + state_bytes() > workspace_bytes) return PTDR_ERR_WORKSPACE;
    if (check_device_ptr(C) != PTDR_OK || check_device_ptr(workspace) != PTDR_OK ||
        check_device_ptr(d_count) != PTDR_OK || check_device_ptr(d_l1) != PTDR_OK ||
        (cap > 0 && (check_device_ptr(d_idx) != PTDR_OK || check_device_ptr(d_val) != PTDR_OK)))
        return PTDR_ERR_INVALID_ARG;
    const uint64_t count = 1ull << (2 * n);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (c_type) {
    case PTDR_C64: e = run_select<float2>(C, count, threshold, k, workspace, d_idx, d_val, cap, d_count, d_l1, s); break;
    case PTDR_C128: e = run_select<double2>(C, count, threshold, k, workspace, d_idx, d_val, cap, d_count, d_l1, s); break;
    case PTDR_F32: e = run_select<float>(C, count, threshold, k, workspace, d_idx, d_val, cap, d_count, d_l1, s); break;
    default: e = run_select<double>(C, count, threshold, k, workspace, d_idx, d_val, cap, d_count, d_l1, s); break;
    }
    return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

} // extern "C"
