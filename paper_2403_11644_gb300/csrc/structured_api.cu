// Band-diagonal (structured) entry points: mask enumeration on the host.
#include "plan.h"

using namespace ptdr;

extern "C" {

// A mask x != 0 with highest set bit h reaches the band iff the smallest
// |row - column| over its XOR-diagonal, 2^h - (x mod 2^h), is at most s
// (Sec. IV.A: diagonal, Thm 3 tridiagonal, Thm 4 band-diagonal).
ptdr_status ptdr_structured_masks(int n, int s, uint64_t* h_masks, size_t* count)
{
    if (!count || n < 1 || n > 40 || s < 0) return PTDR_ERR_INVALID_ARG;
    const uint64_t N = 1ull << n;
    const size_t cap = h_masks ? *count : 0;
    size_t cnt = 0;
    auto emit = [&](uint64_t x) {
        if (h_masks && cnt < cap) h_masks[cnt] = x;
        ++cnt;
    };
    emit(0);
    for (int h = 0; h < n; ++h) {
        const uint64_t top = 1ull << h;
        // x = top + rest with rest < top; reachable iff top - rest <= s,
        // i.e. rest >= top - s (all rest when s >= top).
        const uint64_t lo = (uint64_t)s >= top ? 0 : top - (uint64_t)s;
        for (uint64_t rest = lo; rest < top; ++rest) {
            if (top + rest >= N) break;
            emit(top + rest);
        }
    }
    *count = cnt;
    if (h_masks && cnt > cap) return PTDR_ERR_INVALID_ARG;
    return PTDR_OK;
}

} // extern "C"

// ---------------------------------------------------------------- planning

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "structured.h"

namespace {

struct MaskPlan {
    uint64_t x;
    int h1, zc, f, npairs;
    uint64_t t[kMaxBandPairs];
    int64_t d[kMaxBandPairs];
};

int msb1(uint64_t x)
{
    int h = 0;
    while (x >> h) ++h;
    return h; // msb + 1, 0 for x = 0
}

// T_x = { t subset of x : |x - 2t| <= s }: t lies in [(x-s)/2, (x+s)/2].
MaskPlan plan_mask(int n, int s, uint64_t x)
{
    MaskPlan m{};
    m.x = x;
    m.h1 = msb1(x);
    m.zc = m.h1 - __builtin_popcountll(x);
    m.f = n - __builtin_popcountll(x);
    const int64_t lo = ((int64_t)x - s + 1) / 2 > 0 ? ((int64_t)x - s + 1) / 2 : 0;
    const int64_t hi = ((int64_t)x + s) / 2;
    for (int64_t t = lo; t <= hi; ++t) {
        if (((uint64_t)t & ~x) != 0) continue;
        const int64_t d = (int64_t)x - 2 * t;
        if (d < -s || d > s) continue;
        m.t[m.npairs] = (uint64_t)t;
        m.d[m.npairs] = d;
        ++m.npairs;
    }
    return m;
}

// Bytes of one row value: real bands are transformed as real rows.
size_t calc_bytes(ptdr_precision p, ptdr_dtype b_t)
{
    const size_t c = p == PTDR_PREC_FP64 ? 16 : 8;
    return dtype_complex(b_t) ? c : c / 2;
}

ptdr_status validate_structured(const void* bands, ptdr_dtype b_t, int n, int s,
                                const uint64_t* h_masks, size_t n_masks, ptdr_dtype c_t,
                                ptdr_precision prec)
{
    if (!bands || !h_masks || n_masks == 0) return PTDR_ERR_INVALID_ARG;
    if (n < 1 || n > 30 || s < 0) return PTDR_ERR_INVALID_ARG;
    const uint64_t N = 1ull << n;
    if ((uint64_t)s >= N) return PTDR_ERR_INVALID_ARG;
    if (s >= kMaxBandPairs) return PTDR_ERR_UNSUPPORTED;
    if ((int)b_t < PTDR_C64 || (int)b_t > PTDR_F64 || (int)c_t < PTDR_C64 || (int)c_t > PTDR_F64)
        return PTDR_ERR_INVALID_ARG;
    if ((int)prec < PTDR_PREC_FP64 || (int)prec > PTDR_PREC_FIXED_I128) return PTDR_ERR_INVALID_ARG;
    if (prec != PTDR_PREC_FP64 && prec != PTDR_PREC_FP32) return PTDR_ERR_UNSUPPORTED;
    if (!dtype_complex(c_t) && dtype_complex(b_t)) return PTDR_ERR_UNSUPPORTED;
    for (size_t i = 0; i < n_masks; ++i)
        if (h_masks[i] >= N) return PTDR_ERR_INVALID_ARG;
    return PTDR_OK;
}

// The masks are independent: each is a chain first pass -> strided passes ->
// expansion through its own V rows.  Run on one stream, the chains of the
// many short masks (a few CTAs each: FP64 work on a few SMs runs at a few
// 1/152 of the GPU's FP64 rate) leave the GPU idle, so the masks are dealt
// to up to kChains chains, longest first to the least loaded (work =
// transform and expansion values), each chain on a library stream with its
// own V region.  The plan depends only on the mask list, so the workspace
// query and the call agree.
constexpr int kChains = 8;

struct ChainPlan {
    std::vector<int> chain;      // chain of each mask
    size_t region[kChains] = {}; // V bytes of each chain (its largest mask), 256-aligned
    int chains = 0;
    size_t total = 0;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

ChainPlan plan_chains(int n, int s, const uint64_t* h_masks, size_t n_masks, ptdr_precision prec,
                      ptdr_dtype b_t)
{
    ChainPlan cp;
    cp.chain.assign(n_masks, 0);
    cp.chains = (int)std::min<size_t>(n_masks, kChains);
    std::vector<std::pair<double, size_t>> order(n_masks);
    std::vector<size_t> vbytes(n_masks);
    for (size_t i = 0; i < n_masks; ++i) {
        const MaskPlan m = plan_mask(n, s, h_masks[i]);
        vbytes[i] = ((size_t)m.npairs << m.f) * calc_bytes(prec, b_t);
        const double work = (double)m.npairs * (m.f + 1) * std::ldexp(1.0, m.f) + std::ldexp(1.0, n);
        order[i] = {work, i};
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<double, size_t>& a, const std::pair<double, size_t>& b) {
                         return a.first > b.first;
                     });
    double load[kChains] = {};
    for (const auto& wi : order) {
        int c = 0;
        for (int k = 1; k < cp.chains; ++k)
            if (load[k] < load[c]) c = k;
        load[c] += wi.first;
        cp.chain[wi.second] = c;
        cp.region[c] = std::max(cp.region[c], align256(vbytes[wi.second]));
    }
    for (int c = 0; c < cp.chains; ++c) cp.total += cp.region[c];
    return cp;
}

size_t structured_ws(int n, int s, const uint64_t* h_masks, size_t n_masks, ptdr_precision prec,
                     ptdr_dtype b_t)
{
    return plan_chains(n, s, h_masks, n_masks, prec, b_t).total;
}

// Library streams of the chains, one set per device, created on first use.
struct ChainStreams {
    bool ready = false;
    cudaStream_t s[kChains] = {};
    cudaEvent_t fork = nullptr, join[kChains] = {};
};
std::mutex g_chain_mu; // also serialises the enqueue of concurrent calls
ChainStreams g_chain[128];

ptdr_status chain_streams(int dev, ChainStreams** out)
{
    ChainStreams& c = g_chain[dev];
    if (!c.ready) {
        bool ok = cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; k < kChains && ok; ++k)
            ok = cudaStreamCreateWithFlags(&c.s[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c.join[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return PTDR_ERR_CUDA;
        }
        c.ready = true;
    }
    *out = &c;
    return PTDR_OK;
}


} // namespace

extern "C" {

ptdr_status ptdr_structured_workspace_size(int n, int s, const uint64_t* h_masks, size_t n_masks,
                                           ptdr_dtype b_type, ptdr_dtype c_type,
                                           ptdr_precision prec, size_t* bytes)
{
    if (!bytes) return PTDR_ERR_INVALID_ARG;
    // bands pointer not needed for sizing: pass a dummy non-null value
    ptdr_status v = validate_structured((const void*)1, b_type, n, s, h_masks, n_masks, c_type, prec);
    if (v != PTDR_OK) return v;
    *bytes = structured_ws(n, s, h_masks, n_masks, prec, b_type);
    return PTDR_OK;
}

// The band path for band storage and masks h_masks; with anti_masks the
// storage is that of B = A J (an anti-band A) and h_masks[i] = anti_masks[i] ^
// (2^n - 1), and row i receives the coefficients of A's mask anti_masks[i].
static ptdr_status decompose_band(const void* bands, ptdr_dtype b_type, int n, int s, const uint64_t* h_masks,
                                  size_t n_masks, void* C, ptdr_dtype c_type, ptdr_precision prec, void* workspace,
                                  size_t workspace_bytes, void* stream, const uint64_t* anti_masks)
{
    if (!C) return PTDR_ERR_INVALID_ARG;
    ptdr_status v = validate_structured(bands, b_type, n, s, h_masks, n_masks, c_type, prec);
    if (v != PTDR_OK) return v;
    const uint64_t N = 1ull << n;
    const size_t band_bytes = (size_t)(2 * s + 1) * N * dtype_bytes(b_type);
    const size_t out_bytes = n_masks * N * dtype_bytes(c_type);
    if ((uintptr_t)bands % dtype_bytes(b_type) || (uintptr_t)C % dtype_bytes(c_type))
        return PTDR_ERR_INVALID_ARG;
    if (overlaps(bands, band_bytes, C, out_bytes)) return PTDR_ERR_INVALID_ARG;
    const size_t need = structured_ws(n, s, h_masks, n_masks, prec, b_type);
    if (need > 0 && (!workspace || workspace_bytes < need)) return PTDR_ERR_WORKSPACE;
    if (need > 0 && overlaps(workspace, need, C, out_bytes)) return PTDR_ERR_INVALID_ARG;
    if (fault_injected("plan")) return PTDR_ERR_INTERNAL;
    int dev = 0;
    v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(bands) != PTDR_OK || check_device_ptr(C) != PTDR_OK ||
        (need > 0 && check_device_ptr(workspace) != PTDR_OK))
        return PTDR_ERR_INVALID_ARG;
    unsigned int* st = nullptr;
    v = status_word(dev, &st);
    if (v != PTDR_OK) return v;
    if (fault_injected("launch")) return PTDR_ERR_CUDA;

    cudaStream_t cs = (cudaStream_t)stream;
    const ChainPlan cp = plan_chains(n, s, h_masks, n_masks, prec, b_type);
    size_t region_off[kChains] = {};
    for (int c = 1; c < cp.chains; ++c) region_off[c] = region_off[c - 1] + cp.region[c - 1];
    std::unique_lock<std::mutex> lk(g_chain_mu, std::defer_lock);
    ChainStreams* chs = nullptr;
    if (cp.chains > 1) {
        lk.lock();
        v = chain_streams(dev, &chs);
        if (v != PTDR_OK) return v;
        // the chains follow whatever the caller enqueued on its stream before
        if (cudaEventRecord(chs->fork, cs) != cudaSuccess) return PTDR_ERR_CUDA;
        for (int c = 0; c < cp.chains; ++c)
            if (cudaStreamWaitEvent(chs->s[c], chs->fork, 0) != cudaSuccess) return PTDR_ERR_CUDA;
    }
    const Calc calc = prec == PTDR_PREC_FP64 ? Calc::F64 : Calc::F32;
    const size_t S = calc_bytes(prec, b_type);
    const bool real = !dtype_complex(b_type);
    int single_log = 0, tile_log = 0;
    while (((size_t)2 << single_log) * S <= kRowTileBytes) ++single_log;
    while (((size_t)2 << tile_log) * S <= kTileBytes) ++tile_log;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < n_masks && e == cudaSuccess; ++i) {
        MaskPlan m = plan_mask(n, s, h_masks[i]);
        const int c = cp.chain[i];
        cudaStream_t ms = cp.chains > 1 ? chs->s[c] : cs;
        void* vws = workspace ? (void*)((char*)workspace + region_off[c]) : nullptr;
        BandMaskLaunch p{};
        p.bands = bands;
        p.b_t = b_type;
        p.c_t = c_type;
        p.calc = calc;
        p.real = real;
        p.anti = anti_masks != nullptr;
        p.anti_x = anti_masks ? anti_masks[i] : 0;
        p.n = n;
        p.s = s;
        p.x = m.x;
        p.h1 = m.h1;
        p.zc = m.zc;
        p.f = m.f;
        p.npairs = m.npairs;
        for (int j = 0; j < m.npairs; ++j) {
            p.t[j] = m.t[j];
            p.d[j] = m.d[j];
        }
        p.ws = vws;
        p.ws_elems = (uint64_t)m.npairs << m.f;
        p.out = C;
        p.out_row = i;
        p.out_elems = (uint64_t)n_masks * N;
        p.scale = std::ldexp(1.0, -n);
        const bool single = m.f <= single_log;
        p.log_l = single ? m.f : tile_log;
        p.threads = ((size_t)1 << p.log_l) * S >= 32 * 1024 && calc != Calc::F64 ? 512 : 256;
        // A mask the band cannot reach has no pairs: its row is written as zeros.
        if (m.npairs > 0) e = launch_band_first(p, st, ms);
        if (e == cudaSuccess && m.npairs > 0 && !single) {
            std::vector<StridedPass> passes = strided_schedule(p.log_l, m.f, S);
            for (size_t q = 0; q < passes.size() && e == cudaSuccess; ++q) {
                StridedLaunch sl{};
                sl.src = vws;
                sl.dst = vws;
                sl.calc = calc;
                sl.store = Store::RowBuf;
                sl.n = m.f;
                sl.b0 = passes[q].b0;
                sl.b1 = passes[q].b1;
                sl.log_w = passes[q].log_w;
                sl.x_begin = 0;
                sl.x_count = (uint64_t)m.npairs;
                sl.src_row0 = 0;
                sl.dst_row0 = 0;
                sl.src_elems = p.ws_elems;
                sl.dst_elems = p.ws_elems;
                sl.scale = 1.0;
                sl.threads = calc == Calc::F64 ? 256 : 512;
                sl.real = real;
                e = launch_strided(sl, st, ms);
            }
        }
        if (e == cudaSuccess) e = launch_band_expand(p, st, ms);
    }
    // the caller's stream completes after every chain (also after an error:
    // the joins keep the library streams ordered for the next call)
    if (cp.chains > 1)
        for (int c = 0; c < cp.chains; ++c) {
            const bool ok = cudaEventRecord(chs->join[c], chs->s[c]) == cudaSuccess &&
                            cudaStreamWaitEvent(cs, chs->join[c], 0) == cudaSuccess;
            if (!ok && e == cudaSuccess) e = cudaErrorUnknown;
        }
    return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

ptdr_status ptdr_decompose_structured(const void* bands, ptdr_dtype b_type, int n, int s,
                                      const uint64_t* h_masks, size_t n_masks, void* C,
                                      ptdr_dtype c_type, ptdr_precision prec, void* workspace,
                                      size_t workspace_bytes, void* stream)
{
    PTDR_TRACE();
    return decompose_band(bands, b_type, n, s, h_masks, n_masks, C, c_type, prec, workspace, workspace_bytes,
                          stream, nullptr);
}

// Anti-band matrices (Remark 1 of Sec. IV.A: I and Z swap roles with X and Y):
// A J is a band matrix for J = X (x) ... (x) X, so the masks are the band's
// masks XOR (2^n - 1).
ptdr_status ptdr_antistructured_masks(int n, int s, uint64_t* h_masks, size_t* count)
{
    ptdr_status v = ptdr_structured_masks(n, s, h_masks, count);
    if (v != PTDR_OK || !h_masks) return v;
    const uint64_t all = (1ull << n) - 1;
    for (size_t i = 0; i < *count; ++i) h_masks[i] ^= all;
    std::sort(h_masks, h_masks + *count);
    return PTDR_OK;
}

static ptdr_status band_masks_of(int n, const uint64_t* h_masks, size_t n_masks, std::vector<uint64_t>* out)
{
    if (!h_masks || n < 1 || n > 30) return PTDR_ERR_INVALID_ARG;
    const uint64_t all = (1ull << n) - 1;
    out->resize(n_masks);
    for (size_t i = 0; i < n_masks; ++i) {
        if (h_masks[i] > all) return PTDR_ERR_INVALID_ARG;
        (*out)[i] = h_masks[i] ^ all;
    }
    return PTDR_OK;
}

ptdr_status ptdr_antistructured_workspace_size(int n, int s, const uint64_t* h_masks, size_t n_masks,
                                               ptdr_dtype b_type, ptdr_dtype c_type, ptdr_precision prec,
                                               size_t* bytes)
{
    std::vector<uint64_t> xb;
    ptdr_status v = band_masks_of(n, h_masks, n_masks, &xb);
    if (v != PTDR_OK) return v;
    return ptdr_structured_workspace_size(n, s, xb.data(), n_masks, b_type, c_type, prec, bytes);
}

ptdr_status ptdr_decompose_antistructured(const void* antibands, ptdr_dtype b_type, int n, int s,
                                          const uint64_t* h_masks, size_t n_masks, void* C, ptdr_dtype c_type,
                                          ptdr_precision prec, void* workspace, size_t workspace_bytes, void* stream)
{
    PTDR_TRACE();
    std::vector<uint64_t> xb;
    ptdr_status v = band_masks_of(n, h_masks, n_masks, &xb);
    if (v != PTDR_OK) return v;
    return decompose_band(antibands, b_type, n, s, xb.data(), n_masks, C, c_type, prec, workspace, workspace_bytes,
                          stream, h_masks);
}

} // extern "C"
