// Matrix-free decomposition: the paper notes (Sec. V.B) that the walk never
// needs the whole input stored -- entries that can be computed (from a
// function, say) are enough.  Here the masks are taken in x-blocks of 2^a
// (a = min(7, n)); the entries block xt gathers, A[k ^ x][k] for its 2^a masks
// x and every column k, all lie in the sheared tile set
//     S[i][k] = A[((k >> a) ^ xt) 2^a + i][k],   i < 2^a, k < 2^n,
// i.e. the 2^a x 2^a tiles (cb ^ xt, cb) of A, one per column block cb.  Each
// tile of A belongs to exactly one x-block, so a caller callback that fills S
// block after block produces every entry of A once, and the device holds
// 2^a rows of it instead of 2^n.  The block's masks then run the generic
// kernels with the gather reading row (k ^ x) & (2^a - 1) of S.
#include <algorithm>

#include "plan.h"

using namespace ptdr;

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct FreeLayout {
    DensePlan plan;
    int a;
    size_t s_bytes, buf_bytes, total;
};

ptdr_status free_layout(int n, ptdr_dtype a_t, ptdr_dtype c_t, ptdr_precision prec, FreeLayout* out)
{
    if (n < 1 || n > kMaxDenseN) return PTDR_ERR_INVALID_ARG;
    if ((int)a_t < PTDR_C64 || (int)a_t > PTDR_F64 || (int)c_t < PTDR_C64 || (int)c_t > PTDR_F64)
        return PTDR_ERR_INVALID_ARG;
    if ((int)prec < PTDR_PREC_FP64 || (int)prec > PTDR_PREC_FIXED_I128) return PTDR_ERR_INVALID_ARG;
    if (prec != PTDR_PREC_FP64 && prec != PTDR_PREC_FP32) return PTDR_ERR_UNSUPPORTED;
    DensePlan p;
    ptdr_status v = make_dense_plan(false, n, a_t, c_t, prec, &p);
    if (v != PTDR_OK) return v;
    // the generic kernels: the dedicated n = 9 .. 15 kernels read A directly
    if (p.kernel == DenseKernel::Row14) {
        p.single = true;
        p.log_l = n;
        p.log_r = 0;
        p.threads = 512;
    }
    p.kernel = DenseKernel::Tiles;
    FreeLayout L;
    L.a = std::min(7, n);
    if (p.log_r > L.a) return PTDR_ERR_INTERNAL;
    const size_t N = (size_t)1 << n;
    const size_t S = p.calc == Calc::F64 ? 16 : 8;
    L.s_bytes = align256(((size_t)1 << L.a) * N * dtype_bytes(a_t));
    L.buf_bytes = (!p.single && !p.buf_is_out) ? align256(((size_t)1 << L.a) * N * S) : 0;
    L.total = L.s_bytes + L.buf_bytes;
    L.plan = p;
    *out = L;
    return PTDR_OK;
}

} // namespace

extern "C" {

ptdr_status ptdr_matrix_free_workspace_size(int n, ptdr_dtype a_type, ptdr_dtype c_type, ptdr_precision prec,
                                            size_t* bytes)
{
    if (!bytes) return PTDR_ERR_INVALID_ARG;
    FreeLayout L;
    ptdr_status v = free_layout(n, a_type, c_type, prec, &L);
    if (v != PTDR_OK) return v;
    *bytes = L.total;
    return PTDR_OK;
}

ptdr_status ptdr_decompose_matrix_free(int n, ptdr_dtype a_type, ptdr_tile_fn fill, void* user, void* C,
                                       ptdr_dtype c_type, ptdr_precision prec, void* workspace,
                                       size_t workspace_bytes, void* stream)
{
    PTDR_TRACE();
    if (!fill || !C) return PTDR_ERR_INVALID_ARG;
    FreeLayout L;
    ptdr_status v = free_layout(n, a_type, c_type, prec, &L);
    if (v != PTDR_OK) return v;
    const uint64_t N = 1ull << n;
    if ((uintptr_t)C % dtype_bytes(c_type)) return PTDR_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < L.total || (uintptr_t)workspace % 256) return PTDR_ERR_WORKSPACE;
    if (overlaps(workspace, L.total, C, N * N * dtype_bytes(c_type))) return PTDR_ERR_INVALID_ARG;
    if (fault_injected("plan")) return PTDR_ERR_INTERNAL;
    int dev = 0;
    v = device_ready(&dev);
    if (v != PTDR_OK) return v;
    if (check_device_ptr(C) != PTDR_OK || check_device_ptr(workspace) != PTDR_OK) return PTDR_ERR_INVALID_ARG;
    unsigned int* st = nullptr;
    v = status_word(dev, &st);
    if (v != PTDR_OK) return v;
    if (fault_injected("launch")) return PTDR_ERR_CUDA;

    const DensePlan& p = L.plan;
    const uint64_t B = 1ull << L.a; // masks per x-block
    void* S = workspace;
    void* wbuf = (char*)workspace + L.s_bytes;
    cudaStream_t s = (cudaStream_t)stream;
    const double scale = std::ldexp(1.0, -n);
    cudaError_t e = cudaSuccess;
    for (uint64_t xt = 0; xt < (N >> L.a) && e == cudaSuccess; ++xt) {
        if (fill(user, n, xt, L.a, S, stream) != 0) return PTDR_ERR_INTERNAL;
        const uint64_t x0 = xt * B;
        TileLaunch t{};
        t.src = S;
        t.src_t = a_type;
        t.calc = p.calc;
        t.load = Load::GatherA;
        t.n = n;
        t.log_r = p.log_r;
        t.log_l = p.log_l;
        t.x_begin = x0;
        t.x_count = B;
        t.src_row0 = 0;
        t.src_elems = B * N;
        t.src_row_mask = B - 1;
        t.threads = p.threads;
        if (p.single) {
            t.dst = C;
            t.dst_t = c_type;
            t.store = Store::RowPhaseOut;
            t.dst_row0 = 0;
            t.dst_elems = N * N;
            t.scale = scale;
            e = launch_tile(t, st, s);
            continue;
        }
        // first pass into the intermediate (C itself when it has the compute type),
        // then the strided passes over the high bits; the last one writes C
        void* buf = p.buf_is_out ? C : wbuf;
        const uint64_t buf_row0 = p.buf_is_out ? 0 : x0;
        const uint64_t buf_elems = p.buf_is_out ? N * N : B * N;
        t.dst = buf;
        t.dst_t = c_type;
        t.store = Store::RowBuf;
        t.dst_row0 = buf_row0;
        t.dst_elems = buf_elems;
        t.scale = 1.0;
        e = launch_tile(t, st, s);
        for (size_t i = 0; i < p.passes.size() && e == cudaSuccess; ++i) {
            const bool last = i + 1 == p.passes.size();
            StridedLaunch q{};
            q.src = buf;
            q.src_t = c_type;
            q.calc = p.calc;
            q.n = n;
            q.b0 = p.passes[i].b0;
            q.b1 = p.passes[i].b1;
            q.log_w = p.passes[i].log_w;
            q.x_begin = x0;
            q.x_count = B;
            q.src_row0 = buf_row0;
            q.src_elems = buf_elems;
            q.threads = p.pass_threads;
            if (!last) {
                q.dst = buf;
                q.store = Store::RowBuf;
                q.dst_row0 = buf_row0;
                q.dst_elems = buf_elems;
                q.scale = 1.0;
            } else {
                q.dst = C;
                q.dst_t = c_type;
                q.store = Store::RowPhaseOut;
                q.dst_row0 = 0;
                q.dst_elems = N * N;
                q.scale = scale;
            }
            e = launch_strided(q, st, s);
        }
    }
    return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

} // extern "C"
