// Host-side planning and execution of the dense decompose/compose launches.
#include <algorithm>

#include "plan.h"

namespace ptdr {

static int ilog2(size_t v)
{
    int l = 0;
    while (((size_t)1 << (l + 1)) <= v) ++l;
    return l;
}

std::vector<StridedPass> strided_schedule(int b0, int n, size_t elem_bytes)
{
    return strided_schedule_budget(b0, n, elem_bytes, kTileBytes);
}

std::vector<StridedPass> strided_schedule_budget(int b0, int n, size_t elem_bytes, size_t tile_bytes)
{
    // Each strided tile is 2^nb rows (the bits transformed) x 2^log_w
    // consecutive elements (>= 32 bytes so that every row piece is a whole
    // sector); as many bits per pass as the tile budget allows.
    std::vector<StridedPass> out;
    const int tile_log = ilog2(tile_bytes / elem_bytes);
    const int min_w = std::max(0, ilog2(32 / elem_bytes));
    int b = b0;
    while (b < n) {
        int nb = std::min(n - b, tile_log - min_w);
        int log_w = std::min(tile_log - nb, b); // columns come from the bits below b
        out.push_back({b, b + nb, log_w});
        b += nb;
    }
    return out;
}

ptdr_status make_dense_plan(bool compose, int n, ptdr_dtype in_t, ptdr_dtype out_t,
                            ptdr_precision prec, DensePlan* plan)
{
    if (prec == PTDR_PREC_FIXED_I128) {
        // 32-byte fixed-point complex values: rows of up to 4096 in one tile,
        // longer rows as a first pass and strided passes through an
        // intermediate chunk of masks that stays in L2
        DensePlan p;
        p.compose = compose;
        p.n = n;
        p.in_t = in_t;
        p.out_t = out_t;
        p.prec = prec;
        p.kernel = DenseKernel::Fixed;
        const size_t S = 32, N = (size_t)1 << n, row_bytes = N * S;
        p.threads = 512;
        if (row_bytes <= kRowTileBytes) {
            p.single = true;
            p.log_l = n;
            int lr = 0;
            while (lr < 4 && lr < n && (row_bytes << (lr + 1)) <= std::max(row_bytes, kTileBytes)) ++lr;
            p.log_r = lr;
            p.ws_bytes = fixed_ws_header();
        } else {
            p.single = false;
            p.log_r = compose ? 0 : 2;
            p.log_l = ilog2(kTileBytes / S) - p.log_r;
            p.passes = strided_schedule(p.log_l, n, S);
            p.chunk = std::max<size_t>((size_t)1 << p.log_r, std::min<size_t>(N, kFixedChunkBytes / row_bytes));
            p.ws_bytes = fixed_ws_header() + p.chunk * row_bytes;
        }
        *plan = p;
        return PTDR_OK;
    }
    if (prec == PTDR_PREC_SPLIT_BF16_TC) {
        // the tensor-core path covers the n = 14 complex64 workload (complex64
        // coefficients, or float32 real parts in the Hermitian real-output mode)
        if (compose || n != 14 || in_t != PTDR_C64 || (out_t != PTDR_C64 && out_t != PTDR_F32)) return PTDR_ERR_UNSUPPORTED;
        DensePlan p;
        p.compose = false;
        p.n = n;
        p.in_t = in_t;
        p.out_t = out_t;
        p.prec = prec;
        p.calc = Calc::F32;
        p.kernel = DenseKernel::Tc14;
        p.single = true;
        p.ws_bytes = tc14_pipe_workspace();
        *plan = p;
        return PTDR_OK;
    }
    DensePlan p;
    p.compose = compose;
    p.n = n;
    p.in_t = in_t;
    p.out_t = out_t;
    p.prec = prec;
    p.calc = prec == PTDR_PREC_FP64 ? Calc::F64 : Calc::F32;
    const size_t S = p.calc == Calc::F64 ? 16 : 8;
    const size_t N = (size_t)1 << n;
    const size_t row_bytes = N * S;
    if (compose && n == 14 && p.calc == Calc::F32 && in_t == PTDR_C64 && out_t == PTDR_C64) {
        p.kernel = DenseKernel::Compose14;
        p.single = true;
        p.ws_bytes = compose14_staged_workspace();
        *plan = p;
        return PTDR_OK;
    }
    if (!compose && n == 14 && p.calc == Calc::F32) {
        p.kernel = DenseKernel::Row14;
        p.single = true;
        // the clustered complex64 kernel exchanges through a scratch in the workspace
        if (in_t == PTDR_C64 && out_t == PTDR_C64) p.ws_bytes = dense_staged_workspace(14);
        *plan = p;
        return PTDR_OK;
    }
    if (row_bytes <= kRowTileBytes) {
        p.single = true;
        p.log_l = n;
        int lr = 0;
        while (lr < 4 && lr < n && (row_bytes << (lr + 1)) <= std::max(row_bytes, kTileBytes)) ++lr;
        p.log_r = lr;
        const size_t tile = row_bytes << lr;
        // FP64 tiles run faster as 256-thread CTAs (n = 12: 1.01 -> 0.89 ms)
        p.threads = tile >= 32 * 1024 && p.calc != Calc::F64 ? 512 : 256;
        // the generic fields above remain the fallback for misaligned buffers
        if (!compose && p.calc == Calc::F32 && out_t == PTDR_C64 && in_t == PTDR_C64 && n >= 9 && n <= 12)
            p.kernel = DenseKernel::Rr;
    } else {
        p.single = false;
        // Decompose: 4 masks per first-pass tile, so that each row of A
        // supplies a 4-value piece (a whole 32-byte sector of complex64)
        // instead of one value per sector; A is far larger than L2 here, so
        // the rest of a sector is not there when its own mask is gathered.
        p.log_r = compose ? 0 : 2;
        p.log_l = ilog2(kTileBytes / S) - p.log_r;
        // FP64 tiles and passes run faster as 256-thread CTAs
        p.threads = p.calc == Calc::F64 ? 256 : 512;
        p.pass_threads = p.threads;
        p.passes = strided_schedule(p.log_l, n, S);
        // Decompose can keep the intermediate in C when C has the compute
        // type; compose scatters into A, so its intermediate never aliases A.
        const bool same = (p.calc == Calc::F32 && out_t == PTDR_C64) ||
                          (p.calc == Calc::F64 && out_t == PTDR_C128);
        p.buf_is_out = !compose && same;
        if (p.buf_is_out) {
            p.chunk = N;
            p.ws_bytes = 0;
        } else {
            p.chunk = std::max<size_t>(1, std::min<size_t>(N, kChunkBytes / row_bytes));
            p.ws_bytes = p.chunk * row_bytes;
        }
        if (p.chunk % ((size_t)1 << p.log_r)) { // a chunk holds whole tiles of masks
            p.log_l += p.log_r;
            p.log_r = 0;
            p.passes = strided_schedule(p.log_l, n, S);
        }
        // n = 15 FP32 complex64 -> complex64: the staged two-pass kernel (the
        // multi-pass fields above stay the plan for unaligned buffers)
        if (!compose && n == 15 && p.calc == Calc::F32 && in_t == PTDR_C64 && out_t == PTDR_C64) {
            p.kernel = DenseKernel::Staged15;
            p.ws_bytes = std::max(p.ws_bytes, dense_staged_workspace(15));
        }
    }
    *plan = p;
    return PTDR_OK;
}

bool multipass_tunable(const DensePlan& p)
{
    // (the staged n = 14/15 kernels and the fixed-point path have their own schedules)
    return !p.single && p.kernel == DenseKernel::Tiles;
}

bool apply_multipass_tuning(DensePlan* p, const TuneParams& t)
{
    if (!multipass_tunable(*p)) return false;
    if (t.tile_log2 < 13 || t.tile_log2 > 17 || t.pass_tile_log2 < 13 || t.pass_tile_log2 > 17 ||
        t.masks_log2 < 0 || t.masks_log2 > 4 || (t.threads != 256 && t.threads != 512))
        return false;
    const size_t S = p->calc == Calc::F64 ? 16 : 8;
    const int elems_log = t.tile_log2 - ilog2(S);
    int log_r = p->compose ? 0 : t.masks_log2;
    while (log_r > 0 && p->chunk % ((size_t)1 << log_r)) --log_r; // a chunk holds whole tiles of masks
    const int log_l = elems_log - log_r;
    if (log_l < 5 || log_l >= p->n) return false; // the first pass must leave bits for the strided passes
    DensePlan q = *p;
    q.kernel = DenseKernel::Tiles;
    q.log_r = log_r;
    q.log_l = log_l;
    q.threads = t.threads;
    q.pass_threads = t.threads;
    q.passes = strided_schedule_budget(log_l, p->n, S, (size_t)1 << t.pass_tile_log2);
    *p = q;
    return true;
}

ptdr_status execute_dense(const DensePlan& p, const void* in, void* out, void* ws, double scale,
                          unsigned int* st, cudaStream_t s)
{
    const uint64_t N = 1ull << p.n;
    cudaError_t e = cudaSuccess;
    if (p.kernel == DenseKernel::Fixed) {
        e = launch_fixed(p, in, out, ws, scale, st, s);
        return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
    }
    if (p.kernel == DenseKernel::Tc14) {
        // 32-byte vector loads and stores of A, C and the staging rows
        if ((uintptr_t)in % 32 || (uintptr_t)out % 32 || (uintptr_t)ws % 32) return PTDR_ERR_INVALID_ARG;
        e = launch_tc14_pipe(in, out, p.out_t == PTDR_F32, ws, st, s);
        return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
    }
    if (p.kernel == DenseKernel::Compose14) {
        // 16-byte stores of A rows; otherwise the generic tile kernels
        if (ws && (uintptr_t)out % 16 == 0 && (uintptr_t)in % 8 == 0) {
            e = launch_compose14_staged(in, out, scale, ws, st, s);
            return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
        }
        DensePlan g = p;
        g.kernel = DenseKernel::Tiles;
        g.single = true;
        g.log_l = p.n;
        g.log_r = 0;
        g.threads = 512;
        return execute_dense(g, in, out, ws, scale, st, s);
    }
    if (p.kernel == DenseKernel::Rr) {
        // 16-byte piece copies and 16-byte stores; otherwise the generic tile kernel
        if ((uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0) {
            e = launch_rr_dense(p.n, in, out, scale, st, s);
            return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
        }
        DensePlan g = p;
        g.kernel = DenseKernel::Tiles;
        return execute_dense(g, in, out, ws, scale, st, s);
    }
    if (p.kernel == DenseKernel::Staged15) {
        if (ws && (uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0) {
            e = launch_dense_staged(15, in, out, ws, st, s);
            return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
        }
        DensePlan g = p;
        g.kernel = DenseKernel::Tiles;
        return execute_dense(g, in, out, ws, scale, st, s);
    }
    if (p.kernel == DenseKernel::Row14) {
        // complex64 -> complex64 with a 16-byte aligned input takes the
        // clustered tile kernel; other type pairs the one-mask-per-CTA kernel
        if (ws && p.in_t == PTDR_C64 && p.out_t == PTDR_C64 && (uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0)
            e = launch_dense_staged(14, in, out, ws, st, s);
        else
            e = launch_row14(in, p.in_t, out, p.out_t, st, s);
        return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
    }
    if (p.single) {
        TileLaunch t{};
        t.src = in;
        t.dst = out;
        t.src_t = p.in_t;
        t.dst_t = p.out_t;
        t.calc = p.calc;
        t.load = p.compose ? Load::RowPhaseC : Load::GatherA;
        t.store = p.compose ? Store::ScatterA : Store::RowPhaseOut;
        t.n = p.n;
        t.log_r = p.log_r;
        t.log_l = p.log_l;
        t.x_begin = 0;
        t.x_count = N;
        t.dst_row0 = 0;
        t.src_row0 = 0;
        t.src_elems = N * N;
        t.dst_elems = N * N;
        t.scale = scale;
        t.threads = p.threads;
        e = launch_tile(t, st, s);
        return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
    }
    for (uint64_t x0 = 0; x0 < N && e == cudaSuccess; x0 += p.chunk) {
        void* buf = p.buf_is_out ? out : ws;
        const uint64_t buf_row0 = p.buf_is_out ? 0 : x0;
        const uint64_t buf_elems = p.buf_is_out ? N * N : p.chunk * N;
        TileLaunch t{};
        t.src = in;
        t.dst = buf;
        t.src_t = p.in_t;
        t.dst_t = p.out_t; // unused for RowBuf
        t.calc = p.calc;
        t.load = p.compose ? Load::RowPhaseC : Load::GatherA;
        t.store = Store::RowBuf;
        t.n = p.n;
        t.log_r = p.log_r;
        t.log_l = p.log_l;
        t.x_begin = x0;
        t.x_count = p.chunk;
        t.dst_row0 = buf_row0;
        t.src_row0 = 0;
        t.src_elems = N * N;
        t.dst_elems = buf_elems;
        // compose applies its scale with the phase on load; decompose at the end
        t.scale = p.compose ? scale : 1.0;
        t.threads = p.threads;
        e = launch_tile(t, st, s);
        for (size_t i = 0; i < p.passes.size() && e == cudaSuccess; ++i) {
            const bool last = i + 1 == p.passes.size();
            StridedLaunch q{};
            q.src = buf;
            q.src_t = p.out_t;
            q.calc = p.calc;
            q.n = p.n;
            q.b0 = p.passes[i].b0;
            q.b1 = p.passes[i].b1;
            q.log_w = p.passes[i].log_w;
            q.x_begin = x0;
            q.x_count = p.chunk;
            q.src_row0 = buf_row0;
            q.src_elems = buf_elems;
            q.dst_elems = last ? N * N : buf_elems;
            q.threads = p.pass_threads;
            if (!last) {
                q.dst = buf;
                q.store = Store::RowBuf;
                q.dst_row0 = buf_row0;
                q.scale = 1.0;
            } else {
                q.dst = out;
                q.dst_t = p.out_t;
                q.store = p.compose ? Store::ScatterA : Store::RowPhaseOut;
                q.dst_row0 = 0;
                q.scale = p.compose ? 1.0 : scale;
            }
            e = launch_strided(q, st, s);
        }
    }
    return e == cudaSuccess ? PTDR_OK : PTDR_ERR_CUDA;
}

} // namespace ptdr
