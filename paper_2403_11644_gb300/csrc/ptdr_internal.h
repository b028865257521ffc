// Host-side declarations shared by the libptdr translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ptdr.h"

namespace ptdr {

// An NVTX range named after the entry point around each compute call of the C
// ABI: profilers (Nsight Systems, ncu --nvtx) attribute the kernels to the
// call; without an attached tool the push/pop cost a few nanoseconds.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};
#define PTDR_TRACE() ::ptdr::TraceRange ptdr_trace_range_(__func__)

// Which numeric path a launch takes.
enum class Calc { F32, F64 };

// Element type codes as stored in HBM.
inline size_t dtype_bytes(ptdr_dtype t)
{
    switch (t) {
    case PTDR_C64: return 8;
    case PTDR_C128: return 16;
    case PTDR_F32: return 4;
    case PTDR_F64: return 8;
    }
    return 0;
}
inline bool dtype_complex(ptdr_dtype t) { return t == PTDR_C64 || t == PTDR_C128; }

// Elements of a shared-memory tile of rows x (2^log_ls) complex values,
// padded by one element every 16 and one per row (bank-conflict avoidance).
inline size_t smem_elems(size_t rows, int log_ls)
{
    size_t ls = (size_t)1 << log_ls;
    return rows * (ls + ls / 16 + 1);
}

// ------------------------------------------------------------------ rows

// First pass over a tile of 2^log_r masks x a segment of 2^log_l elements of
// each row: load (gather from A / contiguous with phase from C / contiguous
// from an intermediate buffer), transform over the segment's bits, store
// (final phased output / contiguous intermediate / XOR-scatter into A).
enum class Load { GatherA, RowPhaseC, RowBuf };
enum class Store { RowPhaseOut, RowBuf, ScatterA };

struct TileLaunch {
    const void* src;
    void* dst;
    ptdr_dtype src_t, dst_t;
    Calc calc;
    Load load;
    Store store;
    int n;            // matrix is 2^n x 2^n
    int log_r;        // masks per tile
    int log_l;        // segment length
    uint64_t x_begin; // first mask handled by this launch
    uint64_t x_count; // masks handled (multiple of 2^log_r)
    uint64_t dst_row0; // mask whose row is dst row 0 (buffers may hold a chunk)
    uint64_t src_row0; // mask whose row is src row 0
    uint64_t src_elems, dst_elems; // extents for the checked build's index checks
    double scale;
    int threads;
    uint64_t src_row_mask; // gather from rows r & mask of a sheared tile set (0: all of A)
};

// Strided pass over bits [b0, b1) of each row of an intermediate buffer,
// tile = 2^(b1-b0) x 2^log_w elements.
struct StridedLaunch {
    const void* src; // intermediate buffer (rows of 2^n, row 0 = mask src_row0)
    void* dst;
    ptdr_dtype src_t, dst_t;
    Calc calc;
    Store store;
    int n, b0, b1, log_w;
    uint64_t x_begin, x_count, dst_row0, src_row0;
    uint64_t src_elems, dst_elems; // extents for the checked build's index checks
    double scale;
    int threads;
    bool real = false; // rows of real values (intermediate buffers only: Store::RowBuf)
};

cudaError_t launch_tile(const TileLaunch& p, unsigned int* status, cudaStream_t s);
cudaError_t launch_strided(const StridedLaunch& p, unsigned int* status, cudaStream_t s);

} // namespace ptdr
