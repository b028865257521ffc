// Launch parameters of the batched (persistent, many-matrix) path.
#pragma once

#include "ptdr_internal.h"

namespace ptdr {

constexpr int kBatchMaxN = 13;

// Device tables in the caller's workspace, written by the planner kernel.
struct BatchTables {
    int* hdr;      // [0] queue head, [1] total items, [2] ranked matrices
    int* order;    // matrix index by rank (largest n first)
    int* start;    // first work item of each rank
    int max_items; // capacity check against the host's count
};

struct BatchLaunch {
    const void* const* d_A;
    void* const* d_C;
    const int* d_n;
    int count;
    ptdr_dtype a_t, c_t;
    Calc calc;
    int tile_log; // log2 of the tile budget in elements
    int max_n;
};

cudaError_t launch_batched(const BatchLaunch& p, const BatchTables& tab, unsigned int* status,
                           cudaStream_t s);
int batched_items(int n, int tile_log);

} // namespace ptdr
