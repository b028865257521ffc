// Launch planning for the dense decompose/compose paths (host side).
#pragma once

#include <vector>

#include "ptdr_internal.h"

namespace ptdr {

constexpr int kMaxDenseN = 15;

// Shared-memory budget of one tile of the generic kernels (bytes, unpadded).
constexpr size_t kTileBytes = 64 * 1024;
// A whole row in one tile is allowed up to this size (one CTA per SM).
constexpr size_t kRowTileBytes = 128 * 1024;
// Workspace cap for the intermediate of chunked multi-pass launches.
constexpr size_t kChunkBytes = 256ull << 20;
// Intermediate of the fixed-point path per chunk of masks: small enough to stay in L2.
constexpr size_t kFixedChunkBytes = 128ull << 20;

struct StridedPass {
    int b0, b1, log_w;
};

enum class DenseKernel {
    Tiles,      // generic tile kernels (any n, FP32/FP64)
    Row14,      // n = 14 FP32 decompose: staged two-pass kernel (complex64, 16-byte
                // aligned), otherwise one CTA per mask with register rounds 5/5/4
    Staged15,   // n = 15 FP32 decompose complex64 -> complex64 (16-byte aligned):
                // staged two-pass kernel; otherwise the generic multi-pass plan
    Tc14,       // n = 14 split-bf16 decompose, tensor-core stage over column blocks
    Compose14,  // n = 14 FP32 compose complex64 -> complex64: staged two-pass kernel
    Rr,         // n = 9 .. 12 FP32 decompose complex64 -> complex64 (16-byte aligned):
                // register-round items, one CTA per 2^(13-n) masks; otherwise the generic tiles
    Fixed,      // exact 128-bit fixed-point transform (any n, decompose and compose)
};

struct DensePlan {
    bool compose = false;
    int n = 0;
    ptdr_dtype in_t = PTDR_C64, out_t = PTDR_C64;
    ptdr_precision prec = PTDR_PREC_FP32;
    Calc calc = Calc::F32;
    DenseKernel kernel = DenseKernel::Tiles;
    bool single = true;      // one tile pass covers a whole row
    int log_r = 0, log_l = 0; // first pass tile
    int threads = 256;
    std::vector<StridedPass> passes;
    bool buf_is_out = false; // intermediate lives in the output array
    uint64_t chunk = 0;      // masks per launch chunk (multi-pass)
    int pass_threads = 512;  // threads per CTA of the strided passes
    size_t ws_bytes = 0;
};

// Parameters of a generic multi-pass plan chosen by the autotuner (tune.cu):
// first-pass tile bytes and masks per tile, strided-pass tile bytes, threads.
struct TuneParams {
    int tile_log2, masks_log2, pass_tile_log2, threads;
};
// Whether the plan runs (or falls back to) the generic multi-pass kernels.
bool multipass_tunable(const DensePlan& p);
// Rebuilds the first-pass tile and the strided passes of a multi-pass plan
// with the given parameters (workspace and chunking unchanged); false if the
// plan is not multi-pass or the parameters do not fit it.
bool apply_multipass_tuning(DensePlan* p, const TuneParams& t);
// The tuned parameters cached for this plan on device `dev`, if any.
bool tuned_params_for(int dev, const DensePlan& p, TuneParams* out);

ptdr_status make_dense_plan(bool compose, int n, ptdr_dtype in_t, ptdr_dtype out_t,
                            ptdr_precision prec, DensePlan* plan);
ptdr_status execute_dense(const DensePlan& plan, const void* in, void* out, void* ws,
                          double scale, unsigned int* status, cudaStream_t s);

// Splits bits [b0, n) into strided passes whose tiles fit kTileBytes.
std::vector<StridedPass> strided_schedule(int b0, int n, size_t elem_bytes);
// The same with a tile budget of tile_bytes instead of kTileBytes.
std::vector<StridedPass> strided_schedule_budget(int b0, int n, size_t elem_bytes, size_t tile_bytes);

cudaError_t launch_row14(const void* A, ptdr_dtype a_t, void* C, ptdr_dtype c_t,
                         unsigned int* status, cudaStream_t s);
cudaError_t launch_dense_staged(int n, const void* A, void* C, void* ws, unsigned int* status, cudaStream_t s);
size_t dense_staged_workspace(int n);
cudaError_t launch_tc14_pipe(const void* A, void* C, bool real_out, void* ws, unsigned int* status, cudaStream_t s);
size_t tc14_pipe_workspace();
cudaError_t launch_compose14_staged(const void* C, void* A, double scale, void* ws, unsigned int* status,
                                    cudaStream_t s);
size_t compose14_staged_workspace();
size_t fixed_ws_header();
cudaError_t launch_fixed(const DensePlan& plan, const void* in, void* out, void* ws, double scale,
                         unsigned int* status, cudaStream_t s);
cudaError_t launch_rr_dense(int n, const void* A, void* C, double scale, unsigned int* status, cudaStream_t s);

// shared helpers (ptdr_api.cu)
ptdr_status device_ready(int* dev);
ptdr_status status_word(int dev, unsigned int** out);
ptdr_status check_device_ptr(const void* p);
bool overlaps(const void* a, size_t na, const void* b, size_t nb);
bool fault_injected(const char* what);
// Bound (ns) of the device-side waits of the persistent kernels for other CTAs:
// PTDR_WAIT_NS from the environment at each launch, default 1 s, at most 60 s.
unsigned long long wait_limit_ns();

} // namespace ptdr
