// Launch parameters of the band-diagonal (structured) path.
#pragma once

#include "ptdr_internal.h"

namespace ptdr {

constexpr int kMaxBandPairs = 64; // |T_x| <= s + 1, so s <= 63

// Everything one mask needs, passed by value to its kernels.
struct BandMaskLaunch {
    const void* bands;
    ptdr_dtype b_t, c_t;
    Calc calc;
    int n, s;
    uint64_t x;   // the mask
    int h1;       // msb(x) + 1 (0 for x = 0)
    int zc;       // zero bits of x below h1
    int f;        // free bits n - |x|: each V row has 2^f values
    int log_l;    // first-pass tile length (<= f)
    int npairs;   // |T_x|
    uint64_t t[kMaxBandPairs];
    int64_t d[kMaxBandPairs]; // x - 2 t: the band each pair reads
    bool real;    // real band: V rows hold real values
    bool anti;    // anti-band: the storage is the band matrix B = A J and x = x_A ^ (2^n - 1)
    uint64_t anti_x; // the anti-band mask x_A (phase (-1)^{|z|} (-i)^{|x_A & z|})
    void* ws;     // V rows, npairs x 2^f compute-type values (complex, or real for a real band)
    uint64_t ws_elems;
    void* out;    // output array
    uint64_t out_row, out_elems;
    double scale;
    int threads;
};

cudaError_t launch_band_first(const BandMaskLaunch& p, unsigned int* status, cudaStream_t s);
cudaError_t launch_band_expand(const BandMaskLaunch& p, unsigned int* status, cudaStream_t s);

} // namespace ptdr
