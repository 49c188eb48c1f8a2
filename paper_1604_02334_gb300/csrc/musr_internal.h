// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "musr.h"

namespace musr {

constexpr int kMaxOsc = 2;                         // precession lines per run
constexpr int kMaxRoles = 2 + 4 * kMaxOsc + 2;     // N0, bkg, 4 per line, 2 for KT
constexpr int kBinsPerThread = 8;                  // consecutive bins per thread (2 x float4)
constexpr int kMaxThreads = 256;                   // block size upper bound
constexpr int kMaxWarps = kMaxThreads / 32;

// Kernel "signature": how many precession lines of each relaxation kind and
// whether a static Gaussian Kubo-Toyabe term is present.  Exponential lines
// come first in the kernel's role order, Gaussian lines second.
struct Signature {
    int ne = 0, ng = 0, kt = 0;
    int n_osc() const { return ne + ng; }
    int roles() const { return 2 + 4 * n_osc() + 2 * kt; }
};

// Evaluation modes (kernel template parameter).
enum Mode { kValue = 0, kGrad = 1, kGN = 2, kModel = 3 };

inline int n_acc(int mode, int R) {
    return mode == kValue ? 1 : mode == kGrad ? 1 + R : mode == kGN ? 1 + R + R * (R + 1) / 2 : 0;
}

// Everything one launch of the objective kernel reads or writes.
struct EvalParams {
    // run layout (device)
    const float* data;            // padded, histogram-major
    const int64_t* hist_off;      // [K] float offset of histogram k in data
    const int32_t* hist_nbins;    // [K]
    const int32_t* tile_hist;     // [n_tiles]
    const int32_t* tile_start;    // [n_tiles] first bin of the tile
    const int32_t* hist_first_tile;  // [K]
    const int32_t* hist_ntiles;      // [K]
    const int32_t* role_theta;    // [K][kMaxRoles][2] theta indices (or -1) per role
    const double* theta;          // [P]
    double t0, dt, inv_tau, gamma;
    int K, P, obj;
    // reduction scratch
    double* partial;              // [n_tiles][nacc]
    double* hist_sum;             // [K][nacc]
    unsigned* hist_count;         // [K]   (self-resetting)
    unsigned* global_count;       // [1]   (self-resetting)
    unsigned* flags;              // [1]   (self-resetting)
    const int32_t* csr_ptr;       // [n_out + 1]
    const int32_t* csr_src;       // sources: k * nacc + acc
    int n_out;
    double* out;                  // [n_out]
    int32_t* status_out;          // [1] or null
    // model output (kModel)
    float* model_out;
    const int64_t* model_off;     // [K] offsets into model_out
};

// Launch the objective kernel for a signature / mode (eval_*.cu).
cudaError_t launch_eval(const Signature& sig, int mode, int threads, int n_tiles,
                        cudaStream_t stream, const EvalParams& p);

}  // namespace musr
