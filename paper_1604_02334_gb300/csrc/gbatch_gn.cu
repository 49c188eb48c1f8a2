// Instantiations of the batched adjoint kernel, mode kGN (one translation unit
// per mode keeps the build parallel).
#include "gbatch_kernel.cuh"

namespace musr {
template cudaError_t launch_gbatch_mode<kGN>(const Signature& s, int blocks, int threads, size_t smem,
                                               cudaStream_t st, const GParams& p);
}  // namespace musr
