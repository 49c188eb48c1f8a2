// Instantiations of the objective kernel for mode kValue (one file per mode so
// the build compiles them in parallel).
#include "eval_kernel.cuh"

namespace musr {

cudaError_t launch_eval_mode0(const Signature& s, int threads, int n_tiles, cudaStream_t st,
                                const EvalParams& p) {
#define MUSR_CASE(NE, NG, KT) \
    if (s.ne == NE && s.ng == NG && s.kt == KT) return launch_one<NE, NG, KT, kValue>(threads, n_tiles, st, p);
    MUSR_CASE(0, 0, 0) MUSR_CASE(0, 0, 1)
    MUSR_CASE(1, 0, 0) MUSR_CASE(1, 0, 1)
    MUSR_CASE(0, 1, 0) MUSR_CASE(0, 1, 1)
    MUSR_CASE(2, 0, 0) MUSR_CASE(2, 0, 1)
    MUSR_CASE(1, 1, 0) MUSR_CASE(1, 1, 1)
    MUSR_CASE(0, 2, 0) MUSR_CASE(0, 2, 1)
#undef MUSR_CASE
    return cudaErrorInvalidValue;
}

}  // namespace musr
