// Instantiations of the objective kernel for mode kGrad (one file per mode so
// the build compiles them in parallel).
#include "eval_kernel.cuh"

namespace musr {

cudaError_t launch_eval_mode1(const Signature& s, int threads, int n_tiles, cudaStream_t st,
                                const EvalParams& p) {
#define MUSR_CASE(NE, NG, NS, KT)                                      \
    if (s.ne == NE && s.ng == NG && s.ns == NS && s.kt == KT) \
        return launch_one<NE, NG, NS, KT, kGrad>(threads, n_tiles, st, p);
    MUSR_FOR_EACH_SIGNATURE(MUSR_CASE)
#undef MUSR_CASE
    return cudaErrorInvalidValue;
}

}  // namespace musr
