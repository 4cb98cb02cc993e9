// Batched Gram + FGS kernels for one basis size s (see batch_impl.cuh). build.py compiles
// this file once per s = 1 .. 16 with -DSSTEP_INST_S=<s>.
#include "batch_impl.cuh"

#ifndef SSTEP_INST_S
#error "compile once per basis size with -DSSTEP_INST_S=<s>, 1 <= s <= 16"
#endif

namespace sstep {
template cudaError_t launch_batch_gram_s<SSTEP_INST_S>(const BatchDev&, int, int, bool, const double*, int,
                                                       cudaStream_t);
}  // namespace sstep
