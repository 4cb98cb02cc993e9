// Gram + FGS kernels for one basis size s (see gram_impl.cuh). build.py compiles this file
// once per s = 1 .. 32 with -DSSTEP_INST_S=<s>, so the 32 instantiations, whose cost grows
// steeply with s, compile in parallel.
#include "gram_impl.cuh"

#ifndef SSTEP_INST_S
#error "compile once per basis size with -DSSTEP_INST_S=<s>, 1 <= s <= 32"
#endif

namespace sstep {
template cudaError_t launch_gram_s<SSTEP_INST_S>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<SSTEP_INST_S>(const GramArgs&);
template cudaError_t launch_moments_finish_s<SSTEP_INST_S>(const GramArgs&, const void*, int, double*, int, Ctl*,
                                                           cudaStream_t);
}  // namespace sstep
