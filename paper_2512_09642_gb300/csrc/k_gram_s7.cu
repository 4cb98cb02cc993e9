// Gram + FGS kernels for s = 25 .. 28 (see gram_impl.cuh).
#include "gram_impl.cuh"

namespace sstep {
template cudaError_t launch_gram_s<25>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<26>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<27>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<28>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<25>(const GramArgs&);
template int gram_occupancy_s<26>(const GramArgs&);
template int gram_occupancy_s<27>(const GramArgs&);
template int gram_occupancy_s<28>(const GramArgs&);
}  // namespace sstep
