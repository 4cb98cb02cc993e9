// Gram + FGS kernels for s = 1 .. 4 (see gram_impl.cuh).
#include "gram_impl.cuh"

namespace sstep {
template cudaError_t launch_gram_s<1>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<2>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<3>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<4>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<1>(const GramArgs&);
template int gram_occupancy_s<2>(const GramArgs&);
template int gram_occupancy_s<3>(const GramArgs&);
template int gram_occupancy_s<4>(const GramArgs&);
}  // namespace sstep
