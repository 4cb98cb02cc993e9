// Gram + FGS kernels for s = 5 .. 8 (see gram_impl.cuh).
#include "gram_impl.cuh"

namespace sstep {
template cudaError_t launch_gram_s<5>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<6>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<7>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<8>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<5>(const GramArgs&);
template int gram_occupancy_s<6>(const GramArgs&);
template int gram_occupancy_s<7>(const GramArgs&);
template int gram_occupancy_s<8>(const GramArgs&);
}  // namespace sstep
