// Gram + FGS kernels for s = 13 .. 16 (see gram_impl.cuh).
#include "gram_impl.cuh"

namespace sstep {
template cudaError_t launch_gram_s<13>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<14>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<15>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<16>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<13>(const GramArgs&);
template int gram_occupancy_s<14>(const GramArgs&);
template int gram_occupancy_s<15>(const GramArgs&);
template int gram_occupancy_s<16>(const GramArgs&);
}  // namespace sstep
