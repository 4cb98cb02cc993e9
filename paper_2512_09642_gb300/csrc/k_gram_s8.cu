// Gram + FGS kernels for s = 29 .. 32 (see gram_impl.cuh).
#include "gram_impl.cuh"

namespace sstep {
template cudaError_t launch_gram_s<29>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<30>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<31>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<32>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<29>(const GramArgs&);
template int gram_occupancy_s<30>(const GramArgs&);
template int gram_occupancy_s<31>(const GramArgs&);
template int gram_occupancy_s<32>(const GramArgs&);
}  // namespace sstep
