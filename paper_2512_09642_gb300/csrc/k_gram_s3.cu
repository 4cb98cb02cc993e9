// Gram + FGS kernels for s = 9 .. 12 (see gram_impl.cuh).
#include "gram_impl.cuh"

namespace sstep {
template cudaError_t launch_gram_s<9>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<10>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<11>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<12>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<9>(const GramArgs&);
template int gram_occupancy_s<10>(const GramArgs&);
template int gram_occupancy_s<11>(const GramArgs&);
template int gram_occupancy_s<12>(const GramArgs&);
}  // namespace sstep
