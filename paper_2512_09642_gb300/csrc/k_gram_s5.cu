// Gram + FGS kernels for s = 17 .. 20 (see gram_impl.cuh).
#include "gram_impl.cuh"

namespace sstep {
template cudaError_t launch_gram_s<17>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<18>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<19>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<20>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<17>(const GramArgs&);
template int gram_occupancy_s<18>(const GramArgs&);
template int gram_occupancy_s<19>(const GramArgs&);
template int gram_occupancy_s<20>(const GramArgs&);
}  // namespace sstep
