// Gram + FGS kernels for s = 21 .. 24 (see gram_impl.cuh).
#include "gram_impl.cuh"

namespace sstep {
template cudaError_t launch_gram_s<21>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<22>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<23>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_gram_s<24>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
template int gram_occupancy_s<21>(const GramArgs&);
template int gram_occupancy_s<22>(const GramArgs&);
template int gram_occupancy_s<23>(const GramArgs&);
template int gram_occupancy_s<24>(const GramArgs&);
}  // namespace sstep
