// Batched Gram + FGS kernels for s = 1 .. 8 (see batch_impl.cuh).
#include "batch_impl.cuh"

namespace sstep {
template cudaError_t launch_batch_gram_s<1>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<2>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<3>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<4>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<5>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<6>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<7>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<8>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
}  // namespace sstep
