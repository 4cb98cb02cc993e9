// Batched Gram + FGS kernels for s = 9 .. 16 (see batch_impl.cuh).
#include "batch_impl.cuh"

namespace sstep {
template cudaError_t launch_batch_gram_s<9>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<10>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<11>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<12>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<13>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<14>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<15>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
template cudaError_t launch_batch_gram_s<16>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
}  // namespace sstep
