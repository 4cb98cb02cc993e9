// Dispatch of the batched Gram + FGS kernel over s (instantiated by k_batch_gram_inst.cu, once per s).
#include "batch_impl.cuh"

namespace sstep {

#define SSTEP_EXTERN_BGRAM(S) \
    extern template cudaError_t launch_batch_gram_s<S>(const BatchDev&, int, int, bool, const double*, int, cudaStream_t);
SSTEP_EXTERN_BGRAM(1) SSTEP_EXTERN_BGRAM(2) SSTEP_EXTERN_BGRAM(3) SSTEP_EXTERN_BGRAM(4) SSTEP_EXTERN_BGRAM(5)
SSTEP_EXTERN_BGRAM(6) SSTEP_EXTERN_BGRAM(7) SSTEP_EXTERN_BGRAM(8) SSTEP_EXTERN_BGRAM(9) SSTEP_EXTERN_BGRAM(10)
SSTEP_EXTERN_BGRAM(11) SSTEP_EXTERN_BGRAM(12) SSTEP_EXTERN_BGRAM(13) SSTEP_EXTERN_BGRAM(14) SSTEP_EXTERN_BGRAM(15)
SSTEP_EXTERN_BGRAM(16)
#undef SSTEP_EXTERN_BGRAM

int batch_gram_m(int s) { return s * (s + 1) / 2 + 2 * s; }

cudaError_t launch_batch_gram(const BatchDev& B, int s, int nu, int solver, bool moments, const double* P,
                              cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    switch (s) {
#define SSTEP_CASE(S) case S: return launch_batch_gram_s<S>(B, nu, solver, moments, P, sms, st);
        SSTEP_CASE(1) SSTEP_CASE(2) SSTEP_CASE(3) SSTEP_CASE(4) SSTEP_CASE(5) SSTEP_CASE(6) SSTEP_CASE(7)
        SSTEP_CASE(8) SSTEP_CASE(9) SSTEP_CASE(10) SSTEP_CASE(11) SSTEP_CASE(12) SSTEP_CASE(13) SSTEP_CASE(14)
        SSTEP_CASE(15) SSTEP_CASE(16)
#undef SSTEP_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sstep
