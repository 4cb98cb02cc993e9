// Dispatch of the fused Gram + FGS kernel over the basis size s (instantiated by
// k_gram_inst.cu, compiled once per s so the instantiations build in parallel).
#include "gram_impl.cuh"

namespace sstep {

#define SSTEP_EXTERN_GRAM(S) extern template cudaError_t launch_gram_s<S>(const GramArgs&, double*, Ctl*, int, cudaStream_t);
SSTEP_EXTERN_GRAM(1) SSTEP_EXTERN_GRAM(2) SSTEP_EXTERN_GRAM(3) SSTEP_EXTERN_GRAM(4) SSTEP_EXTERN_GRAM(5)
SSTEP_EXTERN_GRAM(6) SSTEP_EXTERN_GRAM(7) SSTEP_EXTERN_GRAM(8) SSTEP_EXTERN_GRAM(9) SSTEP_EXTERN_GRAM(10)
SSTEP_EXTERN_GRAM(11) SSTEP_EXTERN_GRAM(12) SSTEP_EXTERN_GRAM(13) SSTEP_EXTERN_GRAM(14) SSTEP_EXTERN_GRAM(15)
SSTEP_EXTERN_GRAM(16) SSTEP_EXTERN_GRAM(17) SSTEP_EXTERN_GRAM(18) SSTEP_EXTERN_GRAM(19) SSTEP_EXTERN_GRAM(20)
SSTEP_EXTERN_GRAM(21) SSTEP_EXTERN_GRAM(22) SSTEP_EXTERN_GRAM(23) SSTEP_EXTERN_GRAM(24) SSTEP_EXTERN_GRAM(25)
SSTEP_EXTERN_GRAM(26) SSTEP_EXTERN_GRAM(27) SSTEP_EXTERN_GRAM(28) SSTEP_EXTERN_GRAM(29) SSTEP_EXTERN_GRAM(30)
SSTEP_EXTERN_GRAM(31) SSTEP_EXTERN_GRAM(32)
#undef SSTEP_EXTERN_GRAM
#define SSTEP_EXTERN_FIN(S) \
    extern template cudaError_t launch_moments_finish_s<S>(const GramArgs&, const void*, int, double*, int, Ctl*, cudaStream_t);
SSTEP_EXTERN_FIN(1) SSTEP_EXTERN_FIN(2) SSTEP_EXTERN_FIN(3) SSTEP_EXTERN_FIN(4) SSTEP_EXTERN_FIN(5)
SSTEP_EXTERN_FIN(6) SSTEP_EXTERN_FIN(7) SSTEP_EXTERN_FIN(8) SSTEP_EXTERN_FIN(9) SSTEP_EXTERN_FIN(10)
SSTEP_EXTERN_FIN(11) SSTEP_EXTERN_FIN(12) SSTEP_EXTERN_FIN(13) SSTEP_EXTERN_FIN(14) SSTEP_EXTERN_FIN(15)
SSTEP_EXTERN_FIN(16) SSTEP_EXTERN_FIN(17) SSTEP_EXTERN_FIN(18) SSTEP_EXTERN_FIN(19) SSTEP_EXTERN_FIN(20)
SSTEP_EXTERN_FIN(21) SSTEP_EXTERN_FIN(22) SSTEP_EXTERN_FIN(23) SSTEP_EXTERN_FIN(24) SSTEP_EXTERN_FIN(25)
SSTEP_EXTERN_FIN(26) SSTEP_EXTERN_FIN(27) SSTEP_EXTERN_FIN(28) SSTEP_EXTERN_FIN(29) SSTEP_EXTERN_FIN(30)
SSTEP_EXTERN_FIN(31) SSTEP_EXTERN_FIN(32)
#undef SSTEP_EXTERN_FIN
#define SSTEP_EXTERN_OCC(S) extern template int gram_occupancy_s<S>(const GramArgs&);
SSTEP_EXTERN_OCC(1) SSTEP_EXTERN_OCC(2) SSTEP_EXTERN_OCC(3) SSTEP_EXTERN_OCC(4) SSTEP_EXTERN_OCC(5)
SSTEP_EXTERN_OCC(6) SSTEP_EXTERN_OCC(7) SSTEP_EXTERN_OCC(8) SSTEP_EXTERN_OCC(9) SSTEP_EXTERN_OCC(10)
SSTEP_EXTERN_OCC(11) SSTEP_EXTERN_OCC(12) SSTEP_EXTERN_OCC(13) SSTEP_EXTERN_OCC(14) SSTEP_EXTERN_OCC(15)
SSTEP_EXTERN_OCC(16) SSTEP_EXTERN_OCC(17) SSTEP_EXTERN_OCC(18) SSTEP_EXTERN_OCC(19) SSTEP_EXTERN_OCC(20)
SSTEP_EXTERN_OCC(21) SSTEP_EXTERN_OCC(22) SSTEP_EXTERN_OCC(23) SSTEP_EXTERN_OCC(24) SSTEP_EXTERN_OCC(25)
SSTEP_EXTERN_OCC(26) SSTEP_EXTERN_OCC(27) SSTEP_EXTERN_OCC(28) SSTEP_EXTERN_OCC(29) SSTEP_EXTERN_OCC(30)
SSTEP_EXTERN_OCC(31) SSTEP_EXTERN_OCC(32)
#undef SSTEP_EXTERN_OCC

static int gram_m(int s, bool dvec) { return s * (s + 1) / 2 + s + (dvec ? s : 0); }   // >= the moments form's 2s (+ s)

static int gram_occupancy(const GramArgs& g) {
    switch (g.s) {
#define SSTEP_CASE(S) case S: return gram_occupancy_s<S>(g);
        SSTEP_CASE(1) SSTEP_CASE(2) SSTEP_CASE(3) SSTEP_CASE(4) SSTEP_CASE(5) SSTEP_CASE(6) SSTEP_CASE(7)
        SSTEP_CASE(8) SSTEP_CASE(9) SSTEP_CASE(10) SSTEP_CASE(11) SSTEP_CASE(12) SSTEP_CASE(13) SSTEP_CASE(14)
        SSTEP_CASE(15) SSTEP_CASE(16) SSTEP_CASE(17) SSTEP_CASE(18) SSTEP_CASE(19) SSTEP_CASE(20) SSTEP_CASE(21)
        SSTEP_CASE(22) SSTEP_CASE(23) SSTEP_CASE(24) SSTEP_CASE(25) SSTEP_CASE(26) SSTEP_CASE(27) SSTEP_CASE(28)
        SSTEP_CASE(29) SSTEP_CASE(30) SSTEP_CASE(31) SSTEP_CASE(32)
#undef SSTEP_CASE
        default: return 1;
    }
}

int gram_blocks(const GramArgs& g, int sm_count) {
    // as many 512-thread blocks as fit on the SMs at once (the variant's register use decides:
    // the FP64 forms are FP64-pipe bound with one, the lighter variants need more memory
    // parallelism), fewer when the vector is short (one element per thread at most)
    const int64_t per_block = (int64_t)GRAM_WARPS * 32;
    int64_t want = (g.n + per_block - 1) / per_block;
    if (want < 1) want = 1;
    const int64_t cap = (int64_t)sm_count * gram_occupancy(g);
    return (int)(want < cap ? want : cap);
}

size_t gram_partials_needed(const GramArgs& g, int nblocks) { return (size_t)nblocks * gram_m(g.s, g.dvec); }

cudaError_t launch_gram(const GramArgs& g, double* partials, Ctl* ctl, int nblocks, cudaStream_t st) {
    switch (g.s) {
#define SSTEP_CASE(S) case S: return launch_gram_s<S>(g, partials, ctl, nblocks, st);
        SSTEP_CASE(1) SSTEP_CASE(2) SSTEP_CASE(3) SSTEP_CASE(4) SSTEP_CASE(5) SSTEP_CASE(6) SSTEP_CASE(7)
        SSTEP_CASE(8) SSTEP_CASE(9) SSTEP_CASE(10) SSTEP_CASE(11) SSTEP_CASE(12) SSTEP_CASE(13) SSTEP_CASE(14)
        SSTEP_CASE(15) SSTEP_CASE(16) SSTEP_CASE(17) SSTEP_CASE(18) SSTEP_CASE(19) SSTEP_CASE(20) SSTEP_CASE(21)
        SSTEP_CASE(22) SSTEP_CASE(23) SSTEP_CASE(24) SSTEP_CASE(25) SSTEP_CASE(26) SSTEP_CASE(27) SSTEP_CASE(28)
        SSTEP_CASE(29) SSTEP_CASE(30) SSTEP_CASE(31) SSTEP_CASE(32)
#undef SSTEP_CASE
        default: return cudaErrorInvalidValue;
    }
}

// one finish block per 128 step blocks: its warps' loads of the partials form short chains
// (measured with 1024 step blocks: 4 finish blocks 30.7 us, 8 blocks 28.7 us, 2 blocks 34.8 us)
int moments_finish_blocks(int nblk) {
    const int r = (nblk + 127) / 128;
    return r < 1 ? 1 : (r > MAX_FIN_BLOCKS ? MAX_FIN_BLOCKS : r);
}

cudaError_t launch_moments_finish(const GramArgs& g, const void* part, int nblk, double* part2, Ctl* ctl,
                                  cudaStream_t st) {
    const int nfin = moments_finish_blocks(nblk);
    switch (g.s) {
#define SSTEP_CASE(S) case S: return launch_moments_finish_s<S>(g, part, nblk, part2, nfin, ctl, st);
        SSTEP_CASE(1) SSTEP_CASE(2) SSTEP_CASE(3) SSTEP_CASE(4) SSTEP_CASE(5) SSTEP_CASE(6) SSTEP_CASE(7)
        SSTEP_CASE(8) SSTEP_CASE(9) SSTEP_CASE(10) SSTEP_CASE(11) SSTEP_CASE(12) SSTEP_CASE(13) SSTEP_CASE(14)
        SSTEP_CASE(15) SSTEP_CASE(16) SSTEP_CASE(17) SSTEP_CASE(18) SSTEP_CASE(19) SSTEP_CASE(20) SSTEP_CASE(21)
        SSTEP_CASE(22) SSTEP_CASE(23) SSTEP_CASE(24) SSTEP_CASE(25) SSTEP_CASE(26) SSTEP_CASE(27) SSTEP_CASE(28)
        SSTEP_CASE(29) SSTEP_CASE(30) SSTEP_CASE(31) SSTEP_CASE(32)
#undef SSTEP_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sstep
