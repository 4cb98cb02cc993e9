// Batched kernels: one launch per phase covers every still-running system of the batch.
//
// Work items are stencil tiles (Chebyshev step, residual) and element chunks (Gram, update);
// both lists are sorted by system, so a system's items are a contiguous range. A system whose
// control block says done is skipped by every item. Reductions are per system: each item
// writes its partial sums, and the item that arrives last for its system (a per-system
// counter) sums that system's partials in item order and finishes the system's Gram solve
// (column scaling + FGS, the same code as the single-system kernel) in warp 0 of its block.
// No block waits for another; nothing spins.
#pragma once

#include "batch.h"
#include "gram_impl.cuh"

namespace sstep {

constexpr int BGRAM_THREADS = GRAM_THREADS;

template <int S>
__global__ void __launch_bounds__(BGRAM_THREADS, 1) k_batch_gram(BatchDev B, const double* __restrict__ P,
                                                                GramParams gp0) {
    constexpr int MV = GramShape<S, true>::M;    // partial stride: the larger entry set
    constexpr int A1 = GramShape<S, true>::NSLAB * GramShape<S, true>::M;
    constexpr int A2 = GramShape<S, false>::NSLAB * GramShape<S, false>::M;
    constexpr int A3 = 2 * S * S + 4 * S;
    constexpr int NSM = A1 > A2 ? (A1 > A3 ? A1 : A3) : (A2 > A3 ? A2 : A3);
    __shared__ double smem[NSM];
    __shared__ double tot[MV];
    __shared__ int is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = blockIdx.x; c < B.nchunks; c += gridDim.x) {
        const BChunk ch = B.chunks[c];
        const BSys sy = B.sys[ch.sys];
        Ctl* ctl = B.ctl + ch.sys;
        if (ctl->done) continue;   // same value for the whole block: the system's finish
                                   // happens after all of its chunks have arrived
        const bool dv = !sy.poisson;
        const double* Ps = P + sy.off;
        int M;
        if (dv) {
            constexpr int G = GramShape<S, true>::G, NSL = GramShape<S, true>::NSLAB;
            M = GramShape<S, true>::M;
            gram_role_dispatch<S, true>(warp % G, Ps, B.ld, B.diag + sy.off, ch.e1, ch.e0 + (warp / G) * 32 + lane,
                                        (int64_t)NSL * 32, smem, warp / G);
            __syncthreads();
            for (int k = threadIdx.x; k < M; k += BGRAM_THREADS) {
                double v = 0.0;
                for (int sl = 0; sl < NSL; ++sl) v += smem[sl * M + k];
                B.gram_partials[(size_t)c * MV + k] = v;
            }
        } else {
            constexpr int G = GramShape<S, false>::G, NSL = GramShape<S, false>::NSLAB;
            M = GramShape<S, false>::M;
            gram_role_dispatch<S, false>(warp % G, Ps, B.ld, nullptr, ch.e1, ch.e0 + (warp / G) * 32 + lane,
                                         (int64_t)NSL * 32, smem, warp / G);
            __syncthreads();
            for (int k = threadIdx.x; k < M; k += BGRAM_THREADS) {
                double v = 0.0;
                for (int sl = 0; sl < NSL; ++sl) v += smem[sl * M + k];
                B.gram_partials[(size_t)c * MV + k] = v;
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) is_last = (atomicAdd(&ctl->counter, 1u) == (unsigned)(sy.chunk1 - sy.chunk0 - 1));
        __syncthreads();
        if (is_last) {
            __threadfence();
            for (int k = warp; k < M; k += BGRAM_THREADS / 32) {
                double v = 0.0;
                for (int cc = sy.chunk0 + lane; cc < sy.chunk1; cc += 32)
                    v += ((volatile double*)B.gram_partials)[(size_t)cc * MV + k];
                v = warp_sum(v);
                if (lane == 0) tot[k] = v;
            }
            __syncthreads();
            if (warp == 0) {
                if (lane == 0) ctl->counter = 0u;
                GramParams gp = gp0;
                gp.theta = sy.theta;
                gp.sigma = sy.sigma;
                gp.dfac = sy.poisson ? 2.0 * sy.dim : 1.0;
                if (dv) gram_finish<S, true>(tot, gp, ctl, smem);
                else gram_finish<S, false>(tot, gp, ctl, smem);
                __syncwarp();
                if (lane == 0 && ctl->done != RUNNING) atomicSub(B.running, 1);
            }
        }
        __syncthreads();
    }
}

template <int S>
cudaError_t launch_batch_gram_s(const BatchDev& B, int nu, int solver, const double* P, int nblocks,
                                cudaStream_t st) {
    GramParams gp{};
    gp.nu = nu;
    gp.solver = solver;
    gp.check = 1;
    k_batch_gram<S><<<nblocks, BGRAM_THREADS, 0, st>>>(B, P, gp);
    return cudaGetLastError();
}

}  // namespace sstep
