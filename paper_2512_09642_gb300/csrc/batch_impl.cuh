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

template <int S, bool DV, bool MOM>
constexpr int bgram_slab_size() { return GramShape<S, DV, MOM>::NSLAB * GramShape<S, DV, MOM>::M; }

template <int S, bool MOM>
__global__ void __launch_bounds__(BGRAM_THREADS, 1) k_batch_gram(BatchDev B, const double* __restrict__ P,
                                                                GramParams gp0) {
    constexpr int MV = GramShape<S, true, false>::M;   // partial stride: the largest entry set
    constexpr int A1 = bgram_slab_size<S, true, MOM>();
    constexpr int A2 = bgram_slab_size<S, false, MOM>();
    constexpr int A3 = 2 * S * S + 4 * S;
    constexpr int NSM = A1 > A2 ? (A1 > A3 ? A1 : A3) : (A2 > A3 ? A2 : A3);
    __shared__ double smem[NSM];
    __shared__ double tot[MV];
    __shared__ int is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nact = B.act_n[0], nch = B.act_n[2];
    int idx = -1;
    for (int ca = blockIdx.x; ca < nch; ca += gridDim.x) {
        idx = batch_find(B.act_chunk_prefix, nact, ca, idx);
        const BSys sy = B.sys[B.act_sys[idx]];
        const int c = sy.chunk0 + (ca - B.act_chunk_prefix[idx]);   // global chunk index
        const BChunk ch = B.chunks[c];
        Ctl* ctl = B.ctl + ch.sys;
        if (ctl->done) continue;   // same value for the whole block: the system's finish
                                   // happens after all of its chunks have arrived
        const bool dv = !sy.poisson;
        const double* Ps = P + sy.off;
        int M;
        if (dv) {
            using GS = GramShape<S, true, MOM>;
            M = GS::M;
            gram_role_dispatch<S, true, 0, MOM>(warp % GS::G, Ps, B.ld, B.diag + sy.off, ch.e1,
                                                ch.e0 + (warp / GS::G) * 32 + lane, (int64_t)GS::NSLAB * 32, smem,
                                                warp / GS::G);
            __syncthreads();
            for (int k = threadIdx.x; k < M; k += BGRAM_THREADS) {
                double v = 0.0;
                for (int sl = 0; sl < GS::NSLAB; ++sl) v += smem[sl * M + k];
                B.gram_partials[(size_t)c * MV + k] = v;
            }
        } else {
            using GS = GramShape<S, false, MOM>;
            M = GS::M;
            gram_role_dispatch<S, false, 0, MOM>(warp % GS::G, Ps, B.ld, nullptr, ch.e1,
                                                 ch.e0 + (warp / GS::G) * 32 + lane, (int64_t)GS::NSLAB * 32, smem,
                                                 warp / GS::G);
            __syncthreads();
            for (int k = threadIdx.x; k < M; k += BGRAM_THREADS) {
                double v = 0.0;
                for (int sl = 0; sl < GS::NSLAB; ++sl) v += smem[sl * M + k];
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
                if (dv) gram_finish<S, true, MOM>(tot, gp, ctl, smem);
                else gram_finish<S, false, MOM>(tot, gp, ctl, smem);
                __syncwarp();
                if (lane == 0 && ctl->done != RUNNING) atomicSub(B.running, 1);
            }
        }
        __syncthreads();
    }
}

// Grid: as many blocks as are resident at once (the variant's register use decides), at most
// one per chunk.
template <int S>
cudaError_t launch_batch_gram_s(const BatchDev& B, int nu, int solver, bool moments, const double* P, int sm_count,
                                cudaStream_t st) {
    GramParams gp{};
    gp.nu = nu;
    gp.solver = solver;
    gp.check = 1;
    int occ = 1;
    cudaError_t e = moments ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_gram<S, true>, BGRAM_THREADS, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_gram<S, false>, BGRAM_THREADS, 0);
    if (e != cudaSuccess) return e;
    const int64_t cap = (int64_t)sm_count * (occ < 1 ? 1 : occ);
    const int nblocks = (int)(B.nchunks < cap ? B.nchunks : cap);
    if (moments) k_batch_gram<S, true><<<nblocks, BGRAM_THREADS, 0, st>>>(B, P, gp);
    else k_batch_gram<S, false><<<nblocks, BGRAM_THREADS, 0, st>>>(B, P, gp);
    return cudaGetLastError();
}

}  // namespace sstep
