// Batched form: many independent stencil systems solved together (internal definitions).
#pragma once

#include "kernels.h"

namespace sstep {

constexpr int BT_X = 32, BT_Y = 8, BT_Z = 8;   // stencil tile (x, y threads; z planes per thread)

// One system of the batch (device copy). Its vectors occupy elements [off, off + n) of every
// concatenated vector; the basis column j of all systems is one vector at j * ld_total.
struct BSys {
    int dim, nx, ny, nz;
    int64_t off, n;
    int tile0, tile1;      // its stencil tiles in the tile list
    int chunk0, chunk1;    // its element chunks in the chunk list
    double theta, sigma;
    int poisson;           // 1: constant-coefficient Poisson (no face arrays)
    int pad;
};

struct BTile { int sys, i0, j0, k0; };
struct BChunk { int sys; int pad; int64_t e0, e1; };   // local element range of the system

struct BatchDev {
    const BSys* sys;
    const BTile* tiles;
    const BChunk* chunks;
    int ntiles, nchunks, count;
    int64_t ld;            // length of one concatenated vector (padded)
    const double* wx;      // concatenated face weights / diagonal / 2 theta_i / diag
    const double* wy;
    const double* wz;
    const double* diag;
    const double* cdinv;
    Ctl* ctl;              // one control block per system
    int* running;          // systems still iterating
    double* gram_partials; // [nchunks][M]
    double* tile_partials; // [ntiles]
    int ctas_per_sm;       // grid of the stencil kernels: ctas_per_sm x SMs (capped by the tiles)
    // active work of the current outer iteration (k_batch_compact): running systems and the
    // prefix sums of their tile and chunk counts; act_n = {systems, tiles, chunks}
    int* act_sys;
    int* act_tile_prefix;
    int* act_chunk_prefix;
    int* act_n;
};

// Locates active work item t: returns the index into act_sys whose prefix range holds t,
// starting the forward scan at `hint` (items are visited in increasing order by a block).
__device__ __forceinline__ int batch_find(const int* prefix, int nact, int t, int hint) {
    int lo = hint;
    if (lo < 0 || lo >= nact || prefix[lo] > t) {
        lo = 0;
        int hi = nact;   // binary search: prefix[lo] <= t < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= t) lo = mid; else hi = mid;
        }
        return lo;
    }
    while (lo + 1 < nact && prefix[lo + 1] <= t) ++lo;
    return lo;
}

cudaError_t launch_batch_cheb(const BatchDev& B, const double* p, const double* q, double* out, bool first,
                              cudaStream_t st);
cudaError_t launch_batch_gram(const BatchDev& B, int s, int nu, int solver, bool moments, const double* P,
                              cudaStream_t st);
cudaError_t launch_batch_update(const BatchDev& B, int s, const double* P, double* x, cudaStream_t st);
cudaError_t launch_batch_residual(const BatchDev& B, const double* b, const double* x, double* r, int mode,
                                  cudaStream_t st);
cudaError_t launch_batch_init(const BatchDev& B, double tol_sq, int max_outer, cudaStream_t st);
cudaError_t launch_batch_cond(cudaGraphConditionalHandle h, const int* running, cudaStream_t st);
cudaError_t launch_batch_compact(const BatchDev& B, cudaStream_t st);
int batch_gram_m(int s);

}  // namespace sstep
