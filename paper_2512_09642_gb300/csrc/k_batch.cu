// Batched kernels except the Gram (batch_impl.cuh): Chebyshev step, residual with per-system
// norms, update, control-block initialisation and the graph loop condition.
#include "batch.h"

namespace sstep {
namespace {

constexpr int BU = 256;

// Per-system residual epilogue (modes as in k_operator.cu: 0 initial, 1 true residual).
__device__ void batch_residual_epilogue(Ctl* ctl, int mode, double tot) {
    if (mode == 0) ctl->r0_sq = tot;
    else ctl->true_sq = tot;
}

// Off-diagonal part of (A p)_e for one system: Poisson sum of the in-grid neighbours, or the
// diffusion sum of face weight x neighbour (pdn / pup: the z-neighbours, 0 in 2D).
__device__ __forceinline__ double batch_offdiag(const BSys& sy, const double* __restrict__ ps,
                                                const double* __restrict__ wx, const double* __restrict__ wy,
                                                const double* __restrict__ wz, int64_t e, int i, int j, int k,
                                                int64_t sxy, double pdn, double pup) {
    const int nx = sy.nx, ny = sy.ny, nz = sy.nz;
    if (sy.poisson) {
        double s = (i > 0) ? __ldg(ps + e - 1) : 0.0;
        if (i < nx - 1) s += __ldg(ps + e + 1);
        if (j > 0) s += __ldg(ps + e - nx);
        if (j < ny - 1) s += __ldg(ps + e + nx);
        if (sy.dim == 3) {
            if (k > 0) s += pdn;
            if (k < nz - 1) s += pup;
        }
        return s;
    }
    double s = (i > 0) ? __ldg(wx + e - 1) * __ldg(ps + e - 1) : 0.0;
    if (i < nx - 1) s = fma(__ldg(wx + e), __ldg(ps + e + 1), s);
    if (j > 0) s = fma(__ldg(wy + e - nx), __ldg(ps + e - nx), s);
    if (j < ny - 1) s = fma(__ldg(wy + e), __ldg(ps + e + nx), s);
    if (sy.dim == 3) {
        if (k > 0) s = fma(__ldg(wz + e - sxy), pdn, s);
        if (k < nz - 1) s = fma(__ldg(wz + e), pup, s);
    }
    return s;
}

// Visits the points of one tile: 3D tiles march over BT_Z planes with the z-neighbours in
// registers; 2D tiles cover BT_Z groups of BT_Y rows, independent of each other (so their
// loads overlap). f(e, i, j, k, pc, pdn, pup).
template <typename F>
__device__ __forceinline__ void batch_tile_points(const BSys& sy, const BTile& tl, const double* __restrict__ ps, F f) {
    const int nx = sy.nx, ny = sy.ny, nz = sy.nz;
    const int i = tl.i0 + threadIdx.x;
    if (i >= nx) return;
    if (sy.dim == 2) {
#pragma unroll 4
        for (int m = 0; m < BT_Z; ++m) {
            const int j = tl.j0 + threadIdx.y + BT_Y * m;
            if (j >= ny) break;
            const int64_t e = i + (int64_t)nx * j;
            f(e, i, j, 0, __ldg(ps + e), 0.0, 0.0);
        }
        return;
    }
    const int j = tl.j0 + threadIdx.y;
    if (j >= ny) return;
    const int64_t sxy = (int64_t)nx * ny;
    const int k0 = tl.k0, k1 = min(nz, tl.k0 + BT_Z);
    int64_t e = i + (int64_t)nx * j + sxy * k0;
    double pdn = (k0 > 0) ? __ldg(ps + e - sxy) : 0.0;
    double pc = __ldg(ps + e);
    for (int k = k0; k < k1; ++k, e += sxy) {
        const double pup = (k < nz - 1) ? __ldg(ps + e + sxy) : 0.0;
        f(e, i, j, k, pc, pdn, pup);
        pdn = pc;
        pc = pup;
    }
}

__global__ void __launch_bounds__(BT_X* BT_Y) k_batch_cheb(BatchDev B, const double* __restrict__ p,
                                                           const double* __restrict__ q, double* __restrict__ out,
                                                           int first) {
    const int nact = B.act_n[0], ntiles = B.act_n[1];
    int idx = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        idx = batch_find(B.act_tile_prefix, nact, t, idx);
        const BSys sy = B.sys[B.act_sys[idx]];
        const BTile tl = B.tiles[sy.tile0 + (t - B.act_tile_prefix[idx])];
        const double c = first ? sy.theta : 2.0 * sy.theta;
        const double c1 = c * (1.0 - sy.sigma);
        const double c2 = -c / (2.0 * sy.dim);
        const double cs = first ? 0.5 : 1.0;
        const double* ps = p + sy.off;
        const double* qs = q + sy.off;
        double* os = out + sy.off;
        const double* wx = B.wx + sy.off;
        const double* wy = B.wy + sy.off;
        const double* wz = B.wz + sy.off;
        const double* cd = B.cdinv + sy.off;
        const int64_t sxy = (int64_t)sy.nx * sy.ny;
        batch_tile_points(sy, tl, ps, [&](int64_t e, int i, int j, int k, double pc, double pdn, double pup) {
            const double qv = first ? 0.0 : __ldg(qs + e);
            const double s = batch_offdiag(sy, ps, wx, wy, wz, e, i, j, k, sxy, pdn, pup);
            const double o = sy.poisson ? fma(c2, s, fma(c1, pc, -qv)) : fma(-(__ldg(cd + e) * cs), s, fma(c1, pc, -qv));
            os[e] = o;
        });
    }
}

__global__ void __launch_bounds__(BT_X* BT_Y) k_batch_residual(BatchDev B, const double* __restrict__ b,
                                                               const double* __restrict__ x, double* __restrict__ r,
                                                               int mode) {
    __shared__ double sh[BT_X * BT_Y / 32];
    __shared__ int is_last;
    const int tid = threadIdx.x + BT_X * threadIdx.y;
    for (int t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
        const BTile tl = B.tiles[t];
        const BSys sy = B.sys[tl.sys];
        Ctl* ctl = B.ctl + tl.sys;
        const double* xs = x + sy.off;
        const double* bs = b + sy.off;
        double* rs = r + sy.off;
        const double* wx = B.wx + sy.off;
        const double* wy = B.wy + sy.off;
        const double* wz = B.wz + sy.off;
        const double* dg = B.diag + sy.off;
        const double d2 = 2.0 * sy.dim;
        const int64_t sxy = (int64_t)sy.nx * sy.ny;
        double ss = 0.0;
        batch_tile_points(sy, tl, xs, [&](int64_t e, int i, int j, int k, double pc, double pdn, double pup) {
            const double s = batch_offdiag(sy, xs, wx, wy, wz, e, i, j, k, sxy, pdn, pup);
            const double ax = sy.poisson ? fma(d2, pc, -s) : fma(__ldg(dg + e), pc, -s);
            const double rv = __ldg(bs + e) - ax;
            rs[e] = rv;
            ss = fma(rv, rv, ss);
        });
        const double v = warp_sum(ss);
        if ((tid & 31) == 0) sh[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int k = 0; k < BT_X * BT_Y / 32; ++k) tot += sh[k];
            B.tile_partials[t] = tot;
            __threadfence();
            is_last = (atomicAdd(&ctl->counter2, 1u) == (unsigned)(sy.tile1 - sy.tile0 - 1));
        }
        __syncthreads();
        if (is_last) {
            __threadfence();
            double acc = 0.0;
            for (int tt = sy.tile0 + tid; tt < sy.tile1; tt += BT_X * BT_Y)
                acc += ((volatile double*)B.tile_partials)[tt];
            acc = warp_sum(acc);
            __syncthreads();
            if ((tid & 31) == 0) sh[tid >> 5] = acc;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int k = 0; k < BT_X * BT_Y / 32; ++k) tot += sh[k];
                batch_residual_epilogue(ctl, mode, tot);
                ctl->counter2 = 0u;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(BU) k_batch_update(BatchDev B, int s, const double* __restrict__ P,
                                                     double* __restrict__ x) {
    __shared__ double al[MAXS], be[MAXC];
    const int nact = B.act_n[0], nch = B.act_n[2];
    int idx = -1;
    for (int ca = blockIdx.x; ca < nch; ca += gridDim.x) {
        idx = batch_find(B.act_chunk_prefix, nact, ca, idx);
        const int sysi = B.act_sys[idx];
        const BSys sy = B.sys[sysi];
        const BChunk ch = B.chunks[sy.chunk0 + (ca - B.act_chunk_prefix[idx])];
        const Ctl* ctl = B.ctl + ch.sys;
        if (ctl->done) continue;   // finished in this outer iteration's Gram
        __syncthreads();
        if (threadIdx.x < s) al[threadIdx.x] = ctl->alpha[threadIdx.x];
        if (threadIdx.x <= s) be[threadIdx.x] = ctl->beta[threadIdx.x];
        __syncthreads();
        const double* Ps = P + sy.off;
        double* xs = x + sy.off;
        double* rs = (double*)P + sy.off;   // column 0: the residual, updated in place
        const double* dg = B.diag + sy.off;
        for (int64_t e = ch.e0 + threadIdx.x; e < ch.e1; e += BU) {
            const double p0 = __ldg(Ps + e);
            double xv = fma(al[0], p0, xs[e]);
            double rv = be[0] * p0;
            for (int jj = 1; jj < s; ++jj) {
                const double pv = __ldg(Ps + jj * B.ld + e);
                xv = fma(al[jj], pv, xv);
                rv = fma(be[jj], pv, rv);
            }
            rv = fma(be[s], __ldg(Ps + s * B.ld + e), rv);
            xs[e] = xv;
            rs[e] = sy.poisson ? rv : fma(-__ldg(dg + e), rv, p0);
        }
    }
}

__global__ void k_batch_init(BatchDev B, double tol_sq, int max_outer) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B.count; i += gridDim.x * blockDim.x) {
        Ctl* c = B.ctl + i;
        c->done = RUNNING;
        c->outer = 0;
        c->max_outer = max_outer;
        c->tol_sq = tol_sq;
        c->min_gii = INFINITY;
        c->counter = 0u;
        c->counter2 = 0u;
        c->delta = 0.0;
        c->rk_sq = 0.0;
        c->scale = 1.0;
        c->scale_next = 1.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *B.running = B.count;
}

// One warp: lists the running systems and the prefix sums of their tile and chunk counts.
__global__ void k_batch_compact(BatchDev B) {
    const int lane = threadIdx.x;
    int nact = 0, ntiles = 0, nchunks = 0;
    for (int base = 0; base < B.count; base += 32) {
        const int i = base + lane;
        const bool a = i < B.count && B.ctl[i].done == RUNNING;
        int nt = 0, nc = 0;
        if (a) {
            const BSys& sy = B.sys[i];
            nt = sy.tile1 - sy.tile0;
            nc = sy.chunk1 - sy.chunk0;
        }
        int ia = a ? 1 : 0, it = nt, ic = nc;   // inclusive warp scans
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(0xffffffffu, ia, o);
            const int yt = __shfl_up_sync(0xffffffffu, it, o);
            const int yc = __shfl_up_sync(0xffffffffu, ic, o);
            if (lane >= o) { ia += ya; it += yt; ic += yc; }
        }
        if (a) {
            const int pos = nact + ia - 1;
            B.act_sys[pos] = i;
            B.act_tile_prefix[pos] = ntiles + it - nt;
            B.act_chunk_prefix[pos] = nchunks + ic - nc;
        }
        nact += __shfl_sync(0xffffffffu, ia, 31);
        ntiles += __shfl_sync(0xffffffffu, it, 31);
        nchunks += __shfl_sync(0xffffffffu, ic, 31);
    }
    if (lane == 0) {
        B.act_tile_prefix[nact] = ntiles;
        B.act_chunk_prefix[nact] = nchunks;
        B.act_n[0] = nact;
        B.act_n[1] = ntiles;
        B.act_n[2] = nchunks;
    }
}

__global__ void k_batch_cond(cudaGraphConditionalHandle h, const int* running) {
    cudaGraphSetConditional(h, *running > 0 ? 1u : 0u);
}

int cap(int64_t items, int per_sm) {
    const int64_t c = (int64_t)per_sm * device_sm_count();
    return (int)(items < 1 ? 1 : (items < c ? items : c));
}

// Blocks per SM for a grid-stride kernel: the requested count, but no more than fit at once
// (a block that cannot be resident would start its share of the items only at the end).
template <typename K>
int resident(K kernel, int threads, int want) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess || occ < 1) return want;
    return want < occ ? want : occ;
}

}  // namespace

cudaError_t launch_batch_cheb(const BatchDev& B, const double* p, const double* q, double* out, bool first,
                              cudaStream_t st) {
    const int per_sm = resident(k_batch_cheb, BT_X * BT_Y, B.ctas_per_sm);
    k_batch_cheb<<<cap(B.ntiles, per_sm), dim3(BT_X, BT_Y), 0, st>>>(B, p, q, out, first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_batch_residual(const BatchDev& B, const double* b, const double* x, double* r, int mode,
                                  cudaStream_t st) {
    const int per_sm = resident(k_batch_residual, BT_X * BT_Y, B.ctas_per_sm);
    k_batch_residual<<<cap(B.ntiles, per_sm), dim3(BT_X, BT_Y), 0, st>>>(B, b, x, r, mode);
    return cudaGetLastError();
}

cudaError_t launch_batch_update(const BatchDev& B, int s, const double* P, double* x, cudaStream_t st) {
    k_batch_update<<<cap(B.nchunks, 4), BU, 0, st>>>(B, s, P, x);
    return cudaGetLastError();
}

cudaError_t launch_batch_init(const BatchDev& B, double tol_sq, int max_outer, cudaStream_t st) {
    k_batch_init<<<(B.count + 255) / 256, 256, 0, st>>>(B, tol_sq, max_outer);
    return cudaGetLastError();
}

cudaError_t launch_batch_compact(const BatchDev& B, cudaStream_t st) {
    k_batch_compact<<<1, 32, 0, st>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_batch_cond(cudaGraphConditionalHandle h, const int* running, cudaStream_t st) {
    k_batch_cond<<<1, 1, 0, st>>>(h, running);
    return cudaGetLastError();
}

}  // namespace sstep
