// FGS as the AMG coarse-grid solver (Section 6, "AMG Coarse-Grid Extension") on the handle's
// stencil operator A_f with an aggregation prolongation P: column i of P is the indicator of
// aggregate i, a bx x by x bz box of the grid (ids x fastest over the coarse grid). nu forward
// Gauss-Seidel sweeps on A_c y = g, A_c = P^T A_f P, rows in increasing order, D = diag(A_c):
//   formed     A_c is assembled (dense, one thread per coarse row, in a fixed order) and one
//              block sweeps its rows, y held in shared memory;
//   streaming  A_c is never formed: z = P y is kept on the fine grid, (A_c y)_i is the sum
//              of (A_f z) over aggregate i, and y_i += delta adds delta to z on the aggregate
//              (one block walks the aggregates in order).
// Gauss-Seidel is sequential over the coarse rows; the parallelism is within a row (the dense
// row's dot product, or the aggregate's points).
#include "kernels.h"

namespace sstep {
namespace {

struct Agg {
    int nx, ny, nz, bx, by, bz, cx, cy, cz;
    __device__ __forceinline__ int of(int i, int j, int k) const { return i / bx + cx * (j / by + cy * (k / bz)); }
};

// Calls f(column index, value) for every entry of row (i, j, k) of the stencil operator.
template <typename F>
__device__ __forceinline__ void stencil_row(const OpDesc& op, int i, int j, int k, F f) {
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t e = i + (int64_t)nx * j + sxy * k;
    if (op.box) {
        const int kd = op.dim == 3 ? 1 : 0;
        for (int dz = -kd; dz <= kd; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int ii = i + dx, jj = j + dy, kk = k + dz;
                    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
                    const bool c = dx == 0 && dy == 0 && dz == 0;
                    f(ii + (int64_t)nx * jj + sxy * kk, c ? op.dconst : -1.0);
                }
        return;
    }
    if (op.wx == nullptr) {   // Poisson
        f(e, op.dconst);
        if (i > 0) f(e - 1, -1.0);
        if (i < nx - 1) f(e + 1, -1.0);
        if (j > 0) f(e - nx, -1.0);
        if (j < ny - 1) f(e + nx, -1.0);
        if (op.dim == 3) {
            if (k > 0) f(e - sxy, -1.0);
            if (k < nz - 1) f(e + sxy, -1.0);
        }
        return;
    }
    f(e, op.diag[e]);   // diffusion: face weights to the + neighbour
    if (i > 0) f(e - 1, -op.wx[e - 1]);
    if (i < nx - 1) f(e + 1, -op.wx[e]);
    if (j > 0) f(e - nx, -op.wy[e - nx]);
    if (j < ny - 1) f(e + nx, -op.wy[e]);
    if (op.dim == 3) {
        if (k > 0) f(e - sxy, -op.wz[e - sxy]);
        if (k < nz - 1) f(e + sxy, -op.wz[e]);
    }
}

__device__ __forceinline__ void fine_coords(const OpDesc& op, int64_t e, int& i, int& j, int& k) {
    const int64_t sxy = (int64_t)op.nx * op.ny;
    k = (int)(e / sxy);
    const int64_t r = e - sxy * k;
    j = (int)(r / op.nx);
    i = (int)(r - (int64_t)op.nx * j);
}

// The p-th point (0 <= p < size) of aggregate a, as grid coordinates; false past its end.
__device__ __forceinline__ bool agg_point(const Agg& g, int a, int p, int& i, int& j, int& k) {
    const int ci = a % g.cx, cj = (a / g.cx) % g.cy, ck = a / (g.cx * g.cy);
    const int i0 = ci * g.bx, j0 = cj * g.by, k0 = ck * g.bz;
    const int dx = min(g.bx, g.nx - i0), dy = min(g.by, g.ny - j0), dz = min(g.bz, g.nz - k0);
    if (p >= dx * dy * dz) return false;
    i = i0 + p % dx;
    j = j0 + (p / dx) % dy;
    k = k0 + p / (dx * dy);
    return true;
}

__device__ __forceinline__ int agg_size(const Agg& g) { return g.bx * g.by * g.bz; }

// z = P y0 (one thread per fine point).
__global__ void k_coarse_prolong(OpDesc op, Agg g, const double* __restrict__ y, double* __restrict__ z) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < op.n; e += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        fine_coords(op, e, i, j, k);
        z[e] = y[g.of(i, j, k)];
    }
}

// diag(A_c)_a = sum of A_f over rows and columns of aggregate a (one thread per aggregate).
__global__ void k_coarse_diag(OpDesc op, Agg g, int nc, double* __restrict__ dc) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nc; a += gridDim.x * blockDim.x) {
        double s = 0.0;
        int i, j, k;
        for (int p = 0; agg_point(g, a, p, i, j, k); ++p)
            stencil_row(op, i, j, k, [&](int64_t col, double v) {
                int ii, jj, kk;
                fine_coords(op, col, ii, jj, kk);
                if (g.of(ii, jj, kk) == a) s += v;
            });
        dc[a] = s;
    }
}

constexpr int CS = 256;   // threads of the streaming block

// Streaming sweeps: one block walks the aggregates in increasing order; its threads share an
// aggregate's points. The block barrier after the z update orders it before the next row.
__global__ void __launch_bounds__(CS) k_coarse_stream(OpDesc op, Agg g, int nc, int nu, const double* __restrict__ gv,
                                                      const double* __restrict__ dc, double* __restrict__ y,
                                                      double* z) {
    __shared__ double red[CS / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int cap = agg_size(g);
    for (int sweep = 0; sweep < nu; ++sweep) {
        for (int a = 0; a < nc; ++a) {
            double s = 0.0;
            for (int p = t; p < cap; p += CS) {
                int i, j, k;
                if (!agg_point(g, a, p, i, j, k)) break;
                stencil_row(op, i, j, k, [&](int64_t col, double v) { s = fma(v, z[col], s); });
            }
            s = warp_sum(s);
            if (lane == 0) red[warp] = s;
            __syncthreads();
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < CS / 32; ++w) tot += red[w];
            const double d = dc[a];
            const double delta = d != 0.0 ? (gv[a] - tot) / d : 0.0;
            if (t == 0) y[a] += delta;
            for (int p = t; p < cap; p += CS) {
                int i, j, k;
                if (!agg_point(g, a, p, i, j, k)) break;
                z[i + (int64_t)op.nx * j + (int64_t)op.nx * op.ny * k] += delta;
            }
            __syncthreads();   // z updates (and the reads of red) complete before the next row
        }
    }
}

// Assembly of the dense A_c (zeroed by the caller): thread a accumulates row a in the order of
// its aggregate's points and their stencil entries (deterministic).
__global__ void k_coarse_form(OpDesc op, Agg g, int nc, double* __restrict__ Ac) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nc; a += gridDim.x * blockDim.x) {
        double* row = Ac + (size_t)a * nc;
        int i, j, k;
        for (int p = 0; agg_point(g, a, p, i, j, k); ++p)
            stencil_row(op, i, j, k, [&](int64_t col, double v) {
                int ii, jj, kk;
                fine_coords(op, col, ii, jj, kk);
                row[g.of(ii, jj, kk)] += v;
            });
    }
}

constexpr int CF = 1024;   // threads of the formed-sweep block

// Formed sweeps: one block, y in shared memory; row a's dot product over all threads.
// (Loading the next row into registers during the reduction measured slower: 0.37 -> 0.63 s
// for 20 sweeps at n_c = 4096.)
__global__ void __launch_bounds__(CF) k_coarse_fgs_formed(const double* __restrict__ Ac, int nc, int nu,
                                                          const double* __restrict__ gv, double* __restrict__ y) {
    extern __shared__ double ys[];
    __shared__ double red[CF / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int c = t; c < nc; c += CF) ys[c] = y[c];
    __syncthreads();
    for (int sweep = 0; sweep < nu; ++sweep) {
        for (int a = 0; a < nc; ++a) {
            const double* row = Ac + (size_t)a * nc;
            double s = 0.0;
            for (int c = t; c < nc; c += CF) s = fma(row[c], ys[c], s);
            s = warp_sum(s);
            if (lane == 0) red[warp] = s;
            __syncthreads();
            if (t == 0) {
                double tot = 0.0;
                for (int w = 0; w < CF / 32; ++w) tot += red[w];
                const double d = row[a];
                const double delta = d != 0.0 ? (gv[a] - tot) / d : 0.0;
                ys[a] += delta;
            }
            __syncthreads();
        }
    }
    for (int c = t; c < nc; c += CF) y[c] = ys[c];
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t c = 8 * (int64_t)device_sm_count();
    return (int)(b < 1 ? 1 : (b > c ? c : b));
}

}  // namespace

int coarse_formed_max_nc() { return 16384; }

cudaError_t launch_coarse_fgs(const OpDesc& op, int bx, int by, int bz, int nc, const double* g, double* y, int nu,
                              int streaming, double* z, double* dc, double* Ac, cudaStream_t st) {
    Agg a{};
    a.nx = op.nx;
    a.ny = op.ny;
    a.nz = op.nz;
    a.bx = bx;
    a.by = by;
    a.bz = bz;
    a.cx = (op.nx + bx - 1) / bx;
    a.cy = (op.ny + by - 1) / by;
    a.cz = (op.nz + bz - 1) / bz;
    if (streaming) {
        k_coarse_prolong<<<grid_for(op.n, 256), 256, 0, st>>>(op, a, y, z);
        k_coarse_diag<<<grid_for(nc, 128), 128, 0, st>>>(op, a, nc, dc);
        k_coarse_stream<<<1, CS, 0, st>>>(op, a, nc, nu, g, dc, y, z);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(Ac, 0, sizeof(double) * (size_t)nc * nc, st);
    if (e != cudaSuccess) return e;
    k_coarse_form<<<grid_for(nc, 128), 128, 0, st>>>(op, a, nc, Ac);
    const size_t smem = sizeof(double) * (size_t)nc;
    e = cudaFuncSetAttribute(k_coarse_fgs_formed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_coarse_fgs_formed<<<1, CF, smem, st>>>(Ac, nc, nu, g, y);
    return cudaGetLastError();
}

}  // namespace sstep
