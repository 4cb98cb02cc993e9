// Gradient of a loss L(x) through the solve x = A(kappa)^-1 b with respect to the per-cell
// coefficient kappa of the cell-centred diffusion stencil (the differentiable form of the
// solve; the paper has no adjoint). With A symmetric the adjoint system is A lambda = dL/dx,
// solved by the same s-step CG handle, and
//
//   dL/dkappa_c = -lambda^T (dA/dkappa_c) x
//               = - sum_{interior faces f = (c, o)} dw_f/dkappa_c (lambda_c - lambda_o)(x_c - x_o)
//                 - 2 nbf_c lambda_c x_c,
//
// where w_f = 2 kc ko / (kc + ko) (so dw_f/dkappa_c = 2 ko^2 / (kc + ko)^2) and nbf_c counts
// the boundary faces of cell c (each contributes 2 kappa_c e_c e_c^T to A).
#include "kernels.h"

namespace sstep {
namespace {

constexpr int AB = 256;

__device__ __forceinline__ double face_term(double kc, double ko, double lc, double lo, double xc, double xo) {
    const double s = kc + ko;
    return 2.0 * ko * ko / (s * s) * ((lc - lo) * (xc - xo));
}

__global__ void __launch_bounds__(AB) k_grad_kappa(int dim, int nx, int ny, int nz, const double* __restrict__ kappa,
                                                   const double* __restrict__ x, const double* __restrict__ lam,
                                                   double* __restrict__ g) {
    const int64_t n = (int64_t)nx * ny * nz, sxy = (int64_t)nx * ny;
    for (int64_t e = blockIdx.x * (int64_t)AB + threadIdx.x; e < n; e += (int64_t)gridDim.x * AB) {
        const int i = (int)(e % nx);
        const int j = (int)((e / nx) % ny);
        const int k = (int)(e / sxy);
        const double kc = kappa[e], xc = x[e], lc = lam[e];
        double acc = 0.0;
        int nbf = 0;
        if (i > 0) acc += face_term(kc, kappa[e - 1], lc, lam[e - 1], xc, x[e - 1]); else ++nbf;
        if (i < nx - 1) acc += face_term(kc, kappa[e + 1], lc, lam[e + 1], xc, x[e + 1]); else ++nbf;
        if (j > 0) acc += face_term(kc, kappa[e - nx], lc, lam[e - nx], xc, x[e - nx]); else ++nbf;
        if (j < ny - 1) acc += face_term(kc, kappa[e + nx], lc, lam[e + nx], xc, x[e + nx]); else ++nbf;
        if (dim == 3) {
            if (k > 0) acc += face_term(kc, kappa[e - sxy], lc, lam[e - sxy], xc, x[e - sxy]); else ++nbf;
            if (k < nz - 1) acc += face_term(kc, kappa[e + sxy], lc, lam[e + sxy], xc, x[e + sxy]); else ++nbf;
        }
        g[e] = -(acc + 2.0 * nbf * lc * xc);
    }
}

}  // namespace

cudaError_t launch_grad_kappa(int dim, int nx, int ny, int nz, const double* kappa, const double* x,
                              const double* lam, double* g, cudaStream_t st) {
    const int64_t n = (int64_t)nx * ny * nz;
    int64_t b = (n + AB - 1) / AB;
    if (b > 8 * (int64_t)device_sm_count()) b = 8 * (int64_t)device_sm_count();
    k_grad_kappa<<<(int)b, AB, 0, st>>>(dim, nx, ny, nz, kappa, x, lam, g);
    return cudaGetLastError();
}

}  // namespace sstep
