// Set-up kernels run once per handle (not on the outer-iteration path): the diagonal of a
// CSR matrix, the face weights of the diffusion stencil, 2 theta / diag, FP32 copies, the
// Gershgorin row bound, and the vector pieces of the Lanczos spectral estimate (Section 8).
#include "kernels.h"

namespace sstep {

int device_sm_count() {
    constexpr int MAXDEV = 64;
    static int cache[MAXDEV] = {};   // a benign race: every writer stores the same value
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return 152;
    if (cache[dev] <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 152;
        cache[dev] = v;
    }
    return cache[dev];
}

namespace {

constexpr int TB = 256;

int nblocks(int64_t n) {
    const int64_t b = (n + TB - 1) / TB, cap = 8 * (int64_t)device_sm_count();
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

__global__ void k_csr_diag(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                           const double* __restrict__ vals, int64_t n, double* __restrict__ diag, int* bad) {
    for (int64_t r = blockIdx.x * (int64_t)TB + threadIdx.x; r < n; r += (int64_t)gridDim.x * TB) {
        double d = 0.0;
        bool found = false;
        for (int32_t t = rowptr[r]; t < rowptr[r + 1]; ++t)
            if (colind[t] == r) { d += vals[t]; found = true; }
        diag[r] = d;
        if (!found || !(d > 0.0) || !isfinite(d)) atomicExch(bad, 1);
    }
}

__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

__global__ void k_faces(int dim, int nx, int ny, int nz, const double* __restrict__ kappa, double* wx, double* wy,
                        double* wz, double* diag, int* bad) {
    const int64_t n = (int64_t)nx * ny * nz, sxy = (int64_t)nx * ny;
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB) {
        const int i = (int)(e % nx);
        const int j = (int)((e / nx) % ny);
        const int k = (int)(e / sxy);
        const double kc = kappa[e];
        if (!(kc > 0.0) || !isfinite(kc)) atomicExch(bad, 1);
        double d = 0.0;
        double w;
        w = i < nx - 1 ? harmonic(kc, kappa[e + 1]) : 0.0;
        wx[e] = w;
        d += i < nx - 1 ? w : 2.0 * kc;
        d += i > 0 ? harmonic(kappa[e - 1], kc) : 2.0 * kc;
        w = j < ny - 1 ? harmonic(kc, kappa[e + nx]) : 0.0;
        wy[e] = w;
        d += j < ny - 1 ? w : 2.0 * kc;
        d += j > 0 ? harmonic(kappa[e - nx], kc) : 2.0 * kc;
        if (dim == 3) {
            w = k < nz - 1 ? harmonic(kc, kappa[e + sxy]) : 0.0;
            wz[e] = w;
            d += k < nz - 1 ? w : 2.0 * kc;
            d += k > 0 ? harmonic(kappa[e - sxy], kc) : 2.0 * kc;
        }
        diag[e] = d;
    }
}

__global__ void k_div(const double* __restrict__ diag, double c, double* __restrict__ out, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB) out[e] = c / diag[e];
}

__global__ void k_rsqrt(const double* __restrict__ diag, double* __restrict__ out, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB) out[e] = 1.0 / sqrt(diag[e]);
}

__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB) out[e] = (float)in[e];
}

__global__ void k_copy(const double* __restrict__ in, double* __restrict__ out, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB) out[e] = in[e];
}

// per-block max over rows of sum_j |a_ij| / |a_ii| (Jacobi) - CSR
__global__ void k_gersh_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                            const double* __restrict__ vals, const double* __restrict__ diag, int64_t n,
                            double* blockmax) {
    __shared__ double sh[TB];
    double m = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)TB + threadIdx.x; r < n; r += (int64_t)gridDim.x * TB) {
        double s = 0.0;
        for (int32_t t = rowptr[r]; t < rowptr[r + 1]; ++t) s += fabs(vals[t]);
        m = fmax(m, diag ? s / fabs(diag[r]) : s);
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = TB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) blockmax[blockIdx.x] = sh[0];
}

// same for the diffusion stencil: row sum = diag + sum of interior face weights
__global__ void k_gersh_faces(int dim, int nx, int ny, int nz, const double* __restrict__ wx,
                              const double* __restrict__ wy, const double* __restrict__ wz,
                              const double* __restrict__ diag, bool jacobi, double* blockmax) {
    __shared__ double sh[TB];
    const int64_t n = (int64_t)nx * ny * nz, sxy = (int64_t)nx * ny;
    double m = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB) {
        const int i = (int)(e % nx);
        const int j = (int)((e / nx) % ny);
        const int k = (int)(e / sxy);
        double s = diag[e] + wx[e] + wy[e] + (i > 0 ? wx[e - 1] : 0.0) + (j > 0 ? wy[e - nx] : 0.0);
        if (dim == 3) s += wz[e] + (k > 0 ? wz[e - sxy] : 0.0);
        m = fmax(m, jacobi ? s / diag[e] : s);
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = TB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) blockmax[blockIdx.x] = sh[0];
}

// v_i = 2 u_i - 1, u_i = (splitmix64 draw i >> 11) * 2^-53, draw i = mix(seed + (i+1) * golden)
// (Steele, Lea, Flood 2014; Vigna's finaliser constants).
__global__ void k_splitmix(uint64_t seed, double* __restrict__ v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        v[i] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
    }
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* partials) {
    __shared__ double sh[TB / 32];
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB) s = fma(a[e], b[e], s);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < TB / 32; ++k) t += sh[k];
        partials[blockIdx.x] = t;
    }
}

__global__ void k_mul(const double* __restrict__ a, double ac, const double* __restrict__ b, double* __restrict__ out,
                      int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB)
        out[e] = (a ? a[e] : ac) * b[e];
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)TB + threadIdx.x; e < n; e += (int64_t)gridDim.x * TB) y[e] = a * x[e] + b * y[e];
}

}  // namespace

cudaError_t launch_csr_diag(const OpDesc& op, double* diag, int* bad, cudaStream_t st) {
    k_csr_diag<<<nblocks(op.n), TB, 0, st>>>(op.rowptr, op.colind, op.vals, op.n, diag, bad);
    return cudaGetLastError();
}
cudaError_t launch_stencil_faces(int dim, int nx, int ny, int nz, const double* kappa, double* wx, double* wy,
                                 double* wz, double* diag, int* bad, cudaStream_t st) {
    const int64_t n = (int64_t)nx * ny * nz;
    k_faces<<<nblocks(n), TB, 0, st>>>(dim, nx, ny, nz, kappa, wx, wy, wz, diag, bad);
    return cudaGetLastError();
}
cudaError_t launch_scale_vec(const double* diag, double c, double* out, int64_t n, cudaStream_t st) {
    k_div<<<nblocks(n), TB, 0, st>>>(diag, c, out, n);
    return cudaGetLastError();
}
cudaError_t launch_rsqrt_vec(const double* diag, double* out, int64_t n, cudaStream_t st) {
    k_rsqrt<<<nblocks(n), TB, 0, st>>>(diag, out, n);
    return cudaGetLastError();
}
cudaError_t launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t st) {
    k_to_f32<<<nblocks(n), TB, 0, st>>>(in, out, n);
    return cudaGetLastError();
}
cudaError_t launch_copy_f64(const double* src, double* dst, int64_t n, cudaStream_t st) {
    k_copy<<<nblocks(n), TB, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}
cudaError_t launch_gershgorin(const OpDesc& op, bool jacobi, double* blockmax, int nblk, cudaStream_t st) {
    if (op.kind == OP_CSR)
        k_gersh_csr<<<nblk, TB, 0, st>>>(op.rowptr, op.colind, op.vals, jacobi ? op.diag : nullptr, op.n, blockmax);
    else
        k_gersh_faces<<<nblk, TB, 0, st>>>(op.dim, op.nx, op.ny, op.nz, op.wx, op.wy, op.wz, op.diag, jacobi,
                                           blockmax);
    return cudaGetLastError();
}
cudaError_t launch_splitmix_uniform(uint64_t seed, double* v, int64_t n, cudaStream_t st) {
    k_splitmix<<<nblocks(n), TB, 0, st>>>(seed, v, n);
    return cudaGetLastError();
}
cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* partials, int nblk, cudaStream_t st) {
    k_dot<<<nblk, TB, 0, st>>>(a, b, n, partials);
    return cudaGetLastError();
}
cudaError_t launch_lanczos_apply(const OpDesc& op, const double* dhalf, double dhc, const double* q, double* w,
                                 cudaStream_t st) {
    // w = Dh A (Dh q) with Dh = D^-1/2 (vector dhalf or constant dhc); w doubles as scratch.
    k_mul<<<nblocks(op.n), TB, 0, st>>>(dhalf, dhc, q, w, op.n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // A (Dh q) needs a second buffer: the caller passes w adjacent to a scratch of n doubles
    e = launch_apply(op, w, w + op.n, st);
    if (e != cudaSuccess) return e;
    k_mul<<<nblocks(op.n), TB, 0, st>>>(dhalf, dhc, w + op.n, w, op.n);
    return cudaGetLastError();
}
cudaError_t launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st) {
    k_axpby<<<nblocks(n), TB, 0, st>>>(a, x, b, y, n);
    return cudaGetLastError();
}

}  // namespace sstep
