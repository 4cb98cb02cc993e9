// Outer-iteration update (Section 2): x_(k+1) = x_k + P alpha and the residual
// r_(k+1) = r_k - A P alpha, the latter through the change of basis A P = M P_+ B:
// r_(k+1) = p_0 - M P_+ beta with beta = B alpha (p_0 = r_k), so A P is never stored.
// With a constant M the Gram kernel folds M and p_0 into gamma: r_(k+1) = sum_k gamma_k p_k.
// The new residual overwrites column 0 of P_+ in place.
#include "kernels.h"

namespace sstep {
namespace {

constexpr int UB = 256;

template <bool DV>
__global__ void __launch_bounds__(UB) k_update_f64(const double* __restrict__ P, int64_t ld, int s,
                                                   const double* __restrict__ diag, int64_t n, double* __restrict__ x,
                                                   double* __restrict__ r, bool skip_r, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    __shared__ double al[MAXS], be[MAXC];
    if (threadIdx.x < s) al[threadIdx.x] = ctl->alpha[threadIdx.x];
    if (threadIdx.x <= s) be[threadIdx.x] = ctl->beta[threadIdx.x];
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)UB + threadIdx.x; e < n; e += (int64_t)gridDim.x * UB) {
        const double p0 = __ldg(P + e);
        double xs = fma(al[0], p0, __ldg(x + e));
        double rs = be[0] * p0;
#pragma unroll 4
        for (int j = 1; j < s; ++j) {
            const double p = __ldg(P + j * ld + e);
            xs = fma(al[j], p, xs);
            rs = fma(be[j], p, rs);
        }
        x[e] = xs;
        if (!skip_r) {
            rs = fma(be[s], __ldg(P + s * ld + e), rs);
            r[e] = DV ? fma(-__ldg(diag + e), rs, p0) : rs;
        }
    }
}

// Mixed form (FP32 basis p^_j = scale * p_j): x += (sum_j alpha_j p^_j) / scale, the sum
// taken in FP32 in the scaled domain (where its terms are O(1)) with alpha rounded to FP32, and
// added to x in FP64 through an exact conversion (one FMA on the FP64 pipe per unknown). The
// increment only has to be accurate relative to itself: its FP32 rounding (about 1e-7 of the
// terms) is part of the next residual, which the FP64 refresh r = b - A x recomputes, as in
// iterative refinement.
// WR (the next outer iteration does not refresh): also the recursive residual in the same
// scaled domain, written over p^_0 in FP32: r^ = sum_k gamma_k p^_k (constant M) or
// r^ = p^_0 - d (sum_k beta_k p^_k) (vector M = diag d). Its FP32 rounding drifts from
// b - A x until the next refresh, which restores it.
template <int S, bool WR, bool DV>
__global__ void __launch_bounds__(UB) k_update_mixed(float* __restrict__ P, int64_t ld, int64_t n,
                                                     double* __restrict__ x, const float* __restrict__ diag,
                                                     const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    __shared__ float af[S], gf[S + 1];
    if (threadIdx.x < S) af[threadIdx.x] = __double2float_rn(ctl->alpha[threadIdx.x]);
    if (WR && threadIdx.x <= S) gf[threadIdx.x] = __double2float_rn(ctl->beta[threadIdx.x]);
    __syncthreads();
    const double inv_scale = 1.0 / ctl->scale;   // exact: scale is a power of two
    constexpr int NC = WR ? S + 1 : S;
    // two consecutive unknowns per thread and iteration: 8-byte loads of the FP32 columns (ld
    // is even, the columns 8-byte aligned) and 16-byte loads and stores of x (16-byte aligned),
    // half the load instructions of one unknown at a time; an odd last unknown alone
    const int64_t npair = n / 2;
    for (int64_t e2 = blockIdx.x * (int64_t)UB + threadIdx.x; e2 < npair; e2 += (int64_t)gridDim.x * UB) {
        const int64_t e = 2 * e2;
        float2 pv[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) pv[j] = __ldg(reinterpret_cast<const float2*>(P + j * ld + e));
        float sx0 = 0.f, sx1 = 0.f;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            sx0 = fmaf(af[j], pv[j].x, sx0);
            sx1 = fmaf(af[j], pv[j].y, sx1);
        }
        double2 xv = *reinterpret_cast<const double2*>(x + e);
        xv.x = fma(f2d_exact(sx0), inv_scale, xv.x);
        xv.y = fma(f2d_exact(sx1), inv_scale, xv.y);
        *reinterpret_cast<double2*>(x + e) = xv;
        if (WR) {
            float sr0 = 0.f, sr1 = 0.f;
#pragma unroll
            for (int k = 0; k <= S; ++k) {
                sr0 = fmaf(gf[k], pv[k].x, sr0);
                sr1 = fmaf(gf[k], pv[k].y, sr1);
            }
            float2 rv;
            if (DV) {
                const float2 d = __ldg(reinterpret_cast<const float2*>(diag + e));
                rv.x = fmaf(-d.x, sr0, pv[0].x);
                rv.y = fmaf(-d.y, sr1, pv[0].y);
            } else {
                rv.x = sr0;
                rv.y = sr1;
            }
            *reinterpret_cast<float2*>(P + e) = rv;
        }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t e = n - 1;
        float pv[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) pv[j] = P[j * ld + e];
        float sx = 0.f;
#pragma unroll
        for (int j = 0; j < S; ++j) sx = fmaf(af[j], pv[j], sx);
        x[e] = fma(f2d_exact(sx), inv_scale, x[e]);
        if (WR) {
            float sr = 0.f;
#pragma unroll
            for (int k = 0; k <= S; ++k) sr = fmaf(gf[k], pv[k], sr);
            P[e] = DV ? fmaf(-diag[e], sr, pv[0]) : sr;
        }
    }
}

// Body of the graph's while node: keep looping while the outer iteration is running.
__global__ void k_loop_cond(cudaGraphConditionalHandle handle, const Ctl* __restrict__ ctl) {
    cudaGraphSetConditional(handle, ctl->done == RUNNING ? 1u : 0u);
}

// Grid: per_sm blocks per SM at most (the FP64 update is FP64-pipe bound and runs best with
// 4, the HBM-bound mixed update with 8 in flight), fewer for short vectors.
int blocks_for(int64_t n, int per_sm) {
    const int64_t b = (n + UB - 1) / UB;
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace

cudaError_t launch_loop_cond(cudaGraphConditionalHandle handle, const Ctl* ctl, cudaStream_t st) {
    k_loop_cond<<<1, 1, 0, st>>>(handle, ctl);
    return cudaGetLastError();
}

cudaError_t launch_update_mixed(float* P, int64_t ld, int s, int64_t n, double* x, const Ctl* ctl, cudaStream_t st,
                                bool write_r, const float* diag) {
    // the paired loads need 8-byte aligned FP32 columns and diagonal and a 16-byte aligned x
    if ((ld & 1) || ((uintptr_t)P & 7u) || ((uintptr_t)x & 15u) || (diag && ((uintptr_t)diag & 7u)))
        return cudaErrorMisalignedAddress;
    const int nb = blocks_for((n + 1) / 2, 8);
    switch (s) {
#define SSTEP_CASE(S)                                                                                  \
    case S:                                                                                            \
        if (!write_r) k_update_mixed<S, false, false><<<nb, UB, 0, st>>>(P, ld, n, x, nullptr, ctl);    \
        else if (diag) k_update_mixed<S, true, true><<<nb, UB, 0, st>>>(P, ld, n, x, diag, ctl);        \
        else k_update_mixed<S, true, false><<<nb, UB, 0, st>>>(P, ld, n, x, nullptr, ctl);              \
        break;
        SSTEP_CASE(1) SSTEP_CASE(2) SSTEP_CASE(3) SSTEP_CASE(4) SSTEP_CASE(5) SSTEP_CASE(6) SSTEP_CASE(7)
        SSTEP_CASE(8) SSTEP_CASE(9) SSTEP_CASE(10) SSTEP_CASE(11) SSTEP_CASE(12) SSTEP_CASE(13) SSTEP_CASE(14)
        SSTEP_CASE(15) SSTEP_CASE(16) SSTEP_CASE(17) SSTEP_CASE(18) SSTEP_CASE(19) SSTEP_CASE(20) SSTEP_CASE(21)
        SSTEP_CASE(22) SSTEP_CASE(23) SSTEP_CASE(24) SSTEP_CASE(25) SSTEP_CASE(26) SSTEP_CASE(27) SSTEP_CASE(28)
        SSTEP_CASE(29) SSTEP_CASE(30) SSTEP_CASE(31) SSTEP_CASE(32)
#undef SSTEP_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_update(const UpdateArgs& u, const Ctl* ctl, cudaStream_t st) {
    if (u.fp32) return cudaErrorNotSupported;
    const double* P = (const double*)u.P;
    double* r = (double*)u.P;   // column 0
    if (u.dvec)
        k_update_f64<true><<<blocks_for(u.n, 4), UB, 0, st>>>(P, u.ld, u.s, u.diag, u.n, u.x, r, u.skip_r, ctl);
    else
        k_update_f64<false><<<blocks_for(u.n, 4), UB, 0, st>>>(P, u.ld, u.s, nullptr, u.n, u.x, r, u.skip_r, ctl);
    return cudaGetLastError();
}

}  // namespace sstep
