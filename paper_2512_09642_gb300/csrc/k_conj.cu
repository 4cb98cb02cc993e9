// Block-conjugated s-step CG (the Chronopoulos-Gear s-step CG that Section 1 names as the
// origin of the method): the two streaming passes it adds to an outer iteration.
//
// Workspace columns at stride ld: P_+ = [p_0 .. p_s] (0 .. s, p_0 = r_k), Q_(k-1) (s+1 .. 2s),
// A Q_(k-1) (2s+1 .. 3s). Outer iteration k:
//   k_conj_cd      C = (A Q_(k-1))^T P_k and d = Q_(k-1)^T r_k, per-block partials that the Gram
//                  kernel's last block sums (deterministic order) before its s x s work
//                  (conj_transform: B = W_(k-1)^-1 C, W_k, g, then the Gram solve for alpha);
//   k_update_conj  Q_k = P_k - Q_(k-1) B, A Q_k = A P_k - A Q_(k-1) B, x += Q_k alpha,
//                  r_(k+1) = r_k - A Q_k alpha, in place. A P_k is never stored: A p_j =
//                  M (sigma p_j + h_j (p_(j+1) + p_(j-1))), h_0 = 1/theta, h_j = 1/(2 theta),
//                  from the Chebyshev recurrence (Section 2, Definition).
// Both are FP64-pipe bound on this part (s^2 + s and 2 s^2 + 6 s FP64 operations per unknown).
#include "kernels.h"

namespace sstep {
namespace {

constexpr int CJ_THREADS = 512, CJ_WARPS = CJ_THREADS / 32;
constexpr int UC = 256;   // update block

template <int S>
struct ConjShape {
    static constexpr int RPR = S <= 4 ? S : 2;           // rows of C per warp role
    static constexpr int R = (S + RPR - 1) / RPR;        // warp roles
    static constexpr int NSL = CJ_WARPS / R;             // element slabs per block
    static constexpr int M = S * S + S;                  // entries: C (row-major), then d
};

template <int S>
__global__ void __launch_bounds__(CJ_THREADS, 1) k_conj_cd(const double* __restrict__ W, int64_t ld, int64_t n,
                                                          double* __restrict__ partials,
                                                          const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    using CS = ConjShape<S>;
    __shared__ double sm[CS::NSL * CS::M];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp % CS::R, slab = warp / CS::R;
    const int i0 = q * CS::RPR;
    if (slab < CS::NSL) {
        double acc[CS::RPR][S], accd[CS::RPR];
#pragma unroll
        for (int ii = 0; ii < CS::RPR; ++ii) {
            accd[ii] = 0.0;
#pragma unroll
            for (int j = 0; j < S; ++j) acc[ii][j] = 0.0;
        }
        const int64_t stride = (int64_t)gridDim.x * CS::NSL * 32;
        for (int64_t e = ((int64_t)blockIdx.x * CS::NSL + slab) * 32 + lane; e < n; e += stride) {
            double p[S];
#pragma unroll
            for (int j = 0; j < S; ++j) p[j] = __ldg(W + j * ld + e);
#pragma unroll
            for (int ii = 0; ii < CS::RPR; ++ii) {
                const int i = i0 + ii;
                if (i < S) {
                    const double aq = __ldg(W + (2 * S + 1 + i) * ld + e);
                    const double qq = __ldg(W + (S + 1 + i) * ld + e);
#pragma unroll
                    for (int j = 0; j < S; ++j) acc[ii][j] = fma(aq, p[j], acc[ii][j]);
                    accd[ii] = fma(qq, p[0], accd[ii]);
                }
            }
        }
#pragma unroll
        for (int ii = 0; ii < CS::RPR; ++ii) {
            const int i = i0 + ii;
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const double v = warp_sum(acc[ii][j]);
                if (lane == 0 && i < S) sm[slab * CS::M + i * S + j] = v;
            }
            const double v = warp_sum(accd[ii]);
            if (lane == 0 && i < S) sm[slab * CS::M + S * S + i] = v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < CS::M; k += CJ_THREADS) {
        double v = 0.0;
        for (int sl = 0; sl < CS::NSL; ++sl) v += sm[sl * CS::M + k];
        partials[(size_t)blockIdx.x * CS::M + k] = v;
    }
}

template <int S, bool DV>
__global__ void __launch_bounds__(UC, 2) k_update_conj(double* __restrict__ W, int64_t ld, int64_t n,
                                                    const double* __restrict__ diag, double mconst, double sig,
                                                    double h0, double h1, const double* __restrict__ cj,
                                                    double* __restrict__ x, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    __shared__ double Bs[S * S], al[S];
    for (int idx = threadIdx.x; idx < S * S; idx += UC) Bs[idx] = cj[S * S + idx];
    if (threadIdx.x < S) al[threadIdx.x] = ctl->alpha[threadIdx.x];
    __syncthreads();
    // B is read from shared memory at each use (volatile): kept in registers across the
    // element loop it would take S^2 of them and spill.
    const volatile double* Bv = Bs;
#pragma unroll 1
    for (int64_t e = blockIdx.x * (int64_t)UC + threadIdx.x; e < n; e += (int64_t)gridDim.x * UC) {
        double p[S + 1], qn[S], aqn[S];
#pragma unroll
        for (int j = 0; j <= S; ++j) p[j] = W[j * ld + e];
        const double m = DV ? __ldg(diag + e) : mconst;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const double nb = j == 0 ? p[1] : p[j + 1] + p[j - 1];
            qn[j] = p[j];
            aqn[j] = m * fma(j == 0 ? h0 : h1, nb, sig * p[j]);   // (A P_k)_j
        }
        // rank-1 updates with the previous block's columns, one column at a time
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const double qo = W[(S + 1 + i) * ld + e];
            const double aqo = W[(2 * S + 1 + i) * ld + e];
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const double b = Bv[i * S + j];
                qn[j] = fma(-qo, b, qn[j]);
                aqn[j] = fma(-aqo, b, aqn[j]);
            }
        }
        double xs = x[e], rs = p[0];
#pragma unroll
        for (int j = 0; j < S; ++j) {
            W[(S + 1 + j) * ld + e] = qn[j];
            W[(2 * S + 1 + j) * ld + e] = aqn[j];
            xs = fma(al[j], qn[j], xs);
            rs = fma(-al[j], aqn[j], rs);
        }
        x[e] = xs;
        W[e] = rs;
    }
}

template <int S>
int conj_occupancy() {
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_conj_cd<S>, CJ_THREADS, 0) != cudaSuccess || occ < 1)
        occ = 1;
    return occ;
}

}  // namespace

int conj_cd_blocks(int s, int64_t n, int sm_count) {
    int occ = 1, nsl = 1;
    switch (s) {
#define SSTEP_CASE(S) case S: occ = conj_occupancy<S>(); nsl = ConjShape<S>::NSL; break;
        SSTEP_CASE(1) SSTEP_CASE(2) SSTEP_CASE(3) SSTEP_CASE(4) SSTEP_CASE(5) SSTEP_CASE(6) SSTEP_CASE(7)
        SSTEP_CASE(8) SSTEP_CASE(9) SSTEP_CASE(10) SSTEP_CASE(11) SSTEP_CASE(12) SSTEP_CASE(13) SSTEP_CASE(14)
        SSTEP_CASE(15) SSTEP_CASE(16)
#undef SSTEP_CASE
        default: return 1;
    }
    const int64_t per_block = (int64_t)nsl * 32;
    int64_t want = (n + per_block - 1) / per_block;
    if (want < 1) want = 1;
    const int64_t cap = (int64_t)sm_count * occ;
    return (int)(want < cap ? want : cap);
}

cudaError_t launch_conj_cd(int s, const double* W, int64_t ld, int64_t n, double* partials, int nblk, const Ctl* ctl,
                           cudaStream_t st) {
    switch (s) {
#define SSTEP_CASE(S) case S: k_conj_cd<S><<<nblk, CJ_THREADS, 0, st>>>(W, ld, n, partials, ctl); break;
        SSTEP_CASE(1) SSTEP_CASE(2) SSTEP_CASE(3) SSTEP_CASE(4) SSTEP_CASE(5) SSTEP_CASE(6) SSTEP_CASE(7)
        SSTEP_CASE(8) SSTEP_CASE(9) SSTEP_CASE(10) SSTEP_CASE(11) SSTEP_CASE(12) SSTEP_CASE(13) SSTEP_CASE(14)
        SSTEP_CASE(15) SSTEP_CASE(16)
#undef SSTEP_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_update_conj(int s, double* W, int64_t ld, int64_t n, const double* diag, double dconst,
                               double theta, double sigma, const double* cj, double* x, const Ctl* ctl,
                               cudaStream_t st) {
    int64_t b = (n + UC - 1) / UC;
    const int64_t cap = 4 * (int64_t)device_sm_count();
    const int nb = (int)(b < 1 ? 1 : (b < cap ? b : cap));
    const double h0 = 1.0 / theta, h1 = 0.5 / theta;
    const bool dv = diag != nullptr;
    switch (s) {
#define SSTEP_CASE(S)                                                                                          \
    case S:                                                                                                    \
        if (dv) k_update_conj<S, true><<<nb, UC, 0, st>>>(W, ld, n, diag, dconst, sigma, h0, h1, cj, x, ctl);  \
        else k_update_conj<S, false><<<nb, UC, 0, st>>>(W, ld, n, diag, dconst, sigma, h0, h1, cj, x, ctl);    \
        break;
        SSTEP_CASE(1) SSTEP_CASE(2) SSTEP_CASE(3) SSTEP_CASE(4) SSTEP_CASE(5) SSTEP_CASE(6) SSTEP_CASE(7)
        SSTEP_CASE(8) SSTEP_CASE(9) SSTEP_CASE(10) SSTEP_CASE(11) SSTEP_CASE(12) SSTEP_CASE(13) SSTEP_CASE(14)
        SSTEP_CASE(15) SSTEP_CASE(16)
#undef SSTEP_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sstep
