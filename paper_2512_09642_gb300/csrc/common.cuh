// Internal definitions shared by the kernels and the host driver of the s-step CG library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sstep_cg.h"

namespace sstep {

constexpr int MAXS = SSTEP_MAX_S;
constexpr int MAXC = MAXS + 1;            // basis columns p_0 .. p_s

// Termination states written by the Gram kernel's last block into Ctl::done.
enum Done : int { RUNNING = 0, CONVERGED = 1, MAX_OUTER = 2, NUMERICAL = 3 };

// Device-resident control block of one handle. Kernels of an outer iteration communicate
// through it (the Gram solve writes alpha/beta, the update reads them), and every kernel
// returns immediately once `done` is set, so surplus outer iterations queued after
// convergence cost one launch each and change nothing.
struct Ctl {
    double alpha[MAXS];       // alpha = S a: coefficients of the basis in x += P alpha
    double beta[MAXC];        // residual update r <- p_0 - sum_k beta_k (D p_k) (see update)
    double d[MAXS];           // column scaling d_i = G_ii^-1/2 (0 = dropped column)
    double ct[MAXS];          // c~ = S P^T r
    double Gt[MAXS * MAXS];   // G~ = S G S, row-major (diagnostics and tests)
    double r0_sq;             // ||r_0||^2
    double rk_sq;             // ||r_k||^2 seen by the latest Gram
    double true_sq;           // ||b - A x||^2 of the latest true-residual evaluation
    double min_gii;           // smallest G_ii seen
    double delta;             // ||c~ - G~ a|| / ||c~|| of the last FGS solve
    double tol_sq;            // tol^2
    double scale;             // mixed form: power of two applied to p_0 in this outer iteration
    double scale_next;        // mixed form: power of two the next refresh applies
    int done;
    int conj_valid;           // block-conjugated form: 1 once a previous block (W, Q, AQ) exists
    int outer;                // outer iterations applied
    int max_outer;
    int launches;             // not maintained on device; reserved
    unsigned int counter;     // last-block arrival counter (Gram)
    unsigned int counter2;    // last-block arrival counter (norm reductions)
};

// ---- host error plumbing ----------------------------------------------------------------
const char* cuda_err_name(cudaError_t e);

// ---- device helpers ---------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exact float -> double by rebuilding the IEEE-754 fields with integer instructions (FP32
// exponent e + 896 = FP64 exponent, mantissa shifted left by 29). Keeps the conversion off
// the FP64 pipe, which converts at the FP64 rate on this part. Zero keeps its sign;
// subnormal, infinite and NaN inputs take the hardware conversion.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xffu;
    if (ex == 0u) {
        if ((u & 0x7fffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
        return (double)f;
    }
    if (ex == 0xffu) return (double)f;
    const unsigned hi = (u & 0x80000000u) | ((ex + 896u) << 20) | ((u >> 3) & 0xfffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
}

// float(v * 2^k), rounded to nearest (ties to even), built from the IEEE-754 fields with
// integer instructions: the FP64 exponent is rebiased by k - 896 and the 52-bit mantissa is
// rounded to 23 bits (a round-up that overflows the mantissa carries into the exponent, which
// is the correct result). Zero, subnormal, infinite and NaN inputs, and results outside the
// normal FP32 range, take the FP64 path.
__device__ __forceinline__ float d2f_scaled(double v, int k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32);
    const int ex = (int)((hi >> 20) & 0x7ffu);
    const int fe = ex - 1023 + 127 + k;
    if (ex == 0 || ex == 0x7ff || fe <= 0 || fe >= 254) return __double2float_rn(ldexp(v, k));
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    const unsigned m = (unsigned)(mant >> 29);
    const unsigned rest = (unsigned)(mant & 0x1FFFFFFFull);
    unsigned bits = ((unsigned)fe << 23) | m;
    if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) bits += 1u;
    return __uint_as_float((hi & 0x80000000u) | bits);
}

// Compensated FP32 arithmetic (Knuth's TwoSum, FMA-based TwoProduct; Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 2005). The _rn intrinsics are
// never contracted into FMAs, which the error-free transformations rely on.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (sh, sl) += x * y with the product's rounding error carried in sl.
__device__ __forceinline__ void dot2_acc(float x, float y, float& sh, float& sl) {
    const float ph = __fmul_rn(x, y);
    const float pl = fmaf(x, y, -ph);
    float t, e;
    two_sum(sh, ph, t, e);
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(e, pl));
}

}  // namespace sstep
