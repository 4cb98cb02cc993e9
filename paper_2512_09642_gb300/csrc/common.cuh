// Internal definitions shared by the kernels and the host driver of the s-step CG library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sstep_cg.h"
#include "ieee_conv.cuh"

namespace sstep {

constexpr int MAXS = SSTEP_MAX_S;
constexpr int MAXC = MAXS + 1;            // basis columns p_0 .. p_s

// Termination states written by the Gram kernel's last block into Ctl::done (TIMED_OUT: a
// bounded device-side wait of a step kernel expired).
enum Done : int { RUNNING = 0, CONVERGED = 1, MAX_OUTER = 2, NUMERICAL = 3, TIMED_OUT = 4 };

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

// Exact float -> double and float(v * 2^k), rounded to nearest, built with integer
// instructions from the IEEE-754 fields (ieee_conv.cuh): this part converts between FP32 and
// FP64 at the FP64 rate, and no input class takes a hardware conversion.
__device__ __forceinline__ double f2d_exact(float f) {
    return __longlong_as_double((long long)f32_to_f64_bits(__float_as_uint(f)));
}

__device__ __forceinline__ float d2f_scaled(double v, int k) {
    return __uint_as_float(f64_to_f32_scaled_bits((uint64_t)__double_as_longlong(v), k));
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
