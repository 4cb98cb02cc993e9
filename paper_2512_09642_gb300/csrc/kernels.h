// Host-side launchers of the library's kernels (internal; not part of the C ABI).
#pragma once

#include <cuda.h>   // CUtensorMap

#include "common.cuh"

namespace sstep {

// The two events that time one solve, destroyed on every return path of the solve.
struct SolveEvents {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SolveEvents() = default;
    SolveEvents(const SolveEvents&) = delete;
    SolveEvents& operator=(const SolveEvents&) = delete;
    ~SolveEvents() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Operator description handed to kernels (plain pointers, no ownership).
struct OpDesc {
    int kind;            // OP_CSR or OP_STENCIL
    int64_t n;
    // CSR
    const int32_t* rowptr;
    const int32_t* colind;
    const double* vals;
    const float* vals32;   // FP32 copy (mixed precision), may be null
    // stencil
    int dim, nx, ny, nz;
    int box;               // 1: box stencil (all 3^dim - 1 neighbours, Poisson weights)
    const double* wx;      // face weights, null for the Poisson stencil
    const double* wy;
    const double* wz;
    const float* wx32;     // FP32 copies (mixed precision)
    const float* wy32;
    const float* wz32;
    // diagonal of A and 2 theta / diag (null when the diagonal is the constant dconst)
    const double* diag;
    const double* cdinv;
    const float* diag32;
    const float* cdinv32;
    double dconst;
};
enum { OP_CSR = 0, OP_STENCIL = 1 };

// One Chebyshev step (Section 2, Definition): out = c (M^-1 A p - sigma p) - q,
// c = theta for the first step (q absent) and 2 theta after. `first` selects the form.
// Precision T = double (FP64) or float (mixed form basis). mom != null (stencil operators
// only): the step also writes its per-block partials of <p, p> and <p, out> there (the fused
// moments of gram_form FUSED; FP64 double[2][nblk], FP32 float[4][nblk] with nblk =
// cheb_step_blocks(op, fp32)).
template <typename T>
cudaError_t launch_cheb_step(const OpDesc& op, const T* p, const T* q, T* out, double theta,
                             double sigma, bool first, bool jacobi, const Ctl* ctl, cudaStream_t st,
                             void* mom = nullptr);
// Blocks of the stencil step kernel launch_cheb_step uses for op in FP32 or FP64 (0 for CSR),
// or, with tma, those of launch_cheb_step_tma.
int cheb_step_blocks(const OpDesc& op, bool fp32, bool tma = false);

// FP32 7-point Poisson step through tensor-map (TMA) tiles: 3D, nx a multiple of 4. Each
// basis column needs two maps, made once: `mp` (the column read as p, tiles with a halo) and
// `mq` (read as q). step_tma_maps returns cudaErrorNotSupported when the shape does not allow
// it or the driver has no tensor-map encoder. launch_cheb_step_tma computes the same step as
// launch_cheb_step<float> (bitwise) from the maps of p and q (mq unused when first); a
// bounded wait that expires sets ctl->done = TIMED_OUT.
bool step_tma_shape(const OpDesc& op);
cudaError_t step_tma_maps(const OpDesc& op, float* column, CUtensorMap* mp, CUtensorMap* mq);
cudaError_t launch_cheb_step_tma(const OpDesc& op, const CUtensorMap& mp, const CUtensorMap& mq, float* out,
                                 double theta, double sigma, bool first, bool jacobi, Ctl* ctl, cudaStream_t st,
                                 void* mom = nullptr);
// Self-test of the TMA step's bounded waits: one launch on a 64 x 8 x 4 grid whose stages
// expect more bytes than their copies deliver, with a short wait limit; done_state receives
// the control block's state afterwards (TIMED_OUT when the waits gave up as designed).
cudaError_t tma_wait_selftest(int* done_state);

// r = b - A x in FP64; writes r (double, if non-null) and, if r32 != null, the FP32 copy
// scaled by ctl->scale_next (mode 2); reduces ||r||^2 through `partials` (one double per
// block): mode 0 -> ctl->r0_sq (initial residual), 1 -> ctl->true_sq (exit check),
// 2 -> ctl->rk_sq plus the stopping test (mixed-form refresh; skipped once ctl->done).
cudaError_t launch_residual(const OpDesc& op, const double* b, const double* x, double* r, float* r32,
                            double* partials, Ctl* ctl, int mode, cudaStream_t st);
size_t residual_partials_needed(const OpDesc& op);

// Mixed-form conversions on n values: out = float(in * 2^k) (d2f_scaled), back = double(out)
// (f2d_exact).
cudaError_t launch_convert_check(const double* in, int k, float* out, double* back, int64_t n, cudaStream_t st);

// y = A x (FP64).
cudaError_t launch_apply(const OpDesc& op, const double* x, double* y, cudaStream_t st);

// Gram reduction + column scaling + FGS (or Cholesky) on P_+ = [p_0 .. p_s] (FP64 or FP32
// columns at stride ld). Per-block partials go to `partials` (gram_partials_needed doubles).
struct GramArgs {
    int s, nu, solver, form;
    // stopping test in the Gram finish: 0 none (the mixed form's FP64 refresh tests), 1 on
    // c_0 = ||r_k||^2, 2 on c_0 / scale^2 (mixed form, outer iterations without a refresh)
    int check;
    // per-outer record ring (hist_cap records of 4 doubles), or null
    double* hist;
    int hist_cap;
    double theta, sigma;
    bool dvec;                 // D is the vector op.diag (else the constant op.dconst)
    double dconst;
    const double* diag;
    const float* diag32;
    int64_t n, ld;
    const void* P;             // column-major n x (s+1), double or float
    bool fp32;
    // block-conjugated form (FP64, s <= 16): C / d partials of launch_conj_cd and the state
    // [W_(k-1) | B_k]; conj = 0 for the plain iteration
    int conj, conj_nblk;
    const double* conj_partials;
    double* cj;
};
cudaError_t launch_gram(const GramArgs& g, double* partials, Ctl* ctl, int nblocks, cudaStream_t st);
// Gram finish of the fused moments form: sums the s step kernels' partials (part, nblk blocks
// per step, layout of launch_cheb_step's mom) through part2 (moments_finish_blocks(nblk) x 2s
// doubles) and runs the column scaling and Gram solve (M = g.dconst I).
constexpr int MAX_FIN_BLOCKS = 64;
int moments_finish_blocks(int nblk);
cudaError_t launch_moments_finish(const GramArgs& g, const void* part, int nblk, double* part2, Ctl* ctl,
                                  cudaStream_t st);
int gram_blocks(const GramArgs& g, int sm_count);
size_t gram_partials_needed(const GramArgs& g, int nblocks);

// x += P alpha; r <- p_0 - D P_+ beta (written to column 0) unless skip_r.
struct UpdateArgs {
    int s;
    bool dvec;
    const double* diag;
    int64_t n, ld;
    const void* P;
    bool fp32;
    double* x;
    bool skip_r;
};
cudaError_t launch_update(const UpdateArgs& u, const Ctl* ctl, cudaStream_t st);
// Mixed form: x += P alpha / scale with FP32 P (compensated FP32 sum, exact FP64 add-in);
// write_r: also the recursive FP32 residual over column 0 (diag: the vector M, else M const).
cudaError_t launch_update_mixed(float* P, int64_t ld, int s, int64_t n, double* x, const Ctl* ctl, cudaStream_t st,
                                bool write_r, const float* diag);

// Block-conjugated form (FP64, s <= 16). The workspace holds, at stride ld, the columns
// P_+ = [p_0 .. p_s] (0 .. s), Q_(k-1) (s+1 .. 2s) and A Q_(k-1) (2s+1 .. 3s).
// launch_conj_cd: per-block partials of C = (A Q_(k-1))^T P_k (s x s, row i = column i of
// A Q) and d = Q_(k-1)^T r_k (s), S*S + S doubles per block, for the Gram kernel's last block.
// launch_update_conj: Q_k = P_k - Q_(k-1) B, A Q_k = A P_k - A Q_(k-1) B (A P_k through the
// Chebyshev change of basis), x += Q_k alpha, r = r_k - A Q_k alpha, all in place.
cudaError_t launch_conj_cd(int s, const double* W, int64_t ld, int64_t n, double* partials, int nblk, const Ctl* ctl,
                           cudaStream_t st);
int conj_cd_blocks(int s, int64_t n, int sm_count);
cudaError_t launch_update_conj(int s, double* W, int64_t ld, int64_t n, const double* diag, double dconst,
                               double theta, double sigma, const double* cj, double* x, const Ctl* ctl,
                               cudaStream_t st);

// FGS as the AMG coarse-grid solver (Section 6) on a stencil operator with bx x by x bz box
// aggregation: nu sweeps on A_c y = g (y in place). streaming = 0: A_c formed into Ac
// (nc * nc doubles, nc <= coarse_formed_max_nc()); 1: z (n doubles) and dc (nc doubles) as
// scratch, A_c never formed.
int coarse_formed_max_nc();
cudaError_t launch_coarse_fgs(const OpDesc& op, int bx, int by, int bz, int nc, const double* g, double* y, int nu,
                              int streaming, double* z, double* dc, double* Ac, cudaStream_t st);

// Sets the graph while-node condition to (ctl->done == RUNNING).
cudaError_t launch_loop_cond(cudaGraphConditionalHandle handle, const Ctl* ctl, cudaStream_t st);

// Adjoint: dL/dkappa of the diffusion stencil from x and lambda (see k_adjoint.cu).
cudaError_t launch_grad_kappa(int dim, int nx, int ny, int nz, const double* kappa, const double* x,
                              const double* lam, double* g, cudaStream_t st);

// Streaming multiprocessors of the current device (queried once per device; the launchers
// size their grids as a multiple of it).
int device_sm_count();

// Setup kernels.
cudaError_t launch_csr_diag(const OpDesc& op, double* diag, int* bad, cudaStream_t st);
cudaError_t launch_stencil_faces(int dim, int nx, int ny, int nz, const double* kappa, double* wx, double* wy,
                                 double* wz, double* diag, int* bad, cudaStream_t st);
cudaError_t launch_scale_vec(const double* diag, double c, double* out, int64_t n, cudaStream_t st);
cudaError_t launch_rsqrt_vec(const double* diag, double* out, int64_t n, cudaStream_t st);
cudaError_t launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t st);
cudaError_t launch_gershgorin(const OpDesc& op, bool jacobi, double* blockmax, int nblk, cudaStream_t st);
// Lanczos helpers on B = D^-1/2 A D^-1/2 (D^-1/2 = dhalf or a constant).
cudaError_t launch_splitmix_uniform(uint64_t seed, double* v, int64_t n, cudaStream_t st);
cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* partials, int nblk, cudaStream_t st);
cudaError_t launch_lanczos_apply(const OpDesc& op, const double* dhalf, double dhc, const double* q, double* w,
                                 cudaStream_t st);
cudaError_t launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st);
cudaError_t launch_copy_f64(const double* src, double* dst, int64_t n, cudaStream_t st);

}  // namespace sstep
