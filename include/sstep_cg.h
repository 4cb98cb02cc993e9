/*
 * sstep_cg.h - C ABI of a GB300 (sm_103a) library for Chebyshev-basis s-step Conjugate
 * Gradient with Forward Gauss-Seidel (FGS) Gram solves.
 *
 * Method: Thomas and D'Ambra, "Inexact Gauss-Seidel Coarse Solvers for AMG and s-step CG",
 * arXiv 2512.09642. Section 2 ("Preliminaries") defines the outer iteration on
 * K_s(M^-1 A, r_k): a basis P, the Gram system G alpha = P^T r_k with G = P^T A P, and the
 * update x_(k+1) = x_k + P alpha. Section 2, Definition "Chebyshev Polynomial Basis" gives the
 * basis recurrence; Section 2, "Column scaling" the scaling d_i = (p_i^T A p_i)^-1/2 and the
 * FGS iteration (I + L) a^(l+1) = P~^T r_k - L^T a^(l), a^(0) = 0. Section 8 gives the
 * stopping rule ||r_k|| / ||r_0|| < tol and the Lanczos spectral estimate.
 *
 * Conventions shared by every entry point:
 *  - Pointers whose name ends in _d are DEVICE pointers (CUDA global memory of the current
 *    device); _h marks HOST pointers. Device arrays must be 16-byte aligned.
 *  - Vectors have n double entries. Grid unknown (i, j, k) of an nx*ny*nz grid has index
 *    i + nx * (j + ny * k).
 *  - The caller owns every array it passes; the library never frees it. Arrays passed to a
 *    create call are BORROWED for the handle's lifetime and must stay valid and unchanged
 *    until sstep_cg_destroy. The handle owns its workspace.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream); every kernel
 *    of the handle runs on it, and calls return with work possibly still queued on it,
 *    except where a call says it synchronises.
 *  - Errors are status codes; nothing throws or exits across the ABI. The text of the last
 *    error on a handle is kept (sstep_cg_last_error). A CUDA error leaves the handle
 *    unusable except for sstep_cg_destroy.
 */
#ifndef SSTEP_CG_H
#define SSTEP_CG_H

#include <stdint.h>

#if defined(__GNUC__)
#define SSTEP_API __attribute__((visibility("default")))
#else
#define SSTEP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sstep_cg_s* sstep_cg_t;

typedef enum {
    SSTEP_OK = 0,
    SSTEP_ERR_INVALID_ARG = 1,     /* bad size, option, pointer or alignment */
    SSTEP_ERR_CUDA = 2,            /* a CUDA runtime call or kernel failed */
    SSTEP_ERR_OOM = 3,             /* workspace allocation failed */
    SSTEP_ERR_NUMERICAL = 4,       /* NaN/Inf in the Gram system, or every column dropped */
    SSTEP_ERR_NO_CONVERGENCE = 5,  /* max_outer reached, or the true residual stayed above tol */
    SSTEP_ERR_TIMEOUT = 6,         /* a bounded device-side wait expired */
    SSTEP_ERR_UNSUPPORTED = 7      /* valid request the library does not implement */
} sstep_status;

enum { SSTEP_BOUNDS_GIVEN = 0, SSTEP_BOUNDS_GERSH_LANCZOS10 = 1, SSTEP_BOUNDS_LANCZOS10 = 2 };
enum { SSTEP_GRAM_SOLVE_FGS = 0, SSTEP_GRAM_SOLVE_CHOLESKY = 1 };
enum { SSTEP_PRECISION_FP64 = 0, SSTEP_PRECISION_MIXED = 1 };
enum { SSTEP_PRECOND_NONE = 0, SSTEP_PRECOND_JACOBI = 1 };
enum { SSTEP_START_R = 0 };
/* How G = P^T A P and c = P^T r_k are formed (the Gram system of Section 2). A P is never
 * stored: with the recurrence of the Definition "Chebyshev Polynomial Basis", A P = M P_+ B
 * (P_+ = [p_0 .. p_s], B the tridiagonal change of basis).
 *  DIRECT: one pass over P_+ reduces the s(s+1)/2 + s inner products <p_a, p_b>_M.
 *  MOMENTS: p_j = T_j(A^) p_0 with A^ = theta (M^-1 A - sigma) self-adjoint in <u, v>_M, so
 *    <p_i, p_j>_M = (mu_(i+j) + mu_|i-j|) / 2 with the Chebyshev moments mu_k = <p_0, T_k(A^) p_0>_M
 *    (the spectral expansion of Section 4); one pass over P_+ reduces the 2s moments.
 *  FUSED: the same moments, with no pass over the basis: the step kernel that writes p_(j+1)
 *    also reduces <p_j, p_j>_M and <p_j, p_(j+1)>_M (mu_2j = 2 <p_j, p_j>_M - mu_0, mu_(2j+1) =
 *    2 <p_j, p_(j+1)>_M - mu_1), so each basis vector is read once per outer iteration. Needs a
 *    stencil operator with a constant M (the Poisson or box stencil, or precond NONE; otherwise
 *    SSTEP_ERR_UNSUPPORTED) and block_conjugate = 0. */
enum { SSTEP_GRAM_FORM_DIRECT = 0, SSTEP_GRAM_FORM_MOMENTS = 1, SSTEP_GRAM_FORM_FUSED = 2 };
enum { SSTEP_STEP_AUTO = 0, SSTEP_STEP_TMA = 1, SSTEP_STEP_PLAIN = 2 };

#define SSTEP_MAX_S 32

typedef struct {
    int s;                 /* basis size, 1 <= s <= SSTEP_MAX_S (default 8) */
    int nu;                /* FGS sweeps per Gram solve, 1 <= nu <= 10000 (default 25) */
    double lambda_min;     /* spectral bounds of M^-1 A when bounds_mode = GIVEN */
    double lambda_max;     /*   (0 <= lambda_min < lambda_max) */
    int bounds_mode;       /* SSTEP_BOUNDS_*: GIVEN, or estimated at create time (Section 8) */
    double tol;            /* relative residual ||r|| / ||r_0|| to stop at (default 1e-8) */
    int max_outer;         /* outer-iteration limit (default 100000) */
    int gram_solver;       /* SSTEP_GRAM_SOLVE_FGS (paper) or _CHOLESKY (baseline) */
    int precision;         /* SSTEP_PRECISION_FP64 or _MIXED (FP32 basis, FP64 Gram/x/residual) */
    int precond;           /* SSTEP_PRECOND_JACOBI (M = diag A) or _NONE (M = I) */
    int basis_start;       /* SSTEP_START_R: p_0 = r_k as written in Section 2 */
    int gram_form;         /* how G is formed: SSTEP_GRAM_FORM_DIRECT, _MOMENTS or _FUSED */
    int refresh_period;    /* MIXED: recompute r = b - A x in FP64 in the first outer iteration of
                              every group of this many (>= 1, default 1); the others update the
                              FP32 residual recursively (r -= A P alpha through the change of
                              basis) and test convergence on it. FP64: unused */
    int max_refresh;       /* true-residual restarts after recursive convergence (default 3) */
    uint64_t seed;         /* splitmix64 stream of the Lanczos start vector (default 5000) */
    int use_graph;         /* 1: run the outer loop as a CUDA graph with a device-side while
                              condition; 0: host loop that checks every check_every outers. The
                              handle keeps the graph of the last (b, x) pointer pair it solved;
                              a call with another pair captures and instantiates it again (host
                              time), so repeated solves should reuse their b and x buffers */
    int check_every;       /* host loop only: outers launched between convergence checks */
    int profile_every;     /* > 0: time each kernel of one outer iteration in every this many
                              check intervals with CUDA events (sstep_cg_info.prof_*); 0: off */
    int batch_chunk;       /* batched form: unknowns per Gram/update work item (0: 8192) */
    int batch_ctas_per_sm; /* batched form: resident blocks per SM of the stencil kernels (0: 6) */
    int block_conjugate;   /* 1: make each Chebyshev block A-conjugate to the previous one (the
                              Chronopoulos-Gear s-step CG cited in Section 1): Q_k = P_k -
                              Q_(k-1) W_(k-1)^-1 (A Q_(k-1))^T P_k, x += Q_k alpha; B is solved
                              with the same scaled FGS as alpha. FP64, s <= 16 (else
                              SSTEP_ERR_UNSUPPORTED); 2s more basis-length vectors of workspace.
                              0 (default): the restarted iteration of Section 2 as written */
    int history;           /* > 0: keep a record of the last `history` outer iterations on the
                              device (sstep_cg_history): the relative residual entering it, the
                              Gram solve's inexactness delta_k (Section 7) and the smallest
                              unscaled G_ii; 0 (default): none */
    int step_kernel;       /* MIXED, 3D Poisson stencil with nx a multiple of 4: how the FP32
                              Chebyshev step reads its planes. SSTEP_STEP_AUTO (default): through
                              tensor-map (TMA) tiles when the step's three vectors exceed the L2
                              cache, else plain loads; SSTEP_STEP_TMA / SSTEP_STEP_PLAIN force one
                              (TMA falls back to plain loads where the shape does not allow it).
                              Both give the same basis bit for bit; with FUSED the moments'
                              per-block partial sums follow each kernel's blocks, so the solves
                              agree to FP32 rounding. Elsewhere: unused */
} sstep_cg_opts;

typedef struct {
    int outer_iters;           /* outer iterations applied (Gram solves that updated x) */
    int refreshes;             /* true-residual restarts taken */
    int status;                /* sstep_status of the solve */
    double r0_norm;            /* ||b - A x_0|| */
    double rel_res_recursive;  /* ||r_k|| / ||r_0|| of the recursively updated residual */
    double rel_res_true;       /* ||b - A x|| / ||r_0|| recomputed at exit */
    double lambda_min_used;    /* spectral bounds used by the basis */
    double lambda_max_used;
    double min_gii;            /* smallest Gram diagonal seen (breakdown diagnostic) */
    double delta_last;         /* ||c~ - G~ a|| / ||c~|| of the last Gram solve (Section 7) */
    float ms;                  /* device time of the solve (CUDA events on the stream) */
    int kernel_launches;       /* kernels of this library launched by the solve */
    float prof_ms[4];          /* profile_every > 0: summed device time of the sampled launches of
                                  [0] Chebyshev steps, [1] Gram + FGS, [2] update, [3] residual */
    int prof_launches[4];      /* number of sampled launches behind each prof_ms entry */
    int step_tma;              /* 1: the FP32 Chebyshev steps read their planes through tensor-map
                                  (TMA) tiles (opts.step_kernel), 0: plain loads */
} sstep_cg_info;

/* Fills *opts with the defaults listed above (s = 8, nu = 25, tol = 1e-8, Jacobi, FGS,
 * FP64, bounds GERSH_LANCZOS10, direct Gram, graph off, check_every 8). */
SSTEP_API void sstep_cg_default_opts(sstep_cg_opts* opts);

/* Handle over a CSR matrix (Section 2: A SPD and sparse). rowptr_d: int32[n+1],
 * colind_d: int32[nnz], vals_d: double[nnz], nnz = rowptr[n] < 2^31, row-major, any column
 * order. A must be symmetric positive definite with a positive diagonal (not checked beyond
 * the diagonal sign). Computes M^-1, the spectral bounds (bounds_mode) and allocates the
 * basis workspace ((s+1) vectors, plus an FP32 copy of vals in MIXED precision).
 * Synchronises `stream`. */
SSTEP_API sstep_status sstep_cg_create_csr(sstep_cg_t* handle, int64_t n, const int32_t* rowptr_d,
                                 const int32_t* colind_d, const double* vals_d,
                                 const sstep_cg_opts* opts, void* stream);

/* Matrix-free handle over a structured grid with homogeneous Dirichlet boundaries: the
 * synthetic Poisson problems of Section 8 (its 27-point stencil is sstep_cg_create_box_stencil)
 * and a diffusion operator the paper does not discretise (the reading below).
 * dim = 2 (nz must be 1) or 3. kappa_d = NULL: the unscaled Poisson stencil, diagonal 2*dim
 * and -1 per in-grid neighbour (5- or 7-point). kappa_d = double[n] > 0: cell-centred
 * diffusion -div(kappa grad u); an interior face between cells a, b has weight
 * 2 ka kb / (ka + kb), a boundary face adds 2 kappa_cell to the diagonal. Grid extents:
 * nx, ny, nz >= 1, ny <= 524280 and, in 3D, nz <= 524280; anything else gives
 * SSTEP_ERR_INVALID_ARG before any CUDA call. Synchronises `stream`. */
SSTEP_API sstep_status sstep_cg_create_stencil(sstep_cg_t* handle, int dim, int nx, int ny, int nz,
                                     const double* kappa_d, const sstep_cg_opts* opts,
                                     void* stream);

/* Matrix-free handle over the box-stencil Poisson operator on a structured grid with
 * homogeneous Dirichlet boundaries: every grid point of the unit box around a point (3^dim - 1
 * of them: faces, edges and corners) is a neighbour with weight -1 and the diagonal is
 * 3^dim - 1. In 3D this is the 27-point finite-difference Laplacian of the experiments in
 * Section 8 (unscaled: the h^-2 factor changes neither the Jacobi-preconditioned iteration
 * nor the relative residual); in 2D the 9-point one. dim = 2 (nz must be 1) or 3. M = D is
 * the constant 3^dim - 1, so the moments Gram form applies. The Gershgorin bound of D^-1 A
 * is 2, well above the spectrum's end near 36/26 in 3D; the paper's Lanczos-10 bounds
 * (bounds_mode LANCZOS10) are tighter. Grid extents: nx, ny, nz >= 1, ny <= 524280 and, in
 * 3D, nz <= 1048560; anything else gives SSTEP_ERR_INVALID_ARG before any CUDA call.
 * Synchronises `stream`. */
SSTEP_API sstep_status sstep_cg_create_box_stencil(sstep_cg_t* handle, int dim, int nx, int ny, int nz,
                                                   const sstep_cg_opts* opts, void* stream);

/* Solves A x = b by the s-step CG outer iteration of Section 2 (Chebyshev basis, Gram system,
 * column scaling, nu FGS sweeps, update of x and r), stopped by the rule of Section 8 on the
 * relative residual (the recursive one, with the true residual b - A x checked at exit).
 * b_d, x_d: device double[n], 16-byte aligned, caller-owned (in: x_0, out: x); info (host)
 * may be NULL. Synchronises the handle's stream (it reads the convergence state). Returns
 * SSTEP_OK when ||b - A x|| / ||b - A x_0|| < tol, SSTEP_ERR_NO_CONVERGENCE when max_outer
 * outers or max_refresh restarts did not get there (x holds the last iterate),
 * SSTEP_ERR_NUMERICAL when the Gram system breaks down (every column dropped, a non-finite
 * entry), SSTEP_ERR_TIMEOUT when a bounded device-side wait expired, SSTEP_ERR_INVALID_ARG for
 * a null or misaligned pointer. */
SSTEP_API sstep_status sstep_cg_solve(sstep_cg_t handle, const double* b_d, double* x_d, sstep_cg_info* info);

/* The solve of sstep_cg_solve (Section 2) with HOST arrays b_h, x_h (double[n], pinned or
 * pageable, caller-owned): copies b and x_0 to device buffers the handle owns (allocated on
 * the first call), solves, copies x back; info.ms includes the copies. Same statuses; x_h is
 * written unless the solve failed with a CUDA, memory or timeout error. Synchronises. */
SSTEP_API sstep_status sstep_cg_solve_host(sstep_cg_t handle, const double* b_h, double* x_h, sstep_cg_info* info);

/* Differentiable solve (adjoint): for a diffusion stencil handle (created with kappa_d) and a
 * loss L(x) with x = A(kappa)^-1 b, given x_d and the adjoint solution lambda_d of
 * A lambda = dL/dx (A is symmetric, so the same handle's sstep_cg_solve gives it), writes
 *   gkappa_d[c] = dL/dkappa_c = -lambda^T (dA/dkappa_c) x
 *              = -sum_{faces (c,o)} 2 ko^2/(kc+ko)^2 (lambda_c-lambda_o)(x_c-x_o) - 2 nbf_c lambda_c x_c
 * (nbf_c: boundary faces of cell c). dL/db = lambda. All arrays double[n] on the device.
 * The paper has no adjoint; this is the gradient of the solve it describes (Section 2).
 * SSTEP_ERR_INVALID_ARG for a CSR or Poisson handle. */
SSTEP_API sstep_status sstep_cg_grad_kappa(sstep_cg_t handle, const double* x_d, const double* lambda_d,
                                           double* gkappa_d);

/* Per-outer-iteration record of the last solve, oldest first (opts.history > 0): out_h (host,
 * double[4 * capacity]) receives up to `capacity` records of 4 values each: the outer
 * iteration's number (1-based), ||r_(k-1)||^2 / ||r_0||^2 of the residual it started from (the
 * recursive residual; the mixed form's FP64 refresh where one ran), the inexactness
 * delta_k = ||c~ - G~ a|| / ||c~|| of its Gram solve (Section 7's inexact s-step CG) and its
 * smallest Gram diagonal G_ii before scaling. *count = the number of records written (at most
 * min(outer iterations, opts.history, capacity)). SSTEP_ERR_INVALID_ARG when the handle keeps
 * no history. Synchronises the handle's stream. */
SSTEP_API sstep_status sstep_cg_history(sstep_cg_t handle, double* out_h, int capacity, int* count);

/* Changes the tolerance of Section 8's stopping rule and the outer-iteration limit of an
 * existing handle (for example a looser tolerance for an adjoint solve that reuses the
 * forward handle). SSTEP_ERR_INVALID_ARG unless tol > 0 is finite and max_outer >= 0. */
SSTEP_API sstep_status sstep_cg_set_tolerance(sstep_cg_t handle, double tol, int max_outer);

/* Releases the handle and everything it owns (synchronises its stream). NULL is a no-op. */
SSTEP_API sstep_status sstep_cg_destroy(sstep_cg_t handle);

/* Static description of a status code. */
SSTEP_API const char* sstep_cg_status_string(sstep_status status);

/* Text of the last error recorded on the handle ("" if none). */
SSTEP_API const char* sstep_cg_last_error(sstep_cg_t handle);

/* --- operator and pipeline pieces (the solve is composed of these kernels) ----------- */

/* y_d = A x_d with the handle's operator, the A of Section 2's system (device double[n]
 * each, caller-owned). Asynchronous on the handle's stream. */
SSTEP_API sstep_status sstep_cg_apply(sstep_cg_t handle, const double* x_d, double* y_d);

/* Chebyshev basis of Section 2 (Definition): column j of P_d (leading dimension ldp >= n,
 * column-major, double[ldp * ncols]) receives p_j for j = 0 .. ncols-1, p_0 = r_d,
 * with the handle's theta, sigma and M. 1 <= ncols <= SSTEP_MAX_S + 1. */
SSTEP_API sstep_status sstep_cg_basis(sstep_cg_t handle, const double* r_d, double* P_d, int64_t ldp, int ncols);

/* One Gram reduction and Gram solve on the handle's current basis and residual, as in the
 * solve (Section 2): writes to out_h (host, double[3 * s + s * s]) the vector
 * alpha = S a (s), the scaling d (s), c~ = S P^T r (s), and G~ = S G S (s*s, row-major).
 * Run after sstep_cg_load_basis. Synchronises. */
SSTEP_API sstep_status sstep_cg_gram_solve(sstep_cg_t handle, double* out_h);

/* Copies a caller basis P_d (the P_+ = [p_0 .. p_s] of Section 2: device doubles, n x (s+1),
 * column-major, leading dimension ldp >= n; column 0 = r) into the handle's basis workspace,
 * for sstep_cg_gram_solve. SSTEP_ERR_INVALID_ARG for a null pointer or ldp < n. */
SSTEP_API sstep_status sstep_cg_load_basis(sstep_cg_t handle, const double* P_d, int64_t ldp);

/* Spectral bounds the handle uses (given, or Section 8's Gershgorin / Lanczos estimates,
 * computed at create): lambda_min, lambda_max (host doubles). */
SSTEP_API sstep_status sstep_cg_get_bounds(sstep_cg_t handle, double* lambda_min, double* lambda_max);

/* Writes the handle's current residual r_k of Section 2 (column 0 of the basis workspace) to
 * r_d (device double[n]). Asynchronous on the handle's stream. */
SSTEP_API sstep_status sstep_cg_get_residual(sstep_cg_t handle, double* r_d);

/* Lanczos tridiagonal of Section 8's estimate: k steps on D^-1/2 A D^-1/2 from the seeded
 * start vector; writes alpha (k) and beta (k-1) to host arrays. Synchronises. */
SSTEP_API sstep_status sstep_cg_lanczos(sstep_cg_t handle, int k, uint64_t seed, double* alpha_h, double* beta_h,
                              int* steps_done);

/* The two conversions of the mixed form (FP32 basis, FP64 Gram and x; the paper has no mixed
 * form), exposed for testing: out_d[i] = float(in_d[i] * 2^k)
 * rounded to nearest even, computed from the IEEE-754 fields with integer instructions, and
 * back_d[i] = double(out_d[i]), exact. Device arrays of n elements; asynchronous on stream. */
SSTEP_API sstep_status sstep_convert_check(const double* in_d, int k, float* out_d, double* back_d, int64_t n,
                                           void* stream);

/* --- AMG coarse-grid FGS ----------------------------------------------------------------- */

enum { SSTEP_COARSE_FORMED = 0, SSTEP_COARSE_STREAMING = 1 };

/* FGS as the AMG coarse-grid solver (Section 6, "AMG Coarse-Grid Extension") on the handle's
 * matrix-free stencil operator A_f (sstep_cg_create_stencil or sstep_cg_create_box_stencil;
 * CSR handles give SSTEP_ERR_UNSUPPORTED). The prolongation P aggregates bx x by x bz boxes of
 * the grid (the last box along an axis may be smaller): column i of P is the indicator of
 * aggregate i, ids x fastest over the ceil(nx/bx) x ceil(ny/by) x ceil(nz/bz) coarse grid
 * (bz must be 1 in 2D). Runs nu forward Gauss-Seidel sweeps on A_c y = g with A_c = P^T A_f P,
 * rows in increasing order, D = diag(A_c), starting from y_d: y_i += (g_i - (A_c y)_i) /
 * (A_c)_ii.
 *   mode SSTEP_COARSE_FORMED: A_c is assembled as a dense n_c x n_c matrix (n_c <= 16384;
 *     n_c^2 doubles allocated for the call) and swept;
 *   mode SSTEP_COARSE_STREAMING: A_c is never formed (Section 6's streaming form): P y is kept
 *     on the fine grid and row i of A_c y is the sum of A_f (P y) over aggregate i; memory
 *     O(n_f + n_c), n_c < 2^31.
 * g_d (double[n_c]) and y_d (double[n_c], in: y^(0), out: y^(nu)) are device arrays; the
 * handle's residual scratch is used. Synchronises the handle's stream. */
SSTEP_API sstep_status sstep_coarse_fgs(sstep_cg_t handle, int bx, int by, int bz, const double* g_d, double* y_d,
                                        int nu, int mode);

/* --- batched form -------------------------------------------------------------------- */

typedef struct sstep_cg_batch_s* sstep_cg_batch_t;

/* `count` independent stencil systems solved together (the batched form of the method of
 * Section 2): every phase of an outer iteration (s Chebyshev steps, the Gram reduction with
 * each system's column scaling and FGS, the update) is ONE launch over all systems that are
 * still iterating; a system that has converged drops out of every later launch. With
 * opts->use_graph the outer loop is one CUDA graph whose while node runs until no system is
 * left. grids_h: host int[4 * count], (dim, nx, ny, nz) per system as in
 * sstep_cg_create_stencil. kappa_d: NULL (all Poisson) or a host array of count device
 * pointers, each NULL (Poisson) or double[n_i] (diffusion). Per-system spectral bounds
 * follow opts->bounds_mode (GIVEN: the same bounds for all). Jacobi, FP64, s <= 16; the
 * Gram in either opts->gram_form (DIRECT or MOMENTS). Other options give SSTEP_ERR_UNSUPPORTED.
 * Vectors of all systems are concatenated: system i occupies [offset_i, offset_i + n_i) of
 * b and x (sstep_cg_batch_layout). Synchronises `stream`. */
SSTEP_API sstep_status sstep_cg_batch_create(sstep_cg_batch_t* batch, int count, const int* grids_h,
                                             const double* const* kappa_d, const sstep_cg_opts* opts, void* stream);

/* Layout of the batched form (not in the paper; the per-system solve is Section 2's):
 * offsets_h (host int64[count], may be NULL): start of each system in the concatenated
 * vectors; total: their length; lambda_h (host double[2*count], may be NULL): the bounds. */
SSTEP_API sstep_status sstep_cg_batch_layout(sstep_cg_batch_t batch, int64_t* offsets_h, int64_t* total,
                                             double* lambda_h);

/* Solves all systems by Section 2's outer iteration, each with its own Gram system and
 * Section 8's stopping rule, from x_0 = x_d (concatenated, device, caller-owned; b_d alike).
 * infos_h (host, count entries, may be NULL) receives each system's result; summary (may be
 * NULL) the largest outer count, the worst true relative residual and the device time.
 * Returns SSTEP_OK when every system reached tol, else the first failing status. Synchronises. */
SSTEP_API sstep_status sstep_cg_batch_solve(sstep_cg_batch_t batch, const double* b_d, double* x_d,
                                            sstep_cg_info* infos_h, sstep_cg_info* summary);

/* Releases the batch and everything it owns (synchronises its stream). NULL is a no-op. */
SSTEP_API sstep_status sstep_cg_batch_destroy(sstep_cg_batch_t batch);

/* Text of the last error recorded on the batch; with batch = NULL, the reason of the last
 * failed create (as sstep_cg_last_error(NULL); "" if none). */
SSTEP_API const char* sstep_cg_batch_last_error(sstep_cg_batch_t batch);

/* --- allocation-free variant ---------------------------------------------------------- */

/* The Gram reduction, column scaling and FGS (or Cholesky) solve of one outer iteration
 * (Section 2's Gram system and scaling, Section 3's sweeps) - the same kernel and results as
 * sstep_cg_gram_solve - for callers that cannot allocate
 * device memory, e.g. because a caching allocator already owns the device's memory or
 * because cudaMalloc/cudaFree would synchronise the device inside a latency-bound loop. It
 * needs no handle and allocates nothing: its scratch (per-block partial sums and a control
 * block, about 224 KB) is a static array inside the library, which every GPU that loads the
 * library holds until the process exits. The paper has no counterpart; it is a calling
 * convention of this library.
 *
 * Inputs: P_d, the basis [p_0 .. p_s] (column-major double, leading dimension ldp >= n,
 * p_0 = r_k, built as in sstep_cg_basis); mdiag_d, the diagonal of the preconditioner M
 * (double[n]) or NULL for M = mconst * I (mconst > 0); lambda_min < lambda_max, the bounds the
 * basis was built with; nu sweeps; gram_solver SSTEP_GRAM_SOLVE_FGS or _CHOLESKY.
 * Output out_d (device, double[3s + s*s + 1]): alpha = S a (s), d (s), c~ (s), G~ (s*s,
 * row-major), then the termination state (0 = solved, 3 = numerical breakdown: the other
 * entries are then NaN).
 * Limit: 1 <= s <= 16 (SSTEP_ERR_INVALID_ARG beyond, with the reason in
 * sstep_cg_last_error(NULL)). Asynchronous on `stream`.
 * The device address of the static scratch is looked up (cudaGetSymbolAddress with the device
 * current) on the first call on a device and on every call whose stream is not capturing, as
 * a device reset (cudaDeviceReset) moves it; a call during stream capture reuses the address
 * of the device's last call outside capture. So make a first call on each device before any
 * stream capture, and again after a device reset (a first call during capture gives
 * SSTEP_ERR_INVALID_ARG).
 * All calls on a device share the scratch and it keeps the last call's contents (each call
 * re-initialises what must start at zero): calls whose work can overlap on the GPU, such as
 * calls on two streams, race - serialise them. */
SSTEP_API sstep_status sstep_gram_fgs_noalloc(int64_t n, int s, int nu, int gram_solver, const double* P_d,
                                              int64_t ldp, const double* mdiag_d, double mconst,
                                              double lambda_min, double lambda_max, double* out_d, void* stream);

/* Self-test of the bounded device-side waits of the mixed form's TMA step (the path
 * opts.step_kernel selects): runs that kernel once on a 64 x 8 x 4 grid of its own whose
 * shared-memory stages expect 16 bytes more than their tensor-map copies deliver, so that no
 * wait completes, with a limit of 4096 polls per wait. *done_state (host) receives the
 * control block's termination state afterwards: 4 (timed out) is the designed outcome, and
 * the CUDA context stays usable. Returns SSTEP_ERR_UNSUPPORTED when the driver has no
 * tensor-map encoder, SSTEP_ERR_CUDA when a CUDA call failed, SSTEP_ERR_INVALID_ARG for a
 * null pointer. Allocates and frees its own 8 KB and control block on the current device
 * (synchronous). */
SSTEP_API sstep_status sstep_selftest_tma_timeout(int* done_state);

#ifdef __cplusplus
}
#endif
#endif /* SSTEP_CG_H */
