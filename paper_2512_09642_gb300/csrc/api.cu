// C ABI of the s-step CG library: handle life cycle, validation, spectral bounds, and the
// host driver of the outer iteration (Section 2 of arXiv 2512.09642; stopping rule and
// Lanczos estimate of Section 8). Everything numeric runs in the kernels of k_*.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.h"

using namespace sstep;

struct sstep_cg_s {
    OpDesc op{};
    sstep_cg_opts opts{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 152;
    double lmin = 0, lmax = 0, theta = 0, sigma = 0;
    bool jacobi = true;
    // owned device memory
    double* diag = nullptr;     // diag(A) (CSR, diffusion)
    double* cdinv = nullptr;    // 2 theta / diag (Jacobi)
    double* faces = nullptr;    // wx | wy | wz (diffusion)
    const double* kappa = nullptr;   // borrowed per-cell coefficient (diffusion stencil)
    double* P = nullptr;        // basis P_+ = [p_0 .. p_s], column-major, leading dimension ld
    int64_t ld = 0;
    bool mixed = false;         // FP32 basis (form 1)
    float* P32 = nullptr;       // mixed form: FP32 basis, same layout as P
    bool tma = false;           // mixed form: FP32 steps through tensor-map tiles (step_kernel)
    std::vector<CUtensorMap> tmaps;   // per FP32 column j: [2j] read as p, [2j + 1] read as q
    float* ops32 = nullptr;     // mixed form: FP32 copies of the operator arrays
    double* rtrue = nullptr;    // true residual b - A x
    double* gram_partials = nullptr;
    int gram_nblk = 0;
    bool fused = false;         // gram_form FUSED: moments reduced by the step kernels
    void* mom_part = nullptr;   // their per-block partials, s steps x 16 bytes x mom_nblk
    int mom_nblk = 0;
    double* mom_part2 = nullptr;   // the finish kernel's per-block sums
    double* hist = nullptr;     // per-outer records (opts.history > 0)
    double* res_partials = nullptr;
    bool conj = false;          // block-conjugated form: P holds P_+, Q_(k-1), A Q_(k-1)
    double* conj_partials = nullptr;
    int conj_nblk = 0;
    double* cj = nullptr;       // [W_(k-1) | B_k], s x s each
    Ctl* ctl = nullptr;
    Ctl* ctl_h = nullptr;       // pinned mirror
    double* bx_dev = nullptr;   // device b, x for sstep_cg_solve_host
    // graph mode: one while-node graph per (b, x) pair, captured on cap_stream
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const double* g_b = nullptr;
    double* g_x = nullptr;
    cudaEvent_t ev[SSTEP_MAX_S + 4] = {};   // profiling: boundaries of one outer iteration
    cudaEvent_t rev[2] = {};                // profiling: residual kernel
    char err[512] = {0};
};

namespace {

void set_err(sstep_cg_t h, const char* fmt, ...) {
    if (!h) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            set_err(h, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? SSTEP_ERR_OOM : SSTEP_ERR_CUDA;            \
        }                                                                                      \
    } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

sstep_status validate_opts(sstep_cg_t h, const sstep_cg_opts* o) {
    if (o->s < 1 || o->s > SSTEP_MAX_S) { set_err(h, "s = %d outside [1, %d]", o->s, SSTEP_MAX_S); return SSTEP_ERR_INVALID_ARG; }
    if (o->nu < 1 || o->nu > 10000) { set_err(h, "nu = %d outside [1, 10000]", o->nu); return SSTEP_ERR_INVALID_ARG; }
    if (!(o->tol > 0.0) || !std::isfinite(o->tol)) { set_err(h, "tol must be positive"); return SSTEP_ERR_INVALID_ARG; }
    if (o->max_outer < 0) { set_err(h, "max_outer < 0"); return SSTEP_ERR_INVALID_ARG; }
    if (o->max_refresh < 0) { set_err(h, "max_refresh < 0"); return SSTEP_ERR_INVALID_ARG; }
    if (o->bounds_mode == SSTEP_BOUNDS_GIVEN) {
        if (!(o->lambda_min >= 0.0) || !(o->lambda_max > o->lambda_min) || !std::isfinite(o->lambda_max)) {
            set_err(h, "need 0 <= lambda_min < lambda_max (got %g, %g)", o->lambda_min, o->lambda_max);
            return SSTEP_ERR_INVALID_ARG;
        }
    } else if (o->bounds_mode != SSTEP_BOUNDS_GERSH_LANCZOS10 && o->bounds_mode != SSTEP_BOUNDS_LANCZOS10) {
        set_err(h, "unknown bounds_mode %d", o->bounds_mode);
        return SSTEP_ERR_INVALID_ARG;
    }
    if (o->gram_solver != SSTEP_GRAM_SOLVE_FGS && o->gram_solver != SSTEP_GRAM_SOLVE_CHOLESKY) {
        set_err(h, "unknown gram_solver %d", o->gram_solver);
        return SSTEP_ERR_INVALID_ARG;
    }
    if (o->precond != SSTEP_PRECOND_JACOBI && o->precond != SSTEP_PRECOND_NONE) {
        set_err(h, "unknown precond %d", o->precond);
        return SSTEP_ERR_INVALID_ARG;
    }
    if (o->basis_start != SSTEP_START_R) { set_err(h, "basis_start %d not supported", o->basis_start); return SSTEP_ERR_UNSUPPORTED; }
    if (o->precision != SSTEP_PRECISION_FP64 && o->precision != SSTEP_PRECISION_MIXED) {
        set_err(h, "unknown precision %d", o->precision);
        return SSTEP_ERR_INVALID_ARG;
    }
    if (o->refresh_period < 1) { set_err(h, "refresh_period < 1"); return SSTEP_ERR_INVALID_ARG; }
    if (o->block_conjugate != 0 && o->block_conjugate != 1) {
        set_err(h, "block_conjugate must be 0 or 1");
        return SSTEP_ERR_INVALID_ARG;
    }
    if (o->block_conjugate && (o->precision != SSTEP_PRECISION_FP64 || o->s > 16)) {
        set_err(h, "block_conjugate needs FP64 and s <= 16");
        return SSTEP_ERR_UNSUPPORTED;
    }
    if (o->refresh_period > 1000000) { set_err(h, "refresh_period > 10^6"); return SSTEP_ERR_INVALID_ARG; }
    if (o->gram_form != SSTEP_GRAM_FORM_DIRECT && o->gram_form != SSTEP_GRAM_FORM_MOMENTS &&
        o->gram_form != SSTEP_GRAM_FORM_FUSED) {
        set_err(h, "unknown gram_form %d", o->gram_form);
        return SSTEP_ERR_INVALID_ARG;
    }
    if (o->gram_form == SSTEP_GRAM_FORM_FUSED && o->block_conjugate) {
        set_err(h, "gram_form FUSED does not combine with block_conjugate");
        return SSTEP_ERR_UNSUPPORTED;
    }

    if (o->check_every < 1) { set_err(h, "check_every < 1"); return SSTEP_ERR_INVALID_ARG; }
    if (o->profile_every < 0) { set_err(h, "profile_every < 0"); return SSTEP_ERR_INVALID_ARG; }
    if (o->history < 0 || o->history > (1 << 20)) { set_err(h, "history outside [0, 2^20]"); return SSTEP_ERR_INVALID_ARG; }
    if (o->step_kernel < SSTEP_STEP_AUTO || o->step_kernel > SSTEP_STEP_PLAIN) {
        set_err(h, "step_kernel must be SSTEP_STEP_AUTO, _TMA or _PLAIN");
        return SSTEP_ERR_INVALID_ARG;
    }
    return SSTEP_OK;
}

// Eigenvalues (ascending) of the symmetric tridiagonal (a, b) by Sturm-count bisection.
std::vector<double> tridiag_eigs(const std::vector<double>& a, const std::vector<double>& b) {
    const int m = (int)a.size();
    std::vector<double> out;
    if (m == 0) return out;
    double lo0 = a[0], hi0 = a[0];
    for (int i = 0; i < m; ++i) {
        double r = 0.0;
        if (i > 0) r += std::fabs(b[i - 1]);
        if (i < m - 1) r += std::fabs(b[i]);
        lo0 = std::fmin(lo0, a[i] - r);
        hi0 = std::fmax(hi0, a[i] + r);
    }
    auto count_below = [&](double x) {
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < m; ++i) {
            q = a[i] - x - (i > 0 ? b[i - 1] * b[i - 1] / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++c;
        }
        return c;
    };
    for (int k = 0; k < m; ++k) {
        double lo = lo0, hi = hi0;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (count_below(mid) > k) hi = mid; else lo = mid;
        }
        out.push_back(0.5 * (lo + hi));
    }
    return out;
}

sstep_status host_dot(sstep_cg_t h, const double* a, const double* b, double* partials, int nblk, double* out) {
    CK(launch_dot(a, b, h->op.n, partials, nblk, h->stream));
    std::vector<double> hp(nblk);
    CK(cudaMemcpyAsync(hp.data(), partials, sizeof(double) * nblk, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double s = 0.0;
    for (int i = 0; i < nblk; ++i) s += hp[i];
    *out = s;
    return SSTEP_OK;
}

int setup_nblk(int64_t n) {
    const int64_t b = (n + 255) / 256;
    const int64_t cap = 8 * (int64_t)device_sm_count();
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// k Lanczos steps on B = M^-1/2 A M^-1/2 (Section 8), start vector splitmix64(seed) U(-1,1).
sstep_status lanczos(sstep_cg_t h, int k, uint64_t seed, std::vector<double>& al, std::vector<double>& be) {
    const int64_t n = h->op.n;
    double *q = nullptr, *qp = nullptr, *w = nullptr, *dh = nullptr, *parts = nullptr;
    const int nblk = setup_nblk(n);
    sstep_status st = SSTEP_OK;
    // w holds 2n doubles: the product and the scratch of launch_lanczos_apply
    auto cleanup = [&]() {
        cudaFree(q); cudaFree(qp); cudaFree(w); cudaFree(dh); cudaFree(parts);
    };
    if (cudaMalloc(&q, sizeof(double) * n) != cudaSuccess || cudaMalloc(&qp, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&w, sizeof(double) * 2 * n) != cudaSuccess || cudaMalloc(&parts, sizeof(double) * nblk) != cudaSuccess) {
        cleanup();
        set_err(h, "Lanczos workspace allocation failed");
        return SSTEP_ERR_OOM;
    }
    double dhc = 1.0;   // M^-1/2 when M is a multiple of I
    if (h->jacobi) {
        if (h->diag) {
            if (cudaMalloc(&dh, sizeof(double) * n) != cudaSuccess) { cleanup(); return SSTEP_ERR_OOM; }
            if (launch_rsqrt_vec(h->diag, dh, n, h->stream) != cudaSuccess) { cleanup(); return SSTEP_ERR_CUDA; }
        } else {
            dhc = 1.0 / std::sqrt(h->op.dconst);
        }
    }
    auto fail = [&](const char* what) { cleanup(); set_err(h, "Lanczos: %s", what); return SSTEP_ERR_CUDA; };
    if (launch_splitmix_uniform(seed, q, n, h->stream) != cudaSuccess) return fail("start vector");
    double nrm2 = 0.0;
    if ((st = host_dot(h, q, q, parts, nblk, &nrm2)) != SSTEP_OK) { cleanup(); return st; }
    if (!(nrm2 > 0.0)) { cleanup(); set_err(h, "zero Lanczos start vector"); return SSTEP_ERR_NUMERICAL; }
    if (launch_axpby(0.0, q, 1.0 / std::sqrt(nrm2), q, n, h->stream) != cudaSuccess) return fail("normalise");
    if (cudaMemsetAsync(qp, 0, sizeof(double) * n, h->stream) != cudaSuccess) return fail("memset");
    double beta_prev = 0.0;
    al.clear();
    be.clear();
    for (int j = 0; j < k; ++j) {
        if (launch_lanczos_apply(h->op, dh, dhc, q, w, h->stream) != cudaSuccess) return fail("apply");
        if (launch_axpby(-beta_prev, qp, 1.0, w, n, h->stream) != cudaSuccess) return fail("axpby");
        double a = 0.0;
        if ((st = host_dot(h, q, w, parts, nblk, &a)) != SSTEP_OK) { cleanup(); return st; }
        if (launch_axpby(-a, q, 1.0, w, n, h->stream) != cudaSuccess) return fail("axpby");
        al.push_back(a);
        double b2 = 0.0;
        if ((st = host_dot(h, w, w, parts, nblk, &b2)) != SSTEP_OK) { cleanup(); return st; }
        const double b = std::sqrt(b2);
        if (j == k - 1 || b == 0.0) break;
        be.push_back(b);
        // qp <- q ; q <- w / b
        if (launch_copy_f64(q, qp, n, h->stream) != cudaSuccess) return fail("copy");
        if (launch_axpby(1.0 / b, w, 0.0, q, n, h->stream) != cudaSuccess) return fail("scale");
        beta_prev = b;
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail("sync");
    cleanup();
    return SSTEP_OK;
}

sstep_status gershgorin(sstep_cg_t h, double* out) {
    if (h->op.kind == OP_STENCIL && h->op.box) {
        // box stencil: row sum of |a_ij| = (3^dim - 1) + (in-grid box neighbours), maximal in
        // the interior, where every extent contributes min(3, n_axis) points
        const int D = h->op.dim == 3 ? 26 : 8;
        int pts = (h->op.nx < 3 ? h->op.nx : 3) * (h->op.ny < 3 ? h->op.ny : 3);
        if (h->op.dim == 3) pts *= (h->op.nz < 3 ? h->op.nz : 3);
        *out = h->jacobi ? (double)(D + pts - 1) / D : (double)(D + pts - 1);
        return SSTEP_OK;
    }
    if (h->op.kind == OP_STENCIL && h->op.wx == nullptr) {
        // Poisson: row sum of |a_ij| = 2 dim + (in-grid neighbours); maximal in the interior
        const int d2 = 2 * h->op.dim;
        int nbr = (h->op.nx > 2 ? 2 : h->op.nx - 1) + (h->op.ny > 2 ? 2 : h->op.ny - 1);
        if (h->op.dim == 3) nbr += (h->op.nz > 2 ? 2 : h->op.nz - 1);
        *out = h->jacobi ? (double)(d2 + nbr) / d2 : (double)(d2 + nbr);
        return SSTEP_OK;
    }
    const int nblk = setup_nblk(h->op.n);
    double* bm = nullptr;
    CK(cudaMalloc(&bm, sizeof(double) * nblk));
    cudaError_t e = launch_gershgorin(h->op, h->jacobi, bm, nblk, h->stream);
    std::vector<double> hb(nblk);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), bm, sizeof(double) * nblk, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(bm);
    if (e != cudaSuccess) { set_err(h, "Gershgorin: %s", cudaGetErrorString(e)); return SSTEP_ERR_CUDA; }
    double m = 0.0;
    for (double v : hb) m = std::fmax(m, v);
    *out = m;
    return SSTEP_OK;
}

sstep_status compute_bounds(sstep_cg_t h) {
    const sstep_cg_opts& o = h->opts;
    if (o.bounds_mode == SSTEP_BOUNDS_GIVEN) {
        h->lmin = o.lambda_min;
        h->lmax = o.lambda_max;
        return SSTEP_OK;
    }
    std::vector<double> al, be;
    sstep_status st = lanczos(h, 10, o.seed, al, be);
    if (st != SSTEP_OK) return st;
    std::vector<double> ev = tridiag_eigs(al, be);
    const double tmin = ev.front(), tmax = ev.back();
    h->lmin = 0.9 * tmin;
    if (o.bounds_mode == SSTEP_BOUNDS_LANCZOS10) {
        h->lmax = 1.1 * tmax;
    } else {
        double g = 0.0;
        if ((st = gershgorin(h, &g)) != SSTEP_OK) return st;
        h->lmax = g;
    }
    if (!(h->lmax > h->lmin) || !(h->lmin >= 0.0)) {
        set_err(h, "estimated bounds unusable: [%g, %g]", h->lmin, h->lmax);
        return SSTEP_ERR_NUMERICAL;
    }
    return SSTEP_OK;
}

}  // namespace

namespace sstep {
// Spectral bounds of one operator as a handle would compute them (used by the batched form):
// runs the same Lanczos / Gershgorin code on a temporary, workspace-free handle.
sstep_status estimate_bounds(const OpDesc& op, const double* diag, bool jacobi, const sstep_cg_opts& opts,
                             cudaStream_t stream, double* lmin, double* lmax, char* err, size_t errlen) {
    sstep_cg_s tmp;
    tmp.op = op;
    tmp.opts = opts;
    tmp.stream = stream;
    tmp.jacobi = jacobi;
    tmp.diag = const_cast<double*>(diag);
    sstep_status st = compute_bounds(&tmp);
    tmp.diag = nullptr;   // borrowed
    *lmin = tmp.lmin;
    *lmax = tmp.lmax;
    if (st != SSTEP_OK && err) std::snprintf(err, errlen, "%s", tmp.err);
    return st;
}
}  // namespace sstep

namespace {

GramArgs gram_args(sstep_cg_t h) {
    GramArgs g{};
    g.s = h->opts.s;
    g.nu = h->opts.nu;
    g.solver = h->opts.gram_solver;
    // the fused form's moments come from the step kernels; a Gram pass over a given basis
    // (sstep_cg_gram_solve) forms the same moments itself
    g.form = h->opts.gram_form == SSTEP_GRAM_FORM_FUSED ? SSTEP_GRAM_FORM_MOMENTS : h->opts.gram_form;
    g.check = h->mixed ? 0 : 1;
    g.theta = h->theta;
    g.sigma = h->sigma;
    g.dvec = h->jacobi && h->diag != nullptr;
    g.dconst = h->jacobi ? h->op.dconst : 1.0;
    g.diag = h->diag;
    g.n = h->op.n;
    g.ld = h->ld;
    g.P = h->mixed ? (const void*)h->P32 : (const void*)h->P;
    g.diag32 = h->op.diag32;
    g.fp32 = h->mixed;
    return g;
}

// The same, with the block-conjugated form's inputs and the record ring (used by the outer
// iteration only).
GramArgs gram_args_outer(sstep_cg_t h) {
    GramArgs g = gram_args(h);
    g.hist = h->hist;
    g.hist_cap = h->opts.history;
    if (h->conj) {
        g.conj = 1;
        g.conj_nblk = h->conj_nblk;
        g.conj_partials = h->conj_partials;
        g.cj = h->cj;
    }
    return g;
}

// FP32 copies of the operator for the mixed form's basis (rounded to nearest).
sstep_status make_f32_operator(sstep_cg_t h) {
    const int64_t n = h->op.n;
    int64_t nnz = 0;
    if (h->op.kind == OP_CSR) {
        int32_t last = 0;
        CK(cudaMemcpyAsync(&last, h->op.rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        nnz = last;
    }
    const bool faces = h->op.kind == OP_STENCIL && h->faces;
    // every array starts on a 128-byte boundary (the FP32 Gram reads diag32 in 8-byte pairs)
    auto pad = [](int64_t m) { return (m + 31) / 32 * 32; };
    const int64_t total = pad(nnz) + (faces ? 3 * pad(n) : 0) + (h->diag ? pad(n) : 0) + (h->cdinv ? pad(n) : 0);
    if (total == 0) return SSTEP_OK;
    CK(cudaMalloc(&h->ops32, sizeof(float) * total));
    float* q = h->ops32;
    if (nnz) { CK(launch_to_f32(h->op.vals, q, nnz, h->stream)); h->op.vals32 = q; q += pad(nnz); }
    if (faces) {
        for (int f = 0; f < 3; ++f) CK(launch_to_f32(h->faces + f * n, q + f * pad(n), n, h->stream));
        h->op.wx32 = q; h->op.wy32 = q + pad(n); h->op.wz32 = q + 2 * pad(n);
        q += 3 * pad(n);
    }
    if (h->diag) { CK(launch_to_f32(h->diag, q, n, h->stream)); h->op.diag32 = q; q += pad(n); }
    if (h->cdinv) { CK(launch_to_f32(h->cdinv, q, n, h->stream)); h->op.cdinv32 = q; q += pad(n); }
    return SSTEP_OK;
}

sstep_status finish_create(sstep_cg_t h) {
    const int64_t n = h->op.n;
    // Jacobi coefficients need the bounds; bounds (Lanczos) need the diagonal.
    sstep_status st = compute_bounds(h);
    if (st != SSTEP_OK) return st;
    h->theta = 2.0 / (h->lmax - h->lmin);
    h->sigma = 0.5 * (h->lmax + h->lmin);
    if (h->jacobi && h->diag) {
        CK(cudaMalloc(&h->cdinv, sizeof(double) * n));
        CK(launch_scale_vec(h->diag, 2.0 * h->theta, h->cdinv, n, h->stream));
        h->op.cdinv = h->cdinv;
    }
    h->ld = (n + 31) / 32 * 32;
    // P_+ (s+1 columns); the conjugated form adds Q_(k-1) and A Q_(k-1) (s columns each)
    const int ncols = h->conj ? 3 * h->opts.s + 1 : h->opts.s + 1;
    CK(cudaMalloc(&h->P, sizeof(double) * h->ld * ncols));
    if (h->conj) {
        const int s = h->opts.s;
        h->conj_nblk = conj_cd_blocks(s, n, h->sm_count);
        CK(cudaMalloc(&h->conj_partials, sizeof(double) * (size_t)h->conj_nblk * (s * s + s)));
        CK(cudaMalloc(&h->cj, sizeof(double) * 2 * s * s));
    }
    if (h->mixed) {
        CK(cudaMalloc(&h->P32, sizeof(float) * h->ld * (h->opts.s + 1)));
        if ((st = make_f32_operator(h)) != SSTEP_OK) return st;
        // FP32 steps through TMA tiles: forced, or (AUTO) when the step's three FP32 vectors
        // exceed L2 (below that the plain-load kernel is faster); plain loads when the shape
        // or the driver does not allow it
        int l2 = 0;
        CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device));
        const bool want = h->opts.step_kernel == SSTEP_STEP_TMA ||
                          (h->opts.step_kernel == SSTEP_STEP_AUTO && 3.0 * sizeof(float) * (double)n > (double)l2);
        if (want && step_tma_shape(h->op)) {
            h->tmaps.resize(2 * (size_t)(h->opts.s + 1));
            bool ok = true;
            for (int j = 0; j <= h->opts.s && ok; ++j)
                ok = step_tma_maps(h->op, h->P32 + (int64_t)j * h->ld, &h->tmaps[2 * j], &h->tmaps[2 * j + 1]) == cudaSuccess;
            h->tma = ok;
            if (!ok) h->tmaps.clear();
        }
    }
    CK(cudaMalloc(&h->rtrue, sizeof(double) * n));
    if (h->opts.history > 0) {
        CK(cudaMalloc(&h->hist, sizeof(double) * 4 * h->opts.history));
        CK(cudaMemsetAsync(h->hist, 0, sizeof(double) * 4 * h->opts.history, h->stream));
    }
    if (h->fused) {
        // the step kernels reduce the moments: a stencil operator with a constant M (Poisson
        // star or box stencil, or no preconditioner)
        if (h->op.kind != OP_STENCIL || (h->jacobi && h->diag)) {
            set_err(h, "gram_form FUSED needs a stencil operator with a constant preconditioner (Poisson or "
                       "box stencil, or precond NONE)");
            return SSTEP_ERR_UNSUPPORTED;
        }
        h->mom_nblk = cheb_step_blocks(h->op, h->mixed, h->tma);
        CK(cudaMalloc(&h->mom_part, (size_t)16 * h->mom_nblk * h->opts.s));
        CK(cudaMalloc(&h->mom_part2, sizeof(double) * MAX_FIN_BLOCKS * 2 * h->opts.s));
    }
    GramArgs g = gram_args(h);
    h->gram_nblk = gram_blocks(g, h->sm_count);
    CK(cudaMalloc(&h->gram_partials, sizeof(double) * gram_partials_needed(g, h->gram_nblk)));
    CK(cudaMalloc(&h->res_partials, sizeof(double) * residual_partials_needed(h->op)));
    CK(cudaMalloc(&h->ctl, sizeof(Ctl)));
    CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
    CK(cudaMallocHost(&h->ctl_h, sizeof(Ctl)));
    std::memset(h->ctl_h, 0, sizeof(Ctl));
    CK(cudaStreamSynchronize(h->stream));
    return SSTEP_OK;
}

sstep_status begin_create(sstep_cg_t* out, const sstep_cg_opts* opts, void* stream, sstep_cg_t* hp) {
    if (!out) return SSTEP_ERR_INVALID_ARG;
    *out = nullptr;
    sstep_cg_t h = new (std::nothrow) sstep_cg_s();
    if (!h) return SSTEP_ERR_OOM;
    *hp = h;
    sstep_cg_opts o;
    if (opts) o = *opts; else sstep_cg_default_opts(&o);
    sstep_status st = validate_opts(h, &o);
    if (st != SSTEP_OK) return st;
    h->opts = o;
    h->stream = (cudaStream_t)stream;
    h->jacobi = o.precond == SSTEP_PRECOND_JACOBI;
    h->mixed = o.precision == SSTEP_PRECISION_MIXED;
    h->conj = o.block_conjugate != 0;
    h->fused = o.gram_form == SSTEP_GRAM_FORM_FUSED;
    return SSTEP_OK;
}

// First CUDA call of a create: after every argument has been validated on the host.
sstep_status bind_device(sstep_cg_t h) {
    CK(cudaGetDevice(&h->device));
    CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
    return SSTEP_OK;
}

// Error message buffer for failures without a handle (create calls, handle-free entry points).
thread_local char g_create_err[512];

sstep_status fail_create(sstep_cg_t h, sstep_status st) {
    if (h) {
        std::snprintf(g_create_err, sizeof(g_create_err), "%s", h->err);
        sstep_cg_destroy(h);
    }
    return st;
}

// Kernels of one outer iteration (refresh: the mixed form's FP64 residual refresh runs).
int outer_kernels(sstep_cg_t h, bool refresh) {
    return h->opts.s + 2 + (h->mixed && refresh ? 1 : 0) + (h->conj ? 1 : 0);
}

// One outer iteration: s Chebyshev steps, the Gram + FGS (or the fused form's finish), the
// update (FP64 form); or, in the mixed form, the FP64 residual refresh when `refresh` is set
// (else the FP32 p_0 the previous update wrote), s FP32 Chebyshev steps, the Gram + FGS and the
// x update, which also writes the next FP32 p_0 when `write_r` is set (the next outer
// iteration does not refresh). With `prof`, events ev[0..] bracket every kernel.
sstep_status launch_outer(sstep_cg_t h, const double* b, double* x, int* launches, bool prof, bool refresh = true,
                          bool write_r = false) {
    const int s = h->opts.s;
    int ev = 0;
    if (prof) CK(cudaEventRecord(h->ev[ev++], h->stream));
    if (h->mixed && refresh) {
        CK(launch_residual(h->op, b, x, nullptr, h->P32, h->res_partials, h->ctl, 2, h->stream));
        if (prof) CK(cudaEventRecord(h->ev[ev++], h->stream));
    }
    for (int j = 0; j < s; ++j) {
        void* mom = h->fused ? (void*)((char*)h->mom_part + (size_t)16 * h->mom_nblk * j) : nullptr;
        if (h->mixed) {
            const float* p = h->P32 + (int64_t)j * h->ld;
            const float* q = j > 0 ? h->P32 + (int64_t)(j - 1) * h->ld : nullptr;
            float* o = h->P32 + (int64_t)(j + 1) * h->ld;
            if (h->tma)
                CK(launch_cheb_step_tma(h->op, h->tmaps[2 * j], h->tmaps[j > 0 ? 2 * j - 1 : 2 * j], o, h->theta,
                                        h->sigma, j == 0, h->jacobi, h->ctl, h->stream, mom));
            else
                CK(launch_cheb_step<float>(h->op, p, q, o, h->theta, h->sigma, j == 0, h->jacobi, h->ctl, h->stream, mom));
        } else {
            const double* p = h->P + (int64_t)j * h->ld;
            const double* q = j > 0 ? h->P + (int64_t)(j - 1) * h->ld : nullptr;
            double* o = h->P + (int64_t)(j + 1) * h->ld;
            CK(launch_cheb_step<double>(h->op, p, q, o, h->theta, h->sigma, j == 0, h->jacobi, h->ctl, h->stream, mom));
        }
        if (prof) CK(cudaEventRecord(h->ev[ev++], h->stream));
    }
    GramArgs g = gram_args_outer(h);
    if (h->mixed) g.check = refresh ? 0 : 2;
    if (h->conj)   // C and d for the block conjugation (timed with the Gram)
        CK(launch_conj_cd(s, h->P, h->ld, h->op.n, h->conj_partials, h->conj_nblk, h->ctl, h->stream));
    if (h->fused) {
        g.fp32 = h->mixed;
        CK(launch_moments_finish(g, h->mom_part, h->mom_nblk, h->mom_part2, h->ctl, h->stream));
    } else {
        CK(launch_gram(g, h->gram_partials, h->ctl, h->gram_nblk, h->stream));
    }
    if (prof) CK(cudaEventRecord(h->ev[ev++], h->stream));
    if (h->mixed) {
        CK(launch_update_mixed(h->P32, h->ld, s, h->op.n, x, h->ctl, h->stream, write_r, g.dvec ? h->op.diag32 : nullptr));
    } else if (h->conj) {
        CK(launch_update_conj(s, h->P, h->ld, h->op.n, g.dvec ? h->diag : nullptr, g.dconst, h->theta, h->sigma,
                              h->cj, x, h->ctl, h->stream));
    } else {
        UpdateArgs u{};
        u.s = s;
        u.dvec = g.dvec;
        u.diag = h->diag;
        u.n = h->op.n;
        u.ld = h->ld;
        u.P = h->P;
        u.fp32 = false;
        u.x = x;
        u.skip_r = false;
        CK(launch_update(u, h->ctl, h->stream));
    }
    if (prof) CK(cudaEventRecord(h->ev[ev++], h->stream));
    *launches += outer_kernels(h, refresh);
    return SSTEP_OK;
}

// Outer iterations per group: the mixed form refreshes the FP64 residual in the first outer
// iteration of each group of refresh_period; the FP64 form keeps its recursive residual.
int group_size(sstep_cg_t h) { return h->mixed ? h->opts.refresh_period : 1; }

// Adds the kernel times of the last profiled outer iteration (events complete) to inf.
sstep_status collect_outer_profile(sstep_cg_t h, sstep_cg_info* inf, bool refreshed) {
    const int s = h->opts.s;
    float ms = 0.f;
    int ev = 0;
    if (h->mixed && refreshed) {
        CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
        inf->prof_ms[3] += ms;
        inf->prof_launches[3] += 1;
        ev = 1;
    }
    for (int j = 0; j < s; ++j, ++ev) {
        CK(cudaEventElapsedTime(&ms, h->ev[ev], h->ev[ev + 1]));
        inf->prof_ms[0] += ms;
        inf->prof_launches[0] += 1;
    }
    CK(cudaEventElapsedTime(&ms, h->ev[ev], h->ev[ev + 1]));
    inf->prof_ms[1] += ms;
    inf->prof_launches[1] += 1;
    ++ev;
    CK(cudaEventElapsedTime(&ms, h->ev[ev], h->ev[ev + 1]));
    inf->prof_ms[2] += ms;
    inf->prof_launches[2] += 1;
    return SSTEP_OK;
}

sstep_status ensure_events(sstep_cg_t h) {
    if (h->rev[1]) return SSTEP_OK;   // the last one created: all exist
    for (int i = 0; i < SSTEP_MAX_S + 4; ++i)
        if (!h->ev[i]) CK(cudaEventCreate(&h->ev[i]));
    if (!h->rev[0]) CK(cudaEventCreate(&h->rev[0]));
    CK(cudaEventCreate(&h->rev[1]));
    return SSTEP_OK;
}

// Residual kernel, optionally bracketed by events and added to inf->prof_*[3].
sstep_status launch_residual_timed(sstep_cg_t h, const double* b, const double* x, double* r, int mode,
                                   sstep_cg_info* inf, bool prof) {
    if (prof) CK(cudaEventRecord(h->rev[0], h->stream));
    CK(launch_residual(h->op, b, x, r, nullptr, h->res_partials, h->ctl, mode, h->stream));
    if (prof) {
        CK(cudaEventRecord(h->rev[1], h->stream));
        CK(cudaEventSynchronize(h->rev[1]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->rev[0], h->rev[1]));
        inf->prof_ms[3] += ms;
        inf->prof_launches[3] += 1;
    }
    return SSTEP_OK;
}

void drop_graph(sstep_cg_t h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    h->g_b = nullptr;
    h->g_x = nullptr;
}

// The outer loop as one graph: a while node whose body is one outer iteration followed by
// k_loop_cond, which keeps the node looping while ctl->done == RUNNING. Captured on an
// internal stream (the caller's may be the legacy stream, which cannot be captured).
sstep_status build_graph(sstep_cg_t h, const double* b, double* x) {
    drop_graph(h);
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaGraphCreate(&h->graph, 0));
    cudaGraphConditionalHandle ch;
    CK(cudaGraphConditionalHandleCreate(&ch, h->graph, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = ch;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    int dummy = 0;
    sstep_status st = SSTEP_OK;
    const int grp = group_size(h);
    for (int m = 0; m < grp && st == SSTEP_OK; ++m) st = launch_outer(h, b, x, &dummy, false, m == 0, m + 1 < grp);
    cudaError_t e = st == SSTEP_OK ? launch_loop_cond(ch, h->ctl, h->cap_stream) : cudaSuccess;
    h->stream = user;
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &captured);
    if (st != SSTEP_OK) { drop_graph(h); return st; }
    CK(e);
    CK(e2);
    CK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
    h->g_b = b;
    h->g_x = x;
    return SSTEP_OK;
}

sstep_status read_ctl(sstep_cg_t h) {
    CK(cudaMemcpyAsync(h->ctl_h, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SSTEP_OK;
}

sstep_status solve_impl(sstep_cg_t h, const double* b, double* x, sstep_cg_info* info) {
    sstep_cg_info inf{};
    inf.lambda_min_used = h->lmin;
    inf.lambda_max_used = h->lmax;
    SolveEvents tev;
    CK(cudaEventCreate(&tev.e0));
    CK(cudaEventCreate(&tev.e1));
    CK(cudaEventRecord(tev.e0, h->stream));
    // control block: running, zero outers, tolerance
    Ctl init{};
    init.tol_sq = h->opts.tol * h->opts.tol;
    init.max_outer = h->opts.max_outer;
    init.min_gii = INFINITY;
    init.scale = 1.0;
    init.scale_next = 1.0;
    std::memcpy(h->ctl_h, &init, sizeof(Ctl));
    CK(cudaMemcpyAsync(h->ctl, h->ctl_h, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));
    int launches = 0;
    const bool profiling = h->opts.profile_every > 0;
    sstep_status st;
    if (profiling && (st = ensure_events(h)) != SSTEP_OK) return st;
    // initial residual r_0 (FP64 form: straight into p_0; mixed form: only ||r_0||, the first
    // outer iteration's refresh writes the FP32 p_0)
    if ((st = launch_residual_timed(h, b, x, h->mixed ? nullptr : h->P, 0, &inf, profiling)) != SSTEP_OK) return st;
    ++launches;
    sstep_status status = SSTEP_OK;
    int refreshes = 0;
    const int grp = group_size(h);
    // kernels of one pass of the graph body: a group of outer iterations and the condition
    const int body_launches = outer_kernels(h, true) + (grp - 1) * outer_kernels(h, false) + 1;
    // conjugated form: the first block has no predecessor (Q_(-1) = A Q_(-1) = 0)
    if (h->conj)
        CK(cudaMemsetAsync(h->P + (int64_t)(h->opts.s + 1) * h->ld, 0, sizeof(double) * 2 * h->opts.s * h->ld,
                           h->stream));
    // outer iterations launched in the current group sequence: the mixed form refreshes the FP64
    // residual in outer iterations with in_group % refresh_period == 0, as the graph body does
    long in_group = 0;
    for (long chunk = 0;; ++chunk) {
        if (h->opts.use_graph) {
            if (!h->gexec || h->g_b != b || h->g_x != x)
                if ((st = build_graph(h, b, x)) != SSTEP_OK) return st;
            const int before = h->ctl_h->outer;
            CK(cudaGraphLaunch(h->gexec, h->stream));
            if ((st = read_ctl(h)) != SSTEP_OK) return st;
            // kernels that ran: every body pass launches its group's kernels and the condition;
            // the pass that saw the stop is the last
            launches += ((h->ctl_h->outer - before) / grp + 1) * body_launches;
        } else {
            const bool prof = profiling && chunk % h->opts.profile_every == 0;
            // the sampled outer iteration is the chunk's second (the very first outer iteration
            // of a solve is not typical: in the conjugated form its previous block is zero)
            // (the mixed form with refresh_period > 1 samples the chunk's first outer iteration,
            // which normally refreshes the FP64 residual)
            const int sample = (h->mixed && grp > 1) || h->opts.check_every == 1 ? 0 : 1;
            const int before = h->ctl_h->outer;
            const long m0 = in_group;
            for (int m = 0; m < h->opts.check_every; ++m, ++in_group)
                if ((st = launch_outer(h, b, x, &launches, prof && m == sample, in_group % grp == 0,
                                       (in_group + 1) % grp != 0)) != SSTEP_OK)
                    return st;
            if ((st = read_ctl(h)) != SSTEP_OK) return st;
            // keep the sample only if that outer iteration did its work (its kernels exit at once
            // after convergence)
            if (prof && h->ctl_h->outer > before + sample &&
                (st = collect_outer_profile(h, &inf, (m0 + sample) % grp == 0)) != SSTEP_OK)
                return st;
        }
        const int done = h->ctl_h->done;
        if (done == RUNNING) continue;
        // true residual b - A x (Section 8 stopping rule is checked on it at exit)
        if ((st = launch_residual_timed(h, b, x, h->rtrue, 1, &inf, profiling)) != SSTEP_OK) return st;
        ++launches;
        if ((st = read_ctl(h)) != SSTEP_OK) return st;
        const Ctl& c = *h->ctl_h;
        const bool true_ok = c.r0_sq == 0.0 || c.true_sq < c.tol_sq * c.r0_sq;
        if (done == CONVERGED && !true_ok && refreshes < h->opts.max_refresh) {
            ++refreshes;
            in_group = 0;   // the mixed form's next outer iteration loads the replaced residual
            CK(cudaMemcpyAsync(h->P, h->rtrue, sizeof(double) * h->op.n, cudaMemcpyDeviceToDevice, h->stream));
            const int zero = RUNNING;
            CK(cudaMemcpyAsync(&h->ctl->done, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
            // a replaced residual restarts the block conjugation (the next block is Q = P)
            if (h->conj) CK(cudaMemcpyAsync(&h->ctl->conj_valid, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            continue;
        }
        if (done == NUMERICAL) status = SSTEP_ERR_NUMERICAL;
        else if (done == TIMED_OUT) status = SSTEP_ERR_TIMEOUT;
        else if (done == MAX_OUTER || !true_ok) status = SSTEP_ERR_NO_CONVERGENCE;
        break;
    }
    CK(cudaEventRecord(tev.e1, h->stream));
    CK(cudaEventSynchronize(tev.e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, tev.e0, tev.e1));
    const Ctl& c = *h->ctl_h;
    inf.outer_iters = c.outer;
    inf.refreshes = refreshes;
    inf.status = status;
    inf.r0_norm = std::sqrt(c.r0_sq);
    inf.rel_res_recursive = c.r0_sq > 0 ? std::sqrt(c.rk_sq / c.r0_sq) : 0.0;
    inf.rel_res_true = c.r0_sq > 0 ? std::sqrt(c.true_sq / c.r0_sq) : 0.0;
    inf.min_gii = c.min_gii;
    inf.delta_last = c.delta;
    inf.ms = ms;
    inf.kernel_launches = launches;
    inf.step_tma = h->tma ? 1 : 0;
    if (info) *info = inf;
    if (status != SSTEP_OK)
        set_err(h, "solve ended with %s after %d outer iterations (true rel. residual %.3e)",
                sstep_cg_status_string(status), c.outer, inf.rel_res_true);
    return status;
}

}  // namespace

namespace sstep {
void set_global_error(const char* msg) { std::snprintf(g_create_err, sizeof(g_create_err), "%s", msg); }
}  // namespace sstep

extern "C" {

void sstep_cg_default_opts(sstep_cg_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->s = 8;
    o->nu = 25;
    o->lambda_min = 0.0;
    o->lambda_max = 0.0;
    o->bounds_mode = SSTEP_BOUNDS_GERSH_LANCZOS10;
    o->tol = 1e-8;
    o->max_outer = 100000;
    o->gram_solver = SSTEP_GRAM_SOLVE_FGS;
    o->precision = SSTEP_PRECISION_FP64;
    o->precond = SSTEP_PRECOND_JACOBI;
    o->basis_start = SSTEP_START_R;
    o->gram_form = SSTEP_GRAM_FORM_DIRECT;
    o->refresh_period = 1;
    o->max_refresh = 3;
    o->seed = 5000;
    o->use_graph = 0;
    o->check_every = 8;
    o->profile_every = 0;
    o->batch_chunk = 0;
    o->batch_ctas_per_sm = 0;
    o->block_conjugate = 0;
    o->history = 0;
    o->step_kernel = SSTEP_STEP_AUTO;
}

sstep_status sstep_cg_create_csr(sstep_cg_t* out, int64_t n, const int32_t* rowptr_d, const int32_t* colind_d,
                                 const double* vals_d, const sstep_cg_opts* opts, void* stream) {
    sstep_cg_t h = nullptr;
    sstep_status st = begin_create(out, opts, stream, &h);
    if (st != SSTEP_OK) return fail_create(h, st);
    if (n < 1 || n > 2147483647LL) { set_err(h, "n = %lld outside [1, 2^31)", (long long)n); return fail_create(h, SSTEP_ERR_INVALID_ARG); }
    if (!rowptr_d || !colind_d || !vals_d || !aligned16(rowptr_d) || !aligned16(colind_d) || !aligned16(vals_d)) {
        set_err(h, "CSR arrays must be non-null 16-byte aligned device pointers");
        return fail_create(h, SSTEP_ERR_INVALID_ARG);
    }
    if ((st = bind_device(h)) != SSTEP_OK) return fail_create(h, st);
    h->op.kind = OP_CSR;
    h->op.n = n;
    h->op.rowptr = rowptr_d;
    h->op.colind = colind_d;
    h->op.vals = vals_d;
    h->op.dconst = 1.0;
    int* bad = nullptr;
    cudaError_t e = cudaMalloc(&h->diag, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), h->stream);
    h->op.diag = h->diag;
    if (e == cudaSuccess) e = launch_csr_diag(h->op, h->diag, bad, h->stream);
    int hb = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(bad);
    if (e != cudaSuccess) { set_err(h, "CSR set-up: %s", cudaGetErrorString(e)); return fail_create(h, SSTEP_ERR_CUDA); }
    if (hb) { set_err(h, "a diagonal entry is missing, non-positive or not finite"); return fail_create(h, SSTEP_ERR_INVALID_ARG); }
    if (!h->jacobi) { /* M = I: Gram weights are 1 */ }
    st = finish_create(h);
    if (st != SSTEP_OK) return fail_create(h, st);
    *out = h;
    return SSTEP_OK;
}

sstep_status sstep_cg_create_stencil(sstep_cg_t* out, int dim, int nx, int ny, int nz, const double* kappa_d,
                                     const sstep_cg_opts* opts, void* stream) {
    sstep_cg_t h = nullptr;
    sstep_status st = begin_create(out, opts, stream, &h);
    if (st != SSTEP_OK) return fail_create(h, st);
    // ny and nz bound the grid's y and z extents at 8 rows and 8 planes per block
    if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1) || ny > 65535 * 8 ||
        (dim == 3 && nz > 65535 * 8)) {
        set_err(h, "bad grid: dim %d, %d x %d x %d", dim, nx, ny, nz);
        return fail_create(h, SSTEP_ERR_INVALID_ARG);
    }
    if (kappa_d && !aligned16(kappa_d)) { set_err(h, "kappa must be 16-byte aligned"); return fail_create(h, SSTEP_ERR_INVALID_ARG); }
    if ((st = bind_device(h)) != SSTEP_OK) return fail_create(h, st);
    const int64_t n = (int64_t)nx * ny * nz;
    h->op.kind = OP_STENCIL;
    h->op.n = n;
    h->op.dim = dim;
    h->op.nx = nx;
    h->op.ny = ny;
    h->op.nz = nz;
    h->op.dconst = 2.0 * dim;
    if (kappa_d) {
        int* bad = nullptr;
        cudaError_t e = cudaMalloc(&h->faces, sizeof(double) * 3 * n);
        if (e == cudaSuccess) e = cudaMalloc(&h->diag, sizeof(double) * n);
        if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->faces, 0, sizeof(double) * 3 * n, h->stream);
        h->op.wx = h->faces;
        h->op.wy = h->faces + n;
        h->op.wz = h->faces + 2 * n;
        h->op.diag = h->diag;
        if (e == cudaSuccess)
            e = launch_stencil_faces(dim, nx, ny, nz, kappa_d, h->faces, h->faces + n, h->faces + 2 * n, h->diag, bad, h->stream);
        int hb = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(bad);
        if (e != cudaSuccess) { set_err(h, "stencil set-up: %s", cudaGetErrorString(e)); return fail_create(h, e == cudaErrorMemoryAllocation ? SSTEP_ERR_OOM : SSTEP_ERR_CUDA); }
        if (hb) { set_err(h, "kappa must be positive and finite"); return fail_create(h, SSTEP_ERR_INVALID_ARG); }
        h->kappa = kappa_d;
    }
    st = finish_create(h);
    if (st != SSTEP_OK) return fail_create(h, st);
    *out = h;
    return SSTEP_OK;
}

sstep_status sstep_cg_create_box_stencil(sstep_cg_t* out, int dim, int nx, int ny, int nz, const sstep_cg_opts* opts,
                                         void* stream) {
    sstep_cg_t h = nullptr;
    sstep_status st = begin_create(out, opts, stream, &h);
    if (st != SSTEP_OK) return fail_create(h, st);
    if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1) || ny > 65535 * 8 ||
        (dim == 3 && nz > 65535 * 16)) {
        set_err(h, "bad grid: dim %d, %d x %d x %d", dim, nx, ny, nz);
        return fail_create(h, SSTEP_ERR_INVALID_ARG);
    }
    if ((st = bind_device(h)) != SSTEP_OK) return fail_create(h, st);
    h->op.kind = OP_STENCIL;
    h->op.box = 1;
    h->op.n = (int64_t)nx * ny * nz;
    h->op.dim = dim;
    h->op.nx = nx;
    h->op.ny = ny;
    h->op.nz = nz;
    h->op.dconst = dim == 3 ? 26.0 : 8.0;
    st = finish_create(h);
    if (st != SSTEP_OK) return fail_create(h, st);
    *out = h;
    return SSTEP_OK;
}

sstep_status sstep_coarse_fgs(sstep_cg_t h, int bx, int by, int bz, const double* g_d, double* y_d, int nu, int mode) {
    if (!h) return SSTEP_ERR_INVALID_ARG;
    if (h->op.kind != OP_STENCIL) {
        set_err(h, "coarse FGS needs a stencil handle (box aggregation of its grid)");
        return SSTEP_ERR_UNSUPPORTED;
    }
    if (bx < 1 || by < 1 || bz < 1 || (h->op.dim == 2 && bz != 1) || nu < 1 || !g_d || !y_d ||
        (mode != SSTEP_COARSE_FORMED && mode != SSTEP_COARSE_STREAMING)) {
        set_err(h, "coarse FGS: need aggregate sizes >= 1 (bz = 1 in 2D), nu >= 1, device g and y, a known mode");
        return SSTEP_ERR_INVALID_ARG;
    }
    const int64_t nc = (int64_t)((h->op.nx + bx - 1) / bx) * ((h->op.ny + by - 1) / by) * ((h->op.nz + bz - 1) / bz);
    if (nc > 2147483647LL) {
        set_err(h, "coarse FGS: n_c = %lld aggregates, above 2^31 - 1", (long long)nc);
        return SSTEP_ERR_INVALID_ARG;
    }
    if (mode == SSTEP_COARSE_FORMED && nc > coarse_formed_max_nc()) {
        set_err(h, "coarse FGS: formed A_c limited to n_c <= %d (got %lld); use the streaming mode",
                coarse_formed_max_nc(), (long long)nc);
        return SSTEP_ERR_INVALID_ARG;
    }
    double* dc = nullptr;
    double* Ac = nullptr;
    cudaError_t e = cudaSuccess;
    if (mode == SSTEP_COARSE_STREAMING) e = cudaMalloc(&dc, sizeof(double) * nc);
    else e = cudaMalloc(&Ac, sizeof(double) * nc * nc);
    if (e == cudaSuccess)
        e = launch_coarse_fgs(h->op, bx, by, bz, (int)nc, g_d, y_d, nu, mode == SSTEP_COARSE_STREAMING, h->rtrue, dc,
                              Ac, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dc);
    cudaFree(Ac);
    if (e != cudaSuccess) {
        set_err(h, "coarse FGS: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SSTEP_ERR_OOM : SSTEP_ERR_CUDA;
    }
    return SSTEP_OK;
}

sstep_status sstep_cg_solve(sstep_cg_t h, const double* b_d, double* x_d, sstep_cg_info* info) {
    if (!h) return SSTEP_ERR_INVALID_ARG;
    if (!b_d || !x_d || !aligned16(b_d) || !aligned16(x_d)) {
        set_err(h, "b and x must be non-null 16-byte aligned device pointers");
        return SSTEP_ERR_INVALID_ARG;
    }
    return solve_impl(h, b_d, x_d, info);
}

sstep_status sstep_cg_solve_host(sstep_cg_t h, const double* b_h, double* x_h, sstep_cg_info* info) {
    if (!h || !b_h || !x_h) return SSTEP_ERR_INVALID_ARG;
    const int64_t n = h->op.n;
    if (!h->bx_dev) CK(cudaMalloc(&h->bx_dev, sizeof(double) * 2 * ((n + 31) / 32 * 32)));
    double* bd = h->bx_dev;
    double* xd = h->bx_dev + (n + 31) / 32 * 32;
    SolveEvents tev;
    CK(cudaEventCreate(&tev.e0));
    CK(cudaEventCreate(&tev.e1));
    CK(cudaEventRecord(tev.e0, h->stream));
    CK(cudaMemcpyAsync(bd, b_h, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(xd, x_h, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
    sstep_cg_info inf{};
    sstep_status st = solve_impl(h, bd, xd, &inf);
    if (st != SSTEP_OK && st != SSTEP_ERR_NO_CONVERGENCE && st != SSTEP_ERR_NUMERICAL) return st;
    CK(cudaMemcpyAsync(x_h, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaEventRecord(tev.e1, h->stream));
    CK(cudaEventSynchronize(tev.e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, tev.e0, tev.e1));
    inf.ms = ms;
    if (info) *info = inf;
    return st;
}

sstep_status sstep_cg_destroy(sstep_cg_t h) {
    if (!h) return SSTEP_OK;
    cudaStreamSynchronize(h->stream);
    cudaFree(h->diag);
    cudaFree(h->cdinv);
    cudaFree(h->faces);
    cudaFree(h->P);
    cudaFree(h->P32);
    cudaFree(h->ops32);
    cudaFree(h->rtrue);
    cudaFree(h->gram_partials);
    cudaFree(h->mom_part);
    cudaFree(h->mom_part2);
    cudaFree(h->hist);
    cudaFree(h->res_partials);
    cudaFree(h->conj_partials);
    cudaFree(h->cj);
    cudaFree(h->ctl);
    cudaFree(h->bx_dev);
    drop_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->ctl_h) cudaFreeHost(h->ctl_h);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->rev)
        if (e) cudaEventDestroy(e);
    delete h;
    return SSTEP_OK;
}

const char* sstep_cg_status_string(sstep_status s) {
    switch (s) {
        case SSTEP_OK: return "SSTEP_OK";
        case SSTEP_ERR_INVALID_ARG: return "SSTEP_ERR_INVALID_ARG";
        case SSTEP_ERR_CUDA: return "SSTEP_ERR_CUDA";
        case SSTEP_ERR_OOM: return "SSTEP_ERR_OOM";
        case SSTEP_ERR_NUMERICAL: return "SSTEP_ERR_NUMERICAL";
        case SSTEP_ERR_NO_CONVERGENCE: return "SSTEP_ERR_NO_CONVERGENCE";
        case SSTEP_ERR_TIMEOUT: return "SSTEP_ERR_TIMEOUT";
        case SSTEP_ERR_UNSUPPORTED: return "SSTEP_ERR_UNSUPPORTED";
    }
    return "unknown status";
}

const char* sstep_cg_last_error(sstep_cg_t h) { return h ? h->err : g_create_err; }

sstep_status sstep_cg_apply(sstep_cg_t h, const double* x_d, double* y_d) {
    if (!h || !x_d || !y_d) return SSTEP_ERR_INVALID_ARG;
    CK(launch_apply(h->op, x_d, y_d, h->stream));
    return SSTEP_OK;
}

sstep_status sstep_cg_basis(sstep_cg_t h, const double* r_d, double* P_d, int64_t ldp, int ncols) {
    if (!h || !r_d || !P_d || ldp < h->op.n || ncols < 1 || ncols > SSTEP_MAX_S + 1) return SSTEP_ERR_INVALID_ARG;
    // reset the control block so the step kernels run
    const int zero = RUNNING;
    CK(cudaMemcpyAsync(&h->ctl->done, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(P_d, r_d, sizeof(double) * h->op.n, cudaMemcpyDeviceToDevice, h->stream));
    for (int j = 0; j + 1 < ncols; ++j) {
        const double* p = P_d + (int64_t)j * ldp;
        const double* q = j > 0 ? P_d + (int64_t)(j - 1) * ldp : nullptr;
        CK(launch_cheb_step<double>(h->op, p, q, P_d + (int64_t)(j + 1) * ldp, h->theta, h->sigma, j == 0, h->jacobi,
                                    h->ctl, h->stream));
    }
    return SSTEP_OK;
}

sstep_status sstep_cg_load_basis(sstep_cg_t h, const double* P_d, int64_t ldp) {
    if (!h || !P_d || ldp < h->op.n) return SSTEP_ERR_INVALID_ARG;
    for (int j = 0; j <= h->opts.s; ++j)
        CK(cudaMemcpyAsync(h->P + (int64_t)j * h->ld, P_d + (int64_t)j * ldp, sizeof(double) * h->op.n,
                           cudaMemcpyDeviceToDevice, h->stream));
    return SSTEP_OK;
}

sstep_status sstep_cg_gram_solve(sstep_cg_t h, double* out_h) {
    if (!h || !out_h) return SSTEP_ERR_INVALID_ARG;
    Ctl init{};
    init.tol_sq = 0.0;
    init.r0_sq = 1.0;
    init.max_outer = 1;
    init.min_gii = INFINITY;
    std::memcpy(h->ctl_h, &init, sizeof(Ctl));
    CK(cudaMemcpyAsync(h->ctl, h->ctl_h, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));
    GramArgs g = gram_args(h);
    g.fp32 = false;   // this entry point works on the FP64 basis loaded by sstep_cg_load_basis
    g.P = h->P;
    CK(launch_gram(g, h->gram_partials, h->ctl, h->gram_nblk, h->stream));
    sstep_status st = read_ctl(h);
    if (st != SSTEP_OK) return st;
    const Ctl& c = *h->ctl_h;
    if (c.done == NUMERICAL) { set_err(h, "Gram system not usable"); return SSTEP_ERR_NUMERICAL; }
    const int s = h->opts.s;
    for (int i = 0; i < s; ++i) {
        out_h[i] = c.alpha[i];
        out_h[s + i] = c.d[i];
        out_h[2 * s + i] = c.ct[i];
    }
    for (int i = 0; i < s * s; ++i) out_h[3 * s + i] = c.Gt[i];
    return SSTEP_OK;
}

sstep_status sstep_cg_get_bounds(sstep_cg_t h, double* lmin, double* lmax) {
    if (!h || !lmin || !lmax) return SSTEP_ERR_INVALID_ARG;
    *lmin = h->lmin;
    *lmax = h->lmax;
    return SSTEP_OK;
}

sstep_status sstep_cg_get_residual(sstep_cg_t h, double* r_d) {
    if (!h || !r_d) return SSTEP_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(r_d, h->P, sizeof(double) * h->op.n, cudaMemcpyDeviceToDevice, h->stream));
    return SSTEP_OK;
}

sstep_status sstep_convert_check(const double* in_d, int k, float* out_d, double* back_d, int64_t n, void* stream) {
    if (!in_d || !out_d || !back_d || n < 0) return SSTEP_ERR_INVALID_ARG;
    if (n == 0) return SSTEP_OK;
    cudaError_t e = launch_convert_check(in_d, k, out_d, back_d, n, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        sstep::set_global_error(cudaGetErrorString(e));
        return SSTEP_ERR_CUDA;
    }
    return SSTEP_OK;
}

sstep_status sstep_cg_history(sstep_cg_t h, double* out_h, int capacity, int* count) {
    if (!h || !out_h || capacity < 1 || !count) return SSTEP_ERR_INVALID_ARG;
    *count = 0;
    if (!h->hist) {
        set_err(h, "the handle keeps no history (opts.history = 0)");
        return SSTEP_ERR_INVALID_ARG;
    }
    sstep_status st = read_ctl(h);
    if (st != SSTEP_OK) return st;
    const int cap = h->opts.history, outer = h->ctl_h->outer;
    int m = outer < cap ? outer : cap;
    if (m > capacity) m = capacity;
    std::vector<double> ring((size_t)4 * cap);
    CK(cudaMemcpyAsync(ring.data(), h->hist, sizeof(double) * 4 * cap, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < m; ++k) {   // the newest m records, oldest first
        const int o = outer - m + k;   // 0-based outer index
        for (int q = 0; q < 4; ++q) out_h[4 * k + q] = ring[(size_t)4 * (o % cap) + q];
    }
    *count = m;
    return SSTEP_OK;
}

sstep_status sstep_cg_set_tolerance(sstep_cg_t h, double tol, int max_outer) {
    if (!h) return SSTEP_ERR_INVALID_ARG;
    if (!(tol > 0.0) || !std::isfinite(tol) || max_outer < 0) {
        set_err(h, "need tol > 0 and max_outer >= 0");
        return SSTEP_ERR_INVALID_ARG;
    }
    h->opts.tol = tol;
    h->opts.max_outer = max_outer;
    return SSTEP_OK;
}

sstep_status sstep_cg_grad_kappa(sstep_cg_t h, const double* x_d, const double* lambda_d, double* gkappa_d) {
    if (!h || !x_d || !lambda_d || !gkappa_d) return SSTEP_ERR_INVALID_ARG;
    if (h->op.kind != OP_STENCIL || !h->kappa) {
        set_err(h, "sstep_cg_grad_kappa needs a diffusion stencil handle (created with kappa)");
        return SSTEP_ERR_INVALID_ARG;
    }
    CK(launch_grad_kappa(h->op.dim, h->op.nx, h->op.ny, h->op.nz, h->kappa, x_d, lambda_d, gkappa_d, h->stream));
    return SSTEP_OK;
}

sstep_status sstep_cg_lanczos(sstep_cg_t h, int k, uint64_t seed, double* alpha_h, double* beta_h, int* steps) {
    if (!h || k < 1 || !alpha_h || !beta_h) return SSTEP_ERR_INVALID_ARG;
    std::vector<double> al, be;
    sstep_status st = lanczos(h, k, seed, al, be);
    if (st != SSTEP_OK) return st;
    for (size_t i = 0; i < al.size(); ++i) alpha_h[i] = al[i];
    for (size_t i = 0; i < be.size(); ++i) beta_h[i] = be[i];
    if (steps) *steps = (int)al.size();
    return SSTEP_OK;
}

sstep_status sstep_selftest_tma_timeout(int* done_state) {
    if (!done_state) return SSTEP_ERR_INVALID_ARG;
    const cudaError_t e = tma_wait_selftest(done_state);
    if (e == cudaErrorNotSupported) {
        sstep::set_global_error("no tensor-map encoder in this driver");
        return SSTEP_ERR_UNSUPPORTED;
    }
    if (e != cudaSuccess) {
        sstep::set_global_error(cudaGetErrorString(e));
        return SSTEP_ERR_CUDA;
    }
    return SSTEP_OK;
}

}  // extern "C"
