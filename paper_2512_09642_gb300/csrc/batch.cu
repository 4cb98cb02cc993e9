// Batched form (host): create, solve and destroy a batch of independent stencil systems.
// Every phase of an outer iteration is one launch over all still-running systems
// (batch_impl.cuh, k_batch.cu); the outer loop is either host-driven or one CUDA graph whose
// while node loops as long as any system is running.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "batch.h"

namespace sstep {
sstep_status estimate_bounds(const OpDesc& op, const double* diag, bool jacobi, const sstep_cg_opts& opts,
                             cudaStream_t stream, double* lmin, double* lmax, char* err, size_t errlen);
void set_global_error(const char* msg);
}  // namespace sstep

using namespace sstep;

struct sstep_cg_batch_s {
    int count = 0;
    sstep_cg_opts opts{};
    cudaStream_t stream = nullptr;
    int64_t ld = 0;
    std::vector<BSys> sys;
    std::vector<BTile> tiles;
    std::vector<BChunk> chunks;
    BSys* sys_d = nullptr;
    BTile* tiles_d = nullptr;
    BChunk* chunks_d = nullptr;
    double* arrays = nullptr;     // wx | wy | wz | diag | cdinv, each ld long
    double* P = nullptr;          // (s+1) x ld
    double* rtrue = nullptr;
    double* gram_partials = nullptr;
    double* tile_partials = nullptr;
    Ctl* ctl = nullptr;
    Ctl* ctl_h = nullptr;
    int* running = nullptr;
    int* running_h = nullptr;
    int* act = nullptr;          // act_sys | act_tile_prefix | act_chunk_prefix | act_n
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const double* g_b = nullptr;
    double* g_x = nullptr;
    char err[512] = {0};
};

namespace {


void berr(sstep_cg_batch_t h, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
}

#define BCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            berr(h, "%s failed: %s", #call, cudaGetErrorString(e_));                           \
            return e_ == cudaErrorMemoryAllocation ? SSTEP_ERR_OOM : SSTEP_ERR_CUDA;            \
        }                                                                                      \
    } while (0)

BatchDev dev_view(sstep_cg_batch_t h) {
    BatchDev B{};
    B.sys = h->sys_d;
    B.tiles = h->tiles_d;
    B.chunks = h->chunks_d;
    B.ntiles = (int)h->tiles.size();
    B.nchunks = (int)h->chunks.size();
    B.count = h->count;
    B.ld = h->ld;
    B.wx = h->arrays;
    B.wy = h->arrays + h->ld;
    B.wz = h->arrays + 2 * h->ld;
    B.diag = h->arrays + 3 * h->ld;
    B.cdinv = h->arrays + 4 * h->ld;
    B.ctl = h->ctl;
    B.running = h->running;
    B.gram_partials = h->gram_partials;
    B.tile_partials = h->tile_partials;
    B.ctas_per_sm = h->opts.batch_ctas_per_sm > 0 ? h->opts.batch_ctas_per_sm : 6;
    B.act_sys = h->act;
    B.act_tile_prefix = h->act + h->count;
    B.act_chunk_prefix = h->act + 2 * h->count + 1;
    B.act_n = h->act + 3 * h->count + 2;
    return B;
}

sstep_status batch_outer(sstep_cg_batch_t h, cudaStream_t st) {
    const BatchDev B = dev_view(h);
    const int s = h->opts.s;
    BCK(launch_batch_compact(B, st));
    for (int j = 0; j < s; ++j) {
        const double* p = h->P + (int64_t)j * h->ld;
        const double* q = j > 0 ? h->P + (int64_t)(j - 1) * h->ld : h->P;
        BCK(launch_batch_cheb(B, p, q, h->P + (int64_t)(j + 1) * h->ld, j == 0, st));
    }
    BCK(launch_batch_gram(B, s, h->opts.nu, h->opts.gram_solver, h->opts.gram_form == SSTEP_GRAM_FORM_MOMENTS, h->P,
                          st));
    return SSTEP_OK;
}

sstep_status batch_outer_update(sstep_cg_batch_t h, double* x, cudaStream_t st) {
    BCK(launch_batch_update(dev_view(h), h->opts.s, h->P, x, st));
    return SSTEP_OK;
}

void drop_graph(sstep_cg_batch_t h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
    h->g_b = nullptr;
    h->g_x = nullptr;
}

sstep_status build_graph(sstep_cg_batch_t h, const double* b, double* x) {
    drop_graph(h);
    if (!h->cap_stream) BCK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    BCK(cudaGraphCreate(&h->graph, 0));
    cudaGraphConditionalHandle ch;
    BCK(cudaGraphConditionalHandleCreate(&ch, h->graph, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = ch;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    BCK(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    BCK(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    sstep_status st = batch_outer(h, h->cap_stream);
    if (st == SSTEP_OK) st = batch_outer_update(h, x, h->cap_stream);
    cudaError_t e = st == SSTEP_OK ? launch_batch_cond(ch, h->running, h->cap_stream) : cudaSuccess;
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &captured);
    if (st != SSTEP_OK) { drop_graph(h); return st; }
    BCK(e);
    BCK(e2);
    BCK(cudaGraphInstantiate(&h->gexec, h->graph, 0));
    h->g_b = b;
    h->g_x = x;
    return SSTEP_OK;
}

}  // namespace

extern "C" {

sstep_status sstep_cg_batch_create(sstep_cg_batch_t* out, int count, const int* grids_h,
                                   const double* const* kappa_d, const sstep_cg_opts* opts, void* stream) {
    if (!out) return SSTEP_ERR_INVALID_ARG;
    *out = nullptr;
    sstep_cg_batch_t h = new (std::nothrow) sstep_cg_batch_s();
    if (!h) return SSTEP_ERR_OOM;
    auto fail = [&](sstep_status st) {
        set_global_error(h->err);
        sstep_cg_batch_destroy(h);
        return st;
    };
    sstep_cg_opts o;
    if (opts) o = *opts; else sstep_cg_default_opts(&o);
    if (count < 1 || !grids_h) { berr(h, "count must be >= 1 with a grid per system"); return fail(SSTEP_ERR_INVALID_ARG); }
    if (o.s < 1 || o.s > 16) { berr(h, "batched form: s = %d outside [1, 16]", o.s); return fail(SSTEP_ERR_INVALID_ARG); }
    if (o.nu < 1 || o.nu > 10000 || !(o.tol > 0.0) || !std::isfinite(o.tol) || o.max_outer < 0 || o.max_refresh < 0 ||
        o.check_every < 1) {
        berr(h, "invalid nu, tol, max_outer, max_refresh or check_every");
        return fail(SSTEP_ERR_INVALID_ARG);
    }
    if (o.gram_solver != SSTEP_GRAM_SOLVE_FGS && o.gram_solver != SSTEP_GRAM_SOLVE_CHOLESKY) {
        berr(h, "unknown gram_solver");
        return fail(SSTEP_ERR_INVALID_ARG);
    }
    if (o.precond != SSTEP_PRECOND_JACOBI || o.precision != SSTEP_PRECISION_FP64 || o.basis_start != SSTEP_START_R ||
        o.block_conjugate != 0 ||
        (o.gram_form != SSTEP_GRAM_FORM_DIRECT && o.gram_form != SSTEP_GRAM_FORM_MOMENTS)) {
        berr(h, "batched form: Jacobi, FP64 and p_0 = r only");
        return fail(SSTEP_ERR_UNSUPPORTED);
    }
    if (o.bounds_mode == SSTEP_BOUNDS_GIVEN && !(o.lambda_max > o.lambda_min && o.lambda_min >= 0.0 &&
                                                 std::isfinite(o.lambda_max))) {
        berr(h, "need 0 <= lambda_min < lambda_max");
        return fail(SSTEP_ERR_INVALID_ARG);
    }
    if (o.bounds_mode != SSTEP_BOUNDS_GIVEN && o.bounds_mode != SSTEP_BOUNDS_GERSH_LANCZOS10 &&
        o.bounds_mode != SSTEP_BOUNDS_LANCZOS10) {
        berr(h, "unknown bounds_mode %d", o.bounds_mode);
        return fail(SSTEP_ERR_INVALID_ARG);
    }
    if (o.batch_chunk < 0 || (o.batch_chunk > 0 && o.batch_chunk < 256) || o.batch_ctas_per_sm < 0 ||
        o.batch_ctas_per_sm > 8) {
        berr(h, "batch_chunk must be 0 or >= 256; batch_ctas_per_sm in [0, 8]");
        return fail(SSTEP_ERR_INVALID_ARG);
    }
    const int64_t CHUNK = o.batch_chunk > 0 ? o.batch_chunk : 8192;
    h->count = count;
    h->opts = o;
    h->stream = (cudaStream_t)stream;
    // layout: systems back to back, each padded to 32 elements; tiles and chunks per system
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        const int dim = grids_h[4 * i], nx = grids_h[4 * i + 1], ny = grids_h[4 * i + 2], nz = grids_h[4 * i + 3];
        if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1)) {
            berr(h, "system %d: bad grid dim %d, %d x %d x %d", i, dim, nx, ny, nz);
            return fail(SSTEP_ERR_INVALID_ARG);
        }
        BSys sy{};
        sy.dim = dim;
        sy.nx = nx;
        sy.ny = ny;
        sy.nz = nz;
        sy.n = (int64_t)nx * ny * nz;
        sy.off = off;
        sy.poisson = (kappa_d == nullptr || kappa_d[i] == nullptr) ? 1 : 0;
        off += (sy.n + 31) / 32 * 32;
        sy.tile0 = (int)h->tiles.size();
        // 3D tile: 32 x 8 points x 8 planes; 2D tile: 32 x 64 points (8 row groups of 8)
        for (int k0 = 0; k0 < nz; k0 += (dim == 3 ? BT_Z : 1))
            for (int j0 = 0; j0 < ny; j0 += (dim == 3 ? BT_Y : BT_Y * BT_Z))
                for (int i0 = 0; i0 < nx; i0 += BT_X) h->tiles.push_back(BTile{i, i0, j0, k0});
        sy.tile1 = (int)h->tiles.size();
        sy.chunk0 = (int)h->chunks.size();
        for (int64_t e0 = 0; e0 < sy.n; e0 += CHUNK) h->chunks.push_back(BChunk{i, 0, e0, std::min(sy.n, e0 + CHUNK)});
        sy.chunk1 = (int)h->chunks.size();
        h->sys.push_back(sy);
    }
    h->ld = off;
    const int64_t ld = h->ld;
    const int s = o.s;
    if (cudaMalloc(&h->arrays, sizeof(double) * 5 * ld) != cudaSuccess ||
        cudaMalloc(&h->P, sizeof(double) * (s + 1) * ld) != cudaSuccess ||
        cudaMalloc(&h->rtrue, sizeof(double) * ld) != cudaSuccess ||
        cudaMalloc(&h->gram_partials, sizeof(double) * h->chunks.size() * batch_gram_m(s)) != cudaSuccess ||
        cudaMalloc(&h->tile_partials, sizeof(double) * h->tiles.size()) != cudaSuccess ||
        cudaMalloc(&h->ctl, sizeof(Ctl) * count) != cudaSuccess || cudaMalloc(&h->running, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&h->ctl_h, sizeof(Ctl) * count) != cudaSuccess ||
        cudaMallocHost(&h->running_h, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&h->sys_d, sizeof(BSys) * count) != cudaSuccess ||
        cudaMalloc(&h->tiles_d, sizeof(BTile) * h->tiles.size()) != cudaSuccess ||
        cudaMalloc(&h->chunks_d, sizeof(BChunk) * h->chunks.size()) != cudaSuccess ||
        cudaMalloc(&h->act, sizeof(int) * (3 * count + 5)) != cudaSuccess) {
        berr(h, "batched form: out of device memory (%lld unknowns)", (long long)ld);
        return fail(SSTEP_ERR_OOM);
    }
    cudaStream_t st = h->stream;
    double* wx = h->arrays;
    double* wy = wx + ld;
    double* wz = wy + ld;
    double* dg = wz + ld;
    double* cd = dg + ld;
    int* bad = nullptr;
    if (cudaMalloc(&bad, sizeof(int)) != cudaSuccess) return fail(SSTEP_ERR_OOM);
    cudaMemsetAsync(bad, 0, sizeof(int), st);
    cudaMemsetAsync(h->arrays, 0, sizeof(double) * 5 * ld, st);
    cudaMemsetAsync(h->ctl, 0, sizeof(Ctl) * count, st);
    for (int i = 0; i < count; ++i) {
        BSys& sy = h->sys[i];
        if (!sy.poisson)
            if (launch_stencil_faces(sy.dim, sy.nx, sy.ny, sy.nz, kappa_d[i], wx + sy.off, wy + sy.off, wz + sy.off,
                                     dg + sy.off, bad, st) != cudaSuccess) {
                cudaFree(bad);
                berr(h, "system %d: face set-up failed", i);
                return fail(SSTEP_ERR_CUDA);
            }
    }
    int hb = 0;
    cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(bad);
    if (e != cudaSuccess) { berr(h, "set-up: %s", cudaGetErrorString(e)); return fail(SSTEP_ERR_CUDA); }
    if (hb) { berr(h, "kappa must be positive and finite"); return fail(SSTEP_ERR_INVALID_ARG); }
    // per-system spectral bounds (given, or estimated as for a single handle), 2 theta / diag
    for (int i = 0; i < count; ++i) {
        BSys& sy = h->sys[i];
        double lmin = o.lambda_min, lmax = o.lambda_max;
        if (o.bounds_mode != SSTEP_BOUNDS_GIVEN) {
            OpDesc op{};
            op.kind = OP_STENCIL;
            op.n = sy.n;
            op.dim = sy.dim;
            op.nx = sy.nx;
            op.ny = sy.ny;
            op.nz = sy.nz;
            op.dconst = 2.0 * sy.dim;
            if (!sy.poisson) {
                op.wx = wx + sy.off;
                op.wy = wy + sy.off;
                op.wz = wz + sy.off;
                op.diag = dg + sy.off;
            }
            char msg[256] = {0};
            sstep_status bst = estimate_bounds(op, sy.poisson ? nullptr : dg + sy.off, true, o, st, &lmin, &lmax, msg,
                                               sizeof(msg));
            if (bst != SSTEP_OK) { berr(h, "system %d bounds: %s", i, msg); return fail(bst); }
        }
        sy.theta = 2.0 / (lmax - lmin);
        sy.sigma = 0.5 * (lmax + lmin);
        if (!sy.poisson && launch_scale_vec(dg + sy.off, 2.0 * sy.theta, cd + sy.off, sy.n, st) != cudaSuccess) {
            berr(h, "system %d: 2 theta / diag failed", i);
            return fail(SSTEP_ERR_CUDA);
        }
    }
    if (cudaMemcpyAsync(h->sys_d, h->sys.data(), sizeof(BSys) * count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(h->tiles_d, h->tiles.data(), sizeof(BTile) * h->tiles.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(h->chunks_d, h->chunks.data(), sizeof(BChunk) * h->chunks.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        berr(h, "batched form: descriptor upload failed");
        return fail(SSTEP_ERR_CUDA);
    }
    *out = h;
    return SSTEP_OK;
}

sstep_status sstep_cg_batch_layout(sstep_cg_batch_t h, int64_t* offsets_h, int64_t* total, double* lambda_h) {
    if (!h) return SSTEP_ERR_INVALID_ARG;
    for (int i = 0; i < h->count; ++i) {
        if (offsets_h) offsets_h[i] = h->sys[i].off;
        if (lambda_h) {
            const double half = 1.0 / h->sys[i].theta;   // (lmax - lmin) / 2
            lambda_h[2 * i] = h->sys[i].sigma - half;
            lambda_h[2 * i + 1] = h->sys[i].sigma + half;
        }
    }
    if (total) *total = h->ld;
    return SSTEP_OK;
}

sstep_status sstep_cg_batch_solve(sstep_cg_batch_t h, const double* b_d, double* x_d, sstep_cg_info* infos_h,
                                  sstep_cg_info* summary) {
    if (!h || !b_d || !x_d) return SSTEP_ERR_INVALID_ARG;
    cudaStream_t st = h->stream;
    const int count = h->count;
    const BatchDev B = dev_view(h);
    SolveEvents tev;
    BCK(cudaEventCreate(&tev.e0));
    BCK(cudaEventCreate(&tev.e1));
    BCK(cudaEventRecord(tev.e0, st));
    BCK(launch_batch_init(B, h->opts.tol * h->opts.tol, h->opts.max_outer, st));
    BCK(launch_batch_residual(B, b_d, x_d, h->P, 0, st));
    std::vector<int> refreshes(count, 0);
    long launches = 2;
    const int per_outer = h->opts.s + 3;
    for (;;) {
        if (h->opts.use_graph) {
            if (!h->gexec || h->g_b != b_d || h->g_x != x_d) {
                sstep_status gs = build_graph(h, b_d, x_d);
                if (gs != SSTEP_OK) return gs;
            }
            BCK(cudaGraphLaunch(h->gexec, st));
            BCK(cudaMemcpyAsync(h->running_h, h->running, sizeof(int), cudaMemcpyDeviceToHost, st));
            BCK(cudaStreamSynchronize(st));
        } else {
            for (;;) {
                for (int m = 0; m < h->opts.check_every; ++m) {
                    sstep_status os = batch_outer(h, st);
                    if (os == SSTEP_OK) os = batch_outer_update(h, x_d, st);
                    if (os != SSTEP_OK) return os;
                    launches += per_outer;
                }
                BCK(cudaMemcpyAsync(h->running_h, h->running, sizeof(int), cudaMemcpyDeviceToHost, st));
                BCK(cudaStreamSynchronize(st));
                if (*h->running_h == 0) break;
            }
        }
        // true residual of every system; restart the ones whose recursive residual converged
        // but whose true residual did not (at most max_refresh times each)
        BCK(launch_batch_residual(B, b_d, x_d, h->rtrue, 1, st));
        ++launches;
        BCK(cudaMemcpyAsync(h->ctl_h, h->ctl, sizeof(Ctl) * count, cudaMemcpyDeviceToHost, st));
        BCK(cudaStreamSynchronize(st));
        int restart = 0;
        for (int i = 0; i < count; ++i) {
            Ctl& c = h->ctl_h[i];
            const bool ok = c.r0_sq == 0.0 || c.true_sq < c.tol_sq * c.r0_sq;
            if (c.done == CONVERGED && !ok && refreshes[i] < h->opts.max_refresh) {
                ++refreshes[i];
                ++restart;
                const BSys& sy = h->sys[i];
                BCK(cudaMemcpyAsync(h->P + sy.off, h->rtrue + sy.off, sizeof(double) * sy.n, cudaMemcpyDeviceToDevice, st));
                const int running = RUNNING;
                BCK(cudaMemcpyAsync(&h->ctl[i].done, &running, sizeof(int), cudaMemcpyHostToDevice, st));
            }
        }
        if (!restart) break;
        BCK(cudaMemcpyAsync(h->running, &restart, sizeof(int), cudaMemcpyHostToDevice, st));
        BCK(cudaStreamSynchronize(st));
    }
    BCK(cudaEventRecord(tev.e1, st));
    BCK(cudaEventSynchronize(tev.e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tev.e0, tev.e1);
    sstep_status overall = SSTEP_OK;
    int max_outer = 0, n_ok = 0;
    double worst = 0.0;
    for (int i = 0; i < count; ++i) {
        const Ctl& c = h->ctl_h[i];
        sstep_cg_info inf{};
        const bool ok = c.r0_sq == 0.0 || c.true_sq < c.tol_sq * c.r0_sq;
        sstep_status stt = SSTEP_OK;
        if (c.done == NUMERICAL) stt = SSTEP_ERR_NUMERICAL;
        else if (c.done == MAX_OUTER || !ok) stt = SSTEP_ERR_NO_CONVERGENCE;
        inf.outer_iters = c.outer;
        inf.refreshes = refreshes[i];
        inf.status = stt;
        inf.r0_norm = std::sqrt(c.r0_sq);
        inf.rel_res_recursive = c.r0_sq > 0 ? std::sqrt(c.rk_sq / c.r0_sq) : 0.0;
        inf.rel_res_true = c.r0_sq > 0 ? std::sqrt(c.true_sq / c.r0_sq) : 0.0;
        inf.lambda_min_used = h->sys[i].sigma - 1.0 / h->sys[i].theta;
        inf.lambda_max_used = h->sys[i].sigma + 1.0 / h->sys[i].theta;
        inf.min_gii = c.min_gii;
        inf.delta_last = c.delta;
        inf.ms = ms;
        if (infos_h) infos_h[i] = inf;
        if (stt != SSTEP_OK && overall == SSTEP_OK) overall = stt;
        if (stt == SSTEP_OK) ++n_ok;
        max_outer = std::max(max_outer, c.outer);
        worst = std::max(worst, inf.rel_res_true);
    }
    if (summary) {
        sstep_cg_info sm{};
        sm.outer_iters = max_outer;
        sm.status = overall;
        sm.rel_res_true = worst;
        sm.ms = ms;
        sm.kernel_launches = (int)std::min<long>(launches, 2147483647L);
        *summary = sm;
    }
    if (overall != SSTEP_OK) berr(h, "%d of %d systems did not reach tol (%s)", count - n_ok, count, sstep_cg_status_string(overall));
    return overall;
}

sstep_status sstep_cg_batch_destroy(sstep_cg_batch_t h) {
    if (!h) return SSTEP_OK;
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->arrays);
    cudaFree(h->P);
    cudaFree(h->rtrue);
    cudaFree(h->gram_partials);
    cudaFree(h->tile_partials);
    cudaFree(h->ctl);
    cudaFree(h->running);
    cudaFree(h->sys_d);
    cudaFree(h->tiles_d);
    cudaFree(h->chunks_d);
    cudaFree(h->act);
    if (h->ctl_h) cudaFreeHost(h->ctl_h);
    if (h->running_h) cudaFreeHost(h->running_h);
    delete h;
    return SSTEP_OK;
}

const char* sstep_cg_batch_last_error(sstep_cg_batch_t h) { return h ? h->err : sstep_cg_last_error(nullptr); }

}  // extern "C"
