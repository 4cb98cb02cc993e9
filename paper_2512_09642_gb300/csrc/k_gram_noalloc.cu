// sstep_gram_fgs_noalloc: the fused Gram reduction + column scaling + FGS of an outer
// iteration for callers that cannot allocate device memory. The kernel is the same one
// sstep_cg_solve and sstep_cg_gram_solve launch; only the scratch differs: the per-block
// partial sums and the control block live in one file-scope device array instead of memory
// a handle allocated.
//
// Who needs it: code that must not call cudaMalloc/cudaFree while it runs, for example
// because a caching allocator already owns (nearly) all of the device's memory, or because
// cudaMalloc and cudaFree can synchronise the device and stall a latency-bound loop.
//
// The array (NOALLOC_SCRATCH_BYTES, about 224 KB) is part of the library image: every GPU
// that loads the library holds it until the process exits. Its device address is looked up
// per device with that device current (cudaGetSymbolAddress): on the device's first call, and
// again on every call whose stream is not capturing, since a device reset reloads the module
// and moves the array; a call made during stream capture uses the address of the device's
// last call outside capture, so make a first call before any capture, and one after any
// device reset before capturing again. Each device has its own copy,
// so calls on different devices do not interact. On one device all calls share the array,
// which keeps the last call's contents: each call first re-initialises the control block
// (including the block-arrival counter, which must start at zero), and calls whose work can
// overlap on the GPU (for example on two streams) race on the array - serialise them.
#include <cstdio>
#include <mutex>

#include "kernels.h"

namespace sstep {

void set_global_error(const char* msg);

namespace {

constexpr int NOALLOC_MAX_S = 16;
constexpr int NOALLOC_MAX_BLOCKS = 160;
constexpr int NOALLOC_MAX_M = NOALLOC_MAX_S * (NOALLOC_MAX_S + 1) / 2 + 2 * NOALLOC_MAX_S;   // 168
constexpr size_t CTL_BYTES = (sizeof(Ctl) + 255) / 256 * 256;
constexpr size_t PARTIAL_BYTES = sizeof(double) * NOALLOC_MAX_BLOCKS * NOALLOC_MAX_M;
constexpr size_t NOALLOC_SCRATCH_BYTES = CTL_BYTES + PARTIAL_BYTES;

// [ Ctl | per-block partials ]; every GPU that loads the library holds one copy.
static __device__ __align__(256) unsigned char g_gram_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};
int g_sm_count[MAX_DEVICES] = {};

__global__ void k_noalloc_init(Ctl* ctl) {
    // What the Gram kernel reads before writing: the arrival counter, the termination state
    // and the stopping inputs (no stopping test here: r0 = 1, tol = 0, one outer allowed).
    ctl->counter = 0u;
    ctl->counter2 = 0u;
    ctl->done = RUNNING;
    ctl->outer = 0;
    ctl->max_outer = 1;
    ctl->r0_sq = 1.0;
    ctl->tol_sq = 0.0;
    ctl->rk_sq = 0.0;
    ctl->min_gii = INFINITY;
    ctl->delta = 0.0;
    ctl->scale = 1.0;
    ctl->scale_next = 1.0;
}

// Copies the results out of the shared control block. A solve that stopped early (numerical
// breakdown) wrote none of them, so the scratch still holds an earlier call's values: the
// outputs are then NaN, never another system's numbers.
__global__ void k_noalloc_export(const Ctl* ctl, int s, double* out) {
    const bool ok = ctl->done == RUNNING;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
        out[i] = ok ? ctl->alpha[i] : nan;
        out[s + i] = ok ? ctl->d[i] : nan;
        out[2 * s + i] = ok ? ctl->ct[i] : nan;
    }
    for (int i = threadIdx.x; i < s * s; i += blockDim.x) out[3 * s + i] = ok ? ctl->Gt[i] : nan;
    if (threadIdx.x == 0) out[3 * s + s * s] = (double)ctl->done;
}

}  // namespace

}  // namespace sstep

using namespace sstep;

extern "C" sstep_status sstep_gram_fgs_noalloc(int64_t n, int s, int nu, int gram_solver, const double* P_d,
                                               int64_t ldp, const double* mdiag_d, double mconst, double lambda_min,
                                               double lambda_max, double* out_d, void* stream) {
    if (s < 1 || s > NOALLOC_MAX_S) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "sstep_gram_fgs_noalloc: s = %d outside [1, %d] (its static scratch holds "
                      "the partial sums of s <= %d)", s, NOALLOC_MAX_S, NOALLOC_MAX_S);
        set_global_error(msg);
        return SSTEP_ERR_INVALID_ARG;
    }
    if (n < 1 || ldp < n || nu < 1 || nu > 10000 || !P_d || !out_d ||
        (gram_solver != SSTEP_GRAM_SOLVE_FGS && gram_solver != SSTEP_GRAM_SOLVE_CHOLESKY) ||
        !(lambda_max > lambda_min) || !(lambda_min >= 0.0) || (!mdiag_d && !(mconst > 0.0))) {
        set_global_error("sstep_gram_fgs_noalloc: invalid argument (n, ldp >= n, nu, solver, bounds, P, out, "
                         "or M: mdiag or a positive mconst)");
        return SSTEP_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        set_global_error("sstep_gram_fgs_noalloc: no usable current device");
        return SSTEP_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    int sms = 0;
    cudaStream_t st = (cudaStream_t)stream;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cap);
        if (e != cudaSuccess) {
            set_global_error("sstep_gram_fgs_noalloc: cudaStreamIsCapturing failed");
            return SSTEP_ERR_CUDA;
        }
        if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
            if (cap != cudaStreamCaptureStatusNone) {
                set_global_error("sstep_gram_fgs_noalloc: the first call on a device must come before stream capture");
                return SSTEP_ERR_INVALID_ARG;
            }
            // this device is current: the host-side symbol is only a stand-in, kernels need the
            // device address (looked up again outside capture: a device reset moves the array)
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_gram_scratch);
            if (e != cudaSuccess) {
                set_global_error("sstep_gram_fgs_noalloc: cudaGetSymbolAddress of the static scratch failed");
                return SSTEP_ERR_CUDA;
            }
            e = cudaDeviceGetAttribute(&g_sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) {
                set_global_error("sstep_gram_fgs_noalloc: cudaDeviceGetAttribute failed");
                return SSTEP_ERR_CUDA;
            }
            g_scratch_addr[dev] = (unsigned char*)p;
        }
        base = g_scratch_addr[dev];
        sms = g_sm_count[dev];
    }
    Ctl* ctl = (Ctl*)base;
    double* partials = (double*)(base + CTL_BYTES);

    const double theta = 2.0 / (lambda_max - lambda_min);
    const double sigma = 0.5 * (lambda_max + lambda_min);
    GramArgs g{};
    g.s = s;
    g.nu = nu;
    g.solver = gram_solver;
    g.form = SSTEP_GRAM_FORM_DIRECT;
    g.theta = theta;
    g.sigma = sigma;
    g.dvec = mdiag_d != nullptr;
    g.dconst = mdiag_d ? 1.0 : mconst;
    g.diag = mdiag_d;
    g.n = n;
    g.ld = ldp;
    g.P = P_d;
    g.fp32 = false;
    g.check = 1;
    int nblk = gram_blocks(g, sms < NOALLOC_MAX_BLOCKS ? sms : NOALLOC_MAX_BLOCKS);
    if (nblk > NOALLOC_MAX_BLOCKS) nblk = NOALLOC_MAX_BLOCKS;

    k_noalloc_init<<<1, 1, 0, st>>>(ctl);
    if ((e = cudaGetLastError()) == cudaSuccess) e = launch_gram(g, partials, ctl, nblk, st);
    if (e == cudaSuccess) {
        k_noalloc_export<<<1, 256, 0, st>>>(ctl, s, out_d);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_global_error("sstep_gram_fgs_noalloc: kernel launch failed");
        return SSTEP_ERR_CUDA;
    }
    return SSTEP_OK;
}
