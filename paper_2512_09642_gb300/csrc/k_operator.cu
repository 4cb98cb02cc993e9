// Operator kernels: the Chebyshev matrix-powers step (Section 2, Definition "Chebyshev
// Polynomial Basis"), r = b - A x with its norm, and y = A x, for CSR matrices and for the
// matrix-free 5-/7-point Poisson, 9-/27-point box Poisson (Section 8's operator) and
// cell-centred diffusion stencils.
//
// GB300 notes: FP64 issues at ~1/74 of the FP32 rate on this part, so the FP64 forms are
// written to minimise FP64 instructions per unknown (7-point step: 5 adds + 2 FMAs; 27-point
// step: about 9 operations through separable box sums), and every index is computed from
// the launch grid, never by 64-bit division. Stencil kernels march along z with the
// z-neighbours (or z-plane sums) held in registers. The 5-/7-point and diffusion kernels read
// their x/y neighbours through L1 (staging planes in shared memory made them slower: the
// barriers expose each plane's load latency); the box kernels stage each plane with its
// halo in shared memory, where it serves 9 products per point.
#include <type_traits>

#include "kernels.h"

namespace sstep {

namespace {

constexpr int BX = 32, BY = 8, KC = 8;      // stencil block (x, y) and z planes per block
// z planes per block of the 5/7-point and diffusion kernels by precision: 8 for the FP64
// steps, 16 for the FP32 steps and the FP64 residual (measured at 256^3: the FP32 step 42.6 ->
// 40.8 us, the mixed refresh 0.284 -> 0.268 ms with 16; the FP64 step 0.233 -> 0.242 ms with
// 16, 0.233 with 4); KC for the rest
template <typename T> constexpr int kz_step() { return sizeof(T) == 4 ? 16 : 8; }
constexpr int KZ_RES = 16;
constexpr int RB = 256;                      // CSR / vector kernels: threads per block

template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// a + b written as fma(a, one, b) with one = 1 passed at run time (so the compiler cannot fold
// it back into an add): the same correctly rounded sum, bit for bit, but this part issues FP64
// FMAs at 627 G/s and FP64 adds at only 528 G/s (measured with independent chains at full
// occupancy), so the FP64-pipe bound stencils run their additions as FMAs.
template <typename T> __device__ __forceinline__ T add1(T a, T b, T one) { return fma(a, one, b); }

// Fused moments (gram_form FUSED): the step that writes p_(j+1) also reduces a_j = <p_j, p_j>
// and b_j = <p_j, p_(j+1)> (unweighted; M is a constant multiple of I), from which the Gram
// finish forms every Chebyshev moment, so no pass re-reads the basis. Per-thread sums in the
// step's precision over the thread's points (2 per plane for the pair kernel, over 8 planes
// in FP64 and 16 in FP32; 8 or 16 otherwise), then a fixed
// warp butterfly and a fixed order over the block's warps; one partial per block and value:
// FP64 double[2][nblk] (a, b), FP32 float[4][nblk] (a_hi, a_lo, b_hi, b_lo). In FP32 the
// per-thread sums are plain FMAs (their rounding is independent from thread to thread, so
// the million per-thread errors of about 1e-7 average out in the FP64 total) and everything
// from the warp butterfly on is exact pair arithmetic (TwoSum on the high parts); the FP32
// form adds no FP64 instruction to the step.
template <typename T> struct MomAcc;
template <> struct MomAcc<double> {
    double a = 0.0, b = 0.0;
    __device__ __forceinline__ void add(double pj, double pn) {
        a = fma(pj, pj, a);
        b = fma(pj, pn, b);
    }
};
template <> struct MomAcc<float> {
    float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
    __device__ __forceinline__ void add(float pj, float pn) {
        ah = fmaf(pj, pj, ah);
        bh = fmaf(pj, pn, bh);
    }
};

// (h, l) += (h2, l2): TwoSum on the high parts, the low parts and the error summed.
__device__ __forceinline__ void pair_add(float& h, float& l, float h2, float l2) {
    float t, e;
    two_sum(h, h2, t, e);
    h = t;
    l = __fadd_rn(__fadd_rn(l, l2), e);
}

// Block reduction of the accumulators and the store of this block's partials. Every thread
// of the block calls it (blocks of NT threads, 32 in x; any grid shape).
template <int NT = BX * BY>
__device__ __forceinline__ void mom_block_store(const MomAcc<double>& m, void* part, int nblk) {
    __shared__ double sh[NT / 32][2];
    const int t = threadIdx.x + BX * threadIdx.y, lane = t & 31, w = t >> 5;
    // lanes of even index carry a, odd ones b after the first exchange: one FP64 add per level
    double v = (lane & 1) ? m.b : m.a;
    const double give = (lane & 1) ? m.a : m.b;
    v += __shfl_xor_sync(0xffffffffu, give, 1);
#pragma unroll
    for (int o = 2; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane < 2) sh[w][lane] = v;
    __syncthreads();
    if (t < 2) {
        double acc = sh[0][t];
#pragma unroll
        for (int k = 1; k < NT / 32; ++k) acc += sh[k][t];
        const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        ((double*)part)[(size_t)t * nblk + blk] = acc;
    }
}

template <int NT = BX * BY>
__device__ __forceinline__ void mom_block_store(const MomAcc<float>& m, void* part, int nblk) {
    __shared__ float sh[NT / 32][4];
    const int t = threadIdx.x + BX * threadIdx.y, lane = t & 31, w = t >> 5;
    float ah = m.ah, al = m.al, bh = m.bh, bl = m.bl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pair_add(ah, al, __shfl_xor_sync(0xffffffffu, ah, o), __shfl_xor_sync(0xffffffffu, al, o));
        pair_add(bh, bl, __shfl_xor_sync(0xffffffffu, bh, o), __shfl_xor_sync(0xffffffffu, bl, o));
    }
    if (lane == 0) {
        sh[w][0] = ah;
        sh[w][1] = al;
        sh[w][2] = bh;
        sh[w][3] = bl;
    }
    __syncthreads();
    if (w == 0) {
        // the block's warps, lane k holding warp k's pairs: a butterfly over lanes 0..NW-1
        constexpr int NW = NT / 32;
        static_assert(NW >= 2 && NW <= 32 && (NW & (NW - 1)) == 0, "warps per block: a power of 2 up to 32");
        const bool has = lane < NW;
        ah = has ? sh[lane][0] : 0.f;
        al = has ? sh[lane][1] : 0.f;
        bh = has ? sh[lane][2] : 0.f;
        bl = has ? sh[lane][3] : 0.f;
#pragma unroll
        for (int o = NW / 2; o > 0; o >>= 1) {
            pair_add(ah, al, __shfl_xor_sync(0xffffffffu, ah, o), __shfl_xor_sync(0xffffffffu, al, o));
            pair_add(bh, bl, __shfl_xor_sync(0xffffffffu, bh, o), __shfl_xor_sync(0xffffffffu, bl, o));
        }
    }
    if (t == 0) {
        const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        float* pf = (float*)part;
        pf[blk] = ah;
        pf[(size_t)nblk + blk] = al;
        pf[2 * (size_t)nblk + blk] = bh;
        pf[3 * (size_t)nblk + blk] = bl;
    }
}


// Face weights of the diffusion stencil in precision T.
template <typename T> struct Faces { const T* wx; const T* wy; const T* wz; const T* diag; const T* cdinv; };

// (A p)_e of the diffusion stencil split as diag_e p_e - s, with s = sum_f w_f p_nbr(f).
template <typename T, int DIM>
__device__ __forceinline__ T diffusion_offdiag_sum(const T* __restrict__ p, const Faces<T>& f, int64_t e, int i,
                                                   int j, int k, int nx, int ny, int nz, int64_t sxy, T pdn, T pup) {
    T s = (i > 0) ? ldg(f.wx + e - 1) * ldg(p + e - 1) : T(0);
    if (i < nx - 1) s = fma(ldg(f.wx + e), ldg(p + e + 1), s);
    if (j > 0) s = fma(ldg(f.wy + e - nx), ldg(p + e - nx), s);
    if (j < ny - 1) s = fma(ldg(f.wy + e), ldg(p + e + nx), s);
    if (DIM == 3) {
        if (k > 0) s = fma(ldg(f.wz + e - sxy), pdn, s);
        if (k < nz - 1) s = fma(ldg(f.wz + e), pup, s);
    }
    return s;
}

// Chebyshev step on a structured grid. POISSON: out = c1 p + c2 sum(nbrs) - q with the
// constants folded on the host. Diffusion: out = c1 p - cdv_e s - q (Jacobi, cdv_e = c /
// diag_e) or out = c ((diag_e - sigma) p - s) - q (no preconditioner). GRAM: also the fused
// moments a_j, b_j of this block (mom: this step's partials, nblk blocks in the grid).
template <typename T, int DIM, bool POISSON, bool JACOBI, bool FIRST, bool GRAM, int KZ = kz_step<T>()>
__global__ void __launch_bounds__(BX* BY) k_cheb_stencil(const T* __restrict__ p, const T* __restrict__ q,
                                                         T* __restrict__ out, int nx, int ny, int nz, Faces<T> f,
                                                         T c1, T c2, T csig, T cscale, const Ctl* __restrict__ ctl,
                                                         T one, void* mom, int nblk) {
    if (ctl->done) return;
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    MomAcc<T> acc;
    if (i < nx && j < ny) {
        const int64_t sxy = (int64_t)nx * ny;
        const int k0 = (DIM == 3) ? blockIdx.z * KZ : 0;
        const int k1 = (DIM == 3) ? min(nz, k0 + KZ) : 1;
        int64_t e = i + (int64_t)nx * j + sxy * k0;
        T pdn = (DIM == 3 && k0 > 0) ? ldg(p + e - sxy) : T(0);
        T pc = ldg(p + e);
#pragma unroll 2
        for (int k = k0; k < k1; ++k, e += sxy) {
            const T pup = (DIM == 3 && k < nz - 1) ? ldg(p + e + sxy) : T(0);
            const T qv = FIRST ? T(0) : ldg(q + e);
            T o;
            if (POISSON) {
                // neighbour sum as a depth-3 tree (x pair, y pair, z pair): same 5 adds, shorter chain
                const T xm = (i > 0) ? ldg(p + e - 1) : T(0);
                const T xp = (i < nx - 1) ? ldg(p + e + 1) : T(0);
                const T ym = (j > 0) ? ldg(p + e - nx) : T(0);
                const T yp = (j < ny - 1) ? ldg(p + e + nx) : T(0);
                T s = add1(add1(xm, xp, one), add1(ym, yp, one), one);
                if (DIM == 3) s = add1(s, add1(k > 0 ? pdn : T(0), k < nz - 1 ? pup : T(0), one), one);
                o = FIRST ? fma(c2, s, c1 * pc) : fma(c2, s, fma(c1, pc, -qv));
            } else {
                const T s = diffusion_offdiag_sum<T, DIM>(p, f, e, i, j, k, nx, ny, nz, sxy, pdn, pup);
                if (JACOBI) {
                    T cdv = ldg(f.cdinv + e);
                    if (FIRST) cdv *= cscale;
                    o = FIRST ? fma(-cdv, s, c1 * pc) : fma(-cdv, s, fma(c1, pc, -qv));
                } else {
                    const T t = fma(ldg(f.diag + e) - csig, pc, -s);
                    o = FIRST ? c1 * t : fma(c1, t, -qv);
                }
            }
            out[e] = o;
            if (GRAM) acc.add(pc, o);
            pdn = pc;
            pc = pup;
        }
    }
    if (GRAM) mom_block_store(acc, mom, nblk);
}

// Poisson step with each thread on two x-adjacent points (nx even): 16-byte (8-byte in FP32)
// loads and stores of the pair, the x-neighbours from the adjacent lanes by warp shuffles
// (the warp's two edge points from memory), so a point costs 3 load instructions instead of
// 6. Measured at 256^3: FP32 (HBM-bound) 0.0448 -> 0.0398 ms per step; FP64 unchanged (the
// FP64 pipe stays the limit). Same sums in the same order as k_cheb_stencil.
template <typename T> struct Pair;
template <> struct Pair<double> { using type = double2; };
template <> struct Pair<float> { using type = float2; };

template <typename T, int DIM, bool FIRST, bool GRAM, int KZ = kz_step<T>()>
__global__ void __launch_bounds__(BX* BY) k_cheb_poisson_pair(const T* __restrict__ p, const T* __restrict__ q,
                                                              T* __restrict__ out, int nx, int ny, int nz, T c1, T c2,
                                                              const Ctl* __restrict__ ctl, T one, void* mom, int nblk) {
    if (ctl->done) return;
    using V = typename Pair<T>::type;
    const int lane = threadIdx.x;   // BX = 32: one warp per row of the tile
    const int i0 = blockIdx.x * (2 * BX);
    const int i = i0 + 2 * lane;
    const int j = blockIdx.y * BY + threadIdx.y;
    const bool in = i < nx && j < ny;   // nx even: i + 1 < nx as well
    const int64_t sxy = (int64_t)nx * ny;
    const int k0 = (DIM == 3) ? blockIdx.z * KZ : 0;
    const int k1 = (DIM == 3) ? min(nz, k0 + KZ) : 1;
    const int64_t ij = in ? i + (int64_t)nx * j : 0;
    const V zero{T(0), T(0)};
    auto ld2 = [&](int64_t e) { return __ldg(reinterpret_cast<const V*>(p + e)); };
    V pdn = (DIM == 3 && in && k0 > 0) ? ld2(ij + sxy * (k0 - 1)) : zero;
    V pc = in ? ld2(ij + sxy * k0) : zero;
    MomAcc<T> acc;
    for (int k = k0; k < k1; ++k) {
        const int64_t e = ij + sxy * k;
        const V pup = (DIM == 3 && in && k < nz - 1) ? ld2(e + sxy) : zero;
        const V ym = (in && j > 0) ? ld2(e - nx) : zero;
        const V yp = (in && j < ny - 1) ? ld2(e + nx) : zero;
        const V qv = (FIRST || !in) ? zero : __ldg(reinterpret_cast<const V*>(q + e));
        // left of the pair: the lane below's right point; right of the pair: the lane above's
        // left point (0 from lanes outside the grid, which is the Dirichlet value there)
        T xl = __shfl_up_sync(0xffffffffu, pc.y, 1);
        T xr = __shfl_down_sync(0xffffffffu, pc.x, 1);
        if (lane == 0) xl = (in && i0 > 0) ? ldg(p + e - 1) : T(0);
        if (lane == BX - 1) xr = (in && i + 2 < nx) ? ldg(p + e + 2) : T(0);
        if (in) {
            T s0 = add1(add1(xl, pc.y, one), add1(ym.x, yp.x, one), one);
            T s1 = add1(add1(pc.x, xr, one), add1(ym.y, yp.y, one), one);
            if (DIM == 3) {
                s0 = add1(s0, add1(pdn.x, pup.x, one), one);
                s1 = add1(s1, add1(pdn.y, pup.y, one), one);
            }
            V o;
            o.x = FIRST ? fma(c2, s0, c1 * pc.x) : fma(c2, s0, fma(c1, pc.x, -qv.x));
            o.y = FIRST ? fma(c2, s1, c1 * pc.y) : fma(c2, s1, fma(c1, pc.y, -qv.y));
            *reinterpret_cast<V*>(out + e) = o;
            if (GRAM) {
                acc.add(pc.x, o.x);
                acc.add(pc.y, o.y);
            }
        }
        pdn = pc;
        pc = pup;
    }
    if (GRAM) mom_block_store(acc, mom, nblk);
}

// FP32 7-point step through tensor-map tiles (3D, nx a multiple of 4). The mixed form's FP32
// step is memory-bound and its loads wait on HBM: with the loads in registers the pair kernel
// runs at 0.78 of the measured HBM rate at 256^3. Here each block's 64 x 8 tile of a 32-plane
// slab arrives by TMA into a ring of STMA shared-memory stages tracked by mbarriers: plane k
// of p as a 72 x 10 box (x from i0 - 4, so the x coordinate stays on a 16-byte boundary, and
// y from j0 - 1; the hardware fills what lies outside the grid with zeros, the Dirichlet
// values) together with the tile of q. One thread issues the copies; every thread reads its
// pair, its x and y neighbours and the next plane's pair from shared memory. The sums and
// their order are those of k_cheb_poisson_pair (bitwise equal outputs). Every wait is bounded:
// one that expires sets ctl->done = TIMED_OUT, the block leaves the plane loop with all its
// threads, waits (bounded) for its copies in flight and returns. Measured at 256^3: 0.0382 ->
// 0.0349 ms per step, 0.0401 -> 0.0362 with the fused moments (0.86 and 0.83 of HBM); at
// 192^3, where a step's three vectors fit in L2, the pair kernel is faster (0.0144 against
// 0.0176 ms), so the host picks this kernel only when they do not.
constexpr int TMX = 64, TMY = 8, TMKZ = 32, STMA = 6;
constexpr int TPX = TMX + 8, TPY = TMY + 2;   // the p box: x from i0 - 4, y from j0 - 1
constexpr uint32_t TP_BYTES = TPX * TPY * 4, TQ_BYTES = TMX * TMY * 4;
constexpr int TP_STRIDE = (TP_BYTES + 127) / 128 * 128, TQ_STRIDE = (TQ_BYTES + 127) / 128 * 128;
constexpr int TSTAGE = TP_STRIDE + TQ_STRIDE;
constexpr long long TMA_WAIT_LIMIT = 1ll << 22;   // polls of one wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this thread's earlier generic accesses of shared memory before later TMA writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// false when the phase of the given parity has not completed after `limit` polls
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// SELFTEST (the self-test of the bounded waits only): every stage expects 16 bytes more than
// its copies deliver, so no wait completes, and a wait gives up after 4096 polls. The launch
// bound keeps 7 blocks resident per SM (the most its 30 KB of shared memory allows): at 34
// registers the fused step held 6 and ran 15% slower.
template <bool FIRST, bool GRAM, bool SELFTEST = false>
__global__ void __launch_bounds__(32 * TMY, 7) k_cheb_poisson_tma(const __grid_constant__ CUtensorMap tp,
                                                                  const __grid_constant__ CUtensorMap tq,
                                                                  float* __restrict__ out, int nx, int ny, int nz,
                                                                  float c1, float c2, Ctl* __restrict__ ctl, float one,
                                                                  void* mom, int nblk) {
    constexpr uint32_t extra_tx = SELFTEST ? 16u : 0u;
    constexpr long long wait_limit = SELFTEST ? 4096 : TMA_WAIT_LIMIT;
    if (ctl->done) return;
    __shared__ alignas(128) unsigned char sbuf[STMA * TSTAGE];
    __shared__ alignas(8) unsigned long long bar[STMA];
    __shared__ int aborted;
    const int lane = threadIdx.x, w = threadIdx.y, tid = lane + 32 * w;
    const int i0 = blockIdx.x * TMX, j0 = blockIdx.y * TMY;
    const int k0 = blockIdx.z * TMKZ, k1 = min(nz, k0 + TMKZ);
    const int npl = k1 - k0 + 2;   // planes k0 - 1 .. k1, plane t = k0 - 1 + t in stage t % STMA
    auto sp = [&](int t) { return reinterpret_cast<const float*>(sbuf + (t % STMA) * TSTAGE); };
    auto sq = [&](int t) { return reinterpret_cast<const float*>(sbuf + (t % STMA) * TSTAGE + TP_STRIDE); };
    auto issue = [&](int t) {
        const int s = t % STMA, kk = k0 - 1 + t;
        const bool wq = !FIRST && kk >= k0 && kk < k1;
        mbar_expect_tx(&bar[s], TP_BYTES + (wq ? TQ_BYTES : 0u) + extra_tx);
        tma_load_3d(sbuf + s * TSTAGE, &tp, i0 - 4, j0 - 1, kk, &bar[s]);
        if (wq) tma_load_3d(sbuf + s * TSTAGE + TP_STRIDE, &tq, i0, j0, kk, &bar[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < STMA; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
        aborted = 0;
    }
    __syncthreads();
    int issued = 0;   // thread 0's count of planes issued
    if (tid == 0) {
        issued = STMA < npl ? STMA : npl;
        for (int t = 0; t < issued; ++t) issue(t);
    }
    auto wait_plane = [&](int t) {
        if (!mbar_wait(&bar[t % STMA], (uint32_t)((t / STMA) & 1), wait_limit)) {
            aborted = 1;
            atomicExch(&ctl->done, (int)TIMED_OUT);
        }
    };
    const int i = i0 + 2 * lane, j = j0 + w;
    const bool in = i < nx && j < ny;   // nx even: i + 1 < nx as well
    const int cx = 4 + 2 * lane;        // the pair's column in the p box
    MomAcc<float> acc;
    wait_plane(0);
    float2 pdn = *reinterpret_cast<const float2*>(sp(0) + (w + 1) * TPX + cx);
    wait_plane(1);
    for (int k = k0; k < k1; ++k) {
        const int t = k - k0 + 1;
        wait_plane(t + 1);
        const float* P = sp(t);
        const float2 pc = *reinterpret_cast<const float2*>(P + (w + 1) * TPX + cx);
        const float xl = P[(w + 1) * TPX + cx - 1], xr = P[(w + 1) * TPX + cx + 2];
        const float2 ym = *reinterpret_cast<const float2*>(P + w * TPX + cx);
        const float2 yp = *reinterpret_cast<const float2*>(P + (w + 2) * TPX + cx);
        const float2 pup = *reinterpret_cast<const float2*>(sp(t + 1) + (w + 1) * TPX + cx);
        const float2 qv = FIRST ? make_float2(0.f, 0.f) : *reinterpret_cast<const float2*>(sq(t) + w * TMX + 2 * lane);
        if (in) {
            float s0 = add1(add1(xl, pc.y, one), add1(ym.x, yp.x, one), one);
            float s1 = add1(add1(pc.x, xr, one), add1(ym.y, yp.y, one), one);
            s0 = add1(s0, add1(pdn.x, pup.x, one), one);
            s1 = add1(s1, add1(pdn.y, pup.y, one), one);
            float2 o;
            o.x = FIRST ? fma(c2, s0, c1 * pc.x) : fma(c2, s0, fma(c1, pc.x, -qv.x));
            o.y = FIRST ? fma(c2, s1, c1 * pc.y) : fma(c2, s1, fma(c1, pc.y, -qv.y));
            *reinterpret_cast<float2*>(out + i + (int64_t)nx * j + (int64_t)nx * ny * k) = o;
            if (GRAM) {
                acc.add(pc.x, o.x);
                acc.add(pc.y, o.y);
            }
        }
        pdn = pc;
        __syncthreads();   // every thread is done with plane t: its stage takes plane t + STMA
        if (aborted) break;
        if (tid == 0 && issued < npl) {
            fence_proxy_async();
            issue(issued);
            ++issued;
        }
    }
    if (aborted && tid == 0)   // the copies in flight land before the block's shared memory goes
        for (int t = 0; t < issued; ++t) mbar_wait(&bar[t % STMA], (uint32_t)((t / STMA) & 1), wait_limit);
    if (GRAM) mom_block_store<32 * TMY>(acc, mom, nblk);
}

// CSR Chebyshev step, one thread per row: y = A p, out = cdv (y) - c sigma p - q. A warp's
// loads of vals / colind are strided by the row length, but the warp's rows share their
// cache lines, which L1 keeps between the row's iterations: measured at 0.95 (FP64) and 0.93
// (FP32) of the HBM rate for the 7-point matrix at 256^3. Staging each 256-row tile's entries
// in shared memory with coalesced loads first was measured 1.6x slower (its barriers expose
// the load latency).
template <typename T, bool FIRST, bool JACOBI>
__global__ void __launch_bounds__(RB) k_cheb_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                                 const T* __restrict__ vals, const T* __restrict__ cdinv,
                                                 const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ out,
                                                 int64_t n, T c, T csig, T cscale, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    for (int64_t r = blockIdx.x * (int64_t)RB + threadIdx.x; r < n; r += (int64_t)gridDim.x * RB) {
        const int32_t b = ldg(rowptr + r), en = ldg(rowptr + r + 1);
        T y = T(0);
        for (int32_t t = b; t < en; ++t) y = fma(ldg(vals + t), ldg(p + ldg(colind + t)), y);
        T cdv = JACOBI ? ldg(cdinv + r) : c;
        if (FIRST && JACOBI) cdv *= cscale;
        const T pc = ldg(p + r);
        out[r] = FIRST ? fma(cdv, y, -csig * pc) : fma(cdv, y, fma(-csig, pc, -ldg(q + r)));
    }
}

// Block-wide sum of one double per thread, result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < NT / 32; ++k) t += sh[k];
    return t;
}

// Power of two 2^-e with rms = sqrt(sq / n) in [2^(e-1), 2^e): applied to the FP32 copy of
// the residual so that its entries sit near 1 whatever the scale of b (mixed form).
__device__ double pow2_scale(double sq, int64_t n) {
    const double rms = sqrt(sq / (double)n);
    if (!(rms > 0.0) || !isfinite(rms)) return 1.0;
    int e = 0;
    frexp(rms, &e);
    return ldexp(1.0, -e);
}

// What the last block does with ||r||^2. mode 0: initial residual (r_0, and the first scale);
// 1: true residual at exit; 2: mixed-form refresh of an outer iteration (stopping test of
// Section 8 on the FP64 residual, scale bookkeeping).
__device__ void residual_epilogue(Ctl* ctl, int mode, double tot, int64_t n) {
    if (mode == 0) {
        ctl->r0_sq = tot;
        ctl->scale_next = pow2_scale(tot, n);
    } else if (mode == 1) {
        ctl->true_sq = tot;
    } else {
        ctl->rk_sq = tot;
        ctl->scale = ctl->scale_next;
        ctl->scale_next = pow2_scale(tot, n);
        int done = RUNNING;
        if (!isfinite(tot)) done = NUMERICAL;
        else if (ctl->r0_sq == 0.0 || tot < ctl->tol_sq * ctl->r0_sq) done = CONVERGED;
        else if (ctl->outer >= ctl->max_outer) done = MAX_OUTER;
        ctl->done = done;
    }
}

// Fixed-order sum of per-block partials by the last block to arrive (deterministic for a
// fixed grid), then the epilogue. `counter` is reset for the next launch.
__device__ void last_block_finish(double mine, double* partials, unsigned int* counter, Ctl* ctl, int mode,
                                  int64_t n, int nblk) {
    __shared__ bool last;
    __shared__ double sh[32];
    const int t = threadIdx.x + blockDim.x * threadIdx.y;   // blocks may be 2D
    if (t == 0) {
        partials[blockIdx.x + (size_t)gridDim.x * blockIdx.y + (size_t)gridDim.x * gridDim.y * blockIdx.z] = mine;
        __threadfence();
        const unsigned int prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned int)nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nt = blockDim.x * blockDim.y;
    double acc = 0.0;
    for (int k = t; k < nblk; k += nt) acc += ((volatile double*)partials)[k];
    acc = warp_sum(acc);
    if ((t & 31) == 0) sh[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double tot = 0.0;
        for (int k = 0; k < nt / 32; ++k) tot += sh[k];
        residual_epilogue(ctl, mode, tot, n);
        *counter = 0u;
    }
}

// r = b - A x (FP64) on the stencil, with ||r||^2.
template <int DIM, bool POISSON, int KZ = KZ_RES>
__global__ void __launch_bounds__(BX* BY) k_residual_stencil(const double* __restrict__ b, const double* __restrict__ x,
                                                             double* __restrict__ r, float* __restrict__ r32, int nx,
                                                             int ny, int nz, Faces<double> f, double d2,
                                                             double* partials, Ctl* ctl, int mode, double one) {
    if (mode == 2 && ctl->done) return;
    int kscale = 0;   // scale_next = 2^kscale
    if (mode == 2) {
        frexp(ctl->scale_next, &kscale);
        kscale -= 1;
    }
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const bool act = i < nx && j < ny;
    double ss = 0.0;
    if (act) {
        const int64_t sxy = (int64_t)nx * ny;
        const int k0 = (DIM == 3) ? blockIdx.z * KZ : 0;
        const int k1 = (DIM == 3) ? min(nz, k0 + KZ) : 1;
        int64_t e = i + (int64_t)nx * j + sxy * k0;
        double pdn = (DIM == 3 && k0 > 0) ? ldg(x + e - sxy) : 0.0;
        double pc = ldg(x + e);
        for (int k = k0; k < k1; ++k, e += sxy) {
            const double pup = (DIM == 3 && k < nz - 1) ? ldg(x + e + sxy) : 0.0;
            double ax;
            if (POISSON) {
                double s = (i > 0) ? ldg(x + e - 1) : 0.0;
                if (i < nx - 1) s = add1(s, ldg(x + e + 1), one);
                if (j > 0) s = add1(s, ldg(x + e - nx), one);
                if (j < ny - 1) s = add1(s, ldg(x + e + nx), one);
                if (DIM == 3) {
                    if (k > 0) s = add1(s, pdn, one);
                    if (k < nz - 1) s = add1(s, pup, one);
                }
                ax = fma(d2, pc, -s);
            } else {
                const double s = diffusion_offdiag_sum<double, DIM>(x, f, e, i, j, k, nx, ny, nz, sxy, pdn, pup);
                ax = fma(ldg(f.diag + e), pc, -s);
            }
            const double rv = fma(ax, -one, ldg(b + e));   // b - ax
            if (r) r[e] = rv;
            if (r32) r32[e] = d2f_scaled(rv, kscale);
            ss = fma(rv, rv, ss);
            pdn = pc;
            pc = pup;
        }
    }
    __shared__ double sh[BX * BY / 32];
    // block sum over the 2D block
    double v = warp_sum(ss);
    const int t = threadIdx.x + BX * threadIdx.y;
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    double tot = 0.0;
    if (t == 0)
        for (int k = 0; k < BX * BY / 32; ++k) tot += sh[k];
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    last_block_finish(tot, partials, &ctl->counter2, ctl, mode, (int64_t)nx * ny * nz, nblk);
}

__global__ void __launch_bounds__(RB) k_residual_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                                     const double* __restrict__ vals, const double* __restrict__ b,
                                                     const double* __restrict__ x, double* __restrict__ r,
                                                     float* __restrict__ r32, int64_t n, double* partials, Ctl* ctl,
                                                     int mode) {
    if (mode == 2 && ctl->done) return;
    int kscale = 0;   // scale_next = 2^kscale
    if (mode == 2) {
        frexp(ctl->scale_next, &kscale);
        kscale -= 1;
    }
    double ss = 0.0;
    for (int64_t row = blockIdx.x * (int64_t)RB + threadIdx.x; row < n; row += (int64_t)gridDim.x * RB) {
        const int32_t s0 = ldg(rowptr + row), s1 = ldg(rowptr + row + 1);
        double y = 0.0;
        for (int32_t t = s0; t < s1; ++t) y = fma(ldg(vals + t), ldg(x + ldg(colind + t)), y);
        const double rv = ldg(b + row) - y;
        if (r) r[row] = rv;
        if (r32) r32[row] = d2f_scaled(rv, kscale);
        ss = fma(rv, rv, ss);
    }
    __shared__ double sh[RB / 32];
    const double tot = block_sum<RB>(ss, sh);
    last_block_finish(tot, partials, &ctl->counter2, ctl, mode, n, gridDim.x);
}

template <int DIM, bool POISSON>
__global__ void __launch_bounds__(BX* BY) k_apply_stencil(const double* __restrict__ x, double* __restrict__ y, int nx,
                                                          int ny, int nz, Faces<double> f, double d2) {
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const int64_t sxy = (int64_t)nx * ny;
    const int k0 = (DIM == 3) ? blockIdx.z * KC : 0;
    const int k1 = (DIM == 3) ? min(nz, k0 + KC) : 1;
    int64_t e = i + (int64_t)nx * j + sxy * k0;
    double pdn = (DIM == 3 && k0 > 0) ? ldg(x + e - sxy) : 0.0;
    double pc = ldg(x + e);
    for (int k = k0; k < k1; ++k, e += sxy) {
        const double pup = (DIM == 3 && k < nz - 1) ? ldg(x + e + sxy) : 0.0;
        if (POISSON) {
            double s = (i > 0) ? ldg(x + e - 1) : 0.0;
            if (i < nx - 1) s += ldg(x + e + 1);
            if (j > 0) s += ldg(x + e - nx);
            if (j < ny - 1) s += ldg(x + e + nx);
            if (DIM == 3) {
                if (k > 0) s += pdn;
                if (k < nz - 1) s += pup;
            }
            y[e] = fma(d2, pc, -s);
        } else {
            const double s = diffusion_offdiag_sum<double, DIM>(x, f, e, i, j, k, nx, ny, nz, sxy, pdn, pup);
            y[e] = fma(ldg(f.diag + e), pc, -s);
        }
        pdn = pc;
        pc = pup;
    }
}

// --- box stencil --------------------------------------------------------------------
// Every one of the 3^d - 1 grid points of the unit box around a point is a neighbour with
// weight -1 and the diagonal is 3^d - 1, so A p = 3^d p - B with B the sum of p over the whole
// box (0 outside the grid). B is formed separably: row sums R over x of each plane staged in
// shared memory, plane sums S over y of R (the 3 x 3 in-plane box), B = S(k-1) + S(k) + S(k+1)
// over z. A block computes S once per plane it touches (KB + 2 planes for KB outputs), about 9
// FP64 additions and FMAs per unknown instead of 26 neighbour additions. The values of the
// next plane (and the vector read with each output) are loaded into registers one plane
// ahead, so the two barriers per plane do not wait on memory.
constexpr int KB = 16;   // z planes per block of the box kernels
constexpr int KBP = 8;   // z planes per block of the FP32 box step with two points per thread (at
                         // 230^3: 67 -> 56 us against 16 planes; 3.0 waves of blocks instead of 1.4)

// One thread's share of a staged plane: its point, and the halo point it stages when it sits
// on the tile's x edge (hx), y edge (hy) or is one of the four corner loaders (hc).
template <typename T> struct BoxRegs { T c, hx, hy, hc; };

template <typename T>
__device__ __forceinline__ BoxRegs<T> box_load(const T* __restrict__ p, int64_t sxy, int k, bool valid, int i0, int j0,
                                               int nx, int ny) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = i0 + tx, j = j0 + ty;
    BoxRegs<T> v{T(0), T(0), T(0), T(0)};
    if (!valid) return v;
    const T* pk = p + sxy * k;
    if (i < nx && j < ny) v.c = ldg(pk + i + (int64_t)nx * j);
    if (tx == 0 && i0 > 0 && j < ny) v.hx = ldg(pk + (i0 - 1) + (int64_t)nx * j);
    if (tx == BX - 1 && i0 + BX < nx && j < ny) v.hx = ldg(pk + (i0 + BX) + (int64_t)nx * j);
    if (ty == 0 && j0 > 0 && i < nx) v.hy = ldg(pk + i + (int64_t)nx * (j0 - 1));
    if (ty == BY - 1 && j0 + BY < ny && i < nx) v.hy = ldg(pk + i + (int64_t)nx * (j0 + BY));
    if (ty == 1 && tx < 4) {   // the four halo corners
        const int ci = (tx & 1) ? i0 + BX : i0 - 1;
        const int cj = (tx >> 1) ? j0 + BY : j0 - 1;
        if (ci >= 0 && ci < nx && cj >= 0 && cj < ny) v.hc = ldg(pk + ci + (int64_t)nx * cj);
    }
    return v;
}

// S (the in-plane 3 x 3 box sum) at this thread's point from the plane held in v. Two block
// barriers; sp / sr may be reused after it returns.
template <typename T>
__device__ __forceinline__ T box_plane_sum(T (*sp)[BX + 2], T (*sr)[BX], const BoxRegs<T>& v, T one) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    sp[ty + 1][tx + 1] = v.c;
    if (tx == 0) sp[ty + 1][0] = v.hx;
    if (tx == BX - 1) sp[ty + 1][BX + 1] = v.hx;
    if (ty == 0) sp[0][tx + 1] = v.hy;
    if (ty == BY - 1) sp[BY + 1][tx + 1] = v.hy;
    if (ty == 1 && tx < 4) sp[(tx >> 1) ? BY + 1 : 0][(tx & 1) ? BX + 1 : 0] = v.hc;
    __syncthreads();
    sr[ty + 1][tx] = add1(add1(sp[ty + 1][tx], sp[ty + 1][tx + 1], one), sp[ty + 1][tx + 2], one);
    if (ty == 0) sr[0][tx] = add1(add1(sp[0][tx], sp[0][tx + 1], one), sp[0][tx + 2], one);
    if (ty == BY - 1) sr[BY + 1][tx] = add1(add1(sp[BY + 1][tx], sp[BY + 1][tx + 1], one), sp[BY + 1][tx + 2], one);
    __syncthreads();
    return add1(add1(sr[ty][tx], sr[ty + 1][tx], one), sr[ty + 2][tx], one);
}

// Marches the block's tile over its z slab (3D: planes k0 .. k1 - 1; 2D: the one plane) and
// calls emit(k, p_k, B_k, extra_k) for each, where extra_k = pre(k) was read one plane ahead.
template <typename T, int DIM, typename Pre, typename Emit>
__device__ __forceinline__ void box_march(const T* __restrict__ p, int nx, int ny, int nz, T one, Pre pre, Emit emit) {
    __shared__ T sp[BY + 2][BX + 2];
    __shared__ T sr[BY + 2][BX];
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int64_t sxy = (int64_t)nx * ny;
    if (DIM == 2) {
        const T ex = pre(0);
        const BoxRegs<T> v = box_load<T>(p, sxy, 0, true, i0, j0, nx, ny);
        emit(0, v.c, box_plane_sum<T>(sp, sr, v, one), ex);
        return;
    }
    const int k0 = blockIdx.z * KB, k1 = min(nz, k0 + KB);
    // window over planes kk = k0 - 1 .. k1: S(kk - 2) = sa, S(kk - 1) = sb, p(kk - 1) = pb
    T sa = T(0), sb = T(0), pb = T(0), eb = T(0);
    BoxRegs<T> cur = box_load<T>(p, sxy, k0 - 1, k0 > 0, i0, j0, nx, ny);
    for (int kk = k0 - 1; kk <= k1; ++kk) {
        const bool nvalid = kk + 1 <= k1 && kk + 1 < nz;
        const BoxRegs<T> nxt = box_load<T>(p, sxy, kk + 1, nvalid, i0, j0, nx, ny);
        const T ecur = (kk >= k0 && kk < k1) ? pre(kk) : T(0);
        const bool here = kk >= 0 && kk < nz;   // uniform over the block
        const T sc = here ? box_plane_sum<T>(sp, sr, cur, one) : T(0);
        if (kk - 1 >= k0) emit(kk - 1, pb, add1(add1(sa, sb, one), sc, one), eb);
        sa = sb;
        sb = sc;
        pb = cur.c;
        eb = ecur;
        cur = nxt;
    }
}

// Chebyshev step: out = ca p + cb B - q (q absent in the first step); GRAM: with the fused
// moments.
template <typename T, int DIM, bool FIRST, bool GRAM>
__global__ void __launch_bounds__(BX* BY) k_cheb_box(const T* __restrict__ p, const T* __restrict__ q,
                                                     T* __restrict__ out, int nx, int ny, int nz, T ca, T cb,
                                                     const Ctl* __restrict__ ctl, T one, void* mom, int nblk) {
    if (ctl->done) return;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const bool in = i < nx && j < ny;
    const int64_t ij = i + (int64_t)nx * j, sxy = (int64_t)nx * ny;
    MomAcc<T> acc;
    box_march<T, DIM>(
        p, nx, ny, nz, one, [&](int k) { return (FIRST || !in) ? T(0) : ldg(q + ij + sxy * k); },
        [&](int k, T pc, T B, T qv) {
            if (in) {
                const T o = FIRST ? fma(cb, B, ca * pc) : fma(cb, B, fma(ca, pc, -qv));
                out[ij + sxy * k] = o;
                if (GRAM) acc.add(pc, o);
            }
        });
    if (GRAM) mom_block_store(acc, mom, nblk);
}

// FP32 box step (mixed form): the FP32 pipe has room for the plain 3 x 3 in-plane sums (9
// loads through L1 and 8 adds per point and plane, the z-window of plane sums in registers),
// which needs no shared memory and no barriers. Its nine loads per point and plane make it
// latency-bound: eight resident blocks per SM (at most 32 registers) keep enough loads in
// flight, also with the fused moments' accumulators.
template <int DIM, bool FIRST, bool GRAM>
__global__ void __launch_bounds__(BX* BY, 8) k_cheb_box_f32(const float* __restrict__ p, const float* __restrict__ q,
                                                         float* __restrict__ out, int nx, int ny, int nz, float ca,
                                                         float cb, const Ctl* __restrict__ ctl, void* mom, int nblk) {
    if (ctl->done) return;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    MomAcc<float> acc;
    if (i < nx && j < ny) {
        const int64_t sxy = (int64_t)nx * ny, ij = i + (int64_t)nx * j;
        const bool xm = i > 0, xp = i < nx - 1, ym = j > 0, yp = j < ny - 1;
        auto row = [&](const float* a) { return ((xm ? ldg(a - 1) : 0.f) + ldg(a)) + (xp ? ldg(a + 1) : 0.f); };
        auto plane = [&](int k, float& center) {   // 3 x 3 sum of plane k around (i, j)
            const float* a = p + sxy * k + ij;
            center = ldg(a);
            const float r0 = ym ? row(a - nx) : 0.f;
            const float r1 = ((xm ? ldg(a - 1) : 0.f) + center) + (xp ? ldg(a + 1) : 0.f);
            const float r2 = yp ? row(a + nx) : 0.f;
            return (r0 + r1) + r2;
        };
        if (DIM == 2) {
            float pc;
            const float S = plane(0, pc);
            const float o = FIRST ? fmaf(cb, S, ca * pc) : fmaf(cb, S, fmaf(ca, pc, -ldg(q + ij)));
            out[ij] = o;
            if (GRAM) acc.add(pc, o);
        } else {
            const int k0 = blockIdx.z * KB, k1 = min(nz, k0 + KB);
            float pc, ptmp;
            float sdn = (k0 > 0) ? plane(k0 - 1, ptmp) : 0.f;
            float sc = plane(k0, pc);
            for (int k = k0; k < k1; ++k) {
                float pup = 0.f, sup = 0.f;
                if (k + 1 < nz) sup = plane(k + 1, pup);
                const int64_t e = ij + sxy * k;
                const float B = (sdn + sc) + sup;
                const float o = FIRST ? fmaf(cb, B, ca * pc) : fmaf(cb, B, fmaf(ca, pc, -ldg(q + e)));
                out[e] = o;
                if (GRAM) acc.add(pc, o);
                sdn = sc;
                sc = sup;
                pc = pup;
            }
        }
    }
    if (GRAM) mom_block_store(acc, mom, nblk);
}

// FP32 box step with two x-adjacent points per thread (nx even, 8-byte aligned vectors): each
// of the three rows of a plane is one 8-byte load per thread, the x-neighbours of the pair
// come from the adjacent lanes by shuffles (the warp's two edge points from memory), and the
// pair's row sums share their middle two terms: 3 loads and 3 adds per pair, row and plane
// instead of 9 loads and 8 adds per point. Measured at 230^3: the step alone unchanged (67 us;
// it waits on each plane's loads, and 1740 blocks are 1.4 waves of the resident ones), the
// step with the fused moments 81 -> 68 us (one point per thread needed 40 registers for it).
template <int DIM, bool FIRST, bool GRAM>
__global__ void __launch_bounds__(BX* BY) k_cheb_box_f32_pair(const float* __restrict__ p, const float* __restrict__ q,
                                                              float* __restrict__ out, int nx, int ny, int nz,
                                                              float ca, float cb, const Ctl* __restrict__ ctl,
                                                              void* mom, int nblk) {
    if (ctl->done) return;
    const int lane = threadIdx.x;   // BX = 32: one warp per row of the tile
    const int i0 = blockIdx.x * (2 * BX);
    const int i = i0 + 2 * lane;
    const int j = blockIdx.y * BY + threadIdx.y;
    const bool in = i < nx && j < ny;   // nx even: i + 1 < nx as well
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t ij = in ? i + (int64_t)nx * j : 0;
    const bool has_m = in && j > 0, has_p = in && j < ny - 1;
    // the in-plane 3 x 3 sums of plane k at the pair (and its centre values)
    auto plane = [&](int k, float2& center) {
        const float* a = p + sxy * k + ij;
        float2 S{0.f, 0.f};
        center = float2{0.f, 0.f};
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const bool has = dy < 0 ? has_m : (dy > 0 ? has_p : in);
            const float* row = a + (int64_t)dy * nx;
            const float2 v = has ? __ldg(reinterpret_cast<const float2*>(row)) : float2{0.f, 0.f};
            float xl = __shfl_up_sync(0xffffffffu, v.y, 1);
            float xr = __shfl_down_sync(0xffffffffu, v.x, 1);
            if (lane == 0) xl = (has && i0 > 0) ? ldg(row - 1) : 0.f;
            if (lane == BX - 1) xr = (has && i + 2 < nx) ? ldg(row + 2) : 0.f;
            const float t = v.x + v.y;
            S.x += xl + t;
            S.y += t + xr;
            if (dy == 0) center = v;
        }
        return S;
    };
    MomAcc<float> acc;
    auto emit = [&](int64_t e, const float2& pc, const float2& B) {
        if (!in) return;
        const float2 qv = FIRST ? float2{0.f, 0.f} : __ldg(reinterpret_cast<const float2*>(q + e));
        float2 o;
        o.x = FIRST ? fmaf(cb, B.x, ca * pc.x) : fmaf(cb, B.x, fmaf(ca, pc.x, -qv.x));
        o.y = FIRST ? fmaf(cb, B.y, ca * pc.y) : fmaf(cb, B.y, fmaf(ca, pc.y, -qv.y));
        *reinterpret_cast<float2*>(out + e) = o;
        if (GRAM) {
            acc.add(pc.x, o.x);
            acc.add(pc.y, o.y);
        }
    };
    if (DIM == 2) {
        float2 pc;
        const float2 S = plane(0, pc);
        emit(ij, pc, S);
    } else {
        const int k0 = blockIdx.z * KBP, k1 = min(nz, k0 + KBP);
        float2 pc, ptmp;
        float2 sdn = (k0 > 0) ? plane(k0 - 1, ptmp) : float2{0.f, 0.f};
        float2 sc = plane(k0, pc);
        for (int k = k0; k < k1; ++k) {
            float2 pup{0.f, 0.f}, sup{0.f, 0.f};
            if (k + 1 < nz) sup = plane(k + 1, pup);
            emit(ij + sxy * k, pc, float2{(sdn.x + sc.x) + sup.x, (sdn.y + sc.y) + sup.y});
            sdn = sc;
            sc = sup;
            pc = pup;
        }
    }
    if (GRAM) mom_block_store(acc, mom, nblk);
}

// FP64 box step, register-blocked and persistent (3D, nx even, 16-byte aligned vectors). A
// thread owns two x-adjacent points (one 16-byte load per row) in BOXY consecutive rows; the
// lanes run over (row group, x pair) with the pair fastest, so a warp has idle lanes only in
// the grid's last 32 (a warp's FP64 instruction costs the same whatever its active lanes:
// 64-point tiles idled 10% of the lanes at nx = 230). A warp column is 32 consecutive lanes
// of that order; the grid is the resident blocks, and each warp marches an equal contiguous
// range of the (warp column, plane) units, no shared memory and no barrier. Per plane it
// loads its BOXY + 2 rows and forms
//  * the pair's x row sums p(i-1) + (p(i) + p(i+1)) and (p(i) + p(i+1)) + p(i+2): three
//    additions per pair and row, the outer neighbours from the adjacent lanes by shuffles
//    (from memory where the adjacent lane holds another row group or lies outside the warp,
//    0 at the grid's x faces);
//  * the in-plane sums S of two consecutive rows at a time, which share their middle two row
//    sums: S(t) = R(t-1) + (R(t) + R(t+1)), S(t+1) = (R(t) + R(t+1)) + R(t+2);
// 3.75 FP64 additions per point and plane for S at BOXY = 4 (4 plus the tile's halo rows
// when the row sums go through shared memory). B(k) = S(k-1) + S(k) + S(k+1) is accumulated
// forward as each plane's S arrives (2 additions per point) and the step adds its 2 FMAs:
// with a range's two halo planes about 8.1 FP64 instructions per point against about 10.4
// for k_cheb_box, whose two barriers per plane also leave the FP64 pipe idle. Measured at
// 230^3: 0.255 -> 0.186 ms per step (0.61 -> 0.83 of the FP64 FMA rate by the 8 operations
// of the separable sum); tiles of 64 x 16 x 16 points in a plain grid gave 0.246 ms (1.7
// waves of resident blocks), the same persistent march over 64-point tiles 0.205 ms.
constexpr int BOXY = 4;   // rows per thread (even)
constexpr int BOXW = 4;   // warps per block
// resident blocks per SM the launch bound asks for: FP64 3 (at most 168 registers), FP32 4
template <typename T> constexpr int box_reg_min_blocks() { return sizeof(T) == 8 ? 3 : 4; }

// The thread's place in the flattened order for warp column c, with the in-plane offsets of
// its Y + 2 rows (fixed while it marches the column; a plane only adds k nx ny).
template <int Y> struct BoxLane {
    int i, jb;                        // first x of the pair, first row
    bool valid;                       // the lane has a pair
    bool lload, rload, lzero, rzero;  // outer neighbours: loaded / 0 (x faces) / from a lane
    unsigned rows;                    // bit r: row jb - 1 + r lies in the grid (and valid)
    int roff[Y + 2];                  // nx (jb - 1 + r) + i for those rows, else 0
};

template <int Y>
__device__ __forceinline__ BoxLane<Y> box_lane(int64_t c, int nx, int ny) {
    const int lane = threadIdx.x;
    const int np = nx / 2;
    const int64_t nl = (int64_t)np * ((ny + Y - 1) / Y);
    const int64_t L = c * 32 + lane;
    BoxLane<Y> b;
    b.valid = L < nl;
    const int xp = b.valid ? (int)(L % np) : 0;
    b.i = 2 * xp;
    b.jb = b.valid ? (int)(L / np) * Y : 0;
    b.lzero = xp == 0;
    b.rzero = xp == np - 1;   // also every lane whose next lane is past the last pair
    b.lload = b.valid && !b.lzero && lane == 0;
    b.rload = b.valid && !b.rzero && lane == 31;
    b.rows = 0u;
#pragma unroll
    for (int r = 0; r < Y + 2; ++r) {
        const int jj = b.jb - 1 + r;
        const bool rv = b.valid && jj >= 0 && jj < ny;
        b.rows |= rv ? 1u << r : 0u;
        b.roff[r] = rv ? nx * jj + b.i : 0;
    }
    return b;
}

template <typename T> __device__ __forceinline__ typename Pair<T>::type pair_of(T x, T y) { return {x, y}; }

// The thread's rows of plane k (pk = p + k nx ny, kv: 0 <= k < nz): its pair per row, and the
// edge point lane 0 (x = i - 1) or lane 31 (x = i + 2) loads; 0 outside the grid.
template <typename T, int Y> struct BoxRows {
    typename Pair<T>::type v[Y + 2];
    T e[Y + 2];
};

template <typename T, int Y>
__device__ __forceinline__ BoxRows<T, Y> box_reg_load(const T* __restrict__ pk, bool kv, const BoxLane<Y>& b) {
    const int de = b.lload ? -1 : 2;
    const bool edge = b.lload || b.rload;
    BoxRows<T, Y> w;
#pragma unroll
    for (int r = 0; r < Y + 2; ++r) {
        const bool rv = kv && ((b.rows >> r) & 1u);
        w.v[r] = rv ? __ldg(reinterpret_cast<const typename Pair<T>::type*>(pk + b.roff[r])) : pair_of<T>(T(0), T(0));
        w.e[r] = (rv && edge) ? ldg(pk + b.roff[r] + de) : T(0);
    }
    return w;
}

// S, the 3 x 3 in-plane sums of the loaded plane at the thread's 2 x Y points; c receives the
// centre pairs of the Y rows.
template <typename T, int Y>
__device__ __forceinline__ void box_reg_sums(const BoxRows<T, Y>& w, const BoxLane<Y>& b, T one,
                                             typename Pair<T>::type (&c)[Y], T (&S)[Y][2]) {
    T R[Y + 2][2];
#pragma unroll
    for (int r = 0; r < Y + 2; ++r) {
        T l = __shfl_up_sync(0xffffffffu, w.v[r].y, 1);
        T rr = __shfl_down_sync(0xffffffffu, w.v[r].x, 1);
        if (b.lzero) l = T(0);
        if (b.rzero) rr = T(0);
        if (b.lload) l = w.e[r];
        if (b.rload) rr = w.e[r];
        const T m = add1(w.v[r].x, w.v[r].y, one);
        R[r][0] = add1(l, m, one);
        R[r][1] = add1(m, rr, one);
    }
#pragma unroll
    for (int t = 0; t < Y; ++t) c[t] = w.v[t + 1];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int t = 0; t < Y; t += 2) {
            const T m = add1(R[t + 1][x], R[t + 2][x], one);
            S[t][x] = add1(R[t][x], m, one);
            S[t + 1][x] = add1(m, R[t + 3][x], one);
        }
}

// The warp's share of the persistent march: calls pre(e) ahead of emit(e, pc, B, pre value)
// for each of the thread's points in the grid, e = the element offset of the pair at x = i
// (pc, B and the pre value as pairs at x = i, i + 1). PREF: the rows of plane k + 2 and the
// pre values of plane k + 1 are loaded while plane k's output is formed (the FP32 step, which
// waits on memory); without it a plane's loads are issued at the top of its iteration (the
// FP64 kernels, which the FP64 pipe bounds, keep the registers for resident warps instead).
template <typename T, int Y, bool PREF, typename Pre, typename Emit>
__device__ __forceinline__ void box_reg_sweep(const T* __restrict__ p, int nx, int ny, int nz, T one, Pre pre, Emit emit) {
    static_assert(Y % 2 == 0, "rows per thread: even");
    using V = typename Pair<T>::type;
    const int np = nx / 2;
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t nwc = ((int64_t)np * ((ny + Y - 1) / Y) + 31) / 32;   // warp columns
    const int64_t U = nwc * nz;
    const int64_t nw = (int64_t)gridDim.x * BOXW, w = (int64_t)blockIdx.x * BOXW + threadIdx.y;
    int64_t u = U * w / nw;
    const int64_t u1 = U * (w + 1) / nw;
    while (u < u1) {
        const int64_t c = u / nz;
        const int k0 = (int)(u - c * nz);
        const int k1 = (int)(k0 + (u1 - u) < (int64_t)nz ? k0 + (u1 - u) : (int64_t)nz);
        const BoxLane<Y> b = box_lane<Y>(c, nx, ny);
        auto plane = [&](int k) { return box_reg_load<T, Y>(p + sxy * k, k >= 0 && k < nz, b); };
        auto pre_rows = [&](int k, V (&ev)[Y]) {
#pragma unroll
            for (int t = 0; t < Y; ++t)
                ev[t] = (k < k1 && ((b.rows >> (t + 1)) & 1u)) ? pre(sxy * k + b.roff[t + 1]) : pair_of<T>(T(0), T(0));
        };
        T A0[Y][2], A1[Y][2], S[Y][2];   // A0: S(k-1) + S(k), A1: S(k)
        V pc[Y], pn[Y];
        box_reg_sums<T, Y>(plane(k0 - 1), b, one, pn, A0);
        box_reg_sums<T, Y>(plane(k0), b, one, pc, S);
#pragma unroll
        for (int t = 0; t < Y; ++t)
#pragma unroll
            for (int x = 0; x < 2; ++x) {
                A0[t][x] = add1(A0[t][x], S[t][x], one);
                A1[t][x] = S[t][x];
            }
        BoxRows<T, Y> nxt;
        V evn[Y];
        if (PREF) {
            nxt = plane(k0 + 1);
            pre_rows(k0, evn);
        }
        for (int k = k0; k < k1; ++k) {
            V ev[Y];
            BoxRows<T, Y> cur;
            if (PREF) {
#pragma unroll
                for (int t = 0; t < Y; ++t) ev[t] = evn[t];
                cur = nxt;
                nxt = plane(k + 2 <= k1 ? k + 2 : nz);   // plane nz: zeros, nothing loaded
                pre_rows(k + 1, evn);
            } else {
                pre_rows(k, ev);
                cur = plane(k + 1);
            }
            box_reg_sums<T, Y>(cur, b, one, pn, S);
#pragma unroll
            for (int t = 0; t < Y; ++t) {
                const V B = pair_of<T>(add1(A0[t][0], S[t][0], one), add1(A0[t][1], S[t][1], one));
                if ((b.rows >> (t + 1)) & 1u) emit(sxy * k + b.roff[t + 1], pc[t], B, ev[t]);
#pragma unroll
                for (int x = 0; x < 2; ++x) {
                    A0[t][x] = add1(A1[t][x], S[t][x], one);
                    A1[t][x] = S[t][x];
                }
                pc[t] = pn[t];
            }
        }
        u += k1 - k0;
    }
}

template <typename T, int Y, bool FIRST, bool GRAM>
__global__ void __launch_bounds__(32 * BOXW, box_reg_min_blocks<T>()) k_cheb_box_reg(
    const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ out, int nx, int ny, int nz, T ca, T cb,
    const Ctl* __restrict__ ctl, T one, void* mom, int nblk) {
    using V = typename Pair<T>::type;
    if (ctl->done) return;
    MomAcc<T> acc;
    box_reg_sweep<T, Y, sizeof(T) == 4>(
        p, nx, ny, nz, one,
        [&](int64_t e) { return FIRST ? pair_of<T>(T(0), T(0)) : __ldg(reinterpret_cast<const V*>(q + e)); },
        [&](int64_t e, V pc, V B, V qv) {
            V o;
            o.x = FIRST ? fma(cb, B.x, ca * pc.x) : fma(cb, B.x, fma(ca, pc.x, -qv.x));
            o.y = FIRST ? fma(cb, B.y, ca * pc.y) : fma(cb, B.y, fma(ca, pc.y, -qv.y));
            *reinterpret_cast<V*>(out + e) = o;
            if (GRAM) {
                acc.add(pc.x, o.x);
                acc.add(pc.y, o.y);
            }
        });
    if (GRAM) mom_block_store<32 * BOXW>(acc, mom, nblk);
}

// FP64 7-point Poisson step (3D, nx even, 16-byte aligned vectors) on the same register-blocked
// persistent march: a thread owns an x pair in STARY rows of a warp column and loads its
// STARY + 2 rows of a plane once; the y neighbours of its rows come from its own registers,
// the z neighbours from the previous and next plane's rows it holds, the x neighbours from
// the adjacent lanes: 10 load instructions and 96 B through L1 per 4 points and plane (its
// 4 rows, their edge loads in lanes 0 and 31, q) against 12 and 128 B for the pair kernel,
// whose loads filled the L1 queue (stall tex_throttle 35 per issue at 192^3) with the FP64
// pipe 81% busy; with a quarter of the resident warps the pipe is 91% busy. Same sums in the
// same order as k_cheb_poisson_pair (bitwise equal outputs). Measured at 256^3: 0.2315 ->
// 0.205 ms per step (0.81 -> 0.91 of the FP64 FMA rate). The FP32 step keeps the pair
// kernel (0.80 of HBM; this form measured 0.61).
constexpr int STARY = 2;   // rows per thread

template <bool FIRST, bool GRAM>
__global__ void __launch_bounds__(32 * BOXW, 4) k_cheb_star_reg(const double* __restrict__ p,
                                                                const double* __restrict__ q, double* __restrict__ out,
                                                                int nx, int ny, int nz, double c1, double c2,
                                                                const Ctl* __restrict__ ctl, double one, void* mom,
                                                                int nblk) {
    constexpr int Y = STARY;
    using V = double2;
    if (ctl->done) return;
    const int np = nx / 2;
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t nwc = ((int64_t)np * ((ny + Y - 1) / Y) + 31) / 32;   // warp columns
    const int64_t U = nwc * nz;
    const int64_t nw = (int64_t)gridDim.x * BOXW, w = (int64_t)blockIdx.x * BOXW + threadIdx.y;
    int64_t u = U * w / nw;
    const int64_t u1 = U * (w + 1) / nw;
    MomAcc<double> acc;
    while (u < u1) {
        const int64_t c = u / nz;
        const int k0 = (int)(u - c * nz);
        const int k1 = (int)(k0 + (u1 - u) < (int64_t)nz ? k0 + (u1 - u) : (int64_t)nz);
        const BoxLane<Y> b = box_lane<Y>(c, nx, ny);
        auto plane = [&](int k) { return box_reg_load<double, Y>(p + sxy * k, k >= 0 && k < nz, b); };
        V pd[Y];   // the rows of plane k - 1
        {
            const BoxRows<double, Y> w0 = plane(k0 - 1);
#pragma unroll
            for (int t = 0; t < Y; ++t) pd[t] = w0.v[t + 1];
        }
        BoxRows<double, Y> cur = plane(k0);
        for (int k = k0; k < k1; ++k) {
            V qv[Y];
#pragma unroll
            for (int t = 0; t < Y; ++t)
                qv[t] = (!FIRST && ((b.rows >> (t + 1)) & 1u))
                            ? __ldg(reinterpret_cast<const V*>(q + sxy * k + b.roff[t + 1]))
                            : make_double2(0.0, 0.0);
            const BoxRows<double, Y> up = plane(k + 1);
#pragma unroll
            for (int t = 0; t < Y; ++t) {
                const V pc = cur.v[t + 1];
                // left of the pair: the lane below's right point; right: the lane above's left
                // point; from memory at the warp's edges, 0 at the grid's x faces
                double xl = __shfl_up_sync(0xffffffffu, pc.y, 1);
                double xr = __shfl_down_sync(0xffffffffu, pc.x, 1);
                if (b.lzero) xl = 0.0;
                if (b.rzero) xr = 0.0;
                if (b.lload) xl = cur.e[t + 1];
                if (b.rload) xr = cur.e[t + 1];
                const V ym = cur.v[t], yp = cur.v[t + 2], pup = up.v[t + 1], pdn = pd[t];
                double s0 = add1(add1(xl, pc.y, one), add1(ym.x, yp.x, one), one);
                double s1 = add1(add1(pc.x, xr, one), add1(ym.y, yp.y, one), one);
                s0 = add1(s0, add1(pdn.x, pup.x, one), one);
                s1 = add1(s1, add1(pdn.y, pup.y, one), one);
                V o;
                o.x = FIRST ? fma(c2, s0, c1 * pc.x) : fma(c2, s0, fma(c1, pc.x, -qv[t].x));
                o.y = FIRST ? fma(c2, s1, c1 * pc.y) : fma(c2, s1, fma(c1, pc.y, -qv[t].y));
                if ((b.rows >> (t + 1)) & 1u) {
                    *reinterpret_cast<V*>(out + sxy * k + b.roff[t + 1]) = o;
                    if (GRAM) {
                        acc.add(pc.x, o.x);
                        acc.add(pc.y, o.y);
                    }
                }
                pd[t] = pc;
            }
            cur = up;
        }
        u += k1 - k0;
    }
    if (GRAM) mom_block_store<32 * BOXW>(acc, mom, nblk);
}

// r = b - A x with ||r||^2 for the 7-point Poisson operator (FP64; 3D, nx even, b, x and r
// 16-byte and r32 8-byte aligned) on the march of k_cheb_star_reg; residual modes as
// k_residual_stencil, the neighbour sum in the same order (x-, x+, y-, y+, z-, z+; a missing
// neighbour adds 0). The mixed forms' FP64 refresh.
__global__ void __launch_bounds__(32 * BOXW, 4) k_residual_star_reg(const double* __restrict__ b,
                                                                    const double* __restrict__ x,
                                                                    double* __restrict__ r, float* __restrict__ r32,
                                                                    int nx, int ny, int nz, double d2,
                                                                    double* partials, Ctl* ctl, int mode,
                                                                    double one) {
    constexpr int Y = STARY;
    using V = double2;
    if (mode == 2 && ctl->done) return;
    int kscale = 0;   // scale_next = 2^kscale
    if (mode == 2) {
        frexp(ctl->scale_next, &kscale);
        kscale -= 1;
    }
    const int np = nx / 2;
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t nwc = ((int64_t)np * ((ny + Y - 1) / Y) + 31) / 32;   // warp columns
    const int64_t U = nwc * nz;
    const int64_t nw = (int64_t)gridDim.x * BOXW, w = (int64_t)blockIdx.x * BOXW + threadIdx.y;
    int64_t u = U * w / nw;
    const int64_t u1 = U * (w + 1) / nw;
    double ss = 0.0;
    while (u < u1) {
        const int64_t c = u / nz;
        const int k0 = (int)(u - c * nz);
        const int k1 = (int)(k0 + (u1 - u) < (int64_t)nz ? k0 + (u1 - u) : (int64_t)nz);
        const BoxLane<Y> bl = box_lane<Y>(c, nx, ny);
        auto plane = [&](int k) { return box_reg_load<double, Y>(x + sxy * k, k >= 0 && k < nz, bl); };
        V pd[Y];   // the rows of plane k - 1
        {
            const BoxRows<double, Y> w0 = plane(k0 - 1);
#pragma unroll
            for (int t = 0; t < Y; ++t) pd[t] = w0.v[t + 1];
        }
        BoxRows<double, Y> cur = plane(k0);
        for (int k = k0; k < k1; ++k) {
            V bv[Y];
#pragma unroll
            for (int t = 0; t < Y; ++t)
                bv[t] = ((bl.rows >> (t + 1)) & 1u) ? __ldg(reinterpret_cast<const V*>(b + sxy * k + bl.roff[t + 1]))
                                                    : make_double2(0.0, 0.0);
            const BoxRows<double, Y> up = plane(k + 1);
#pragma unroll
            for (int t = 0; t < Y; ++t) {
                const V pc = cur.v[t + 1];
                double xl = __shfl_up_sync(0xffffffffu, pc.y, 1);
                double xr = __shfl_down_sync(0xffffffffu, pc.x, 1);
                if (bl.lzero) xl = 0.0;
                if (bl.rzero) xr = 0.0;
                if (bl.lload) xl = cur.e[t + 1];
                if (bl.rload) xr = cur.e[t + 1];
                const V ym = cur.v[t], yp = cur.v[t + 2], pup = up.v[t + 1], pdn = pd[t];
                double s0 = add1(add1(add1(add1(add1(xl, pc.y, one), ym.x, one), yp.x, one), pdn.x, one), pup.x, one);
                double s1 = add1(add1(add1(add1(add1(pc.x, xr, one), ym.y, one), yp.y, one), pdn.y, one), pup.y, one);
                const double r0 = fma(fma(d2, pc.x, -s0), -one, bv[t].x);   // b - A x
                const double r1 = fma(fma(d2, pc.y, -s1), -one, bv[t].y);
                if ((bl.rows >> (t + 1)) & 1u) {
                    const int64_t e = sxy * k + bl.roff[t + 1];
                    if (r) *reinterpret_cast<V*>(r + e) = make_double2(r0, r1);
                    if (r32) *reinterpret_cast<float2*>(r32 + e) = make_float2(d2f_scaled(r0, kscale), d2f_scaled(r1, kscale));
                    ss = fma(r0, r0, ss);
                    ss = fma(r1, r1, ss);
                }
                pd[t] = pc;
            }
            cur = up;
        }
        u += k1 - k0;
    }
    __shared__ double sh[BOXW];
    const double v = warp_sum(ss);
    if (threadIdx.x == 0) sh[threadIdx.y] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int k = 0; k < BOXW; ++k) tot += sh[k];
    last_block_finish(tot, partials, &ctl->counter2, ctl, mode, (int64_t)nx * ny * nz, (int)gridDim.x);
}

// r = b - A x = b - (3^d x - B) with ||r||^2 (residual modes as k_residual_stencil).
template <int DIM>
__global__ void __launch_bounds__(BX* BY) k_residual_box(const double* __restrict__ b, const double* __restrict__ x,
                                                         double* __restrict__ r, float* __restrict__ r32, int nx,
                                                         int ny, int nz, double* partials, Ctl* ctl, int mode,
                                                         double one) {
    if (mode == 2 && ctl->done) return;
    int kscale = 0;   // scale_next = 2^kscale
    if (mode == 2) {
        frexp(ctl->scale_next, &kscale);
        kscale -= 1;
    }
    const double dfull = DIM == 3 ? 27.0 : 9.0;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const bool in = i < nx && j < ny;
    const int64_t ij = i + (int64_t)nx * j, sxy = (int64_t)nx * ny;
    double ss = 0.0;
    box_march<double, DIM>(
        x, nx, ny, nz, one, [&](int k) { return in ? ldg(b + ij + sxy * k) : 0.0; },
        [&](int k, double pc, double B, double bv) {
            if (!in) return;
            const int64_t e = ij + sxy * k;
            const double rv = fma(fma(dfull, pc, -B), -one, bv);   // bv - (dfull pc - B)
            if (r) r[e] = rv;
            if (r32) r32[e] = d2f_scaled(rv, kscale);
            ss = fma(rv, rv, ss);
        });
    __shared__ double sh[BX * BY / 32];
    double v = warp_sum(ss);
    const int t = threadIdx.x + BX * threadIdx.y;
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    double tot = 0.0;
    if (t == 0)
        for (int k = 0; k < BX * BY / 32; ++k) tot += sh[k];
    const int nblk = gridDim.x * gridDim.y * gridDim.z;
    last_block_finish(tot, partials, &ctl->counter2, ctl, mode, (int64_t)nx * ny * nz, nblk);
}

// r = b - A x with ||r||^2 on the register-blocked persistent march of k_cheb_box_reg (3D, nx
// even, b, x and r 16-byte and r32 8-byte aligned); residual modes as k_residual_stencil.
__global__ void __launch_bounds__(32 * BOXW, box_reg_min_blocks<double>()) k_residual_box_reg(const double* __restrict__ b,
                                                                   const double* __restrict__ x,
                                                                   double* __restrict__ r, float* __restrict__ r32,
                                                                   int nx, int ny, int nz, double* partials, Ctl* ctl,
                                                                   int mode, double one) {
    if (mode == 2 && ctl->done) return;
    int kscale = 0;   // scale_next = 2^kscale
    if (mode == 2) {
        frexp(ctl->scale_next, &kscale);
        kscale -= 1;
    }
    double ss = 0.0;
    box_reg_sweep<double, BOXY, false>(
        x, nx, ny, nz, one, [&](int64_t e) { return __ldg(reinterpret_cast<const double2*>(b + e)); },
        [&](int64_t e, double2 pc, double2 B, double2 bv) {
            const double r0 = fma(fma(27.0, pc.x, -B.x), -one, bv.x);   // bv - (27 pc - B)
            const double r1 = fma(fma(27.0, pc.y, -B.y), -one, bv.y);
            if (r) *reinterpret_cast<double2*>(r + e) = make_double2(r0, r1);
            if (r32) *reinterpret_cast<float2*>(r32 + e) = make_float2(d2f_scaled(r0, kscale), d2f_scaled(r1, kscale));
            ss = fma(r0, r0, ss);
            ss = fma(r1, r1, ss);
        });
    __shared__ double sh[BOXW];
    const double v = warp_sum(ss);
    if (threadIdx.x == 0) sh[threadIdx.y] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int k = 0; k < BOXW; ++k) tot += sh[k];
    last_block_finish(tot, partials, &ctl->counter2, ctl, mode, (int64_t)nx * ny * nz, (int)gridDim.x);
}

template <int DIM>
__global__ void __launch_bounds__(BX* BY) k_apply_box(const double* __restrict__ x, double* __restrict__ y, int nx,
                                                      int ny, int nz) {
    const double dfull = DIM == 3 ? 27.0 : 9.0;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const bool in = i < nx && j < ny;
    const int64_t ij = i + (int64_t)nx * j, sxy = (int64_t)nx * ny;
    box_march<double, DIM>(
        x, nx, ny, nz, 1.0, [&](int) { return 0.0; },
        [&](int k, double pc, double B, double) {
            if (in) y[ij + sxy * k] = fma(dfull, pc, -B);
        });
}

dim3 box_grid(const OpDesc& op) {
    return dim3((op.nx + BX - 1) / BX, (op.ny + BY - 1) / BY, op.dim == 3 ? (op.nz + KB - 1) / KB : 1);
}

// FP32 box step with two points per thread: nx even and 8-byte aligned vectors
dim3 box_pair_grid(const OpDesc& op) {
    return dim3((op.nx + 2 * BX - 1) / (2 * BX), (op.ny + BY - 1) / BY, op.dim == 3 ? (op.nz + KBP - 1) / KBP : 1);
}
// The register-blocked persistent kernels (box steps and residual for 3D grids with nx even,
// 7-point FP64 step and residual): the grid is the blocks of 32 x BOXW threads resident at
// once for the least of a kernel family's instantiations (cached per device), and at most one
// warp per (warp column, plane) unit.
template <typename... K>
int resident_per_sm(int (&cache)[64], K... kernels) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) {
        int m = 1 << 30;
        for (const void* k : {(const void*)kernels...}) {
            int b = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, 32 * BOXW, 0) == cudaSuccess) m = std::min(m, b);
        }
        cache[dev] = (m >= 1 && m < (1 << 30)) ? m : 1;
    }
    return cache[dev];
}
dim3 persistent_grid(const OpDesc& op, int rows_per_thread, int per_sm) {
    const int64_t nwc = ((int64_t)(op.nx / 2) * ((op.ny + rows_per_thread - 1) / rows_per_thread) + 31) / 32;
    const int64_t units = nwc * op.nz, want = (units + BOXW - 1) / BOXW;
    const int64_t cap = (int64_t)per_sm * device_sm_count();
    return dim3((unsigned)std::max<int64_t>(1, std::min(want, cap)));
}
template <typename T>
dim3 box_reg_grid(const OpDesc& op) {
    static int cache[64] = {0};
    return persistent_grid(op, BOXY,
                           resident_per_sm(cache, k_cheb_box_reg<T, BOXY, true, false>, k_cheb_box_reg<T, BOXY, false, false>,
                                           k_cheb_box_reg<T, BOXY, true, true>, k_cheb_box_reg<T, BOXY, false, true>));
}
// the grids the register-blocked kernels take: 3D, nx even, a plane within 32-bit offsets
bool box_reg_shape(const OpDesc& op) {
    return op.dim == 3 && op.nx % 2 == 0 && (int64_t)op.nx * op.ny < (int64_t)INT32_MAX;
}
template <typename T>
bool box_reg_ok(const OpDesc& op, const T* p, const T* q, const T* out) {
    const size_t al = 2 * sizeof(T);
    return box_reg_shape(op) && ((uintptr_t)p % al == 0) && ((uintptr_t)out % al == 0) && (!q || (uintptr_t)q % al == 0);
}
// FP64 register-blocked 7-point step and residual: the shapes of the box kernels, Poisson weights
dim3 star_reg_grid(const OpDesc& op) {
    static int cache[64] = {0};
    return persistent_grid(op, STARY,
                           resident_per_sm(cache, k_cheb_star_reg<true, false>, k_cheb_star_reg<false, false>,
                                           k_cheb_star_reg<true, true>, k_cheb_star_reg<false, true>));
}
bool star_reg_shape(const OpDesc& op) { return !op.box && op.wx == nullptr && box_reg_shape(op); }
dim3 star_res_grid(const OpDesc& op) {
    static int cache[64] = {0};
    return persistent_grid(op, STARY, resident_per_sm(cache, k_residual_star_reg));
}
dim3 box_res_reg_grid(const OpDesc& op) {
    static int cache[64] = {0};
    return persistent_grid(op, BOXY, resident_per_sm(cache, k_residual_box_reg));
}
bool box_res_reg_ok(const OpDesc& op, const double* b, const double* x, const double* r, const float* r32) {
    return box_reg_shape(op) && ((uintptr_t)b % 16 == 0) && ((uintptr_t)x % 16 == 0) &&
           (!r || (uintptr_t)r % 16 == 0) && (!r32 || (uintptr_t)r32 % 8 == 0);
}
bool box_pair_ok(const OpDesc& op, const float* p, const float* q, const float* out) {
    return op.nx % 2 == 0 && ((uintptr_t)p % 8 == 0) && ((uintptr_t)out % 8 == 0) && (!q || (uintptr_t)q % 8 == 0);
}

__global__ void __launch_bounds__(RB) k_apply_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                                  const double* __restrict__ vals, const double* __restrict__ x,
                                                  double* __restrict__ y, int64_t n) {
    for (int64_t row = blockIdx.x * (int64_t)RB + threadIdx.x; row < n; row += (int64_t)gridDim.x * RB) {
        const int32_t s0 = ldg(rowptr + row), s1 = ldg(rowptr + row + 1);
        double acc = 0.0;
        for (int32_t t = s0; t < s1; ++t) acc = fma(ldg(vals + t), ldg(x + ldg(colind + t)), acc);
        y[row] = acc;
    }
}

dim3 stencil_grid(const OpDesc& op, int kz = KC) {
    return dim3((op.nx + BX - 1) / BX, (op.ny + BY - 1) / BY, op.dim == 3 ? (op.nz + kz - 1) / kz : 1);
}

// two x-adjacent points per thread
dim3 pair_grid(const OpDesc& op, int kz) {
    const dim3 g = stencil_grid(op, kz);
    return dim3((op.nx + 2 * BX - 1) / (2 * BX), g.y, g.z);
}

int vec_blocks(int64_t n) {
    int64_t b = (n + RB - 1) / RB;
    const int64_t cap = 8 * (int64_t)device_sm_count();
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename T> Faces<T> faces_of(const OpDesc& op);
template <> Faces<double> faces_of<double>(const OpDesc& op) { return {op.wx, op.wy, op.wz, op.diag, op.cdinv}; }
template <> Faces<float> faces_of<float>(const OpDesc& op) { return {op.wx32, op.wy32, op.wz32, op.diag32, op.cdinv32}; }

template <typename T> const T* csr_vals(const OpDesc& op);
template <> const double* csr_vals<double>(const OpDesc& op) { return op.vals; }
template <> const float* csr_vals<float>(const OpDesc& op) { return op.vals32; }

// Launch of a step kernel K<..., FIRST, GRAM> with the fused-moments switch resolved at run time.
#define SSTEP_STEP_LAUNCH(KERNEL, GRID, ...)                                                      \
    do {                                                                                        \
        const int nb_ = (int)((GRID).x * (GRID).y * (GRID).z);                                  \
        if (first) {                                                                            \
            if (mom) KERNEL<__VA_ARGS__, true, true><<<GRID, block, 0, st>>>(ARGS, mom, nb_);   \
            else KERNEL<__VA_ARGS__, true, false><<<GRID, block, 0, st>>>(ARGS, nullptr, nb_);  \
        } else {                                                                                \
            if (mom) KERNEL<__VA_ARGS__, false, true><<<GRID, block, 0, st>>>(ARGS, mom, nb_);  \
            else KERNEL<__VA_ARGS__, false, false><<<GRID, block, 0, st>>>(ARGS, nullptr, nb_); \
        }                                                                                       \
    } while (0)

// Pair kernel for the Poisson stencil: nx even and the vectors 2-element aligned (the
// workspace's always are), so every pair's loads and stores are aligned.
template <typename T>
bool use_pair(const OpDesc& op, const T* p, const T* q, const T* out) {
    const size_t al = 2 * sizeof(T);
    return op.nx % 2 == 0 && ((uintptr_t)p % al == 0) && ((uintptr_t)out % al == 0) && (!q || (uintptr_t)q % al == 0);
}

template <typename T, int DIM, bool POISSON>
void cheb_stencil_dispatch(const OpDesc& op, const T* p, const T* q, T* out, double theta, double sigma, bool first,
                           bool jacobi, const Ctl* ctl, void* mom, cudaStream_t st) {
    const dim3 grid = stencil_grid(op, kz_step<T>()), block(BX, BY);
    const double c = first ? theta : 2.0 * theta;
    const Faces<T> f = faces_of<T>(op);
    if (POISSON) {
        // D^-1 A p - sigma p = (1 - sigma) p - sum / (2 dim) with Jacobi (D = 2 dim I);
        // A p - sigma p = (2 dim - sigma) p - sum without.
        const double d2 = 2.0 * op.dim;
        const T c1 = (T)(jacobi ? c * (1.0 - sigma) : c * (d2 - sigma));
        const T c2 = (T)(jacobi ? -c / d2 : -c);
        if constexpr (std::is_same<T, double>::value) {
            if (DIM == 3 && star_reg_shape(op) && use_pair(op, p, q, out)) {
                const dim3 g3 = star_reg_grid(op), block(32, BOXW);
#define ARGS p, q, out, op.nx, op.ny, op.nz, c1, c2, ctl, 1.0
                if (first) {
                    if (mom) k_cheb_star_reg<true, true><<<g3, block, 0, st>>>(ARGS, mom, (int)g3.x);
                    else k_cheb_star_reg<true, false><<<g3, block, 0, st>>>(ARGS, nullptr, (int)g3.x);
                } else {
                    if (mom) k_cheb_star_reg<false, true><<<g3, block, 0, st>>>(ARGS, mom, (int)g3.x);
                    else k_cheb_star_reg<false, false><<<g3, block, 0, st>>>(ARGS, nullptr, (int)g3.x);
                }
#undef ARGS
                return;
            }
        }
        if (use_pair(op, p, q, out)) {
            const dim3 g2 = pair_grid(op, kz_step<T>());
#define ARGS p, q, out, op.nx, op.ny, op.nz, c1, c2, ctl, T(1)
            SSTEP_STEP_LAUNCH(k_cheb_poisson_pair, g2, T, DIM);
#undef ARGS
            return;
        }
#define ARGS p, q, out, op.nx, op.ny, op.nz, f, c1, c2, T(0), T(1), ctl, T(1)
        SSTEP_STEP_LAUNCH(k_cheb_stencil, grid, T, DIM, true, true);
#undef ARGS
        return;
    }
    if (jacobi) {
        const T c1 = (T)(c * (1.0 - sigma));
        const T csc = first ? T(0.5) : T(1);
#define ARGS p, q, out, op.nx, op.ny, op.nz, f, c1, T(0), T(0), csc, ctl, T(1)
        SSTEP_STEP_LAUNCH(k_cheb_stencil, grid, T, DIM, false, true);
#undef ARGS
    } else {
        const T cc = (T)c, cs = (T)sigma;
#define ARGS p, q, out, op.nx, op.ny, op.nz, f, cc, T(0), cs, T(1), ctl, T(1)
        SSTEP_STEP_LAUNCH(k_cheb_stencil, grid, T, DIM, false, false);
#undef ARGS
    }
}

}  // namespace

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// the driver's tensor-map encoder, resolved once (null when the driver has none)
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}
// an nx x ny x nz FP32 array read in bx x by x 1 boxes, zeros outside
bool encode_box_map(float* base, const OpDesc& op, int bx, int by, CUtensorMap* m) {
    const cuuint64_t gdim[3] = {(cuuint64_t)op.nx, (cuuint64_t)op.ny, (cuuint64_t)op.nz};
    const cuuint64_t gstride[2] = {(cuuint64_t)op.nx * 4, (cuuint64_t)op.nx * op.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estride[3] = {1, 1, 1};
    return encode_tiled()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, gdim, gstride, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
dim3 step_tma_grid(const OpDesc& op) {
    return dim3((op.nx + TMX - 1) / TMX, (op.ny + TMY - 1) / TMY, (op.nz + TMKZ - 1) / TMKZ);
}
}  // namespace

bool step_tma_shape(const OpDesc& op) {
    return op.kind == OP_STENCIL && !op.box && op.wx == nullptr && op.dim == 3 && op.nx % 4 == 0 && op.nx >= 4 &&
           op.ny >= 1 && op.nz >= 1;
}

cudaError_t step_tma_maps(const OpDesc& op, float* column, CUtensorMap* mp, CUtensorMap* mq) {
    if (!step_tma_shape(op) || (uintptr_t)column % 16 != 0 || !encode_tiled()) return cudaErrorNotSupported;
    if (!encode_box_map(column, op, TPX, TPY, mp) || !encode_box_map(column, op, TMX, TMY, mq))
        return cudaErrorNotSupported;
    return cudaSuccess;
}

cudaError_t launch_cheb_step_tma(const OpDesc& op, const CUtensorMap& mp, const CUtensorMap& mq, float* out,
                                 double theta, double sigma, bool first, bool jacobi, Ctl* ctl, cudaStream_t st,
                                 void* mom) {
    if (!step_tma_shape(op)) return cudaErrorInvalidValue;
    // the constants of cheb_stencil_dispatch's Poisson branch
    const double c = first ? theta : 2.0 * theta, d2 = 2.0 * op.dim;
    const float c1 = (float)(jacobi ? c * (1.0 - sigma) : c * (d2 - sigma));
    const float c2 = (float)(jacobi ? -c / d2 : -c);
    const dim3 g = step_tma_grid(op), block(32, TMY);
    const int nb = (int)(g.x * g.y * g.z);
    if (first) {
        if (mom) k_cheb_poisson_tma<true, true><<<g, block, 0, st>>>(mp, mq, out, op.nx, op.ny, op.nz, c1, c2, ctl, 1.f, mom, nb);
        else k_cheb_poisson_tma<true, false><<<g, block, 0, st>>>(mp, mq, out, op.nx, op.ny, op.nz, c1, c2, ctl, 1.f, nullptr, nb);
    } else {
        if (mom) k_cheb_poisson_tma<false, true><<<g, block, 0, st>>>(mp, mq, out, op.nx, op.ny, op.nz, c1, c2, ctl, 1.f, mom, nb);
        else k_cheb_poisson_tma<false, false><<<g, block, 0, st>>>(mp, mq, out, op.nx, op.ny, op.nz, c1, c2, ctl, 1.f, nullptr, nb);
    }
    return cudaGetLastError();
}

cudaError_t tma_wait_selftest(int* done_state) {
    *done_state = -1;
    OpDesc op{};
    op.kind = OP_STENCIL;
    op.dim = 3;
    op.nx = 64;
    op.ny = 8;
    op.nz = 4;
    op.n = (int64_t)op.nx * op.ny * op.nz;
    float* v = nullptr;
    Ctl* ctl = nullptr;
    cudaError_t e = cudaMalloc(&v, sizeof(float) * 2 * op.n);
    if (e == cudaSuccess) e = cudaMalloc(&ctl, sizeof(Ctl));
    CUtensorMap mp, mq;
    if (e == cudaSuccess) e = cudaMemset(v, 0, sizeof(float) * 2 * op.n);
    if (e == cudaSuccess) e = cudaMemset(ctl, 0, sizeof(Ctl));
    if (e == cudaSuccess) e = step_tma_maps(op, v, &mp, &mq);
    if (e == cudaSuccess) {
        // one block; its copies deliver 16 bytes less than each stage expects, and each wait
        // gives up after 4096 polls
        k_cheb_poisson_tma<false, false, true><<<step_tma_grid(op), dim3(32, TMY)>>>(mp, mq, v + op.n, op.nx, op.ny,
                                                                                    op.nz, 1.f, -1.f, ctl, 1.f, nullptr, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    Ctl h{};
    if (e == cudaSuccess) e = cudaMemcpy(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) *done_state = h.done;
    cudaFree(v);
    cudaFree(ctl);
    return e;
}

int cheb_step_blocks(const OpDesc& op, bool fp32, bool tma) {
    if (op.kind != OP_STENCIL) return 0;
    if (tma && fp32 && step_tma_shape(op)) {
        const dim3 g = step_tma_grid(op);
        return (int)(g.x * g.y * g.z);
    }
    const int kz = fp32 ? kz_step<float>() : kz_step<double>();
    dim3 g;
    if (op.box) {
        if (box_reg_shape(op)) g = fp32 ? box_reg_grid<float>(op) : box_reg_grid<double>(op);
        else g = fp32 && op.nx % 2 == 0 ? box_pair_grid(op) : box_grid(op);
    }
    else if (!fp32 && star_reg_shape(op)) g = star_reg_grid(op);
    else if (op.wx == nullptr && op.nx % 2 == 0) g = pair_grid(op, kz);
    else g = stencil_grid(op, kz);
    return (int)(g.x * g.y * g.z);
}

template <typename T>
cudaError_t launch_cheb_step(const OpDesc& op, const T* p, const T* q, T* out, double theta, double sigma, bool first,
                             bool jacobi, const Ctl* ctl, cudaStream_t st, void* mom) {
    if (mom) {
        // the fused moments need a stencil operator and the block count cheb_step_blocks reports
        if (op.kind != OP_STENCIL) return cudaErrorInvalidValue;
        if (!op.box && op.wx == nullptr && op.nx % 2 == 0 && !use_pair(op, p, q, out)) return cudaErrorInvalidValue;
        if (op.box && box_reg_shape(op) && !box_reg_ok<T>(op, p, q, out)) return cudaErrorInvalidValue;
        if (op.box && !box_reg_shape(op) && std::is_same<T, float>::value && op.nx % 2 == 0 &&
            !box_pair_ok(op, (const float*)p, (const float*)q, (const float*)out))
            return cudaErrorInvalidValue;
    }
    if (op.kind == OP_STENCIL && op.box) {
        // c (M^-1 A p - sigma p) = c (D + 1 - sigma) p - c B without a preconditioner and
        // c (1 - sigma + 1 / D) p - (c / D) B with Jacobi (D = 3^dim - 1)
        const double c = first ? theta : 2.0 * theta;
        const double D = op.dim == 3 ? 26.0 : 8.0;
        const T ca = (T)(jacobi ? c * (1.0 - sigma) + c / D : c * (D + 1.0 - sigma));
        const T cb = (T)(jacobi ? -c / D : -c);
        if (box_reg_ok<T>(op, p, q, out)) {
            const dim3 g3 = box_reg_grid<T>(op), block(32, BOXW);
#define ARGS p, q, out, op.nx, op.ny, op.nz, ca, cb, ctl, T(1)
            SSTEP_STEP_LAUNCH(k_cheb_box_reg, g3, T, BOXY);
#undef ARGS
            return cudaGetLastError();
        }
        const dim3 grid = box_grid(op), block(BX, BY);
        if (std::is_same<T, float>::value) {
            const float* pf = (const float*)p;
            const float* qf = (const float*)q;
            float* of = (float*)out;
            const float caf = (float)ca, cbf = (float)cb;
#define ARGS pf, qf, of, op.nx, op.ny, op.nz, caf, cbf, ctl
            if (box_pair_ok(op, pf, qf, of)) {
                const dim3 g2 = box_pair_grid(op);
                if (op.dim == 3) SSTEP_STEP_LAUNCH(k_cheb_box_f32_pair, g2, 3);
                else SSTEP_STEP_LAUNCH(k_cheb_box_f32_pair, g2, 2);
            } else {
                if (op.dim == 3) SSTEP_STEP_LAUNCH(k_cheb_box_f32, grid, 3);
                else SSTEP_STEP_LAUNCH(k_cheb_box_f32, grid, 2);
            }
#undef ARGS
            return cudaGetLastError();
        }
#define ARGS p, q, out, op.nx, op.ny, op.nz, ca, cb, ctl, T(1)
        if (op.dim == 3) SSTEP_STEP_LAUNCH(k_cheb_box, grid, T, 3);
        else SSTEP_STEP_LAUNCH(k_cheb_box, grid, T, 2);
#undef ARGS
        return cudaGetLastError();
    }
    if (op.kind == OP_STENCIL) {
        const bool poisson = op.wx == nullptr;
        if (op.dim == 3) {
            if (poisson) cheb_stencil_dispatch<T, 3, true>(op, p, q, out, theta, sigma, first, jacobi, ctl, mom, st);
            else cheb_stencil_dispatch<T, 3, false>(op, p, q, out, theta, sigma, first, jacobi, ctl, mom, st);
        } else {
            if (poisson) cheb_stencil_dispatch<T, 2, true>(op, p, q, out, theta, sigma, first, jacobi, ctl, mom, st);
            else cheb_stencil_dispatch<T, 2, false>(op, p, q, out, theta, sigma, first, jacobi, ctl, mom, st);
        }
        return cudaGetLastError();
    }
    const double c = first ? theta : 2.0 * theta;
    const int nb = vec_blocks(op.n);
    const T* cd = jacobi ? (std::is_same<T, double>::value ? (const T*)op.cdinv : (const T*)op.cdinv32) : nullptr;
    const T* v = csr_vals<T>(op);
    if (first) {
        if (jacobi) k_cheb_csr<T, true, true><<<nb, RB, 0, st>>>(op.rowptr, op.colind, v, cd, p, q, out, op.n, (T)c, (T)(c * sigma), T(0.5), ctl);
        else k_cheb_csr<T, true, false><<<nb, RB, 0, st>>>(op.rowptr, op.colind, v, cd, p, q, out, op.n, (T)c, (T)(c * sigma), T(1), ctl);
    } else {
        if (jacobi) k_cheb_csr<T, false, true><<<nb, RB, 0, st>>>(op.rowptr, op.colind, v, cd, p, q, out, op.n, (T)c, (T)(c * sigma), T(1), ctl);
        else k_cheb_csr<T, false, false><<<nb, RB, 0, st>>>(op.rowptr, op.colind, v, cd, p, q, out, op.n, (T)c, (T)(c * sigma), T(1), ctl);
    }
    return cudaGetLastError();
}
#undef SSTEP_STEP_LAUNCH

template cudaError_t launch_cheb_step<double>(const OpDesc&, const double*, const double*, double*, double, double,
                                              bool, bool, const Ctl*, cudaStream_t, void*);
template cudaError_t launch_cheb_step<float>(const OpDesc&, const float*, const float*, float*, double, double, bool,
                                             bool, const Ctl*, cudaStream_t, void*);

size_t residual_partials_needed(const OpDesc& op) {
    if (op.kind == OP_STENCIL && op.box) {
        // either kernel may run (the register-blocked one needs aligned vectors)
        const dim3 g = box_grid(op);
        const size_t n1 = (size_t)g.x * g.y * g.z;
        if (!box_reg_shape(op)) return n1;
        return std::max(n1, (size_t)box_res_reg_grid(op).x);
    }
    if (op.kind == OP_STENCIL) {
        // either kernel may run for the 7-point operator (the register-blocked one needs
        // aligned vectors)
        const dim3 g = stencil_grid(op, KZ_RES);
        const size_t n1 = (size_t)g.x * g.y * g.z;
        return star_reg_shape(op) ? std::max(n1, (size_t)star_res_grid(op).x) : n1;
    }
    return (size_t)vec_blocks(op.n);
}

cudaError_t launch_residual(const OpDesc& op, const double* b, const double* x, double* r, float* r32,
                            double* partials, Ctl* ctl, int mode, cudaStream_t st) {
    if (op.kind == OP_STENCIL && op.box) {
        if (box_res_reg_ok(op, b, x, r, r32)) {
            k_residual_box_reg<<<box_res_reg_grid(op), dim3(32, BOXW), 0, st>>>(b, x, r, r32, op.nx, op.ny, op.nz,
                                                                               partials, ctl, mode, 1.0);
            return cudaGetLastError();
        }
        const dim3 grid = box_grid(op), block(BX, BY);
        if (op.dim == 3) k_residual_box<3><<<grid, block, 0, st>>>(b, x, r, r32, op.nx, op.ny, op.nz, partials, ctl, mode, 1.0);
        else k_residual_box<2><<<grid, block, 0, st>>>(b, x, r, r32, op.nx, op.ny, op.nz, partials, ctl, mode, 1.0);
        return cudaGetLastError();
    }
    if (op.kind == OP_STENCIL && star_reg_shape(op) && (uintptr_t)b % 16 == 0 && (uintptr_t)x % 16 == 0 &&
        (!r || (uintptr_t)r % 16 == 0) && (!r32 || (uintptr_t)r32 % 8 == 0)) {
        k_residual_star_reg<<<star_res_grid(op), dim3(32, BOXW), 0, st>>>(b, x, r, r32, op.nx, op.ny, op.nz,
                                                                          2.0 * op.dim, partials, ctl, mode, 1.0);
        return cudaGetLastError();
    }
    if (op.kind == OP_STENCIL) {
        const dim3 grid = stencil_grid(op, KZ_RES), block(BX, BY);
        const Faces<double> f = faces_of<double>(op);
        const double d2 = 2.0 * op.dim;
        const bool poisson = op.wx == nullptr;
        if (op.dim == 3) {
            if (poisson) k_residual_stencil<3, true><<<grid, block, 0, st>>>(b, x, r, r32, op.nx, op.ny, op.nz, f, d2, partials, ctl, mode, 1.0);
            else k_residual_stencil<3, false><<<grid, block, 0, st>>>(b, x, r, r32, op.nx, op.ny, op.nz, f, d2, partials, ctl, mode, 1.0);
        } else {
            if (poisson) k_residual_stencil<2, true><<<grid, block, 0, st>>>(b, x, r, r32, op.nx, op.ny, op.nz, f, d2, partials, ctl, mode, 1.0);
            else k_residual_stencil<2, false><<<grid, block, 0, st>>>(b, x, r, r32, op.nx, op.ny, op.nz, f, d2, partials, ctl, mode, 1.0);
        }
        return cudaGetLastError();
    }
    k_residual_csr<<<vec_blocks(op.n), RB, 0, st>>>(op.rowptr, op.colind, op.vals, b, x, r, r32, op.n, partials, ctl, mode);
    return cudaGetLastError();
}

namespace {
__global__ void k_convert_check(const double* __restrict__ in, int k, float* __restrict__ out, double* __restrict__ back,
                                int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)RB + threadIdx.x; e < n; e += (int64_t)gridDim.x * RB) {
        const float f = d2f_scaled(in[e], k);
        out[e] = f;
        back[e] = f2d_exact(f);
    }
}
}  // namespace

cudaError_t launch_convert_check(const double* in, int k, float* out, double* back, int64_t n, cudaStream_t st) {
    k_convert_check<<<vec_blocks(n), RB, 0, st>>>(in, k, out, back, n);
    return cudaGetLastError();
}

cudaError_t launch_apply(const OpDesc& op, const double* x, double* y, cudaStream_t st) {
    if (op.kind == OP_STENCIL && op.box) {
        const dim3 grid = box_grid(op), block(BX, BY);
        if (op.dim == 3) k_apply_box<3><<<grid, block, 0, st>>>(x, y, op.nx, op.ny, op.nz);
        else k_apply_box<2><<<grid, block, 0, st>>>(x, y, op.nx, op.ny, op.nz);
        return cudaGetLastError();
    }
    if (op.kind == OP_STENCIL) {
        const dim3 grid = stencil_grid(op), block(BX, BY);
        const Faces<double> f = faces_of<double>(op);
        const double d2 = 2.0 * op.dim;
        const bool poisson = op.wx == nullptr;
        if (op.dim == 3) {
            if (poisson) k_apply_stencil<3, true><<<grid, block, 0, st>>>(x, y, op.nx, op.ny, op.nz, f, d2);
            else k_apply_stencil<3, false><<<grid, block, 0, st>>>(x, y, op.nx, op.ny, op.nz, f, d2);
        } else {
            if (poisson) k_apply_stencil<2, true><<<grid, block, 0, st>>>(x, y, op.nx, op.ny, op.nz, f, d2);
            else k_apply_stencil<2, false><<<grid, block, 0, st>>>(x, y, op.nx, op.ny, op.nz, f, d2);
        }
        return cudaGetLastError();
    }
    k_apply_csr<<<vec_blocks(op.n), RB, 0, st>>>(op.rowptr, op.colind, op.vals, x, y, op.n);
    return cudaGetLastError();
}

}  // namespace sstep
