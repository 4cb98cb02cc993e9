// Fused Gram reduction + column scaling + FGS Gram solve (one launch per outer iteration).
//
// What it computes (arXiv 2512.09642, Section 2): G = P^T A P and c = P^T r_k for the
// Chebyshev basis P = [p_0 .. p_(s-1)], p_0 = r_k; the scaling d_i = G_ii^-1/2 with
// G~ = S G S, c~ = S c; nu FGS sweeps (I + L) a^(l+1) = c~ - L^T a^(l), a^(0) = 0; alpha = S a.
//
// How (GB300 design):
//  * A P is never formed. With M the preconditioner of the recurrence, the basis satisfies
//    A p_j = M (p_(j+1) + p_(j-1)) / (2 theta) + sigma M p_j (j >= 1), A p_0 = M p_1 / theta
//    + sigma M p_0, i.e. A P = M P_+ B with P_+ = [P, p_s] and B the (s+1) x s tridiagonal
//    change-of-basis matrix. One streaming pass over P_+ therefore reduces W = P^T M P_+
//    (s(s+1)/2 symmetric entries + s entries against p_s) and, when M is not a multiple of I,
//    c = P^T p_0; G = W B is assembled at the end.
//  * Each warp owns a compile-time subset of the entries (s <= 8: all of them), so the
//    accumulators stay in registers and each FP64 FMA is useful work.
//  * Deterministic: fixed per-thread order, fixed butterfly, fixed order over warps, then
//    the last block to arrive sums the per-block partials in block order.
//  * The last block then runs the s x s work in one warp: lane j owns row j of G~, and each
//    FGS sweep is s dependent warp-wide FMAs (a warp FP64 instruction costs the same with
//    one active lane as with 32 on this part, so the sweep keeps all lanes busy).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace sstep {

constexpr int GRAM_THREADS = 512;
constexpr int GRAM_WARPS = GRAM_THREADS / 32;

// Entry count M of one Gram pass and the number G of warp roles that split it: the smallest
// G in {1, 2, 4, 8, 16} that keeps a role's accumulators within budget (FP64: 46 doubles;
// mixed form: 28 compensated FP32 pairs).
__host__ __device__ constexpr int gram_roles(int m, int budget) {
    int g = 1;
    while (g < 16 && (m + g - 1) / g > budget) g *= 2;
    return g;
}

template <int S, bool DV, bool MOM = false>
struct GramShape {
    static constexpr int NSYM = S * (S + 1) / 2;    // p_a^T M p_b, 0 <= a <= b < S
    static constexpr int NLAST = S;                 // p_a^T M p_S
    // direct: the NSYM + NLAST entries of W; moments: the 2S moments' inner products
    static constexpr int M = (MOM ? 2 * S : NSYM + NLAST) + (DV ? S : 0);
    static constexpr int G = gram_roles(M, 46);     // warp roles, FP64 form
    static constexpr int NSLAB = GRAM_WARPS / G;
    static constexpr int G32 = gram_roles(M, 16);   // warp roles, mixed form (two blocks per SM)
    static constexpr int NSLAB32 = GRAM_WARPS / G32;
};

struct AB { int a, b, kind; };  // kind 0: p_a^T M p_b, 1: p_a^T p_0 (unweighted c)

// Moments form (gram_form MOMENTS): the basis is p_j = T_j(A^) p_0 with A^ = theta (M^-1 A -
// sigma) self-adjoint in <u, v>_M = u^T M v, so <p_i, p_j>_M = (mu_(i+j) + mu_|i-j|) / 2 with
// mu_k = <p_0, T_k(A^) p_0>_M (the spectral expansion used in Section 4's proof). The entries
// are mu_k = <p_0, p_k>_M for k <= s and, for s < k < 2s, <p_m, p_m>_M (k = 2m, giving
// mu_k = 2 <p_m, p_m>_M - mu_0) or <p_(m+1), p_m>_M (k = 2m + 1, mu_k = 2 <.,.>_M - mu_1).
template <int S, bool DV, bool MOM = false>
__host__ __device__ constexpr AB gram_entry(int e) {
    constexpr int NSYM = S * (S + 1) / 2;
    if (MOM) {
        if (e <= S) return AB{0, e, 0};
        if (e < 2 * S) {
            const int k = e;
            return (k % 2 == 0) ? AB{k / 2, k / 2, 0} : AB{(k - 1) / 2, (k + 1) / 2, 0};
        }
        return AB{e - 2 * S, 0, 1};
    }
    if (e < NSYM) {
        int a = 0, len = S;
        while (e >= len) { e -= len; ++a; --len; }
        return AB{a, a + e, 0};
    }
    e -= NSYM;
    if (e < S) return AB{e, S, 0};
    e -= S;
    return AB{e, 0, 1};
}

// Compile-time list of the entries owned by warp role Q (entries e with e % G == Q).
template <int S, bool DV, int Q, int G_ = GramShape<S, DV>::G, bool MOM = false>
struct RoleTable {
    static constexpr int G = G_;
    static constexpr int M = GramShape<S, DV, MOM>::M;
    static constexpr int MQ = (M - Q + G - 1) / G;
    int a[MQ > 0 ? MQ : 1], b[MQ > 0 ? MQ : 1], kind[MQ > 0 ? MQ : 1], e[MQ > 0 ? MQ : 1];
    __host__ __device__ constexpr RoleTable() : a(), b(), kind(), e() {
        int k = 0;
        for (int ee = Q; ee < M; ee += G) {
            const AB ab = gram_entry<S, DV, MOM>(ee);
            a[k] = ab.a;
            b[k] = ab.b;
            kind[k] = ab.kind;
            e[k] = ee;
            ++k;
        }
    }
};

// Per-role accumulation over this thread's elements, then warp reduction and one write per
// entry into smem[slab * M + entry] by lane 0.
template <int S, bool DV, int Q, bool MOM = false>
__device__ __forceinline__ void gram_role_f64(const double* __restrict__ P, int64_t ld, const double* __restrict__ diag,
                                              int64_t n, int64_t e0, int64_t stride, double* smem, int slab) {
    constexpr int G = GramShape<S, DV, MOM>::G;
    constexpr int M = GramShape<S, DV, MOM>::M;
    constexpr int MQ = (M - Q + G - 1) / G;
    constexpr RoleTable<S, DV, Q, G, MOM> RT{};
    double acc[MQ > 0 ? MQ : 1];
#pragma unroll
    for (int k = 0; k < MQ; ++k) acc[k] = 0.0;
    for (int64_t e = e0; e < n; e += stride) {
        double pv[S + 1];
#pragma unroll
        for (int c = 0; c <= S; ++c) pv[c] = __ldg(P + c * ld + e);
        double dq[S];
        if constexpr (DV) {
            const double dv = __ldg(diag + e);
#pragma unroll
            for (int a = 0; a < S; ++a) dq[a] = dv * pv[a];
        } else {
#pragma unroll
            for (int a = 0; a < S; ++a) dq[a] = pv[a];
        }
#pragma unroll
        for (int k = 0; k < MQ; ++k)
            acc[k] = fma(RT.kind[k] == 0 ? dq[RT.a[k]] : pv[RT.a[k]], pv[RT.b[k]], acc[k]);
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < MQ; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) smem[slab * M + RT.e[k]] = v;
    }
}

template <int S, bool DV, int Q = 0, bool MOM = false>
__device__ __forceinline__ void gram_role_dispatch(int q, const double* P, int64_t ld, const double* diag, int64_t n,
                                                   int64_t e0, int64_t stride, double* smem, int slab) {
    if constexpr (Q < GramShape<S, DV, MOM>::G) {
        if (q == Q) gram_role_f64<S, DV, Q, MOM>(P, ld, diag, n, e0, stride, smem, slab);
        else gram_role_dispatch<S, DV, Q + 1, MOM>(q, P, ld, diag, n, e0, stride, smem, slab);
    }
}

// Mixed form: P holds FP32 vectors. Each product p_a p_b is formed exactly (FMA-based
// TwoProduct) and summed per thread in a compensated FP32 pair (Dot2 of Ogita, Rump and
// Oishi, about 48 significant bits); the per-thread sums are converted exactly to FP64 and
// all further reduction (warps, blocks, grid) is in FP64.
template <int S, bool DV, int Q, bool MOM = false>
__device__ __forceinline__ void gram_role_f32(const float* __restrict__ P, int64_t ld, const float* __restrict__ diag,
                                              int64_t n, int64_t e0, int64_t stride, double* smem, int slab) {
    constexpr int G = GramShape<S, DV, MOM>::G32;
    constexpr int M = GramShape<S, DV, MOM>::M;
    constexpr int MQ = (M - Q + G - 1) / G;
    constexpr RoleTable<S, DV, Q, G, MOM> RT{};
    float ah[MQ > 0 ? MQ : 1], al[MQ > 0 ? MQ : 1];
#pragma unroll
    for (int k = 0; k < MQ; ++k) ah[k] = al[k] = 0.f;
    auto element = [&](const float* pv, float dv) {
        float dq[S];
        if constexpr (DV) {
#pragma unroll
            for (int a = 0; a < S; ++a) dq[a] = __fmul_rn(dv, pv[a]);
        } else {
#pragma unroll
            for (int a = 0; a < S; ++a) dq[a] = pv[a];
        }
#pragma unroll
        for (int k = 0; k < MQ; ++k) dot2_acc(RT.kind[k] == 0 ? dq[RT.a[k]] : pv[RT.a[k]], pv[RT.b[k]], ah[k], al[k]);
    };
    // moments form: two consecutive elements per thread and iteration, loaded as 8-byte pairs
    // (ld is even and the columns 8-byte aligned): twice the loads in flight per warp, which
    // this latency-bound pass needs (0.175 -> 0.143 ms at 256^3, s = 8); an odd last element
    // is read alone. The direct form, with more accumulators per role, keeps one element per
    // iteration, as does s = 4 with a vector M: two spilled registers there.
    if constexpr (!MOM || (DV && S == 4)) {
        for (int64_t e = e0; e < n; e += stride) {
            float pv[S + 1];
#pragma unroll
            for (int c = 0; c <= S; ++c) pv[c] = __ldg(P + c * ld + e);
            element(pv, DV ? __ldg(diag + e) : 1.f);
        }
    } else {
        for (int64_t e = 2 * e0; e < n; e += 2 * stride) {
            float pa[S + 1], pb[S + 1];
            float da = 1.f, db = 1.f;
            if (e + 1 < n) {
#pragma unroll
                for (int c = 0; c <= S; ++c) {
                    const float2 v = __ldg(reinterpret_cast<const float2*>(P + c * ld + e));
                    pa[c] = v.x;
                    pb[c] = v.y;
                }
                if constexpr (DV) {
                    if (((uintptr_t)diag & 7u) == 0u) {
                        const float2 d2 = __ldg(reinterpret_cast<const float2*>(diag + e));
                        da = d2.x;
                        db = d2.y;
                    } else {
                        da = __ldg(diag + e);
                        db = __ldg(diag + e + 1);
                    }
                }
                element(pa, da);
                element(pb, db);
            } else {
#pragma unroll
                for (int c = 0; c <= S; ++c) pa[c] = __ldg(P + c * ld + e);
                if constexpr (DV) da = __ldg(diag + e);
                element(pa, da);
            }
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < MQ; ++k) {
        const double v = warp_sum(f2d_exact(ah[k]) + f2d_exact(al[k]));
        if (lane == 0) smem[slab * M + RT.e[k]] = v;
    }
}

template <int S, bool DV, int Q = 0, bool MOM = false>
__device__ __forceinline__ void gram_role_dispatch32(int q, const float* P, int64_t ld, const float* diag, int64_t n,
                                                     int64_t e0, int64_t stride, double* smem, int slab) {
    if constexpr (Q < GramShape<S, DV, MOM>::G32) {
        if (q == Q) gram_role_f32<S, DV, Q, MOM>(P, ld, diag, n, e0, stride, smem, slab);
        else gram_role_dispatch32<S, DV, Q + 1, MOM>(q, P, ld, diag, n, e0, stride, smem, slab);
    }
}

struct GramParams {
    int nu, solver;
    int check;                   // 1: convergence / max-outer test on c_0 = ||r_k||^2 (FP64 form);
                                 // 2: the same on c_0 / scale^2 (mixed form between refreshes);
                                 // 0: done by the FP64 residual refresh (mixed form)
    double theta, sigma, dfac;   // dfac: constant diagonal of M (1 when M = I); unused if DV
    // block-conjugated form (conj = 1): per-block partials of C = (A Q_(k-1))^T P_k and
    // d = Q_(k-1)^T r_k from k_conj_cd, and the state cj = [W_(k-1) | B_k] (row-major s x s each)
    int conj, conj_nblk;
    const double* conj_partials;
    double* cj;
    int fp32;                    // the basis is the mixed form's scaled FP32 copy
    double* hist;                // per-outer record ring (outer, ||r||^2 / ||r_0||^2, delta, min G_ii)
    int hist_cap;
};

// nu forward Gauss-Seidel sweeps on one right-hand side, lane j owning row j (lanes >= S and
// rows whose bit is clear in `kept` hold 0): grow = row `lane` of the scaled matrix divided by
// its diagonal, chat = the scaled right-hand side over the same diagonal. A sweep is S
// warp-wide steps: step i broadcasts a_i = w_i and every other row takes its product into its
// accumulator w, which row i then restarts at chat; so when step j reads it, w_j = chat_j -
// sum_(i > j) G^_ji a_i (previous sweep) - sum_(i < j) G^_ji a_i (this sweep), the terms in
// the order of i. The dropped rows and columns are zeroed once up front (their a_i stay 0),
// so a step's dependent chain is one shuffle, one FMA and one select. Returns a_lane.
template <int S>
__device__ __forceinline__ double fgs_lane(const double (&grow_in)[S], double chat, unsigned kept, int nu) {
    const int lane = threadIdx.x & 31;
    const bool kj = lane < S && ((kept >> lane) & 1u);
    double grow[S];
#pragma unroll
    for (int i = 0; i < S; ++i) grow[i] = (kj && ((kept >> i) & 1u)) ? grow_in[i] : 0.0;
    if (!kj) chat = 0.0;
    double a = 0.0, w = chat;
    for (int sweep = 0; sweep < nu; ++sweep) {
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const double ai = __shfl_sync(0xffffffffu, w, i);
            const double wn = fma(-grow[i], ai, w);
            if (lane == i) a = ai;
            w = lane == i ? chat : wn;
        }
    }
    return a;
}

// Block conjugation (the Chronopoulos-Gear s-step CG cited in Section 1), applied to the
// s x s quantities of outer iteration k before its Gram solve (warp 0). With Q_k = P_k -
// Q_(k-1) B_k, B_k = W_(k-1)^-1 C, C = (A Q_(k-1))^T P_k:
//   W_k = Q_k^T A Q_k = G - C^T B - B^T C + B^T W_(k-1) B,   g = Q_k^T r_k = c - B^T d,
// with G = P_k^T A P_k, c = P_k^T r_k and d = Q_(k-1)^T r_k. B is solved column by column
// with the same column scaling and nu FGS sweeps as the Gram system. Gs / cs hold G and c on
// entry and W_k and g on exit; cj receives W_k and B for the next iteration and the update.
// scr: >= 3 S^2 + S doubles. The first block (conj_valid = 0) has Q = P, B = 0.
template <int S>
__device__ void conj_transform(double* Gs, double* cs, const double* totc, const GramParams& gp, Ctl* ctl,
                               double* scr) {
    const int lane = threadIdx.x;
    double* B = scr;
    double* T = scr + S * S;
    double* Wp = scr + 2 * S * S;
    double* dw = scr + 3 * S * S;
    const double* C = totc;            // C[i * S + j] = (A q_i)^T p_j
    const double* dq = totc + S * S;   // d[i] = q_i^T r
    const bool valid = ctl->conj_valid != 0;
    if (!valid) {
        for (int idx = lane; idx < S * S; idx += 32) B[idx] = 0.0;
        __syncwarp();
    } else {
        for (int idx = lane; idx < S * S; idx += 32) Wp[idx] = gp.cj[idx];
        __syncwarp();
        const double gjj = lane < S ? Wp[lane * S + lane] : 0.0;
        const bool keep = lane < S && gjj > 0.0 && isfinite(gjj);
        const double dj = keep ? 1.0 / sqrt(gjj) : 0.0;
        if (lane < S) dw[lane] = dj;
        const unsigned kept = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (gp.solver == SSTEP_GRAM_SOLVE_FGS) {
            const double gd = keep ? dj * gjj * dj : 1.0;
            const double inv = keep ? 1.0 / gd : 0.0;
            double grow[S];
#pragma unroll
            for (int i = 0; i < S; ++i) grow[i] = lane < S ? dj * Wp[lane * S + i] * dw[i] * inv : 0.0;
            for (int j = 0; j < S; ++j) {
                const double chat = lane < S ? dj * C[lane * S + j] * inv : 0.0;
                const double a = fgs_lane<S>(grow, chat, kept, gp.nu);
                if (lane < S) B[lane * S + j] = dj * a;
            }
        } else if (lane == 0) {
            // Cholesky of the scaled kept block of W_(k-1) (R in T's storage), then the S columns
            double* R = T;
            bool ok = true;
            for (int j = 0; j < S && ok; ++j) {
                if (!((kept >> j) & 1u)) continue;
                double accd = dw[j] * Wp[j * S + j] * dw[j];
                for (int k = 0; k < j; ++k)
                    if ((kept >> k) & 1u) accd -= R[k * S + j] * R[k * S + j];
                if (!(accd > 0.0)) { ok = false; break; }
                R[j * S + j] = sqrt(accd);
                for (int i = j + 1; i < S; ++i) {
                    if (!((kept >> i) & 1u)) continue;
                    double v = dw[j] * Wp[j * S + i] * dw[i];
                    for (int k = 0; k < j; ++k)
                        if ((kept >> k) & 1u) v -= R[k * S + j] * R[k * S + i];
                    R[j * S + i] = v / R[j * S + j];
                }
            }
            for (int col = 0; col < S; ++col) {
                double y[S], a[S];
                for (int i = 0; i < S; ++i) {
                    y[i] = 0.0;
                    if (!ok || !((kept >> i) & 1u)) continue;
                    double v = dw[i] * C[i * S + col];
                    for (int k = 0; k < i; ++k)
                        if ((kept >> k) & 1u) v -= R[k * S + i] * y[k];
                    y[i] = v / R[i * S + i];
                }
                for (int i = S - 1; i >= 0; --i) {
                    a[i] = 0.0;
                    if (!ok || !((kept >> i) & 1u)) continue;
                    double v = y[i];
                    for (int k = i + 1; k < S; ++k)
                        if ((kept >> k) & 1u) v -= R[i * S + k] * a[k];
                    a[i] = v / R[i * S + i];
                }
                for (int i = 0; i < S; ++i) B[i * S + col] = dw[i] * a[i];
            }
            if (!ok) ctl->done = NUMERICAL;
        }
        __syncwarp();
        if (ctl->done != RUNNING) return;
        // T = W_(k-1) B
        for (int idx = lane; idx < S * S; idx += 32) {
            const int i = idx / S, b = idx % S;
            double v = 0.0;
            for (int k = 0; k < S; ++k) v = fma(Wp[i * S + k], B[k * S + b], v);
            T[idx] = v;
        }
        __syncwarp();
        // W_k from its lower triangle, mirrored
        for (int idx = lane; idx < S * S; idx += 32) {
            const int a = idx / S, b = idx % S;
            if (a < b) continue;
            double w = Gs[a * S + b];
            for (int i = 0; i < S; ++i) {
                w = fma(-C[i * S + a], B[i * S + b], w);
                w = fma(-B[i * S + a], C[i * S + b], w);
                w = fma(B[i * S + a], T[i * S + b], w);
            }
            Gs[a * S + b] = w;
            Gs[b * S + a] = w;
        }
        double g = 0.0;
        if (lane < S) {
            g = cs[lane];
            for (int i = 0; i < S; ++i) g = fma(-B[i * S + lane], dq[i], g);
        }
        __syncwarp();
        if (lane < S) cs[lane] = g;
        __syncwarp();
    }
    for (int idx = lane; idx < S * S; idx += 32) {
        gp.cj[idx] = Gs[idx];
        gp.cj[S * S + idx] = B[idx];
    }
    __syncwarp();
}

// The s x s work of one outer iteration, executed by warp 0 of the last block.
// tot[]: reduced entries (layout of gram_entry). Writes ctl.
template <int S, bool DV, bool MOM = false>
__device__ void gram_finish(const double* tot, const GramParams& gp, Ctl* ctl, double* sm /* >= 2*S*S + 4*S doubles */,
                            const double* totc = nullptr, double* cscr = nullptr) {
    const int lane = threadIdx.x;   // warp 0 only
    constexpr int NSYM = S * (S + 1) / 2;
    constexpr int NW = MOM ? 2 * S : NSYM + S;   // where the unweighted c entries start
    // the control block's inputs, read once up front (independent loads whose latency the
    // assembly of G hides; every lane takes the same decisions from them)
    const double c_scale = ctl->scale, c_r0 = ctl->r0_sq, c_tol = ctl->tol_sq, c_ming = ctl->min_gii;
    const int c_outer = ctl->outer, c_maxo = ctl->max_outer;
    double* Gs = sm;                // G~, row-major S x S
    double* cs = sm + S * S;        // c~
    double* ds = cs + S;            // d
    double* as = ds + S;            // a (scaled solution) then alpha
    double* mu = sm + S * S + 4 * S;   // moments form: mu_0 .. mu_(2S-1)
    if (MOM) {
        for (int k = lane; k < 2 * S; k += 32) {
            double m;
            if (k <= S) m = tot[k];
            else m = 2.0 * tot[k] - tot[k % 2];   // 2 <p_a, p_b>_M - mu_(a-b), a - b = k mod 2
            mu[k] = m;
        }
        __syncwarp();
    }
    auto Wsym = [&](int a, int b) -> double {   // p_a^T M p_b for a, b < S
        if (MOM) return 0.5 * (mu[a + b] + mu[a > b ? a - b : b - a]);
        if (a > b) { const int t = a; a = b; b = t; }
        return tot[a * S - a * (a - 1) / 2 + (b - a)];
    };
    auto W = [&](int i, int k) -> double {
        if (MOM) return 0.5 * (mu[i + k] + mu[i > k ? i - k : k - i]);
        return k < S ? Wsym(i, k) : tot[NSYM + i];
    };
    const double h0 = 1.0 / gp.theta, h1 = 0.5 / gp.theta;
    const double sc = DV ? 1.0 : gp.dfac;
    // G (lower triangle, mirrored) and c
    for (int idx = lane; idx < S * S; idx += 32) {
        const int i = idx / S, j = idx % S;
        const int ii = i >= j ? i : j, jj = i >= j ? j : i;  // compute from the lower triangle
        double g = gp.sigma * W(ii, jj);
        const double hj = jj == 0 ? h0 : h1;
        double nb = W(ii, jj + 1);
        if (jj >= 1) nb += W(ii, jj - 1);
        g = fma(hj, nb, g);
        Gs[idx] = sc * g;
    }
    if (lane < S) cs[lane] = DV ? tot[NW + lane] : Wsym(lane, 0);
    __syncwarp();
    // c_0 = ||p_0||^2; the mixed form's FP32 p_0 carries the power-of-two scale of its outer
    // iteration, which the stopping test between FP64 refreshes (check 2) takes out
    const double cs0 = cs[0];   // c_0 = ||p_0||^2 before the scaling (kept for the record)
    const double rk_sq = gp.check == 2 ? cs0 / (c_scale * c_scale) : cs0;
    {
        int done = RUNNING;
        if (!(rk_sq >= 0.0) || !isfinite(rk_sq)) done = NUMERICAL;
        if (gp.check) {
            if (done == RUNNING && (c_r0 == 0.0 || rk_sq < c_tol * c_r0)) done = CONVERGED;
            else if (done == RUNNING && c_outer >= c_maxo) done = MAX_OUTER;
        } else if (done == RUNNING && rk_sq == 0.0) {
            done = CONVERGED;   // the refreshed residual rounded to zero in FP32
        }
        if (lane == 0) {
            if (gp.check) ctl->rk_sq = rk_sq;
            ctl->done = done;
        }
        if (done != RUNNING) return;
    }
    if constexpr (S <= 16) {
        if (totc) {
            conj_transform<S>(Gs, cs, totc, gp, ctl, cscr);
            __syncwarp();
            if (ctl->done != RUNNING) return;
        }
    }
    // column scaling (Section 2, "Column scaling")
    double gjj = lane < S ? Gs[lane * S + lane] : 0.0;
    const bool keep = lane < S && gjj > 0.0 && isfinite(gjj);
    const double dj = keep ? 1.0 / sqrt(gjj) : 0.0;
    if (lane < S) ds[lane] = dj;
    double mg = lane < S ? gjj : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mg = fmin(mg, __shfl_xor_sync(0xffffffffu, mg, o));
    const unsigned kept = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    for (int idx = lane; idx < S * S; idx += 32) Gs[idx] = ds[idx / S] * Gs[idx] * ds[idx % S];
    if (lane < S) cs[lane] = dj * cs[lane];
    __syncwarp();
    bool finite = true;
    for (int idx = lane; idx < S * S; idx += 32) finite &= (bool)isfinite(Gs[idx]);
    if (lane < S) finite &= (bool)isfinite(cs[lane]);
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) ctl->min_gii = fmin(c_ming, mg);
    if (kept == 0u || !finite) {
        if (lane == 0) ctl->done = NUMERICAL;
        return;
    }
    double a = 0.0;   // a_lane
    if (gp.solver == SSTEP_GRAM_SOLVE_FGS) {
        // row lane of G~ normalised by its diagonal: a_j = c^_j - sum_{i != j} G^_ji a_i
        const double gd = lane < S ? Gs[lane * S + lane] : 1.0;
        const bool kj = (kept >> lane) & 1u;
        const double inv = kj ? 1.0 / gd : 0.0;
        double grow[S];
#pragma unroll
        for (int i = 0; i < S; ++i) grow[i] = lane < S ? Gs[lane * S + i] * inv : 0.0;
        const double chat = lane < S ? cs[lane] * inv : 0.0;
        a = fgs_lane<S>(grow, chat, kept, gp.nu);
    } else {
        // Cholesky of the kept block of G~ (lane 0, sequential), the O(s^3) baseline.
        double* R = sm + S * S + 4 * S;   // S*S scratch
        if (lane == 0) {
            bool ok = true;
            for (int j = 0; j < S && ok; ++j) {
                if (!((kept >> j) & 1u)) continue;
                double accd = Gs[j * S + j];
                for (int k = 0; k < j; ++k)
                    if ((kept >> k) & 1u) accd -= R[k * S + j] * R[k * S + j];
                if (!(accd > 0.0)) { ok = false; break; }
                R[j * S + j] = sqrt(accd);
                for (int i = j + 1; i < S; ++i) {
                    if (!((kept >> i) & 1u)) continue;
                    double t = Gs[j * S + i];
                    for (int k = 0; k < j; ++k)
                        if ((kept >> k) & 1u) t -= R[k * S + j] * R[k * S + i];
                    R[j * S + i] = t / R[j * S + j];
                }
            }
            if (ok) {
                double y[S];
                for (int i = 0; i < S; ++i) {
                    y[i] = 0.0;
                    if (!((kept >> i) & 1u)) continue;
                    double t = cs[i];
                    for (int k = 0; k < i; ++k)
                        if ((kept >> k) & 1u) t -= R[k * S + i] * y[k];
                    y[i] = t / R[i * S + i];
                }
                for (int i = S - 1; i >= 0; --i) {
                    as[i] = 0.0;
                    if (!((kept >> i) & 1u)) continue;
                    double t = y[i];
                    for (int k = i + 1; k < S; ++k)
                        if ((kept >> k) & 1u) t -= R[i * S + k] * as[k];
                    as[i] = t / R[i * S + i];
                }
            } else {
                ctl->done = NUMERICAL;
            }
        }
        __syncwarp();
        if (ctl->done != RUNNING) return;
        a = lane < S ? as[lane] : 0.0;
    }
    // inexactness delta = ||c~ - G~ a|| / ||c~|| (Section 7)
    if (lane < S) as[lane] = a;
    __syncwarp();
    double res = 0.0, cn = 0.0;
    if (lane < S) {
        double t = cs[lane];
        for (int i = 0; i < S; ++i) t = fma(-Gs[lane * S + i], as[i], t);
        res = t * t;
        cn = cs[lane] * cs[lane];
    }
    res = warp_sum(res);
    cn = warp_sum(cn);
    // alpha = S a; beta = B alpha (residual update coefficients)
    const double al = lane < S ? ds[lane] * a : 0.0;
    __syncwarp();
    if (lane < S) as[lane] = al;
    __syncwarp();
    for (int k = lane; k <= S; k += 32) {
        double b = k < S ? gp.sigma * as[k] : 0.0;
        if (k >= 1) b = fma(k - 1 == 0 ? h0 : h1, as[k - 1], b);
        if (k + 1 < S) b = fma(h1, as[k + 1], b);
        // const M: r = sum_k gamma_k p_k with gamma_0 = 1 - m beta_0, gamma_k = -m beta_k
        if (!DV) b = (k == 0) ? fma(-sc, b, 1.0) : -sc * b;
        ctl->beta[k] = b;
    }
    if (lane < S) {
        ctl->alpha[lane] = al;
        ctl->d[lane] = ds[lane];
        ctl->ct[lane] = cs[lane];
    }
    for (int idx = lane; idx < S * S; idx += 32) ctl->Gt[idx] = Gs[idx];
    if (lane == 0) {
        const double delta = cn > 0.0 ? sqrt(res / cn) : 0.0;
        ctl->delta = delta;
        ctl->outer = c_outer + 1;
        if (gp.hist) {
            const double r2 = gp.fp32 ? cs0 / (c_scale * c_scale) : cs0;
            double* rec = gp.hist + 4 * (size_t)(c_outer % gp.hist_cap);
            rec[0] = (double)(c_outer + 1);
            rec[1] = c_r0 > 0.0 ? r2 / c_r0 : 0.0;
            rec[2] = delta;
            rec[3] = mg;
        }
        if (totc) ctl->conj_valid = 1;
    }
}

// One block per SM for the FP64 forms (FP64-pipe bound); the FP32 (mixed) form is latency
// bound and runs two blocks per SM (registers capped at 64).
template <int S, bool DV, typename T, bool MOM>
__global__ void __launch_bounds__(GRAM_THREADS, std::is_same<T, float>::value ? 2 : 1) k_gram(const T* __restrict__ P, int64_t ld,
                                                         const T* __restrict__ diag, int64_t n,
                                                         double* partials, Ctl* ctl, GramParams gp) {
    if (ctl->done) return;
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int G = F32 ? GramShape<S, DV, MOM>::G32 : GramShape<S, DV, MOM>::G;
    constexpr int NSLAB = F32 ? GramShape<S, DV, MOM>::NSLAB32 : GramShape<S, DV, MOM>::NSLAB;
    constexpr int M = GramShape<S, DV, MOM>::M;
    constexpr int NSM = (NSLAB * M) > S * S * 2 + 4 * S ? NSLAB * M : S * S * 2 + 4 * S;
    __shared__ double smem[NSM];
    __shared__ double tot[M];
    __shared__ bool is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp % G, slab = warp / G;
    const int64_t e0 = ((int64_t)blockIdx.x * NSLAB + slab) * 32 + lane;
    const int64_t stride = (int64_t)gridDim.x * NSLAB * 32;
    if constexpr (F32) gram_role_dispatch32<S, DV, 0, MOM>(q, P, ld, diag, n, e0, stride, smem, slab);
    else gram_role_dispatch<S, DV, 0, MOM>(q, P, ld, diag, n, e0, stride, smem, slab);
    __syncthreads();
    for (int k = threadIdx.x; k < M; k += GRAM_THREADS) {
        double v = 0.0;
        for (int sl = 0; sl < NSLAB; ++sl) v += smem[sl * M + k];
        partials[(size_t)blockIdx.x * M + k] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&ctl->counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const int nblk = gridDim.x;
    for (int k = warp; k < M; k += GRAM_WARPS) {
        double v = 0.0;
        for (int b = lane; b < nblk; b += 32) v += ((volatile double*)partials)[(size_t)b * M + k];
        v = warp_sum(v);
        if (lane == 0) tot[k] = v;
    }
    // block-conjugated form (FP64, S <= 16): the C and d partials of k_conj_cd, summed in block
    // order like the Gram's
    constexpr bool CJ = !F32 && S <= 16;
    constexpr int MC = CJ ? S * S + S : 1;
    __shared__ double totc[MC];
    __shared__ double cscr[CJ ? 3 * S * S + S : 1];
    if (CJ && gp.conj) {
        for (int k = warp; k < MC; k += GRAM_WARPS) {
            double v = 0.0;
            for (int b = lane; b < gp.conj_nblk; b += 32) v += gp.conj_partials[(size_t)b * MC + k];
            v = warp_sum(v);
            if (lane == 0) totc[k] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) ctl->counter = 0u;
    if (warp == 0) {
        if (CJ && gp.conj) gram_finish<S, DV, MOM>(tot, gp, ctl, smem, totc, cscr);
        else gram_finish<S, DV, MOM>(tot, gp, ctl, smem);
    }
}

// Resident blocks per SM of the kernel variant g selects (for sizing the grid).
template <int S>
int gram_occupancy_s(const GramArgs& g) {
    int occ = 1;
    const bool mom = g.form == SSTEP_GRAM_FORM_MOMENTS;
    cudaError_t e;
#define SSTEP_OCC(DV, T, MOM) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram<S, DV, T, MOM>, GRAM_THREADS, 0)
    if (g.fp32) {
        if (g.dvec) { if (mom) SSTEP_OCC(true, float, true); else SSTEP_OCC(true, float, false); }
        else { if (mom) SSTEP_OCC(false, float, true); else SSTEP_OCC(false, float, false); }
    } else {
        if (g.dvec) { if (mom) SSTEP_OCC(true, double, true); else SSTEP_OCC(true, double, false); }
        else { if (mom) SSTEP_OCC(false, double, true); else SSTEP_OCC(false, double, false); }
    }
#undef SSTEP_OCC
    return (e == cudaSuccess && occ > 0) ? occ : 1;
}

inline GramParams gram_params(const GramArgs& g) {
    GramParams gp{};
    gp.nu = g.nu;
    gp.solver = g.solver;
    gp.check = g.check;
    gp.theta = g.theta;
    gp.sigma = g.sigma;
    gp.dfac = g.dconst;
    gp.conj = g.conj;
    gp.conj_nblk = g.conj_nblk;
    gp.conj_partials = g.conj_partials;
    gp.cj = g.cj;
    gp.fp32 = g.fp32 ? 1 : 0;
    gp.hist = g.hist;
    gp.hist_cap = g.hist_cap;
    return gp;
}

template <int S>
cudaError_t launch_gram_s(const GramArgs& g, double* partials, Ctl* ctl, int nblocks, cudaStream_t st) {
    const GramParams gp = gram_params(g);
    const bool mom = g.form == SSTEP_GRAM_FORM_MOMENTS;
#define SSTEP_GRAM_LAUNCH(DV, T, MOM, DIAG) \
    k_gram<S, DV, T, MOM><<<nblocks, GRAM_THREADS, 0, st>>>((const T*)g.P, g.ld, DIAG, g.n, partials, ctl, gp)
    if (g.fp32) {
        if (g.dvec) {
            if (mom) SSTEP_GRAM_LAUNCH(true, float, true, g.diag32);
            else SSTEP_GRAM_LAUNCH(true, float, false, g.diag32);
        } else {
            if (mom) SSTEP_GRAM_LAUNCH(false, float, true, (const float*)nullptr);
            else SSTEP_GRAM_LAUNCH(false, float, false, (const float*)nullptr);
        }
    } else {
        if (g.dvec) {
            if (mom) SSTEP_GRAM_LAUNCH(true, double, true, g.diag);
            else SSTEP_GRAM_LAUNCH(true, double, false, g.diag);
        } else {
            if (mom) SSTEP_GRAM_LAUNCH(false, double, true, (const double*)nullptr);
            else SSTEP_GRAM_LAUNCH(false, double, false, (const double*)nullptr);
        }
    }
#undef SSTEP_GRAM_LAUNCH
    return cudaGetLastError();
}

// Fused moments (gram_form FUSED): the s step kernels of an outer iteration left per-block
// partials of a_j = <p_j, p_j> and b_j = <p_j, p_(j+1)>, j = 0 .. s-1 (unweighted: M = m I).
// With A^ = theta (M^-1 A - sigma) self-adjoint in <., .>_M and p_j = T_j(A^) p_0, the
// product rule 2 T_m T_n = T_(m+n) + T_|m-n| gives every moment mu_k = <p_0, T_k(A^) p_0>
// (up to the constant m) from them: mu_0 = a_0, mu_1 = b_0, mu_2m = 2 a_m - mu_0 and
// mu_(2m+1) = 2 b_m - mu_1, which is all the Gram system needs (k < 2s). Blocks sum fixed,
// contiguous ranges of the partials in FP64 (FP32 partials: hi + lo converted exactly); the
// last block to arrive sums the per-block results in block order (deterministic), lays the
// moments out as the moments form's entries and runs the same scaling and solve.
constexpr int FIN_THREADS = 512;
constexpr int FIN_WARPS = FIN_THREADS / 32;

template <int S, typename T>
__global__ void __launch_bounds__(FIN_THREADS) k_moments_finish(const T* __restrict__ part, int nblk, double* part2,
                                                               Ctl* ctl, GramParams gp) {
    if (ctl->done) return;
    constexpr int NV = 2 * S;                   // a_0, b_0, a_1, b_1, ...
    constexpr int NC = sizeof(T) == 8 ? 1 : 2;  // components of one partial (FP32: hi, lo)
    __shared__ double tot[NV];
    __shared__ double ent[2 * S];
    __shared__ double sm[2 * S * S + 4 * S];
    __shared__ bool is_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int R = gridDim.x;
    const int lo = (int)((int64_t)nblk * blockIdx.x / R), hi = (int)((int64_t)nblk * (blockIdx.x + 1) / R);
    for (int v = warp; v < NV; v += FIN_WARPS) {
        // value v = (j, q): step j's partials start at j * 2 NC nblk, component c of q at
        // (2 q + c) nblk (FP64: q nblk)
        const int j = v >> 1, q = v & 1;
        const T* base = part + (size_t)(2 * j + q) * NC * nblk;
        auto val = [&](int b) -> double {
            if constexpr (NC == 2) return f2d_exact(__ldg(base + b)) + f2d_exact(__ldg(base + nblk + b));
            else return __ldg(base + b);
        };
        double acc = 0.0;
        int b = lo + lane;
        // eight values per lane in flight at once, summed in the order of b
        for (; b + 7 * 32 < hi; b += 8 * 32) {
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = val(b + 32 * u);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc += x[u];
        }
        for (; b < hi; b += 32) acc += val(b);
        acc = warp_sum(acc);
        if (lane == 0) part2[(size_t)blockIdx.x * NV + v] = acc;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&ctl->counter, 1u) == (unsigned)R - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int v = warp; v < NV; v += FIN_WARPS) {
        double acc = 0.0;
        for (int r = lane; r < R; r += 32) acc += ((volatile double*)part2)[(size_t)r * NV + v];
        acc = warp_sum(acc);
        if (lane == 0) tot[v] = acc;
    }
    __syncthreads();
    // entries in the layout of the moments form: e <= S: mu_e; S < e < 2S: <p_m, p_m> (e = 2m)
    // or <p_m, p_(m+1)> (e = 2m + 1), from which gram_finish forms mu_e
    for (int e = threadIdx.x; e < 2 * S; e += FIN_THREADS) {
        const double am = tot[2 * (e >> 1)], bm = tot[2 * (e >> 1) + 1];   // a_(e/2), b_(e/2)
        double v;
        if (e <= 1) v = e == 0 ? tot[0] : tot[1];
        else if (e <= S) v = (e % 2 == 0) ? 2.0 * am - tot[0] : 2.0 * bm - tot[1];
        else v = (e % 2 == 0) ? am : bm;
        ent[e] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) ctl->counter = 0u;
    if (warp == 0) gram_finish<S, false, true>(ent, gp, ctl, sm);
}

template <int S>
cudaError_t launch_moments_finish_s(const GramArgs& g, const void* part, int nblk, double* part2, int nfin, Ctl* ctl,
                                    cudaStream_t st) {
    const GramParams gp = gram_params(g);
    if (g.fp32)
        k_moments_finish<S, float><<<nfin, FIN_THREADS, 0, st>>>((const float*)part, nblk, part2, ctl, gp);
    else
        k_moments_finish<S, double><<<nfin, FIN_THREADS, 0, st>>>((const double*)part, nblk, part2, ctl, gp);
    return cudaGetLastError();
}

}  // namespace sstep
