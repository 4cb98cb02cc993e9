// Latency on one warp: dependent DFMA chains with 32 lanes and with one lane active, dependent
// shuffles of a double, and an s = 8 FGS solve in the lane-parallel form (lane j owns row j;
// this copy keeps two accumulators per lane, the library's earlier form: fgs_sweep_forms.cu
// compares it with the current one) against single-thread sequential forms; also the
// globaltimer rate against CUDA events. Standalone; not part of the library.
// Build and run from the repository root:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/warp_fp64_latency paper_2512_09642_gb300/microbench/warp_fp64_latency.cu
//   /tmp/warp_fp64_latency
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); exit(1); } } while (0)

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr int S = 8;

// the library's form: lane j holds row j of G^ (normalised) and c^_j
__device__ __forceinline__ double fgs_lane(const double (&grow)[S], double chat, unsigned kept, int nu) {
    const int lane = threadIdx.x & 31;
    double a = 0.0;
    double u = chat, v = chat;
    for (int sweep = 0; sweep < nu; ++sweep) {
#pragma unroll
        for (int i = 0; i < S; ++i) {
            double ai = __shfl_sync(0xffffffffu, u, i);
            if (!((kept >> i) & 1u)) ai = 0.0;
            if (lane == i) a = ai;
            double w = lane > i ? u : v;
            w = fma(-grow[i], ai, w);
            if (lane > i) u = w;
            else if (lane < i) v = w;
        }
        u = v;
        v = chat;
    }
    return a;
}

// sequential in one thread: a_i = c^_i - sum_{k<i} G^_ik a_k(new) - sum_{k>i} G^_ik a_k(old)
// as running sums: after a_i is final, every other row's sum takes its term.
__device__ __forceinline__ void fgs_seq(const double* G /* S*S normalised rows */, const double* c, unsigned kept,
                                        int nu, double* a_out) {
    double g[S][S], ch[S], a[S], u[S], v[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
        ch[i] = c[i];
#pragma unroll
        for (int k = 0; k < S; ++k) g[i][k] = G[i * S + k];
        u[i] = ch[i];
        v[i] = ch[i];
        a[i] = 0.0;
    }
    for (int sweep = 0; sweep < nu; ++sweep) {
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const double ai = ((kept >> i) & 1u) ? u[i] : 0.0;
            a[i] = ai;
#pragma unroll
            for (int j = 0; j < S; ++j) {
                if (j > i) u[j] = fma(-g[j][i], ai, u[j]);
                else if (j < i) v[j] = fma(-g[j][i], ai, v[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {
            u[j] = v[j];
            v[j] = ch[j];
        }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) a_out[i] = a[i];
}

__global__ void k_lane(const double* G, const double* c, int nu, double* out, long long* cyc, unsigned long long* gt) {
    const int lane = threadIdx.x;
    double grow[S];
#pragma unroll
    for (int i = 0; i < S; ++i) grow[i] = lane < S ? G[lane * S + i] : 0.0;
    const double chat = lane < S ? c[lane] : 0.0;
    __syncwarp();
    const long long c0 = clock64();
    const unsigned long long g0 = gtimer();
    const double a = fgs_lane(grow, chat, 0xffu, nu);
    const double as = __shfl_sync(0xffffffffu, a, 0);
    const long long c1 = clock64();
    const unsigned long long g1 = gtimer();
    if (lane < S) out[lane] = a;
    if (lane == 0) { cyc[0] = c1 - c0 + (as == 12345.0); gt[0] = g1 - g0; }
}

template <bool ONE>
__global__ void k_seq(const double* G, const double* c, int nu, double* out, long long* cyc, unsigned long long* gt) {
    const int lane = threadIdx.x;
    __shared__ double sG[S * S], sc[S];
    for (int i = lane; i < S * S; i += 32) sG[i] = G[i];
    if (lane < S) sc[lane] = c[lane];
    __syncwarp();
    double a[S];
    const long long c0 = clock64();
    const unsigned long long g0 = gtimer();
    if (!ONE || lane == 0) fgs_seq(sG, sc, 0xffu, nu, a);
    __syncwarp();
    const long long c1 = clock64();
    const unsigned long long g1 = gtimer();
    if (lane == 0) {
        for (int i = 0; i < S; ++i) out[i] = a[i];
        cyc[0] = c1 - c0;
        gt[0] = g1 - g0;
    }
}

__global__ void k_dfma_chain(const double* in, int n, double* out, long long* cyc) {
    double x = in[threadIdx.x], m = in[32 + threadIdx.x], y = in[64 + threadIdx.x];
    const long long c0 = clock64();
    for (int i = 0; i < n; ++i) x = fma(x, m, y);
    const long long c1 = clock64();
    out[threadIdx.x] = x;
    if (threadIdx.x == 0) cyc[0] = c1 - c0;
}

__global__ void k_dfma_chain_one(const double* in, int n, double* out, long long* cyc) {
    double x = in[threadIdx.x], m = in[32 + threadIdx.x], y = in[64 + threadIdx.x];
    const long long c0 = clock64();
    if (threadIdx.x == 0)
        for (int i = 0; i < n; ++i) x = fma(x, m, y);
    __syncwarp();
    const long long c1 = clock64();
    out[threadIdx.x] = x;
    if (threadIdx.x == 0) cyc[0] = c1 - c0;
}

__global__ void k_shfl_chain(const double* in, int n, double* out, long long* cyc) {
    double x = in[threadIdx.x];
    const long long c0 = clock64();
    for (int i = 0; i < n; ++i) x = __shfl_sync(0xffffffffu, x, (i + 1) & 31);
    const long long c1 = clock64();
    out[threadIdx.x] = x;
    if (threadIdx.x == 0) cyc[0] = c1 - c0;
}

__global__ void k_spin(int n, double* out, unsigned long long* gt, long long* cyc) {
    const long long c0 = clock64();
    const unsigned long long g0 = gtimer();
    float x = (float)threadIdx.x;
    for (int i = 0; i < n; ++i) x = fmaf(x, 0.999f, 0.5f);
    const long long c1 = clock64();
    const unsigned long long g1 = gtimer();
    out[threadIdx.x] = x;
    if (threadIdx.x == 0) { gt[0] = g1 - g0; cyc[0] = c1 - c0; }
}

int main() {
    // a well-conditioned SPD G (diagonally dominant), normalised rows: G^_ik = G_ik / G_ii
    double G[S * S], c[S], Gn[S * S], cn[S];
    srand(3);
    for (int i = 0; i < S; ++i)
        for (int k = 0; k <= i; ++k) {
            const double v = (k == i) ? 2.0 + i * 0.1 : 0.3 * ((rand() % 1000) / 1000.0 - 0.5);
            G[i * S + k] = G[k * S + i] = v;
        }
    for (int i = 0; i < S; ++i) c[i] = 1.0 + 0.1 * i;
    for (int i = 0; i < S; ++i) {
        for (int k = 0; k < S; ++k) Gn[i * S + k] = G[i * S + k] / G[i * S + i];
        cn[i] = c[i] / G[i * S + i];
    }
    double *dG, *dc, *dout, *din;
    long long* dcyc;
    unsigned long long* dgt;
    CK(cudaMalloc(&dG, sizeof(Gn)));
    CK(cudaMalloc(&dc, sizeof(cn)));
    CK(cudaMalloc(&dout, 64 * sizeof(double)));
    CK(cudaMalloc(&din, 96 * sizeof(double)));
    CK(cudaMalloc(&dcyc, 8 * sizeof(long long)));
    CK(cudaMalloc(&dgt, 8 * sizeof(unsigned long long)));
    CK(cudaMemcpy(dG, Gn, sizeof(Gn), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dc, cn, sizeof(cn), cudaMemcpyHostToDevice));
    double hin[96];
    for (int i = 0; i < 96; ++i) hin[i] = i < 32 ? 1.0 : (i < 64 ? 0.999 : 0.001);
    CK(cudaMemcpy(din, hin, sizeof(hin), cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    long long cyc;
    unsigned long long gt;
    float ms;
    // globaltimer rate against events and clock64
    for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(e0));
        k_spin<<<1, 32>>>(20000000, dout, dgt, dcyc);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        CK(cudaMemcpy(&cyc, dcyc, 8, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&gt, dgt, 8, cudaMemcpyDeviceToHost));
        printf("spin: events %.3f ms, globaltimer %.3f ms, clock64 %lld (%.0f MHz by events)\n", ms, gt / 1e6, cyc,
               cyc / (ms * 1e3));
    }
    const int n = 4096;
    for (int rep = 0; rep < 2; ++rep) {
        k_dfma_chain<<<1, 32>>>(din, n, dout, dcyc);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(&cyc, dcyc, 8, cudaMemcpyDeviceToHost));
        printf("dependent DFMA, 32 lanes: %.1f cycles each\n", (double)cyc / n);
        k_dfma_chain_one<<<1, 32>>>(din, n, dout, dcyc);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(&cyc, dcyc, 8, cudaMemcpyDeviceToHost));
        printf("dependent DFMA, 1 lane: %.1f cycles each\n", (double)cyc / n);
        k_shfl_chain<<<1, 32>>>(din, n, dout, dcyc);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(&cyc, dcyc, 8, cudaMemcpyDeviceToHost));
        printf("dependent SHFL of a double: %.1f cycles each\n", (double)cyc / n);
    }
    double ref[S], hout[S];
    for (int nu : {1, 25}) {
        for (int rep = 0; rep < 2; ++rep) {
            k_lane<<<1, 32>>>(dG, dc, nu, dout, dcyc, dgt);
            CK(cudaDeviceSynchronize());
            CK(cudaMemcpy(&cyc, dcyc, 8, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(&gt, dgt, 8, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(ref, dout, sizeof(ref), cudaMemcpyDeviceToHost));
            printf("nu %2d lane-parallel: %lld cycles (%.1f per row step), %.2f us globaltimer\n", nu, cyc,
                   (double)cyc / (nu * S), gt / 1e3);
            k_seq<false><<<1, 32>>>(dG, dc, nu, dout, dcyc, dgt);
            CK(cudaDeviceSynchronize());
            CK(cudaMemcpy(&cyc, dcyc, 8, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(&gt, dgt, 8, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(hout, dout, sizeof(hout), cudaMemcpyDeviceToHost));
            bool same = true;
            for (int i = 0; i < S; ++i) same &= hout[i] == ref[i];
            printf("nu %2d sequential, 32 lanes: %lld cycles (%.1f per row step), %.2f us, bitwise %s\n", nu, cyc,
                   (double)cyc / (nu * S), gt / 1e3, same ? "equal" : "DIFFERENT");
            k_seq<true><<<1, 32>>>(dG, dc, nu, dout, dcyc, dgt);
            CK(cudaDeviceSynchronize());
            CK(cudaMemcpy(&cyc, dcyc, 8, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(&gt, dgt, 8, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(hout, dout, sizeof(hout), cudaMemcpyDeviceToHost));
            same = true;
            for (int i = 0; i < S; ++i) same &= hout[i] == ref[i];
            printf("nu %2d sequential, lane 0: %lld cycles (%.1f per row step), %.2f us, bitwise %s\n", nu, cyc,
                   (double)cyc / (nu * S), gt / 1e3, same ? "equal" : "DIFFERENT");
        }
    }
    return 0;
}
