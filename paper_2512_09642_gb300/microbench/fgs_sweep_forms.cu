// The library's FGS sweep (fgs_lane of gram_impl.cuh: one accumulator per lane) against the
// earlier two-accumulator form: results compared with == (zero signs may differ), cycles per
// step timed in one warp. Standalone; not part of the library.
// Build and run from the repository root:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 --expt-relaxed-constexpr -Iinclude \
//        -o /tmp/fgs_sweep_forms paper_2512_09642_gb300/microbench/fgs_sweep_forms.cu
//   /tmp/fgs_sweep_forms
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include "../csrc/gram_impl.cuh"

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); exit(1); } } while (0)
namespace sstep { const char* cuda_err_name(cudaError_t e) { return cudaGetErrorString(e); } }
using namespace sstep;

template <int S>
__device__ __forceinline__ double fgs_old(const double (&grow)[S], double chat, unsigned kept, int nu) {
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

template <int S, bool OLD>
__global__ void k_fgs(const double* G, const double* c, unsigned kept, int nu, double* out, long long* cyc) {
    const int lane = threadIdx.x;
    const bool kj = lane < S && ((kept >> lane) & 1u);
    const double inv = kj ? 1.0 / G[lane * S + lane] : 0.0;
    double grow[S];
#pragma unroll
    for (int i = 0; i < S; ++i) grow[i] = lane < S ? G[lane * S + i] * inv : 0.0;
    const double chat = lane < S ? c[lane] * inv : 0.0;
    __syncwarp();
    const long long c0 = clock64();
    const double a = OLD ? fgs_old<S>(grow, chat, kept, nu) : fgs_lane<S>(grow, chat, kept, nu);
    const double as = __shfl_sync(0xffffffffu, a, 0);
    const long long c1 = clock64();
    if (lane < S) out[lane] = a;
    if (lane == 0) cyc[0] = c1 - c0 + (as == 12345.0);
}

template <int S>
void run(unsigned kept, int nu, int seed) {
    double G[S * S], c[S];
    srand(seed);
    for (int i = 0; i < S; ++i)
        for (int k = 0; k <= i; ++k) {
            const double v = (k == i) ? 1.0 + 0.2 * (rand() % 100) / 100.0 : 0.6 * ((rand() % 1000) / 1000.0 - 0.5);
            G[i * S + k] = G[k * S + i] = v;
        }
    for (int i = 0; i < S; ++i) c[i] = (rand() % 1000) / 500.0 - 1.0;
    // dropped columns: zero their rows and columns (as the scaling leaves them)
    for (int i = 0; i < S; ++i)
        if (!((kept >> i) & 1u))
            for (int k = 0; k < S; ++k) G[i * S + k] = G[k * S + i] = 0.0;
    double *dG, *dc, *o1, *o2;
    long long* cy;
    CK(cudaMalloc(&dG, sizeof(G)));
    CK(cudaMalloc(&dc, sizeof(c)));
    CK(cudaMalloc(&o1, 32 * 8));
    CK(cudaMalloc(&o2, 32 * 8));
    CK(cudaMalloc(&cy, 16));
    CK(cudaMemcpy(dG, G, sizeof(G), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dc, c, sizeof(c), cudaMemcpyHostToDevice));
    long long t1 = 0, t2 = 0;
    for (int r = 0; r < 3; ++r) {
        k_fgs<S, true><<<1, 32>>>(dG, dc, kept, nu, o1, cy);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(&t1, cy, 8, cudaMemcpyDeviceToHost));
        k_fgs<S, false><<<1, 32>>>(dG, dc, kept, nu, o2, cy);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(&t2, cy, 8, cudaMemcpyDeviceToHost));
    }
    double h1[S], h2[S];
    CK(cudaMemcpy(h1, o1, sizeof(h1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(h2, o2, sizeof(h2), cudaMemcpyDeviceToHost));
    bool same = true;
    for (int i = 0; i < S; ++i) same &= h1[i] == h2[i];
    printf("S %2d kept %08x nu %2d: two accumulators %6lld cycles (%.1f per step), one accumulator %6lld (%.1f); equal %s\n",
           S, kept, nu, t1, (double)t1 / (nu * S), t2, (double)t2 / (nu * S), same ? "yes" : "NO");
    cudaFree(dG); cudaFree(dc); cudaFree(o1); cudaFree(o2); cudaFree(cy);
}

int main() {
    for (int nu : {1, 25}) {
        run<8>(0xffu, nu, 1);
        run<8>(0xbbu, nu, 2);
        run<12>(0xfffu, nu, 3);
        run<16>(0xffffu, nu, 4);
        run<16>(0xf7efu, nu, 5);
    }
    return 0;
}
