// FP64 issue-rate microbenchmark (the denominator of the FP64 stencils' roofline fractions): CH
// independent FMA/ADD/MUL chains per thread at full occupancy, operands loaded from memory
// (random non-zero or zero), CUDA-event timing. Standalone; not part of the library.
// Build and run from the repository root:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/fp64_rate paper_2512_09642_gb300/microbench/fp64_rate.cu
//   /tmp/fp64_rate
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); exit(1); } } while (0)

template <int CH, int OP>
__global__ void __launch_bounds__(256) k_fp64(const double* __restrict__ in, double* __restrict__ out, int iters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double a[CH];
    const double m = in[(t * 7) & 4095];
    const double c = in[(t * 13 + 5) & 4095];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = in[(t + k * 97) & 4095];
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            if (OP == 0) a[k] = fma(a[k], m, c);
            else if (OP == 1) a[k] = a[k] + c;
            else a[k] = a[k] * m;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) s += a[k];
    if (s == 12345.678) out[t] = s;   // keeps the chains live, never taken
}

// OP 3: a + c written as fma(a, one, c) with one = 1.0 from memory (bitwise the same sum)
// OP 4: the 7-point step's mix, 5 adds + 2 FMAs per chain element; OP 5: the same with the
// adds as fma(., one, .)
template <int CH, int OP>
__global__ void __launch_bounds__(256) k_fp64b(const double* __restrict__ in, const double* __restrict__ onep,
                                                double* __restrict__ out, int iters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double a[CH];
    const double one = onep[0];
    const double m = in[(t * 7) & 4095];
    const double c = in[(t * 13 + 5) & 4095];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = in[(t + k * 97) & 4095];
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            if (OP == 3) a[k] = fma(a[k], one, c);
            else if (OP == 4) {
                double v = a[k] + c; v = v + m; v = v + c; v = v + m; v = v + c;
                v = fma(v, m, c); a[k] = fma(v, m, -c);
            } else {
                double v = fma(a[k], one, c); v = fma(v, one, m); v = fma(v, one, c); v = fma(v, one, m);
                v = fma(v, one, c); v = fma(v, m, c); a[k] = fma(v, m, -c);
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CH; ++k) s += a[k];
    if (s == 12345.678) out[t] = s;
}

template <int CH>
__global__ void __launch_bounds__(256) k_fp32(const float* __restrict__ in, float* __restrict__ out, int iters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float a[CH];
    const float m = in[(t * 7) & 4095];
    const float c = in[(t * 13 + 5) & 4095];
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = in[(t + k * 97) & 4095];
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CH; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CH; ++k) s += a[k];
    if (s == 12345.678f) out[t] = s;
}

template <typename K>
float timeit(K launch, int reps) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int w = 0; w < 3; ++w) launch();
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0));
    for (int r = 0; r < reps; ++r) launch();
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    return ms / reps;
}

int main() {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    std::vector<double> h(4096), z(4096, 0.0);
    uint64_t st = 12345;
    for (auto& v : h) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        v = 0.999 + 0.001 * ((st >> 11) * (1.0 / 9007199254740992.0));   // in [0.999, 1)
    }
    std::vector<float> hf(h.begin(), h.end());
    double *din, *dz, *dout;
    float *fin, *fout;
    CK(cudaMalloc(&din, 4096 * 8));
    CK(cudaMalloc(&dz, 4096 * 8));
    CK(cudaMalloc(&fin, 4096 * 4));
    const int blocks = sms * 8, threads = 256;   // 2048 threads per SM
    CK(cudaMalloc(&dout, sizeof(double) * blocks * threads));
    CK(cudaMalloc(&fout, sizeof(float) * blocks * threads));
    CK(cudaMemcpy(din, h.data(), 4096 * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dz, z.data(), 4096 * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(fin, hf.data(), 4096 * 4, cudaMemcpyHostToDevice));
    const double nthr = (double)blocks * threads;
    const int iters = 4096;
    printf("sms %d blocks %d threads %d iters %d\n", sms, blocks, threads, iters);
    auto rep = [&](const char* name, int ch, float ms) {
        const double ops = nthr * iters * ch;
        printf("%-28s chains %2d: %.3f ms  %.1f G lane-ops/s\n", name, ch, ms, ops / (ms * 1e-3) / 1e9);
    };
#define RUN64(CH, OP, SRC, NAME) rep(NAME, CH, timeit([&] { k_fp64<CH, OP><<<blocks, threads>>>(SRC, dout, iters); }, 5))
    RUN64(4, 0, din, "fp64 fma random");
    RUN64(8, 0, din, "fp64 fma random");
    RUN64(16, 0, din, "fp64 fma random");
    RUN64(8, 1, din, "fp64 add random");
    RUN64(8, 2, din, "fp64 mul random");
    RUN64(8, 0, dz, "fp64 fma zero operands");
    RUN64(8, 1, dz, "fp64 add zero operands");
    RUN64(16, 0, din, "fp64 fma random (again)");
    {
        double* d1;
        const double onev = 1.0;
        CK(cudaMalloc(&d1, 8));
        CK(cudaMemcpy(d1, &onev, 8, cudaMemcpyHostToDevice));
        rep("fp64 add as fma(a, one, c)", 8, timeit([&] { k_fp64b<8, 3><<<blocks, threads>>>(din, d1, dout, iters); }, 5));
        float ms = timeit([&] { k_fp64b<8, 4><<<blocks, threads>>>(din, d1, dout, iters / 4); }, 5);
        printf("%-28s chains  8: %.3f ms  %.1f G lane-ops/s\n", "5 add + 2 fma (dependent)", ms, nthr * (iters / 4) * 8 * 7 / (ms * 1e-3) / 1e9);
        ms = timeit([&] { k_fp64b<8, 5><<<blocks, threads>>>(din, d1, dout, iters / 4); }, 5);
        printf("%-28s chains  8: %.3f ms  %.1f G lane-ops/s\n", "7 fma (adds via one)", ms, nthr * (iters / 4) * 8 * 7 / (ms * 1e-3) / 1e9);
    }
    rep("fp32 fma random", 8, timeit([&] { k_fp32<8><<<blocks, threads>>>(fin, fout, iters * 8); }, 5) / 8);
    // the same with fewer resident threads: 1 block of 256 per SM, 4 blocks per SM
    {
        const int b1 = sms, b4 = sms * 4;
        float ms = timeit([&] { k_fp64<8, 0><<<b1, threads>>>(din, dout, iters); }, 5);
        printf("%-28s chains  8: %.3f ms  %.1f G lane-ops/s\n", "fp64 fma 256 thr/SM", ms, (double)b1 * threads * iters * 8 / (ms * 1e-3) / 1e9);
        ms = timeit([&] { k_fp64<8, 0><<<b4, threads>>>(din, dout, iters); }, 5);
        printf("%-28s chains  8: %.3f ms  %.1f G lane-ops/s\n", "fp64 fma 1024 thr/SM", ms, (double)b4 * threads * iters * 8 / (ms * 1e-3) / 1e9);
    }
    // a long loop (about 2 s) for the clock sampler
    {
        float ms = timeit([&] { k_fp64<8, 0><<<blocks, threads>>>(din, dout, iters * 16); }, 10);
        printf("%-28s chains  8: %.3f ms  %.1f G lane-ops/s (long run)\n", "fp64 fma random", ms, nthr * iters * 16 * 8 / (ms * 1e-3) / 1e9);
    }
    return 0;
}
