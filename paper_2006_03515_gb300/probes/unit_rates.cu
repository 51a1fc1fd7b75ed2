// Throughput of the special-function unit (ex2.approx, rsqrt.approx) and of FP64 FMA on the
// current GPU: independent dependency chains per thread, 4 blocks of 256 threads per SM, timed
// with CUDA events. Prints results per SM per clock at the device's maximum SM clock; these
// rates are the peaks of the pair-kernel and FP64 rooflines.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o unit_rates unit_rates.cu && ./unit_rates
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqa(float x) {
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <int KIND>
__global__ void sfu(float* out, int iters) {
    float a[8];
    for (int k = 0; k < 8; ++k) a[k] = 0.5f + 1e-3f * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = KIND == 0 ? ex2a(a[k]) : rsqa(a[k]);
    }
    float s = 0.f;
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// one pair of the near-field kernel's special functions: two ex2 and one rsqrt, independent
__global__ void sfu_mix(float* out, int iters) {
    float a[4], b[4], c[4];
    for (int k = 0; k < 4; ++k) a[k] = b[k] = c[k] = 0.5f + 1e-3f * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = ex2a(a[k]);
            b[k] = ex2a(b[k]);
            c[k] = rsqa(c[k]);
        }
    }
    float s = 0.f;
    for (int k = 0; k < 4; ++k) s += a[k] + b[k] + c[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void dfma(double* out, int iters) {
    double a[16];
    for (int k = 0; k < 16; ++k) a[k] = 1e-3 * (threadIdx.x + k);
    const double m = 0.999999, c = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = fma(a[k], m, c);
    }
    double s = 0;
    for (int k = 0; k < 16; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
    int dev = 0, sms = 0, clk = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);   // kHz
    const int blocks = sms * 4, threads = 256;
    float* f = nullptr;
    double* d = nullptr;
    if (cudaMalloc(&f, (size_t)blocks * threads * 4) != cudaSuccess ||
        cudaMalloc(&d, (size_t)blocks * threads * 8) != cudaSuccess) {
        printf("allocation failed\n");
        return 1;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const char* names[4] = {"ex2.approx.f32", "rsqrt.approx.f32", "FP64 FMA", "2 ex2 + 1 rsqrt"};
    for (int rep = 0; rep < 2; ++rep) {
        for (int kind = 0; kind < 4; ++kind) {
            const int it = kind == 2 ? 2048 : 8192;
            cudaEventRecord(e0);
            if (kind == 0) sfu<0><<<blocks, threads>>>(f, it);
            else if (kind == 1) sfu<1><<<blocks, threads>>>(f, it);
            else if (kind == 2) dfma<<<blocks, threads>>>(d, it);
            else sfu_mix<<<blocks, threads>>>(f, it);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double ops = (kind == 2 ? 16.0 : (kind == 3 ? 4.0 : 8.0)) * it * blocks * threads;
            const double rate = ops / (ms * 1e-3);
            if (rep)
                printf("%-18s %10.1f G/s  %6.2f per SM per clock at %.0f MHz%s\n", names[kind], rate / 1e9,
                       rate / sms / (clk * 1e3), clk / 1e3,
                       kind == 2 ? "  (x2 flop per FMA)" : (kind == 3 ? "  (triples)" : ""));
        }
    }
    cudaError_t e = cudaGetLastError();
    printf("%s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
