// Measures the arithmetic peaks that bound the FP64 path of the solver on
// this GPU: FP64 and FP32 fused multiply-add throughput and FP64 division
// throughput.  Every SM runs several blocks of independent dependency
// chains; the result is printed as one JSON line.
#include <cstdio>
#include <cuda_runtime.h>

template <class T>
__global__ void fma_chains(T* out, int iters, T b, T c) {
    T x0 = (T)threadIdx.x * (T)1e-6, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * b + c; x1 = x1 * b + c; x2 = x2 * b + c; x3 = x3 * b + c;
        x4 = x4 * b + c; x5 = x5 * b + c; x6 = x6 * b + c; x7 = x7 * b + c;
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1) out[blockIdx.x] = s;   // keeps the chains live
}

__global__ void div_chains(double* out, int iters, double b) {
    double x0 = 1.0 + threadIdx.x * 1e-6, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    for (int i = 0; i < iters; ++i) {
        x0 = b / x0; x1 = b / x1; x2 = b / x2; x3 = b / x3;
    }
    const double s = x0 + x1 + x2 + x3;
    if (s == -1.0) out[blockIdx.x] = s;
}

template <class K>
float time_ms(K k) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k();
    cudaEventRecord(a);
    k();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

int main() {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = sms * 8, threads = 256;
    double* out;
    if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) return 1;
    const int it64 = 4096, it32 = 65536, itd = 1024;
    const float m64 = time_ms([&] { fma_chains<double><<<blocks, threads>>>(out, it64, 1.0000001, 1e-9); });
    const float m32 = time_ms([&] { fma_chains<float><<<blocks, threads>>>((float*)out, it32, 1.0000001f, 1e-9f); });
    const float md = time_ms([&] { div_chains<<<blocks, threads>>>(out, itd, 1.5); });
    const double n = (double)blocks * threads;
    const double f64 = 2.0 * 8 * it64 * n / (m64 * 1e-3) / 1e12;
    const double f32 = 2.0 * 8 * it32 * n / (m32 * 1e-3) / 1e12;
    const double dv = 4.0 * itd * n / (md * 1e-3) / 1e9;
    if (cudaGetLastError() != cudaSuccess) return 2;
    printf("{\"sms\": %d, \"fp64_fma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, \"fp64_div_gops\": %.2f}\n", sms,
           f64, f32, dv);
    cudaFree(out);
    return 0;
}
