// FMA throughput probe: the ALU roofline denominators (FP64 and FP32 CUDA-core
// FMA rate of this GPU), measured with independent FMA chains on every SM.
#include <cuda_runtime.h>

#include "../../include/hlu.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T *out, int iters, T b, T c) {
    T x0 = T(threadIdx.x) * T(1e-7), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, b, c);
        x1 = fma(x1, b, c);
        x2 = fma(x2, b, c);
        x3 = fma(x3, b, c);
        x4 = fma(x4, b, c);
        x5 = fma(x5, b, c);
        x6 = fma(x6, b, c);
        x7 = fma(x7, b, c);
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == T(-12345.678)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

template <class T>
double measure(int iters) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chains<T><<<blocks, threads>>>(out, iters / 8, T(0.999999), T(1e-7));  // warm-up
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0);
        k_fma_chains<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    return flops / (best * 1e-3) / 1e12;
}

}  // namespace

extern "C" int hlu_probe_alu_peaks(double *fp64_tflops, double *fp32_tflops) {
    if (fp64_tflops) *fp64_tflops = measure<double>(1 << 12);
    if (fp32_tflops) *fp32_tflops = measure<float>(1 << 16);
    return (fp64_tflops && *fp64_tflops < 0) || (fp32_tflops && *fp32_tflops < 0) ? HLU_ECUDA : HLU_OK;
}
