// ALU peak probe: FP32 / FP64 fused multiply-add throughput of this GPU,
// measured with independent FMA chains (the roofline denominator of the
// arithmetic-bound pair kernels; not part of the method).
//
// Every thread runs CHAINS independent recurrences x <- x a + b for `iters`
// rounds (a = 1 - 2^-20, b = 2^-20 keep x near 1), so the FMA pipe sees
// CHAINS independent instructions per round per thread; one launch covers
// 8 blocks of 256 threads per SM.  Flops = 2 * CHAINS * iters * threads.
#include <cuda_runtime.h>

#include "ffmin.h"

namespace ffm {

constexpr int PEAK_CHAINS = 8, PEAK_THREADS = 256, PEAK_BLOCKS_PER_SM = 8;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(T *out, int iters, T a, T b) {
    T x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; c++) x[c] = T(1) + T(c) * b;
    for (int k = 0; k < iters; k++) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; c++) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; c++) s += x[c];
    out[(size_t)blockIdx.x * PEAK_THREADS + threadIdx.x] = s;
}

}  // namespace ffm

using namespace ffm;

extern "C" ffmin_status ffmin_alu_peak(int32_t precision, int32_t reps, double *tflops) {
    if (!tflops || reps < 1 || (precision != FFMIN_FP64 && precision != FFMIN_MIXED))
        return FFMIN_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FFMIN_ERR_CUDA;
    const int blocks = sms * PEAK_BLOCKS_PER_SM;
    const bool f64 = precision == FFMIN_FP64;
    const int iters = f64 ? 256 : 8192;
    void *out = nullptr;
    const size_t bytes = (size_t)blocks * PEAK_THREADS * (f64 ? 8 : 4);
    if (cudaMalloc(&out, bytes) != cudaSuccess) return FFMIN_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ffmin_status st = FFMIN_OK;
    float ms = 0.f;
    auto launch = [&]() {
        if (f64)
            k_fma_peak<double><<<blocks, PEAK_THREADS>>>((double *)out, iters, 1.0 - 0x1p-20, 0x1p-20);
        else
            k_fma_peak<float><<<blocks, PEAK_THREADS>>>((float *)out, iters, 1.0f - 0x1p-20f, 0x1p-20f);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = FFMIN_ERR_CUDA;
    } else {
        for (int w = 0; w < 3; w++) launch();  // warm-up (clocks ramp)
        cudaEventRecord(e0);
        for (int r = 0; r < reps; r++) launch();
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess)
            st = FFMIN_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (st != FFMIN_OK) return st;
    const double flops = 2.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_THREADS * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return FFMIN_OK;
}
