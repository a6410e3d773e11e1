// Training of the per-atom preconditioner network on the GPU: mean squared
// error between z(f) and the recorded target t over a data set, plain
// backpropagation through the two layers, and Adam (Kingma & Ba 2015).
// Hand-written kernels, FP32 arithmetic; weights are handed to inference as
// FP16.  Minibatches are drawn with the SplitMix64 counter stream.
//
// Loss per sample: (z - t)^2; minibatch loss = mean.  Gradients:
//   dz = 2 (z - t) / B,  dw2_k = dz h_k,  db2 = dz,
//   dh_k = dz w2_k [a_k > 0],  dW1_ki = dh_k f_i,  db1_k = dh_k.
// Per-block partial gradients are summed in block order by a second kernel,
// so a step is deterministic.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "ffmin.h"
#include "mlp.cuh"

namespace ffm {

constexpr int MT = 128;          // threads per training block
constexpr int MLP_BLOCKS = 256;  // blocks per minibatch gradient

__device__ __forceinline__ uint64_t mix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// partial gradient of one block over its share of the minibatch; samples of
// the minibatch are index (base + k) of the SplitMix64 stream when sample
// != 0, else rows [0, batch) of the data in order
__global__ void __launch_bounds__(MT) k_mlp_grad(const float *feat, const float *target, int64_t n,
                                                 const float *w32, int batch, uint64_t seed, uint64_t base,
                                                 int sample, float *part, float *loss_part) {
    __shared__ float w[MLP_NW];
    __shared__ float acc[MLP_NW];
    __shared__ float lsum[MT];
    for (int k = threadIdx.x; k < MLP_NW; k += MT) { w[k] = w32[k]; acc[k] = 0.f; }
    __syncthreads();
    float g[MLP_NW];  // per-thread gradient accumulator (registers / local)
    for (int k = 0; k < MLP_NW; k++) g[k] = 0.f;
    float loss = 0.f;
    const float inv_b = 1.0f / (float)batch;
    for (int s = blockIdx.x * MT + threadIdx.x; s < batch; s += gridDim.x * MT) {
        int64_t row = sample ? (int64_t)__umul64hi(mix64(seed, base + s), (uint64_t)n) : s;
        float f[MLP_IN], h[MLP_H];
        for (int i = 0; i < MLP_IN; i++) f[i] = feat[row * MLP_IN + i];
        const float z = mlp_forward(w, f, h);
        const float r = z - target[row];
        loss += r * r;
        const float dz = 2.f * r * inv_b;
        g[MLP_B2] += dz;
        for (int k = 0; k < MLP_H; k++) {
            g[MLP_W2 + k] += dz * h[k];
            const float dh = h[k] > 0.f ? dz * w[MLP_W2 + k] : 0.f;
            g[MLP_B1 + k] += dh;
            for (int i = 0; i < MLP_IN; i++) g[MLP_W1 + k * MLP_IN + i] += dh * f[i];
        }
    }
    // block sum in thread order, one parameter at a time
    for (int k = 0; k < MLP_NW; k++) {
        lsum[threadIdx.x] = g[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int j = 0; j < MT; j++) t += lsum[j];
            acc[k] = t;
        }
        __syncthreads();
    }
    lsum[threadIdx.x] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int j = 0; j < MT; j++) t += lsum[j];
        loss_part[blockIdx.x] = t;
    }
    for (int k = threadIdx.x; k < MLP_NW; k += MT) part[(int64_t)blockIdx.x * MLP_NW + k] = acc[k];
}

// sum of the block partials in block order; then one Adam step on the FP32
// master weights (when lr > 0) and the FP16 copy for inference
__global__ void k_mlp_adam(const float *part, const float *loss_part, int nblocks, int batch, float *w32,
                           float *adam, int step, float lr, float *grad_out, float *loss_out,
                           uint16_t *w16) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int k = threadIdx.x; k < MLP_NW; k += blockDim.x) {
        float gk = 0.f;
        for (int b = 0; b < nblocks; b++) gk += part[(int64_t)b * MLP_NW + k];
        if (grad_out) grad_out[k] = gk;
        if (lr > 0.f) {
            float m = adam[k] = b1 * adam[k] + (1.f - b1) * gk;
            float v = adam[MLP_NW + k] = b2 * adam[MLP_NW + k] + (1.f - b2) * gk * gk;
            const float mh = m / (1.f - powf(b1, (float)step));
            const float vh = v / (1.f - powf(b2, (float)step));
            w32[k] -= lr * mh / (sqrtf(vh) + eps);
        }
        if (w16) {
            __half hv = __float2half_rn(w32[k]);
            w16[k] = *reinterpret_cast<uint16_t *>(&hv);
        }
    }
    if (threadIdx.x == 0 && loss_out) {
        float t = 0.f;
        for (int b = 0; b < nblocks; b++) t += loss_part[b];
        *loss_out = t / (float)batch;
    }
}

}  // namespace ffm

using namespace ffm;

extern "C" ffmin_status ffmin_mlp_train(const float *feat_dev, const float *target_dev, int64_t n_samples,
                                        int32_t steps, int32_t batch, float lr, uint64_t seed, float *w32_dev,
                                        float *adam_dev, float *work_dev, float *loss_host, uint16_t *w16_dev,
                                        void *cuda_stream) {
    if (!feat_dev || !target_dev || n_samples < 1 || steps < 0 || batch < 1 || !w32_dev || !work_dev)
        return FFMIN_ERR_INVALID_ARG;
    if (steps > 0 && (!adam_dev || !(lr > 0.f))) return FFMIN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float *part = work_dev;                                    // [MLP_BLOCKS][MLP_NW]
    float *loss_part = work_dev + (size_t)MLP_BLOCKS * MLP_NW; // [MLP_BLOCKS]
    float *loss_dev = loss_part + MLP_BLOCKS;                  // [1]
    float *grad_dev = loss_dev + 1;                            // [MLP_NW]
    const int nsteps = steps > 0 ? steps : 1;
    for (int t = 0; t < nsteps; t++) {
        const int sample = steps > 0 ? 1 : 0;
        const int b = steps > 0 ? batch : (int)std::min<int64_t>(batch, n_samples);
        k_mlp_grad<<<MLP_BLOCKS, MT, 0, s>>>(feat_dev, target_dev, n_samples, w32_dev, b, seed,
                                             (uint64_t)t * (uint64_t)batch, sample, part, loss_part);
        k_mlp_adam<<<1, 512, 0, s>>>(part, loss_part, MLP_BLOCKS, b, w32_dev, adam_dev, t + 1,
                                     steps > 0 ? lr : 0.f, grad_dev, loss_dev, w16_dev);
        if (loss_host) {
            if (cudaMemcpyAsync(loss_host + t, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return FFMIN_ERR_CUDA;
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return FFMIN_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? FFMIN_OK : FFMIN_ERR_CUDA;
}

extern "C" int64_t ffmin_mlp_work_floats(void) {
    return (int64_t)MLP_BLOCKS * MLP_NW + MLP_BLOCKS + 1 + MLP_NW;
}
