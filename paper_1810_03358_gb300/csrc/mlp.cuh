// The per-atom preconditioner network: features f (5) -> h = relu(W1 f + b1)
// (64) -> z = w2 . h + b2; the L-BFGS initial Hessian is scaled per atom by
// d = exp(clamp(z, -3, 3)) (an extension of Algorithm 3, not in the paper).
// Weights are stored as 449 values: W1 [64][5], b1 [64], w2 [64], b2.
#pragma once

#include <cuda_fp16.h>

namespace ffm {

constexpr int MLP_IN = 5, MLP_H = 64;
constexpr int MLP_NW = MLP_H * MLP_IN + MLP_H + MLP_H + 1;  // 449
constexpr int MLP_W1 = 0, MLP_B1 = MLP_H * MLP_IN, MLP_W2 = MLP_B1 + MLP_H, MLP_B2 = MLP_W2 + MLP_H;

// features of an atom: charge, sigma, epsilon, (neighbours within 8 A)/64,
// log(1 + |grad_i|)
__device__ __forceinline__ void mlp_features(float q, float sigma, float eps, int n8, float gnorm,
                                             float *f) {
    f[0] = q;
    f[1] = sigma;
    f[2] = eps;
    f[3] = (float)n8 * (1.0f / 64.0f);
    f[4] = log1pf(gnorm);
}

// forward pass with FP32 accumulation; w in FP32 (converted once from the
// FP16 weights into shared memory by the caller); returns z, fills h (may be
// nullptr when not needed)
__device__ __forceinline__ float mlp_forward(const float *w, const float *f, float *h) {
    float z = w[MLP_B2];
#pragma unroll 8
    for (int k = 0; k < MLP_H; k++) {
        float a = w[MLP_B1 + k];
#pragma unroll
        for (int i = 0; i < MLP_IN; i++) a = fmaf(w[MLP_W1 + k * MLP_IN + i], f[i], a);
        a = fmaxf(a, 0.0f);
        if (h) h[k] = a;
        z = fmaf(w[MLP_W2 + k], a, z);
    }
    return z;
}

__device__ __forceinline__ float mlp_scale(const float *w, const float *f) {
    const float z = mlp_forward(w, f, nullptr);
    return expf(fminf(fmaxf(z, -3.0f), 3.0f));
}

}  // namespace ffm
