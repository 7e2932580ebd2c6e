// mlp.cuh -- the learned proposal: a 3-layer MLP (n_in -> 64 -> 64 -> 3,
// SiLU) with BF16 weights and FP32 accumulation, predicting a system's first
// step size, spectral-radius bound and integration cost.
#pragma once
#include <cstdint>

namespace bode {

constexpr int kMlpHidden = 64;
constexpr int kMlpMaxIn = 33;  // up to 32 state components + 1 parameter
constexpr int kMlpOut = 3;     // log h0, log sigma, log cost (right-hand-side evaluations)

// Parameter layout (one flat array): W1 [64][n_in], b1 [64], W2 [64][64],
// b2 [64], W3 [3][64], b3 [3].
__host__ __device__ constexpr int mlp_w1(int) { return 0; }
__host__ __device__ constexpr int mlp_b1(int n_in) { return kMlpHidden * n_in; }
__host__ __device__ constexpr int mlp_w2(int n_in) { return mlp_b1(n_in) + kMlpHidden; }
__host__ __device__ constexpr int mlp_b2(int n_in) { return mlp_w2(n_in) + kMlpHidden * kMlpHidden; }
__host__ __device__ constexpr int mlp_w3(int n_in) { return mlp_b2(n_in) + kMlpHidden; }
__host__ __device__ constexpr int mlp_b3(int n_in) { return mlp_w3(n_in) + kMlpOut * kMlpHidden; }
__host__ __device__ constexpr int mlp_nparams(int n_in) { return mlp_b3(n_in) + kMlpOut; }

// Feature normalisation and the input box the network was trained on.
struct MlpNorm {
    float x_mean[kMlpMaxIn], x_scale[kMlpMaxIn], x_min[kMlpMaxIn], x_max[kMlpMaxIn];
    float y_mean[kMlpOut], y_scale[kMlpOut];
};

// SiLU and its derivative.
__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

}  // namespace bode
