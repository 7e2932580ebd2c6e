// mlp.cu -- training and inference kernels of the learned proposal.
//
// The network maps the features of a system's initial state (log |y_k| per
// component and the raw parameter, normalised) to (log h0, log sigma,
// log cost): the first accepted step size and the power-method
// spectral-radius bound the FP64 solver found for it, and the number of
// right-hand-side evaluations the whole integration took (the key that
// orders a batch longest-first).  Weights are kept as FP32 masters and used in
// BF16 (round-to-nearest-even) for every forward pass; all sums are FP32.
//
// Losses: squared error on log h0 and log cost; pinball (quantile tau = 0.9)
// on log sigma, so the network leans to over-estimating sigma -- the stable
// side for RKC.
//
// Kernels:
//   k_mlp_grad    one block = 64 threads = one thread per hidden neuron,
//                 samples streamed through shared memory; forward, loss,
//                 backward and the per-block weight-gradient sums in
//                 registers, then one atomicAdd per parameter per block.
//   k_adam        one thread per parameter (bias-corrected Adam), writes the
//                 FP32 master and its BF16 copy, clears the gradient.
//   k_mlp_apply   one thread per sample, weights in shared memory.
//   k_pack        the inference copy the integration kernels evaluate
//                 in-kernel (mlp_warp.cuh): B fragments of mma.m16n8k16 in
//                 fragment-major order, biases, normalisation and the box.
//
// A NaN target is no target (no loss, no gradient, not in the statistics),
// so records with a spectral-radius target only train beside full ones.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "batchode.h"
#include "mlp.cuh"
#include "mlp_warp.cuh"

namespace bode {
int set_last_error(int code, const char* msg);
void clear_last_error();
}  // namespace bode

using namespace bode;

namespace {

constexpr int kH = kMlpHidden;
constexpr float kTau = 0.9f;  // pinball quantile of the log-sigma loss

struct Mlp {
    int n_in = 0;
    int nparams = 0;
    int dev = 0;
    float* master = nullptr;
    __nv_bfloat16* w16 = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;  // device scalar
    MlpNorm norm;
    bool has_norm = false;
    int64_t step = 0;
    MlpPacked* packed = nullptr;  // inference copy for the integration kernels
};

constexpr float kBoxMargin = 0.05f;  // in-kernel proposals: the training box widened by 5 % of its width

std::mutex g_mu;
std::map<int32_t, Mlp> g_mlps;
int32_t g_next = 1;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

int cuda_fail(cudaError_t e, const char* what) { return fail(ODE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e)); }

// ---------------------------------------------------------------- kernels

// Weights (BF16 -> float) into shared memory.
__device__ void load_weights(const __nv_bfloat16* w16, float* sw, int np) {
    for (int k = threadIdx.x; k < np; k += blockDim.x) sw[k] = __bfloat162float(w16[k]);
    __syncthreads();
}

__device__ __forceinline__ float loss_grad(int o, float p, float t, float* loss) {
    if (isnan(t)) return 0.0f;  // no target
    if (o != 1) {  // squared error: log h0, log cost
        const float r = p - t;
        *loss += r * r;
        return 2.0f * r;
    }
    const float r = t - p;  // pinball: tau r for r > 0, (tau - 1) r otherwise
    *loss += r > 0.0f ? kTau * r : (kTau - 1.0f) * r;
    return r > 0.0f ? -kTau : (1.0f - kTau);
}

// Gradient of the summed loss over samples [0, n) (rows of X / Y, optionally
// through a permutation), accumulated into grad; the summed loss into *loss.
__global__ void __launch_bounds__(kH) k_mlp_grad(const __nv_bfloat16* __restrict__ w16, const MlpNorm norm, int n_in,
                                                  const float* __restrict__ X, const float* __restrict__ Y,
                                                  const int32_t* __restrict__ perm, int64_t n, int per_block,
                                                  float* __restrict__ grad, float* __restrict__ loss) {
    extern __shared__ float sm[];
    const int np = mlp_nparams(n_in);
    float* sw = sm;                 // weights
    float* sx = sw + np;            // normalised input of the current sample
    float* sa1 = sx + kMlpMaxIn;    // layer-1 activations
    float* sa2 = sa1 + kH;          // layer-2 activations
    float* sd2 = sa2 + kH;          // layer-2 deltas
    float* sg3 = sd2 + kH;          // output gradients (kMlpOut)
    load_weights(w16, sw, np);
    const int j = threadIdx.x;
    const float* W1 = sw + mlp_w1(n_in);
    const float* B1 = sw + mlp_b1(n_in);
    const float* W2 = sw + mlp_w2(n_in);
    const float* B2 = sw + mlp_b2(n_in);
    const float* W3 = sw + mlp_w3(n_in);
    const float* B3 = sw + mlp_b3(n_in);
    float gW1[kMlpMaxIn], gW2[kH], gB1 = 0.f, gB2 = 0.f, gW3[kMlpOut], gB3[kMlpOut];
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) gW3[o] = gB3[o] = 0.f;
#pragma unroll
    for (int k = 0; k < kMlpMaxIn; ++k) gW1[k] = 0.f;
#pragma unroll
    for (int k = 0; k < kH; ++k) gW2[k] = 0.f;
    float lsum = 0.f;
    const int64_t s0 = (int64_t)blockIdx.x * per_block;
    const int64_t s1 = min(n, s0 + per_block);
    for (int64_t q = s0; q < s1; ++q) {
        const int64_t r = perm ? perm[q] : q;
        if (j < n_in) sx[j] = (X[r * n_in + j] - norm.x_mean[j]) / norm.x_scale[j];
        __syncthreads();
        float z1 = B1[j];
        for (int k = 0; k < n_in; ++k) z1 += W1[j * n_in + k] * sx[k];
        sa1[j] = silu(z1);
        __syncthreads();
        float z2 = B2[j];
#pragma unroll 8
        for (int k = 0; k < kH; ++k) z2 += W2[j * kH + k] * sa1[k];
        sa2[j] = silu(z2);
        __syncthreads();
        if (j < kMlpOut) {
            float z3 = B3[j];
            for (int k = 0; k < kH; ++k) z3 += W3[j * kH + k] * sa2[k];
            const float t = (Y[r * kMlpOut + j] - norm.y_mean[j]) / norm.y_scale[j];
            sg3[j] = loss_grad(j, z3, t, &lsum);
        }
        __syncthreads();
        float back3 = 0.f;
#pragma unroll
        for (int o = 0; o < kMlpOut; ++o) {
            const float g = sg3[o];
            gW3[o] += g * sa2[j];
            gB3[o] += g;  // summed by thread 0 only
            back3 += W3[o * kH + j] * g;
        }
        const float d2 = back3 * silu_grad(z2);
        sd2[j] = d2;
        gB2 += d2;
#pragma unroll 8
        for (int k = 0; k < kH; ++k) gW2[k] += d2 * sa1[k];
        __syncthreads();
        float back = 0.f;
#pragma unroll 8
        for (int k = 0; k < kH; ++k) back += W2[k * kH + j] * sd2[k];
        const float d1 = back * silu_grad(z1);
        gB1 += d1;
        for (int k = 0; k < n_in; ++k) gW1[k] += d1 * sx[k];
        __syncthreads();
    }
    if (s0 >= s1) return;
    for (int k = 0; k < n_in; ++k) atomicAdd(grad + mlp_w1(n_in) + j * n_in + k, gW1[k]);
    atomicAdd(grad + mlp_b1(n_in) + j, gB1);
#pragma unroll 8
    for (int k = 0; k < kH; ++k) atomicAdd(grad + mlp_w2(n_in) + j * kH + k, gW2[k]);
    atomicAdd(grad + mlp_b2(n_in) + j, gB2);
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) atomicAdd(grad + mlp_w3(n_in) + o * kH + j, gW3[o]);
    if (j == 0)
#pragma unroll
        for (int o = 0; o < kMlpOut; ++o) atomicAdd(grad + mlp_b3(n_in) + o, gB3[o]);
    if (j < kMlpOut) atomicAdd(loss, lsum);
}

__global__ void k_adam(float* master, __nv_bfloat16* w16, float* m, float* v, float* grad, int np, float inv_n,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const float g = grad[k] * inv_n;
    const float mk = b1 * m[k] + (1.0f - b1) * g;
    const float vk = b2 * v[k] + (1.0f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    const float w = master[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    master[k] = w;
    w16[k] = __float2bfloat16_rn(w);
    grad[k] = 0.0f;
}

__global__ void k_to_bf16(const float* master, __nv_bfloat16* w16, int np) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < np) w16[k] = __float2bfloat16_rn(master[k]);
}

// Forward pass of one normalised input row; returns the de-normalised
// outputs (log h0, log sigma, log cost).
__device__ void mlp_forward(const float* sw, int n_in, const float* x, const MlpNorm& norm, float* out) {
    const float* W1 = sw + mlp_w1(n_in);
    const float* B1 = sw + mlp_b1(n_in);
    const float* W2 = sw + mlp_w2(n_in);
    const float* B2 = sw + mlp_b2(n_in);
    const float* W3 = sw + mlp_w3(n_in);
    const float* B3 = sw + mlp_b3(n_in);
    float a1[kH];
#pragma unroll
    for (int jj = 0; jj < kH; ++jj) {
        float z = B1[jj];
        for (int k = 0; k < n_in; ++k) z += W1[jj * n_in + k] * x[k];
        a1[jj] = silu(z);
    }
    float o[kMlpOut];
#pragma unroll
    for (int q = 0; q < kMlpOut; ++q) o[q] = B3[q];
    for (int jj = 0; jj < kH; ++jj) {
        float z = B2[jj];
#pragma unroll
        for (int k = 0; k < kH; ++k) z += W2[jj * kH + k] * a1[k];
        const float a2 = silu(z);
#pragma unroll
        for (int q = 0; q < kMlpOut; ++q) o[q] += W3[q * kH + jj] * a2;
    }
#pragma unroll
    for (int q = 0; q < kMlpOut; ++q) out[q] = o[q] * norm.y_scale[q] + norm.y_mean[q];
}

// Outputs for feature rows X [n][n_in] (raw features, normalised here).
__global__ void k_mlp_apply(const __nv_bfloat16* w16, const MlpNorm norm, int n_in, const float* X, int64_t n,
                            float* out) {
    extern __shared__ float sw[];
    load_weights(w16, sw, mlp_nparams(n_in));
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[kMlpMaxIn];
    for (int k = 0; k < n_in; ++k) x[k] = (X[r * n_in + k] - norm.x_mean[k]) / norm.x_scale[k];
    mlp_forward(sw, n_in, x, norm, out + r * kMlpOut);
}

// Proposals for an SoA batch: features log max(|y_k|, 1e-30) and the raw
// parameter; NaN outputs (no proposal) outside the training input box
// (widened by `margin` of its width) or when not finite.  The predicted
// cost (optional) is written wherever it is finite.
__global__ void k_mlp_propose(const __nv_bfloat16* w16, const MlpNorm norm, int n_in, int64_t nsys, int neq,
                              const double* y0, const double* params, float margin, float* h0, float* sigma0,
                              float* cost) {
    extern __shared__ float sw[];
    load_weights(w16, sw, mlp_nparams(n_in));
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsys) return;
    float x[kMlpMaxIn];
    bool inside = true;
    for (int k = 0; k < n_in; ++k) {
        const double raw = k < neq ? log(fmax(fabs(y0[i + nsys * (int64_t)k]), 1e-30)) : params[i];
        const float xr = (float)raw;
        const float w = norm.x_max[k] - norm.x_min[k];
        if (!(xr >= norm.x_min[k] - margin * w && xr <= norm.x_max[k] + margin * w)) inside = false;
        x[k] = (xr - norm.x_mean[k]) / norm.x_scale[k];
    }
    float out[kMlpOut];
    mlp_forward(sw, n_in, x, norm, out);
    const float h = expf(out[0]), s = expf(out[1]);
    const bool ok = inside && isfinite(h) && isfinite(s) && h > 0.f && s > 0.f;
    h0[i] = ok ? h : __int_as_float(0x7fffffff);
    sigma0[i] = ok ? s : __int_as_float(0x7fffffff);
    if (cost) {
        const float c = expf(out[2]);
        cost[i] = isfinite(c) ? c : __int_as_float(0x7fffffff);
    }
}

// Per-block partial sums / extrema / counts of the finite values of the
// feature and target columns.
__global__ void k_stats(const float* X, const float* Y, int64_t n, int n_in, double* part) {
    const int F = n_in + kMlpOut;
    const int f = threadIdx.x;  // one column per thread
    if (f >= F) return;
    double s = 0.0, ss = 0.0, cnt = 0.0;
    float lo = 3.0e38f, hi = -3.0e38f;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const float x = f < n_in ? X[r * n_in + f] : Y[r * kMlpOut + (f - n_in)];
        if (!isfinite(x)) continue;
        s += x;
        ss += (double)x * x;
        cnt += 1.0;
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
    }
    double* p = part + ((int64_t)blockIdx.x * F + f) * 5;
    p[0] = s;
    p[1] = ss;
    p[2] = lo;
    p[3] = hi;
    p[4] = cnt;
}

// The inference copy: B fragments (lane l of n-tile nt, k-step ks holds
// W[8 nt + l / 4][16 ks + 2 (l % 4) + {0, 1, 8, 9}], BF16 pairs, the lower
// column in the low half), zero outside the layer; biases as the BF16
// values the other kernels use, widened to FP32.
__global__ void k_pack(const __nv_bfloat16* __restrict__ w16, int n_in, MlpPacked* out) {
    const uint16_t* w = reinterpret_cast<const uint16_t*>(w16);
    auto el = [&](int off, int rows, int cols, int r, int c) -> uint32_t {
        return (r < rows && c < cols) ? (uint32_t)w[off + r * cols + c] : 0u;
    };
    auto frag = [&](int off, int rows, int cols, int KS, int idx) {
        const int nt = idx / (KS * 32), ks = (idx / 32) % KS, l = idx % 32;
        const int r = 8 * nt + (l >> 2), c = 16 * ks + 2 * (l & 3);
        return make_uint2(el(off, rows, cols, r, c) | (el(off, rows, cols, r, c + 1) << 16),
                          el(off, rows, cols, r, c + 8) | (el(off, rows, cols, r, c + 9) << 16));
    };
    for (int k = threadIdx.x; k < 8 * kMlpWarpKs1 * 32; k += blockDim.x)
        out->w1[k] = frag(mlp_w1(n_in), kH, n_in, kMlpWarpKs1, k);
    for (int k = threadIdx.x; k < 8 * 4 * 32; k += blockDim.x) out->w2[k] = frag(mlp_w2(n_in), kH, kH, 4, k);
    for (int k = threadIdx.x; k < 4 * 32; k += blockDim.x) out->w3[k] = frag(mlp_w3(n_in), kMlpOut, kH, 4, k);
    for (int k = threadIdx.x; k < kH; k += blockDim.x) {
        out->b1[k] = __bfloat162float(w16[mlp_b1(n_in) + k]);
        out->b2[k] = __bfloat162float(w16[mlp_b2(n_in) + k]);
    }
    if (threadIdx.x < 8) out->b3[threadIdx.x] = threadIdx.x < kMlpOut ? __bfloat162float(w16[mlp_b3(n_in) + threadIdx.x]) : 0.0f;
}

// Outputs 0 and 1 of raw feature rows through the in-kernel evaluation:
// one warp per 32 rows (KS k-steps of 16 inputs), the BF16 features staged
// in a shared-memory row per thread as the integration kernels stage them.
template <int KS>
__global__ void __launch_bounds__(128) k_mlp_apply_warp(const MlpPacked* __restrict__ net, const float* __restrict__ X,
                                                         int64_t n, float* __restrict__ out) {
    constexpr int kStride = 8 * KS + 1;  // words per row (odd: fewer bank conflicts)
    __shared__ uint32_t rows[128 * kStride];
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool have = r < n;
    const unsigned take = __ballot_sync(0xffffffffu, have);
    const int n_in = net->n_in;
    uint32_t* mine = rows + threadIdx.x * kStride;
    uint16_t* fr = reinterpret_cast<uint16_t*>(mine);
    for (int k = 0; k < 16 * KS; ++k)
        fr[k] = to_bf16((have && k < n_in) ? (X[r * n_in + k] - net->x_mean[k]) * net->x_iscale[k] : 0.0f);
    __syncwarp();
    float o0 = 0.0f, o1 = 0.0f;
    mlp_warp_eval<KS>(net, take, mine, kStride, o0, o1);
    if (!have) return;
    out[2 * r] = o0 * net->y_scale[0] + net->y_mean[0];
    out[2 * r + 1] = o1 * net->y_scale[1] + net->y_mean[1];
}

size_t grad_smem(int n_in) { return sizeof(float) * (mlp_nparams(n_in) + kMlpMaxIn + 3 * kH + kMlpOut); }
size_t apply_smem(int n_in) { return sizeof(float) * mlp_nparams(n_in); }

int get(int32_t h, Mlp** out) {
    auto it = g_mlps.find(h);
    if (it == g_mlps.end()) return fail(ODE_ERR_HANDLE, "unknown mlp handle %d", h);
    *out = &it->second;
    return ODE_OK;
}

// Rebuilds the inference copy from the BF16 weights and the normalisation
// (after every change of either); synchronous on s.
int refresh_packed(Mlp& net, cudaStream_t s) {
    if (!net.packed) return ODE_OK;
    k_pack<<<1, 256, 0, s>>>(net.w16, net.n_in, net.packed);
    MlpPacked h;  // the host-built part: normalisation and the widened box
    std::memset(&h, 0, sizeof(h));
    for (int k = 0; k < kMlpMaxIn; ++k) {
        h.x_mean[k] = net.norm.x_mean[k];
        h.x_iscale[k] = 1.0f / net.norm.x_scale[k];
        const float w = net.norm.x_max[k] - net.norm.x_min[k];
        h.x_lo[k] = net.norm.x_min[k] - kBoxMargin * w;
        h.x_hi[k] = net.norm.x_max[k] + kBoxMargin * w;
    }
    for (int k = 0; k < kMlpOut; ++k) {
        h.y_mean[k] = net.norm.y_mean[k];
        h.y_scale[k] = net.norm.y_scale[k];
    }
    h.n_in = net.n_in;
    const size_t off = offsetof(MlpPacked, x_mean);
    cudaError_t e = cudaMemcpyAsync(reinterpret_cast<char*>(net.packed) + off, reinterpret_cast<const char*>(&h) + off,
                                    sizeof(MlpPacked) - off, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? ODE_OK : cuda_fail(e, "network inference copy");
}

// gradient of the summed loss over n rows (device X, Y) into net.grad / net.loss
int run_grad(Mlp& net, const float* X, const float* Y, const int32_t* perm, int64_t n, cudaStream_t s) {
    const int per_block = 32;
    const int64_t blocks = (n + per_block - 1) / per_block;
    k_mlp_grad<<<(unsigned)blocks, kH, grad_smem(net.n_in), s>>>(net.w16, net.norm, net.n_in, X, Y, perm, n, per_block,
                                                                  net.grad, net.loss);
    return cudaGetLastError() == cudaSuccess ? ODE_OK : ODE_ERR_CUDA;
}

}  // namespace

namespace bode {
// The inference copy of network `handle` for an integration whose systems
// have n_in - 1 components (ODE_ERR_HANDLE / ODE_ERR_ARG otherwise).
int mlp_packed_for(int32_t handle, int n_in, const MlpPacked** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (net->n_in != n_in) return fail(ODE_ERR_ARG, "network takes %d inputs, the systems have %d + 1", net->n_in, n_in - 1);
    *out = net->packed;
    return ODE_OK;
}
}  // namespace bode

extern "C" {

int ode_mlp_create(int32_t n_in, uint64_t seed, int32_t* handle) {
    clear_last_error();
    if (!handle) return fail(ODE_ERR_ARG, "handle is NULL");
    if (n_in < 1 || n_in > kMlpMaxIn) return fail(ODE_ERR_ARG, "n_in must be in [1, %d]", kMlpMaxIn);
    Mlp net;
    net.n_in = n_in;
    net.nparams = mlp_nparams(n_in);
    cudaError_t e = cudaGetDevice(&net.dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    // Glorot-uniform weights, zero biases
    std::vector<float> w(net.nparams, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int rows, int cols) {
        const float a = std::sqrt(6.0f / (float)(rows + cols));
        std::uniform_real_distribution<float> u(-a, a);
        for (int k = 0; k < rows * cols; ++k) w[off + k] = u(rng);
    };
    fill(mlp_w1(n_in), kH, n_in);
    fill(mlp_w2(n_in), kH, kH);
    fill(mlp_w3(n_in), kMlpOut, kH);
    const size_t nb = sizeof(float) * net.nparams;
    e = cudaMalloc(&net.master, nb);
    if (e == cudaSuccess) e = cudaMalloc(&net.w16, sizeof(__nv_bfloat16) * net.nparams);
    if (e == cudaSuccess) e = cudaMalloc(&net.m, nb);
    if (e == cudaSuccess) e = cudaMalloc(&net.v, nb);
    if (e == cudaSuccess) e = cudaMalloc(&net.grad, nb);
    if (e == cudaSuccess) e = cudaMalloc(&net.loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net.packed, sizeof(MlpPacked));
    if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "mlp allocation failed");
    cudaMemcpy(net.master, w.data(), nb, cudaMemcpyHostToDevice);
    cudaMemset(net.m, 0, nb);
    cudaMemset(net.v, 0, nb);
    cudaMemset(net.grad, 0, nb);
    k_to_bf16<<<(net.nparams + 255) / 256, 256>>>(net.master, net.w16, net.nparams);
    for (int k = 0; k < kMlpMaxIn; ++k) {
        net.norm.x_mean[k] = 0.f;
        net.norm.x_scale[k] = 1.f;
        net.norm.x_min[k] = -3.0e38f;
        net.norm.x_max[k] = 3.0e38f;
    }
    for (int k = 0; k < kMlpOut; ++k) {
        net.norm.y_mean[k] = 0.f;
        net.norm.y_scale[k] = 1.f;
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "mlp initialisation");
    if (int rc = refresh_packed(net, nullptr)) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    *handle = g_next++;
    g_mlps[*handle] = net;
    return ODE_OK;
}

int ode_mlp_release(int32_t handle) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    cudaFree(net->master);
    cudaFree(net->w16);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->grad);
    cudaFree(net->loss);
    cudaFree(net->packed);
    g_mlps.erase(handle);
    return ODE_OK;
}

int ode_mlp_fit_normalization(int32_t handle, const float* X, const float* Y, int64_t n, void* stream) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (!X || !Y || n < 2) return fail(ODE_ERR_ARG, "need device X, Y and n >= 2");
    const int F = net->n_in + kMlpOut;
    const int blocks = 1024;
    double* part = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&part, sizeof(double) * blocks * F * 5);
    if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "statistics buffer");
    k_stats<<<blocks, 64, 0, s>>>(X, Y, n, net->n_in, part);
    std::vector<double> h((size_t)blocks * F * 5);
    e = cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(part);
    if (e != cudaSuccess) return cuda_fail(e, "statistics");
    for (int f = 0; f < F; ++f) {
        double sum = 0, sq = 0, lo = 3e38, hi = -3e38, cnt = 0;
        for (int b = 0; b < blocks; ++b) {
            const double* p = &h[((size_t)b * F + f) * 5];
            sum += p[0];
            sq += p[1];
            lo = std::min(lo, p[2]);
            hi = std::max(hi, p[3]);
            cnt += p[4];
        }
        if (cnt < 2) {  // no statistics: identity normalisation, unbounded box
            sum = sq = 0;
            cnt = 1;
            lo = -3e38;
            hi = 3e38;
        }
        const double mean = sum / cnt;
        const double sd = std::sqrt(std::max(sq / cnt - mean * mean, 0.0));
        const float scale = (float)(sd > 1e-12 ? sd : 1.0);
        if (f < net->n_in) {
            net->norm.x_mean[f] = (float)mean;
            net->norm.x_scale[f] = scale;
            net->norm.x_min[f] = (float)lo;
            net->norm.x_max[f] = (float)hi;
        } else {
            net->norm.y_mean[f - net->n_in] = (float)mean;
            net->norm.y_scale[f - net->n_in] = scale;
        }
    }
    net->has_norm = true;
    return refresh_packed(*net, s);
}

int ode_mlp_gradient(int32_t handle, const float* X, const float* Y, int64_t n, float* grad_out, float* loss_out,
                     void* stream) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (!X || !Y || !grad_out || n < 1) return fail(ODE_ERR_ARG, "need device X, Y, grad_out and n >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(net->grad, 0, sizeof(float) * net->nparams, s);
    cudaMemsetAsync(net->loss, 0, sizeof(float), s);
    if (run_grad(*net, X, Y, nullptr, n, s)) return cuda_fail(cudaGetLastError(), "gradient kernel");
    // mean over the rows
    std::vector<float> g(net->nparams);
    float l = 0;
    cudaError_t e = cudaMemcpyAsync(g.data(), net->grad, sizeof(float) * net->nparams, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, net->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "gradient copy");
    for (auto& x : g) x /= (float)n;
    cudaMemsetAsync(net->grad, 0, sizeof(float) * net->nparams, s);
    e = cudaMemcpyAsync(grad_out, g.data(), sizeof(float) * net->nparams, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "gradient copy");
    if (loss_out) *loss_out = l / (float)n;
    return ODE_OK;
}

int ode_mlp_train(int32_t handle, const float* X, const float* Y, int64_t n, const ode_train_opts* o,
                  float* loss_history, void* stream) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (!X || !Y || !o || n < 1) return fail(ODE_ERR_ARG, "need device X, Y, options and n >= 1");
    if (o->epochs < 1 || o->batch < 1 || !(o->lr > 0)) return fail(ODE_ERR_ARG, "need epochs >= 1, batch >= 1, lr > 0");
    if (!net->has_norm) return fail(ODE_ERR_ARG, "call ode_mlp_fit_normalization first");
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* perm = nullptr;
    cudaError_t e = cudaMalloc(&perm, sizeof(int32_t) * n);
    if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "permutation buffer");
    std::vector<int32_t> hp(n);
    std::mt19937_64 rng(o->seed);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < o->epochs; ++ep) {
        for (int64_t k = 0; k < n; ++k) hp[k] = (int32_t)k;
        std::shuffle(hp.begin(), hp.end(), rng);
        cudaMemcpyAsync(perm, hp.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(net->loss, 0, sizeof(float), s);
        for (int64_t b0 = 0; b0 < n; b0 += o->batch) {
            const int64_t bn = std::min<int64_t>(o->batch, n - b0);
            if (run_grad(*net, X, Y, perm + b0, bn, s)) {
                cudaFree(perm);
                return cuda_fail(cudaGetLastError(), "gradient kernel");
            }
            net->step += 1;
            const float c1 = 1.0f - std::pow(b1, (float)net->step), c2 = 1.0f - std::pow(b2, (float)net->step);
            k_adam<<<(net->nparams + 255) / 256, 256, 0, s>>>(net->master, net->w16, net->m, net->v, net->grad,
                                                             net->nparams, 1.0f / (float)bn, o->lr, b1, b2, eps, c1, c2);
        }
        float l = 0;
        e = cudaMemcpyAsync(&l, net->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(perm);
            return cuda_fail(e, "training");
        }
        if (loss_history) loss_history[ep] = l / (float)n;
    }
    cudaFree(perm);
    return refresh_packed(*net, s);
}

int ode_mlp_apply(int32_t handle, const float* X, int64_t n, float* out, void* stream) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (!X || !out || n < 0) return fail(ODE_ERR_ARG, "need device X and out");
    if (n == 0) return ODE_OK;
    k_mlp_apply<<<(unsigned)((n + 127) / 128), 128, apply_smem(net->n_in), (cudaStream_t)stream>>>(
        net->w16, net->norm, net->n_in, X, n, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ODE_OK : cuda_fail(e, "mlp apply");
}

int ode_mlp_propose(int32_t handle, int64_t nsys, int32_t neq, const double* y0, const double* params, float margin,
                    float* h0, float* sigma0, float* cost, void* stream) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (neq + 1 != net->n_in) return fail(ODE_ERR_ARG, "network takes %d inputs, state has %d + 1", net->n_in, neq);
    if (!y0 || !params || !h0 || !sigma0 || nsys < 0) return fail(ODE_ERR_ARG, "need device y0, params, h0, sigma0");
    if (nsys == 0) return ODE_OK;
    k_mlp_propose<<<(unsigned)((nsys + 127) / 128), 128, apply_smem(net->n_in), (cudaStream_t)stream>>>(
        net->w16, net->norm, net->n_in, nsys, neq, y0, params, margin, h0, sigma0, cost);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ODE_OK : cuda_fail(e, "mlp proposal");
}

int ode_mlp_get_params(int32_t handle, float* params, float* norm) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (params) {
        cudaError_t e = cudaMemcpy(params, net->master, sizeof(float) * net->nparams, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "parameter copy");
    }
    if (norm) std::memcpy(norm, &net->norm, sizeof(MlpNorm));
    return ODE_OK;
}

int ode_mlp_set_params(int32_t handle, const float* params, const float* norm) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (params) {
        cudaError_t e = cudaMemcpy(net->master, params, sizeof(float) * net->nparams, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "parameter copy");
        k_to_bf16<<<(net->nparams + 255) / 256, 256>>>(net->master, net->w16, net->nparams);
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "parameter copy");
    }
    if (norm) {
        std::memcpy(&net->norm, norm, sizeof(MlpNorm));
        net->has_norm = true;
    }
    return refresh_packed(*net, nullptr);
}

int ode_mlp_apply_warp(int32_t handle, const float* X, int64_t n, float* out, void* stream) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    Mlp* net;
    int rc = get(handle, &net);
    if (rc) return rc;
    if (!X || !out || n < 0) return fail(ODE_ERR_ARG, "need device X and out");
    if (n == 0) return ODE_OK;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    cudaStream_t s = (cudaStream_t)stream;
    const int ks = (net->n_in + 15) / 16;
    if (ks == 1)
        k_mlp_apply_warp<1><<<blocks, 128, 0, s>>>(net->packed, X, n, out);
    else if (ks == 2)
        k_mlp_apply_warp<2><<<blocks, 128, 0, s>>>(net->packed, X, n, out);
    else
        k_mlp_apply_warp<3><<<blocks, 128, 0, s>>>(net->packed, X, n, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ODE_OK : cuda_fail(e, "mlp warp apply");
}

int ode_mlp_num_params(int32_t n_in) { return n_in >= 1 && n_in <= kMlpMaxIn ? mlp_nparams(n_in) : -1; }

}  // extern "C"
