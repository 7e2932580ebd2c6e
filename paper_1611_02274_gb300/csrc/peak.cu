// peak.cu -- FMA-chain throughput microbenchmark (include/batchode_bench.h).
#include <cuda_runtime.h>

#include "batchode.h"
#include "batchode_bench.h"

namespace {

constexpr int kIlp = 8;

template <class T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, int iters, T a, T b) {
    T x[kIlp];
#pragma unroll
    for (int i = 0; i < kIlp; ++i) x[i] = (T)(threadIdx.x & 7) + (T)i;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < kIlp; ++i) x[i] = fma(x[i], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int i = 0; i < kIlp; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int run(int iters, double* gflops, double* ms) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ODE_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ODE_ERR_CUDA;
    const int block = 256, grid = sms * 8;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * grid * block) != cudaSuccess) return ODE_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chain<T><<<grid, block>>>(out, iters / 4 + 1, (T)0.999999, (T)1e-6);  // warm-up
    cudaEventRecord(e0);
    k_fma_chain<T><<<grid, block>>>(out, iters, (T)0.999999, (T)1e-6);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return ODE_ERR_CUDA;
    *ms = t;
    *gflops = 2.0 * kIlp * (double)iters * grid * block / (t * 1e-3) / 1e9;
    return ODE_OK;
}

}  // namespace

extern "C" int bode_fma_peak(int fp64, int32_t iters, double* gflops, double* ms) {
    if (iters < 1 || !gflops || !ms) return ODE_ERR_ARG;
    return fp64 ? run<double>(iters, gflops, ms) : run<float>(iters, gflops, ms);
}
