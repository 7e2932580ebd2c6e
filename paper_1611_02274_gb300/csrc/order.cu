// order.cu -- longest-first order of a batch from per-system cost estimates.
//
// A counting sort on a 16-bit cost class.  Positive floats order like their
// bit patterns, and the bit pattern is close to a scaled log2 of the value,
// so the classes split the range [lo, hi] of the batch's positive costs'
// bit patterns into 65535 equal steps (about log-uniform): class
// 1 + (bits - lo) * 65535 / (hi - lo + 1); NaN and values <= 0 form class 0.
// Classes that narrow matter: systems of almost equal cost follow almost the
// same step sequence, so a warp of them stays in phase (merging neighbouring
// costs of a few parts in a thousand measurably costs time), and a few
// outliers must not widen the classes much.  Four launches:
//   k_order_range    lo and hi (block reductions, one atomic each per warp);
//   k_order_hist     class histogram (global atomics, aggregated over the
//                    lanes of a warp that share a class);
//   k_order_scan     one block: descending exclusive scan, so the most
//                    expensive class starts at position 0;
//   k_order_scatter  each system's position from its class's running
//                    offset (lanes of a warp with the same class take
//                    consecutive positions with one atomic).
// Systems of one class land in an unspecified order; the integration
// results do not depend on it.
#include <cuda_runtime.h>

#include <cstdint>

#include "order.h"

namespace bode {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kBinsPerThread = kOrderBins / kScanThreads;
static_assert(kOrderBins % kScanThreads == 0, "bins split evenly over the scan block");

// a cost as float: float32 estimates, or int32 counts (e.g. n_rhs)
__device__ __forceinline__ float cost_at(const void* cost, int kind, int64_t i) {
    return kind == 1 ? (float)static_cast<const int32_t*>(cost)[i] : static_cast<const float*>(cost)[i];
}

// range[0] = lo, range[1] = hi (bit patterns of the positive costs)
__device__ __forceinline__ int cost_class(float c, const uint32_t* range) {
    if (!(c > 0.0f)) return 0;  // NaN, zero and negative estimates: cheapest
    const uint32_t lo = range[0], hi = range[1];
    const uint64_t step = (uint64_t)(__float_as_uint(c) - lo) * (uint64_t)(kOrderBins - 1);
    return 1 + (int)(step / ((uint64_t)(hi - lo) + 1u));
}

__global__ void k_order_range(const void* __restrict__ cost, int kind, int64_t n, uint32_t* __restrict__ range) {
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float c = cost_at(cost, kind, i);
        if (c > 0.0f) {
            lo = min(lo, __float_as_uint(c));
            hi = max(hi, __float_as_uint(c));
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0 && hi >= lo) {
        atomicMin(&range[0], lo);
        atomicMax(&range[1], hi);
    }
}

__global__ void k_order_hist(const void* __restrict__ cost, int kind, int64_t n, const uint32_t* __restrict__ range,
                             int32_t* __restrict__ hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    if (!live) return;
    const int cls = cost_class(cost_at(cost, kind, i), range);
    const unsigned peers = __match_any_sync(active, cls);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[cls], __popc(peers));
}

// offset[b] = number of systems in classes above b
__global__ void __launch_bounds__(kScanThreads) k_order_scan(const int32_t* __restrict__ hist,
                                                             int32_t* __restrict__ offset) {
    __shared__ int32_t warp_sums[kScanThreads / 32];
    const int t = threadIdx.x;
    // thread t owns classes top - kBinsPerThread t - q, q = 0 .. kBinsPerThread - 1
    const int top = kOrderBins - 1 - kBinsPerThread * t;
    int32_t local = 0;
    for (int q = 0; q < kBinsPerThread; ++q) local += hist[top - q];
    // inclusive scan over the threads (warp shuffles, then the warp totals)
    int32_t x = local;
    const int lane = t & 31, warp = t >> 5;
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    int32_t run = x - local + (warp > 0 ? warp_sums[warp - 1] : 0);  // exclusive prefix of this thread
    for (int q = 0; q < kBinsPerThread; ++q) {
        offset[top - q] = run;
        run += hist[top - q];
    }
}

__global__ void k_order_scatter(const void* __restrict__ cost, int kind, int64_t n,
                                 const uint32_t* __restrict__ range, int32_t* __restrict__ offset,
                                 int32_t* __restrict__ index) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < n;
    const int cls = live ? cost_class(cost_at(cost, kind, i), range) : -1;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    if (!live) return;
    const unsigned peers = __match_any_sync(active, cls);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(&offset[cls], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    index[base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)i;
}

}  // namespace

cudaError_t order_by_cost(const void* cost, int kind, int64_t n, int32_t* bins, int32_t* index, int sm_count,
                          cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int32_t* hist = bins;
    int32_t* offset = bins + kOrderBins;
    uint32_t* range = reinterpret_cast<uint32_t*>(bins + 2 * kOrderBins);
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * kOrderBins, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(range, 0xff, sizeof(uint32_t), s);      // lo = max
    if (e == cudaSuccess) e = cudaMemsetAsync(range + 1, 0, sizeof(uint32_t), s);     // hi = 0
    if (e != cudaSuccess) return e;
    const int64_t blocks = (n + 255) / 256;
    const unsigned grid = (unsigned)(blocks < 4 * (int64_t)sm_count ? blocks : 4 * (int64_t)sm_count);
    k_order_range<<<grid, 256, 0, s>>>(cost, kind, n, range);
    k_order_hist<<<(unsigned)blocks, 256, 0, s>>>(cost, kind, n, range, hist);
    k_order_scan<<<1, kScanThreads, 0, s>>>(hist, offset);
    k_order_scatter<<<(unsigned)blocks, 256, 0, s>>>(cost, kind, n, range, offset, index);
    return cudaGetLastError();
}

}  // namespace bode
