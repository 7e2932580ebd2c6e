// order.h -- longest-first batch order from per-system cost estimates.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace bode {

// Cost classes of the counting sort: class 0 for NaN and values <= 0, then
// 65535 about log-uniform steps over the batch's range of positive costs.
constexpr int kOrderBins = 65536;
// int32 words of device scratch order_by_cost needs
constexpr int kOrderScratchWords = 2 * kOrderBins + 2;

// Writes index[0..n) = the systems 0..n-1, most expensive class first,
// on stream s.  bins: device scratch of kOrderScratchWords int32; index:
// n int32.  cost: device [n], float32 (kind 0) or int32 (kind 1).
cudaError_t order_by_cost(const void* cost, int kind, int64_t n, int32_t* bins, int32_t* index, int sm_count,
                          cudaStream_t s);

}  // namespace bode
