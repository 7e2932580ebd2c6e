// team.cuh -- a team of W consecutive lanes of one warp that owns one ODE
// system.  W = 1 is the paper's one-thread-per-system mapping; W = 32 is
// one warp per system.  Every lane holds PER "slots" of each state vector;
// which component a slot holds is defined by the right-hand-side model.
// Reductions are butterfly shuffles inside the team, so every lane ends with
// the bitwise-identical result and all control decisions stay team-uniform.
#pragma once
#include <cstdint>

#include "f2.cuh"

namespace bode {

// shuffles and maxima through overloadable names (f2.cuh adds the two-float pair)
template <class T>
__device__ __forceinline__ T shfl_xor(unsigned m, T v, int o, int w) { return __shfl_xor_sync(m, v, o, w); }
template <class T>
__device__ __forceinline__ T shfl_idx(unsigned m, T v, int s, int w) { return __shfl_sync(m, v, s, w); }
template <class T>
__device__ __forceinline__ T shfl_up(unsigned m, T v, int d, int w) { return __shfl_up_sync(m, v, d, w); }
template <class T>
__device__ __forceinline__ T shfl_down(unsigned m, T v, int d, int w) { return __shfl_down_sync(m, v, d, w); }
template <class T>
__device__ __forceinline__ T vmax(T a, T b) { return fmax(a, b); }

template <int W_>
struct Team {
    static constexpr int W = W_;
    static_assert(W == 1 || W == 2 || W == 4 || W == 8 || W == 16 || W == 32, "team width");
    int lane;       // 0..W-1
    unsigned mask;  // lanes of this team within the warp

    __device__ static Team make() {
        Team t;
        const int l = threadIdx.x & 31;
        t.lane = l % W;
        t.mask = (W == 32) ? 0xffffffffu : (((1u << W) - 1u) << ((l / W) * W));
        return t;
    }
    template <class T>
    __device__ T sum(T x) const {
        if constexpr (W > 1) {
#pragma unroll
            for (int o = W / 2; o > 0; o >>= 1) x = x + shfl_xor(mask, x, o, W);
        }
        return x;
    }
    template <class T>
    __device__ T max(T x) const {
        if constexpr (W > 1) {
#pragma unroll
            for (int o = W / 2; o > 0; o >>= 1) x = vmax(x, shfl_xor(mask, x, o, W));
        }
        return x;
    }
    __device__ bool any(bool p) const {
        if constexpr (W > 1) return __any_sync(mask, p);
        return p;
    }
    template <class T>
    __device__ T bcast(T x, int src) const {
        if constexpr (W > 1) return shfl_idx(mask, x, src, W);
        return x;
    }
    // value held by lane - 1 (own value on lane 0) and lane + 1 (own value on the last lane)
    template <class T>
    __device__ T from_left(T x) const {
        if constexpr (W > 1) return shfl_up(mask, x, 1, W);
        return x;
    }
    template <class T>
    __device__ T from_right(T x) const {
        if constexpr (W > 1) return shfl_down(mask, x, 1, W);
        return x;
    }
};

}  // namespace bode
