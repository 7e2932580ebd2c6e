// mlp_warp.cuh -- the proposal network evaluated inside an integration
// kernel by one warp for its 32 systems, on the tensor cores.
//
// The RKC kernels call it where the Appendix's power method would run (the
// 25-step schedule and the start; never after a rejection): the lanes that
// need a spectral-radius bound pass their features, the warp evaluates the
// n_in -> 64 -> 64 -> 3 network as three small matrix products with
// mma.sync m16n8k16 (BF16 operands, FP32 accumulation), 16 systems per
// tile, and each lane gets its own row's outputs back.  The step-end hold
// keeps the lanes of a warp on the same accepted-step count, so their
// schedule points coincide and one evaluation serves most of the warp.
//
// Why mma.sync and not tcgen05: the products are 16 x {16..48} x 64 per
// tile, issued from inside a per-thread phase machine whose warps are at
// arbitrary points of their loops; tcgen05 wants a single issuing thread,
// operands in shared memory and an accumulator allocation in tensor memory
// -- all of it shared-memory and synchronisation traffic larger than the
// few dozen warp-level instructions used here.
//
// Layer outputs feed the next layer's A operand straight from the
// accumulator registers: in the m16n8k16 layouts, the accumulator of
// n-tiles 2k and 2k+1 holds exactly the A fragment of k-step k.  Inputs
// come from shared memory: each lane writes its normalised features as BF16
// into a row of its own, and the A fragments are read from the rows.
#pragma once
#include <cstdint>

#include "mlp.cuh"

namespace bode {

constexpr int kMlpWarpKs1 = 3;  // k-steps of the first layer: inputs up to 48 (33 used)

// Inference copy of a network, built by the library from its BF16 weights
// (fragment-major: lane l's B fragment of n-tile nt and k-step ks at
// [(nt * KS + ks) * 32 + l], two BF16 pairs) and its normalisation.
struct MlpPacked {
    uint2 w1[8 * kMlpWarpKs1 * 32];  // W1 [64][n_in], zero past n_in
    uint2 w2[8 * 4 * 32];            // W2 [64][64]
    uint2 w3[1 * 4 * 32];            // W3 [3][64], rows 3..7 zero
    float b1[kMlpHidden], b2[kMlpHidden], b3[8];
    float x_mean[kMlpMaxIn], x_iscale[kMlpMaxIn];  // features normalised as (x - mean) * iscale
    float x_lo[kMlpMaxIn], x_hi[kMlpMaxIn];       // the training box widened by the margin
    float y_mean[kMlpOut], y_scale[kMlpOut];
    int32_t n_in;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// c += a * b for one 16 x 8 tile (k = 16), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// Weight and bias loads with L1 priority: the 12 KB the evaluation reads are
// fetched by every warp of the SM at its schedule points, far apart in time;
// evict_last keeps them in L1 against the kernel's own traffic there.
__device__ __forceinline__ uint2 ld_keep(const uint2* p) {
    uint2 v;
    asm volatile("ld.global.nc.L1::evict_last.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float2 ld_keep(const float* p) {
    float2 v;
    asm volatile("ld.global.nc.L1::evict_last.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ uint16_t to_bf16(float x) {
    uint16_t r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}

// Normalised outputs 0 (log h0) and 1 (log sigma) of this lane's row for the
// lanes in `take` (a warp-uniform mask; all 32 lanes call).  Each lane's
// normalised features are BF16 values in shared memory, 16 KS of them
// (zero past n_in), in a row of `stride` 32-bit words; `row` is this lane's
// row and lane L's is row + (L - lane) stride.  Tiles (16 lanes each) with
// no lane in `take` are skipped.
//
// The code is kept small on purpose: it runs rarely, so its instructions are
// fetched cold each time, and that fetch -- not the few dozen products --
// sets its cost.  Layer 1 is computed two n-tiles at a time inside the
// loop that accumulates layer 2 (layer-1 n-tiles 2k and 2k+1 are layer 2's
// A fragment k), and layer 3 consumes layer 2's accumulators two n-tiles
// per pass, the rest moved down a place; both loops stay rolled.
template <int KS>
__device__ __forceinline__ void mlp_warp_eval(const MlpPacked* __restrict__ net, unsigned take,
                                              const uint32_t* row, int stride, float& out0, float& out1) {
    static_assert(KS >= 1 && KS <= kMlpWarpKs1, "inputs up to 48");
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll 1
    for (int t = 0; t < 2; ++t) {
        if (((take >> (16 * t)) & 0xffffu) == 0u) continue;
        // rows g and g + 8 of the tile: lanes 16 t + g and 16 t + g + 8
        const uint32_t* ra = row + (16 * t + g - lane) * stride;
        const uint32_t* rb = ra + 8 * stride;
        uint32_t a1[KS][4];
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            a1[ks][0] = ra[8 * ks + q];
            a1[ks][1] = rb[8 * ks + q];
            a1[ks][2] = ra[8 * ks + 4 + q];
            a1[ks][3] = rb[8 * ks + 4 + q];
        }
        float c[8][4];  // layer-2 accumulators
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 b = ld_keep(net->b2 + 8 * nt + 2 * q);
            c[nt][0] = c[nt][2] = b.x;
            c[nt][1] = c[nt][3] = b.y;
        }
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            uint2 w1f[2][KS], w2f[8];
            float2 b1f[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                b1f[e] = ld_keep(net->b1 + 8 * (2 * k + e) + 2 * q);
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) w1f[e][ks] = ld_keep(&net->w1[((2 * k + e) * kMlpWarpKs1 + ks) * 32 + lane]);
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) w2f[nt] = ld_keep(&net->w2[(nt * 4 + k) * 32 + lane]);
            float z[2][4];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                z[e][0] = z[e][2] = b1f[e].x;
                z[e][1] = z[e][3] = b1f[e].y;
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) mma_16816(z[e], a1[ks], w1f[e][ks]);
            }
            const uint32_t a2[4] = {pack_bf16x2(silu_fast(z[0][0]), silu_fast(z[0][1])),
                                    pack_bf16x2(silu_fast(z[0][2]), silu_fast(z[0][3])),
                                    pack_bf16x2(silu_fast(z[1][0]), silu_fast(z[1][1])),
                                    pack_bf16x2(silu_fast(z[1][2]), silu_fast(z[1][3]))};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) mma_16816(c[nt], a2, w2f[nt]);
        }
        float o[4];
        {
            const float2 b = ld_keep(net->b3 + 2 * q);
            o[0] = o[2] = b.x;
            o[1] = o[3] = b.y;
        }
#pragma unroll 1
        for (int k3 = 0; k3 < 4; ++k3) {
            const uint2 w3f = ld_keep(&net->w3[k3 * 32 + lane]);
            const uint32_t a3[4] = {pack_bf16x2(silu_fast(c[0][0]), silu_fast(c[0][1])),
                                    pack_bf16x2(silu_fast(c[0][2]), silu_fast(c[0][3])),
                                    pack_bf16x2(silu_fast(c[1][0]), silu_fast(c[1][1])),
                                    pack_bf16x2(silu_fast(c[1][2]), silu_fast(c[1][3]))};
            mma_16816(o, a3, w3f);
#pragma unroll
            for (int nt = 0; nt < 6; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) c[nt][e] = c[nt + 2][e];
        }
        // row r of the tile: columns 0 and 1 sit in lane 4 (r mod 8), registers 0/1 (r < 8) or 2/3
        const int r = (lane - 16 * t) & 15, src = 4 * (r & 7);
        const float v0 = __shfl_sync(0xffffffffu, o[0], src), v1 = __shfl_sync(0xffffffffu, o[1], src);
        const float v2 = __shfl_sync(0xffffffffu, o[2], src), v3 = __shfl_sync(0xffffffffu, o[3], src);
        if ((lane >> 4) == t) {
            out0 = r < 8 ? v0 : v2;
            out1 = r < 8 ? v1 : v3;
        }
    }
}

}  // namespace bode
