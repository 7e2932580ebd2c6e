// k_table.cu -- RKC stage-coefficient tables, built once per device.
#include "integrators.cuh"
#include "launch.cuh"

namespace bode {

__global__ void k_build_rkc_table(double* tab64, float4* tab32, int mmax) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x + 2;
    if (m > mmax) return;
    RkcStageGen g;
    g.start(m);
    const int base = rkc_tab_index(m, 1);
    double* e = tab64 + 8 * base;
    e[0] = 0.0;
    e[1] = 0.0;
    e[2] = 0.0;
    e[3] = g.mut1;
    e[4] = 0.0;
    e[5] = 0.0;
    e[6] = 0.0;
    e[7] = 0.0;
    tab32[base] = make_float4(0.0f, 0.0f, (float)g.mut1, 0.0f);
    // trailing words of the two-float coefficients in the entry's last 16 bytes
    reinterpret_cast<float4*>(e + 6)[0] = make_float4(0.0f, 0.0f, F2(g.mut1).lo, 0.0f);
    for (int j = 2; j <= m; ++j) {
        const StageCoef s = g.next();
        e = tab64 + 8 * (base + j - 1);
        e[0] = s.cy;
        e[1] = s.mu;
        e[2] = s.nu;
        e[3] = s.mut;
        e[4] = s.gt;
        e[5] = s.cprev;
        tab32[base + j - 1] = make_float4((float)s.mu, (float)s.nu, (float)s.mut, (float)s.gt);
        reinterpret_cast<float4*>(e + 6)[0] = make_float4(F2(s.mu).lo, F2(s.nu).lo, F2(s.mut).lo, F2(s.gt).lo);
    }
}

cudaError_t build_rkc_tables(double* tab64, float4* tab32, int mmax, cudaStream_t s) {
    const int count = mmax - 1;
    k_build_rkc_table<<<(count + 63) / 64, 64, 0, s>>>(tab64, tab32, mmax);
    return cudaGetLastError();
}

}  // namespace bode
