// stoich_bench.cu -- is the stoichiometry product of a mass-action
// right-hand side worth the tensor cores?  (include/batchode_bench.h)
//
// One mass-action evaluation computes the reaction rates r_j (products of a
// rate constant and concentrations) and then f = N r, N the S x R matrix of
// net stoichiometric coefficients (Section 4.2's omega_i sums).  For a warp
// of 32 systems in step that second part is the product
// F[32 x S] = R[32 x R] N^T[R x S], which fits the tensor cores' shapes.
// Three kernels are generated for the registered network and timed on the
// same synthetic rates:
//   variant 0  the sparse form the generated integrators use: one FP32
//              add or subtract per nonzero coefficient occurrence, each
//              species' sum in reaction order;
//   variant 1  mma.sync m16n8k8 with TF32 operands, the rates split into a
//              leading and a trailing TF32 word (two products per tile;
//              the coefficients are small integers, exact in TF32), FP32
//              accumulation: FP32-class accuracy, as the FP32 forms need;
//              the warp stages its rates through shared memory into the
//              A-fragment layout and its results back to one row per lane;
//   variant 2  the sparse form in FP64 (the accuracy reference).
// Each kernel evaluates the product `reps` times per system (rates scaled
// by 1 + rep 1e-7 so that no repetition can be hoisted), stores the last
// and a checksum of all of them (so that none is dead code); the time of
// one product is (t(reps) - t(0)) / reps, so generating the rates and
// storing the results cancel out.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <sstream>
#include <string>
#include <vector>

#include "batchode.h"
#include "batchode_bench.h"
#include "jit.h"
#include "launch.cuh"

namespace bode {
bool registry_lookup(int32_t handle, RhsEntry* out);
int set_last_error(int code, const char* msg);
void clear_last_error();
}  // namespace bode

using namespace bode;

namespace {

int fail(int code, const std::string& msg) { return set_last_error(code, msg.c_str()); }

// Net coefficient of species s in reaction j (products minus reactants).
int coef(const MassActionNet& n, int j, int s) {
    int c = 0;
    for (int q = 0; q < n.n_reac[j]; ++q) c -= n.reac[j][q] == s;
    for (int q = 0; q < n.n_prod[j]; ++q) c += n.prod[j][q] == s;
    return c;
}

std::string program(const MassActionNet& n) {
    const int S = n.n_species, R = n.n_reactions;
    std::ostringstream o;
    o << "#include \"common.cuh\"\n"
      << "namespace {\n"
      << "constexpr int S = " << S << ", R = " << R << ";\n"
      // synthetic rates: log-uniform in [1e-8, 1e4] from an integer hash
      << "__device__ __forceinline__ float rate(long long i, int j) {\n"
      << "  unsigned long long x = (unsigned long long)i * 0x9E3779B97F4A7C15ull + (unsigned long long)(j + 1) * 0xC2B2AE3D27D4EB4Full;\n"
      << "  x ^= x >> 31; x *= 0xBF58476D1CE4E5B9ull; x ^= x >> 29;\n"
      << "  const float u = (float)(x >> 40) * (1.0f / 16777216.0f);\n"
      << "  return exp2f(-26.575f + 39.863f * u);\n"
      << "}\n";
    // the sparse scatter, in reaction order (reactants then products)
    auto scatter = [&](const char* T) {
        std::ostringstream b;
        for (int s = 0; s < S; ++s) b << "    " << T << " a" << s << " = 0;\n";
        for (int j = 0; j < R; ++j) {
            b << "    { const " << T << " q = r[" << j << "] * sc;";
            for (int q = 0; q < n.n_reac[j]; ++q) b << " a" << (int)n.reac[j][q] << " -= q;";
            for (int q = 0; q < n.n_prod[j]; ++q) b << " a" << (int)n.prod[j][q] << " += q;";
            b << " }\n";
        }
        for (int s = 0; s < S; ++s) b << "    f[" << s << "] = a" << s << ";\n";
        return b.str();
    };
    o << "}  // namespace\n";
    // variant 0: FP32 sparse
    // (every repetition's results go into a stored checksum, so none can be
    // dropped as dead code; both variants add the same 13 terms per repetition)
    o << "extern \"C\" __global__ void __launch_bounds__(128) k_stoich_sparse(long long nsys, int reps, float* out, float* chk) {\n"
      << "  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n"
      << "  if (i >= nsys) return;\n"
      << "  float r[R], f[S], c = 0.0f;\n"
      << "  for (int j = 0; j < R; ++j) r[j] = rate(i, j);\n"
      << "  for (int s = 0; s < S; ++s) f[s] = 0.0f;\n"
      << "  for (int rep = 0; rep < reps; ++rep) {\n"
      << "    const float sc = 1.0f + (float)rep * 1e-7f;\n"
      << scatter("float")
      << "    for (int s = 0; s < S; ++s) c += f[s];\n"
      << "  }\n"
      << "  for (int s = 0; s < S; ++s) out[i * S + s] = f[s];\n"
      << "  chk[i] = c;\n"
      << "}\n";
    // variant 2: FP64 sparse reference, the last repetition's scale
    o << "extern \"C\" __global__ void __launch_bounds__(128) k_stoich_ref(long long nsys, int reps, double* out, double* mag) {\n"
      << "  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n"
      << "  if (i >= nsys) return;\n"
      << "  double r[R], f[S];\n"
      << "  for (int j = 0; j < R; ++j) r[j] = (double)rate(i, j);\n"
      << "  const double sc = (double)(1.0f + (float)(reps - 1) * 1e-7f);\n"
      << "  {\n" << scatter("double") << "  }\n"
      << "  for (int s = 0; s < S; ++s) out[i * S + s] = f[s];\n";
    // sum of |terms| per species over every reactant and product occurrence
    // (the sums the sparse form and the oracle accumulate): the scale of the
    // FP32 rounding of either form
    o << "  double m[S];\n  for (int s = 0; s < S; ++s) m[s] = 0.0;\n";
    for (int j = 0; j < R; ++j) {
        for (int q = 0; q < n.n_reac[j]; ++q) o << "  m[" << (int)n.reac[j][q] << "] += fabs(r[" << j << "] * sc);\n";
        for (int q = 0; q < n.n_prod[j]; ++q) o << "  m[" << (int)n.prod[j][q] << "] += fabs(r[" << j << "] * sc);\n";
    }
    o << "  for (int s = 0; s < S; ++s) mag[i * S + s] = m[s];\n"
      << "}\n";
    // variant 1: warp-level TF32 tensor-core product
    const int KT = (R + 7) / 8, NT = (S + 7) / 8;  // k-steps of 8 reactions, n-tiles of 8 species
    o << "constexpr int KT = " << KT << ", NT = " << NT << ", RP = " << (8 * KT + 4) << ", FP = " << (8 * NT + 1)
      << ";\n"
      << "__constant__ float kN[" << 8 * KT << "][" << 8 * NT << "] = {\n";
    for (int j = 0; j < 8 * KT; ++j) {
        o << "  {";
        for (int s = 0; s < 8 * NT; ++s) o << (j < R && s < S ? coef(n, j, s) : 0) << (s + 1 < 8 * NT ? ", " : "");
        o << "}" << (j + 1 < 8 * KT ? "," : "") << "\n";
    }
    o << "};\n"
      << "__device__ __forceinline__ unsigned tf32(float x) { unsigned t; asm(\"cvt.rna.tf32.f32 %0, %1;\" : \"=r\"(t) : \"f\"(x)); return t; }\n"
      << "__device__ __forceinline__ void mma(float* d, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0, unsigned b1) {\n"
      << "  asm volatile(\"mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\"\n"
      << "               : \"+f\"(d[0]), \"+f\"(d[1]), \"+f\"(d[2]), \"+f\"(d[3])\n"
      << "               : \"r\"(a0), \"r\"(a1), \"r\"(a2), \"r\"(a3), \"r\"(b0), \"r\"(b1));\n"
      << "}\n"
      << "extern \"C\" __global__ void __launch_bounds__(128) k_stoich_tc(long long nsys, int reps, float* out, float* chk) {\n"
      << "  __shared__ float sr[4][32][RP];\n"
      << "  __shared__ float sf[4][32][FP];\n"
      << "  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;\n"
      << "  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // nsys: a multiple of 128\n"
      << "  float r[R], f[S], c = 0.0f;\n"
      << "  for (int j = 0; j < R; ++j) r[j] = rate(i, j);\n"
      << "  for (int j = R; j < 8 * KT; ++j) sr[w][lane][j] = 0.0f;\n"
      << "  for (int s = 0; s < S; ++s) f[s] = 0.0f;\n"
      // B fragments: row (reaction) tig / tig + 4 of k-step ks, column (species) gid of n-tile nt
      << "  unsigned b[NT][KT][2];\n"
      << "  for (int nt = 0; nt < NT; ++nt)\n"
      << "    for (int ks = 0; ks < KT; ++ks) {\n"
      << "      b[nt][ks][0] = tf32(kN[8 * ks + tig][8 * nt + gid]);\n"
      << "      b[nt][ks][1] = tf32(kN[8 * ks + tig + 4][8 * nt + gid]);\n"
      << "    }\n"
      << "  for (int rep = 0; rep < reps; ++rep) {\n"
      << "    const float sc = 1.0f + (float)rep * 1e-7f;\n"
      << "    for (int j = 0; j < R; ++j) sr[w][lane][j] = r[j] * sc;\n"
      << "    __syncwarp();\n"
      << "    float d[2][NT][4];\n"
      << "    for (int mt = 0; mt < 2; ++mt) for (int nt = 0; nt < NT; ++nt) for (int q = 0; q < 4; ++q) d[mt][nt][q] = 0.0f;\n"
      << "    for (int ks = 0; ks < KT; ++ks)\n"
      << "      for (int mt = 0; mt < 2; ++mt) {\n"
      << "        const int r0 = 16 * mt + gid, c0 = 8 * ks + tig;\n"
      << "        const float x0 = sr[w][r0][c0], x1 = sr[w][r0 + 8][c0], x2 = sr[w][r0][c0 + 4], x3 = sr[w][r0 + 8][c0 + 4];\n"
      << "        const unsigned h0 = tf32(x0), h1 = tf32(x1), h2 = tf32(x2), h3 = tf32(x3);\n"
      << "        const unsigned l0 = tf32(x0 - __uint_as_float(h0)), l1 = tf32(x1 - __uint_as_float(h1));\n"
      << "        const unsigned l2 = tf32(x2 - __uint_as_float(h2)), l3 = tf32(x3 - __uint_as_float(h3));\n"
      << "        for (int nt = 0; nt < NT; ++nt) {\n"
      << "          mma(d[mt][nt], l0, l1, l2, l3, b[nt][ks][0], b[nt][ks][1]);\n"
      << "          mma(d[mt][nt], h0, h1, h2, h3, b[nt][ks][0], b[nt][ks][1]);\n"
      << "        }\n"
      << "      }\n"
      // accumulator fragments: rows gid / gid + 8 of the m-tile, columns 2 tig, 2 tig + 1 of the n-tile
      << "    for (int mt = 0; mt < 2; ++mt)\n"
      << "      for (int nt = 0; nt < NT; ++nt) {\n"
      << "        const int r0 = 16 * mt + gid, c0 = 8 * nt + 2 * tig;\n"
      << "        sf[w][r0][c0] = d[mt][nt][0]; sf[w][r0][c0 + 1] = d[mt][nt][1];\n"
      << "        sf[w][r0 + 8][c0] = d[mt][nt][2]; sf[w][r0 + 8][c0 + 1] = d[mt][nt][3];\n"
      << "      }\n"
      << "    __syncwarp();\n"
      << "    for (int s = 0; s < S; ++s) f[s] = sf[w][lane][s];\n"
      << "    for (int s = 0; s < S; ++s) c += f[s];\n"
      << "    __syncwarp();\n"
      << "  }\n"
      << "  for (int s = 0; s < S; ++s) out[i * S + s] = f[s];\n"
      << "  chk[i] = c;\n"
      << "}\n";
    return o.str();
}

}  // namespace

extern "C" int bode_stoich_bench(int32_t rhs_handle, int32_t variant, int64_t nsys, int32_t reps, double* ms,
                                 double* max_err) {
    clear_last_error();
    RhsEntry r;
    if (!registry_lookup(rhs_handle, &r)) return fail(ODE_ERR_HANDLE, "unknown rhs handle");
    if (r.kind != ODE_RHS_MASSACTION) return fail(ODE_ERR_ARG, "the stoichiometry product needs a mass-action network");
    if (variant < 0 || variant > 1) return fail(ODE_ERR_ARG, "variant must be 0 (sparse FP32) or 1 (TF32 tensor cores)");
    if (nsys < 128 || nsys % 128 || nsys > ((int64_t)1 << 26) || reps < 0 || reps > 100000 || !ms)
        return fail(ODE_ERR_ARG, "need 128 <= nsys <= 2^26, a multiple of 128, 0 <= reps <= 100000");
    if (r.net.n_species > 16 || r.net.n_reactions > 32)
        return fail(ODE_ERR_UNSUPPORTED, "the product kernels take up to 16 species and 32 reactions");
    std::vector<cudaKernel_t> k;
    std::string why;
    int rc = jit_program(program(r.net), {"k_stoich_sparse", "k_stoich_tc", "k_stoich_ref"}, &k, &why);
    if (rc) return fail(rc, why);
    const int S = r.net.n_species;
    float *out = nullptr, *chk = nullptr;
    double *ref = nullptr, *mag = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(float) * S * nsys);
    if (e == cudaSuccess) e = cudaMalloc(&chk, sizeof(float) * nsys);
    if (e == cudaSuccess) e = cudaMalloc(&ref, sizeof(double) * S * nsys);
    if (e == cudaSuccess) e = cudaMalloc(&mag, sizeof(double) * S * nsys);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const unsigned grid = (unsigned)(nsys / 128);
    cudaKernel_t kv = variant == 0 ? k[0] : k[1];
    long long n = nsys;
    int reps_run = reps;
    void* args[] = {&n, &reps_run, &out, &chk};
    float t = 0.0f;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // pass 0 warms up
        e = cudaEventRecord(e0);
        if (e == cudaSuccess) e = cudaLaunchKernel((const void*)kv, dim3(grid), dim3(128), args, 0, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    }
    if (e == cudaSuccess) *ms = t;
    if (e == cudaSuccess && max_err && reps > 0) {
        // FP64 reference of the last repetition, error relative to the sum
        // of |terms| of each species (the scale the sums round at)
        void* rargs[] = {&n, &reps_run, &ref, &mag};
        e = cudaLaunchKernel((const void*)k[2], dim3(grid), dim3(128), rargs, 0, nullptr);
        std::vector<float> hf(S * nsys);
        std::vector<double> hr(S * nsys), hm(S * nsys);
        if (e == cudaSuccess) e = cudaMemcpy(hf.data(), out, sizeof(float) * S * nsys, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(hr.data(), ref, sizeof(double) * S * nsys, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(hm.data(), mag, sizeof(double) * S * nsys, cudaMemcpyDeviceToHost);
        double worst = 0.0;
        for (size_t q = 0; q < hf.size() && e == cudaSuccess; ++q)
            if (hm[q] > 0.0) worst = std::fmax(worst, std::fabs((double)hf[q] - hr[q]) / hm[q]);
        *max_err = worst;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(chk);
    cudaFree(ref);
    cudaFree(mag);
    if (e != cudaSuccess) return fail(ODE_ERR_CUDA, std::string("stoichiometry product bench: ") + cudaGetErrorString(e));
    return ODE_OK;
}
