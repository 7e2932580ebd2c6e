// jit.cu -- run-time specialisation of the integrator kernels for a
// registered mass-action network.
//
// The generic mass-action kernels read the network from kernel parameters,
// so every species index is a run-time value and the state vector must be
// addressed through local memory.  Here the network is written out as
// straight-line device code (one statement per rate product and per
// accumulation, in the order the reactions list them), compiled with NVRTC
// together with the integrator templates, and loaded as a CUDA library:
// every index is then a compile-time constant and the state stays in
// registers.  NVRTC is resolved with dlopen at first use, so the library
// has no link-time dependency on it; compiled kernels are cached per device
// in memory and as cubins on disk (BATCHODE_CACHE_DIR, else
// $HOME/.cache/batchode).
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "jit.h"

namespace bode {
namespace {

#include "jit_sources.inc"  // kJitHeaderNames / kJitHeaderSources / kJitHeaderCount (generated)

// Stand-ins for the host headers the device headers include.
const char* const kStubNames[] = {"cstdint", "stdint.h", "cmath", "cuda_runtime.h"};
const char* const kStubSources[] = {
    "#pragma once\ntypedef signed char int8_t; typedef short int16_t; typedef int int32_t;\n"
    "typedef long long int64_t; typedef unsigned char uint8_t; typedef unsigned short uint16_t;\n"
    "typedef unsigned int uint32_t; typedef unsigned long long uint64_t;\n",
    "#pragma once\n#include <cstdint>\n",
    "#pragma once\n#define INFINITY (__int_as_float(0x7f800000))\n#define NAN (__int_as_float(0x7fffffff))\n",
    "#pragma once\n",
};

struct Nvrtc {
    bool ok = false;
    std::string why;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcAddNameExpression) add_name = nullptr;
    decltype(&nvrtcGetLoweredName) lowered = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) errstr = nullptr;
};

Nvrtc load_nvrtc() {
    Nvrtc n;
    std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
    for (const char* env : {"CUDA_HOME", "CUDA_PATH"}) {
        const char* p = getenv(env);
        if (p) names.push_back(std::string(p) + "/lib64/libnvrtc.so.13");
    }
    names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    void* h = nullptr;
    for (const auto& name : names)
        if ((h = dlopen(name.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
        n.why = "libnvrtc.so.13 not found";
        return n;
    }
#define BODE_SYM(field, sym)                                          \
    n.field = reinterpret_cast<decltype(n.field)>(dlsym(h, #sym));    \
    if (!n.field) {                                                   \
        n.why = "missing symbol " #sym;                               \
        return n;                                                     \
    }
    BODE_SYM(create, nvrtcCreateProgram)
    BODE_SYM(compile, nvrtcCompileProgram)
    BODE_SYM(log_size, nvrtcGetProgramLogSize)
    BODE_SYM(log, nvrtcGetProgramLog)
    BODE_SYM(cubin_size, nvrtcGetCUBINSize)
    BODE_SYM(cubin, nvrtcGetCUBIN)
    BODE_SYM(add_name, nvrtcAddNameExpression)
    BODE_SYM(lowered, nvrtcGetLoweredName)
    BODE_SYM(destroy, nvrtcDestroyProgram)
    BODE_SYM(errstr, nvrtcGetErrorString)
#undef BODE_SYM
    n.ok = true;
    return n;
}

Nvrtc& nvrtc() {
    static Nvrtc n = load_nvrtc();
    return n;
}

// Resident blocks of 128 threads per SM the generated kernels are compiled
// for (a register budget of 65536 / (128 n) per thread).  Measured on the
// 13-species network: the mixed forms run best at 3 (168 registers; 2 and
// 4 are slower), the plain FP64 form at 2 (its FP64 state spills at 168
// registers); the two-float forms, with their rate constants and d_{j-2} in
// shared memory, at 3 (168 registers, ~130 B spilled).  BATCHODE_JIT_MINBLOCKS overrides both (1 = no budget).
int jit_min_blocks(int prec) {
    const int def = prec == ODE_PREC_FP64 ? 2 : 3;
    const char* v = getenv("BATCHODE_JIT_MINBLOCKS");
    const int n = v ? atoi(v) : def;
    return n >= 1 && n <= 16 ? n : def;
}

// Block lockstep of the generated one-launch kernels (BODE_LOCKSTEP in
// kernels.cuh): the two-float forms take 2, the block-wide step-end hold.
// Their evaluation and step code is several times the FP32 forms' and the
// kernel waits on instruction fetch; with the hold, the four warps of a
// block run the same phase of the step at the same time.  Measured per
// 1M-system mass-action step, results bit-identical: two-float with FP32
// scalars 156.5 -> 133.0 ms (cost-ordered) and 207 -> 184 ms (unordered);
// with FP64 bookkeeping 229 -> 210 ms.  The FP32 forms lose with it (lean
// 40.4 -> 42.2 ms, the specified split 121 -> 126 ms) and FP64 is
// unchanged, so they keep 0.  BATCHODE_JIT_LOCKSTEP (0-2) overrides.
int jit_lockstep(int prec) {
    const int def = prec_is_f2(prec) ? 2 : 0;
    const char* v = getenv("BATCHODE_JIT_LOCKSTEP");
    const int n = v ? atoi(v) : def;
    return n >= 0 && n <= 2 ? n : def;
}

std::string lit(double x) {
    char buf[64];
    snprintf(buf, sizeof(buf), "%.17g", x);
    std::string s(buf);
    if (s.find_first_of(".eEn") == std::string::npos) s += ".0";
    return "(" + s + ")";
}

// The network as a Model (see rhs.cuh for the interface): rate constants in
// registers, f written as straight-line code whose per-species accumulation
// order is the reaction order (reactants, then products).
std::string model_source(const RhsEntry& r) {
    const MassActionNet& net = r.net;
    const int S = net.n_species, NR = net.n_reactions;
    std::ostringstream o;
    o << "struct JitMass {\n"
      << "  static constexpr int W = 1, PER = " << S << ";\n"
      << "  using Ctx = bode::NoCtx;\n"
      << "  template <class R> struct Sys {\n"
      << "    bode::ConstStore<R, " << NR << "> k;  // registers, or a shared-memory row (two-float forms)\n"
      << "    static constexpr int CONST_SMEM = bode::ConstStore<R, " << NR << ">::SMEM_FLOATS;\n"
      << "    __device__ void bind_consts(float* row) { k.bind(row); }\n"
      << "    int n;\n"
      << "    __device__ static double clip(double k) { return fmin(fmax(k, " << lit(net.kmin) << "), " << lit(net.kmax)
      << "); }\n"
      << "    __device__ void load(const Ctx&, const bode::Team<1>&, double T, int neq) {\n"
      << "      n = neq;\n"
      << "      if constexpr (sizeof(R) == 8) {\n"
      << "        const double lnT = bode::xm::log_series(T);\n";
    for (int j = 0; j < NR; ++j)
        o << "        k[" << j << "] = clip(bode::xm::exp_series(bode::xm::kLn10 * " << lit(net.log10A[j]) << " + "
          << lit(net.beta[j]) << " * lnT - " << lit(net.Ea[j]) << " / T));\n";
    o << "      } else {\n"
      << "        const double lnT = log(T), invT = 1.0 / T;\n";
    for (int j = 0; j < NR; ++j)
        o << "        { const double l2 = (2.302585092994046 * " << lit(net.log10A[j]) << " + " << lit(net.beta[j])
          << " * lnT - " << lit(net.Ea[j]) << " * invT) * 1.4426950408889634; const double li = floor(l2);"
          << " k[" << j << "] = (R)clip((double)ldexpf(exp2f((float)(l2 - li)), (int)li)); }\n";
    o << "      }\n"
      << "    }\n"
      // the two-float forms read the constants that bode_jit_rates wrote
      // (the same FP64 series, once per system, in a kernel of its own):
      // a system's set-up then runs no series, which matters in the work
      // queue, where set-ups interleave with the evaluation loop and their
      // code would push the loop's out of the instruction cache
      << "    static constexpr bool kPreConsts = true;\n"
      << "    __device__ void load_pre(const bode::F2* tab, long long i, long long stride, int neq) {\n"
      << "      n = neq;\n"
      << "      if constexpr (bode::ConstStore<R, " << NR << ">::SMEM_FLOATS > 0)\n"
      << "        for (int j = 0; j < " << NR << "; ++j) k[j] = tab[(long long)j * stride + i];\n"
      << "    }\n"
      << "    __device__ int comp(const bode::Team<1>&, int s) const { return s; }\n"
      << "    template <class T> __device__ T ordered_sum(const bode::Team<1>&, const T* x) const {\n"
      << "      T acc = T(0);\n";
    for (int s = 0; s < S; ++s) o << "      acc = acc + x[" << s << "];\n";
    o << "      return acc;\n"
      << "    }\n"
      << "    __device__ void rhs(const bode::Team<1>&, R, const R* y, R* f) const {\n";
    // each species' accumulator starts from its first term (0 - r or 0 + r,
    // the values an accumulator started at zero takes); the products and
    // sums go through the lazy two-float forms (the plain operations for
    // float and double), normalised once per species at the end
    std::vector<int> seen(S, 0);
    for (int s = 0; s < S; ++s) o << "      R a" << s << ";\n";
    for (int j = 0; j < NR; ++j) {
        o << "      { R r = k[" << j << "];";
        for (int q = 0; q < net.n_reac[j]; ++q) o << " r = bode::mul_lazy(r, y[" << (int)net.reac[j][q] << "]);";
        for (int q = 0; q < net.n_reac[j]; ++q) {
            const int sp = net.reac[j][q];
            if (!seen[sp])
                o << " a" << sp << " = bode::acc_first_sub(r);";
            else
                o << " a" << sp << " = bode::acc_sub(a" << sp << ", r);";
            seen[sp] = 1;
        }
        for (int q = 0; q < net.n_prod[j]; ++q) {
            const int sp = net.prod[j][q];
            if (!seen[sp])
                o << " a" << sp << " = bode::acc_first_add(r);";
            else
                o << " a" << sp << " = bode::acc_add(a" << sp << ", r);";
            seen[sp] = 1;
        }
        o << " }\n";
    }
    for (int s = 0; s < S; ++s)
        if (!seen[s]) o << "      a" << s << " = R(0);\n";
    for (int s = 0; s < S; ++s) o << "      f[" << s << "] = bode::acc_value(a" << s << ");\n";
    o << "    }\n";
    // Gershgorin bound, row by row: J_sl accumulates reaction by reaction
    // -dr_j/dC_l per reactant occurrence of s, +dr_j/dC_l per product
    // occurrence, dr_j/dC_l summed over the reactant occurrences of l; the
    // row sum runs over the touched columns in increasing order
    o << "    __device__ R gershgorin(const bode::Team<1>&, const R* y) const {\n"
      << "      R g = R(0);\n";
    for (int s = 0; s < S; ++s) {
        std::vector<int> touched(S, 0);
        std::ostringstream body;
        for (int j = 0; j < NR; ++j) {
            const int nr = net.n_reac[j];
            int occ = 0, pocc = 0;
            for (int q = 0; q < nr; ++q) occ += net.reac[j][q] == s;
            for (int q = 0; q < net.n_prod[j]; ++q) pocc += net.prod[j][q] == s;
            if (!occ && !pocc) continue;
            body << "        {";
            if (nr == 1)
                body << " const R d0 = k[" << j << "];";
            else
                body << " const R d0 = k[" << j << "] * y[" << (int)net.reac[j][1] << "]; const R d1 = k[" << j
                     << "] * y[" << (int)net.reac[j][0] << "];";
            for (int l = 0; l < S; ++l) {
                bool any = false;
                for (int q = 0; q < nr; ++q) any = any || net.reac[j][q] == l;
                if (!any) continue;
                touched[l] = 1;
                body << " { R dl = R(0);";
                for (int q = 0; q < nr; ++q)
                    if (net.reac[j][q] == l) body << " dl = dl + d" << q << ";";
                for (int q = 0; q < occ; ++q) body << " J" << l << " = J" << l << " - dl;";
                for (int q = 0; q < pocc; ++q) body << " J" << l << " = J" << l << " + dl;";
                body << " }";
            }
            body << " }\n";
        }
        o << "      {\n";
        for (int l = 0; l < S; ++l)
            if (touched[l]) o << "        R J" << l << " = R(0);\n";
        o << body.str() << "        R acc = R(0);";
        for (int l = 0; l < S; ++l)
            if (touched[l]) o << " acc = acc + bode::rabs(J" << l << ");";
        o << "\n        g = bode::rmax(g, acc);\n"
          << "      }\n";
    }
    o << "      return g;\n"
      << "    }\n"
      << "  };\n"
      << "};\n";
    // every system's rate constants from its temperature params[i] as
    // two-float pairs, reaction-major (out[j * nsys + i]); the expression of
    // the FP64 branch of load() above
    o << "extern \"C\" __global__ void bode_jit_rates(const double* __restrict__ Tv, long long nsys,\n"
      << "                                             bode::F2* __restrict__ out) {\n"
      << "  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n"
      << "  if (i >= nsys) return;\n"
      << "  using S = JitMass::Sys<bode::F2>;\n"
      << "  const double T = Tv[i];\n"
      << "  const double lnT = bode::xm::log_series(T);\n";
    for (int j = 0; j < NR; ++j)
        o << "  out[" << j << "LL * nsys + i] = bode::F2(S::clip(bode::xm::exp_series(bode::xm::kLn10 * "
          << lit(net.log10A[j]) << " + " << lit(net.beta[j]) << " * lnT - " << lit(net.Ea[j]) << " / T)));\n";
    o << "}\n";
    return o.str();
}

uint64_t fnv1a(const std::string& s) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : s) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

std::string cache_dir() {
    const char* d = getenv("BATCHODE_CACHE_DIR");
    if (d && *d) return d;
    const char* home = getenv("HOME");
    if (!home || !*home) return "";
    std::string base = std::string(home) + "/.cache";
    mkdir(base.c_str(), 0755);
    return base + "/batchode";
}

bool read_file(const std::string& path, std::vector<char>* out) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    out->assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
    return !out->empty();
}

void write_file(const std::string& dir, const std::string& path, const std::vector<char>& data) {
    if (dir.empty()) return;
    mkdir(dir.c_str(), 0755);
    const std::string tmp = path + ".tmp" + std::to_string(getpid());
    {
        std::ofstream f(tmp, std::ios::binary);
        if (!f) return;
        f.write(data.data(), (std::streamsize)data.size());
    }
    rename(tmp.c_str(), path.c_str());
}

struct JitKernels {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kstatic = nullptr, kqueue = nullptr, krates = nullptr;
    int smem_floats = 0;  // dynamic shared memory per thread, as the integrator declares it
};

std::mutex g_jit_mu;
std::map<std::string, JitKernels> g_cache;  // key: device + source hash + form

// net: the two-float variant with the warp-level code (work queue, in-kernel
// network); the other forms have one variant
std::string method_type(int method, int prec, bool net) {
    const std::string nv = net ? "true" : "false";
    if (prec == ODE_PREC_F2) return "bode::RkcF2<JitMass, true, " + nv + ">";
    if (prec == ODE_PREC_F2_LEAN) return "bode::RkcF2<JitMass, false, " + nv + ">";
    if (method == kMethodRkck)
        return prec == ODE_PREC_FP64 ? "bode::RkckF64<JitMass>"
               : prec == ODE_PREC_MIXED ? "bode::RkckMixed<JitMass, true>" : "bode::RkckMixed<JitMass, false>";
    if (prec == ODE_PREC_FP64) return "bode::RkcF64<JitMass>";
    return prec == ODE_PREC_MIXED ? "bode::RkcMixed<JitMass, true>" : "bode::RkcMixed<JitMass, false>";
}

struct JitImage {
    std::string low_static, low_queue;
    std::vector<char> cubin;
};

int compile_image(const RhsEntry& r, int method, int prec, bool net, JitImage* img, std::string* err) {
    const std::string model = model_source(r);
    const std::string meth = method_type(method, prec, net);
    const std::string nstatic = "bode::k_static<" + meth + ", bode::NoCtx>";
    const std::string nqueue = "bode::k_queue<" + meth + ", bode::NoCtx>";
    // the two kernels are instantiated through their name expressions
    // the module also exports the integrator's shared-memory need per thread,
    // which the launcher reads back instead of restating the layout
    std::string src = "#include \"rhs.cuh\"\n#include \"integrators.cuh\"\n#include \"kernels.cuh\"\n" + model +
                      "extern \"C\" __device__ const int bode_jit_smem_floats = " + meth + "::SMEM_FLOATS;\n";
    std::vector<std::string> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo",
                                     prec == ODE_PREC_FP64 ? "--fmad=false" : "--fmad=true"};
    // occupancy tuning: blocks of at most 128 threads with a register budget
    // for BATCHODE_JIT_MINBLOCKS resident blocks per SM
    const int minb = jit_min_blocks(prec);
    if (minb > 1) {
        opts.push_back("-DBODE_MAX_THREADS=128");
        opts.push_back("-DBODE_MIN_BLOCKS=" + std::to_string(minb));
    }
    if (jit_lockstep(prec) > 0) opts.push_back("-DBODE_LOCKSTEP=" + std::to_string(jit_lockstep(prec)));
    const char* verbose = getenv("BATCHODE_JIT_VERBOSE");  // print the ptxas resource report
    if (verbose && *verbose == '1') opts.push_back("-Xptxas=-v");
    std::string key_text = src + "\n" + nstatic + "\n" + nqueue;
    for (const auto& o : opts) key_text += "\n" + o;
    for (int k = 0; k < kJitHeaderCount; ++k) key_text += kJitHeaderSources[k];
    char hash[32];
    snprintf(hash, sizeof(hash), "%016llx", (unsigned long long)fnv1a(key_text));
    const std::string dir = cache_dir();
    const std::string path = dir.empty() ? "" : dir + "/jit_" + hash + ".bin";

    // cached cubin: the two lowered names, then the image
    std::vector<char> blob;
    std::string& low_static = img->low_static;
    std::string& low_queue = img->low_queue;
    std::vector<char>& cubin = img->cubin;
    if (!path.empty() && read_file(path, &blob)) {
        const char* p = blob.data();
        const size_t n = blob.size();
        const size_t a = strnlen(p, n);
        if (a < n) {
            const size_t b = strnlen(p + a + 1, n - a - 1);
            if (a + 1 + b < n) {
                low_static.assign(p, a);
                low_queue.assign(p + a + 1, b);
                cubin.assign(p + a + b + 2, p + n);
            }
        }
    }
    if (cubin.empty()) {
        Nvrtc& nv = nvrtc();
        if (!nv.ok) {
            *err = "NVRTC unavailable: " + nv.why;
            return ODE_ERR_UNSUPPORTED;
        }
        std::vector<const char*> hnames, hsrcs;
        for (int k = 0; k < kJitHeaderCount; ++k) {
            hnames.push_back(kJitHeaderNames[k]);
            hsrcs.push_back(kJitHeaderSources[k]);
        }
        for (int k = 0; k < 4; ++k) {
            hnames.push_back(kStubNames[k]);
            hsrcs.push_back(kStubSources[k]);
        }
        nvrtcProgram prog;
        nvrtcResult rc = nv.create(&prog, src.c_str(), "jit_mass.cu", (int)hnames.size(), hsrcs.data(), hnames.data());
        if (rc != NVRTC_SUCCESS) {
            *err = std::string("nvrtcCreateProgram: ") + nv.errstr(rc);
            return ODE_ERR_UNSUPPORTED;
        }
        nv.add_name(prog, nstatic.c_str());
        nv.add_name(prog, nqueue.c_str());
        std::vector<const char*> copts;
        for (const auto& o : opts) copts.push_back(o.c_str());
        rc = nv.compile(prog, (int)copts.size(), copts.data());
        if (rc != NVRTC_SUCCESS) {
            size_t ls = 0;
            nv.log_size(prog, &ls);
            std::string logtxt(ls, '\0');
            nv.log(prog, &logtxt[0]);
            nv.destroy(&prog);
            *err = "NVRTC compile failed: " + logtxt.substr(0, 2000);
            return ODE_ERR_UNSUPPORTED;
        }
        if (verbose && *verbose == '1') {
            size_t ls = 0;
            nv.log_size(prog, &ls);
            std::string logtxt(ls, '\0');
            nv.log(prog, &logtxt[0]);
            fprintf(stderr, "%s\n", logtxt.c_str());
        }
        const char* l1 = nullptr;
        const char* l2 = nullptr;
        nv.lowered(prog, nstatic.c_str(), &l1);
        nv.lowered(prog, nqueue.c_str(), &l2);
        low_static = l1 ? l1 : "";
        low_queue = l2 ? l2 : "";
        size_t cs = 0;
        nv.cubin_size(prog, &cs);
        cubin.resize(cs);
        nv.cubin(prog, cubin.data());
        nv.destroy(&prog);
        if (!path.empty()) {
            std::vector<char> out(low_static.begin(), low_static.end());
            out.push_back('\0');
            out.insert(out.end(), low_queue.begin(), low_queue.end());
            out.push_back('\0');
            out.insert(out.end(), cubin.begin(), cubin.end());
            write_file(dir, path, out);
        }
    }
    return ODE_OK;
}

int load_image(const JitImage& img, JitKernels* out, std::string* err) {
    cudaError_t e = cudaLibraryLoadData(&out->lib, img.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&out->kstatic, out->lib, img.low_static.c_str());
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&out->kqueue, out->lib, img.low_queue.c_str());
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&out->krates, out->lib, "bode_jit_rates");
    void* dptr = nullptr;
    size_t bytes = 0;
    if (e == cudaSuccess) e = cudaLibraryGetGlobal(&dptr, &bytes, out->lib, "bode_jit_smem_floats");
    if (e == cudaSuccess && bytes != sizeof(int)) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaMemcpy(&out->smem_floats, dptr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && (out->smem_floats < 0 || out->smem_floats > 4096)) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        *err = std::string("loading generated kernels: ") + cudaGetErrorString(e);
        return ODE_ERR_CUDA;
    }
    return ODE_OK;
}

std::string cache_key(const RhsEntry& r, int method, int prec, bool net, int dev) {
    char key[128];
    snprintf(key, sizeof(key), "%d/%d/%d/%d/%016llx/%d/%d", dev, method, prec, (int)net,
             (unsigned long long)fnv1a(model_source(r)), jit_min_blocks(prec), jit_lockstep(prec));
    return key;
}

// whether a launch takes the two-float variant with the warp-level code
bool wants_net(int prec, const BatchArgs& a, int mapping) {
    return prec_is_f2(prec) && (a.mlp != nullptr || mapping == ODE_MAP_QUEUE);
}

// kernels for the current device, built and loaded at first use
int get_kernels(const RhsEntry& r, int method, int prec, bool net, JitKernels* k, std::string* err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return ODE_ERR_CUDA;
    }
    const std::string key = cache_key(r, method, prec, net, dev);
    std::lock_guard<std::mutex> lk(g_jit_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *k = it->second;
        return ODE_OK;
    }
    JitImage img;
    int rc = compile_image(r, method, prec, net, &img, err);
    if (rc == ODE_OK) rc = load_image(img, k, err);
    if (rc == ODE_OK) g_cache[key] = *k;
    return rc;
}

// Compiles a stand-alone device program (the library's device headers
// available) for sm_103a and loads it on the current device; kernels by
// name expression.  Cached in memory per device and source.
struct JitProgram {
    cudaLibrary_t lib = nullptr;
    std::vector<cudaKernel_t> kernels;
};
std::map<std::string, JitProgram> g_programs;

int compile_program(const std::string& src, const std::vector<std::string>& names, JitProgram* out,
                    std::string* err) {
    Nvrtc& nv = nvrtc();
    if (!nv.ok) {
        *err = "NVRTC unavailable: " + nv.why;
        return ODE_ERR_UNSUPPORTED;
    }
    std::vector<const char*> hnames, hsrcs;
    for (int k = 0; k < kJitHeaderCount; ++k) {
        hnames.push_back(kJitHeaderNames[k]);
        hsrcs.push_back(kJitHeaderSources[k]);
    }
    for (int k = 0; k < 4; ++k) {
        hnames.push_back(kStubNames[k]);
        hsrcs.push_back(kStubSources[k]);
    }
    nvrtcProgram prog;
    nvrtcResult rc = nv.create(&prog, src.c_str(), "jit_program.cu", (int)hnames.size(), hsrcs.data(), hnames.data());
    if (rc != NVRTC_SUCCESS) {
        *err = std::string("nvrtcCreateProgram: ") + nv.errstr(rc);
        return ODE_ERR_UNSUPPORTED;
    }
    for (const auto& n : names) nv.add_name(prog, n.c_str());
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo"};
    rc = nv.compile(prog, 3, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t ls = 0;
        nv.log_size(prog, &ls);
        std::string logtxt(ls, '\0');
        nv.log(prog, &logtxt[0]);
        nv.destroy(&prog);
        *err = "NVRTC compile failed: " + logtxt.substr(0, 2000);
        return ODE_ERR_UNSUPPORTED;
    }
    std::vector<std::string> lowered;
    for (const auto& n : names) {
        const char* l = nullptr;
        nv.lowered(prog, n.c_str(), &l);
        lowered.push_back(l ? l : "");
    }
    size_t cs = 0;
    nv.cubin_size(prog, &cs);
    std::vector<char> cubin(cs);
    nv.cubin(prog, cubin.data());
    nv.destroy(&prog);
    cudaError_t e = cudaLibraryLoadData(&out->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    out->kernels.assign(names.size(), nullptr);
    for (size_t k = 0; k < names.size() && e == cudaSuccess; ++k)
        e = cudaLibraryGetKernel(&out->kernels[k], out->lib, lowered[k].c_str());
    if (e != cudaSuccess) {
        *err = std::string("loading a generated program: ") + cudaGetErrorString(e);
        return ODE_ERR_CUDA;
    }
    return ODE_OK;
}

}  // namespace

int jit_max_block(int prec) { return jit_min_blocks(prec) > 1 ? 128 : 256; }

int jit_program(const std::string& src, const std::vector<std::string>& names, std::vector<cudaKernel_t>* kernels,
                std::string* err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return ODE_ERR_CUDA;
    }
    std::string key = std::to_string(dev) + "/" + std::to_string(fnv1a(src));
    for (const auto& n : names) key += "/" + n;
    std::lock_guard<std::mutex> lk(g_jit_mu);
    auto it = g_programs.find(key);
    if (it == g_programs.end()) {
        JitProgram p;
        const int rc = compile_program(src, names, &p, err);
        if (rc) return rc;
        it = g_programs.emplace(key, p).first;
    }
    *kernels = it->second.kernels;
    return ODE_OK;
}

bool jit_available() { return nvrtc().ok; }

int jit_prepare(const RhsEntry& r, int method, int prec, std::string* err) {
    int ndev = 0;
    // the two-float forms in both variants (the work queue and the in-kernel
    // network take the one with the warp-level code)
    const int variants = prec_is_f2(prec) ? 2 : 1;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();  // clear the no-device error
        for (int v = 0; v < variants; ++v) {
            JitImage img;
            const int rc = compile_image(r, method, prec, v == 1, &img, err);
            if (rc) return rc;
        }
        return ODE_OK;
    }
    for (int v = 0; v < variants; ++v) {
        JitKernels k;
        const int rc = get_kernels(r, method, prec, v == 1, &k, err);
        if (rc) return rc;
    }
    return ODE_OK;
}

int jit_rates(const RhsEntry& r, int method, int prec, const double* T, int64_t nsys, void* out, cudaStream_t s,
              std::string* err) {
    JitKernels k;
    int rc = get_kernels(r, method, prec, false, &k, err);
    if (rc) return rc;
    if (nsys <= 0) return ODE_OK;
    long long n = (long long)nsys;
    void* params[] = {(void*)&T, &n, &out};
    const cudaError_t e = cudaLaunchKernel((const void*)k.krates, dim3((unsigned)((nsys + 255) / 256)), dim3(256), params, 0, s);
    if (e != cudaSuccess) {
        *err = std::string("rate-constant kernel launch: ") + cudaGetErrorString(e);
        return ODE_ERR_CUDA;
    }
    return ODE_OK;
}

int jit_launch(const RhsEntry& r, int method, int prec, const BatchArgs& a, const LaunchCfg& c, std::string* err) {
    JitKernels k;
    int rc = get_kernels(r, method, prec, wants_net(prec, a, c.mapping), &k, err);
    if (rc) return rc;
    NoCtx ctx;
    BatchArgs args = a;
    void* params[] = {&args, &ctx};
    const int block = c.block > jit_max_block(prec) ? jit_max_block(prec) : c.block;
    // the generated model is one thread per system with PER = species count
    const size_t smem = sizeof(float) * (size_t)k.smem_floats * (size_t)block;
    const int64_t threads = a.nsys;  // one thread per system
    cudaError_t e;
    if (smem > 48 * 1024) {  // above the default dynamic shared-memory limit: opt in
        e = cudaFuncSetAttribute((const void*)k.kstatic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)k.kqueue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            *err = std::string("shared-memory opt-in: ") + cudaGetErrorString(e);
            return ODE_ERR_CUDA;
        }
    }
    if (c.mapping == ODE_MAP_QUEUE) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k.kqueue, block, smem);
        if (e != cudaSuccess) {
            *err = std::string("occupancy query: ") + cudaGetErrorString(e);
            return ODE_ERR_CUDA;
        }
        if (per_sm < 1) per_sm = 1;
        int64_t grid = (int64_t)per_sm * c.sm_count;
        const int64_t need = (threads + block - 1) / block;
        if (grid > need) grid = need;
        args.warp_sched = 1;
        e = cudaLaunchKernel((const void*)k.kqueue, dim3((unsigned)grid), dim3(block), params, smem, c.stream);
    } else {
        const int64_t grid = (threads + block - 1) / block;
        e = cudaLaunchKernel((const void*)k.kstatic, dim3((unsigned)grid), dim3(block), params, smem, c.stream);
    }
    if (e != cudaSuccess) {
        *err = std::string("generated kernel launch: ") + cudaGetErrorString(e);
        return ODE_ERR_CUDA;
    }
    return ODE_OK;
}

std::string jit_model_source(const RhsEntry& r) { return model_source(r); }

}  // namespace bode
