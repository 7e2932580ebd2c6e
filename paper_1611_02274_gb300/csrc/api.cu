// api.cu -- the C ABI (include/batchode.h): RHS registry, argument
// validation, workspace, host-buffer staging and kernel dispatch.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>
#include <algorithm>

#include "batchode.h"
#include "jit.h"
#include "launch.cuh"
#include "order.h"

using namespace bode;

namespace bode {
int mlp_packed_for(int32_t handle, int n_in, const MlpPacked** out);  // mlp.cu
}  // namespace bode

namespace {

thread_local std::string g_err;
std::mutex g_mu;
std::map<int32_t, RhsEntry> g_reg;
int32_t g_next_handle = 1;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(ODE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Per-device workspace: a ring of queue cursors and a grow-only staging
// buffer for host-pointer calls.
constexpr int kCursorRing = 1024;
constexpr int kRkcTabMax = 256;  // stage counts with tabulated coefficients
struct Workspace {
    unsigned long long* cursors = nullptr;  // kCursorRing + 1: the last one for tuning runs
    int next_cursor = 0;
    double* tune_y = nullptr;  // output of mapping-tuning runs, grow-only
    size_t tune_bytes = 0;
    // cost-ordering buffers per stream (grow-only): calls on one stream run
    // in order, calls on different streams get their own buffers
    struct OrderBuf {
        int32_t* bins = nullptr;
        int32_t* index = nullptr;
        int64_t cap = 0;
    };
    std::map<cudaStream_t, OrderBuf> order;
    // precomputed right-hand-side constants per stream (grow-only)
    struct ConstBuf {
        void* ptr = nullptr;
        size_t bytes = 0;
    };
    std::map<cudaStream_t, ConstBuf> consts;
    double* tab64 = nullptr;
    float4* tab32 = nullptr;
    void* stage = nullptr;
    size_t stage_bytes = 0;
    int sm_count = 0;
};
std::map<int, Workspace> g_ws;

int get_workspace(Workspace** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    Workspace& w = g_ws[dev];
    if (!w.cursors) {
        e = cudaMalloc(&w.cursors, sizeof(unsigned long long) * (kCursorRing + 1));
        if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "workspace allocation failed: %s", cudaGetErrorString(e));
        e = cudaDeviceGetAttribute(&w.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        const int entries = rkc_tab_index(kRkcTabMax + 1, 1);
        e = cudaMalloc(&w.tab64, sizeof(double) * 8 * entries);
        if (e == cudaSuccess) e = cudaMalloc(&w.tab32, sizeof(float4) * entries);
        if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "coefficient table allocation failed: %s", cudaGetErrorString(e));
        e = build_rkc_tables(w.tab64, w.tab32, kRkcTabMax, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "coefficient table build");
    }
    *out = &w;
    return ODE_OK;
}

int validate_desc(const ode_rhs_desc* d, RhsEntry* r) {
    if (!d) return fail(ODE_ERR_ARG, "desc is NULL");
    std::memset(r, 0, sizeof(*r));
    r->kind = d->kind;
    r->neq = d->neq;
    r->n_params = d->n_params;
    if (d->n_params != 1) return fail(ODE_ERR_ARG, "n_params must be 1 for every built-in family (got %d)", d->n_params);
    switch (d->kind) {
    case ODE_RHS_VDP:
        if (d->neq != 2) return fail(ODE_ERR_ARG, "van der Pol has neq 2 (got %d)", d->neq);
        return ODE_OK;
    case ODE_RHS_VDP_CHAIN:
        if (d->neq < 2 || d->neq > 128 || d->neq % 2) return fail(ODE_ERR_ARG, "chain neq must be even in [2, 128]");
        if (!std::isfinite(d->coupling)) return fail(ODE_ERR_ARG, "coupling must be finite");
        r->coupling = d->coupling;
        return ODE_OK;
    case ODE_RHS_BRUSS1D:
        if (d->neq < 2 || d->neq > 256 || d->neq % 2) return fail(ODE_ERR_ARG, "Brusselator neq must be even in [2, 256]");
        r->bruss_A = d->bruss_A;
        r->bruss_B = d->bruss_B;
        r->bruss_ubc = d->bruss_ubc;
        r->bruss_vbc = d->bruss_vbc;
        return ODE_OK;
    case ODE_RHS_KINETICS: {
        const int S = d->neq - 1, R = d->n_reactions;
        if (S < 1 || S > kKinMaxSpecies) return fail(ODE_ERR_ARG, "kinetics neq must be in [2, %d]", kKinMaxSpecies + 1);
        if (R < 1 || R > kKinMaxReactions) return fail(ODE_ERR_ARG, "kinetics reaction count must be in [1, %d]", kKinMaxReactions);
        if (!d->n_reac || !d->reac || !d->n_prod || !d->prod || !d->log10A || !d->beta || !d->Ea || !d->mol_weights ||
            !d->thermo)
            return fail(ODE_ERR_ARG, "kinetics mechanism arrays must be non-NULL");
        if (!(d->kmin > 0.0) || !(d->kmax >= d->kmin)) return fail(ODE_ERR_ARG, "need 0 < kmin <= kmax");
        for (int i = 0; i < S; ++i) {
            if (!(d->mol_weights[i] > 0.0) || !std::isfinite(d->mol_weights[i]))
                return fail(ODE_ERR_ARG, "species %d: molecular weight must be finite and > 0", i);
            for (int q = 0; q < 4; ++q)
                if (!std::isfinite(d->thermo[4 * i + q])) return fail(ODE_ERR_ARG, "species %d: non-finite thermo", i);
        }
        // incidence lists: per species, one packed word per occurrence
        // (kin_inc_word), j ascending, reactants first
        std::vector<std::vector<int>> inc(S);
        for (int j = 0; j < R; ++j) {
            const int nr = d->n_reac[j], np = d->n_prod[j];
            if (nr < 1 || nr > 2 || np < 1 || np > 2) return fail(ODE_ERR_ARG, "reaction %d: 1-2 reactants and products", j);
            if (!std::isfinite(d->log10A[j]) || !std::isfinite(d->beta[j]) || !std::isfinite(d->Ea[j]))
                return fail(ODE_ERR_ARG, "reaction %d: non-finite Arrhenius parameter", j);
            for (int q = 0; q < nr + np; ++q) {
                const int i = q < nr ? d->reac[2 * j + q] : d->prod[2 * j + q - nr];
                if (i < 0 || i >= S) return fail(ODE_ERR_ARG, "reaction %d: species index out of range", j);
            }
            const int r0 = d->reac[2 * j], r1 = nr == 2 ? d->reac[2 * j + 1] : kKinOne;
            for (int q = 0; q < nr; ++q) inc[d->reac[2 * j + q]].push_back(kin_inc_word(j, false, r0, r1));
            for (int q = 0; q < np; ++q) inc[d->prod[2 * j + q]].push_back(kin_inc_word(j, true, r0, r1));
        }
        std::vector<double> dv;
        dv.insert(dv.end(), d->mol_weights, d->mol_weights + S);
        dv.insert(dv.end(), d->thermo, d->thermo + 4 * S);
        dv.insert(dv.end(), d->log10A, d->log10A + R);
        dv.insert(dv.end(), d->beta, d->beta + R);
        dv.insert(dv.end(), d->Ea, d->Ea + R);
        if (dv.size() % 2) dv.push_back(0.0);  // the float4 section starts 16-byte aligned
        std::vector<float> fv;
        const double log2_10 = 3.321928094887362, log2_e = 1.4426950408889634, r_gas = 8.314462618;
        for (int j = 0; j < R; ++j) {
            fv.push_back((float)(log2_10 * d->log10A[j]));
            fv.push_back((float)d->beta[j]);
            fv.push_back((float)(log2_e * d->Ea[j]));
            fv.push_back(0.0f);
        }
        for (int i = 0; i < S; ++i) {
            for (int q = 0; q < 4; ++q) fv.push_back((float)d->thermo[4 * i + q]);
            fv.push_back((float)(r_gas / d->mol_weights[i]));
            fv.push_back((float)d->mol_weights[i]);
            fv.push_back((float)(1.0 / d->mol_weights[i]));
            fv.push_back(0.0f);
        }
        // omega schedule: species by descending list length, each to the
        // lane with the least work so far (ties: the lowest lane)
        std::vector<int> by_len(S);
        for (int i = 0; i < S; ++i) by_len[i] = i;
        std::stable_sort(by_len.begin(), by_len.end(),
                         [&](int x, int y) { return inc[x].size() > inc[y].size(); });
        std::vector<std::vector<int>> lane_sp(32);
        std::vector<size_t> load(32, 0);
        for (int i : by_len) {
            const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            lane_sp[l].push_back(i);
            load[l] += inc[i].size() + 1;  // the +1 keeps empty lists spread too
        }
        int sched_k = 0;
        for (const auto& v : lane_sp) sched_k = std::max(sched_k, (int)v.size());
        std::vector<int> iv;
        iv.push_back(0);
        for (int i = 0; i < S; ++i) iv.push_back(iv.back() + (int)inc[i].size());
        for (int i = 0; i < S; ++i) iv.insert(iv.end(), inc[i].begin(), inc[i].end());
        const size_t sched_pos = iv.size();
        for (int k = 0; k < sched_k; ++k)
            for (int l = 0; l < 32; ++l) iv.push_back(k < (int)lane_sp[l].size() ? lane_sp[l][k] : -1);
        const size_t dbytes = sizeof(double) * dv.size(), fbytes = sizeof(float) * fv.size(),
                     ibytes = sizeof(int) * iv.size();
        void* mem = nullptr;
        cudaError_t e = cudaMalloc(&mem, dbytes + fbytes + ibytes);
        if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "mechanism allocation: %s", cudaGetErrorString(e));
        e = cudaMemcpy(mem, dv.data(), dbytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy((char*)mem + dbytes, fv.data(), fbytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy((char*)mem + dbytes + fbytes, iv.data(), ibytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(mem);
            return cuda_fail(e, "mechanism copy");
        }
        const double* dp = (const double*)mem;
        const float4* fp = (const float4*)((char*)mem + dbytes);
        const int* ip = (const int*)((char*)mem + dbytes + fbytes);
        KinDevice& kd = r->kin;
        kd.S = S;
        kd.R = R;
        kd.kmin = d->kmin;
        kd.kmax = d->kmax;
        kd.W = dp;
        kd.thermo = dp + S;
        kd.log10A = dp + 5 * S;
        kd.beta = kd.log10A + R;
        kd.Ea = kd.beta + R;
        kd.rate32 = fp;
        kd.thermo32 = fp + R;
        kd.inc_off = ip;
        kd.inc = ip + S + 1;
        kd.sched = ip + sched_pos;
        kd.sched_k = sched_k;
        r->kin_alloc = mem;
        return ODE_OK;
    }
    case ODE_RHS_NBODY: {
        if (d->neq < 4 || d->neq > 4 * kMaxBodies || d->neq % 4)
            return fail(ODE_ERR_ARG, "n-body neq must be a multiple of 4 in [4, %d]", 4 * kMaxBodies);
        if (!d->masses) return fail(ODE_ERR_ARG, "n-body masses must be non-NULL");
        for (int b = 0; b < d->neq / 4; ++b) {
            if (!(d->masses[b] > 0.0) || !std::isfinite(d->masses[b]))
                return fail(ODE_ERR_ARG, "body %d: mass must be finite and > 0", b);
            r->masses[b] = d->masses[b];
        }
        return ODE_OK;
    }
    case ODE_RHS_MASSACTION: {
        const int S = d->neq, R = d->n_reactions;
        if (S < 1 || S > kMaxSpecies) return fail(ODE_ERR_ARG, "mass-action species count must be in [1, %d]", kMaxSpecies);
        if (R < 1 || R > kMaxReactions) return fail(ODE_ERR_ARG, "mass-action reaction count must be in [1, %d]", kMaxReactions);
        if (!d->n_reac || !d->reac || !d->n_prod || !d->prod || !d->log10A || !d->beta || !d->Ea)
            return fail(ODE_ERR_ARG, "mass-action network arrays must be non-NULL");
        if (!(d->kmin > 0.0) || !(d->kmax >= d->kmin)) return fail(ODE_ERR_ARG, "need 0 < kmin <= kmax");
        MassActionNet& n = r->net;
        n.n_species = S;
        n.n_reactions = R;
        n.kmin = d->kmin;
        n.kmax = d->kmax;
        for (int j = 0; j < R; ++j) {
            const int nr = d->n_reac[j], np = d->n_prod[j];
            if (nr < 1 || nr > 2 || np < 1 || np > 2) return fail(ODE_ERR_ARG, "reaction %d: 1-2 reactants and products", j);
            n.n_reac[j] = (int8_t)nr;
            n.n_prod[j] = (int8_t)np;
            for (int q = 0; q < 2; ++q) {
                const int rs = q < nr ? d->reac[2 * j + q] : 0;
                const int ps = q < np ? d->prod[2 * j + q] : 0;
                if (rs < 0 || rs >= S || ps < 0 || ps >= S) return fail(ODE_ERR_ARG, "reaction %d: species index out of range", j);
                n.reac[j][q] = (int8_t)rs;
                n.prod[j][q] = (int8_t)ps;
            }
            if (!std::isfinite(d->log10A[j]) || !std::isfinite(d->beta[j]) || !std::isfinite(d->Ea[j]))
                return fail(ODE_ERR_ARG, "reaction %d: non-finite Arrhenius parameter", j);
            n.log10A[j] = d->log10A[j];
            n.beta[j] = d->beta[j];
            n.Ea[j] = d->Ea[j];
        }
        return ODE_OK;
    }
    default:
        return fail(ODE_ERR_ARG, "unknown rhs kind %d", d->kind);
    }
}

enum Method { kRkck = 0, kRkc = 1 };

// One launch of the family's kernel (queue cursor reset included).
int dispatch(const RhsEntry& rhs, int meth, int prec, bool use_jit, const BatchArgs& a, const LaunchCfg& cfg) {
    cudaError_t e;
    if (cfg.mapping == ODE_MAP_QUEUE) {
        e = cudaMemsetAsync(a.cursor, 0, sizeof(unsigned long long), cfg.stream);
        if (e != cudaSuccess) return cuda_fail(e, "cursor reset");
    }
    bool supported = true;
    switch (rhs.kind) {
    case ODE_RHS_VDP: e = launch_vdp(meth, prec, rhs, a, cfg, &supported); break;
    case ODE_RHS_MASSACTION:
        if (use_jit) {
            std::string why;
            const int rc = jit_launch(rhs, meth, prec, a, cfg, &why);
            if (rc) return fail(rc, "%s", why.c_str());
            e = cudaSuccess;
        } else {
            e = launch_mass(meth, prec, rhs, a, cfg, &supported);
        }
        break;
    case ODE_RHS_BRUSS1D: e = launch_bruss(meth, prec, rhs, a, cfg, &supported); break;
    case ODE_RHS_VDP_CHAIN: e = launch_chain(meth, prec, rhs, a, cfg, &supported); break;
    case ODE_RHS_NBODY: e = launch_nbody(meth, prec, rhs, a, cfg, &supported); break;
    case ODE_RHS_KINETICS: e = launch_kinetics(meth, prec, rhs, a, cfg, &supported); break;
    default: supported = false; e = cudaSuccess;
    }
    if (!supported) return fail(ODE_ERR_UNSUPPORTED, "rhs kind %d with neq %d is not built for this method", rhs.kind, rhs.neq);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return ODE_OK;
}

// ODE_MAP_AUTO: the mapping and block size of a (rhs, method, precision,
// code path, device) are timed once on a sample of the first batch that is
// large enough to fill the device, and cached.  Smaller batches, and calls
// on a capturing stream, take the untuned default.
constexpr int64_t kTuneMinSystems = 32768;
std::map<std::tuple<int32_t, int, int, int, int, int>, std::pair<int, int>> g_map_tuned;

// Untuned default: one thread per system, one launch over the batch (lanes
// of a warp then start their systems together and stay in step longer than
// the queue's refills let them).
void default_mapping(LaunchCfg* cfg, int block_req) {
    cfg->mapping = ODE_MAP_THREAD;
    cfg->block = block_req ? block_req : 128;
}

int tune_mapping(Workspace* ws, int32_t handle, const RhsEntry& rhs, int meth, int prec, bool use_jit, int block_req,
                 const BatchArgs& a, LaunchCfg* cfg) {
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(handle, meth, prec, (int)use_jit, dev, block_req);
    auto it = g_map_tuned.find(key);
    if (it != g_map_tuned.end()) {
        cfg->mapping = it->second.first;
        cfg->block = it->second.second;
        return ODE_OK;
    }
    default_mapping(cfg, block_req);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(cfg->stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (a.nsys < kTuneMinSystems || cap != cudaStreamCaptureStatusNone) return ODE_OK;

    // sample: the first systems of the batch, output to a scratch buffer;
    // up to 262,144 systems give the work queue ~4 systems per lane, so that
    // the cost of its system switches shows (at one per lane it never
    // does).  A probe run of the first candidate on 32,768 systems (also the
    // warm-up: code paging, caches) prices a system; the sample then takes
    // what ~50 ms per candidate buys, between 65,536 and 262,144 systems.
    // Cheap systems (van der Pol RKCK in FP64, the FP32 and two-float
    // forms) get the full sample; expensive ones (FP64 mass-action, n-body)
    // keep 65,536, so that the timing costs less than one integration of a
    // 1M batch.
    const int64_t probe = kTuneMinSystems;
    const int64_t cap_sys = std::min<int64_t>(a.nsys, std::max<int64_t>(4096, (1 << 22) / rhs.neq));
    const int64_t sample_max = std::min<int64_t>(cap_sys, 262144);
    const size_t bytes = sizeof(double) * (size_t)sample_max * rhs.neq;
    if (ws->tune_bytes < bytes) {
        if (ws->tune_y) cudaFree(ws->tune_y);
        ws->tune_y = nullptr;
        ws->tune_bytes = 0;
        if (cudaMalloc(&ws->tune_y, bytes) != cudaSuccess) return ODE_OK;  // untuned
        ws->tune_bytes = bytes;
    }
    BatchArgs t = a;
    t.nsys = std::min<int64_t>(probe, sample_max);
    t.ld_in = a.nsys;
    t.ld_out = sample_max;
    t.y_out = ws->tune_y;
    t.n_accept = t.n_reject = t.n_rhs = t.n_specrad = t.status = nullptr;
    t.log_xy = nullptr;
    t.log_sr = nullptr;
    t.carry = nullptr;  // the timing runs neither read nor overwrite the caller's warm-restart state
    t.cursor = ws->cursors + kCursorRing;
    std::vector<std::pair<int, int>> cand;
    // generated kernels with a multi-block register budget launch at most
    // 128 threads per block: a larger candidate would time the same launch
    const int bmax = use_jit ? jit_max_block(prec) : 256;
    for (int b : {64, 128, 256})
        if ((!block_req || b == block_req) && b <= bmax) cand.push_back({ODE_MAP_THREAD, b});
    if (block_req && block_req != 64 && block_req != 128 && block_req != 256 && block_req <= bmax)
        cand.push_back({ODE_MAP_THREAD, block_req});
    if (cand.empty()) cand.push_back({ODE_MAP_THREAD, bmax});
    cand.push_back({ODE_MAP_QUEUE, block_req ? std::min(block_req, bmax) : 128});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    float best = 3.0e38f, best_probe_ms = 0.0f;
    int rc = ODE_OK;
    for (size_t k = 0; k <= cand.size() && rc == ODE_OK; ++k) {
        // k = 0 is the probe (and warm-up) with the first candidate
        LaunchCfg c = *cfg;
        c.mapping = cand[k ? k - 1 : 0].first;
        c.block = cand[k ? k - 1 : 0].second;
        if (k == 1) {  // the sample the probe's price allows
            const double per_sys = (double)best_probe_ms / (double)t.nsys;
            const int64_t want = per_sys > 0.0 ? (int64_t)(50.0 / per_sys) : sample_max;
            t.nsys = std::min<int64_t>(sample_max, std::max<int64_t>(std::min<int64_t>(65536, sample_max), want));
        }
        e = cudaEventRecord(e0, c.stream);
        if (e == cudaSuccess) rc = dispatch(rhs, meth, prec, use_jit, t, c);
        if (rc) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, c.stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "mapping tuning");
            break;
        }
        if (k == 0) best_probe_ms = ms;
        if (k && ms < best) {
            best = ms;
            cfg->mapping = c.mapping;
            cfg->block = c.block;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    g_map_tuned[key] = {cfg->mapping, cfg->block};
    return ODE_OK;
}

int integrate(Method method, int32_t handle, int64_t nsys, const double* y0, const double* params, double t0,
              double tend, double rtol, double atol, const ode_opts* opts_in, double* y_out,
              const ode_stats* stats_in, void* stream_ptr) {
    g_err.clear();
    RhsEntry rhs;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_reg.find(handle);
        if (it == g_reg.end()) return fail(ODE_ERR_HANDLE, "unknown rhs handle %d", handle);
        rhs = it->second;
    }
    ode_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    for (int k = 0; k < 3; ++k)
        if (opts.reserved[k] != 0) return fail(ODE_ERR_ARG, "opts.reserved must be zero");
    if (opts.log_sr && (method != kRkc || opts.precision != ODE_PREC_FP64))
        return fail(ODE_ERR_UNSUPPORTED, "the spectral-radius log is written by the plain FP64 RKC");
    if (opts.log_sr && opts.log_sr_records < 1) return fail(ODE_ERR_ARG, "log_sr needs log_sr_records >= 1");
    if (opts.mlp && (method != kRkc || !prec_is_f2(opts.precision)))
        return fail(ODE_ERR_UNSUPPORTED, "the in-kernel network is built for the two-float RKC forms");
    if (opts.mlp && rhs.n_params < 1) return fail(ODE_ERR_UNSUPPORTED, "the network's last input is the parameter");
    if (opts.specrad < ODE_SPECRAD_POWER || opts.specrad > ODE_SPECRAD_POWER_CAPPED)
        return fail(ODE_ERR_ARG, "unknown specrad mode %d", opts.specrad);
    if (opts.carry_mode != ODE_CARRY_CONTINUE && opts.carry_mode != ODE_CARRY_RESTART)
        return fail(ODE_ERR_ARG, "unknown carry_mode %d", opts.carry_mode);
    if (opts.cost_kind != 0 && opts.cost_kind != 1) return fail(ODE_ERR_ARG, "cost_kind must be 0 or 1");
    if (opts.codegen < ODE_CODEGEN_AUTO || opts.codegen > ODE_CODEGEN_ON) return fail(ODE_ERR_ARG, "unknown codegen mode %d", opts.codegen);
    if (opts.precision < ODE_PREC_FP64 || opts.precision > ODE_PREC_F2_LEAN)
        return fail(ODE_ERR_ARG, "unknown precision %d", opts.precision);
    if (prec_is_f2(opts.precision) && method != kRkc && rhs.kind != ODE_RHS_VDP && rhs.kind != ODE_RHS_VDP_CHAIN)
        return fail(ODE_ERR_UNSUPPORTED, "the two-float RKCK forms are built for van der Pol systems and chains only");
    if (opts.mapping < ODE_MAP_AUTO || opts.mapping > ODE_MAP_QUEUE) return fail(ODE_ERR_ARG, "unknown mapping %d", opts.mapping);
    if (opts.io != ODE_IO_DEVICE && opts.io != ODE_IO_HOST) return fail(ODE_ERR_ARG, "unknown io mode %d", opts.io);
    if (opts.block_size != 0 && (opts.block_size < 32 || opts.block_size > 256 || opts.block_size % 32))
        return fail(ODE_ERR_ARG, "block_size must be 0 or a multiple of 32 in [32, 256]");
    if (nsys < 0) return fail(ODE_ERR_ARG, "nsys must be >= 0");
    if (nsys > ((int64_t)1 << 40)) return fail(ODE_ERR_ARG, "nsys too large");
    if (!(rtol > 0.0) || !std::isfinite(rtol)) return fail(ODE_ERR_ARG, "rtol must be finite and > 0");
    if (!(atol >= 0.0) || !std::isfinite(atol)) return fail(ODE_ERR_ARG, "atol must be finite and >= 0");
    if (!std::isfinite(t0) || !std::isfinite(tend) || tend < t0) return fail(ODE_ERR_ARG, "need finite t0 <= tend");
    if ((opts.h0 == nullptr) != (opts.sigma0 == nullptr)) return fail(ODE_ERR_ARG, "h0 and sigma0 go together");
    if (opts.io == ODE_IO_HOST && (opts.h0 || opts.log_xy || opts.log_sr || opts.cost || opts.carry))
        return fail(ODE_ERR_ARG, "proposals, logs, cost ordering and warm-restart state need device io");
    if (opts.cost && nsys > INT32_MAX) return fail(ODE_ERR_ARG, "cost ordering takes at most 2^31 - 1 systems");
    if (nsys == 0) return ODE_OK;
    if (!y0 || !params || !y_out) return fail(ODE_ERR_ARG, "y0, params and y_out must be non-NULL");

    ode_stats stats;
    std::memset(&stats, 0, sizeof(stats));
    if (stats_in) stats = *stats_in;
    cudaStream_t stream = (cudaStream_t)stream_ptr;

    std::lock_guard<std::mutex> lk(g_mu);
    Workspace* ws = nullptr;
    int rc = get_workspace(&ws);
    if (rc) return rc;

    const size_t ny = (size_t)nsys * rhs.neq, np = (size_t)nsys * rhs.n_params;
    const double* d_y0 = y0;
    const double* d_p = params;
    double* d_yout = y_out;
    ode_stats d_stats = stats;
    cudaError_t e;
    int32_t* const* host_cnt[5] = {&stats.n_accept, &stats.n_reject, &stats.n_rhs, &stats.n_specrad_iter, &stats.status};
    int32_t** dev_cnt[5] = {&d_stats.n_accept, &d_stats.n_reject, &d_stats.n_rhs, &d_stats.n_specrad_iter, &d_stats.status};
    if (opts.io == ODE_IO_HOST) {
        const size_t need = sizeof(double) * (2 * ny + np) + sizeof(int32_t) * 5 * (size_t)nsys + 256 * 4;
        if (ws->stage_bytes < need) {
            if (ws->stage) cudaFree(ws->stage);
            ws->stage = nullptr;
            ws->stage_bytes = 0;
            e = cudaMalloc(&ws->stage, need);
            if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "staging allocation of %zu bytes failed", need);
            ws->stage_bytes = need;
        }
        char* p = (char*)ws->stage;
        auto carve = [&](size_t bytes) {
            char* q = p;
            p += (bytes + 255) / 256 * 256;
            return q;
        };
        double* sy0 = (double*)carve(sizeof(double) * ny);
        double* sp = (double*)carve(sizeof(double) * np);
        d_yout = (double*)carve(sizeof(double) * ny);
        for (int k = 0; k < 5; ++k) *dev_cnt[k] = *host_cnt[k] ? (int32_t*)carve(sizeof(int32_t) * nsys) : nullptr;
        e = cudaMemcpyAsync(sy0, y0, sizeof(double) * ny, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sp, params, sizeof(double) * np, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
        d_y0 = sy0;
        d_p = sp;
    }

    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nsys = nsys;
    a.neq = rhs.neq;
    a.max_attempts = opts.max_attempts > 0 ? opts.max_attempts : 1000000;
    a.y0 = d_y0;
    a.params = d_p;
    a.y_out = d_yout;
    a.t0 = t0;
    a.tend = tend;
    a.rtol = rtol;
    a.atol = atol;
    a.n_accept = d_stats.n_accept;
    a.n_reject = d_stats.n_reject;
    a.n_rhs = d_stats.n_rhs;
    a.n_specrad = d_stats.n_specrad_iter;
    a.status = d_stats.status;
    a.cursor = ws->cursors + ws->next_cursor;
    a.h0 = opts.h0;
    a.sigma0 = opts.sigma0;
    a.log_xy = opts.log_xy;
    a.log_sr = opts.log_sr;
    a.log_sr_every = opts.log_sr_every > 0 ? opts.log_sr_every : 1;
    a.log_sr_records = opts.log_sr_records;
    if (opts.mlp) {
        rc = mlp_packed_for(opts.mlp, rhs.neq + 1, &a.mlp);
        if (rc) return rc;
    }
    a.carry = opts.carry;
    a.carry_mode = opts.carry_mode;
    a.specrad = opts.specrad;
    a.rkc_tab64 = ws->tab64;
    a.rkc_tab32 = ws->tab32;
    a.rkc_tab_max = kRkcTabMax;
    ws->next_cursor = (ws->next_cursor + 1) % kCursorRing;

    LaunchCfg cfg;
    cfg.mapping = opts.mapping;
    cfg.block = opts.block_size ? opts.block_size : 128;
    cfg.team = 0;
    cfg.sm_count = ws->sm_count;
    cfg.stream = stream;
    if (rhs.kind == ODE_RHS_KINETICS && opts.specrad != ODE_SPECRAD_POWER)
        return fail(ODE_ERR_UNSUPPORTED, "kinetics right-hand sides take the power method only (no Jacobian bound)");
    const int meth = method == kRkck ? kMethodRkck : kMethodRkc;
    const bool use_jit = rhs.kind == ODE_RHS_MASSACTION &&
                         (opts.codegen == ODE_CODEGEN_ON || (opts.codegen == ODE_CODEGEN_AUTO && jit_available()));
    if (use_jit && prec_is_f2(opts.precision) && meth == kMethodRkc) {
        // the network's rate constants, once per system, before the
        // integration kernel (and before any tuning run, which reads them too)
        Workspace::ConstBuf& cb = ws->consts[stream];
        const size_t need = 2 * sizeof(float) * (size_t)rhs.net.n_reactions * (size_t)nsys;
        if (cb.bytes < need) {
            cudaFree(cb.ptr);
            cb.ptr = nullptr;
            cb.bytes = 0;
            e = cudaMalloc(&cb.ptr, need);
            if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "rate-constant table of %zu bytes", need);
            cb.bytes = need;
        }
        std::string why;
        rc = jit_rates(rhs, meth, opts.precision, d_p, nsys, cb.ptr, stream, &why);
        if (rc) return fail(rc, "%s", why.c_str());
        a.pre_consts = cb.ptr;
        a.pre_stride = nsys;
    }
    if (opts.mapping == ODE_MAP_AUTO) {
        rc = tune_mapping(ws, handle, rhs, meth, opts.precision, use_jit, opts.block_size, a, &cfg);
        if (rc) return rc;
    }
    if (opts.cost) {
        Workspace::OrderBuf& ob = ws->order[stream];
        if (ob.cap < nsys) {
            cudaFree(ob.index);
            ob.index = nullptr;
            ob.cap = 0;
            e = cudaMalloc(&ob.index, sizeof(int32_t) * (size_t)nsys);
            if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "order buffer of %lld systems", (long long)nsys);
            ob.cap = nsys;
        }
        if (!ob.bins) {
            e = cudaMalloc(&ob.bins, sizeof(int32_t) * kOrderScratchWords);
            if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "order bins");
        }
        e = order_by_cost(opts.cost, opts.cost_kind, nsys, ob.bins, ob.index, ws->sm_count, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cost ordering");
        a.index = ob.index;
    }
    rc = dispatch(rhs, meth, opts.precision, use_jit, a, cfg);
    if (rc) return rc;

    if (opts.io == ODE_IO_HOST) {
        e = cudaMemcpyAsync(y_out, d_yout, sizeof(double) * ny, cudaMemcpyDeviceToHost, stream);
        for (int k = 0; k < 5 && e == cudaSuccess; ++k)
            if (*host_cnt[k]) e = cudaMemcpyAsync(*host_cnt[k], *dev_cnt[k], sizeof(int32_t) * nsys, cudaMemcpyDeviceToHost, stream);
        if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    }
    if (opts.io == ODE_IO_HOST || opts.sync) {
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    }
    return ODE_OK;
}

}  // namespace

namespace bode {

void ragged_tuning_reset();

// Registry and error-string access for the allocation-free entry point
// (noalloc.cu).
bool registry_lookup(int32_t handle, RhsEntry* out) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_reg.find(handle);
    if (it == g_reg.end()) return false;
    *out = it->second;
    return true;
}

int set_last_error(int code, const char* msg) {
    g_err = msg;
    return code;
}

void clear_last_error() { g_err.clear(); }

}  // namespace bode

extern "C" {

int ode_rhs_register(const ode_rhs_desc* desc, int32_t* rhs_handle) {
    g_err.clear();
    if (!rhs_handle) return fail(ODE_ERR_ARG, "rhs_handle is NULL");
    RhsEntry r;
    int rc = validate_desc(desc, &r);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    const int32_t h = g_next_handle++;
    g_reg[h] = r;
    *rhs_handle = h;
    return ODE_OK;
}

int ode_rhs_release(int32_t rhs_handle) {
    g_err.clear();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it_r = g_reg.find(rhs_handle);
    if (it_r == g_reg.end()) return fail(ODE_ERR_HANDLE, "unknown rhs handle %d", rhs_handle);
    if (it_r->second.kin_alloc) cudaFree(it_r->second.kin_alloc);
    g_reg.erase(it_r);
    for (auto it = g_map_tuned.begin(); it != g_map_tuned.end();)
        it = std::get<0>(it->first) == rhs_handle ? g_map_tuned.erase(it) : std::next(it);
    return ODE_OK;
}

int ode_rhs_prepare(int32_t rhs_handle, int32_t method, int32_t precision) {
    g_err.clear();
    if (method != 0 && method != 1) return fail(ODE_ERR_ARG, "method must be 0 (RKCK) or 1 (RKC)");
    if (precision < ODE_PREC_FP64 || precision > ODE_PREC_F2_LEAN) return fail(ODE_ERR_ARG, "unknown precision %d", precision);
    RhsEntry r;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_reg.find(rhs_handle);
        if (it == g_reg.end()) return fail(ODE_ERR_HANDLE, "unknown rhs handle %d", rhs_handle);
        r = it->second;
    }
    if (prec_is_f2(precision) && method == 0 && r.kind != ODE_RHS_VDP && r.kind != ODE_RHS_VDP_CHAIN)
        return fail(ODE_ERR_UNSUPPORTED, "the two-float RKCK forms are built for van der Pol systems and chains only");
    if (r.kind != ODE_RHS_MASSACTION) return ODE_OK;
    std::string why;
    const int rc = jit_prepare(r, method == 0 ? kMethodRkck : kMethodRkc, precision, &why);
    if (rc) return fail(rc, "%s", why.c_str());
    return ODE_OK;
}

int rkck_integrate(int32_t rhs, int64_t nsys, const double* y0, const double* params, double t0, double tend,
                   double rtol, double atol, const ode_opts* opts, double* y_out, const ode_stats* stats,
                   void* stream) {
    return integrate(kRkck, rhs, nsys, y0, params, t0, tend, rtol, atol, opts, y_out, stats, stream);
}

int rkc_integrate(int32_t rhs, int64_t nsys, const double* y0, const double* params, double t0, double tend,
                  double rtol, double atol, const ode_opts* opts, double* y_out, const ode_stats* stats,
                  void* stream) {
    return integrate(kRkc, rhs, nsys, y0, params, t0, tend, rtol, atol, opts, y_out, stats, stream);
}

int ode_mapping_info(int32_t rhs_handle, int32_t method, int32_t precision, int32_t codegen, int32_t block_size,
                     int32_t* mapping, int32_t* block) {
    g_err.clear();
    if (!mapping || !block) return fail(ODE_ERR_ARG, "mapping and block must be non-NULL");
    if (method != 0 && method != 1) return fail(ODE_ERR_ARG, "method must be 0 (RKCK) or 1 (RKC)");
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_reg.find(rhs_handle);
    if (it == g_reg.end()) return fail(ODE_ERR_HANDLE, "unknown rhs handle %d", rhs_handle);
    const bool use_jit = it->second.kind == ODE_RHS_MASSACTION &&
                         (codegen == ODE_CODEGEN_ON || (codegen == ODE_CODEGEN_AUTO && jit_available()));
    int dev = 0;
    cudaGetDevice(&dev);
    const int meth = method == 0 ? kMethodRkck : kMethodRkc;
    auto t = g_map_tuned.find(std::make_tuple(rhs_handle, meth, precision, (int)use_jit, dev, block_size));
    LaunchCfg cfg;
    if (t != g_map_tuned.end()) {
        cfg.mapping = t->second.first;
        cfg.block = t->second.second;
    } else {
        default_mapping(&cfg, block_size);
    }
    if (use_jit && cfg.block > jit_max_block(precision)) cfg.block = jit_max_block(precision);  // what launches
    *mapping = cfg.mapping;
    *block = cfg.block;
    return t != g_map_tuned.end() ? ODE_OK : ODE_ERR_UNSUPPORTED;
}

namespace {
int cost_order_any(const void* cost, int kind, int64_t n, int32_t* index, void* stream_ptr);
}

int ode_cost_order(const float* cost, int64_t n, int32_t* index, void* stream_ptr) {
    return cost_order_any(cost, 0, n, index, stream_ptr);
}

int ode_cost_order_i32(const int32_t* cost, int64_t n, int32_t* index, void* stream_ptr) {
    return cost_order_any(cost, 1, n, index, stream_ptr);
}

}  // extern "C"

namespace {
int cost_order_any(const void* cost, int kind, int64_t n, int32_t* index, void* stream_ptr) {
    g_err.clear();
    if (n < 0 || n > INT32_MAX) return fail(ODE_ERR_ARG, "n must be in [0, 2^31 - 1]");
    if (n == 0) return ODE_OK;
    if (!cost || !index) return fail(ODE_ERR_ARG, "cost and index must be non-NULL");
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace* ws = nullptr;
    int rc = get_workspace(&ws);
    if (rc) return rc;
    Workspace::OrderBuf& ob = ws->order[stream];
    if (!ob.bins) {
        cudaError_t e = cudaMalloc(&ob.bins, sizeof(int32_t) * kOrderScratchWords);
        if (e != cudaSuccess) return fail(ODE_ERR_NOMEM, "order bins");
    }
    cudaError_t e = order_by_cost(cost, kind, n, ob.bins, index, ws->sm_count, stream);
    return e == cudaSuccess ? ODE_OK : cuda_fail(e, "cost ordering");
}
}  // namespace

extern "C" {

int ode_tuning_reset(void) {
    g_err.clear();
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_map_tuned.clear();
    }
    ragged_tuning_reset();
    return ODE_OK;
}

const char* ode_last_error(void) { return g_err.c_str(); }

const char* ode_version(void) { return "batchode 0.1 (sm_103a)"; }

}  // extern "C"
