// ragged.cu -- ragged batches: systems of different families, sizes and
// methods in one plan.
//
// A plan groups the systems into buckets (family, method, size class =
// smallest of 8/16/32/64/128/192/256 unknowns that holds them), orders each
// bucket's queue by size, largest first, picks for each bucket a kernel
// shape -- lanes per system (1, 8, 16 or 32), grid points per lane, block
// size and mapping -- and captures every bucket's cursor reset and
// persistent-queue kernel, on parallel branches, into one CUDA graph.  A
// launch replays the graph: one call integrates the whole batch, and while
// one bucket drains its tail the others fill the freed SMs.
//
// Shapes: ODE_MAP_AUTO times each candidate shape x block size x mapping
// (persistent queue or one launch over the bucket) on a sample of the
// bucket (cached per family / method / precision / size class);
// ODE_MAP_THREAD is the paper's mapping (one thread per system, one
// launch, 64-thread blocks); ODE_MAP_QUEUE uses the default warp-per-system
// shape without tuning.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "batchode.h"
#include "launch.cuh"
#include "rhs.cuh"

namespace bode {
bool registry_lookup(int32_t handle, RhsEntry* out);
int set_last_error(int code, const char* msg);
void clear_last_error();
cudaError_t launch_bruss_shape_team(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok);
cudaError_t launch_bruss_shape_t1(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok);
cudaError_t launch_chain_shape_team(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok);
cudaError_t launch_chain_shape_t1(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok);
cudaError_t launch_bruss_shape_f2(int team, int g, const BatchArgs& a, const GridCtx& ctx, const LaunchCfg& c, bool* ok);
cudaError_t launch_chain_shape_f2(int method, int team, int g, const BatchArgs& a, const GridCtx& ctx,
                                  const LaunchCfg& c, bool* ok);
}  // namespace bode

using namespace bode;

namespace {

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

// 192 splits the largest grids: 65-96 points fill a 32-lane x 3-point team
// instead of padding a 4-point one to 128
const int kClasses[] = {8, 16, 32, 64, 128, 192, 256};

// A kernel shape: lanes per system and grid points per lane (team = 0: the
// family's default kernels, which pick their own shape by size).
struct Shape {
    int team, g, max_neq;
};

// extra shapes, built for the lean mixed form with each family's own method
// (Brusselator grids: RKC, oscillator chains: RKCK)
const Shape kBrussShapes[] = {{1, 4, 8}, {8, 1, 16}, {16, 1, 32}, {32, 2, 128}, {32, 3, 192}, {1, 128, 256}};
const Shape kChainShapes[] = {{1, 4, 8}, {8, 1, 16}, {16, 1, 32}, {1, 64, 128}};
// two-float shapes (FP32 scalars) for the small classes, both families;
// the warp-wide default kernels take the rest
const Shape kF2Shapes[] = {{8, 1, 16}, {16, 1, 32}};

bool tuned_method(int family, int method) {
    return (family == ODE_RHS_BRUSS1D && method == kMethodRkc) || (family == ODE_RHS_VDP_CHAIN && method == kMethodRkck);
}

cudaError_t launch_shape(int family, int method, int prec, const Shape& sh, const RhsEntry& r, const BatchArgs& a,
                         const LaunchCfg& c, bool* ok) {
    const GridCtx g{r.bruss_A, r.bruss_B, r.bruss_ubc, r.bruss_vbc, r.coupling};
    if (sh.team == 0) {
        RhsEntry rr = r;
        rr.neq = sh.max_neq;  // size of the default kernel to use
        return family == ODE_RHS_BRUSS1D ? launch_bruss(method, prec, rr, a, c, ok) : launch_chain(method, prec, rr, a, c, ok);
    }
    if (prec == ODE_PREC_F2_LEAN)
        return family == ODE_RHS_BRUSS1D ? launch_bruss_shape_f2(sh.team, sh.g, a, g, c, ok)
                                         : launch_chain_shape_f2(method, sh.team, sh.g, a, g, c, ok);
    if (family == ODE_RHS_BRUSS1D)
        return sh.team == 1 ? launch_bruss_shape_t1(sh.team, sh.g, a, g, c, ok) : launch_bruss_shape_team(sh.team, sh.g, a, g, c, ok);
    return sh.team == 1 ? launch_chain_shape_t1(sh.team, sh.g, a, g, c, ok) : launch_chain_shape_team(sh.team, sh.g, a, g, c, ok);
}

// The precision a bucket runs in.  A two-float plan takes the two-float
// kernels where they are built (Brusselator grids by RKC, oscillator chains
// by RKCK or RKC) and FP64 for Brusselator grids by RKCK, so that every
// bucket of the plan keeps FP64-class accuracy.
int bucket_prec(int family, int method, int prec) {
    if (!prec_is_f2(prec)) return prec;
    return family == ODE_RHS_BRUSS1D && method == kMethodRkck ? ODE_PREC_FP64 : prec;
}

// candidate shapes for a bucket (the default kernel first)
std::vector<Shape> candidates(int family, int method, int prec, int cls, bool thread_only) {
    std::vector<Shape> out;
    const int def_max = family == ODE_RHS_BRUSS1D ? (cls <= 64 ? 64 : 256) : (cls <= 64 ? 64 : 128);
    if (!thread_only) out.push_back({0, 0, def_max});
    if (prec == ODE_PREC_F2_LEAN && !thread_only) {
        for (const Shape& sh : kF2Shapes)
            if (sh.max_neq >= cls) out.push_back(sh);
        return out;
    }
    if (prec == ODE_PREC_MIXED_LEAN && tuned_method(family, method)) {
        const Shape* s = family == ODE_RHS_BRUSS1D ? kBrussShapes : kChainShapes;
        const int n = family == ODE_RHS_BRUSS1D ? (int)(sizeof(kBrussShapes) / sizeof(Shape))
                                                : (int)(sizeof(kChainShapes) / sizeof(Shape));
        for (int k = 0; k < n; ++k) {
            if (s[k].max_neq < cls) continue;
            if (thread_only != (s[k].team == 1)) continue;
            // a thread-per-system shape only where it is the paper's mapping or small
            if (!thread_only && s[k].team == 1 && s[k].max_neq > 8) continue;
            out.push_back(s[k]);
        }
    }
    return out;
}

struct Bucket {
    int32_t handle;
    RhsEntry rhs;
    int method, cls;
    int prec;  // bucket_prec of the plan's precision
    std::vector<int32_t> sys;
    Shape shape;
    int block, mapping;
    int64_t index_offset;  // into the plan's device index list
};

struct Plan {
    int dev;
    std::vector<Bucket> buckets;
    int64_t* d_offset = nullptr;
    int32_t* d_neq = nullptr;
    int32_t* d_index = nullptr;
    unsigned long long* d_cursor = nullptr;
    double* d_tab64 = nullptr;
    float4* d_tab32 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

std::mutex g_mu;
std::map<int64_t, Plan*> g_plans;
int64_t g_next_plan = 1;
// tuned (shape, block, mapping) per family / method / precision / size class / SM count
struct Tuned {
    Shape shape;
    int block, mapping;
};
std::map<std::tuple<int, int, int, int, int>, Tuned> g_tuned;

constexpr int kTabMax = 256;

int make_args(const Plan& p, const Bucket& b, const ode_ragged_batch& rb, const ode_opts& o, double* y_out,
              const ode_stats& st, int64_t count, unsigned long long* cursor, BatchArgs* out) {
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nsys = count;
    a.neq = b.rhs.neq;
    a.max_attempts = o.max_attempts > 0 ? o.max_attempts : 1000000;
    a.y0 = rb.y0;
    a.params = rb.params;
    a.y_out = y_out;
    a.n_accept = st.n_accept;
    a.n_reject = st.n_reject;
    a.n_rhs = st.n_rhs;
    a.n_specrad = st.n_specrad_iter;
    a.status = st.status;
    a.cursor = cursor;
    a.rkc_tab64 = p.d_tab64;
    a.rkc_tab32 = p.d_tab32;
    a.rkc_tab_max = kTabMax;
    a.index = p.d_index + b.index_offset;
    a.offset = p.d_offset;
    a.neq_arr = p.d_neq;
    a.t0_arr = rb.t0;
    a.tend_arr = rb.tend;
    a.rtol_arr = rb.rtol;
    a.atol_arr = rb.atol;
    *out = a;
    return ODE_OK;
}

int sm_count(int dev) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

int destroy(Plan* p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_offset);
    cudaFree(p->d_neq);
    cudaFree(p->d_index);
    cudaFree(p->d_cursor);
    cudaFree(p->d_tab64);
    cudaFree(p->d_tab32);
    delete p;
    return ODE_OK;
}

}  // namespace

namespace bode {
void ragged_tuning_reset() {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tuned.clear();
}
}  // namespace bode

extern "C" {

int ode_ragged_plan_create(const ode_ragged_batch* rb, const ode_opts* opts_in, double* y_out, const ode_stats* stats_in,
                           void* stream_ptr, int64_t* plan_out) {
    clear_last_error();
    if (!rb || !plan_out || !y_out) return fail(ODE_ERR_ARG, "batch, y_out and plan must be non-NULL");
    const int64_t nsys = rb->nsys;
    if (nsys < 1) return fail(ODE_ERR_ARG, "nsys must be >= 1");
    if (!rb->rhs || !rb->method || !rb->neq || !rb->offset || !rb->y0 || !rb->params || !rb->t0 || !rb->tend ||
        !rb->rtol || !rb->atol)
        return fail(ODE_ERR_ARG, "every batch array must be non-NULL");
    ode_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts_in) o = *opts_in;
    if (o.precision < ODE_PREC_FP64 || o.precision > ODE_PREC_F2_LEAN) return fail(ODE_ERR_ARG, "unknown precision");
    if (o.mlp || o.log_sr) return fail(ODE_ERR_ARG, "networks and the spectral-radius log are not taken by ragged plans");
    if (o.mapping < ODE_MAP_AUTO || o.mapping > ODE_MAP_QUEUE) return fail(ODE_ERR_ARG, "unknown mapping");
    ode_stats st;
    std::memset(&st, 0, sizeof(st));
    if (stats_in) st = *stats_in;
    cudaStream_t user = (cudaStream_t)stream_ptr;

    // buckets
    std::map<std::tuple<int32_t, int, int>, Bucket> by_key;
    for (int64_t i = 0; i < nsys; ++i) {
        RhsEntry r;
        if (!registry_lookup(rb->rhs[i], &r)) return fail(ODE_ERR_HANDLE, "system %lld: unknown rhs handle %d", (long long)i, rb->rhs[i]);
        if (r.kind != ODE_RHS_BRUSS1D && r.kind != ODE_RHS_VDP_CHAIN)
            return fail(ODE_ERR_UNSUPPORTED, "system %lld: ragged batches take Brusselator and chain systems", (long long)i);
        const int n = rb->neq[i], m = rb->method[i];
        if (n < 2 || n % 2 || n > r.neq) return fail(ODE_ERR_ARG, "system %lld: neq %d not even in [2, %d]", (long long)i, n, r.neq);
        if (m != 0 && m != 1) return fail(ODE_ERR_ARG, "system %lld: method must be 0 or 1", (long long)i);
        int cls = 256;
        for (int c : kClasses)
            if (n <= c) {
                cls = c;
                break;
            }
        auto key = std::make_tuple(rb->rhs[i], m, cls);
        Bucket& b = by_key[key];
        if (b.sys.empty()) {
            b.handle = rb->rhs[i];
            b.rhs = r;
            b.method = m == 0 ? kMethodRkck : kMethodRkc;
            b.cls = cls;
            b.prec = bucket_prec(r.kind, b.method, o.precision);
        }
        b.sys.push_back((int32_t)i);
    }

    Plan* p = new Plan();
    cudaGetDevice(&p->dev);
    const int sms = sm_count(p->dev);
    std::vector<int32_t> index;
    for (auto& kv : by_key) {
        Bucket b = kv.second;
        // largest systems first: the queue starts the longest work early
        std::stable_sort(b.sys.begin(), b.sys.end(), [&](int32_t x, int32_t y) { return rb->neq[x] > rb->neq[y]; });
        b.index_offset = (int64_t)index.size();
        index.insert(index.end(), b.sys.begin(), b.sys.end());
        p->buckets.push_back(b);
    }
    const size_t nb = p->buckets.size();
    cudaError_t e = cudaMalloc(&p->d_offset, sizeof(int64_t) * nsys);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_neq, sizeof(int32_t) * nsys);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_index, sizeof(int32_t) * index.size());
    if (e == cudaSuccess) e = cudaMalloc(&p->d_cursor, 256 * (nb + 1));
    const int entries = rkc_tab_index(kTabMax + 1, 1);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tab64, sizeof(double) * 8 * entries);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_tab32, sizeof(float4) * entries);
    if (e != cudaSuccess) {
        destroy(p);
        return fail(ODE_ERR_NOMEM, "plan allocation failed");
    }
    e = cudaMemcpy(p->d_offset, rb->offset, sizeof(int64_t) * nsys, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_neq, rb->neq, sizeof(int32_t) * nsys, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_index, index.data(), sizeof(int32_t) * index.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = build_rkc_tables(p->d_tab64, p->d_tab32, kTabMax, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        destroy(p);
        return cuda_fail(e, "plan set-up");
    }

    // shapes
    double* tune_out = nullptr;
    for (auto& b : p->buckets) {
        const int family = b.rhs.kind;
        if (o.mapping == ODE_MAP_THREAD) {
            auto c = candidates(family, b.method, b.prec, b.cls, true);
            b.shape = c.empty() ? Shape{0, 0, b.cls <= 64 ? 64 : (family == ODE_RHS_BRUSS1D ? 256 : 128)} : c.front();
            b.block = 64;
            b.mapping = ODE_MAP_THREAD;
            continue;
        }
        auto cand = candidates(family, b.method, b.prec, b.cls, false);
        b.shape = cand.front();
        b.block = 128;
        b.mapping = ODE_MAP_QUEUE;
        if (o.mapping == ODE_MAP_QUEUE) continue;
        auto key = std::make_tuple(family, b.method, b.prec, b.cls, sms);
        {
            std::lock_guard<std::mutex> lk(g_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                b.shape = it->second.shape;
                b.block = it->second.block;
                b.mapping = it->second.mapping;
                continue;
            }
        }
        // time each shape, block size and mapping on a sample of this bucket;
        // the sample's results go to a scratch state when the plan
        // integrates in place (they would overwrite initial states)
        if (y_out == rb->y0 && !tune_out) {
            int64_t ny = 0;
            for (int64_t i = 0; i < nsys; ++i) ny = std::max<int64_t>(ny, rb->offset[i] + rb->neq[i]);
            if (cudaMalloc(&tune_out, sizeof(double) * (size_t)ny) != cudaSuccess) {
                tune_out = nullptr;
                continue;  // untuned
            }
        }
        const int64_t sample = std::min<int64_t>((int64_t)b.sys.size(), 8192);
        float best = 3.0e38f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (const Shape& sh : cand) {
            for (int blk : {64, 128, 256}) {
                bool ok = true;
                for (int map : {ODE_MAP_QUEUE, ODE_MAP_THREAD}) {
                    BatchArgs a;
                    make_args(*p, b, *rb, o, tune_out ? tune_out : y_out, st, sample, p->d_cursor + 32 * nb, &a);
                    LaunchCfg cfg{map, blk, sh.team, sms, user};
                    cudaMemsetAsync(a.cursor, 0, 8, user);
                    launch_shape(family, b.method, b.prec, sh, b.rhs, a, cfg, &ok);  // warm-up
                    if (!ok) break;
                    cudaMemsetAsync(a.cursor, 0, 8, user);
                    cudaEventRecord(e0, user);
                    launch_shape(family, b.method, b.prec, sh, b.rhs, a, cfg, &ok);
                    cudaEventRecord(e1, user);
                    e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        cudaFree(tune_out);
                        destroy(p);
                        return cuda_fail(e, "autotuning launch");
                    }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) {
                        best = ms;
                        b.shape = sh;
                        b.block = blk;
                        b.mapping = map;
                    }
                }
                if (!ok) break;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lk(g_mu);
        g_tuned[key] = {b.shape, b.block, b.mapping};
    }
    cudaFree(tune_out);

    // graph: fork one branch per bucket, join
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    std::vector<cudaStream_t> br(nb);
    std::vector<cudaEvent_t> ev(nb + 1);
    for (size_t k = 0; k < nb && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking);
    for (size_t k = 0; k <= nb && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(ev[nb], cap);
    bool supported = true;
    for (size_t k = 0; k < nb && e == cudaSuccess; ++k) {
        const Bucket& b = p->buckets[k];
        BatchArgs a;
        make_args(*p, b, *rb, o, y_out, st, (int64_t)b.sys.size(), p->d_cursor + 32 * k, &a);
        LaunchCfg cfg{b.mapping, b.block, b.shape.team, sms, br[k]};
        e = cudaStreamWaitEvent(br[k], ev[nb], 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.cursor, 0, 8, br[k]);
        if (e == cudaSuccess) e = launch_shape(b.rhs.kind, b.method, b.prec, b.shape, b.rhs, a, cfg, &supported);
        if (e == cudaSuccess && !supported) break;
        if (e == cudaSuccess) e = cudaEventRecord(ev[k], br[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev[k], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(cap, &p->graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && supported) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    for (auto s : br) cudaStreamDestroy(s);
    for (auto x : ev) cudaEventDestroy(x);
    cudaStreamDestroy(cap);
    if (!supported) {
        destroy(p);
        return fail(ODE_ERR_UNSUPPORTED, "a bucket's kernel shape is not built for this precision / method");
    }
    if (e != cudaSuccess) {
        destroy(p);
        return cuda_fail(e, "graph capture");
    }
    std::lock_guard<std::mutex> lk(g_mu);
    *plan_out = g_next_plan++;
    g_plans[*plan_out] = p;
    return ODE_OK;
}

int ode_ragged_plan_launch(int64_t plan, void* stream) {
    clear_last_error();
    Plan* p;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(plan);
        if (it == g_plans.end()) return fail(ODE_ERR_HANDLE, "unknown plan %lld", (long long)plan);
        p = it->second;
    }
    cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? ODE_OK : cuda_fail(e, "graph launch");
}

int ode_ragged_plan_info(int64_t plan, int32_t* n_buckets, int32_t* desc, int32_t capacity) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(plan);
    if (it == g_plans.end()) return fail(ODE_ERR_HANDLE, "unknown plan %lld", (long long)plan);
    const Plan* p = it->second;
    if (n_buckets) *n_buckets = (int32_t)p->buckets.size();
    for (int32_t k = 0; desc && k < capacity && k < (int32_t)p->buckets.size(); ++k) {
        const Bucket& b = p->buckets[k];
        int32_t* d = desc + 8 * k;
        d[0] = b.rhs.kind;
        d[1] = b.method == kMethodRkck ? 0 : 1;
        d[2] = b.cls;
        d[3] = (int32_t)b.sys.size();
        d[4] = b.shape.team == 0 ? 32 : b.shape.team;
        d[5] = b.shape.team == 0 ? 0 : b.shape.g;
        d[6] = b.block;
        d[7] = b.mapping;
    }
    return ODE_OK;
}

int ode_ragged_plan_destroy(int64_t plan) {
    clear_last_error();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(plan);
    if (it == g_plans.end()) return fail(ODE_ERR_HANDLE, "unknown plan %lld", (long long)plan);
    destroy(it->second);
    g_plans.erase(it);
    return ODE_OK;
}

}  // extern "C"
