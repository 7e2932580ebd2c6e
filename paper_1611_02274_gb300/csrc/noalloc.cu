// noalloc.cu -- rkc_integrate_noalloc: RKC integration that allocates no
// GPU memory.  For callers that may not call cudaMalloc (a fixed memory
// budget, another framework's pool, or code that must not fail on an
// allocation mid-job), every byte of scratch -- the work-queue cursor, an
// RKC coefficient table for stage counts up to kTabMax and the staging
// area for the caller's host arrays -- lives in one file-scope device array
// of ODE_NOALLOC_SCRATCH_BYTES.  Each device that loads the library holds
// the array until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "batchode.h"
#include "launch.cuh"

namespace bode {
bool registry_lookup(int32_t handle, RhsEntry* out);
int set_last_error(int code, const char* msg);
void clear_last_error();
}  // namespace bode

using namespace bode;

namespace {

constexpr int kTabMax = 32;                 // tabulated RKC stage counts (beyond: recomputed per stage)
constexpr size_t kAlign = 256;
constexpr size_t kCursorBytes = kAlign;      // one 8-byte counter, padded
constexpr size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kTab64Bytes = round_up(sizeof(double) * 8 * (kTabMax * (kTabMax + 1) / 2 - 1));
constexpr size_t kTab32Bytes = round_up(sizeof(float4) * (kTabMax * (kTabMax + 1) / 2 - 1));
constexpr size_t kStageOffset = kCursorBytes + kTab64Bytes + kTab32Bytes;
constexpr size_t kStageBytes = (size_t)ODE_NOALLOC_SCRATCH_BYTES - kStageOffset;

// The scratch.  In host code this name is only a stand-in for the device
// array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ODE_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;            // serialises calls: they share the array
unsigned char* g_base[kMaxDevices];  // device address of the array, per device (set-up done when non-null)

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

// Once per device, with that device current: the array's device address
// and the coefficient table built into it.
int setup_device(int dev, cudaStream_t stream, unsigned char** base) {
    if (g_base[dev]) {
        *base = g_base[dev];
        return ODE_OK;
    }
    unsigned char* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(ODE_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    e = build_rkc_tables((double*)(ptr + kCursorBytes), (float4*)(ptr + kCursorBytes + kTab64Bytes), kTabMax, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(ODE_ERR_CUDA, "coefficient table set-up: %s", cudaGetErrorString(e));
    g_base[dev] = ptr;
    *base = ptr;
    return ODE_OK;
}

}  // namespace

extern "C" int rkc_integrate_noalloc(int32_t handle, int64_t nsys, const double* y0, const double* params, double t0,
                                     double tend, double rtol, double atol, const ode_opts* opts_in, double* y_out,
                                     const ode_stats* stats_in, void* stream_ptr) {
    clear_last_error();
    RhsEntry rhs;
    if (!registry_lookup(handle, &rhs)) return fail(ODE_ERR_HANDLE, "unknown rhs handle %d", handle);
    ode_opts opts;
    std::memset(&opts, 0, sizeof(opts));
    if (opts_in) opts = *opts_in;
    if (opts.precision < ODE_PREC_FP64 || opts.precision > ODE_PREC_MIXED_LEAN)
        return fail(ODE_ERR_ARG, "precision %d is not built for the allocation-free entry point", opts.precision);
    if (opts.mlp || opts.log_sr)
        return fail(ODE_ERR_ARG, "networks and the spectral-radius log are not taken by the allocation-free entry point");
    if (opts.specrad < ODE_SPECRAD_POWER || opts.specrad > ODE_SPECRAD_POWER_CAPPED)
        return fail(ODE_ERR_ARG, "unknown specrad mode %d", opts.specrad);
    switch (rhs.kind) {  // every built-in family; decided before any GPU work
    case ODE_RHS_VDP:
    case ODE_RHS_MASSACTION:
    case ODE_RHS_BRUSS1D:
    case ODE_RHS_VDP_CHAIN:
    case ODE_RHS_NBODY:
    case ODE_RHS_KINETICS: break;
    default: return fail(ODE_ERR_UNSUPPORTED, "rhs kind %d is not built", rhs.kind);
    }
    if (rhs.kind == ODE_RHS_KINETICS && opts.specrad != ODE_SPECRAD_POWER)
        return fail(ODE_ERR_UNSUPPORTED, "kinetics right-hand sides take the power method only (no Jacobian bound)");
    if (opts.mapping < ODE_MAP_AUTO || opts.mapping > ODE_MAP_QUEUE) return fail(ODE_ERR_ARG, "unknown mapping %d", opts.mapping);
    if (opts.block_size != 0 && (opts.block_size < 32 || opts.block_size > 256 || opts.block_size % 32))
        return fail(ODE_ERR_ARG, "block_size must be 0 or a multiple of 32 in [32, 256]");
    if (nsys < 0) return fail(ODE_ERR_ARG, "nsys must be >= 0");
    if (!(rtol > 0.0) || !std::isfinite(rtol)) return fail(ODE_ERR_ARG, "rtol must be finite and > 0");
    if (!(atol >= 0.0) || !std::isfinite(atol)) return fail(ODE_ERR_ARG, "atol must be finite and >= 0");
    if (!std::isfinite(t0) || !std::isfinite(tend) || tend < t0) return fail(ODE_ERR_ARG, "need finite t0 <= tend");
    if (nsys == 0) return ODE_OK;
    if (!y0 || !params || !y_out) return fail(ODE_ERR_ARG, "y0, params and y_out must be non-NULL");

    ode_stats stats;
    std::memset(&stats, 0, sizeof(stats));
    if (stats_in) stats = *stats_in;
    int32_t* host_cnt[5] = {stats.n_accept, stats.n_reject, stats.n_rhs, stats.n_specrad_iter, stats.status};

    // staging layout: y (in and out, in place), params, requested counters
    const size_t ny = (size_t)nsys * rhs.neq, np = (size_t)nsys * rhs.n_params;
    if (nsys > (int64_t)(kStageBytes / 8)) return fail(ODE_ERR_ARG, "nsys %lld exceeds the static scratch", (long long)nsys);
    size_t need = round_up(sizeof(double) * ny) + round_up(sizeof(double) * np);
    for (int k = 0; k < 5; ++k)
        if (host_cnt[k]) need += round_up(sizeof(int32_t) * (size_t)nsys);
    if (need > kStageBytes)
        return fail(ODE_ERR_ARG,
                    "batch needs %zu bytes of staging but the static scratch holds %zu (ODE_NOALLOC_SCRATCH_BYTES less "
                    "cursor and table); split it into batches of at most %lld systems",
                    need, kStageBytes, (long long)(nsys * (double)kStageBytes / (double)need));

    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ODE_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(ODE_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(ODE_ERR_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    unsigned char* base = nullptr;
    int rc = setup_device(dev, stream, &base);
    if (rc) return rc;

    unsigned char* p = base + kStageOffset;
    double* d_y = (double*)p;
    p += round_up(sizeof(double) * ny);
    double* d_p = (double*)p;
    p += round_up(sizeof(double) * np);
    int32_t* d_cnt[5];
    for (int k = 0; k < 5; ++k) {
        d_cnt[k] = nullptr;
        if (host_cnt[k]) {
            d_cnt[k] = (int32_t*)p;
            p += round_up(sizeof(int32_t) * (size_t)nsys);
        }
    }

    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nsys = nsys;
    a.neq = rhs.neq;
    a.max_attempts = opts.max_attempts > 0 ? opts.max_attempts : 1000000;
    a.y0 = d_y;
    a.params = d_p;
    a.y_out = d_y;  // in place: each system reads its state before writing it
    a.t0 = t0;
    a.tend = tend;
    a.rtol = rtol;
    a.atol = atol;
    a.n_accept = d_cnt[0];
    a.n_reject = d_cnt[1];
    a.n_rhs = d_cnt[2];
    a.n_specrad = d_cnt[3];
    a.status = d_cnt[4];
    a.cursor = (unsigned long long*)base;
    a.rkc_tab64 = (const double*)(base + kCursorBytes);
    a.rkc_tab32 = (const float4*)(base + kCursorBytes + kTab64Bytes);
    a.rkc_tab_max = kTabMax;
    a.specrad = opts.specrad;

    // From the first queued operation on, every return waits for the
    // stream: the copies may still read the caller's arrays, and the next
    // call (under the lock, perhaps on another stream) reuses the scratch.
    auto fail_after_queue = [&](int code, const char* what, cudaError_t err) {
        cudaStreamSynchronize(stream);  // its own status is not the error to report
        return fail(code, "%s: %s", what, cudaGetErrorString(err));
    };
    e = cudaMemsetAsync(a.cursor, 0, sizeof(unsigned long long), stream);  // the queue starts at system 0
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_y, y0, sizeof(double) * ny, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_p, params, sizeof(double) * np, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return fail_after_queue(ODE_ERR_CUDA, "staging copy", e);

    LaunchCfg cfg;
    cfg.mapping = opts.mapping == ODE_MAP_THREAD ? ODE_MAP_THREAD : ODE_MAP_QUEUE;
    cfg.block = opts.block_size ? opts.block_size : 128;
    cfg.team = 0;
    cfg.sm_count = sms;
    cfg.stream = stream;
    bool supported = true;
    switch (rhs.kind) {
    case ODE_RHS_VDP: e = launch_vdp(kMethodRkc, opts.precision, rhs, a, cfg, &supported); break;
    case ODE_RHS_MASSACTION: e = launch_mass(kMethodRkc, opts.precision, rhs, a, cfg, &supported); break;
    case ODE_RHS_BRUSS1D: e = launch_bruss(kMethodRkc, opts.precision, rhs, a, cfg, &supported); break;
    case ODE_RHS_VDP_CHAIN: e = launch_chain(kMethodRkc, opts.precision, rhs, a, cfg, &supported); break;
    case ODE_RHS_NBODY: e = launch_nbody(kMethodRkc, opts.precision, rhs, a, cfg, &supported); break;
    default: e = launch_kinetics(kMethodRkc, opts.precision, rhs, a, cfg, &supported); break;
    }
    if (!supported) {
        cudaStreamSynchronize(stream);
        return fail(ODE_ERR_UNSUPPORTED, "rhs kind %d with neq %d is not built", rhs.kind, rhs.neq);
    }
    if (e != cudaSuccess) return fail_after_queue(ODE_ERR_CUDA, "kernel launch", e);

    e = cudaMemcpyAsync(y_out, d_y, sizeof(double) * ny, cudaMemcpyDeviceToHost, stream);
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        if (host_cnt[k]) e = cudaMemcpyAsync(host_cnt[k], d_cnt[k], sizeof(int32_t) * nsys, cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return fail_after_queue(ODE_ERR_CUDA, "result copy", e);
    e = cudaStreamSynchronize(stream);  // the next call may reuse the array
    if (e != cudaSuccess) return fail(ODE_ERR_CUDA, "stream synchronize: %s", cudaGetErrorString(e));
    return ODE_OK;
}
