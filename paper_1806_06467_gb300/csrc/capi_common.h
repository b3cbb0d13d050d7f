// capi_common.h -- host-side helpers shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/coro.h"

struct coro_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::map<int, void*> tw32;   // twiddles exp(-2 pi i m / n), complex64, per n
    std::map<int, void*> tw64;   // same, complex128
    void* work = nullptr;        // MFT work buffer (grown on demand)
    size_t work_bytes = 0;
    int* err = nullptr;          // device flag set by kernels whose bounded waits expired
};

// Replay of a plan's launch sequence as one CUDA graph. The graph is captured on a private
// stream the first time execute runs with a given set of device pointers (after one eager
// run of the same sequence, which makes every lazily built table exist and produces that
// call's result), and re-captured when the pointers change.
struct PlanGraph {
    bool enabled = false;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
    ~PlanGraph() {
        reset();
        if (cap) cudaStreamDestroy(cap);
    }
};

// Per-unit timing of consecutive executes: `steps` sets of (units + 1) events; execute k of
// an execute_n call records set k before its first unit and after each unit (inside the
// graph when one is used), so unit durations are measured on the stream the kernels run on.
struct PlanTiming {
    int steps = 0, units = 0;
    std::vector<cudaEvent_t> ev;
    void release() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        steps = 0;
    }
    const cudaEvent_t* set(int k) const { return k < steps ? ev.data() + (size_t)k * (units + 1) : nullptr; }
};

// Base of every plan handle (Fresnel systems: kind 1, Lyot coronagraphs: kind 2).
struct coro_plan_s {
    PlanGraph graph;
    PlanTiming timing;
    virtual ~coro_plan_s() {}
    virtual int kind() const = 0;
    virtual int launches() const = 0;
    virtual int timing_units() const = 0;
};

namespace coro {

void set_error(const char* fmt, ...);
void clear_error();
coro_status cuda_fail(cudaError_t e, const char* what);

// Switch to the context's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Run `body` (which launches on ctx->stream) directly, or through the plan's graph: captured
// on first use with `key`, replayed on ctx->stream afterwards. body returns a coro_status.
template <typename F>
coro_status run_graphed(coro_ctx ctx, PlanGraph& g, const std::vector<const void*>& key, F body) {
    if (!g.enabled) return body();
    if (g.exec && key == g.key) {
        const cudaError_t e = cudaGraphLaunch(g.exec, ctx->stream);
        return e == cudaSuccess ? CORO_OK : cuda_fail(e, "cudaGraphLaunch");
    }
    coro_status st = body();                              // eager run: this call's result
    if (st != CORO_OK) return st;
    g.reset();
    cudaError_t e = cudaSuccess;
    if (!g.cap) e = cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate (graph capture)");
    cudaStream_t user = ctx->stream;
    ctx->stream = g.cap;
    e = cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = body();
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(g.cap, &graph);
        if (st == CORO_OK && e2 == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
        else if (e2 != cudaSuccess) e = e2;
        if (graph) cudaGraphDestroy(graph);
    }
    ctx->stream = user;
    if (st != CORO_OK) { g.reset(); return st; }
    if (e != cudaSuccess) { g.reset(); return cuda_fail(e, "graph capture"); }
    g.key = key;
    return CORO_OK;
}

// Record a timing event: a plain record, or an event-record node of the graph while the
// stream is being captured (the external flag is only valid during capture).
inline cudaError_t record_timing_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, s);
}

// Twiddle table for n (built lazily on the context's stream).
const void* get_twiddles(coro_ctx ctx, int n, bool dbl, coro_status* st, bool linear = false);
// The Lyot plan at reference precision (lyot64.cu): complex128 fields, FP64 MFTs, item by item.
coro_status lyot64_create(coro_ctx ctx, const coro_lyot_desc* d, coro_plan* out);
coro_status lyot64_peak(coro_plan plan, const void* pupil, double* peak_out);
int lyot64_batch(coro_plan plan);
coro_status lyot64_execute(coro_plan plan, const void* pupil, const double* peak, float* intensity, void* field,
                           double* dh);


// Stream-ordered copy of a host array into a fresh device block (freed with free_async).
void* upload_async(coro_ctx ctx, const void* host, size_t bytes, coro_status* st);
void free_async(coro_ctx ctx, void* p);

// Grow the context work buffer to at least `bytes` (synchronous allocation).
void* ctx_work(coro_ctx ctx, size_t bytes, coro_status* st);

inline bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// Largest integer m >= 0 with (double)m * (pitch * pitch) <= r * r (strict: <), or -1.
// These are the exact FP64 predicates the masks are defined by.
long long disk_threshold(double r, double pitch, bool strict);
// Largest integer k >= 0 with (double)k * pitch < half, or -1.
long long band_threshold(double half, double pitch);

}  // namespace coro
