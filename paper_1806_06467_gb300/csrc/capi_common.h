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

// Base of every plan handle (Fresnel systems: kind 1, Lyot coronagraphs: kind 2).
struct coro_plan_s {
    virtual ~coro_plan_s() {}
    virtual int kind() const = 0;
    virtual int launches() const = 0;
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

// Twiddle table for n (built lazily on the context's stream).
const void* get_twiddles(coro_ctx ctx, int n, bool dbl, coro_status* st);


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
