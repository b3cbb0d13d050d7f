// noalloc.cu -- dark-hole sum that allocates nothing.
//
// For callers that cannot allocate device memory once they are running: a wavefront-control
// loop that must not take allocator latency or jitter between frames, a host application that
// hands the whole device heap to another framework, or a process whose memory budget is fixed
// at start-up. They keep their own field and host result buffer; the few words of scratch
// the reduction needs (per-item radius bounds, normalisation, accumulators) live in one
// file-scope device array of fixed size instead of a per-call allocation.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "capi_common.h"

namespace {

constexpr int kMaxBatch = CORO_NOALLOC_MAX_BATCH;

struct NoallocItem {
    long long lo, hi;       // integer r^2 bounds of the annulus
    double inv_norm;
    double acc;             // sum accumulated by the kernel (cleared by every call)
};

// The scratch: kMaxBatch items, 32 bytes each (32 KiB). Every GPU that loads the library
// holds it until the process exits.
static __device__ __align__(256) NoallocItem g_scratch[kMaxBatch];

// Per-device address of g_scratch as seen by host code, looked up once per device.
struct ScratchAddr {
    std::mutex mu;
    NoallocItem* ptr[64] = {};
};
ScratchAddr g_addr;

template <typename C>
__global__ void darkhole_noalloc_kernel(const C* __restrict__ e, int n, NoallocItem* __restrict__ items) {
    const int b = blockIdx.y;
    const long long lo = items[b].lo, hi = items[b].hi;
    const C* f = e + (size_t)b * n * n;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * n; i += gridDim.x * blockDim.x) {
        const long long kx = i % n - n / 2, ky = i / n - n / 2;
        const long long r2 = kx * kx + ky * ky;
        if (r2 >= lo && r2 <= hi) {
            const C v = f[i];
            s += (double)v.x * v.x + (double)v.y * v.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(&items[b].acc, s * items[b].inv_norm);
    }
}

}  // namespace

extern "C" coro_status coro_darkhole_sum_noalloc(const coro_wavefront* wf, const double* du, double r_in,
                                                 double r_out, const double* norm, void* stream, double* host_out) {
    coro::clear_error();
    if (!wf || !wf->data || !du || !host_out) {
        coro::set_error("coro_darkhole_sum_noalloc: wavefront, data, du or host_out is NULL");
        return CORO_EINVAL;
    }
    if (wf->dtype != CORO_C64 && wf->dtype != CORO_C128) { coro::set_error("coro_darkhole_sum_noalloc: bad dtype"); return CORO_EINVAL; }
    if (wf->n < 1 || wf->n > 8192) { coro::set_error("coro_darkhole_sum_noalloc: n = %d outside [1, 8192]", wf->n); return CORO_ESIZE; }
    if (wf->batch < 1 || wf->batch > kMaxBatch) {
        coro::set_error("coro_darkhole_sum_noalloc: batch %d exceeds the fixed scratch of %d items", wf->batch, kMaxBatch);
        return CORO_ESIZE;
    }
    if (!(r_in >= 0) || !(r_out >= r_in)) { coro::set_error("coro_darkhole_sum_noalloc: need 0 <= r_in <= r_out"); return CORO_EINVAL; }
    const int batch = wf->batch;
    std::vector<NoallocItem> items(batch);
    for (int b = 0; b < batch; ++b) {
        if (!(du[b] > 0)) { coro::set_error("coro_darkhole_sum_noalloc: du[%d] must be > 0", b); return CORO_EINVAL; }
        if (norm && !(norm[b] > 0)) { coro::set_error("coro_darkhole_sum_noalloc: norm[%d] must be > 0", b); return CORO_EINVAL; }
        items[b].lo = coro::disk_threshold(r_in, du[b], true) + 1;
        items[b].hi = coro::disk_threshold(r_out, du[b], false);
        items[b].inv_norm = norm ? 1.0 / norm[b] : 1.0;
        items[b].acc = 0.0;            // the array keeps the previous call's sums: restart from zero
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return coro::cuda_fail(e, "coro_darkhole_sum_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) { coro::set_error("coro_darkhole_sum_noalloc: device %d out of range", dev); return CORO_EINVAL; }
    {
        // the kernel runs on the current device with that device's scratch: the field must live there
        cudaPointerAttributes pa{};
        e = cudaPointerGetAttributes(&pa, wf->data);
        if (e != cudaSuccess) return coro::cuda_fail(e, "coro_darkhole_sum_noalloc: cudaPointerGetAttributes");
        if (pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered) {
            coro::set_error("coro_darkhole_sum_noalloc: the field is not in device memory");
            return CORO_EINVAL;
        }
        if (pa.type == cudaMemoryTypeDevice && pa.device != dev) {
            coro::set_error("coro_darkhole_sum_noalloc: the field is on device %d but device %d is current", pa.device, dev);
            return CORO_EINVAL;
        }
    }
    NoallocItem* ptr = nullptr;
    {
        // set-up, once per device, with that device current: the host-side name g_scratch
        // is not a device address, so ask the runtime for the real one
        std::lock_guard<std::mutex> lk(g_addr.mu);
        if (!g_addr.ptr[dev]) {
            e = cudaGetSymbolAddress((void**)&g_addr.ptr[dev], g_scratch);
            if (e != cudaSuccess) {
                g_addr.ptr[dev] = nullptr;
                return coro::cuda_fail(e, "coro_darkhole_sum_noalloc: cudaGetSymbolAddress");
            }
        }
        ptr = g_addr.ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(ptr, items.data(), batch * sizeof(NoallocItem), cudaMemcpyHostToDevice, s);
    const int n = wf->n;
    dim3 grid((unsigned)std::min(64, (n * n + 255) / 256), batch);
    if (e == cudaSuccess) {
        if (wf->dtype == CORO_C64) darkhole_noalloc_kernel<float2><<<grid, 256, 0, s>>>((const float2*)wf->data, n, ptr);
        else darkhole_noalloc_kernel<double2><<<grid, 256, 0, s>>>((const double2*)wf->data, n, ptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(items.data(), ptr, batch * sizeof(NoallocItem), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return coro::cuda_fail(e, "coro_darkhole_sum_noalloc");
    for (int b = 0; b < batch; ++b) host_out[b] = items[b].acc;
    return CORO_OK;
}
