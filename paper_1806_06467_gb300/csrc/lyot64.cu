// lyot64.cu -- the batched Lyot coronagraph at reference precision (CORO_MFT_FP64): complex128
// pupils, FP64 CUDA-core MFTs, the same chain and outputs as the split-precision plan,
//   E_B = MFT(E_A), E_C = E_A - MFT^-1(spot . E_B), E_D = E_C . stop, E_det = MFT(E_D),
//   I = |E_det|^2 / peak, S = sum of I over the dark hole,
// run item by item through the library's single calls (each item may have its own occulter
// size and pitches). The peak is the maximum of |E_det|^2 with the occulter removed. Used
// where the split-precision plan's FP32-class GEMM error (about 5e-10 in the dark hole) is too
// large: this path is exact to FP64 rounding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "capi_common.h"

using namespace coro;

namespace {

struct LyotPlan64 : coro_plan_s {
    coro_ctx ctx = nullptr;
    int device = 0;
    int batch = 0, n = 0, m_det = 0, m_occ_max = 0;
    double npix = 0, lyot_frac = 0;
    std::vector<coro_lyot_item> items;
    double2 *occ = nullptr, *pup = nullptr, *det = nullptr;   // work planes, one item each
    unsigned long long* pk = nullptr;                         // |E|^2 maximum as ordered bits
    double *part = nullptr, *dh = nullptr;                    // dark-hole partials, per-item sums
    int kind() const override { return 4; }
    int launches() const override { return 0; }
    int timing_units() const override { return 0; }
    ~LyotPlan64() override {
        DeviceGuard g(device);
        cudaDeviceSynchronize();
        for (void* q : {(void*)occ, (void*)pup, (void*)det, (void*)pk, (void*)part, (void*)dh})
            if (q) cudaFree(q);
    }
};

// out = max over the plane of |e|^2 (non-negative doubles order like their bit patterns).
__global__ void max_abs2_kernel(const double2* __restrict__ e, size_t n, unsigned long long* out) {
    double m = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = e[i];
        m = fmax(m, v.x * v.x + v.y * v.y);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

struct Wf {                           // a single-item complex128 wavefront with its own scalars
    double ps = 1.0, lam = 1.0;
    coro_wavefront w{};
    Wf(void* data, int n, double pitch) : ps(pitch) { w = coro_wavefront{data, CORO_C128, 1, n, &ps, &lam}; }
};

constexpr int kFinishBlocks = 304;

__device__ __forceinline__ long long centred_k2(size_t idx, int m) {
    const long long y = (long long)(idx / m) - m / 2, x = (long long)(idx % m) - m / 2;
    return x * x + y * y;
}

// Binary disk on an m x m plane: zero where (x - m/2)^2 + (y - m/2)^2 > thr (thr < 0: all zero).
// The spot keeps rho <= spot_radius, the Lyot stop r <= lyot_frac * D/2; thresholds come from
// the same exact integer test as the split-precision plan's epilogues.
__global__ void disk_mask_kernel(double2* __restrict__ e, int m, long long thr) {
    const size_t total = (size_t)m * m;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        if (centred_k2(i, m) > thr) e[i] = make_double2(0.0, 0.0);
}

// det holds -E_det: intensity |E|^2 / peak (float), field E_det, and per-block FP64 partial sums
// of the normalised intensity over lo <= k2 <= hi (the dark-hole annulus).
__global__ void finish_kernel(const double2* __restrict__ det, int m, double peak, long long lo, long long hi,
                              float* __restrict__ inten, double2* __restrict__ field, double* __restrict__ part) {
    const size_t total = (size_t)m * m;
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = det[i];
        const double I = (v.x * v.x + v.y * v.y) / peak;
        if (inten) inten[i] = (float)I;
        if (field) field[i] = make_double2(-v.x, -v.y);
        const long long k2 = centred_k2(i, m);
        if (k2 >= lo && k2 <= hi) acc += I;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// out = sum of part[0 .. count) in a fixed order (one warp).
__global__ void sum_parts_kernel(const double* __restrict__ part, int count, double* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += 32) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
}

int grid_for(size_t total) { return (int)std::min<size_t>((total + 255) / 256, kFinishBlocks); }

cudaError_t mask(cudaStream_t s, double2* e, int m, long long thr) {
    disk_mask_kernel<<<grid_for((size_t)m * m), 256, 0, s>>>(e, m, thr);
    return cudaGetLastError();
}

// E_det of item b in p->det (with the occulter: -E_det, the sign dropped by |.|^2 and fixed
// by finish_kernel where the field is returned).
coro_status item_chain(LyotPlan64* p, int b, const double2* e_a, bool occulter) {
    const coro_lyot_item& it = p->items[b];
    coro_ctx c = p->ctx;
    const int n = p->n;
    Wf a((void*)e_a, n, 1.0 / p->npix), pu(p->pup, n, 1.0 / p->npix), oc(p->occ, it.m_occ, it.du_occ),
        dt(p->det, p->m_det, it.du_det);
    coro_status st;
    cudaError_t e;
    if (occulter) {
        if ((st = coro_propagate_mft(c, &a.w, p->npix, -1, it.m_occ, &it.du_occ, CORO_MFT_FP64, &oc.w)) != CORO_OK) return st;
        if ((e = mask(c->stream, p->occ, it.m_occ, disk_threshold(it.spot_radius, it.du_occ, false))) != cudaSuccess)
            return cuda_fail(e, "lyot fp64: spot");
        if ((st = coro_propagate_mft(c, &oc.w, p->npix, +1, n, &it.du_occ, CORO_MFT_FP64, &pu.w)) != CORO_OK) return st;
        if ((st = coro_wavefront_axpy(c, -1.0, &a.w, &pu.w)) != CORO_OK) return st;   // pup = -E_C
    } else {
        e = cudaMemcpyAsync(p->pup, e_a, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lyot fp64: copy");
    }
    if ((e = mask(c->stream, p->pup, n, disk_threshold(0.5 * p->lyot_frac, 1.0 / p->npix, false))) != cudaSuccess)
        return cuda_fail(e, "lyot fp64: Lyot stop");
    return coro_propagate_mft(c, &pu.w, p->npix, -1, p->m_det, &it.du_det, CORO_MFT_FP64, &dt.w);
}

}  // namespace

namespace coro {

coro_status lyot64_create(coro_ctx ctx, const coro_lyot_desc* d, coro_plan* out) {
    DeviceGuard g(ctx->device);
    auto p = std::unique_ptr<LyotPlan64>(new (std::nothrow) LyotPlan64);
    if (!p) { set_error("out of host memory"); return CORO_ENOMEM; }
    p->ctx = ctx;
    p->device = ctx->device;
    p->batch = d->batch;
    p->n = d->n;
    p->m_det = d->m_det;
    p->npix = d->npix;
    p->lyot_frac = d->lyot_frac;
    p->items.assign(d->items, d->items + d->batch);
    for (const auto& it : p->items) p->m_occ_max = std::max(p->m_occ_max, it.m_occ);
    cudaError_t e = cudaMalloc(&p->occ, (size_t)p->m_occ_max * p->m_occ_max * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->pup, (size_t)p->n * p->n * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->det, (size_t)p->m_det * p->m_det * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->pk, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&p->part, sizeof(double) * kFinishBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&p->dh, sizeof(double) * p->batch);
    if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_create (FP64)");
    *out = p.release();
    return CORO_OK;
}

int lyot64_batch(coro_plan plan) { return static_cast<LyotPlan64*>(plan)->batch; }

coro_status lyot64_peak(coro_plan plan, const void* pupil, double* peak_out) {
    auto* p = static_cast<LyotPlan64*>(plan);
    DeviceGuard g(p->device);
    cudaStream_t s = p->ctx->stream;
    const size_t md2 = (size_t)p->m_det * p->m_det;
    for (int b = 0; b < p->batch; ++b) {
        coro_status st = item_chain(p, b, static_cast<const double2*>(pupil) + (size_t)b * p->n * p->n, false);
        if (st != CORO_OK) return st;
        unsigned long long bits = 0;
        cudaError_t e = cudaMemsetAsync(p->pk, 0, sizeof(bits), s);
        if (e == cudaSuccess) {
            max_abs2_kernel<<<(int)std::min<size_t>((md2 + 255) / 256, 1024), 256, 0, s>>>(p->det, md2, p->pk);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, p->pk, sizeof(bits), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_peak (FP64)");
        std::memcpy(&peak_out[b], &bits, sizeof(double));
    }
    return CORO_OK;
}

coro_status lyot64_execute(coro_plan plan, const void* pupil, const double* peak, float* intensity, void* field,
                           double* dh) {
    auto* p = static_cast<LyotPlan64*>(plan);
    DeviceGuard g(p->device);
    std::vector<double> pk(p->batch, 1.0);                // NULL peak: unnormalised
    coro_status st;
    if (peak) pk.assign(peak, peak + p->batch);
    const size_t md2 = (size_t)p->m_det * p->m_det;
    cudaStream_t s = p->ctx->stream;
    for (int b = 0; b < p->batch; ++b) {
        const coro_lyot_item& it = p->items[b];
        if ((st = item_chain(p, b, static_cast<const double2*>(pupil) + (size_t)b * p->n * p->n, true)) != CORO_OK)
            return st;
        const long long lo = disk_threshold(it.dh_in, it.du_det, true) + 1, hi = disk_threshold(it.dh_out, it.du_det, false);
        finish_kernel<<<grid_for(md2), 256, 0, s>>>(p->det, p->m_det, pk[b], lo, hi,
                                                    intensity ? intensity + b * md2 : nullptr,
                                                    field ? static_cast<double2*>(field) + b * md2 : nullptr, p->part);
        sum_parts_kernel<<<1, 32, 0, s>>>(p->part, grid_for(md2), p->dh + b);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_execute (FP64)");
    }
    if (dh) {
        cudaError_t e = cudaMemcpyAsync(dh, p->dh, sizeof(double) * p->batch, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_execute (FP64): dark-hole sums");
    }
    return CORO_OK;
}

}  // namespace coro
