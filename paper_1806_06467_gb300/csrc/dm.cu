// dm.cu -- deformable-mirror surface synthesis and its adjoint (Sec. 1.2: 32x32 / 48x48
// actuator DMs sampled with hundreds of pixels across the pupil).
//
//   OPD[b][y][x]  = scale * sum_{p,q} h[b][p][q] g(y_c - y_p) g(x_c - x_q)
//   grad[b][p][q] = scale * sum_{y,x} w[b][y][x] g(y_c - y_p) g(x_c - x_q)      (the transpose)
//
// with g(d) = exp(-d^2 / (2 sigma^2)), sigma = fwhm / (2 sqrt(2 ln 2)), pixel centres
// (x - n/2) * dx and actuator centres (q - (na - 1)/2) * pitch. g is separable, so a pixel only
// needs the actuators within the window where g exceeds 1e-20 of its peak (|d| < 9.6 sigma).
#include <cuda_runtime.h>

#include <cmath>

#include "capi_common.h"

namespace {

constexpr double kWindowSigmas = 9.6;     // exp(-9.6^2 / 2) = 1e-20

struct DmGeom {
    int n, na;
    float dx, pitch, inv2s2;              // inv2s2 = 1 / (2 sigma^2)
    int half_win;                         // actuators on each side of the nearest one
};

__device__ __forceinline__ float gauss(float d, float inv2s2) { return __expf(-d * d * inv2s2); }

// One thread per pixel; the (2w+1)^2 actuators around it.
__global__ void dm_opd_kernel(const float* __restrict__ h, DmGeom g, float scale, float* __restrict__ opd) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int b = blockIdx.z;
    if (x >= g.n) return;
    const float xc = (float)(x - g.n / 2) * g.dx, yc = (float)(y - g.n / 2) * g.dx;
    const float c0 = 0.5f * (float)(g.na - 1);
    const int qx = __float2int_rn(xc / g.pitch + c0), qy = __float2int_rn(yc / g.pitch + c0);
    const float* hb = h + (size_t)b * g.na * g.na;
    float acc = 0.f;
    for (int p = max(0, qy - g.half_win); p <= min(g.na - 1, qy + g.half_win); ++p) {
        const float gy = gauss(yc - ((float)p - c0) * g.pitch, g.inv2s2);
        float row = 0.f;
        for (int q = max(0, qx - g.half_win); q <= min(g.na - 1, qx + g.half_win); ++q)
            row = fmaf(hb[p * g.na + q], gauss(xc - ((float)q - c0) * g.pitch, g.inv2s2), row);
        acc = fmaf(gy, row, acc);
    }
    opd[((size_t)b * g.n + y) * g.n + x] = scale * acc;
}

// One block per actuator: sum over the pixels of its window, FP64 block reduction.
__global__ void dm_correlate_kernel(const float* __restrict__ w, DmGeom g, float scale, float* __restrict__ grad) {
    const int q = blockIdx.x, p = blockIdx.y, b = blockIdx.z;
    const float c0 = 0.5f * (float)(g.na - 1);
    const float xa = ((float)q - c0) * g.pitch, ya = ((float)p - c0) * g.pitch;
    const float reach = (float)(g.half_win + 1) * g.pitch;
    const int x0 = max(0, (int)floorf((xa - reach) / g.dx) + g.n / 2), x1 = min(g.n - 1, (int)ceilf((xa + reach) / g.dx) + g.n / 2);
    const int y0 = max(0, (int)floorf((ya - reach) / g.dx) + g.n / 2), y1 = min(g.n - 1, (int)ceilf((ya + reach) / g.dx) + g.n / 2);
    const int wx = x1 - x0 + 1, wy = y1 - y0 + 1;
    const float* wb = w + (size_t)b * g.n * g.n;
    double acc = 0.0;
    for (int i = threadIdx.x; i < wx * wy; i += blockDim.x) {
        const int x = x0 + i % wx, y = y0 + i / wx;
        const float xc = (float)(x - g.n / 2) * g.dx, yc = (float)(y - g.n / 2) * g.dx;
        acc += (double)(wb[(size_t)y * g.n + x] * gauss(xc - xa, g.inv2s2) * gauss(yc - ya, g.inv2s2));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) grad[((size_t)b * g.na + p) * g.na + q] = (float)(acc * scale);
    }
}

coro_status geom(const char* fn, int n, int na, double pitch, double fwhm, double dx, DmGeom* g) {
    if (n < 1 || n > 8192 || na < 1 || na > 1024) { coro::set_error("%s: n = %d, na = %d out of range", fn, n, na); return CORO_ESIZE; }
    if (!(pitch > 0) || !(fwhm > 0) || !(dx > 0)) { coro::set_error("%s: pitch, fwhm and pixelscale must be > 0", fn); return CORO_EINVAL; }
    const double sigma = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    g->n = n;
    g->na = na;
    g->dx = (float)dx;
    g->pitch = (float)pitch;
    g->inv2s2 = (float)(1.0 / (2.0 * sigma * sigma));
    g->half_win = (int)std::ceil(kWindowSigmas * sigma / pitch) + 1;
    return CORO_OK;
}

}  // namespace

extern "C" coro_status coro_dm_opd(coro_ctx ctx, const float* heights, int batch, int na, double pitch, double fwhm,
                                   int n, double pixelscale, double scale, float* opd) {
    coro::clear_error();
    if (!ctx || !heights || !opd) { coro::set_error("coro_dm_opd: NULL argument"); return CORO_EINVAL; }
    if (batch < 1 || batch > 65535) { coro::set_error("coro_dm_opd: batch %d", batch); return CORO_ESIZE; }
    DmGeom g;
    coro_status st = geom("coro_dm_opd", n, na, pitch, fwhm, pixelscale, &g);
    if (st != CORO_OK) return st;
    coro::DeviceGuard dg(ctx->device);
    dim3 grid((n + 127) / 128, n, batch);
    dm_opd_kernel<<<grid, 128, 0, ctx->stream>>>(heights, g, (float)scale, opd);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CORO_OK : coro::cuda_fail(e, "dm_opd_kernel");
}

extern "C" coro_status coro_dm_correlate(coro_ctx ctx, const float* w, int batch, int n, double pixelscale, int na,
                                         double pitch, double fwhm, double scale, float* grad) {
    coro::clear_error();
    if (!ctx || !w || !grad) { coro::set_error("coro_dm_correlate: NULL argument"); return CORO_EINVAL; }
    if (batch < 1 || batch > 65535) { coro::set_error("coro_dm_correlate: batch %d", batch); return CORO_ESIZE; }
    DmGeom g;
    coro_status st = geom("coro_dm_correlate", n, na, pitch, fwhm, pixelscale, &g);
    if (st != CORO_OK) return st;
    coro::DeviceGuard dg(ctx->device);
    dim3 grid(na, na, batch);
    dm_correlate_kernel<<<grid, 256, 0, ctx->stream>>>(w, g, (float)scale, grad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CORO_OK : coro::cuda_fail(e, "dm_correlate_kernel");
}
