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

// ---------------------------------------------------------------------------- tiled forms
// Both sums are separable, so a tile of pixels shares its actuator rows and a block per
// actuator row shares its pixel rows. The windows are those of the per-pixel kernels above
// (pixel (x, y) sees actuator (p, q) iff |q - q(x)| <= hw and |p - p(y)| <= hw, q(x) the
// nearest actuator), so the two-step correlation is the exact transpose of dm_opd_tile, and
// dm_opd_tile reproduces dm_opd_kernel bit for bit (same products, same order).

constexpr int kTileX = 256;

__device__ __forceinline__ int nearest_act(float c, float pitch, float c0) { return __float2int_rn(c / pitch + c0); }

// grid (ceil(n / 256), ceil(n / ty), batch), 256 threads; shared T[pcap][256], gy[ty][pcap].
// T[p][x] = sum_q h[p][q] g(x - x_q) for the tile's actuator rows, then each pixel sums its
// own window of rows p with weights g(y - y_p).
__global__ void __launch_bounds__(kTileX)
dm_opd_tile(const float* __restrict__ h, DmGeom g, float scale, int ty, int pcap, float* __restrict__ opd) {
    extern __shared__ float dsm[];
    float* Ts = dsm;
    float* gys = dsm + pcap * kTileX;
    const int tid = threadIdx.x;
    const int x = blockIdx.x * kTileX + tid;
    const int y0 = blockIdx.y * ty, b = blockIdx.z;
    const int y1 = min(g.n, y0 + ty) - 1;
    const float c0 = 0.5f * (float)(g.na - 1);
    const int pmin = max(0, nearest_act((float)(y0 - g.n / 2) * g.dx, g.pitch, c0) - g.half_win);
    const int pmax = min(min(g.na - 1, nearest_act((float)(y1 - g.n / 2) * g.dx, g.pitch, c0) + g.half_win),
                         pmin + pcap - 1);
    const int P = pmax - pmin + 1;
    float* ob = opd + (size_t)b * g.n * g.n;
    if (P <= 0) {                                   // no actuator reaches these rows
        if (x < g.n)
            for (int y = y0; y <= y1; ++y) ob[(size_t)y * g.n + x] = 0.f;
        return;
    }
    const float* hb = h + (size_t)b * g.na * g.na;
    const float xc = (float)(x - g.n / 2) * g.dx;
    const int qx = nearest_act(xc, g.pitch, c0);
    for (int pp = 0; pp < P; ++pp) Ts[pp * kTileX + tid] = 0.f;
    if (x < g.n) {
        for (int q = max(0, qx - g.half_win); q <= min(g.na - 1, qx + g.half_win); ++q) {
            const float gx = gauss(xc - ((float)q - c0) * g.pitch, g.inv2s2);
            for (int pp = 0; pp < P; ++pp)
                Ts[pp * kTileX + tid] = fmaf(hb[(pmin + pp) * g.na + q], gx, Ts[pp * kTileX + tid]);
        }
    }
    for (int i = tid; i < ty * P; i += kTileX) {
        const int r = i / P, pp = i % P;
        const float yc = (float)(y0 + r - g.n / 2) * g.dx;
        gys[r * pcap + pp] = gauss(yc - ((float)(pmin + pp) - c0) * g.pitch, g.inv2s2);
    }
    __syncthreads();
    if (x >= g.n) return;
    for (int y = y0; y <= y1; ++y) {
        const int r = y - y0;
        const int qy = nearest_act((float)(y - g.n / 2) * g.dx, g.pitch, c0);
        float acc = 0.f;
        for (int p = max(pmin, qy - g.half_win); p <= min(pmax, qy + g.half_win); ++p)
            acc = fmaf(gys[r * pcap + p - pmin], Ts[(p - pmin) * kTileX + tid], acc);
        ob[(size_t)y * g.n + x] = scale * acc;
    }
}

// Pixel window of actuator column q (or row p): candidates xs(q) .. xs(q) + len - 1.
__device__ __forceinline__ int window_start(int a, const DmGeom& g, float c0) {
    const float xa = ((float)a - c0) * g.pitch;
    return (int)floorf((xa - (float)(g.half_win + 1) * g.pitch) / g.dx) + g.n / 2;
}

// The transpose in two steps, U[b][y][q] = sum_{x in X(q)} w[b][y][x] g(x - x_q) for the rows
// the actuators reach, then grad[b][p][q] = scale * sum_{y in Y(p)} g(y - y_p) U[b][y][q].
// Pixel windows start at xs(q) = window_start(q) and span len candidates; gx[q][k] holds
// g(x - x_q) for x = xs(q) + k inside the window (zero elsewhere). Rows run over the union
// of the row windows, y = ys0 + r, r < span.

// gx table, one thread per entry; also the window starts xs[q], which the next two kernels
// read instead of recomputing them (a recomputation compiled with other contractions could
// round to the next pixel and misalign the windows).
__global__ void dm_gx_table(DmGeom g, int len, float* __restrict__ gx, int* __restrict__ xs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.na * len) return;
    const float c0 = 0.5f * (float)(g.na - 1);
    const int q = i / len, x0 = window_start(q, g, c0), x = x0 + i % len;
    if (i % len == 0) xs[q] = x0;
    const float xc = (float)(x - g.n / 2) * g.dx;
    const bool in = x >= 0 && x < g.n && abs(nearest_act(xc, g.pitch, c0) - q) <= g.half_win;
    gx[i] = in ? gauss(xc - ((float)q - c0) * g.pitch, g.inv2s2) : 0.f;
}

// grid (ceil(span / 8), batch), 256 threads: one warp per row, all na columns of U. Shared:
// each warp's row over the union of the windows (span); the gx table is read through L1.
__global__ void __launch_bounds__(256)
dm_correlate_u(const float* __restrict__ w, DmGeom g, int len, int span, const float* __restrict__ gx,
               const int* __restrict__ xs_tab, float* __restrict__ U) {
    extern __shared__ float usm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* row = usm + (size_t)warp * span;
    const int r = blockIdx.x * 8 + warp, b = blockIdx.y;
    if (r >= span) return;                                   // warps are independent
    const int xs0 = xs_tab[0];
    const int y = xs0 + r;
    float* ub = U + ((size_t)b * span + r) * g.na;
    if (y < 0 || y >= g.n) {
        for (int q = lane; q < g.na; q += 32) ub[q] = 0.f;
        return;
    }
    const float* wr = w + ((size_t)b * g.n + y) * g.n;
#pragma unroll 4
    for (int i = lane; i < span; i += 32) {
        const int x = xs0 + i;
        row[i] = (x >= 0 && x < g.n) ? __ldg(wr + x) : 0.f;
    }
    __syncwarp();
    // 32 columns q at a time: every lane sums its strided share of each column's window
    // (p[j] for q = q0 + j), then a transposing butterfly (16 + 8 + 4 + 2 + 1 shuffles)
    // leaves lane j with the total of column q0 + j
    for (int q0 = 0; q0 < g.na; q0 += 32) {
        float p[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int q = q0 + j;
            float acc = 0.f;
            if (q < g.na) {
                const int off = xs_tab[q] - xs0;
                const int kend = min(len, span - off);
                const float* gq = gx + (size_t)q * len;
                for (int k = lane; k < kend; k += 32) acc = fmaf(row[off + k], __ldg(gq + k), acc);
            }
            p[j] = acc;
        }
#pragma unroll
        for (int wdt = 16; wdt >= 1; wdt >>= 1) {
            const bool upper = lane & wdt;
#pragma unroll
            for (int j = 0; j < wdt; ++j) {
                const float send = upper ? p[j] : p[j + wdt];
                const float keep = upper ? p[j + wdt] : p[j];
                p[j] = keep + __shfl_xor_sync(0xffffffffu, send, wdt);
            }
        }
        if (q0 + lane < g.na) ub[q0 + lane] = p[0];
    }
}

// grid (na, batch), 256 threads: block = actuator row p of map b. Warp j takes the rows
// y = ys + j, ys + j + 8, ..., lanes the columns q; the eight warps' FP32 partial sums are
// added in FP64 in warp order.
__global__ void __launch_bounds__(256)
dm_correlate_p(const float* __restrict__ U, const int* __restrict__ xs_tab, DmGeom g, int len, int span,
               float scale, float* __restrict__ grad) {
    __shared__ float part[8][64];
    const int p = blockIdx.x, b = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float c0 = 0.5f * (float)(g.na - 1);
    const int ys0 = xs_tab[0], ys = xs_tab[p];
    const float yp = ((float)p - c0) * g.pitch;
    for (int q0 = 0; q0 < g.na; q0 += 64) {
        float acc0 = 0.f, acc1 = 0.f;
        for (int y = max(0, ys) + warp; y < min(g.n, ys + len); y += 8) {
            const int r = y - ys0;
            if (r < 0 || r >= span) continue;
            const float yc = (float)(y - g.n / 2) * g.dx;
            if (abs(nearest_act(yc, g.pitch, c0) - p) > g.half_win) continue;
            const float gy = gauss(yc - yp, g.inv2s2);
            const float* ur = U + ((size_t)b * span + r) * g.na;
            if (q0 + lane < g.na) acc0 = fmaf(gy, ur[q0 + lane], acc0);
            if (q0 + 32 + lane < g.na) acc1 = fmaf(gy, ur[q0 + 32 + lane], acc1);
        }
        part[warp][lane] = acc0;
        part[warp][32 + lane] = acc1;
        __syncthreads();
        if (threadIdx.x < 64 && q0 + threadIdx.x < g.na) {
            double t = 0.0;
            for (int j = 0; j < 8; ++j) t += (double)part[j][threadIdx.x];
            grad[((size_t)b * g.na + p) * g.na + q0 + threadIdx.x] = (float)(t * scale);
        }
        __syncthreads();
    }
}

// Host side: tile height for dm_opd_tile (0 = use the per-pixel kernel) and its row cap.
int opd_tile_rows(const DmGeom& g, double dx, double pitch, int* pcap) {
    for (int ty : {16, 8, 4, 2, 1}) {
        const int cap = (int)std::ceil((ty - 1) * dx / pitch) + 2 * g.half_win + 4;
        if (cap <= 32) { *pcap = cap; return ty; }
    }
    return 0;
}

// Candidate window length, the number of rows of U (the union of the row windows) and the
// shared bytes of dm_correlate_u for the two-step transpose; 0 when they would not fit (then
// the per-actuator kernel).
size_t correlate_sizes(const DmGeom& g, double dx, double pitch, int* len, int* span) {
    const double l = 2.0 * std::ceil((g.half_win + 1) * pitch / dx) + 3;
    const double sp = std::ceil((g.na - 1) * pitch / dx) + l + 4;
    if (l > 65536 || sp > 65536) return 0;
    *len = (int)l;
    *span = (int)sp;
    const size_t bytes = 8 * (size_t)*span * sizeof(float);
    return bytes <= 200 * 1024 ? bytes : 0;
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
    int pcap = 0;
    const int ty = opd_tile_rows(g, pixelscale, pitch, &pcap);
    if (ty > 0) {
        dim3 grid((n + kTileX - 1) / kTileX, (n + ty - 1) / ty, batch);
        const size_t smem = (size_t)pcap * (kTileX + ty) * sizeof(float);
        dm_opd_tile<<<grid, kTileX, smem, ctx->stream>>>(heights, g, (float)scale, ty, pcap, opd);
    } else {
        dim3 grid((n + 127) / 128, n, batch);
        dm_opd_kernel<<<grid, 128, 0, ctx->stream>>>(heights, g, (float)scale, opd);
    }
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
    int len = 0, span = 0;
    cudaError_t e = cudaSuccess;
    const size_t usmem = na <= 1024 ? correlate_sizes(g, pixelscale, pitch, &len, &span) : 0;
    if (usmem > 48 * 1024) e = cudaFuncSetAttribute(dm_correlate_u, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usmem);
    if (e != cudaSuccess) return coro::cuda_fail(e, "coro_dm_correlate: shared memory");
    if (usmem > 0) {
        // scratch: the gx table and U, stream-ordered
        const size_t xs_bytes = ((size_t)na * sizeof(int) + 255) / 256 * 256;
        const size_t gx_bytes = ((size_t)na * len * sizeof(float) + 255) / 256 * 256;
        const size_t u_bytes = (size_t)batch * span * na * sizeof(float);
        void* scratch = nullptr;
        e = cudaMallocAsync(&scratch, xs_bytes + gx_bytes + u_bytes, ctx->stream);
        if (e != cudaSuccess) return coro::cuda_fail(e, "coro_dm_correlate: scratch");
        int* xs = static_cast<int*>(scratch);
        float* gx = reinterpret_cast<float*>(static_cast<char*>(scratch) + xs_bytes);
        float* U = reinterpret_cast<float*>(static_cast<char*>(scratch) + xs_bytes + gx_bytes);
        dm_gx_table<<<(na * len + 255) / 256, 256, 0, ctx->stream>>>(g, len, gx, xs);
        dm_correlate_u<<<dim3((span + 7) / 8, batch), 256, usmem, ctx->stream>>>(w, g, len, span, gx, xs, U);
        dm_correlate_p<<<dim3(na, batch), 256, 0, ctx->stream>>>(U, xs, g, len, span, (float)scale, grad);
        e = cudaGetLastError();
        const cudaError_t f = cudaFreeAsync(scratch, ctx->stream);
        if (e == cudaSuccess) e = f;
    } else {
        dim3 grid(na, na, batch);
        dm_correlate_kernel<<<grid, 256, 0, ctx->stream>>>(w, g, (float)scale, grad);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? CORO_OK : coro::cuda_fail(e, "dm_correlate_kernel");
}
