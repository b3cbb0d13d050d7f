// cgemm_simt.cu -- CUDA-core batched complex GEMMs: FP32 (the CORO_MFT_FP32 path of the MFT)
// and FP64 on complex128 fields (CORO_MFT_FP64).
// 64 x 64 output tile per block, 16-deep k slices staged in shared memory, each thread a
// 4 x 4 block of complex outputs at stride 16 (conflict-free shared reads, coalesced stores).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/coro.h"
#include "mft_gemm.cuh"

namespace coro {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// splits > 1: split K as in zgemm_simt_kernel below (partials in part[s][b][m][n]).
__global__ void __launch_bounds__(256) cgemm_simt_kernel(const GemmDesc g, int splits, int kc, float2* part) {
    __shared__ float2 As[BK][BM];
    __shared__ float2 Bs[BK][BN];
    const int b = blockIdx.z / splits, sp = blockIdx.z % splits;
    const int k_lo = sp * kc, k_hi = min(g.K, k_lo + kc);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const float2* A = g.A + b * g.sA;
    const float2* B = g.B + b * g.sB;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
        // 1024 samples of each tile, 4 per thread
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = threadIdx.x + r * 256;
            int mm, kk;
            if (g.a_trans) { mm = idx % BM; kk = idx / BM; } else { kk = idx % BK; mm = idx / BK; }
            const int gm = m0 + mm, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gm < g.M && gk < k_hi) v = g.a_trans ? A[(size_t)gk * g.lda + gm] : A[(size_t)gm * g.lda + gk];
            As[kk][mm] = v;
            int nn;
            if (g.b_trans) { kk = idx % BK; nn = idx / BK; } else { nn = idx % BN; kk = idx / BN; }
            const int gn = n0 + nn, gk2 = k0 + kk;
            float2 w = make_float2(0.f, 0.f);
            if (gn < g.N && gk2 < k_hi) w = g.b_trans ? B[(size_t)gn * g.ldb + gk2] : B[(size_t)gk2 * g.ldb + gn];
            Bs[kk][nn] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float2 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(a[i].x, bb[j].x, acc[i][j].x);
                    acc[i][j].x = fmaf(-a[i].y, bb[j].y, acc[i][j].x);
                    acc[i][j].y = fmaf(a[i].x, bb[j].y, acc[i][j].y);
                    acc[i][j].y = fmaf(a[i].y, bb[j].x, acc[i][j].y);
                }
        }
        __syncthreads();
    }
    const bool direct = splits == 1;
    const float s = !direct ? 1.f : g.scale_per_item ? g.scale_per_item[b] : g.alpha;
    float2* C = direct ? g.C + b * g.sC : part + ((size_t)sp * gridDim.z / splits + b) * g.M * g.N;
    const int ldc = direct ? g.ldc : g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn < g.N) C[(size_t)gm * ldc + gn] = make_float2(acc[i][j].x * s, acc[i][j].y * s);
        }
    }
}

__global__ void creduce_kernel(const GemmDesc g, int batch, int splits, const float2* __restrict__ part) {
    const size_t mn = (size_t)g.M * g.N, total = mn * batch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / mn);
        const size_t r = i - (size_t)b * mn;
        const int m = (int)(r / g.N), n = (int)(r - (size_t)m * g.N);
        float2 acc = part[i];
        for (int sp = 1; sp < splits; ++sp) {
            const float2 v = part[(size_t)sp * total + i];
            acc.x += v.x;
            acc.y += v.y;
        }
        const float sc = g.scale_per_item ? g.scale_per_item[b] : g.alpha;
        g.C[b * g.sC + (size_t)m * g.ldc + n] = make_float2(acc.x * sc, acc.y * sc);
    }
}



// FP64 complex GEMM: 64 x 64 output tile, 8-deep k slices, each thread 4 x 4 outputs. With
// splits > 1 (split K: the MFT's products have few output tiles and a long K, and FP64 FMAs
// are scarce, so every SM needs blocks) block z = b * splits + s covers k in
// [s kc, (s + 1) kc) and writes its unscaled partial sum to part[s][b][m][n]; zreduce_kernel
// adds the partials in split order.
constexpr int ZBK = 8;

__global__ void __launch_bounds__(256) zgemm_simt_kernel(const ZGemmDesc g, int splits, int kc, double2* part) {
    __shared__ double2 As[ZBK][BM];
    __shared__ double2 Bs[ZBK][BN];
    const int b = blockIdx.z / splits, sp = blockIdx.z % splits;
    const int k_lo = sp * kc, k_hi = min(g.K, k_lo + kc);
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const double2* A = g.A + b * g.sA;
    const double2* B = g.B + b * g.sB;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

    for (int k0 = k_lo; k0 < k_hi; k0 += ZBK) {
        // 512 samples of each tile, 2 per thread
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = threadIdx.x + r * 256;
            int mm, kk;
            if (g.a_trans) { mm = idx % BM; kk = idx / BM; } else { kk = idx % ZBK; mm = idx / ZBK; }
            const int gm = m0 + mm, gk = k0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (gm < g.M && gk < k_hi) v = g.a_trans ? A[(size_t)gk * g.lda + gm] : A[(size_t)gm * g.lda + gk];
            As[kk][mm] = v;
            int nn;
            if (g.b_trans) { kk = idx % ZBK; nn = idx / ZBK; } else { nn = idx % BN; kk = idx / BN; }
            const int gn = n0 + nn, gk2 = k0 + kk;
            double2 w = make_double2(0.0, 0.0);
            if (gn < g.N && gk2 < k_hi) w = g.b_trans ? B[(size_t)gn * g.ldb + gk2] : B[(size_t)gk2 * g.ldb + gn];
            Bs[kk][nn] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < ZBK; ++k) {
            double2 a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fma(a[i].x, bb[j].x, acc[i][j].x);
                    acc[i][j].x = fma(-a[i].y, bb[j].y, acc[i][j].x);
                    acc[i][j].y = fma(a[i].x, bb[j].y, acc[i][j].y);
                    acc[i][j].y = fma(a[i].y, bb[j].x, acc[i][j].y);
                }
        }
        __syncthreads();
    }
    const bool direct = splits == 1;
    const double s = !direct ? 1.0 : g.scale_per_item ? g.scale_per_item[b] : g.alpha;
    double2* C = direct ? g.C + b * g.sC : part + ((size_t)sp * gridDim.z / splits + b) * g.M * g.N;
    const int ldc = direct ? g.ldc : g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn < g.N) C[(size_t)gm * ldc + gn] = make_double2(acc[i][j].x * s, acc[i][j].y * s);
        }
    }
}

// C[b][m][n] = scale_b * sum_s part[s][b][m][n], the partials added in split order.
__global__ void zreduce_kernel(const ZGemmDesc g, int batch, int splits, const double2* __restrict__ part) {
    const size_t mn = (size_t)g.M * g.N, total = mn * batch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / mn);
        const size_t r = i - (size_t)b * mn;
        const int m = (int)(r / g.N), n = (int)(r - (size_t)m * g.N);
        double2 acc = part[i];
        for (int sp = 1; sp < splits; ++sp) {
            const double2 v = part[(size_t)sp * total + i];
            acc.x += v.x;
            acc.y += v.y;
        }
        const double sc = g.scale_per_item ? g.scale_per_item[b] : g.alpha;
        g.C[b * g.sC + (size_t)m * g.ldc + n] = make_double2(acc.x * sc, acc.y * sc);
    }
}

}  // namespace

namespace {

// Split of K for a GEMM with `tiles` output tiles: enough splits (of at least 32 of K, a
// multiple of `step`) for the blocks to fill `per_sm` resident slots on every SM.
cudaError_t split_k(long long tiles, int per_sm, int K, int step, int* splits, int* kc) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)per_sm * sms;
    int s = tiles >= slots ? 1 : (int)(slots / tiles);
    s = std::max(1, std::min(s, K / 32));
    *kc = ((K + s - 1) / s + step - 1) / step * step;
    *splits = (K + *kc - 1) / *kc;
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_zgemm(const ZGemmDesc& g, int batch, cudaStream_t stream) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batch);
    int splits = 1, kc = g.K;
    cudaError_t e = split_k((long long)grid.x * grid.y * batch, 2, g.K, ZBK, &splits, &kc);   // two blocks per SM
    if (e != cudaSuccess) return e;
    if (splits == 1) {
        zgemm_simt_kernel<<<grid, 256, 0, stream>>>(g, 1, g.K, nullptr);
        return cudaGetLastError();
    }
    const size_t total = (size_t)g.M * g.N * batch;
    double2* part = nullptr;
    if ((e = cudaMallocAsync(&part, total * splits * sizeof(double2), stream)) != cudaSuccess) return e;
    grid.z = batch * splits;
    zgemm_simt_kernel<<<grid, 256, 0, stream>>>(g, splits, kc, part);
    zreduce_kernel<<<(int)std::min<size_t>((total + 255) / 256, 4096), 256, 0, stream>>>(g, batch, splits, part);
    e = cudaGetLastError();
    const cudaError_t f = cudaFreeAsync(part, stream);
    return e != cudaSuccess ? e : f;
}

cudaError_t launch_cgemm(const GemmDesc& g, int batch, int precision, cudaStream_t stream) {
    if (precision != CORO_MFT_FP32) return cudaErrorNotSupported;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batch);
    int splits = 1, kc = g.K;
    cudaError_t e = split_k((long long)grid.x * grid.y * batch, 4, g.K, BK, &splits, &kc);    // four blocks per SM
    if (e != cudaSuccess) return e;
    if (splits == 1) {
        cgemm_simt_kernel<<<grid, 256, 0, stream>>>(g, 1, g.K, nullptr);
        return cudaGetLastError();
    }
    const size_t total = (size_t)g.M * g.N * batch;
    float2* part = nullptr;
    if ((e = cudaMallocAsync(&part, total * splits * sizeof(float2), stream)) != cudaSuccess) return e;
    grid.z = batch * splits;
    cgemm_simt_kernel<<<grid, 256, 0, stream>>>(g, splits, kc, part);
    creduce_kernel<<<(int)std::min<size_t>((total + 255) / 256, 4096), 256, 0, stream>>>(g, batch, splits, part);
    e = cudaGetLastError();
    const cudaError_t f = cudaFreeAsync(part, stream);
    return e != cudaSuccess ? e : f;
}

}  // namespace coro
