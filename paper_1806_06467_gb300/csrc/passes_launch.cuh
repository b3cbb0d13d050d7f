// passes_launch.cuh -- instantiation and launch of the row/column pass kernels for one
// complex type. Included once per precision (passes_f32.cu, passes_f64.cu).
#pragma once
#include <cstring>

#include "passes.cuh"
#include "tc_gemm.cuh"

namespace coro {
namespace detail {

// Raise the dynamic shared-memory limit of a kernel once per device.
template <typename K>
inline cudaError_t ensure_smem(K kernel, size_t bytes, unsigned& done_mask) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned bit = 1u << (dev & 31);
    if (done_mask & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done_mask |= bit;
    return e;
}

// Persistent variant: as many resident blocks as fit, each streaming line groups.
template <typename C, int N>
cudaError_t row_launch_persistent(const RowArgs<C>& a, const PassLaunch& l) {
    using Cfg = PRowCfg<N>;
    static unsigned done = 0;
    static int per_sm[32] = {};
    const size_t smem = Cfg::template smem<C>();
    cudaError_t e = ensure_smem(row_pass_persistent_kernel<C, N>, smem, done);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int& occ = per_sm[dev & 31];
    if (occ == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, row_pass_persistent_kernel<C, N>, Cfg::THREADS, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
    }
    const int groups = l.batch * N / Cfg::L;
    const int grid = groups < sms * occ ? groups : sms * occ;
    row_pass_persistent_kernel<C, N><<<grid, Cfg::THREADS, smem, l.stream>>>(a, groups);
    return cudaGetLastError();
}

template <typename C, int N>
cudaError_t row_launch(const RowArgs<C>& a, const PassLaunch& l) {
    using Cfg = RowCfg<N>;
    static unsigned done = 0;
    // without a transform the shared exchange buffer is never touched
    const bool fft = a.flags & (RF_INV_FIRST | RF_FWD_AFTER);
    const size_t smem = fft ? (size_t)Cfg::L * Cfg::STRIDE * sizeof(C) : 0;
    cudaError_t e = ensure_smem(row_pass_kernel<C, N>, smem, done);
    if (e != cudaSuccess) return e;
    dim3 grid(N / Cfg::L, l.batch);
    row_pass_kernel<C, N><<<grid, Cfg::THREADS, smem, l.stream>>>(a);
    return cudaGetLastError();
}

template <typename C, int N, int L>
cudaError_t col_launch_persistent(const ColArgs<C>& a, const PassLaunch& l) {
    using Cfg = PColCfg<N, L>;
    static unsigned done = 0;
    static int per_sm[32] = {};
    const size_t smem = Cfg::template smem<C>();
    cudaError_t e = ensure_smem(col_pass_persistent_kernel<C, N, L>, smem, done);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int& occ = per_sm[dev & 31];
    if (occ == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, col_pass_persistent_kernel<C, N, L>, Cfg::THREADS, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
    }
    // in place: the same map serves the loads and the stores
    if (a.in != a.out) return cudaErrorInvalidValue;
    CUtensorMap map;
    if ((e = tc_make_field_map(a.in, N, (long long)l.batch * N, L, &map)) != cudaSuccess) return e;
    const int groups = l.batch * N / L;
    const int grid = groups < sms * occ ? groups : sms * occ;
    col_pass_persistent_kernel<C, N, L><<<grid, Cfg::THREADS, smem, l.stream>>>(a, map, groups);
    return cudaGetLastError();
}

template <typename C, int N, int L>
cudaError_t col_launch(const ColArgs<C>& a, const PassLaunch& l) {
    using Cfg = ColCfg<N, L>;
    static unsigned done = 0;
    const size_t smem = (size_t)L * Cfg::STRIDE * sizeof(C);
    cudaError_t e = ensure_smem(col_pass_kernel<C, N, L>, smem, done);
    if (e != cudaSuccess) return e;
    dim3 grid(N / L, l.batch);
    col_pass_kernel<C, N, L><<<grid, Cfg::THREADS, smem, l.stream>>>(a);
    return cudaGetLastError();
}

// Unit-pipelined passes: one block per SM (as many SMs as there are groups).
inline cudaError_t sm_count(int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    return e;
}

template <typename C, int N, int L, int U, int S>
cudaError_t col_launch_units(const ColArgs<C>& a, const PassLaunch& l) {
    using Cfg = UColCfg<N, L, U, S>;
    static unsigned done = 0;
    const size_t smem = Cfg::template smem<C>();
    cudaError_t e = ensure_smem(col_pass_units_kernel<C, N, L, U, S>, smem, done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = sm_count(&sms)) != cudaSuccess) return e;
    if (a.in != a.out) return cudaErrorInvalidValue;   // one tensor map serves loads and stores
    CUtensorMap map;
    if ((e = tc_make_field_map(a.in, N, (long long)l.batch * N, L, &map)) != cudaSuccess) return e;
    const int groups = l.batch * N / L;
    const int grid = groups < sms ? groups : sms;
    col_pass_units_kernel<C, N, L, U, S><<<grid, Cfg::THREADS, smem, l.stream>>>(a, map, groups);
    return cudaGetLastError();
}

// TOUT: out-of-place, the result transposed (out[b][x][y]).
template <int N, int U, int S, bool TOUT = false>
cudaError_t col_launch_pair(const ColArgs<float2>& a, const PassLaunch& l) {
    using Cfg = PColPairCfg<N, U, S>;
    static unsigned done = 0;
    const size_t smem = Cfg::template smem<float2>();
    cudaError_t e = ensure_smem(col_pass_pair_kernel<N, U, S, TOUT>, smem, done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = sm_count(&sms)) != cudaSuccess) return e;
    if ((a.in != a.out) != TOUT) return cudaErrorInvalidValue;
    CUtensorMap map;
    if ((e = tc_make_field_map(a.in, N, (long long)l.batch * N, 2, &map)) != cudaSuccess) return e;
    const int groups = l.batch * N / 2;
    const int grid = groups < sms ? groups : sms;
    col_pass_pair_kernel<N, U, S, TOUT><<<grid, Cfg::THREADS, smem, l.stream>>>(a, map, groups);
    return cudaGetLastError();
}

template <int N>
cudaError_t col_launch_quad(const ColArgs<float2>& a, const PassLaunch& l) {
    using Cfg = QColCfg<N>;
    static unsigned done = 0;
    const size_t smem = Cfg::smem();
    cudaError_t e = ensure_smem(col_pass_quad_kernel<N>, smem, done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = sm_count(&sms)) != cudaSuccess) return e;
    if (a.in != a.out) return cudaErrorInvalidValue;   // one tensor map serves loads and stores
    CUtensorMap map;
    if ((e = tc_make_field_map(a.in, N, (long long)l.batch * N, 4, &map)) != cudaSuccess) return e;
    static int occ = 0;
    if (occ == 0) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, col_pass_quad_kernel<N>, Cfg::THREADS, smem)) != cudaSuccess)
            return e;
        if (occ < 1) occ = 1;
    }
    const int strips = l.batch * N / 4;
    const int grid = strips < sms * occ ? strips : sms * occ;
    col_pass_quad_kernel<N><<<grid, Cfg::THREADS, smem, l.stream>>>(a, map, strips);
    return cudaGetLastError();
}

template <int N>
cudaError_t col_launch_wide(const ColArgs<float2>& a, const PassLaunch& l) {
    using Cfg = WColCfg<N>;
    static unsigned done = 0;
    const size_t smem = Cfg::smem();
    cudaError_t e = ensure_smem(col_pass_wide_kernel<N>, smem, done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = sm_count(&sms)) != cudaSuccess) return e;
    if (a.in != a.out) return cudaErrorInvalidValue;   // one tensor map serves loads and stores
    CUtensorMap map;
    if ((e = tc_make_field_map(a.in, N, (long long)l.batch * N, 4, &map)) != cudaSuccess) return e;
    static int occ = 0;
    if (occ == 0) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, col_pass_wide_kernel<N>, Cfg::THREADS, smem)) != cudaSuccess)
            return e;
        if (occ < 1) occ = 1;
    }
    const int groups = l.batch * N / 4;
    const int grid = groups < sms * occ ? groups : sms * occ;
    col_pass_wide_kernel<N><<<grid, Cfg::THREADS, smem, l.stream>>>(a, map, groups);
    return cudaGetLastError();
}

template <typename C, int N, int U, int S>
cudaError_t row_launch_units(const RowArgs<C>& a, const PassLaunch& l) {
    using Cfg = URowCfg<N, U, S>;
    static unsigned done = 0;
    const size_t smem = Cfg::template smem<C>();
    cudaError_t e = ensure_smem(row_pass_units_kernel<C, N, U, S>, smem, done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = sm_count(&sms)) != cudaSuccess) return e;
    const int rows = l.batch * N;
    const int grid = rows < sms ? rows : sms;
    row_pass_units_kernel<C, N, U, S><<<grid, Cfg::THREADS, smem, l.stream>>>(a, rows);
    return cudaGetLastError();
}

template <int N, int U, int S, bool TIN = false>
cudaError_t row_launch_pair(const RowArgs<float2>& a, const PassLaunch& l) {
    using Cfg = PRowPairCfg<N, U, S>;
    static unsigned done = 0;
    const size_t smem = Cfg::smem();
    cudaError_t e = ensure_smem(row_pass_pair_kernel<N, U, S, TIN>, smem, done);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if ((e = sm_count(&sms)) != cudaSuccess) return e;
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    if constexpr (TIN) {                    // out-of-place; input transposed (in[b][x][y])
        if (a.in == a.out || (a.flags & RF_INIT_ONE)) return cudaErrorInvalidValue;
        if ((e = tc_make_field_map(a.in, N, (long long)l.batch * N, 2, &map)) != cudaSuccess) return e;
    }
    const int pairs = l.batch * N / 2;
    const int grid = pairs < sms ? pairs : sms;
    row_pass_pair_kernel<N, U, S, TIN><<<grid, Cfg::THREADS, smem, l.stream>>>(a, map, pairs);
    return cudaGetLastError();
}

}  // namespace detail
}  // namespace coro
