// mft.cu -- matrix Fourier transform (Sec. 1.1: the semi-analytic coronagraph method of
// Soummer et al. uses "discrete matrix Fourier transforms of modest sized arrays"; Sec. 2.3:
// the "sines and cosines ... needed in the matrix DFT").
//
//   out = s * A_y . in . A_x^T,   A[u][j] = exp(-+ 2 pi i X_j U_u)
//
// evaluated as two batched complex GEMMs. The bases are generated on the device in FP64
// (the phase X_j U_u = j' u' du / npix is an exact integer times one FP64 constant, reduced
// to its fractional cycle before sincospi) and rounded to complex64.
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>
#include <vector>

#include "capi_common.h"
#include "fft_engine.cuh"
#include "mft_gemm.cuh"
#include "tc_gemm.cuh"
#include "tcx_gemm.cuh"

using namespace coro;

namespace {

// basis[b][u][j] = exp(sign 2 pi i (j - n/2)(u - m/2) c_b), c_b = du_b / npix.
template <typename C>
__global__ void mft_basis_kernel(C* basis, int m, int n, const double* __restrict__ c, int sign) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int u = blockIdx.y;
    const int b = blockIdx.z;
    if (j >= n) return;
    const long long jj = (long long)j - n / 2, uu = (long long)u - m / 2;
    double cyc = (double)(jj * uu) * c[b];
    cyc -= rint(cyc);
    double s, co;
    sincospi(2.0 * cyc, &s, &co);
    if (sign < 0) s = -s;
    using R = typename real_of<C>::type;
    basis[((size_t)b * m + u) * n + j] = mk<C>((R)co, (R)s);
}

coro_status check_mft_wf(const char* fn, const coro_wavefront* wf) {
    if (!wf || !wf->data) { coro::set_error("%s: wavefront or data is NULL", fn); return CORO_EINVAL; }
    if (wf->dtype != CORO_C64 && wf->dtype != CORO_C128) { coro::set_error("%s: bad dtype %d", fn, wf->dtype); return CORO_EINVAL; }
    if (wf->batch < 1 || wf->batch > 65535) { coro::set_error("%s: batch %d", fn, wf->batch); return CORO_ESIZE; }
    if (wf->n < 1 || wf->n > 8192) { coro::set_error("%s: size %d outside [1, 8192]", fn, wf->n); return CORO_ESIZE; }
    return CORO_OK;
}

// Split-precision tensor-core MFT: Y1 = X . W^T written transposed and split, then
// out = s (Y1^T . W^T)^T, with W[r][k] = exp(-+2 pi i r' k' du/npix) the MFT basis.
coro_status mft_tensor_core(coro_ctx ctx, const coro_wavefront* in, int direction, int m, const std::vector<double>& c,
                            bool bf16, coro_wavefront* out) {
    coro_status st = CORO_OK;
    const int batch = in->batch;
    const int nin = in->n;                       // X1 rows = cols
    const int nout = m;                          // W rows, output size
    const size_t es = tc_elem_size(bf16);
    const int ld = tc_ld(nin, bf16);
    const size_t x_bytes = (size_t)4 * batch * nin * ld * es;
    const size_t w_bytes = (size_t)4 * batch * nout * ld * es;
    const size_t z_bytes = w_bytes;
    auto align = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
    unsigned char* work = (unsigned char*)coro::ctx_work(ctx, align(x_bytes) + align(w_bytes) + align(z_bytes), &st);
    if (!work) return st;
    TcOperand X{work, batch, nin, nin, ld};
    TcOperand W{work + align(x_bytes), batch, nout, nin, ld};
    TcOperand Z{work + align(x_bytes) + align(w_bytes), batch, nout, nin, ld};
    void* c_d = coro::upload_async(ctx, c.data(), c.size() * sizeof(double), &st);
    if (!c_d) return st;
    std::vector<TcItem> it1(batch), it2(batch);
    for (int b = 0; b < batch; ++b) {
        it1[b] = TcItem{nin, nout, nin, b, b, 0, 0x7fffffff, 1.0f, 1.0f};
        it2[b] = TcItem{nout, nout, nin, b, b, 0, 0x7fffffff, (float)c[b], 1.0f};
    }
    void* i1 = coro::upload_async(ctx, it1.data(), batch * sizeof(TcItem), &st);
    void* i2 = i1 ? coro::upload_async(ctx, it2.data(), batch * sizeof(TcItem), &st) : nullptr;
    cudaError_t e = (i1 && i2) ? cudaSuccess : cudaErrorMemoryAllocation;
    CUtensorMap mx, mw, mz;
    if (e == cudaSuccess) e = tc_split(bf16, (const float2*)in->data, (long long)nin * nin, nin, X, ctx->stream);
    if (e == cudaSuccess) e = tc_basis(bf16, (const double*)c_d, direction < 0 ? -1 : 1, W, ctx->stream);
    if (e == cudaSuccess) e = tc_make_operand_map(X, bf16, &mx);
    if (e == cudaSuccess) e = tc_make_operand_map(W, bf16, &mw);
    if (e == cudaSuccess) e = tc_make_operand_map(Z, bf16, &mz);
    if (e == cudaSuccess) {
        TcArgs a{};
        a.items = (const TcItem*)i1;
        a.err = ctx->err;
        a.dst = Z.base;
        a.dst_bstride = (long long)4 * nout * ld;
        a.dst_rows = nout;
        a.dst_ld = ld;
        e = tc_launch(bf16, TC_EPI_SPLITT, mx, mw, nin, nout, nin, batch, a, ctx->stream);
    }
    if (e == cudaSuccess) {
        TcArgs a{};
        a.items = (const TcItem*)i2;
        a.err = ctx->err;
        a.dst = out->data;
        a.dst_bstride = (long long)nout * nout;
        a.dst_rows = nout;
        a.dst_ld = nout;
        e = tc_launch(bf16, TC_EPI_C64T, mz, mw, nout, nout, nin, batch, a, ctx->stream);
    }
    coro::free_async(ctx, c_d);
    coro::free_async(ctx, i1);
    coro::free_async(ctx, i2);
    if (e == cudaErrorNotSupported) {
        coro::set_error("coro_propagate_mft: tensor maps unavailable (driver entry point missing)");
        return CORO_ENOTIMPL;
    }
    if (e != cudaSuccess) return coro::cuda_fail(e, "tensor-core MFT");
    return CORO_OK;
}

// Extended-precision tensor-core MFT (CORO_MFT_EXT): the same two GEMMs on sliced BF16
// operands (tcx_gemm.cu), the bases sliced straight from their FP64 values.
coro_status mft_ext(coro_ctx ctx, const coro_wavefront* in, int direction, int m, const std::vector<double>& c,
                    coro_wavefront* out) {
    coro_status st = CORO_OK;
    const int batch = in->batch;
    const int nin = in->n, nout = m;
    const int ld = tcx_ld(nin);
    const size_t x_bytes = (size_t)TCX_X_PLANES * batch * nin * ld * 2;
    const size_t w_bytes = (size_t)TCX_W_PLANES * batch * nout * ld * 2;
    const size_t z_bytes = (size_t)TCX_X_PLANES * batch * nout * ld * 2;
    auto align = [](size_t v) { return (v + 1023) & ~(size_t)1023; };
    unsigned char* work = (unsigned char*)coro::ctx_work(ctx, align(x_bytes) + align(w_bytes) + align(z_bytes), &st);
    if (!work) return st;
    TcOperand X{work, batch, nin, nin, ld};
    TcOperand W{work + align(x_bytes), batch, nout, nin, ld};
    TcOperand Z{work + align(x_bytes) + align(w_bytes), batch, nout, nin, ld};
    std::vector<TcItem> it1(batch), it2(batch);
    for (int b = 0; b < batch; ++b) {
        it1[b] = TcItem{nin, nout, nin, b, b, 0, 0x7fffffff, 1.0f, 1.0f};
        it2[b] = TcItem{nout, nout, nin, b, b, 0, 0x7fffffff, (float)c[b], 1.0f};
        it2[b].scale64 = c[b];
    }
    void* i1 = coro::upload_async(ctx, it1.data(), batch * sizeof(TcItem), &st);
    void* i2 = i1 ? coro::upload_async(ctx, it2.data(), batch * sizeof(TcItem), &st) : nullptr;
    cudaError_t e = (i1 && i2) ? cudaSuccess : cudaErrorMemoryAllocation;
    // the first GEMM writes Z's nin valid columns only; its padding up to ld must read as zeros
    if (e == cudaSuccess) e = cudaMemsetAsync(Z.base, 0, z_bytes, ctx->stream);
    CUtensorMap mx, mw, mz;
    if (e == cudaSuccess) e = tcx_split((const float2*)in->data, (long long)nin * nin, nin, X, ctx->stream);
    for (int b = 0; b < batch && e == cudaSuccess; ++b)
        e = tcx_basis_one(c[b], direction < 0 ? -1 : 1, W, b, nout, nin, ctx->stream);
    if (e == cudaSuccess) e = tcx_make_x_map(X, &mx);
    if (e == cudaSuccess) e = tcx_make_w_map(W, &mw);
    if (e == cudaSuccess) e = tcx_make_x_map(Z, &mz);
    if (e == cudaSuccess) {
        TcArgs a{};
        a.items = (const TcItem*)i1;
        a.err = ctx->err;
        a.dst = Z.base;
        a.dst_bstride = (long long)TCX_X_PLANES * nout * ld;
        a.dst_rows = nout;
        a.dst_ld = ld;
        e = tcx_launch(TC_EPI_SPLITT, mx, mw, nin, nout, batch, a, ctx->stream);
    }
    if (e == cudaSuccess) {
        TcArgs a{};
        a.items = (const TcItem*)i2;
        a.err = ctx->err;
        a.dst = out->data;
        a.dst_bstride = (long long)nout * nout;
        a.dst_rows = nout;
        a.dst_ld = nout;
        e = tcx_launch(TC_EPI_C64T, mz, mw, nout, nout, batch, a, ctx->stream);
    }
    coro::free_async(ctx, i1);
    coro::free_async(ctx, i2);
    if (e == cudaErrorNotSupported) {
        coro::set_error("coro_propagate_mft: tensor maps unavailable (driver entry point missing)");
        return CORO_ENOTIMPL;
    }
    if (e != cudaSuccess) return coro::cuda_fail(e, "extended-precision tensor-core MFT");
    return CORO_OK;
}

// CUDA-core MFT: complex64 with FP32 arithmetic or complex128 with FP64 arithmetic.
template <typename C>
coro_status mft_cuda_cores(coro_ctx ctx, const coro_wavefront* in, int direction, int m, const std::vector<double>& c,
                           coro_wavefront* out) {
    using Real = typename real_of<C>::type;
    using Desc = typename std::conditional<std::is_same<C, float2>::value, GemmDesc, ZGemmDesc>::type;
    coro_status st = CORO_OK;
    const int batch = in->batch;
    auto gemm = [&](const Desc& g) -> cudaError_t {
        if constexpr (std::is_same<C, float2>::value) return launch_cgemm(g, batch, CORO_MFT_FP32, ctx->stream);
        else return launch_zgemm(g, batch, ctx->stream);
    };
    // focal-plane side has m (forward) or in->n (inverse) samples; pupil side the other
    const int nf = direction < 0 ? m : in->n;     // focal samples per axis
    const int np = direction < 0 ? in->n : m;     // pupil samples per axis
    const size_t basis_elems = (size_t)batch * nf * np;
    const size_t t_elems = (size_t)batch * (direction < 0 ? (size_t)np * nf : (size_t)nf * np);
    C* work = (C*)coro::ctx_work(ctx, (basis_elems + t_elems) * sizeof(C), &st);
    if (!work) return st;
    C* basis = work;
    C* tmp = work + basis_elems;
    void* c_d = coro::upload_async(ctx, c.data(), c.size() * sizeof(double), &st);
    if (!c_d) return st;
    dim3 bg((np + 127) / 128, nf, batch);
    mft_basis_kernel<C><<<bg, 128, 0, ctx->stream>>>(basis, nf, np, (const double*)c_d, direction < 0 ? -1 : 1);
    cudaError_t e = cudaGetLastError();
    coro::free_async(ctx, c_d);
    if (e != cudaSuccess) return coro::cuda_fail(e, "mft_basis_kernel");

    const C* x = (const C*)in->data;
    C* y = (C*)out->data;
    const long long sb = (long long)nf * np;   // basis batch stride
    Desc g1{}, g2{};
    if (direction < 0) {
        // T[i][u] = sum_j in[i][j] A[u][j]            (M = np, N = nf, K = np)
        g1 = Desc{np, nf, np, x, (long long)np * np, np, false, basis, sb, np, true,
                      tmp, (long long)np * nf, nf, (Real)1};
        // out[v][u] = s sum_i A[v][i] T[i][u]         (M = nf, N = nf, K = np)
        g2 = Desc{nf, nf, np, basis, sb, np, false, tmp, (long long)np * nf, nf, false,
                      y, (long long)nf * nf, nf, (Real)0};
    } else {
        // T[v][j] = sum_u in[v][u] B[u][j]            (M = nf, N = np, K = nf)
        g1 = Desc{nf, np, nf, x, (long long)nf * nf, nf, false, basis, sb, np, false,
                      tmp, (long long)nf * np, np, (Real)1};
        // out[i][j] = s sum_v B[v][i] T[v][j]         (M = np, N = np, K = nf)
        g2 = Desc{np, np, nf, basis, sb, np, true, tmp, (long long)nf * np, np, false,
                      y, (long long)np * np, np, (Real)0};
    }
    std::vector<Real> scale(batch);
    for (int b = 0; b < batch; ++b) scale[b] = (Real)c[b];
    void* s_d = coro::upload_async(ctx, scale.data(), batch * sizeof(Real), &st);
    if (!s_d) return st;
    g2.scale_per_item = (const Real*)s_d;
    e = gemm(g1);
    if (e == cudaSuccess) e = gemm(g2);
    coro::free_async(ctx, s_d);
    if (e == cudaErrorNotSupported) {
        coro::set_error("coro_propagate_mft: CUDA-core GEMM not available in this build");
        return CORO_ENOTIMPL;
    }
    if (e != cudaSuccess) return coro::cuda_fail(e, "mft gemm");
    return CORO_OK;
}

}  // namespace

extern "C" coro_status coro_propagate_mft(coro_ctx ctx, const coro_wavefront* in, double npix, int direction,
                                          int m, const double* du, int precision, coro_wavefront* out) {
    coro::clear_error();
    if (!ctx) { coro::set_error("coro_propagate_mft: ctx is NULL"); return CORO_EINVAL; }
    coro_status st = check_mft_wf("coro_propagate_mft(in)", in);
    if (st != CORO_OK) return st;
    if ((st = check_mft_wf("coro_propagate_mft(out)", out)) != CORO_OK) return st;
    if (direction != -1 && direction != 1) { coro::set_error("coro_propagate_mft: direction must be -1 or +1"); return CORO_EINVAL; }
    if (!(npix > 0)) { coro::set_error("coro_propagate_mft: npix must be > 0"); return CORO_EINVAL; }
    if (!du) { coro::set_error("coro_propagate_mft: du is NULL"); return CORO_EINVAL; }
    if (out->batch != in->batch) { coro::set_error("coro_propagate_mft: batch mismatch"); return CORO_EINVAL; }
    if (out->n != m) { coro::set_error("coro_propagate_mft: out->n (%d) must equal m (%d)", out->n, m); return CORO_EINVAL; }
    if (in->dtype != out->dtype) { coro::set_error("coro_propagate_mft: in and out dtypes differ"); return CORO_EINVAL; }
    const bool dbl = in->dtype == CORO_C128;
    if (dbl ? precision != CORO_MFT_FP64
            : (precision != CORO_MFT_FP32 && precision != CORO_MFT_3XTF32 && precision != CORO_MFT_3XBF16 &&
                 precision != CORO_MFT_EXT)) {
        coro::set_error("coro_propagate_mft: precision %d does not apply to %s fields", precision,
                        dbl ? "complex128 (use CORO_MFT_FP64)" : "complex64");
        return CORO_EINVAL;
    }
    const int batch = in->batch;
    std::vector<double> c(batch);
    for (int b = 0; b < batch; ++b) {
        if (!(du[b] > 0) || !std::isfinite(du[b])) { coro::set_error("coro_propagate_mft: du[%d] must be > 0", b); return CORO_EINVAL; }
        c[b] = du[b] / npix;
    }
    coro::DeviceGuard g(ctx->device);
    if (precision == CORO_MFT_EXT) return mft_ext(ctx, in, direction, m, c, out);
    if (precision == CORO_MFT_3XTF32 || precision == CORO_MFT_3XBF16)
        return mft_tensor_core(ctx, in, direction, m, c, precision == CORO_MFT_3XBF16, out);
    return dbl ? mft_cuda_cores<double2>(ctx, in, direction, m, c, out) : mft_cuda_cores<float2>(ctx, in, direction, m, c, out);
}

