// capi.cu -- C ABI of libcoro: context, wavefront elements, Fresnel propagation, fused
// Fresnel plans and detector reductions. Every compute step runs in the kernels of this
// library; the host side only validates arguments, builds small parameter blocks and
// launches.
#include <cuda_runtime.h>

#include <complex>

#include <cmath>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <memory>
#include <string>

#include "capi_common.h"
#include "passes.cuh"
#include "rader.cuh"
#include "tc_ptx.cuh"

using namespace coro;

// =========================================================================== errors

namespace coro {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}
void clear_error() { g_err.clear(); }

coro_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return e == cudaErrorMemoryAllocation ? CORO_ENOMEM : CORO_ECUDA;
}

long long disk_threshold(double r, double pitch, bool strict) {
    if (!(r >= 0.0)) return -1;
    const double p2 = pitch * pitch, rr = r * r;
    auto ok = [&](long long m) { return strict ? (double)m * p2 < rr : (double)m * p2 <= rr; };
    double guess = std::floor(rr / p2);
    if (guess > 4.0e9) guess = 4.0e9;     // beyond any grid: everything passes
    long long m = (long long)guess;
    while (ok(m + 1) && m < 4000000000LL) ++m;
    while (m >= 0 && !ok(m)) --m;
    return m;
}

long long band_threshold(double half, double pitch) {
    if (!(half > 0.0)) return -1;
    double guess = std::floor(half / pitch);
    if (guess > 1.0e9) guess = 1.0e9;
    long long k = (long long)guess;
    while ((double)(k + 1) * pitch < half && k < 1000000000LL) ++k;
    while (k >= 0 && !((double)k * pitch < half)) --k;
    return k;
}

}  // namespace coro

extern "C" const char* coro_last_error(void) { return g_err.c_str(); }
extern "C" int coro_version(void) { return CORO_VERSION; }

// =========================================================================== FP64 table kernels

namespace {

// Per-pass twiddle blocks of an n-point line FFT (radix 16 then one smaller radix): entry
// m of the block with span ns is W_{ns R}^{r k}, r = 1 + m / ns, k = m % ns, evaluated in FP64
// (sincospi of an exact rational) and rounded. Entries past the last block stay unused.
// W_n^m = exp(-2 pi i m / n) for m in [0, n), FP64-evaluated.
template <typename C>
__global__ void lin_twiddle_kernel(C* tw, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(-2.0 * (double)m / (double)n, &s, &c);
    tw[m] = mk<C>((typename real_of<C>::type)c, (typename real_of<C>::type)s);
}

// Per-stage twiddle blocks of the mixed-radix packed-pair engine (mixed_pair.cuh), stored after
// the linear table: stage s (radix R, span NS > 1) holds W_{NS R}^{r k} at (r - 1) NS + k,
// r = 1 ... R-1, k < NS, so that the twiddles of consecutive butterflies are adjacent.
struct StagePlan {
    int stages;
    int radix[16];
};

template <typename C>
__global__ void stage_twiddle_kernel(C* tw, int count, StagePlan sp) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count) return;
    using R = typename real_of<C>::type;
    int ns = 1, off = 0;
    for (int st = 0; st < sp.stages; ++st) {
        const int r_pass = sp.radix[st];
        if (ns > 1) {
            const int len = (r_pass - 1) * ns;
            if (m < off + len) {
                const int r = 1 + (m - off) / ns, k = (m - off) % ns;
                double s, c;
                sincospi(-2.0 * (double)((long long)r * k) / (double)((long long)ns * r_pass), &s, &c);
                tw[m] = mk<C>((R)c, (R)s);
                return;
            }
            off += len;
        }
        ns *= r_pass;
    }
    // Rader tables of a prime last radix p (rader.cuh): w_L^i, then B_f[k], B_i[k] =
    // (1/L) sum_i b_i w_L^(ik) with b_i = exp(-+2 pi i g^(-i) / p), each term's phase reduced as
    // an exact fraction of a cycle before the FP64 sine and cosine
    const int p = sp.stages > 0 ? sp.radix[sp.stages - 1] : 0;
    const int L = p - 1, i = m - off;
    if (rader_l1(p) && i >= 0 && i < 3 * L) {
        if (i < L) {
            double s, c;
            sincospi(-2.0 * (double)i / (double)L, &s, &c);
            tw[m] = mk<C>((R)c, (R)s);
            return;
        }
        const int k = (i - L) % L;
        const double sgn = i < 2 * L ? -1.0 : 1.0;    // B_f: W_p = exp(-2 pi i / p); B_i: its conjugate
        const int g = rader_root(p);
        double re = 0.0, im = 0.0;
        for (int t = 0; t < L; ++t) {
            const int gi = rader_pow(g, (L - t) % L, p);            // g^(-t) mod p
            // phase in cycles: sgn g^-t / p - t k / L (mod 1)
            double cyc = sgn * (double)gi / (double)p - (double)((t * k) % L) / (double)L;
            cyc -= rint(cyc);
            double s, c;
            sincospi(2.0 * cyc, &s, &c);
            re += c;
            im += s;
        }
        tw[m] = mk<C>((R)(re / L), (R)(im / L));
        return;
    }
    tw[m] = mk<C>(0, 0);
}

template <typename C>
__global__ void twiddle_kernel(C* tw, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    int ns = 16, off = 0;
    while (ns < n) {
        const int r_pass = (n / ns) >= 16 ? 16 : n / ns;
        const int len = (r_pass - 1) * ns;
        if (m < off + len) {
            const int r = 1 + (m - off) / ns, k = (m - off) % ns;
            double s, c;
            sincospi(-2.0 * (double)((long long)r * k) / (double)(ns * r_pass), &s, &c);
            tw[m] = mk<C>((typename real_of<C>::type)c, (typename real_of<C>::type)s);
            return;
        }
        off += len;
        ns *= 16;
    }
    tw[m] = mk<C>(0, 0);
}

// Separable phase table: value[k] = mag * (-1)^(checker*k) * exp(2 pi i sign frac(k'^2 c)),
// k' = k - n/2. The cycle count k'^2 c is reduced to its fractional part in FP64 before the
// sine and cosine (Sec. 2.3: quadratic phase factors reach 1e6-1e7 radians at the array edge).
struct TabSpec {
    double c;        // cycles per k'^2
    double mag_re, mag_im;
    int sign;        // +1 / -1
    int checker;     // multiply by (-1)^k
};

template <typename C>
__global__ void sep_table_kernel(C* out, int n, const TabSpec* spec) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (k >= n) return;
    const TabSpec sp = spec[b];
    const long long kk = (long long)k - n / 2;
    double cyc = (double)(kk * kk) * sp.c;
    cyc -= rint(cyc);
    double s, c;
    sincospi(2.0 * cyc, &s, &c);
    if (sp.sign < 0) s = -s;
    double re = sp.mag_re * c - sp.mag_im * s;
    double im = sp.mag_re * s + sp.mag_im * c;
    if (sp.checker && (k & 1)) { re = -re; im = -im; }
    using R = typename real_of<C>::type;
    out[(size_t)b * n + k] = mk<C>((R)re, (R)im);
}

}  // namespace

namespace coro {

// linear: the table W_n^m of the shared-memory engine even when n is a power of two (kept
// under the key -n beside the per-pass blocks). At a mixed-radix n the complex64 table holds the
// linear table, then the per-stage blocks of the packed-pair engine (stage_twiddle_kernel).
const void* get_twiddles(coro_ctx ctx, int n, bool dbl, coro_status* st, bool linear) {
    auto& cache = dbl ? ctx->tw64 : ctx->tw32;
    const int key = (linear && is_pow2(n)) ? -n : n;
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    StagePlan sp{};
    int extra = 0;
    if (!is_pow2(n) && !dbl) {
        sp.stages = pass_radices(n, true, 0, 0, sp.radix, 16);
        for (int s = 0, ns = 1; s < sp.stages; ns *= sp.radix[s], ++s)
            if (ns > 1) extra += (sp.radix[s] - 1) * ns;
        if (sp.stages > 0) extra += rader_table_len(sp.radix[sp.stages - 1]);
    }
    void* p = nullptr;
    const size_t bytes = (size_t)(n + extra) * (dbl ? sizeof(double2) : sizeof(float2));
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) { *st = cuda_fail(e, "cudaMalloc(twiddles)"); return nullptr; }
    const int th = 256;
    if (!is_pow2(n) || linear) {                // mixed-radix passes: the linear table W_n^m
        if (dbl) lin_twiddle_kernel<double2><<<(n + th - 1) / th, th, 0, ctx->stream>>>((double2*)p, n);
        else lin_twiddle_kernel<float2><<<(n + th - 1) / th, th, 0, ctx->stream>>>((float2*)p, n);
        if (extra > 0)
            stage_twiddle_kernel<float2><<<(extra + th - 1) / th, th, 0, ctx->stream>>>((float2*)p + n, extra, sp);
    } else if (dbl) {
        twiddle_kernel<double2><<<(n + th - 1) / th, th, 0, ctx->stream>>>((double2*)p, n);
    } else {
        twiddle_kernel<float2><<<(n + th - 1) / th, th, 0, ctx->stream>>>((float2*)p, n);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { cudaFree(p); *st = cuda_fail(e, "twiddle_kernel"); return nullptr; }
    cache[key] = p;
    return p;
}

void* upload_async(coro_ctx ctx, const void* host, size_t bytes, coro_status* st) {
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
    if (e != cudaSuccess) { *st = cuda_fail(e, "cudaMallocAsync"); return nullptr; }
    if (host) {
        e = cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) { cudaFreeAsync(p, ctx->stream); *st = cuda_fail(e, "cudaMemcpyAsync"); return nullptr; }
    }
    return p;
}

void free_async(coro_ctx ctx, void* p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

void* ctx_work(coro_ctx ctx, size_t bytes, coro_status* st) {
    if (ctx->work_bytes >= bytes) return ctx->work;
    if (ctx->work) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->work);
        ctx->work = nullptr;
        ctx->work_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->work, bytes);
    if (e != cudaSuccess) { ctx->work = nullptr; *st = cuda_fail(e, "cudaMalloc(work)"); return nullptr; }
    ctx->work_bytes = bytes;
    return ctx->work;
}

}  // namespace coro

// =========================================================================== context

extern "C" coro_status coro_ctx_create(int device, void* stream, coro_ctx* out) {
    clear_error();
    if (!out) { set_error("coro_ctx_create: out is NULL"); return CORO_EINVAL; }
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        set_error("coro_ctx_create: no CUDA device (%s)", cudaGetErrorString(e));
        return CORO_ECUDA;
    }
    if (device < 0 || device >= count) { set_error("coro_ctx_create: device %d of %d", device, count); return CORO_EINVAL; }
    DeviceGuard g(device);
    if (!g.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    auto* c = new (std::nothrow) coro_ctx_s;
    if (!c) { set_error("coro_ctx_create: out of host memory"); return CORO_ENOMEM; }
    c->device = device;
    c->stream = (cudaStream_t)stream;
    e = cudaMalloc(&c->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(int));
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "coro_ctx_create"); }
    *out = c;
    return CORO_OK;
}

extern "C" coro_status coro_ctx_destroy(coro_ctx ctx) {
    clear_error();
    if (!ctx) return CORO_OK;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();          // the borrowed stream may already be gone
        for (auto& kv : ctx->tw32) cudaFree(kv.second);
        for (auto& kv : ctx->tw64) cudaFree(kv.second);
        if (ctx->work) cudaFree(ctx->work);
        if (ctx->err) cudaFree(ctx->err);
    }
    delete ctx;
    return CORO_OK;
}

extern "C" coro_status coro_ctx_set_stream(coro_ctx ctx, void* stream) {
    clear_error();
    if (!ctx) { set_error("coro_ctx_set_stream: ctx is NULL"); return CORO_EINVAL; }
    ctx->stream = (cudaStream_t)stream;
    return CORO_OK;
}

extern "C" coro_status coro_ctx_synchronize(coro_ctx ctx) {
    clear_error();
    if (!ctx) { set_error("coro_ctx_synchronize: ctx is NULL"); return CORO_EINVAL; }
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, ctx->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error flag");
    if (flag) {
        cudaMemset(ctx->err, 0, sizeof(int));
        set_error("a bounded device-side wait expired (code %d); results of the affected launch are invalid", flag);
        return CORO_ETIMEOUT;
    }
    return CORO_OK;
}

// Failure-path check: one thread waits, with a short bound, on an mbarrier that nothing will
// ever complete, so the bounded wait expires and raises the context's error flag exactly as a
// stalled copy or MMA would; the kernel then returns and the context stays usable.
__global__ void wait_timeout_probe_kernel(int* err, int polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    coro::tc::mbar_init(&bar, 1);
    coro::tc::fence_mbar_init();
    coro::tc::mbar_wait(&bar, 0, err, 99, polls);          // phase 0 never completes
}

extern "C" coro_status coro_selftest_wait_timeout(coro_ctx ctx, int polls) {
    clear_error();
    if (!ctx || polls < 1 || polls > (1 << 20)) { set_error("coro_selftest_wait_timeout: bad argument"); return CORO_EINVAL; }
    DeviceGuard g(ctx->device);
    wait_timeout_probe_kernel<<<1, 32, 0, ctx->stream>>>(ctx->err, polls);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "wait_timeout_probe_kernel");
}

// =========================================================================== validation

static coro_status check_wf(const char* fn, coro_ctx ctx, const coro_wavefront* wf, bool need_ps = true) {
    if (!ctx) { set_error("%s: ctx is NULL", fn); return CORO_EINVAL; }
    if (!wf) { set_error("%s: wavefront is NULL", fn); return CORO_EINVAL; }
    if (!wf->data) { set_error("%s: wavefront data is NULL", fn); return CORO_EINVAL; }
    if (wf->dtype != CORO_C64 && wf->dtype != CORO_C128) { set_error("%s: bad dtype %d", fn, wf->dtype); return CORO_EINVAL; }
    if (wf->batch < 1 || wf->batch > 65535) { set_error("%s: batch %d outside [1, 65535]", fn, wf->batch); return CORO_ESIZE; }
    const int nmax = wf->dtype == CORO_C64 ? 8192 : 4096;
    const bool pow2_ok = is_pow2(wf->n) && wf->n >= 32 && wf->n <= nmax;
    if (!pow2_ok && (is_pow2(wf->n) || wf->n > 8192 || !mixed_length_ok(wf->n, wf->dtype == CORO_C128))) {
        set_error("%s: n = %d must be a power of two in [32, %d], or even with prime factors up to 61 "
                  "(complex64: n <= 8192, complex128: n <= 6022)", fn, wf->n, nmax);
        return CORO_ESIZE;
    }
    if (need_ps) {
        if (!wf->pixelscale || !wf->wavelength) { set_error("%s: pixelscale/wavelength arrays are NULL", fn); return CORO_EINVAL; }
        for (int b = 0; b < wf->batch; ++b) {
            if (!(wf->pixelscale[b] > 0.0) || !std::isfinite(wf->pixelscale[b])) { set_error("%s: pixelscale[%d] must be > 0", fn, b); return CORO_EINVAL; }
            if (!(wf->wavelength[b] > 0.0) || !std::isfinite(wf->wavelength[b])) { set_error("%s: wavelength[%d] must be > 0", fn, b); return CORO_EINVAL; }
        }
    }
    return CORO_OK;
}

// =========================================================================== element compiler

namespace {

// Owns the device parameter blocks of compiled elements. Stream-ordered frees unless the
// owner is a plan (then freed at destroy, after a synchronize).
struct DevBlocks {
    coro_ctx ctx = nullptr;
    std::vector<void*> blocks;
    bool plan_owned = false;
    void* add(const void* host, size_t bytes, coro_status* st) {
        void* p = nullptr;
        if (plan_owned) {
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess) { *st = cuda_fail(e, "cudaMalloc(plan params)"); return nullptr; }
            if (host) {
                e = cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, ctx->stream);
                if (e != cudaSuccess) { cudaFree(p); *st = cuda_fail(e, "cudaMemcpyAsync"); return nullptr; }
            }
        } else {
            p = upload_async(ctx, host, bytes, st);
            if (!p) return nullptr;
        }
        blocks.push_back(p);
        return p;
    }
    void release() {
        if (plan_owned) {
            for (void* p : blocks) cudaFree(p);
        } else {
            for (void* p : blocks) free_async(ctx, p);
        }
        blocks.clear();
    }
};

// Separable complex table [batch][n] generated on the device from per-item specs.
void* make_table(DevBlocks& db, bool dbl, int n, const std::vector<TabSpec>& specs, coro_status* st) {
    const int batch = (int)specs.size();
    const size_t elt = dbl ? sizeof(double2) : sizeof(float2);
    void* spec_d = upload_async(db.ctx, specs.data(), specs.size() * sizeof(TabSpec), st);
    if (!spec_d) return nullptr;
    void* tab = db.add(nullptr, (size_t)batch * n * elt, st);
    if (!tab) { free_async(db.ctx, spec_d); return nullptr; }
    dim3 grid((n + 255) / 256, batch);
    if (dbl) sep_table_kernel<double2><<<grid, 256, 0, db.ctx->stream>>>((double2*)tab, n, (const TabSpec*)spec_d);
    else sep_table_kernel<float2><<<grid, 256, 0, db.ctx->stream>>>((float2*)tab, n, (const TabSpec*)spec_d);
    cudaError_t e = cudaGetLastError();
    free_async(db.ctx, spec_d);
    if (e != cudaSuccess) { *st = cuda_fail(e, "sep_table_kernel"); return nullptr; }
    return tab;
}

int clamp_thr(long long v) { return v > 0x3fffffffLL ? 0x3fffffff : (int)v; }

// Noll index -> (n, m), m > 0 cosine, m < 0 sine (Noll 1976 ordering).
void noll_nm(int j, int* n_out, int* m_out) {
    int count = 0;
    for (int n = 0;; ++n) {
        for (int am = n % 2; am <= n; am += 2) {
            if (am == 0) {
                if (++count == j) { *n_out = n; *m_out = 0; return; }
            } else {
                const int first = count + 1, second = count + 2;
                count += 2;
                if (j == first || j == second) { *n_out = n; *m_out = (j % 2 == 0) ? am : -am; return; }
            }
        }
    }
}

double factorial(int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; }

// Combined Zernike polynomial table: A_m(rho^2) multiplies Re(z^m), B_m(rho^2) Im(z^m).
bool zernike_table(const coro_element* el, std::vector<double>& out) {
    std::vector<double> acc(2 * ZM * ZD, 0.0);
    for (int i = 0; i < el->n_coeffs; ++i) {
        int n, m;
        noll_nm(el->j_first + i, &n, &m);
        const int am = m < 0 ? -m : m;
        if (am >= ZM || (n - am) / 2 >= ZD) return false;
        const double norm = m == 0 ? std::sqrt((double)(n + 1)) : std::sqrt(2.0 * (n + 1));
        double* dst = acc.data() + (m < 0 ? ZM * ZD : 0) + am * ZD;
        for (int s = 0; s <= (n - am) / 2; ++s) {
            const double a = ((s % 2) ? -1.0 : 1.0) * factorial(n - s)
                             / (factorial(s) * factorial((n + am) / 2 - s) * factorial((n - am) / 2 - s));
            dst[(n - am) / 2 - s] += el->coeffs[i] * norm * a;
        }
    }
    out.assign(acc.begin(), acc.end());
    return true;
}

// x = hi + lo with hi = float(x): complex64 passes use hi, complex128 passes the FP64 sum
// (about 48 significant bits).
void split_f32(double x, float* hi, float* lo) {
    *hi = (float)x;
    *lo = (float)(x - (double)*hi);
}

// Compile one API element for a batch at the given per-item pixel scales.
coro_status compile_element(DevBlocks& db, const coro_element* el, bool dbl, int n, int batch,
                            const double* ps, const double* lam, DevElem* out) {
    coro_status st = CORO_OK;
    std::memset(out, 0, sizeof(DevElem));
    std::vector<int> ithr((size_t)batch * 4, 0);
    std::vector<float> fpar((size_t)batch * 4, 0.f);   // [batch][4]
    switch (el->kind) {
        case CORO_EL_APERTURE: {
            if (!(el->radius > 0)) { set_error("aperture: radius must be > 0"); return CORO_EINVAL; }
            if (el->n_spiders != 0 && el->n_spiders != 4) { set_error("aperture: n_spiders must be 0 or 4"); return CORO_ENOTIMPL; }
            if (el->obscuration < 0 || el->obscuration >= 1) { set_error("aperture: obscuration in [0, 1)"); return CORO_EINVAL; }
            for (int b = 0; b < batch; ++b) {
                ithr[4 * b + 0] = clamp_thr(disk_threshold(el->radius, ps[b], false));
                const double ro = el->obscuration * el->radius;
                ithr[4 * b + 1] = el->obscuration > 0 ? clamp_thr(disk_threshold(ro, ps[b], true)) : -1;
                ithr[4 * b + 2] = el->n_spiders ? clamp_thr(band_threshold(el->spider_width / 2.0, ps[b])) : -1;
            }
            out->kind = DK_APERTURE;
            break;
        }
        case CORO_EL_CIRCLE: {
            for (int b = 0; b < batch; ++b) ithr[4 * b] = clamp_thr(disk_threshold(el->radius, ps[b], false));
            out->kind = DK_CIRCLE;
            out->flags = (el->flags & CORO_ELF_OPAQUE_INSIDE) ? 1 : 0;
            break;
        }
        case CORO_EL_LENS: {
            if (el->focal_length == 0 || !std::isfinite(el->focal_length)) { set_error("lens: focal length must be finite and nonzero"); return CORO_EINVAL; }
            std::vector<TabSpec> sp(batch);
            for (int b = 0; b < batch; ++b)
                sp[b] = TabSpec{ps[b] * ps[b] / (2.0 * lam[b] * el->focal_length), 1.0, 0.0, -1, 0};
            out->tab = make_table(db, dbl, n, sp, &st);
            if (!out->tab) return st;
            out->kind = DK_TABLE;
            return CORO_OK;
        }
        case CORO_EL_OPD_MAP: {
            if (!el->opd) { set_error("opd map: opd pointer is NULL"); return CORO_EINVAL; }
            for (int b = 0; b < batch; ++b) split_f32(2.0 / lam[b], &fpar[4 * b], &fpar[4 * b + 1]);
            out->kind = DK_OPD_MAP;
            out->map = el->opd;
            out->amp = el->amplitude;
            out->map_bstride = (el->flags & CORO_ELF_MAP_BATCHED) ? (long long)n * n : 0;
            break;
        }
        case CORO_EL_ZERNIKE: {
            if (!el->coeffs || el->n_coeffs < 1 || el->j_first < 1) { set_error("zernike: need coeffs, n_coeffs >= 1, j_first >= 1"); return CORO_EINVAL; }
            if (!(el->radius > 0)) { set_error("zernike: radius must be > 0"); return CORO_EINVAL; }
            std::vector<double> zt;
            if (!zernike_table(el, zt)) { set_error("zernike: Noll index beyond 36 (radial order 7)"); return CORO_ENOTIMPL; }
            for (int b = 0; b < batch; ++b) {
                ithr[4 * b] = clamp_thr(disk_threshold(el->radius, ps[b], false));
                split_f32(2.0 / lam[b], &fpar[4 * b], &fpar[4 * b + 2]);
                split_f32(ps[b] / el->radius, &fpar[4 * b + 1], &fpar[4 * b + 3]);
            }
            if (dbl) {                                   // complex128 passes: FP64 polynomials
                std::vector<double> zd(zt.begin(), zt.end());
                out->zpoly = (const float*)db.add(zd.data(), zd.size() * sizeof(double), &st);
            } else {
                std::vector<float> zf(zt.begin(), zt.end());
                out->zpoly = (const float*)db.add(zf.data(), zf.size() * sizeof(float), &st);
            }
            if (!out->zpoly) return st;
            out->kind = DK_ZERNIKE;
            break;
        }
        case CORO_EL_SINE: {
            for (int b = 0; b < batch; ++b) {
                const double f = el->sine_freq * ps[b];                 // cycles per pixel
                const double fhi = (double)(float)(std::ldexp(std::rint(std::ldexp(f, 11)), -11));
                split_f32(2.0 * el->sine_amplitude / lam[b], &fpar[4 * b], &fpar[4 * b + 3]);
                fpar[4 * b + 1] = (float)fhi;
                fpar[4 * b + 2] = (float)(f - fhi);
            }
            if (dbl) {                                   // complex128 passes: f and 2 amp / lambda in FP64
                std::vector<double> dp((size_t)2 * batch);
                for (int b = 0; b < batch; ++b) {
                    dp[2 * b] = el->sine_freq * ps[b];
                    dp[2 * b + 1] = 2.0 * el->sine_amplitude / lam[b];
                }
                out->zpoly = (const float*)db.add(dp.data(), dp.size() * sizeof(double), &st);
                if (!out->zpoly) return st;
            }
            out->kind = DK_SINE;
            out->flags = el->axis ? 1 : 0;
            break;
        }
        case CORO_EL_SCALAR: {
            for (int b = 0; b < batch; ++b) split_f32(el->scalar, &fpar[4 * b], &fpar[4 * b + 1]);
            out->kind = DK_SCALAR;
            break;
        }
        case CORO_EL_PHASE_GRAD: {
            if (!el->store) { set_error("phase gradient: store must be set"); return CORO_EINVAL; }
            for (int b = 0; b < batch; ++b) split_f32(2.0 * el->scalar / lam[b], &fpar[4 * b], &fpar[4 * b + 1]);
            out->kind = DK_PHASE_GRAD;
            out->dst = el->store;
            out->tab = el->ref;
            out->map_bstride = (long long)n * n;
            break;
        }
        case CORO_EL_CHECKPOINT: {
            if (!el->store) { set_error("checkpoint: store is NULL"); return CORO_EINVAL; }
            out->kind = DK_STORE;
            out->dst = el->store;
            out->map_bstride = (long long)n * n;
            break;
        }
        default:
            set_error("unknown element kind %d", el->kind);
            return CORO_EINVAL;
    }
    out->ithr = (const int*)db.add(ithr.data(), ithr.size() * sizeof(int), &st);
    if (!out->ithr) return st;
    out->fpar = (const float*)db.add(fpar.data(), fpar.size() * sizeof(float), &st);
    if (!out->fpar) return st;
    return CORO_OK;
}

DevElem checker_elem() { DevElem e; std::memset(&e, 0, sizeof(e)); e.kind = DK_CHECKER; return e; }

DevElem table_elem(const void* tab) { DevElem e; std::memset(&e, 0, sizeof(e)); e.kind = DK_TABLE; e.tab = tab; return e; }
DevElem conj_elem() { DevElem e; std::memset(&e, 0, sizeof(e)); e.kind = DK_CONJ; return e; }

// ------------------------------------------------------------------------------ pass ops

struct Op {
    bool row = true;
    int row_flags = 0;
    int col_flags = 0;
    PassElems elems{};
    const void* tab_x = nullptr;
    const void* tab_y = nullptr;
    int lines = 0;        // column passes: 0 default, > 0 block width, < 0 staged kernels (passes_f32.cu)
    int variant = -1;     // row passes: -1 default, 0 persistent, 1 per group, 2 units, 3 pairs
};

// ev (optional, ops.size() + 1 events): recorded before the first pass and after each.
// tbuf: the plane that column passes with lines -6 write transposed and the row passes of
// variant 4 read back (batch x n x n samples); NULL when the ops hold neither.
template <typename C>
coro_status run_ops(coro_ctx ctx, int n, int batch, const std::vector<Op>& ops, void* field,
                    const cudaEvent_t* ev = nullptr, void* tbuf = nullptr) {
    coro_status st = CORO_OK;
    const C* tw = (const C*)get_twiddles(ctx, n, sizeof(C) == sizeof(double2), &st);
    if (!tw) return st;
    const C* tw_lin = nullptr;                          // radix-8 shared-memory engine at a power of two
    for (const Op& op : ops)
        if (!tw_lin && ((op.row && op.variant == 5) || (!op.row && op.lines == -8))) {
            tw_lin = (const C*)get_twiddles(ctx, n, sizeof(C) == sizeof(double2), &st, true);
            if (!tw_lin) return st;
        }
    PassLaunch pl{ctx->stream, batch};
    if (ev) {
        const cudaError_t e0 = record_timing_event(ev[0], ctx->stream);
        if (e0 != cudaSuccess) return cuda_fail(e0, "cudaEventRecord");
    }
    int i = 0;
    for (const Op& op : ops) {
        cudaError_t e;
        const bool t_in = op.row && op.variant == 4, t_out = !op.row && op.lines == -6;
        if ((t_in || t_out) && !tbuf) { set_error("transposed pass without its plane"); return CORO_EINVAL; }
        if (op.row) {
            RowArgs<C> a;
            a.in = (const C*)(t_in ? tbuf : field);
            a.out = (C*)field;
            a.tw = op.variant == 5 ? tw_lin : tw;
            a.flags = op.row_flags;
            a.err = ctx->err;
            a.elems = op.elems;
            pl.variant = op.variant;
            e = launch_row_pass<C>(n, a, pl);
        } else {
            ColArgs<C> a;
            a.in = (const C*)field;
            a.out = (C*)(t_out ? tbuf : field);
            a.tw = op.lines == -8 ? tw_lin : tw;
            a.tab_x = (const C*)op.tab_x;
            a.tab_y = (const C*)op.tab_y;
            a.flags = op.col_flags;
            a.err = ctx->err;
            e = launch_col_pass<C>(n, op.lines, a, pl);
        }
        if (e != cudaSuccess) return cuda_fail(e, op.row ? "row pass" : "column pass");
        ++i;
        if (ev && (e = record_timing_event(ev[i], ctx->stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    }
    return CORO_OK;
}

coro_status run_ops_any(coro_ctx ctx, int dtype, int n, int batch, const std::vector<Op>& ops, void* field,
                        const cudaEvent_t* ev = nullptr, void* tbuf = nullptr) {
    return dtype == CORO_C64 ? run_ops<float2>(ctx, n, batch, ops, field, ev, tbuf)
                             : run_ops<double2>(ctx, n, batch, ops, field, ev, tbuf);
}

// ------------------------------------------------------------------------------ hop tables

// Angular-spectrum transfer function per axis, 1/n folded in (1/n^2 overall for the IDFT).
coro_status as_table(DevBlocks& db, bool dbl, int n, int batch, const double* ps, const double* lam,
                     const double* z, const void** out) {
    coro_status st = CORO_OK;
    std::vector<TabSpec> sp(batch);
    for (int b = 0; b < batch; ++b) {
        const double L = n * ps[b];
        sp[b] = TabSpec{lam[b] * z[b] / (2.0 * L * L), 1.0 / n, 0.0, -1, 0};
    }
    *out = make_table(db, dbl, n, sp, &st);
    return *out ? CORO_OK : st;
}

// Direct Fresnel: input QPF exp(+i pi x^2/(lambda z)); output QPF with (-1)^k folded in, the
// y-table also carrying dx^2 / (i lambda z); output pitch |lambda z / (n dx)|. qin / qout
// drop the input or output QPF (hops from or to a waist in the pilot-beam scheme). For z < 0
// the kernel exp(-2 pi i x u / (lambda z)) is the inverse DFT on the grid u_k = (k - n/2)|du|;
// it is computed as conj(DFT(conj(.))): the tables returned are then the conjugates of the
// input QPF and of the output factor, and the caller conjugates the field before the row FFT
// and after the column pass (the next row pass).
coro_status direct_tables(DevBlocks& db, bool dbl, int n, int batch, const double* ps, const double* lam,
                          const double* z, bool qin_on, bool qout_on, const void** qin, const void** qx,
                          const void** qy, std::vector<double>& ps_out) {
    coro_status st = CORO_OK;
    std::vector<TabSpec> a(batch), bx(batch), by(batch);
    ps_out.resize(batch);
    for (int b = 0; b < batch; ++b) {
        const double dx = ps[b], zb = z[b];
        const double du = std::fabs(lam[b] * zb / (n * dx));
        const int cj = zb < 0 ? -1 : 1;                          // conjugate every table for z < 0
        ps_out[b] = du;
        a[b] = TabSpec{qin_on ? dx * dx / (2.0 * lam[b] * zb) : 0.0, 1.0, 0.0, +cj, 0};
        bx[b] = TabSpec{qout_on ? du * du / (2.0 * lam[b] * zb) : 0.0, 1.0, 0.0, +cj, 1};
        by[b] = TabSpec{qout_on ? du * du / (2.0 * lam[b] * zb) : 0.0, 0.0, -cj * dx * dx / (lam[b] * zb), +cj, 1};
    }
    *qin = nullptr;
    if (qin_on && !(*qin = make_table(db, dbl, n, a, &st))) return st;
    if (!(*qx = make_table(db, dbl, n, bx, &st))) return st;
    if (!(*qy = make_table(db, dbl, n, by, &st))) return st;
    return CORO_OK;
}

coro_status sign_tables(DevBlocks& db, bool dbl, int n, int batch, double mag, const void** out) {
    coro_status st = CORO_OK;
    std::vector<TabSpec> sp(batch, TabSpec{0.0, mag, 0.0, 1, 1});
    *out = make_table(db, dbl, n, sp, &st);
    return *out ? CORO_OK : st;
}

}  // namespace

// =========================================================================== a1: init

namespace {
template <typename C>
__global__ void fill_kernel(C* p, size_t count, double amp) {
    using R = typename real_of<C>::type;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        p[i] = mk<C>((R)amp, (R)0);
}
}  // namespace

extern "C" coro_status coro_wavefront_init(coro_ctx ctx, const coro_wavefront* wf, double amplitude) {
    clear_error();
    coro_status st = check_wf("coro_wavefront_init", ctx, wf, false);
    if (st != CORO_OK) return st;
    DeviceGuard g(ctx->device);
    const size_t count = (size_t)wf->batch * wf->n * wf->n;
    const int blocks = (int)std::min<size_t>((count + 255) / 256, 152 * 16);
    if (wf->dtype == CORO_C64) fill_kernel<float2><<<blocks, 256, 0, ctx->stream>>>((float2*)wf->data, count, amplitude);
    else fill_kernel<double2><<<blocks, 256, 0, ctx->stream>>>((double2*)wf->data, count, amplitude);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "fill_kernel");
}

namespace {
template <typename C>
__global__ void axpy_kernel(typename real_of<C>::type alpha, const C* __restrict__ x, C* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const C a = x[i], b = y[i];
        y[i] = mk<C>(fma(alpha, a.x, b.x), fma(alpha, a.y, b.y));
    }
}
}  // namespace

extern "C" coro_status coro_wavefront_axpy(coro_ctx ctx, double alpha, const coro_wavefront* x, const coro_wavefront* y) {
    clear_error();
    if (!ctx || !x || !y || !x->data || !y->data) { set_error("coro_wavefront_axpy: NULL argument"); return CORO_EINVAL; }
    if (x->dtype != y->dtype || x->batch != y->batch || x->n != y->n) {
        set_error("coro_wavefront_axpy: x and y differ in dtype, batch or n");
        return CORO_EINVAL;
    }
    if ((x->dtype != CORO_C64 && x->dtype != CORO_C128) || x->batch < 1 || x->n < 1) {
        set_error("coro_wavefront_axpy: bad dtype, batch or n");
        return CORO_EINVAL;
    }
    if (!std::isfinite(alpha)) { set_error("coro_wavefront_axpy: alpha must be finite"); return CORO_EINVAL; }
    DeviceGuard g(ctx->device);
    const size_t n = (size_t)x->batch * x->n * x->n;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
    if (x->dtype == CORO_C64)
        axpy_kernel<float2><<<blocks, 256, 0, ctx->stream>>>((float)alpha, (const float2*)x->data, (float2*)y->data, n);
    else
        axpy_kernel<double2><<<blocks, 256, 0, ctx->stream>>>(alpha, (const double2*)x->data, (double2*)y->data, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "axpy_kernel");
}

// =========================================================================== a2/a3: elements

extern "C" coro_status coro_apply_element(coro_ctx ctx, const coro_wavefront* wf, const coro_element* el) {
    clear_error();
    coro_status st = check_wf("coro_apply_element", ctx, wf);
    if (st != CORO_OK) return st;
    if (!el) { set_error("coro_apply_element: element is NULL"); return CORO_EINVAL; }
    DeviceGuard g(ctx->device);
    DevBlocks db;
    db.ctx = ctx;
    Op op;
    op.row = true;
    op.elems.count = 1;
    st = compile_element(db, el, wf->dtype == CORO_C128, wf->n, wf->batch, wf->pixelscale, wf->wavelength, &op.elems.e[0]);
    if (st == CORO_OK) st = run_ops_any(ctx, wf->dtype, wf->n, wf->batch, {op}, wf->data);
    db.release();
    return st;
}

// =========================================================================== a4-a6: Fresnel

extern "C" coro_status coro_propagate_fresnel(coro_ctx ctx, coro_wavefront* wf, double z, int method) {
    clear_error();
    coro_status st = check_wf("coro_propagate_fresnel", ctx, wf);
    if (st != CORO_OK) return st;
    if (!(z != 0.0) || !std::isfinite(z)) { set_error("coro_propagate_fresnel: z must be finite and nonzero"); return CORO_EINVAL; }
    if (method != CORO_FRESNEL_AS && method != CORO_FRESNEL_DIRECT) { set_error("coro_propagate_fresnel: bad method %d", method); return CORO_EINVAL; }
    DeviceGuard g(ctx->device);
    const bool dbl = wf->dtype == CORO_C128;
    const int n = wf->n, batch = wf->batch;
    DevBlocks db;
    db.ctx = ctx;
    std::vector<Op> ops;
    std::vector<double> ps_out;
    const std::vector<double> zb(batch, z);
    if (method == CORO_FRESNEL_AS) {
        const void* h = nullptr;
        st = as_table(db, dbl, n, batch, wf->pixelscale, wf->wavelength, zb.data(), &h);
        if (st == CORO_OK) {
            Op r0; r0.row = true; r0.row_flags = RF_FWD_AFTER; r0.elems.count = 1; r0.elems.e[0] = checker_elem();
            Op c; c.row = false; c.col_flags = CF_FWD | CF_TABLE | CF_INV; c.tab_x = h; c.tab_y = h;
            Op r1; r1.row = true; r1.row_flags = RF_INV_FIRST; r1.elems.count = 1; r1.elems.e[0] = checker_elem();
            ops = {r0, c, r1};
        }
    } else {
        const void *qin = nullptr, *qx = nullptr, *qy = nullptr;
        st = direct_tables(db, dbl, n, batch, wf->pixelscale, wf->wavelength, zb.data(), true, true, &qin, &qx, &qy, ps_out);
        if (st == CORO_OK) {
            Op r0; r0.row = true; r0.row_flags = RF_FWD_AFTER;
            if (z < 0) r0.elems.e[r0.elems.count++] = conj_elem();
            r0.elems.e[r0.elems.count++] = table_elem(qin);
            r0.elems.e[r0.elems.count++] = checker_elem();
            Op c; c.row = false; c.col_flags = CF_FWD | CF_TABLE; c.tab_x = qx; c.tab_y = qy;
            ops = {r0, c};
            if (z < 0) {                                      // undo the conjugation of the output
                Op r1; r1.row = true; r1.elems.count = 1; r1.elems.e[0] = conj_elem();
                ops.push_back(r1);
            }
        }
    }
    if (st == CORO_OK) st = run_ops_any(ctx, wf->dtype, n, batch, ops, wf->data);
    db.release();
    if (st == CORO_OK && method == CORO_FRESNEL_DIRECT)
        for (int b = 0; b < batch; ++b) wf->pixelscale[b] = ps_out[b];
    return st;
}

extern "C" coro_status coro_fft2(coro_ctx ctx, const coro_wavefront* wf, int direction) {
    clear_error();
    coro_status st = check_wf("coro_fft2", ctx, wf, false);
    if (st != CORO_OK) return st;
    if (direction != -1 && direction != 1) { set_error("coro_fft2: direction must be -1 or +1"); return CORO_EINVAL; }
    DeviceGuard g(ctx->device);
    const bool dbl = wf->dtype == CORO_C128;
    DevBlocks db;
    db.ctx = ctx;
    const void* sgn = nullptr;
    st = sign_tables(db, dbl, wf->n, wf->batch, direction < 0 ? 1.0 : 1.0 / wf->n, &sgn);
    std::vector<Op> ops;
    if (st == CORO_OK) {
        if (direction < 0) {
            Op r; r.row = true; r.row_flags = RF_FWD_AFTER; r.elems.count = 1; r.elems.e[0] = checker_elem();
            Op c; c.row = false; c.col_flags = CF_FWD | CF_TABLE; c.tab_x = sgn; c.tab_y = sgn;
            ops = {r, c};
        } else {
            Op c; c.row = false; c.col_flags = CF_TABLE | CF_INV; c.tab_x = sgn; c.tab_y = sgn;
            Op r; r.row = true; r.row_flags = RF_INV_FIRST; r.elems.count = 1; r.elems.e[0] = checker_elem();
            ops = {c, r};
        }
        st = run_ops_any(ctx, wf->dtype, wf->n, wf->batch, ops, wf->data);
    }
    db.release();
    return st;
}

// =========================================================================== fused Fresnel plan

namespace {

// Plan-time autotuner: times the candidate row and column kernels on a scratch field of the
// plan's size and keeps the fastest (CORO_AUTOTUNE=0 keeps the defaults).
bool autotune_enabled() {
    const char* v = std::getenv("CORO_AUTOTUNE");
    return !(v && v[0] == '0');
}

template <typename C>
float time_ops(coro_ctx ctx, int n, int batch, const std::vector<Op>& ops, void* field, int reps,
               void* tbuf = nullptr) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return 1e30f;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return 1e30f; }
    float ms = 1e30f;
    if (run_ops<C>(ctx, n, batch, ops, field, nullptr, tbuf) == CORO_OK) {          // warm-up
        cudaEventRecord(a, ctx->stream);
        bool ok = true;
        for (int r = 0; r < reps && ok; ++r) ok = run_ops<C>(ctx, n, batch, ops, field, nullptr, tbuf) == CORO_OK;
        cudaEventRecord(b, ctx->stream);
        if (ok && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    clear_error();
    return ms;
}

// The ops with the elements that write outside the field (checkpoints, phase-gradient taps)
// left out, for timing runs on a scratch field: tuning never touches the caller's buffers.
std::vector<Op> timing_copy(const std::vector<Op>& ops) {
    std::vector<Op> out = ops;
    for (Op& op : out) {
        int k = 0;
        for (int i = 0; i < op.elems.count; ++i)
            if (op.elems.e[i].kind != DK_STORE && op.elems.e[i].kind != DK_PHASE_GRAD) op.elems.e[k++] = op.elems.e[i];
        op.elems.count = k;
    }
    return out;
}

coro_status autotune_ops(coro_ctx ctx, int dtype, int n, int batch, std::vector<Op>& ops, std::vector<std::string>* log) {
    if (dtype != CORO_C64 || !autotune_enabled()) return CORO_OK;
    int cand[8], rcand[8];
    const int nc = col_candidates(n, cand), nr = row_candidates(n, rcand);
    if (nc < 2 && nr < 2) return CORO_OK;
    coro_status st = CORO_OK;
    void* scratch = upload_async(ctx, nullptr, (size_t)batch * n * n * sizeof(float2), &st);
    if (!scratch) { clear_error(); return CORO_OK; }      // no room to tune: keep the defaults
    cudaMemsetAsync(scratch, 0, (size_t)batch * n * n * sizeof(float2), ctx->stream);
    const std::vector<Op> tops = timing_copy(ops);
    const Op* col = nullptr;
    const Op* row = nullptr;
    for (const Op& op : tops) {
        if (!op.row && !col) col = &op;
        if (op.row && (op.row_flags & (RF_INV_FIRST | RF_FWD_AFTER)) && (!row || (row->row_flags & RF_INIT_ONE))) row = &op;
    }
    int best_lines = 0, best_variant = 0;
    std::vector<std::pair<float, int>> row_ms;
    if (col && nc > 1) {
        float best = 1e30f;
        for (int i = 0; i < nc; ++i) {
            Op t = *col;
            t.lines = cand[i];
            const float ms = time_ops<float2>(ctx, n, batch, {t}, scratch, 3);
            if (log) log->push_back("col lines " + std::to_string(cand[i]) + ": " + std::to_string(ms / 3) + " ms");
            if (ms < best) { best = ms; best_lines = cand[i]; }
        }
    }
    if (row && nr > 1) {
        float best = 1e30f;
        for (int iv = 0; iv < nr; ++iv) {
            const int v = rcand[iv];
            Op t = *row;
            t.variant = v;
            const float ms = time_ops<float2>(ctx, n, batch, {t}, scratch, 3);
            if (log) log->push_back("row variant " + std::to_string(v) + ": " + std::to_string(ms / 3) + " ms");
            if (ms < best) { best = ms; best_variant = v; }
            row_ms.push_back({ms, v});
        }
    }
    // one representative row pass does not rank variants within a few per cent of each other
    // reliably (passes differ in their elements): the two fastest are timed over every pass
    std::sort(row_ms.begin(), row_ms.end());
    if (row_ms.size() >= 2 && row_ms[1].first < 1.1f * row_ms[0].first) {
        float best = 1e30f;
        for (int c = 0; c < 2; ++c) {
            std::vector<Op> t = tops;
            for (Op& op : t) {
                if (op.row) op.variant = row_ms[c].second;
                else op.lines = best_lines;
            }
            const float ms = time_ops<float2>(ctx, n, batch, t, scratch, 3);
            if (log) log->push_back("all passes, row variant " + std::to_string(row_ms[c].second) + ": " + std::to_string(ms / 3) + " ms");
            if (ms < best) { best = ms; best_variant = row_ms[c].second; }
        }
    }
    for (Op& op : ops) {
        if (op.row) op.variant = best_variant;
        else op.lines = best_lines;
    }
    free_async(ctx, scratch);
    return CORO_OK;
}

struct FresnelPlan : coro_plan_s {
    coro_ctx ctx = nullptr;
    int device = 0;                  // kept so that destruction never touches the context
    int dtype = CORO_C64, n = 0, batch = 0;
    std::vector<Op> ops;             // as executed
    std::vector<Op> ops_nat;         // the same passes, every one in place on the natural layout
    void* tbuf = nullptr;            // transposed plane of the alternating layout (owned)
    DevBlocks db;
    std::vector<double> ps_final;
    std::vector<std::string> tune_log;
    std::vector<int> sys_spherical;    // pilot-beam plans: per user plane, 1 = spherical reference
    int sys_direct = -1;               // pilot-beam plans: direct sub-hops (-1: not a system plan)
    std::vector<std::vector<double>> plane_pitch;   // per compiled plane: per-item pixel scale
    std::vector<int> user_plane;                    // pilot-beam plans: compiled index of user plane p
    int kind() const override { return 1; }
    int launches() const override { return (int)ops.size(); }
    int timing_units() const override { return (int)ops.size(); }
    ~FresnelPlan() override {
        DeviceGuard g(device);
        cudaDeviceSynchronize();
        timing.release();
        graph.reset();
        db.release();
        if (tbuf) cudaFree(tbuf);
    }
};

// Alternating layout (complex64, n = 1024 ... 4096): a column pass followed by a row pass is
// run as the packed-pair column kernel writing its result transposed into tbuf (contiguous
// rows) and the packed-pair row kernel reading it back column-wise (TMA boxes), so that each
// of the two passes has one strided side instead of the column pass having two. Every other
// pass stays in place. Returns the number of such pairs.
int transposed_ops(int dtype, int n, const std::vector<Op>& nat, std::vector<Op>* out) {
    if (out) *out = nat;
    if (dtype != CORO_C64 || n < 1024 || n > 4096 || (n & (n - 1))) return 0;
    int pairs = 0;
    for (size_t i = 0; i + 1 < nat.size(); ++i) {
        if (nat[i].row || !nat[i + 1].row || (nat[i + 1].row_flags & RF_INIT_ONE)) continue;
        if (out) {
            (*out)[i].lines = -6;
            (*out)[i + 1].variant = 4;
        }
        ++pairs;
        ++i;
    }
    return pairs;
}

// Switch a plan between the natural (0) and the alternating (1) layout. CORO_ENOTIMPL where
// the plan has no column pass followed by a row pass at a size the pair kernels take.
coro_status set_layout(FresnelPlan* p, int transposed) {
    DeviceGuard g(p->device);
    std::vector<Op> t;
    if (transposed) {
        if (transposed_ops(p->dtype, p->n, p->ops_nat, &t) == 0) {
            set_error("alternating layout: complex64 plans with n = 1024, 2048 or 4096 and a column pass followed by a row pass only");
            return CORO_ENOTIMPL;
        }
        if (!p->tbuf) {
            const cudaError_t e = cudaMalloc(&p->tbuf, (size_t)p->batch * p->n * p->n * sizeof(float2));
            if (e != cudaSuccess) { p->tbuf = nullptr; return cuda_fail(e, "alternating layout plane"); }
        }
        p->ops = t;
    } else {
        p->ops = p->ops_nat;
        if (p->tbuf) {
            cudaDeviceSynchronize();
            cudaFree(p->tbuf);
            p->tbuf = nullptr;
        }
    }
    p->graph.reset();                                   // a captured graph holds the old kernels
    return CORO_OK;
}

}  // namespace

namespace {

// A hop between consecutive planes of a plan: method and per-item signed distance; direct
// hops may omit the input or output quadratic phase (pilot-beam scheme, waist planes).
struct HopSpec {
    int method = CORO_FRESNEL_AS;
    std::vector<double> z;
    bool qin = true, qout = true;
};
// A plane: user elements, then optional per-item quadratic phases exp(i pi r^2 c_b / lambda_b)
// (curvature c_b in 1/m; reference-surface changes and lenses of the pilot-beam scheme).
struct PlaneSpec {
    std::vector<const coro_element*> user;
    std::vector<std::vector<double>> qpf;
};

// exp(i pi r^2 c_b / lambda_b) on the plane's grid as a separable table element.
coro_status qpf_elem(DevBlocks& db, bool dbl, int n, int batch, const double* ps, const double* lam,
                     const std::vector<double>& c, DevElem* out) {
    coro_status st = CORO_OK;
    std::vector<TabSpec> sp(batch);
    for (int b = 0; b < batch; ++b) sp[b] = TabSpec{ps[b] * ps[b] * c[b] / (2.0 * lam[b]), 1.0, 0.0, +1, 0};
    *out = table_elem(make_table(db, dbl, n, sp, &st));
    return out->tab ? CORO_OK : st;
}

// Compile planes and hops into row / column passes (the fused pass scheduler shared by the
// explicit and the pilot-beam plan builders).
coro_status build_passes(FresnelPlan* plan, int n, int batch, const double* ps0, const double* lam,
                         const std::vector<PlaneSpec>& planes, const std::vector<HopSpec>& hops, int flags) {
    coro_status st = CORO_OK;
    const bool dbl = plan->dtype == CORO_C128;
    std::vector<double> ps(ps0, ps0 + batch);
    enum { NATURAL, UNIFORM, SPECTRUM } state = (flags & CORO_PLAN_INIT_UNIFORM) ? UNIFORM : NATURAL;
    bool conj_pending = false;                 // the stored field is the conjugate of the true one
    const int n_planes = (int)planes.size();
    plan->plane_pitch.assign(n_planes, std::vector<double>());
    for (int p = 0; p < n_planes; ++p) {
        plan->plane_pitch[p] = ps;
        PassElems pe{};
        auto push = [&](const DevElem& e) -> bool {
            if (pe.count >= kMaxPassElems - 3) {
                set_error("plane %d: more than %d elements", p, kMaxPassElems - 3);
                return false;
            }
            pe.e[pe.count++] = e;
            return true;
        };
        if (conj_pending) {
            if (!push(conj_elem())) return CORO_ENOTIMPL;
            conj_pending = false;
        }
        for (const coro_element* el : planes[p].user) {
            DevElem e;
            if ((st = compile_element(plan->db, el, dbl, n, batch, ps.data(), lam, &e)) != CORO_OK) return st;
            // after an angular-spectrum hop the row pass holds the field times (-1)^(x+y)
            // (the fftshift sign is carried into the next forward FFT); checkpoints undo it
            if ((e.kind == DK_STORE || e.kind == DK_PHASE_GRAD) && state == SPECTRUM) e.flags |= 1;
            if (!push(e)) return CORO_ENOTIMPL;
        }
        for (const auto& c : planes[p].qpf) {
            DevElem e;
            if ((st = qpf_elem(plan->db, dbl, n, batch, ps.data(), lam, c, &e)) != CORO_OK) return st;
            if (!push(e)) return CORO_ENOTIMPL;
        }
        Op r;
        r.row = true;
        r.elems = pe;
        if (state == SPECTRUM) r.row_flags |= RF_INV_FIRST;
        if (state == UNIFORM) r.row_flags |= RF_INIT_ONE;
        if (p + 1 < n_planes) {
            const HopSpec& h = hops[p];
            r.row_flags |= RF_FWD_AFTER;
            Op c;
            c.row = false;
            if (h.method == CORO_FRESNEL_AS) {
                const void* tab = nullptr;
                if ((st = as_table(plan->db, dbl, n, batch, ps.data(), lam, h.z.data(), &tab)) != CORO_OK) return st;
                if (state != SPECTRUM) r.elems.e[r.elems.count++] = checker_elem();
                c.col_flags = CF_FWD | CF_TABLE | CF_INV;
                c.tab_x = c.tab_y = tab;
                state = SPECTRUM;
            } else {
                const bool neg = h.z[0] < 0;
                for (int b = 1; b < batch; ++b)
                    if ((h.z[b] < 0) != neg) { set_error("hop %d: items disagree on the direction of a direct hop", p); return CORO_ENOTIMPL; }
                const void *qin = nullptr, *qx = nullptr, *qy = nullptr;
                std::vector<double> ps_next;
                if ((st = direct_tables(plan->db, dbl, n, batch, ps.data(), lam, h.z.data(), h.qin, h.qout, &qin, &qx, &qy,
                                        ps_next)) != CORO_OK)
                    return st;
                if (neg) r.elems.e[r.elems.count++] = conj_elem();
                if (qin) r.elems.e[r.elems.count++] = table_elem(qin);
                if (state != SPECTRUM) r.elems.e[r.elems.count++] = checker_elem();
                c.col_flags = CF_FWD | CF_TABLE;
                c.tab_x = qx;
                c.tab_y = qy;
                ps = ps_next;
                state = NATURAL;
                conj_pending = neg;
            }
            plan->ops.push_back(r);
            plan->ops.push_back(c);
        } else {
            if (state == SPECTRUM) r.elems.e[r.elems.count++] = checker_elem();
            if (r.row_flags || r.elems.count) plan->ops.push_back(r);
            state = NATURAL;
        }
    }
    plan->ps_final = ps;
    return CORO_OK;
}

// Layout choice: CORO_LAYOUT=0 / 1 forces the natural / alternating layout; otherwise the
// alternating one is timed against the natural one when tuning is on and kept if faster
// (natural without tuning).
void choose_layout(FresnelPlan* p) {
    if (transposed_ops(p->dtype, p->n, p->ops_nat, nullptr) == 0) return;
    const char* v = std::getenv("CORO_LAYOUT");
    const bool force = v && v[0] == '1';
    if ((v && v[0] == '0') || (!force && !autotune_enabled())) return;
    if (set_layout(p, 1) != CORO_OK) { clear_error(); return; }     // no room: natural layout
    if (force) return;
    coro_status st = CORO_OK;
    const size_t bytes = (size_t)p->batch * p->n * p->n * sizeof(float2);
    void* scratch = upload_async(p->ctx, nullptr, bytes, &st);
    if (!scratch) { clear_error(); return; }
    cudaMemsetAsync(scratch, 0, bytes, p->ctx->stream);
    const float t_nat = time_ops<float2>(p->ctx, p->n, p->batch, timing_copy(p->ops_nat), scratch, 3);
    const float t_alt = time_ops<float2>(p->ctx, p->n, p->batch, timing_copy(p->ops), scratch, 3, p->tbuf);
    free_async(p->ctx, scratch);
    p->tune_log.push_back("layout natural: " + std::to_string(t_nat / 3) + " ms, alternating: " +
                          std::to_string(t_alt / 3) + " ms");
    if (!(t_alt < t_nat)) set_layout(p, 0);
}

coro_status finish_plan(coro_ctx ctx, std::unique_ptr<FresnelPlan>& plan, coro_plan* out, const char* who) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);   // tables ready; plan owns them
    if (e == cudaSuccess) {
        autotune_ops(ctx, plan->dtype, plan->n, plan->batch, plan->ops, &plan->tune_log);
        plan->ops_nat = plan->ops;
        choose_layout(plan.get());
        e = cudaStreamSynchronize(ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, who);
    *out = plan.release();
    return CORO_OK;
}

std::unique_ptr<FresnelPlan> new_plan(coro_ctx ctx, int dtype, int n, int batch) {
    auto plan = std::unique_ptr<FresnelPlan>(new (std::nothrow) FresnelPlan);
    if (!plan) return plan;
    plan->ctx = ctx;
    plan->device = ctx->device;
    plan->dtype = dtype;
    plan->n = n;
    plan->batch = batch;
    plan->db.ctx = ctx;
    plan->db.plan_owned = true;
    return plan;
}

}  // namespace

extern "C" coro_status coro_fresnel_plan_create(coro_ctx ctx, const coro_fresnel_desc* d, coro_plan* out) {
    clear_error();
    if (!ctx || !d || !out) { set_error("coro_fresnel_plan_create: NULL argument"); return CORO_EINVAL; }
    *out = nullptr;
    coro_wavefront probe{(void*)1, d->dtype, d->batch, d->n, const_cast<double*>(d->pixelscale), d->wavelength};
    coro_status st = check_wf("coro_fresnel_plan_create", ctx, &probe);
    if (st != CORO_OK) return st;
    if (d->n_planes < 1) { set_error("coro_fresnel_plan_create: n_planes must be >= 1"); return CORO_EINVAL; }
    if (d->n_planes > 1 && !d->distance) { set_error("coro_fresnel_plan_create: distance is NULL"); return CORO_EINVAL; }
    if (d->n_elements < 0 || (d->n_elements > 0 && !d->elements)) { set_error("coro_fresnel_plan_create: bad element list"); return CORO_EINVAL; }
    for (int p = 0; p + 1 < d->n_planes; ++p) {
        if (!(d->distance[p] != 0.0) || !std::isfinite(d->distance[p])) { set_error("distance[%d] must be finite and nonzero", p); return CORO_EINVAL; }
        const int m = d->method ? d->method[p] : CORO_FRESNEL_AS;
        if (m != CORO_FRESNEL_AS && m != CORO_FRESNEL_DIRECT) { set_error("method[%d] = %d", p, m); return CORO_EINVAL; }
    }
    for (int i = 0; i < d->n_elements; ++i)
        if (d->elements[i].plane < 0 || d->elements[i].plane >= d->n_planes) { set_error("element %d: plane %d out of range", i, d->elements[i].plane); return CORO_EINVAL; }

    DeviceGuard g(ctx->device);
    auto plan = new_plan(ctx, d->dtype, d->n, d->batch);
    if (!plan) { set_error("out of host memory"); return CORO_ENOMEM; }
    std::vector<PlaneSpec> planes(d->n_planes);
    std::vector<HopSpec> hops(d->n_planes > 0 ? d->n_planes - 1 : 0);
    for (int i = 0; i < d->n_elements; ++i) planes[d->elements[i].plane].user.push_back(&d->elements[i]);
    for (int p = 0; p + 1 < d->n_planes; ++p) {
        hops[p].method = d->method ? d->method[p] : CORO_FRESNEL_AS;
        hops[p].z.assign(d->batch, d->distance[p]);
    }
    if ((st = build_passes(plan.get(), d->n, d->batch, d->pixelscale, d->wavelength, planes, hops, d->flags)) != CORO_OK)
        return st;
    return finish_plan(ctx, plan, out, "coro_fresnel_plan_create");
}

// ------------------------------------------------------------------------------ f2: pilot beam

extern "C" coro_status coro_fresnel_system_create(coro_ctx ctx, const coro_fresnel_system_desc* d, coro_plan* out) {
    clear_error();
    if (!ctx || !d || !out) { set_error("coro_fresnel_system_create: NULL argument"); return CORO_EINVAL; }
    *out = nullptr;
    coro_wavefront probe{(void*)1, d->dtype, d->batch, d->n, const_cast<double*>(d->pixelscale), d->wavelength};
    coro_status st = check_wf("coro_fresnel_system_create", ctx, &probe);
    if (st != CORO_OK) return st;
    if (!(d->beam_radius > 0) || !std::isfinite(d->beam_radius)) { set_error("coro_fresnel_system_create: beam_radius must be > 0"); return CORO_EINVAL; }
    if (d->n_planes < 1) { set_error("coro_fresnel_system_create: n_planes must be >= 1"); return CORO_EINVAL; }
    if (d->n_planes > 1 && !d->distance) { set_error("coro_fresnel_system_create: distance is NULL"); return CORO_EINVAL; }
    if (d->n_elements < 0 || (d->n_elements > 0 && !d->elements)) { set_error("coro_fresnel_system_create: bad element list"); return CORO_EINVAL; }
    for (int p = 0; p + 1 < d->n_planes; ++p)
        if (!(d->distance[p] != 0.0) || !std::isfinite(d->distance[p])) { set_error("distance[%d] must be finite and nonzero", p); return CORO_EINVAL; }
    for (int i = 0; i < d->n_elements; ++i) {
        const coro_element& el = d->elements[i];
        if (el.plane < 0 || el.plane >= d->n_planes) { set_error("element %d: plane %d out of range", i, el.plane); return CORO_EINVAL; }
        if (el.kind == CORO_EL_LENS && (el.focal_length == 0 || !std::isfinite(el.focal_length))) {
            set_error("element %d: lens focal length must be finite and nonzero", i);
            return CORO_EINVAL;
        }
    }
    const int B = d->batch;
    // pilot beam per item: q = z - z_waist - i z_R (the sign convention of the Fresnel kernel
    // exp(+i pi r^2/(lambda z)): a Gaussian exp(i pi r^2/(lambda q)) stays Gaussian)
    std::vector<std::complex<double>> q(B);
    for (int b = 0; b < B; ++b) q[b] = std::complex<double>(0.0, -M_PI * d->beam_radius * d->beam_radius / d->wavelength[b]);
    auto inside = [](std::complex<double> v) { return std::fabs(v.real()) < std::fabs(v.imag()); };
    auto agree = [&](const std::vector<std::complex<double>>& v, bool* in) -> bool {
        *in = inside(v[0]);
        for (int b = 1; b < B; ++b)
            if (inside(v[b]) != *in) return false;
        return true;
    };
    std::vector<PlaneSpec> planes;
    std::vector<HopSpec> hops;
    std::vector<int> spherical(d->n_planes, 0);
    int direct = 0;
    bool sph = false;                           // current plane: spherical reference (R = Re q)
    std::vector<int> user_plane(d->n_planes, 0);
    for (int p = 0; p < d->n_planes; ++p) {
        user_plane[p] = (int)planes.size();
        PlaneSpec ps;
        std::vector<double> curv(B, 0.0);
        bool lens = false;
        for (int i = 0; i < d->n_elements; ++i) {
            const coro_element& el = d->elements[i];
            if (el.plane != p) continue;
            if (el.kind != CORO_EL_LENS) { ps.user.push_back(&el); continue; }
            if (!lens && sph)                   // restore the true field: x exp(+i pi r^2/(lambda R))
                for (int b = 0; b < B; ++b) curv[b] += 1.0 / q[b].real();
            lens = true;
            for (int b = 0; b < B; ++b) {
                curv[b] -= 1.0 / el.focal_length;
                q[b] = 1.0 / (1.0 / q[b] - 1.0 / el.focal_length);
            }
        }
        if (lens) {
            bool in = true;
            if (!agree(q, &in)) { set_error("plane %d: items disagree on the pilot-beam regime after the lens", p); return CORO_ENOTIMPL; }
            sph = !in;
            if (sph)
                for (int b = 0; b < B; ++b) curv[b] -= 1.0 / q[b].real();
        }
        if (p + 1 == d->n_planes && sph) {      // hand back the true field on a planar reference
            if (!lens) std::fill(curv.begin(), curv.end(), 0.0);
            for (int b = 0; b < B; ++b) curv[b] += 1.0 / q[b].real();
            lens = true;
        }
        spherical[p] = sph ? 1 : 0;
        bool any = false;
        for (double c : curv) any = any || c != 0.0;
        if (lens && any) ps.qpf.push_back(curv);
        planes.push_back(ps);
        if (p + 1 == d->n_planes) break;
        // hop to plane p + 1
        const double dz = d->distance[p];
        std::vector<std::complex<double>> qb(B);
        for (int b = 0; b < B; ++b) qb[b] = q[b] + dz;
        bool in_a = !sph, in_b = true;
        if (!agree(qb, &in_b)) { set_error("hop %d: items disagree on the pilot-beam regime", p); return CORO_ENOTIMPL; }
        auto add_hop = [&](int method, std::vector<double> z, bool qin, bool qout) {
            HopSpec h;
            h.method = method;
            h.z = std::move(z);
            h.qin = qin;
            h.qout = qout;
            hops.push_back(h);
            if (method == CORO_FRESNEL_DIRECT) ++direct;
        };
        std::vector<double> to_waist(B), from_waist(B), whole(B, dz);
        bool zero_to = true, zero_from = true;
        for (int b = 0; b < B; ++b) {
            to_waist[b] = -q[b].real();
            from_waist[b] = qb[b].real();
            zero_to = zero_to && to_waist[b] == 0.0;
            zero_from = zero_from && from_waist[b] == 0.0;
        }
        if (in_a && in_b) {
            add_hop(CORO_FRESNEL_AS, whole, true, true);
        } else if (in_a) {                      // inside -> outside: to the waist, then WTS
            if (!zero_to) { add_hop(CORO_FRESNEL_AS, to_waist, true, true); planes.push_back(PlaneSpec{}); }
            add_hop(CORO_FRESNEL_DIRECT, from_waist, true, false);
        } else if (in_b) {                      // outside -> inside: STW, then from the waist
            add_hop(CORO_FRESNEL_DIRECT, to_waist, false, true);
            if (!zero_from) { planes.push_back(PlaneSpec{}); add_hop(CORO_FRESNEL_AS, from_waist, true, true); }
        } else {                                // outside -> outside through the waist
            add_hop(CORO_FRESNEL_DIRECT, to_waist, false, true);
            planes.push_back(PlaneSpec{});
            add_hop(CORO_FRESNEL_DIRECT, from_waist, true, false);
        }
        for (int b = 0; b < B; ++b) q[b] = qb[b];
        sph = !in_b;
    }
    DeviceGuard g(ctx->device);
    auto plan = new_plan(ctx, d->dtype, d->n, B);
    if (!plan) { set_error("out of host memory"); return CORO_ENOMEM; }
    plan->sys_spherical = spherical;
    plan->sys_direct = direct;
    plan->user_plane = user_plane;
    if ((st = build_passes(plan.get(), d->n, B, d->pixelscale, d->wavelength, planes, hops, d->flags)) != CORO_OK) return st;
    return finish_plan(ctx, plan, out, "coro_fresnel_system_create");
}

extern "C" coro_status coro_fresnel_system_pitch(coro_plan plan, int plane, double* pitch) {
    clear_error();
    if (!plan || plan->kind() != 1 || !pitch) { set_error("coro_fresnel_system_pitch: bad argument"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    const bool sys = p->sys_direct >= 0;
    const int count = sys ? (int)p->user_plane.size() : (int)p->plane_pitch.size();
    if (plane < 0 || plane >= count) { set_error("coro_fresnel_system_pitch: plane %d of %d", plane, count); return CORO_EINVAL; }
    const std::vector<double>& v = p->plane_pitch[sys ? p->user_plane[plane] : plane];
    std::copy(v.begin(), v.end(), pitch);
    return CORO_OK;
}

extern "C" coro_status coro_fresnel_system_info(coro_plan plan, int* spherical, int* direct_hops) {
    clear_error();
    if (!plan || plan->kind() != 1 || static_cast<FresnelPlan*>(plan)->sys_direct < 0) {
        set_error("coro_fresnel_system_info: not a plan made by coro_fresnel_system_create");
        return CORO_EINVAL;
    }
    auto* p = static_cast<FresnelPlan*>(plan);
    if (spherical) std::copy(p->sys_spherical.begin(), p->sys_spherical.end(), spherical);
    if (direct_hops) *direct_hops = p->sys_direct;
    return CORO_OK;
}

extern "C" coro_status coro_fresnel_plan_execute(coro_plan plan, void* field, double* pixelscale_out) {
    clear_error();
    if (!plan || plan->kind() != 1) { set_error("coro_fresnel_plan_execute: not a Fresnel plan"); return CORO_EINVAL; }
    if (!field) { set_error("coro_fresnel_plan_execute: field is NULL"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    DeviceGuard g(p->ctx->device);
    coro_status st = run_graphed(p->ctx, p->graph, {field, (const void*)1}, [&]() {
        return run_ops_any(p->ctx, p->dtype, p->n, p->batch, p->ops, field, p->timing.set(0), p->tbuf);
    });
    if (st == CORO_OK && pixelscale_out)
        for (int b = 0; b < p->batch; ++b) pixelscale_out[b] = p->ps_final[b];
    return st;
}

extern "C" coro_status coro_fresnel_plan_execute_n(coro_plan plan, void* field, int times) {
    clear_error();
    if (!plan || plan->kind() != 1) { set_error("coro_fresnel_plan_execute_n: not a Fresnel plan"); return CORO_EINVAL; }
    if (!field || times < 1) { set_error("coro_fresnel_plan_execute_n: field NULL or times < 1"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    DeviceGuard g(p->ctx->device);
    return run_graphed(p->ctx, p->graph, {field, (const void*)(intptr_t)times}, [&]() {
        coro_status st = CORO_OK;
        for (int k = 0; k < times && st == CORO_OK; ++k)
            st = run_ops_any(p->ctx, p->dtype, p->n, p->batch, p->ops, field, p->timing.set(k), p->tbuf);
        return st;
    });
}

extern "C" coro_status coro_fresnel_plan_execute_range(coro_plan plan, void* field, int first, int count) {
    clear_error();
    if (!plan || plan->kind() != 1) { set_error("coro_fresnel_plan_execute_range: not a Fresnel plan"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    if (!field || first < 0 || count < 0 || first + count > (int)p->ops.size()) {
        set_error("coro_fresnel_plan_execute_range: bad field or range [%d, %d) of %d", first, first + count, (int)p->ops.size());
        return CORO_EINVAL;
    }
    DeviceGuard g(p->ctx->device);
    std::vector<Op> sub(p->ops_nat.begin() + first, p->ops_nat.begin() + first + count);   // in place
    return run_ops_any(p->ctx, p->dtype, p->n, p->batch, sub, field);
}

extern "C" coro_status coro_fresnel_plan_pass_flops(coro_plan plan, int i, double* flops) {
    clear_error();
    if (!plan || plan->kind() != 1 || !flops) { set_error("coro_fresnel_plan_pass_flops: bad argument"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    if (i < 0 || i >= (int)p->ops.size()) { set_error("coro_fresnel_plan_pass_flops: pass %d of %d", i, (int)p->ops.size()); return CORO_EINVAL; }
    const Op& op = p->ops[i];
    const int transforms = op.row ? ((op.row_flags & RF_INV_FIRST) ? 1 : 0) + ((op.row_flags & RF_FWD_AFTER) ? 1 : 0)
                                  : ((op.col_flags & CF_FWD) ? 1 : 0) + ((op.col_flags & CF_INV) ? 1 : 0);
    const double n = p->n;
    *flops = transforms * 5.0 * n * std::log2(n) * n * p->batch;
    return CORO_OK;
}

extern "C" coro_status coro_fresnel_plan_pass_info(coro_plan plan, int i, int* is_row, double* bytes) {
    clear_error();
    if (!plan || plan->kind() != 1 || !is_row || !bytes) { set_error("coro_fresnel_plan_pass_info: bad argument"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    if (i < 0 || i >= (int)p->ops.size()) { set_error("coro_fresnel_plan_pass_info: pass %d of %d", i, (int)p->ops.size()); return CORO_EINVAL; }
    const Op& op = p->ops[i];
    const double field = (double)p->batch * p->n * p->n * (p->dtype == CORO_C64 ? 8.0 : 16.0);
    const double plane = (double)p->n * p->n * 4.0;
    double b = field;                                   // write
    if (!op.row || !(op.row_flags & RF_INIT_ONE)) b += field;   // read
    if (op.row) {
        for (int k = 0; k < op.elems.count; ++k) {
            const DevElem& e = op.elems.e[k];
            if (e.kind != DK_OPD_MAP) continue;
            const double maps = e.map_bstride ? (double)p->batch : 1.0;
            b += plane * maps * (e.amp ? 2.0 : 1.0);
        }
    }
    *is_row = op.row ? 1 : 0;
    *bytes = b;
    return CORO_OK;
}

extern "C" coro_status coro_fresnel_plan_pass_kernel(coro_plan plan, int i, int* persistent, int* lines) {
    clear_error();
    if (!plan || plan->kind() != 1) { set_error("coro_fresnel_plan_pass_kernel: not a Fresnel plan"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    if (i < 0 || i >= (int)p->ops.size()) { set_error("coro_fresnel_plan_pass_kernel: pass %d of %d", i, (int)p->ops.size()); return CORO_EINVAL; }
    const Op& op = p->ops[i];
    describe_pass(p->n, p->dtype == CORO_C128, op.row, op.variant, op.lines, persistent, lines);
    return CORO_OK;
}

extern "C" coro_status coro_fresnel_plan_pass_radix(coro_plan plan, int i, int* radices, int max_radices, int* stages) {
    clear_error();
    if (!plan || plan->kind() != 1) { set_error("coro_fresnel_plan_pass_radix: not a Fresnel plan"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    if (i < 0 || i >= (int)p->ops.size()) { set_error("coro_fresnel_plan_pass_radix: pass %d of %d", i, (int)p->ops.size()); return CORO_EINVAL; }
    if (max_radices < 0 || (max_radices > 0 && !radices)) { set_error("coro_fresnel_plan_pass_radix: bad radices buffer"); return CORO_EINVAL; }
    const Op& op = p->ops[i];
    int r[16];
    const int k = pass_radices(p->n, op.row, p->dtype == CORO_C64 ? op.variant : 0, p->dtype == CORO_C64 ? op.lines : 0, r, 16);
    for (int j = 0; j < k && j < max_radices; ++j) radices[j] = r[j];
    if (stages) *stages = k;
    return CORO_OK;
}

extern "C" coro_status coro_fresnel_plan_set_pass_kernel(coro_plan plan, int row_variant, int col_lines) {
    clear_error();
    if (!plan || plan->kind() != 1) { set_error("coro_fresnel_plan_set_pass_kernel: not a Fresnel plan"); return CORO_EINVAL; }
    auto* p = static_cast<FresnelPlan*>(plan);
    if (p->dtype != CORO_C64) { set_error("coro_fresnel_plan_set_pass_kernel: complex64 plans only"); return CORO_EINVAL; }
    int rcand[8];
    const int nr = row_candidates(p->n, rcand);
    bool row_ok = false;
    for (int i = 0; i < nr; ++i) row_ok = row_ok || rcand[i] == row_variant;
    if (!row_ok) {
        set_error("coro_fresnel_plan_set_pass_kernel: row variant %d not offered at n=%d", row_variant, p->n);
        return CORO_EINVAL;
    }
    bool col_ok = col_lines == 0;
    int cand[8];
    const int nc = col_candidates(p->n, cand);
    for (int i = 0; i < nc; ++i) col_ok = col_ok || cand[i] == col_lines;
    if (!col_ok) {
        set_error("coro_fresnel_plan_set_pass_kernel: column kernel %d not offered at n=%d", col_lines, p->n);
        return CORO_EINVAL;
    }
    for (Op& op : p->ops_nat) {
        if (op.row) op.variant = row_variant;
        else op.lines = col_lines;
    }
    return set_layout(p, 0);                            // every pass in place with these kernels
}

extern "C" coro_status coro_fresnel_plan_copy_tuning(coro_plan dst, coro_plan src) {
    clear_error();
    if (!dst || !src || dst->kind() != 1 || src->kind() != 1) {
        set_error("coro_fresnel_plan_copy_tuning: not two Fresnel plans");
        return CORO_EINVAL;
    }
    auto* d = static_cast<FresnelPlan*>(dst);
    auto* s = static_cast<const FresnelPlan*>(src);
    bool same = d->dtype == s->dtype && d->n == s->n && d->batch == s->batch && d->ops_nat.size() == s->ops_nat.size();
    for (size_t i = 0; same && i < d->ops_nat.size(); ++i) same = d->ops_nat[i].row == s->ops_nat[i].row;
    if (!same) {
        set_error("coro_fresnel_plan_copy_tuning: plans differ in dtype, size, batch or pass sequence");
        return CORO_EINVAL;
    }
    for (size_t i = 0; i < d->ops_nat.size(); ++i) {
        d->ops_nat[i].variant = s->ops_nat[i].variant;
        d->ops_nat[i].lines = s->ops_nat[i].lines;
    }
    d->ops = d->ops_nat;
    coro_status st = set_layout(d, 0);
    if (st == CORO_OK && s->tbuf) st = set_layout(d, 1);
    return st;
}

extern "C" coro_status coro_fresnel_plan_set_layout(coro_plan plan, int transposed) {
    clear_error();
    if (!plan || plan->kind() != 1) { set_error("coro_fresnel_plan_set_layout: not a Fresnel plan"); return CORO_EINVAL; }
    if (transposed != 0 && transposed != 1) { set_error("coro_fresnel_plan_set_layout: transposed must be 0 or 1"); return CORO_EINVAL; }
    return set_layout(static_cast<FresnelPlan*>(plan), transposed);
}

extern "C" coro_status coro_fresnel_plan_layout(coro_plan plan, int* transposed) {
    clear_error();
    if (!plan || plan->kind() != 1 || !transposed) { set_error("coro_fresnel_plan_layout: bad argument"); return CORO_EINVAL; }
    *transposed = static_cast<FresnelPlan*>(plan)->tbuf ? 1 : 0;
    return CORO_OK;
}

extern "C" coro_status coro_plan_launch_count(coro_plan plan, int* out) {
    clear_error();
    if (!plan || !out) { set_error("coro_plan_launch_count: NULL argument"); return CORO_EINVAL; }
    *out = plan->launches();
    return CORO_OK;
}

extern "C" coro_status coro_plan_set_timing(coro_plan plan, int steps) {
    clear_error();
    if (!plan || steps < 0) { set_error("coro_plan_set_timing: NULL plan or steps < 0"); return CORO_EINVAL; }
    PlanTiming& t = plan->timing;
    cudaDeviceSynchronize();                             // no recorded event may be in flight
    t.release();
    plan->graph.reset();                                 // a captured graph holds the old events
    if (steps == 0) return CORO_OK;
    t.units = plan->timing_units();
    t.ev.resize((size_t)steps * (t.units + 1));
    for (auto& e : t.ev) {
        const cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) {
            e = nullptr;
            for (auto& x : t.ev) if (x) cudaEventDestroy(x);
            t.ev.clear();
            return cuda_fail(r, "coro_plan_set_timing: cudaEventCreate");
        }
    }
    t.steps = steps;
    return CORO_OK;
}

extern "C" coro_status coro_plan_unit_times(coro_plan plan, int steps, float* ms) {
    clear_error();
    if (!plan || !ms || steps < 1 || steps > plan->timing.steps) {
        set_error("coro_plan_unit_times: bad argument (timing holds %d steps)", plan ? plan->timing.steps : 0);
        return CORO_EINVAL;
    }
    const PlanTiming& t = plan->timing;
    cudaError_t e = cudaEventSynchronize(t.ev[(size_t)(steps - 1) * (t.units + 1) + t.units]);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        const cudaEvent_t* s = t.set(k);
        for (int i = 0; i < t.units && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[k * t.units + i], s[i], s[i + 1]);
    }
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "coro_plan_unit_times");
}

extern "C" coro_status coro_plan_set_graph(coro_plan plan, int enable) {
    clear_error();
    if (!plan) { set_error("coro_plan_set_graph: NULL plan"); return CORO_EINVAL; }
    plan->graph.enabled = enable != 0;
    plan->graph.reset();
    return CORO_OK;
}

extern "C" coro_status coro_plan_destroy(coro_plan plan) {
    clear_error();
    delete plan;
    return CORO_OK;
}

// =========================================================================== a9: detector

namespace {

template <typename C>
__global__ void intensity_kernel(const C* __restrict__ e, float* __restrict__ out, size_t per_item,
                                 int batch, const double* __restrict__ inv_norm) {
    const size_t total = per_item * batch;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const C v = e[i];
        const double s = inv_norm[i / per_item];
        out[i] = (float)(((double)v.x * v.x + (double)v.y * v.y) * s);
    }
}

// Dark-hole sum: one block row per item; pixels with lo <= r2 <= hi (integer radii squared).
template <typename C>
__global__ void darkhole_kernel(const C* __restrict__ e, int n, const long long* __restrict__ lohi,
                                const double* __restrict__ inv_norm, double* __restrict__ acc) {
    const int b = blockIdx.y;
    const long long lo = lohi[2 * b], hi = lohi[2 * b + 1];
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
        if (threadIdx.x == 0) atomicAdd(acc + b, s * inv_norm[b]);
    }
}

}  // namespace

extern "C" coro_status coro_intensity(coro_ctx ctx, const coro_wavefront* wf, const double* norm, float* out) {
    clear_error();
    coro_status st = check_wf("coro_intensity", ctx, wf, false);
    if (st != CORO_OK) return st;
    if (!out) { set_error("coro_intensity: out is NULL"); return CORO_EINVAL; }
    std::vector<double> inv(wf->batch, 1.0);
    for (int b = 0; b < wf->batch && norm; ++b) {
        if (!(norm[b] > 0)) { set_error("coro_intensity: norm[%d] must be > 0", b); return CORO_EINVAL; }
        inv[b] = 1.0 / norm[b];
    }
    DeviceGuard g(ctx->device);
    void* inv_d = upload_async(ctx, inv.data(), inv.size() * sizeof(double), &st);
    if (!inv_d) return st;
    const size_t per = (size_t)wf->n * wf->n;
    const int blocks = (int)std::min<size_t>((per * wf->batch + 255) / 256, 152 * 8);
    if (wf->dtype == CORO_C64) intensity_kernel<float2><<<blocks, 256, 0, ctx->stream>>>((const float2*)wf->data, out, per, wf->batch, (const double*)inv_d);
    else intensity_kernel<double2><<<blocks, 256, 0, ctx->stream>>>((const double2*)wf->data, out, per, wf->batch, (const double*)inv_d);
    cudaError_t e = cudaGetLastError();
    free_async(ctx, inv_d);
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "intensity_kernel");
}

extern "C" coro_status coro_darkhole_sum(coro_ctx ctx, const coro_wavefront* wf, const double* du, double r_in,
                                         double r_out, const double* norm, double* host_out) {
    clear_error();
    coro_status st = check_wf("coro_darkhole_sum", ctx, wf, false);
    if (st != CORO_OK) return st;
    if (!du || !host_out) { set_error("coro_darkhole_sum: du/host_out is NULL"); return CORO_EINVAL; }
    if (!(r_in >= 0) || !(r_out >= r_in)) { set_error("coro_darkhole_sum: need 0 <= r_in <= r_out"); return CORO_EINVAL; }
    const int batch = wf->batch;
    std::vector<long long> lohi(2 * batch);
    std::vector<double> inv(batch, 1.0);
    for (int b = 0; b < batch; ++b) {
        if (!(du[b] > 0)) { set_error("coro_darkhole_sum: du[%d] must be > 0", b); return CORO_EINVAL; }
        if (norm) {
            if (!(norm[b] > 0)) { set_error("coro_darkhole_sum: norm[%d] must be > 0", b); return CORO_EINVAL; }
            inv[b] = 1.0 / norm[b];
        }
        // lo = smallest m with m du^2 >= r_in^2 = (largest m with m du^2 < r_in^2) + 1
        lohi[2 * b] = disk_threshold(r_in, du[b], true) + 1;
        lohi[2 * b + 1] = disk_threshold(r_out, du[b], false);
    }
    DeviceGuard g(ctx->device);
    void* lohi_d = upload_async(ctx, lohi.data(), lohi.size() * sizeof(long long), &st);
    if (!lohi_d) return st;
    void* inv_d = upload_async(ctx, inv.data(), inv.size() * sizeof(double), &st);
    void* acc_d = inv_d ? upload_async(ctx, nullptr, batch * sizeof(double), &st) : nullptr;
    cudaError_t e = cudaSuccess;
    if (acc_d) {
        e = cudaMemsetAsync(acc_d, 0, batch * sizeof(double), ctx->stream);
        const int n = wf->n;
        dim3 grid((unsigned)std::min(64, (n * n + 255) / 256), batch);
        if (e == cudaSuccess) {
            if (wf->dtype == CORO_C64) darkhole_kernel<float2><<<grid, 256, 0, ctx->stream>>>((const float2*)wf->data, n, (const long long*)lohi_d, (const double*)inv_d, (double*)acc_d);
            else darkhole_kernel<double2><<<grid, 256, 0, ctx->stream>>>((const double2*)wf->data, n, (const long long*)lohi_d, (const double*)inv_d, (double*)acc_d);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, acc_d, batch * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "coro_darkhole_sum");
    }
    free_async(ctx, lohi_d);
    free_async(ctx, inv_d);
    free_async(ctx, acc_d);
    return st;
}
