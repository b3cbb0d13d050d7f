// wfc.cu -- differentiable wavefront control: dark-hole intensity and its gradient with
// respect to the heights of two deformable mirrors (DM1 at the pupil, DM2 a Fresnel hop z
// away), summed over wavelengths.
//
// Forward, per wavelength (the hop uses the angular-spectrum method of Sec. 1.1):
//   E0 = A exp(i phi1),  E1 = AS(+z) E0,  E2 = E1 exp(i phi2),  E3 = AS(-z) E2,
//   E_A = centre n x n of E3 -> Lyot chain -> S = sum over the dark hole of |E_det|^2 / peak
// with phi = 2 pi OPD / lambda and OPD = 2 x (Gaussian-influence DM surface).
// Adjoint (G = dL/dconj(E), AS(z)^H = AS(-z), phase elements pass G times exp(-i phi)):
//   G3 = pad(dS/dconj(E_A)),  G2 = AS(+z) G3,  dL/dphi2 = 2 Im(G2 conj(E2)),
//   G0 = AS(-z)(exp(-i phi2) G2),  dL/dphi1 = 2 Im(G0 conj(E0)),
//   dL/dh = sum_lambda (4 pi / lambda) G_infl^T (dL/dphi) G_infl.
// The wavelength sum is folded into one weighted map per DM before the DM correlation.
// Each chain runs as one fused Fresnel plan (five row / column passes for the two hops):
// forward  init . aperture . phi1 -> AS(+z) -> [checkpoint E1] . phi2 -> AS(-z)
// adjoint  G3 -> AS(+z) -> exp(-i phi2) . [dL/dphi2 tap vs E1] -> AS(-z)
//          -> aperture . exp(-i phi1) . [dL/dphi1 tap vs 1]
// with the checkpoint and the taps written by the row passes themselves (no separate copies).
// The dphi2 tap uses 2 Im(G2 conj(E2)) = 2 Im(G1 conj(E1)) with G1 = exp(-i phi2) G2, so it
// sits after the conjugate phase and needs only E1; E0 = A exp(i phi1) is known in closed
// form, so 2 Im(G0 conj(E0)) = 2 Im(A exp(-i phi1) G0) is a tap against a unit reference
// after the aperture and the conjugate DM1 phase, and E0 is never stored. Each tap writes one
// weighted map per wavelength; the DM correlation reads them per wavelength and a last
// kernel sums over them.
//
// HBM budget: the three full-grid fields per wavelength (checkpoint E1, the Lyot pupil / tap
// maps, the adjoint field) are 24 N^2 bytes, 1.5 GiB per wavelength at N = 8192. The
// plan keeps at most `resident` wavelengths in memory and runs the band in chunks of that
// many (one set of fused plans and one Lyot plan per chunk, all on the same buffers); the
// gradient sums the chunks' contributions in order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "capi_common.h"

namespace {

// grad[dm][p][q] (+)= sum_b part[dm][b][p][q]  (accumulate: add to what grad holds)
__global__ void sum_items_kernel(const float* __restrict__ part, int batch, int per_dm, int accumulate,
                                 float* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, dm = blockIdx.y;
    if (i >= per_dm) return;
    const float* src = part + (size_t)dm * batch * per_dm + i;
    float acc = accumulate ? grad[(size_t)dm * per_dm + i] : 0.f;
    for (int b = 0; b < batch; ++b) acc += src[(size_t)b * per_dm];
    grad[(size_t)dm * per_dm + i] = acc;
}

// One group of wavelengths [b0, b0 + nb) resident at a time, with its own plans.
struct Chunk {
    int b0 = 0, nb = 0;
    coro_plan lyot = nullptr;
    coro_plan fwd = nullptr, adj = nullptr;     // fused Fresnel plans of the two chains
};

struct WfcPlan : coro_plan_s {
    coro_ctx ctx = nullptr;
    int device = 0;
    coro_wfc_desc d{};
    std::vector<double> lam, ps;
    std::vector<coro_lyot_item> items;
    int resident = 0;                           // wavelengths whose fields fit at once
    std::vector<Chunk> chunks;
    std::vector<void*> bufs;
    float2 *e1 = nullptr, *w = nullptr, *g = nullptr;
    float *opd1 = nullptr, *opd1n = nullptr, *opd2 = nullptr, *opd2n = nullptr, *zero_h = nullptr;
    float* part = nullptr;                      // [2][resident][n_act][n_act] per-wavelength dL/dh
    std::vector<double> peak;
    int kind() const override { return 3; }
    int launches() const override { return 0; }
    int timing_units() const override { return 0; }
    ~WfcPlan() override {
        for (Chunk& ch : chunks) {
            if (ch.lyot) coro_plan_destroy(ch.lyot);
            if (ch.fwd) coro_plan_destroy(ch.fwd);
            if (ch.adj) coro_plan_destroy(ch.adj);
        }
        coro::DeviceGuard gd(device);
        cudaDeviceSynchronize();
        for (void* p : bufs) cudaFree(p);
    }
    void* alloc(size_t bytes, coro_status* st) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) { *st = coro::cuda_fail(e, "coro_wfc_plan_create: cudaMalloc"); return nullptr; }
        bufs.push_back(p);
        return p;
    }
};

coro_element opd_elem(const float* map) {
    coro_element e{};
    e.kind = CORO_EL_OPD_MAP;
    e.opd = map;
    return e;
}

// The DM surfaces of `heights` (shared by every wavelength and chunk).
coro_status dm_maps(WfcPlan* p, const float* heights) {
    const coro_wfc_desc& d = p->d;
    coro_ctx c = p->ctx;
    const int nf = d.n_fresnel, na = d.n_act;
    const double dx = d.diam_m / d.npix;
    coro_status st;
    if ((st = coro_dm_opd(c, heights, 1, na, d.act_pitch_m, d.act_fwhm_m, nf, dx, 2.0, p->opd1)) != CORO_OK) return st;
    if ((st = coro_dm_opd(c, heights, 1, na, d.act_pitch_m, d.act_fwhm_m, nf, dx, -2.0, p->opd1n)) != CORO_OK) return st;
    if ((st = coro_dm_opd(c, heights + na * na, 1, na, d.act_pitch_m, d.act_fwhm_m, nf, dx, 2.0, p->opd2)) != CORO_OK) return st;
    return coro_dm_opd(c, heights + na * na, 1, na, d.act_pitch_m, d.act_fwhm_m, nf, dx, -2.0, p->opd2n);
}

coro_element checkpoint_elem(int plane, void* store) {
    coro_element e{};
    e.kind = CORO_EL_CHECKPOINT;
    e.plane = plane;
    e.store = store;
    return e;
}

// The chunk's plans: Lyot chain and the two fused Fresnel chains (their element maps and
// checkpoint buffers are the WFC plan's own).
coro_status make_chunk(WfcPlan* p, Chunk& ch) {
    const coro_wfc_desc& d = p->d;
    const double z[2] = {d.z_m, -d.z_m};
    const int nf = d.n_fresnel;
    coro_lyot_desc ld{ch.nb, d.npix, (double)d.npix, d.lyot_frac, d.m_det, p->items.data() + ch.b0, d.precision};
    coro_status st = coro_lyot_plan_create(p->ctx, &ld, &ch.lyot);
    if (st != CORO_OK) return st;
    if ((st = coro_lyot_plan_set_pupil_layout(ch.lyot, nf, (long long)nf * nf)) != CORO_OK) return st;
    coro_element fe[4]{};
    fe[0].kind = CORO_EL_APERTURE;
    fe[0].radius = 0.5 * d.diam_m;
    fe[1] = opd_elem(p->opd1);
    fe[2] = checkpoint_elem(1, p->e1);
    fe[3] = opd_elem(p->opd2);
    fe[3].plane = 1;
    coro_fresnel_desc fd{};
    fd.dtype = CORO_C64;
    fd.batch = ch.nb;
    fd.n = d.n_fresnel;
    fd.pixelscale = p->ps.data() + ch.b0;
    fd.wavelength = p->lam.data() + ch.b0;
    fd.n_planes = 3;
    fd.distance = z;
    fd.n_elements = 4;
    fd.elements = fe;
    fd.flags = CORO_PLAN_INIT_UNIFORM;
    if ((st = coro_fresnel_plan_create(p->ctx, &fd, &ch.fwd)) != CORO_OK) return st;
    // per-wavelength dL/dh density maps in w (E3 is no longer needed by then): DM2 first
    const size_t npx = (size_t)d.n_fresnel * d.n_fresnel;
    float* dphi2 = reinterpret_cast<float*>(p->w);
    float* dphi1 = dphi2 + (size_t)ch.nb * npx;
    coro_element ae[5]{};
    ae[0] = opd_elem(p->opd2n);
    ae[0].plane = 1;
    ae[1].kind = CORO_EL_PHASE_GRAD;                 // (4 pi / lambda) 2 Im(G1 conj(E1))
    ae[1].plane = 1;
    ae[1].scalar = 4.0 * M_PI;
    ae[1].ref = p->e1;
    ae[1].store = dphi2;
    ae[2] = fe[0];                                   // A exp(-i phi1) G0 ...
    ae[2].plane = 2;
    ae[3] = opd_elem(p->opd1n);
    ae[3].plane = 2;
    ae[4] = ae[1];                                   // ... (4 pi / lambda) 2 Im(A exp(-i phi1) G0)
    ae[4].plane = 2;
    ae[4].ref = nullptr;
    ae[4].store = dphi1;
    fd.n_elements = 5;
    fd.elements = ae;
    fd.flags = 0;
    if ((st = coro_fresnel_plan_create(p->ctx, &fd, &ch.adj)) != CORO_OK) return st;
    if ((st = coro_plan_set_graph(ch.fwd, 1)) != CORO_OK) return st;
    return coro_plan_set_graph(ch.adj, 1);
}

float2* window(WfcPlan* p, float2* base) {
    const int nf = p->d.n_fresnel, n = p->d.npix;
    const size_t off = (size_t)(nf / 2 - n / 2) * nf + (nf / 2 - n / 2);
    return base + off;
}

}  // namespace

extern "C" coro_status coro_wfc_plan_create(coro_ctx ctx, const coro_wfc_desc* d, coro_plan* out) {
    coro::clear_error();
    if (!ctx || !d || !out || !d->wavelength || !d->items) { coro::set_error("coro_wfc_plan_create: NULL argument"); return CORO_EINVAL; }
    *out = nullptr;
    if (d->batch < 1 || d->batch > 1024) { coro::set_error("coro_wfc_plan_create: batch %d", d->batch); return CORO_ESIZE; }
    if (!coro::is_pow2(d->n_fresnel) || d->n_fresnel < 32 || d->n_fresnel > 8192 || d->npix < 16 || d->npix > d->n_fresnel ||
        (d->npix & 1)) {
        coro::set_error("coro_wfc_plan_create: n_fresnel must be a power of two in [32, 8192], npix even in [16, n_fresnel]");
        return CORO_ESIZE;
    }
    if (!(d->diam_m > 0) || !(d->z_m != 0) || d->n_act < 1 || !(d->act_pitch_m > 0) || !(d->act_fwhm_m > 0)) {
        coro::set_error("coro_wfc_plan_create: need diam, pitch, fwhm > 0, z != 0, n_act >= 1");
        return CORO_EINVAL;
    }
    if (d->max_resident < 0) { coro::set_error("coro_wfc_plan_create: max_resident must be >= 0"); return CORO_EINVAL; }
    for (int b = 0; b < d->batch; ++b)
        if (!(d->wavelength[b] > 0)) { coro::set_error("coro_wfc_plan_create: wavelength[%d] must be > 0", b); return CORO_EINVAL; }
    coro::DeviceGuard gd(ctx->device);
    auto p = std::unique_ptr<WfcPlan>(new (std::nothrow) WfcPlan);
    if (!p) { coro::set_error("out of host memory"); return CORO_ENOMEM; }
    p->ctx = ctx;
    p->device = ctx->device;
    p->d = *d;
    p->lam.assign(d->wavelength, d->wavelength + d->batch);
    p->ps.assign(d->batch, d->diam_m / d->npix);
    p->items.assign(d->items, d->items + d->batch);
    p->d.wavelength = p->lam.data();
    p->d.items = p->items.data();
    const int nf = d->n_fresnel;
    // E1, w, g; plus the transposed planes of the forward and adjoint plans should their
    // tuner pick the alternating layout (n_fresnel 1024 ... 4096)
    const size_t item_bytes = (size_t)(nf >= 1024 && nf <= 4096 ? 5 : 3) * nf * nf * sizeof(float2);
    // wavelengths resident at once: the caller's bound, else what fits in 70 % of the free
    // memory next to a generous allowance for the Lyot plans' own buffers
    int res = d->max_resident > 0 ? d->max_resident : d->batch;
    if (d->max_resident == 0) {
        size_t free_b = 0, total_b = 0;
        cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) return coro::cuda_fail(e, "coro_wfc_plan_create: cudaMemGetInfo");
        const size_t per = item_bytes + (size_t)32 * d->npix * d->npix * sizeof(float2);
        const size_t fit = (size_t)(0.7 * (double)free_b) / per;
        res = (int)std::max<size_t>(1, std::min<size_t>((size_t)d->batch, fit));
    }
    p->resident = std::min(res, d->batch);
    const int R = p->resident;
    coro_status st = CORO_OK;
    const size_t fbytes = (size_t)R * nf * nf * sizeof(float2), mbytes = (size_t)nf * nf * sizeof(float);
    p->e1 = (float2*)p->alloc(fbytes, &st);
    p->w = p->e1 ? (float2*)p->alloc(fbytes, &st) : nullptr;
    p->g = p->w ? (float2*)p->alloc(fbytes, &st) : nullptr;
    p->opd1 = p->g ? (float*)p->alloc(mbytes, &st) : nullptr;
    p->opd1n = p->opd1 ? (float*)p->alloc(mbytes, &st) : nullptr;
    p->opd2 = p->opd1n ? (float*)p->alloc(mbytes, &st) : nullptr;
    p->opd2n = p->opd2 ? (float*)p->alloc(mbytes, &st) : nullptr;
    p->zero_h = p->opd2n ? (float*)p->alloc((size_t)2 * d->n_act * d->n_act * sizeof(float), &st) : nullptr;
    p->part = p->zero_h ? (float*)p->alloc((size_t)2 * R * d->n_act * d->n_act * sizeof(float), &st) : nullptr;
    if (!p->part) return st;
    cudaError_t e = cudaMemsetAsync(p->zero_h, 0, (size_t)2 * d->n_act * d->n_act * sizeof(float), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return coro::cuda_fail(e, "coro_wfc_plan_create");
    for (int b0 = 0; b0 < d->batch; b0 += R) {
        p->chunks.emplace_back();
        Chunk& ch = p->chunks.back();
        ch.b0 = b0;
        ch.nb = std::min(R, d->batch - b0);
        if ((st = make_chunk(p.get(), ch)) != CORO_OK) return st;
    }
    *out = p.release();
    return CORO_OK;
}

extern "C" coro_status coro_wfc_plan_resident(coro_plan plan, int* resident, int* chunks) {
    coro::clear_error();
    if (!plan || plan->kind() != 3) { coro::set_error("coro_wfc_plan_resident: not a wavefront-control plan"); return CORO_EINVAL; }
    auto* p = static_cast<WfcPlan*>(plan);
    if (resident) *resident = p->resident;
    if (chunks) *chunks = (int)p->chunks.size();
    return CORO_OK;
}

extern "C" coro_status coro_wfc_plan_peak(coro_plan plan, double* peak_out) {
    coro::clear_error();
    if (!plan || plan->kind() != 3) { coro::set_error("coro_wfc_plan_peak: not a wavefront-control plan"); return CORO_EINVAL; }
    auto* p = static_cast<WfcPlan*>(plan);
    coro::DeviceGuard gd(p->device);
    if (p->peak.empty()) {
        coro_status st = dm_maps(p, p->zero_h);
        if (st != CORO_OK) return st;
        std::vector<double> pk(p->d.batch, 0.0);
        for (Chunk& ch : p->chunks) {
            if ((st = coro_fresnel_plan_execute(ch.fwd, p->w, nullptr)) != CORO_OK) return st;
            if ((st = coro_lyot_plan_peak(ch.lyot, window(p, p->w), pk.data() + ch.b0)) != CORO_OK) return st;
        }
        p->peak = pk;
    }
    if (peak_out)
        for (int b = 0; b < p->d.batch; ++b) peak_out[b] = p->peak[b];
    return CORO_OK;
}

extern "C" coro_status coro_wfc_plan_evaluate(coro_plan plan, const float* heights, double* loss, double* per_item,
                                              float* grad) {
    coro::clear_error();
    if (!plan || plan->kind() != 3) { coro::set_error("coro_wfc_plan_evaluate: not a wavefront-control plan"); return CORO_EINVAL; }
    if (!heights) { coro::set_error("coro_wfc_plan_evaluate: heights is NULL"); return CORO_EINVAL; }
    auto* p = static_cast<WfcPlan*>(plan);
    coro::DeviceGuard gd(p->device);
    coro_status st;
    if (p->peak.empty() && (st = coro_wfc_plan_peak(plan, nullptr)) != CORO_OK) return st;
    const coro_wfc_desc& d = p->d;
    coro_ctx c = p->ctx;
    const int B = d.batch, nf = d.n_fresnel, na = d.n_act;
    if ((st = dm_maps(p, heights)) != CORO_OK) return st;
    std::vector<double> dh(B, 0.0);
    const size_t npx = (size_t)nf * nf;
    const double dx = d.diam_m / d.npix;
    const int per = na * na;
    for (size_t k = 0; k < p->chunks.size() && st == CORO_OK; ++k) {
        Chunk& ch = p->chunks[k];
        const int nb = ch.nb;
        // E1 checkpoint and E3 (in w)
        if ((st = coro_fresnel_plan_execute(ch.fwd, p->w, nullptr)) != CORO_OK) break;
        if (!grad) {
            st = coro_lyot_plan_execute(ch.lyot, window(p, p->w), p->peak.data() + ch.b0, nullptr, nullptr,
                                        dh.data() + ch.b0);
            continue;
        }
        cudaError_t e = cudaMemsetAsync(p->g, 0, (size_t)nb * npx * sizeof(float2), c->stream);   // pad(): zero outside the window
        if (e != cudaSuccess) return coro::cuda_fail(e, "wfc: memset");
        st = coro_lyot_plan_gradient(ch.lyot, window(p, p->w), p->peak.data() + ch.b0, dh.data() + ch.b0,
                                     window(p, p->g), nf, (long long)nf * nf);
        // G3 -> G0 (in g), the row passes writing the per-wavelength dL/dh density maps into w
        if (st == CORO_OK) st = coro_fresnel_plan_execute(ch.adj, p->g, nullptr);
        const float* dphi2 = reinterpret_cast<const float*>(p->w);
        if (st == CORO_OK)
            st = coro_dm_correlate(c, dphi2 + (size_t)nb * npx, nb, nf, dx, na, d.act_pitch_m, d.act_fwhm_m, 1.0, p->part);
        if (st == CORO_OK)
            st = coro_dm_correlate(c, dphi2, nb, nf, dx, na, d.act_pitch_m, d.act_fwhm_m, 1.0, p->part + (size_t)nb * per);
        if (st == CORO_OK) {
            sum_items_kernel<<<dim3((per + 255) / 256, 2), 256, 0, c->stream>>>(p->part, nb, per, k > 0, grad);
            e = cudaGetLastError();
            if (e != cudaSuccess) st = coro::cuda_fail(e, "sum_items_kernel");
        }
    }
    if (st == CORO_OK && grad) {
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = coro::cuda_fail(e, "coro_wfc_plan_evaluate");
    }
    if (st != CORO_OK) return st;
    double total = 0.0;
    for (int b = 0; b < B; ++b) {
        total += dh[b];
        if (per_item) per_item[b] = dh[b];
    }
    if (loss) *loss = total;
    return CORO_OK;
}
