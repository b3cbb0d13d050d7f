// lyot.cu -- batched semi-analytic Lyot coronagraph (Sec. 1.1: the Soummer et al. method
// built from matrix Fourier transforms of modest arrays around a small focal-plane mask).
//
// Per item (wavelength x probe state), with E_A the pupil field:
//   G1  Z1 = (E_A . A_occ^T)^T                       split, transposed
//   G2  X_B = spot . s_occ (Z1 . A_occ^T)^T           = spot . MFT(E_A)       (pupil -> occulter)
//   G3  Z3 = (X_B . B^T)^T
//   G4  E_D = Lyot . (E_A - s_occ (Z3 . B^T)^T)       Babinet, in place over E_A's planes
//   G5  Z5 = (E_D . A_det^T)^T
//   G6  I = |s_det (Z5 . A_det^T)^T|^2 / peak,   S = sum over the dark-hole annulus of I
// Every G is one launch of the split-precision tensor-core GEMM (tc_gemm.cu) over the whole
// batch; the spot, the Babinet subtraction, the Lyot stop, the intensity and the dark-hole sum
// are epilogues, so the only extra pass is the split of E_A.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <map>
#include <memory>
#include <vector>

#include "capi_common.h"
#include "tc_gemm.cuh"
#include "tcx_gemm.cuh"

using namespace coro;

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct LyotPlan : coro_plan_s {
    coro_ctx ctx = nullptr;
    bool bf16 = false;
    bool ext = false;                  // CORO_MFT_EXT: sliced BF16 operands (tcx_gemm.cu)
    int tile_n = TCX_TILE_N_WIDE;      // CORO_MFT_EXT output tile width (complex columns)
    int batch = 0, n = 0, m_det = 0, m_occ_max = 0;
    double npix = 0;
    std::vector<coro_lyot_item> items;
    std::vector<Buf> bufs;
    TcOperand XA{}, Z1{}, XB{}, Z3{}, Z5{}, W1{}, W2{}, W3{};
    CUtensorMap mXA, mZ1, mXB, mZ3, mZ5, mW1, mW2, mW3;
    TcItem* dev_items = nullptr;       // [9][batch]: G1-G6, then the adjoint's H1, H2, G4 without stop
    std::vector<TcItem> host_items;    // [9][batch]
    int pupil_ld = 0;                  // layout of the pupil argument (elements)
    long long pupil_bstride = 0;
    std::vector<std::pair<double, int>> det_bases;   // (du_det, basis index)
    // adjoint resources, made on the first gradient call
    bool grad_ready = false;
    TcOperand XS{}, Z4{}, W4{};
    CUtensorMap mXS, mZ4, mW4;
    float2* seed = nullptr;            // [batch][m_det][m_det] dS/dconj(E_det)
    int* keep_lyot = nullptr;          // [batch] Lyot-stop radius^2 (pupil pixels)
    double* dh = nullptr;              // [batch]
    float* peak = nullptr;             // [batch]
    double* peak64 = nullptr;          // [batch] (CORO_MFT_EXT)
    int device = 0;                    // kept so that destruction never touches the context
    int kind() const override { return 2; }
    int launches() const override { return 7; }
    int timing_units() const override { return 6; }     // the stages of execute_range
    ~LyotPlan() override {
        DeviceGuard g(device);
        cudaDeviceSynchronize();
        timing.release();
        graph.reset();
        for (auto& b : bufs) cudaFree(b.p);
    }
    void* alloc(size_t bytes, coro_status* st) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) { *st = cuda_fail(e, "coro_lyot_plan_create: cudaMalloc"); return nullptr; }
        bufs.push_back({p, bytes});
        e = cudaMemsetAsync(p, 0, bytes, ctx->stream);   // padding of every operand stays zero
        if (e != cudaSuccess) { *st = cuda_fail(e, "cudaMemsetAsync"); return nullptr; }
        return p;
    }
    // An operand of the plan's GEMM family; basis = a W-type operand (the MFT bases).
    bool make(TcOperand& op, int nb, int rows, int cols, coro_status* st, bool basis = false) {
        op.batch = nb;
        op.rows = rows;
        op.cols = cols;
        if (ext) {
            op.ld = tcx_ld(cols);
            op.base = alloc((size_t)(basis ? TCX_W_PLANES : TCX_X_PLANES) * nb * rows * op.ld * 2, st);
        } else {
            op.ld = tc_ld(cols, bf16);
            op.base = alloc((size_t)4 * nb * rows * op.ld * tc_elem_size(bf16), st);
        }
        return op.base != nullptr;
    }
    cudaError_t map(const TcOperand& op, bool basis, CUtensorMap* m) const {
        if (ext) return basis ? tcx_make_w_map(op, m, tile_n) : tcx_make_x_map(op, m);
        return tc_make_operand_map(op, bf16, m);
    }
    cudaError_t basis(double c, int sign, const TcOperand& dst, int item, int rows, int cols) const {
        return ext ? tcx_basis_one(c, sign, dst, item, rows, cols, ctx->stream)
                   : tc_basis_one(bf16, c, sign, dst, item, rows, cols, ctx->stream);
    }
    cudaError_t split(const float2* src, long long bstride, int ld, const TcOperand& dst, const int* keep = nullptr) const {
        return ext ? tcx_split(src, bstride, ld, dst, ctx->stream, keep)
                   : tc_split(bf16, src, bstride, ld, dst, ctx->stream, keep);
    }
    cudaError_t launch(int epi, const CUtensorMap& mx, const CUtensorMap& mw, int mm, int nn, int kk, const TcArgs& a) const {
        return ext ? tcx_launch(epi, mx, mw, mm, nn, batch, a, ctx->stream, tile_n)
                   : tc_launch(bf16, epi, mx, mw, mm, nn, kk, batch, a, ctx->stream);
    }
    // elements per item of an X-type operand (for the epilogues' batch strides)
    long long xstride(const TcOperand& op) const { return (long long)(ext ? TCX_X_PLANES : 4) * op.rows * op.ld; }
};

int clamp_thr(long long v) { return v > 0x3fffffffLL ? 0x3fffffff : (int)v; }

coro_status tune_tile(LyotPlan* p);

}  // namespace

extern "C" coro_status coro_lyot_plan_create(coro_ctx ctx, const coro_lyot_desc* d, coro_plan* out) {
    clear_error();
    if (!ctx || !d || !out || !d->items) { set_error("coro_lyot_plan_create: NULL argument"); return CORO_EINVAL; }
    *out = nullptr;
    if (d->precision != CORO_MFT_3XTF32 && d->precision != CORO_MFT_3XBF16 && d->precision != CORO_MFT_EXT &&
        d->precision != CORO_MFT_FP64) {
        set_error("coro_lyot_plan_create: precision must be CORO_MFT_3XTF32, CORO_MFT_3XBF16, CORO_MFT_EXT or CORO_MFT_FP64");
        return CORO_EINVAL;
    }
    if (d->batch < 1 || d->batch > 65535) { set_error("coro_lyot_plan_create: batch %d", d->batch); return CORO_ESIZE; }
    if (d->n < 16 || d->n > 8192 || d->m_det < 16 || d->m_det > 8192) {
        set_error("coro_lyot_plan_create: n = %d, m_det = %d outside [16, 8192]", d->n, d->m_det);
        return CORO_ESIZE;
    }
    if (!(d->npix > 0) || !(d->lyot_frac > 0)) { set_error("coro_lyot_plan_create: npix and lyot_frac must be > 0"); return CORO_EINVAL; }
    int m_occ_max = 0;
    for (int b = 0; b < d->batch; ++b) {
        const coro_lyot_item& it = d->items[b];
        if (it.m_occ < 16 || it.m_occ > 8192) { set_error("item %d: m_occ = %d outside [16, 8192]", b, it.m_occ); return CORO_ESIZE; }
        if (!(it.du_occ > 0) || !(it.du_det > 0) || !(it.spot_radius >= 0) || !(it.dh_in >= 0) || !(it.dh_out >= it.dh_in)) {
            set_error("item %d: need du_occ, du_det > 0, spot_radius >= 0, 0 <= dh_in <= dh_out", b);
            return CORO_EINVAL;
        }
        if (it.m_occ > m_occ_max) m_occ_max = it.m_occ;
    }
    if (d->precision == CORO_MFT_FP64) return lyot64_create(ctx, d, out);
    DeviceGuard g(ctx->device);
    auto p = std::unique_ptr<LyotPlan>(new (std::nothrow) LyotPlan);
    if (!p) { set_error("out of host memory"); return CORO_ENOMEM; }
    p->ctx = ctx;
    p->device = ctx->device;
    p->bf16 = d->precision == CORO_MFT_3XBF16;
    p->ext = d->precision == CORO_MFT_EXT;
    p->batch = d->batch;
    p->n = d->n;
    p->npix = d->npix;
    p->m_det = d->m_det;
    p->m_occ_max = m_occ_max;
    p->items.assign(d->items, d->items + d->batch);
    const int B = d->batch, n = d->n, md = d->m_det;

    // distinct bases: occulter (m_occ, du_occ) and detector du_det
    std::map<std::pair<int, double>, int> occ_id;
    std::map<double, int> det_id;
    std::vector<int> oi(B), di(B);
    for (int b = 0; b < B; ++b) {
        auto ko = std::make_pair(d->items[b].m_occ, d->items[b].du_occ);
        if (!occ_id.count(ko)) { const int id = (int)occ_id.size(); occ_id[ko] = id; }
        if (!det_id.count(d->items[b].du_det)) { const int id = (int)det_id.size(); det_id[d->items[b].du_det] = id; }
        oi[b] = occ_id[ko];
        di[b] = det_id[d->items[b].du_det];
    }
    coro_status st = CORO_OK;
    const int no = (int)occ_id.size(), nd = (int)det_id.size();
    if (!p->make(p->XA, B, n, n, &st) || !p->make(p->Z1, B, m_occ_max, n, &st) || !p->make(p->XB, B, m_occ_max, m_occ_max, &st) ||
        !p->make(p->Z3, B, n, m_occ_max, &st) || !p->make(p->Z5, B, md, n, &st) || !p->make(p->W1, no, m_occ_max, n, &st, true) ||
        !p->make(p->W2, no, n, m_occ_max, &st, true) || !p->make(p->W3, nd, md, n, &st, true))
        return st;
    cudaError_t e = cudaSuccess;
    // A_occ[u][j] = exp(-2 pi i u' j' du/npix), B^T[j][u] = exp(+2 pi i j' u' du/npix), A_det likewise
    for (auto& kv : occ_id) {
        const double c = kv.first.second / d->npix;
        const int m = kv.first.first;
        if (e == cudaSuccess) e = p->basis(c, -1, p->W1, kv.second, m, n);
        if (e == cudaSuccess) e = p->basis(c, +1, p->W2, kv.second, n, m);
    }
    for (auto& kv : det_id)
        if (e == cudaSuccess) e = p->basis(kv.first / d->npix, -1, p->W3, kv.second, md, n);
    TcOperand* ops[8] = {&p->XA, &p->Z1, &p->XB, &p->Z3, &p->Z5, &p->W1, &p->W2, &p->W3};
    CUtensorMap* maps[8] = {&p->mXA, &p->mZ1, &p->mXB, &p->mZ3, &p->mZ5, &p->mW1, &p->mW2, &p->mW3};
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = p->map(*ops[i], i >= 5, maps[i]);
    if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_create: bases / tensor maps");

    // per-GEMM item tables
    const double pupil_pitch = 1.0 / d->npix;            // pupil coordinates in units of D
    const int lyot_thr = clamp_thr(disk_threshold(0.5 * d->lyot_frac, pupil_pitch, false));
    const int all = 0x7fffffff;
    p->host_items.resize((size_t)9 * B);
    p->pupil_ld = n;
    p->pupil_bstride = (long long)n * n;
    for (auto& kv : det_id) p->det_bases.push_back({kv.first, kv.second});
    std::vector<int> keep(B, lyot_thr);
    for (int b = 0; b < B; ++b) {
        const coro_lyot_item& it = d->items[b];
        const int mo = it.m_occ;
        const float s_occ = (float)(it.du_occ / d->npix), s_det = (float)(it.du_det / d->npix);
        const int spot = clamp_thr(disk_threshold(it.spot_radius, it.du_occ, false));
        const int dh_lo = clamp_thr(disk_threshold(it.dh_in, it.du_det, true) + 1);
        const int dh_hi = clamp_thr(disk_threshold(it.dh_out, it.du_det, false));
        TcItem* h = p->host_items.data();
        h[0 * B + b] = TcItem{n, mo, n, b, oi[b], 0, all, 1.0f, 1.0f};
        h[1 * B + b] = TcItem{mo, mo, n, b, oi[b], 0, spot, s_occ, 1.0f};
        h[2 * B + b] = TcItem{mo, n, mo, b, oi[b], 0, all, 1.0f, 1.0f};
        h[3 * B + b] = TcItem{n, n, mo, b, oi[b], 0, lyot_thr, s_occ, 1.0f};
        h[4 * B + b] = TcItem{n, md, n, b, di[b], 0, all, 1.0f, 1.0f};
        h[5 * B + b] = TcItem{md, md, n, b, di[b], dh_lo, dh_hi, s_det, 1.0f};
        // adjoint: detector IMFT (two GEMMs, Lyot stop on the second), Babinet block without stop
        h[6 * B + b] = TcItem{md, n, md, b, di[b], 0, all, 1.0f, 1.0f};
        h[7 * B + b] = TcItem{n, n, md, b, di[b], 0, lyot_thr, s_det, 1.0f};
        h[8 * B + b] = TcItem{n, n, mo, b, oi[b], 0, all, s_occ, 1.0f};
        for (int g : {1, 3, 8}) h[g * B + b].scale64 = it.du_occ / d->npix;
        for (int g : {5, 7}) h[g * B + b].scale64 = it.du_det / d->npix;
        // known zeros of the X operands (tc_gemm skips the K slices and tiles they cover):
        // X_B is the spot disk; Z3's columns are X_B's rows, so a band of the spot's width;
        // E_D is the Lyot-stop disk; Z5's columns are E_D's rows, a band of the stop's width
        h[2 * B + b].kr2 = spot;
        h[2 * B + b].kdy = 1;
        h[3 * B + b].kr2 = spot;
        h[3 * B + b].kdy = 0;
        h[4 * B + b].kr2 = lyot_thr;
        h[4 * B + b].kdy = 1;
        h[5 * B + b].kr2 = lyot_thr;
        h[5 * B + b].kdy = 0;
        // adjoint: the seed is zero outside the dark-hole's outer circle, Z4 a band of its
        // width; the stop-less Babinet block reads Z3 as G4 does
        h[6 * B + b].kr2 = dh_hi;
        h[6 * B + b].kdy = 1;
        h[7 * B + b].kr2 = dh_hi;
        h[7 * B + b].kdy = 0;
        h[8 * B + b].kr2 = spot;
        h[8 * B + b].kdy = 0;
    }
    p->dev_items = (TcItem*)p->alloc(p->host_items.size() * sizeof(TcItem), &st);
    p->keep_lyot = p->dev_items ? (int*)p->alloc(B * sizeof(int), &st) : nullptr;
    p->dh = p->keep_lyot ? (double*)p->alloc(B * sizeof(double), &st) : nullptr;
    p->peak = p->dh ? (float*)p->alloc(B * sizeof(float), &st) : nullptr;
    p->peak64 = p->peak ? (double*)p->alloc(B * sizeof(double), &st) : nullptr;
    if (!p->peak64) return st;
    e = cudaMemcpyAsync(p->dev_items, p->host_items.data(), p->host_items.size() * sizeof(TcItem), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->keep_lyot, keep.data(), B * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_create");
    if (p->ext && !(std::getenv("CORO_AUTOTUNE") && std::getenv("CORO_AUTOTUNE")[0] == '0')) {
        const coro_status ts = tune_tile(p.get());
        if (ts != CORO_OK) return ts;
    }
    *out = p.release();
    return CORO_OK;
}

namespace {

// The G6 item table with the intensity normalisation 1/peak (peak NULL: 1), stream-ordered.
cudaError_t upload_det_items(LyotPlan* p, const double* peak_host) {
    const int B = p->batch;
    cudaStream_t s = p->ctx->stream;
    if (peak_host) {
        std::vector<TcItem> g6(p->host_items.begin() + 5 * B, p->host_items.begin() + 6 * B);
        for (int b = 0; b < B; ++b) {
            g6[b].inv_peak = (float)(1.0 / peak_host[b]);
            g6[b].inv_peak64 = 1.0 / peak_host[b];
        }
        return cudaMemcpyAsync(p->dev_items + 5 * B, g6.data(), B * sizeof(TcItem), cudaMemcpyHostToDevice, s);
    }
    return cudaMemcpyAsync(p->dev_items + 5 * B, p->host_items.data() + 5 * B, B * sizeof(TcItem), cudaMemcpyHostToDevice, s);
}

// G5 + G6 on the operand already in XA planes; intensity epilogue (seed: write dS/dconj(E_det)).
// The G6 items must have been uploaded (upload_det_items) before.
cudaError_t detector_gemms(LyotPlan* p, float* intensity, void* field, bool track_peak, float2* seed = nullptr) {
    const int B = p->batch, n = p->n, md = p->m_det;
    cudaStream_t s = p->ctx->stream;
    TcArgs a{};
    a.err = p->ctx->err;
    a.items = p->dev_items + 4 * B;
    a.dst = p->Z5.base;
    a.dst_bstride = p->xstride(p->Z5);
    a.dst_rows = p->Z5.rows;
    a.dst_ld = p->Z5.ld;
    cudaError_t e = p->launch(TC_EPI_SPLITT, p->mXA, p->mW3, n, md, n, a);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p->dh, 0, B * sizeof(double), s);
    if (e == cudaSuccess && track_peak) e = cudaMemsetAsync(p->peak, 0, B * sizeof(float), s);
    if (e == cudaSuccess && track_peak) e = cudaMemsetAsync(p->peak64, 0, B * sizeof(double), s);
    if (e != cudaSuccess) return e;
    TcArgs b6{};
    b6.err = p->ctx->err;
    b6.items = p->dev_items + 5 * B;
    b6.dst = intensity;
    b6.dst_bstride = (long long)md * md;
    b6.dst_rows = md;
    b6.dst_ld = md;
    b6.c64 = seed ? seed : (float2*)field;
    b6.c64_seed = seed ? 1 : 0;
    b6.c64_bstride = (long long)md * md;
    b6.c64_ld = md;
    b6.dh_acc = p->dh;
    b6.peak = track_peak ? p->peak : nullptr;
    b6.peak64 = track_peak ? p->peak64 : nullptr;
    return p->launch(TC_EPI_INTENSITY, p->mZ5, p->mW3, md, md, n, b6);
}

}  // namespace

namespace {

// Stages 0 (split of the pupil), 1-4 (G1-G4), 5 (G5 + G6 with the intensity epilogue; its
// item table must be current, see upload_det_items).
// ev (optional, 7 events): recorded before stage 0 and after each of stages 0-5 (all six run).
cudaError_t run_stages(LyotPlan* p, const void* pupil, float* intensity, void* field, int first, int last,
                       const cudaEvent_t* ev = nullptr) {
    const int B = p->batch, n = p->n, mo = p->m_occ_max;
    cudaStream_t s = p->ctx->stream;
    cudaError_t e = cudaSuccess;
    auto mark = [&](int i) {
        if (ev && e == cudaSuccess) e = record_timing_event(ev[i], s);
    };
    mark(0);
    auto gemm = [&](int gi, int epi, const CUtensorMap& mx, const CUtensorMap& mw, const TcOperand& dst, int mm, int nn, int kk) {
        if (e != cudaSuccess || gi + 1 < first || gi + 1 > last) return;
        TcArgs a{};
        a.err = p->ctx->err;
        a.items = p->dev_items + gi * B;
        a.dst = dst.base;
        a.dst_bstride = p->xstride(dst);
        a.dst_rows = dst.rows;
        a.dst_ld = dst.ld;
        if (epi == TC_EPI_BABINET) {                 // E_A straight from the complex64 pupil
            a.src64 = (const float2*)pupil;
            a.src64_bstride = p->pupil_bstride;
            a.src64_ld = p->pupil_ld;
        }
        e = p->launch(epi, mx, mw, mm, nn, kk, a);
        mark(gi + 2);
    };
    if (first <= 0 && last >= 0) e = p->split((const float2*)pupil, p->pupil_bstride, p->pupil_ld, p->XA);
    mark(1);
    gemm(0, TC_EPI_SPLITT, p->mXA, p->mW1, p->Z1, n, mo, n);     // G1
    gemm(1, TC_EPI_SPLITT, p->mZ1, p->mW1, p->XB, mo, mo, n);    // G2 (x spot)
    gemm(2, TC_EPI_SPLITT, p->mXB, p->mW2, p->Z3, mo, n, mo);    // G3
    gemm(3, TC_EPI_BABINET, p->mZ3, p->mW2, p->XA, n, n, mo);    // G4 (Babinet, x Lyot)
    if (e == cudaSuccess && first <= 5 && last >= 5) e = detector_gemms(p, intensity, field, false);
    mark(6);
    return e;
}

}  // namespace

namespace {

// Re-encode the basis maps for the plan's tile width (their boxes have tile_n rows).
cudaError_t remap_bases(LyotPlan* p) {
    cudaError_t e = p->map(p->W1, true, &p->mW1);
    if (e == cudaSuccess) e = p->map(p->W2, true, &p->mW2);
    if (e == cudaSuccess) e = p->map(p->W3, true, &p->mW3);
    if (e == cudaSuccess && p->grad_ready) e = p->map(p->W4, true, &p->mW4);
    return e;
}

// Plan-time choice of the extended GEMM's tile width: the GEMM stages (1-5) of one execute on
// the plan's own (zero) operands, timed with events for each width; the faster is kept. The
// GEMMs' cost depends on the geometry only (tile counts, support-aware K ranges), not on the
// values. Results do not depend on the choice beyond FP32 rounding order.
coro_status tune_tile(LyotPlan* p) {
    cudaStream_t s = p->ctx->stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 1e30f;
    int best_tile = TCX_TILE_N_WIDE;
    for (int tile : {TCX_TILE_N_WIDE, TCX_TILE_N_NARROW}) {
        if (e != cudaSuccess) break;
        p->tile_n = tile;
        e = remap_bases(p);
        if (e == cudaSuccess) e = run_stages(p, nullptr, nullptr, nullptr, 1, 5);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(a, s);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = run_stages(p, nullptr, nullptr, nullptr, 1, 5);
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && ms < best) { best = ms; best_tile = tile; }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    p->tile_n = best_tile;
    if (e == cudaSuccess) e = remap_bases(p);
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "coro_lyot_plan_create: GEMM tile tuning");
}

}  // namespace

extern "C" coro_status coro_lyot_plan_gemm_tile(coro_plan plan, int* tile_m, int* tile_n) {
    clear_error();
    if (!plan || (plan->kind() != 2 && plan->kind() != 4)) { set_error("coro_lyot_plan_gemm_tile: not a Lyot plan"); return CORO_EINVAL; }
    int m = 0, n = 0;                                    // FP64 plans: CUDA-core GEMMs, no tensor tile
    if (plan->kind() == 2) {
        auto* p = static_cast<LyotPlan*>(plan);
        m = 128;
        n = p->ext ? p->tile_n : 128;
    }
    if (tile_m) *tile_m = m;
    if (tile_n) *tile_n = n;
    return CORO_OK;
}

extern "C" coro_status coro_lyot_plan_set_gemm_tile(coro_plan plan, int tile_n) {
    clear_error();
    if (!plan || plan->kind() != 2) { set_error("coro_lyot_plan_set_gemm_tile: not a tensor-core Lyot plan"); return CORO_EINVAL; }
    auto* p = static_cast<LyotPlan*>(plan);
    if (!p->ext) {
        if (tile_n == 128) return CORO_OK;
        set_error("coro_lyot_plan_set_gemm_tile: the 3xTF32 / 3xBF16 GEMM has one tile width, 128");
        return CORO_EINVAL;
    }
    if (tile_n != TCX_TILE_N_WIDE && tile_n != TCX_TILE_N_NARROW) {
        set_error("coro_lyot_plan_set_gemm_tile: tile width %d (CORO_MFT_EXT offers 64 and 32)", tile_n);
        return CORO_EINVAL;
    }
    DeviceGuard g(p->ctx->device);
    p->graph.reset();                                    // captured launches used the old maps
    p->tile_n = tile_n;
    const cudaError_t e = remap_bases(p);
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "coro_lyot_plan_set_gemm_tile");
}

namespace {
// Items of a split-precision (kind 2) or FP64 (kind 4) Lyot plan.
int lyot_batch(coro_plan plan) { return plan->kind() == 4 ? coro::lyot64_batch(plan) : static_cast<LyotPlan*>(plan)->batch; }
}  // namespace

extern "C" coro_status coro_lyot_plan_execute_range(coro_plan plan, const void* pupil, const double* peak,
                                                    float* intensity, void* field, int first, int count) {
    clear_error();
    if (plan && plan->kind() == 4) { set_error("coro_lyot_plan_execute_range: not available at CORO_MFT_FP64"); return CORO_ENOTIMPL; }
    if (!plan || plan->kind() != 2) { set_error("coro_lyot_plan_execute_range: not a Lyot plan"); return CORO_EINVAL; }
    if (!pupil || first < 0 || count < 0 || first + count > 6) {
        set_error("coro_lyot_plan_execute_range: pupil NULL or stage range [%d, %d) outside [0, 6)", first, first + count);
        return CORO_EINVAL;
    }
    auto* p = static_cast<LyotPlan*>(plan);
    if (peak)
        for (int b = 0; b < p->batch; ++b)
            if (!(peak[b] > 0)) { set_error("coro_lyot_plan_execute_range: peak[%d] must be > 0", b); return CORO_EINVAL; }
    DeviceGuard g(p->ctx->device);
    const int last = first + count - 1;
    cudaError_t e = (first <= 5 && last >= 5) ? upload_det_items(p, peak) : cudaSuccess;
    if (e == cudaSuccess) e = run_stages(p, pupil, intensity, field, first, last);
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "coro_lyot_plan_execute_range");
}

extern "C" coro_status coro_lyot_plan_execute(coro_plan plan, const void* pupil, const double* peak, float* intensity,
                                              void* field, double* dh) {
    clear_error();
    if (!plan || (plan->kind() != 2 && plan->kind() != 4)) { set_error("coro_lyot_plan_execute: not a Lyot plan"); return CORO_EINVAL; }
    if (!pupil) { set_error("coro_lyot_plan_execute: pupil is NULL"); return CORO_EINVAL; }
    const int B = lyot_batch(plan);
    if (peak)
        for (int b = 0; b < B; ++b)
            if (!(peak[b] > 0)) { set_error("coro_lyot_plan_execute: peak[%d] must be > 0", b); return CORO_EINVAL; }
    if (plan->kind() == 4) return lyot64_execute(plan, pupil, peak, intensity, field, dh);
    auto* p = static_cast<LyotPlan*>(plan);
    DeviceGuard g(p->ctx->device);
    cudaStream_t s = p->ctx->stream;
    cudaError_t e = upload_det_items(p, peak);           // outside any graph: plain stream copy
    if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_execute");
    const coro_status st = run_graphed(p->ctx, p->graph, {pupil, intensity, field, (const void*)1}, [&]() -> coro_status {
        const cudaError_t e1 = run_stages(p, pupil, intensity, field, 0, 5, p->timing.set(0));
        return e1 == cudaSuccess ? CORO_OK : cuda_fail(e1, "coro_lyot_plan_execute");
    });
    if (st != CORO_OK) return st;
    s = p->ctx->stream;
    if (e == cudaSuccess && dh) {
        e = cudaMemcpyAsync(dh, p->dh, B * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_execute");
    return CORO_OK;
}

extern "C" coro_status coro_lyot_plan_execute_n(coro_plan plan, const void* pupil, const double* peak, float* intensity,
                                                void* field, int times) {
    clear_error();
    if (!plan || (plan->kind() != 2 && plan->kind() != 4)) { set_error("coro_lyot_plan_execute_n: not a Lyot plan"); return CORO_EINVAL; }
    if (!pupil || times < 1) { set_error("coro_lyot_plan_execute_n: pupil NULL or times < 1"); return CORO_EINVAL; }
    if (plan->kind() == 4) {
        if (peak)
            for (int b = 0; b < lyot_batch(plan); ++b)
                if (!(peak[b] > 0)) { set_error("coro_lyot_plan_execute_n: peak[%d] must be > 0", b); return CORO_EINVAL; }
        coro_status st = CORO_OK;
        for (int k = 0; k < times && st == CORO_OK; ++k) st = lyot64_execute(plan, pupil, peak, intensity, field, nullptr);
        return st;
    }
    auto* p = static_cast<LyotPlan*>(plan);
    if (peak)
        for (int b = 0; b < p->batch; ++b)
            if (!(peak[b] > 0)) { set_error("coro_lyot_plan_execute_n: peak[%d] must be > 0", b); return CORO_EINVAL; }
    DeviceGuard g(p->ctx->device);
    cudaError_t e = upload_det_items(p, peak);
    if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_execute_n");
    return run_graphed(p->ctx, p->graph, {pupil, intensity, field, (const void*)(intptr_t)times}, [&]() -> coro_status {
        cudaError_t e1 = cudaSuccess;
        for (int k = 0; k < times && e1 == cudaSuccess; ++k)
            e1 = run_stages(p, pupil, intensity, field, 0, 5, p->timing.set(k));
        return e1 == cudaSuccess ? CORO_OK : cuda_fail(e1, "coro_lyot_plan_execute_n");
    });
}

extern "C" coro_status coro_lyot_plan_flops(coro_plan plan, double* useful, double* issued) {
    clear_error();
    if (plan && plan->kind() == 4) {                       // no tensor-core work
        if (useful) *useful = 0.0;
        if (issued) *issued = 0.0;
        return CORO_OK;
    }
    if (!plan || plan->kind() != 2) { set_error("coro_lyot_plan_flops: not a Lyot plan"); return CORO_EINVAL; }
    auto* p = static_cast<LyotPlan*>(plan);
    const int B = p->batch, n = p->n, md = p->m_det, mo = p->m_occ_max;
    const int epi[6] = {TC_EPI_SPLITT, TC_EPI_SPLITT, TC_EPI_SPLITT, TC_EPI_BABINET, TC_EPI_SPLITT, TC_EPI_INTENSITY};
    const int mm[6] = {n, mo, mo, n, n, md}, nn[6] = {mo, mo, n, n, md, md};
    double u = 0, is = 0;
    for (int g = 0; g < 6; ++g) {
        if (p->ext) tcx_count_flops(epi[g], p->host_items.data() + (size_t)g * B, B, mm[g], nn[g], &u, &is, p->tile_n);
        else tc_count_flops(p->bf16, epi[g], p->host_items.data() + (size_t)g * B, B, mm[g], nn[g], &u, &is);
    }
    if (useful) *useful = u;
    if (issued) *issued = is;
    return CORO_OK;
}

extern "C" coro_status coro_lyot_plan_peak(coro_plan plan, const void* pupil, double* peak_out) {
    clear_error();
    if (plan && plan->kind() == 4 && pupil && peak_out) return lyot64_peak(plan, pupil, peak_out);
    if (!plan || plan->kind() != 2 || !pupil || !peak_out) { set_error("coro_lyot_plan_peak: bad argument"); return CORO_EINVAL; }
    auto* p = static_cast<LyotPlan*>(plan);
    const int B = p->batch, n = p->n;
    DeviceGuard g(p->ctx->device);
    cudaStream_t s = p->ctx->stream;
    // occulter removed: E_D = E_A . Lyot stop, then the detector MFT
    cudaError_t e = p->split((const float2*)pupil, p->pupil_bstride, p->pupil_ld, p->XA, p->keep_lyot);
    if (e == cudaSuccess) e = upload_det_items(p, nullptr);
    if (e == cudaSuccess) e = detector_gemms(p, nullptr, nullptr, true);
    std::vector<float> pk(B);
    std::vector<double> pk64(B);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pk.data(), p->peak, B * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pk64.data(), p->peak64, B * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_peak");
    for (int b = 0; b < B; ++b) peak_out[b] = p->ext ? pk64[b] : pk[b];
    return CORO_OK;
}

extern "C" coro_status coro_lyot_plan_set_pupil_layout(coro_plan plan, int ld, long long bstride) {
    clear_error();
    if (plan && plan->kind() == 4) {
        set_error("coro_lyot_plan_set_pupil_layout: CORO_MFT_FP64 plans take contiguous [batch][n][n] pupils");
        return CORO_ENOTIMPL;
    }
    if (!plan || plan->kind() != 2) { set_error("coro_lyot_plan_set_pupil_layout: not a Lyot plan"); return CORO_EINVAL; }
    auto* p = static_cast<LyotPlan*>(plan);
    if (ld < p->n || bstride < (long long)ld * (p->n - 1) + p->n) {
        set_error("coro_lyot_plan_set_pupil_layout: ld %d / bstride %lld too small for n = %d", ld, bstride, p->n);
        return CORO_EINVAL;
    }
    p->pupil_ld = ld;
    p->pupil_bstride = bstride;
    return CORO_OK;
}

namespace {

coro_status prepare_gradient(LyotPlan* p) {
    if (p->grad_ready) return CORO_OK;
    coro_status st = CORO_OK;
    const int B = p->batch, n = p->n, md = p->m_det;
    const int nd = (int)p->det_bases.size();
    if (!p->make(p->XS, B, md, md, &st) || !p->make(p->Z4, B, n, md, &st) || !p->make(p->W4, nd, n, md, &st, true))
        return st;
    p->seed = (float2*)p->alloc((size_t)B * md * md * sizeof(float2), &st);
    if (!p->seed) return st;
    cudaError_t e = cudaSuccess;
    // W4[j][u] = exp(+2 pi i j' u' du_det / npix): the detector MFT's conjugate transpose
    for (auto& db : p->det_bases)
        if (e == cudaSuccess) e = p->basis(db.first / p->npix, +1, p->W4, db.second, n, md);
    if (e == cudaSuccess) e = p->map(p->XS, false, &p->mXS);
    if (e == cudaSuccess) e = p->map(p->Z4, false, &p->mZ4);
    if (e == cudaSuccess) e = p->map(p->W4, true, &p->mW4);
    if (e != cudaSuccess) return cuda_fail(e, "coro_lyot_plan_gradient: set-up");
    p->grad_ready = true;
    return CORO_OK;
}

}  // namespace

extern "C" coro_status coro_lyot_plan_gradient(coro_plan plan, const void* pupil, const double* peak, double* dh_out,
                                               void* grad, int grad_ld, long long grad_bstride) {
    clear_error();
    if (plan && plan->kind() == 4) { set_error("coro_lyot_plan_gradient: not available at CORO_MFT_FP64"); return CORO_ENOTIMPL; }
    if (!plan || plan->kind() != 2) { set_error("coro_lyot_plan_gradient: not a Lyot plan"); return CORO_EINVAL; }
    auto* p = static_cast<LyotPlan*>(plan);
    const int B = p->batch, n = p->n, md = p->m_det, mo = p->m_occ_max;
    if (!pupil || !peak || !grad) { set_error("coro_lyot_plan_gradient: pupil, peak and grad are required"); return CORO_EINVAL; }
    if (grad_ld < n || grad_bstride < (long long)grad_ld * (n - 1) + n) {
        set_error("coro_lyot_plan_gradient: grad_ld %d / grad_bstride %lld too small", grad_ld, grad_bstride);
        return CORO_EINVAL;
    }
    for (int b = 0; b < B; ++b)
        if (!(peak[b] > 0)) { set_error("coro_lyot_plan_gradient: peak[%d] must be > 0", b); return CORO_EINVAL; }
    DeviceGuard g(p->ctx->device);
    coro_status st = prepare_gradient(p);
    if (st != CORO_OK) return st;
    cudaStream_t s = p->ctx->stream;
    // forward (stages 0-4), then the detector MFT writing the seed mask . E_det / peak
    cudaError_t e = run_stages(p, pupil, nullptr, nullptr, 0, 4);
    if (e == cudaSuccess) e = upload_det_items(p, peak);
    if (e == cudaSuccess) e = detector_gemms(p, nullptr, nullptr, false, p->seed);
    if (e == cudaSuccess && dh_out) e = cudaMemcpyAsync(dh_out, p->dh, B * sizeof(double), cudaMemcpyDeviceToHost, s);
    // adjoint: G_D = IMFT_det(seed); G_C = Lyot . G_D; G_A = G_C - IMFT_occ(spot . MFT_occ(G_C))
    if (e == cudaSuccess) e = p->split(p->seed, (long long)md * md, md, p->XS);
    auto gemm = [&](int gi, int epi, const CUtensorMap& mx, const CUtensorMap& mw, const TcOperand& dst, int mm, int nn, int kk) {
        if (e != cudaSuccess) return;
        TcArgs a{};
        a.err = p->ctx->err;
        a.items = p->dev_items + gi * B;
        a.dst = dst.base;
        a.dst_bstride = p->xstride(dst);
        a.dst_rows = dst.rows;
        a.dst_ld = dst.ld;
        e = p->launch(epi, mx, mw, mm, nn, kk, a);
    };
    gemm(6, TC_EPI_SPLITT, p->mXS, p->mW4, p->Z4, md, n, md);    // H1
    gemm(7, TC_EPI_SPLITT, p->mZ4, p->mW4, p->XA, n, n, md);     // H2 (x Lyot) -> G_C in XA
    gemm(0, TC_EPI_SPLITT, p->mXA, p->mW1, p->Z1, n, mo, n);     // G1
    gemm(1, TC_EPI_SPLITT, p->mZ1, p->mW1, p->XB, mo, mo, n);    // G2 (x spot)
    gemm(2, TC_EPI_SPLITT, p->mXB, p->mW2, p->Z3, mo, n, mo);    // G3
    gemm(8, TC_EPI_BABINET, p->mZ3, p->mW2, p->XA, n, n, mo);    // G4, no stop -> G_A in XA
    if (e == cudaSuccess)
        e = p->ext ? tcx_merge(p->XA, (float2*)grad, grad_bstride, grad_ld, s)
                   : tc_merge(p->bf16, p->XA, (float2*)grad, grad_bstride, grad_ld, s);
    if (e == cudaSuccess && dh_out) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? CORO_OK : cuda_fail(e, "coro_lyot_plan_gradient");
}
