"""GPU parity: batched semi-analytic Lyot coronagraph (six tensor-core GEMMs with fused
spot / Babinet / Lyot-stop / intensity / dark-hole epilogues) against the FP64 oracle.

Every comparison is the product's own normalised intensity (its own peak) against the oracle's
own (the oracle's peak): nothing is rescaled.

Target: |I_gpu - I_oracle| <= 1e-11 inside the dark hole. On this workload (mean dark-hole
contrast 1.2e-6, 4.3e-5 at the inner edge) FP32-class arithmetic cannot deliver it: the same
chain with complex64 BLAS GEMMs (round-to-nearest FMA) lands at 3.3e-11, because GEMM errors
scale with the peak field while the dark-hole field is 1e-2..1e-3 of it, and the tensor cores'
truncating accumulators in 3xTF32 / 3xBF16 land near 5e-10. Those two precisions are held to
regression bars set from their measured errors (printed on every run). The extended-precision
plan (CORO_MFT_EXT: exact 8-bit BF16 slices, two-float accumulation, FP64 peak) is held to the
1e-11 target itself.
"""
import numpy as np
import pytest
import torch

from oracle import coronagraph, optics
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu

DH_TARGET = 1e-11
# regression bars of the FP32-class precisions (own peak against the oracle's own peak)
DH_TOL_SMALL = {coro.MFT_3XTF32: 5e-9, coro.MFT_3XBF16: 3e-8, coro.MFT_EXT: DH_TARGET}
DH_TOL_FULL = {coro.MFT_3XTF32: 2e-9, coro.MFT_3XBF16: 3e-9, coro.MFT_EXT: DH_TARGET}
PEAK_TOL = {coro.MFT_3XTF32: 1e-5, coro.MFT_3XBF16: 1e-5, coro.MFT_EXT: 1e-9}
PRECS = [coro.MFT_3XTF32, coro.MFT_3XBF16, coro.MFT_EXT]


@pytest.fixture(scope="module")
def ctx(lib):
    c = coro.Context(0)
    yield c
    c.synchronize()


def oracle_psf(e, n, npix, it, lyot_frac, m_det):
    p = coronagraph.LyotParams(n=n, npix=npix, m_occ=it["m_occ"], du_occ=it["du_occ"],
                               spot_radius=it["spot_radius"], lyot_frac=lyot_frac, m_det=m_det,
                               du_det=it["du_det"])
    peak = coronagraph.peak_intensity(e, p)
    i = coronagraph.intensity(coronagraph.lyot_fields(e, p)["det"], peak)
    return i, coronagraph.dark_hole_sum(i, it["du_det"], it["dh_in"], it["dh_out"]), peak


def zernike_pupil(n, npix, lam, seed, rms=5e-9):
    c = inputs.zernike_coefficients(seed, 4, 21, rms)
    opd = optics.zernike_opd(n, 1.0 / npix, 0.5, c, 4)
    return coronagraph.pupil_field(n, npix, lam, opd)


@pytest.mark.parametrize("prec", PRECS)
def test_lyot_small_uneven_batch(ctx, prec):
    n, npix, m_det, lyot = 128, 120, 96, 0.8
    items = [dict(m_occ=40, du_occ=0.25, spot_radius=3.0, du_det=0.5, dh_in=4.0, dh_out=16.0),
             dict(m_occ=37, du_occ=0.27, spot_radius=3.0, du_det=0.45, dh_in=4.0, dh_out=16.0),
             dict(m_occ=45, du_occ=0.22, spot_radius=3.5, du_det=0.55, dh_in=4.5, dh_out=18.0)]
    pupils = np.stack([zernike_pupil(n, npix, 550e-9, s, rms=20e-9) for s in range(3)]).astype(np.complex64)
    x = torch.from_numpy(pupils).cuda()
    plan = coro.LyotPlan(ctx, n=n, npix=npix, lyot_frac=lyot, m_det=m_det, items=items, precision=prec)
    peak = plan.peak(x)
    inten = torch.empty((3, m_det, m_det), dtype=torch.float32, device="cuda")
    dh = plan.execute(x, peak=peak, intensity=inten)
    got = inten.cpu().numpy()
    for b, it in enumerate(items):
        ref_i, ref_s, ref_peak = oracle_psf(pupils[b].astype(np.complex128), n, npix, it, lyot, m_det)
        mask = coronagraph.dark_hole_mask(m_det, it["du_det"], it["dh_in"], it["dh_out"]) > 0
        err = np.max(np.abs(got[b][mask] - ref_i[mask]))
        print(f"prec {prec} item {b}: peak rel {peak[b] / ref_peak - 1:.2e}, max |dI| in dark hole {err:.3e}, "
              f"S {dh[b]:.9e} vs {ref_s:.9e}")
        assert abs(peak[b] / ref_peak - 1) < PEAK_TOL[prec]
        # the intensity output is float32: on this bright (20 nm RMS) dark hole its own rounding,
        # 2^-24 I, reaches 1e-11; the extended plan is held to the bar plus that rounding
        rounding = 2.0 ** -24 * ref_i[mask] if prec == coro.MFT_EXT else 0.0
        assert np.all(np.abs(got[b][mask] - ref_i[mask]) <= DH_TOL_SMALL[prec] + rounding)
        assert abs(dh[b] - ref_s) <= 1e-3 * ref_s + mask.sum() * DH_TOL_SMALL[prec]
        assert np.max(np.abs(got[b] - ref_i)) < 1e-5      # whole detector, relative to the peak


@pytest.mark.parametrize("tile", [64, 32])
def test_lyot_ext_every_gemm_tile(ctx, tile):
    """Both output-tile widths the extended plan's tuner chooses from (128 x 64 and 128 x 32
    complex) meet the extended-precision bar on the uneven batch; the 3xTF32 plan has the one
    128 x 128 tile and refuses others."""
    n, npix, m_det, lyot = 128, 120, 96, 0.8
    items = [dict(m_occ=40, du_occ=0.25, spot_radius=3.0, du_det=0.5, dh_in=4.0, dh_out=16.0),
             dict(m_occ=45, du_occ=0.22, spot_radius=3.5, du_det=0.55, dh_in=4.5, dh_out=18.0)]
    pupils = np.stack([zernike_pupil(n, npix, 550e-9, s, rms=20e-9) for s in range(2)]).astype(np.complex64)
    x = torch.from_numpy(pupils).cuda()
    plan = coro.LyotPlan(ctx, n=n, npix=npix, lyot_frac=lyot, m_det=m_det, items=items, precision=coro.MFT_EXT)
    assert plan.gemm_tile()[0] == 128 and plan.gemm_tile()[1] in (64, 32)
    plan.set_gemm_tile(tile)
    assert plan.gemm_tile() == (128, tile)
    peak = plan.peak(x)
    inten = torch.empty((2, m_det, m_det), dtype=torch.float32, device="cuda")
    plan.execute(x, peak=peak, intensity=inten)
    got = inten.cpu().numpy()
    for b, it in enumerate(items):
        ref_i, _, ref_peak = oracle_psf(pupils[b].astype(np.complex128), n, npix, it, lyot, m_det)
        mask = coronagraph.dark_hole_mask(m_det, it["du_det"], it["dh_in"], it["dh_out"]) > 0
        print(f"tile {tile} item {b}: max |dI| {np.max(np.abs(got[b][mask] - ref_i[mask])):.3e}")
        assert abs(peak[b] / ref_peak - 1) < PEAK_TOL[coro.MFT_EXT]
        assert np.all(np.abs(got[b][mask] - ref_i[mask]) <= DH_TARGET + 2.0 ** -24 * ref_i[mask])
    with pytest.raises(coro.CoroError):
        plan.set_gemm_tile(128)
    p3 = coro.LyotPlan(ctx, n=n, npix=npix, lyot_frac=lyot, m_det=m_det, items=items, precision=coro.MFT_3XTF32)
    assert p3.gemm_tile() == (128, 128)
    p3.set_gemm_tile(128)
    with pytest.raises(coro.CoroError):
        p3.set_gemm_tile(64)


def full_size_error(ctx, prec):
    """1024^2 pupil with 5 nm RMS Zernike 4-21, 256^2 occulter at 0.05 lambda/D with a 5 lambda/D
    spot, Lyot stop 0.8, 512^2 detector at 0.25 lambda/D, dark hole 6-20 lambda/D; returns
    max |dI| over the dark hole (own peaks on both sides)."""
    w = inputs.LyotWorkload()
    pupil = zernike_pupil(w.n, w.npix, w.wavelength_m, w.seed).astype(np.complex64)
    x = torch.from_numpy(pupil).cuda().unsqueeze(0)
    it = dict(m_occ=w.m_occ, du_occ=w.du_occ, spot_radius=w.spot_radius_lamd, du_det=w.du_det,
              dh_in=w.dh_inner, dh_out=w.dh_outer)
    plan = coro.LyotPlan(ctx, n=w.n, npix=w.npix, lyot_frac=w.lyot_frac, m_det=w.m_det, items=[it], precision=prec)
    peak = plan.peak(x)
    inten = torch.empty((1, w.m_det, w.m_det), dtype=torch.float32, device="cuda")
    dh = plan.execute(x, peak=peak, intensity=inten)
    ref_i, ref_s, ref_peak = oracle_psf(pupil.astype(np.complex128), w.n, w.npix, it, w.lyot_frac, w.m_det)
    mask = coronagraph.dark_hole_mask(w.m_det, w.du_det, w.dh_inner, w.dh_outer) > 0
    got = inten.cpu().numpy()[0]
    err = np.max(np.abs(got[mask] - ref_i[mask]))
    print(f"prec {prec}: mean dark-hole contrast {ref_i[mask].mean():.3e}, peak rel {peak[0] / ref_peak - 1:.2e}, "
          f"max |dI| {err:.3e}, S {dh[0]:.9e} vs {ref_s:.9e}")
    assert abs(peak[0] / ref_peak - 1) < PEAK_TOL[prec]
    assert abs(dh[0] - ref_s) < (1e-4 if prec != coro.MFT_EXT else 1e-8) * ref_s
    return err


@pytest.mark.parametrize("prec", [coro.MFT_3XTF32, coro.MFT_3XBF16])
def test_lyot_full_size(ctx, prec):
    assert full_size_error(ctx, prec) < DH_TOL_FULL[prec]


def test_lyot_full_size_darkhole_target(ctx):
    """The split-precision tensor-core plan at extended precision meets the 1e-11 bar."""
    assert full_size_error(ctx, coro.MFT_EXT) <= DH_TARGET


def test_lyot_fp64_chain_meets_darkhole_target(ctx):
    """The full-size Lyot system composed from single FP64 calls on complex128 fields (MFT to
    the occulter, spot, inverse MFT, Babinet subtraction by axpy, Lyot stop, MFT to the
    detector): |dI| <= 1e-11 inside the dark hole, the bar the FP32-class split-precision
    GEMMs cannot reach (see the xfail above)."""
    w = inputs.LyotWorkload()
    pupil = zernike_pupil(w.n, w.npix, w.wavelength_m, w.seed)
    it = dict(m_occ=w.m_occ, du_occ=w.du_occ, spot_radius=w.spot_radius_lamd, du_det=w.du_det,
              dh_in=w.dh_inner, dh_out=w.dh_outer)
    npix = float(w.npix)
    e_a = torch.from_numpy(pupil).cuda().unsqueeze(0)
    stop = coro.element(coro.EL_CIRCLE, radius=0.5 * w.lyot_frac)            # D = 1 m, pitch 1/npix

    def detector(e_c):
        coro.apply_element(ctx, e_c, 1.0 / npix, w.wavelength_m, stop)
        return coro.propagate_mft(ctx, e_c, npix, -1, w.m_det, [w.du_det])

    peak = float((detector(e_a.clone()).abs() ** 2).max())                   # no occulter
    e_b = coro.propagate_mft(ctx, e_a, npix, -1, w.m_occ, [w.du_occ])
    coro.apply_element(ctx, e_b, w.du_occ, w.wavelength_m, coro.element(coro.EL_CIRCLE, radius=w.spot_radius_lamd))
    e_s = coro.propagate_mft(ctx, e_b, npix, +1, w.n, [w.du_occ])
    e_c = coro.wavefront_axpy(ctx, -1.0, e_s, e_a.clone())                   # E_A - IMFT(spot . E_B)
    got = (detector(e_c).abs() ** 2 / peak)[0].cpu().numpy()
    ref_i, ref_s, ref_peak = oracle_psf(pupil, w.n, w.npix, it, w.lyot_frac, w.m_det)
    assert abs(peak / ref_peak - 1) < 1e-12
    mask = coronagraph.dark_hole_mask(w.m_det, w.du_det, w.dh_inner, w.dh_outer) > 0
    err = np.max(np.abs(got[mask] - ref_i[mask]))
    print(f"FP64 chain: max |dI| in the dark hole {err:.3e} (mean contrast {ref_i[mask].mean():.3e})")
    assert err <= DH_TARGET


def test_lyot_plan_fp64_small_uneven_batch(ctx):
    """The plan at CORO_MFT_FP64 (complex128 pupils and fields): per-item peaks, intensities,
    the E_det field and dark-hole sums against the oracle on an uneven batch."""
    n, npix, m_det, lyot = 128, 120, 96, 0.8
    items = [dict(m_occ=40, du_occ=0.25, spot_radius=3.0, du_det=0.5, dh_in=4.0, dh_out=16.0),
             dict(m_occ=37, du_occ=0.27, spot_radius=3.0, du_det=0.45, dh_in=4.0, dh_out=16.0),
             dict(m_occ=45, du_occ=0.22, spot_radius=3.5, du_det=0.55, dh_in=4.5, dh_out=18.0)]
    pupils = np.stack([zernike_pupil(n, npix, 550e-9, s, rms=20e-9) for s in range(3)])
    x = torch.from_numpy(pupils).cuda()
    plan = coro.LyotPlan(ctx, n=n, npix=npix, lyot_frac=lyot, m_det=m_det, items=items, precision=coro.MFT_FP64)
    peak = plan.peak(x)
    inten = torch.empty((3, m_det, m_det), dtype=torch.float32, device="cuda")
    field = torch.empty((3, m_det, m_det), dtype=torch.complex128, device="cuda")
    dh = plan.execute(x, peak=peak, intensity=inten, field=field)
    got, got_f = inten.cpu().numpy(), field.cpu().numpy()
    for b, it in enumerate(items):
        ref_i, ref_s, ref_peak = oracle_psf(pupils[b], n, npix, it, lyot, m_det)
        p = coronagraph.LyotParams(n=n, npix=npix, m_occ=it["m_occ"], du_occ=it["du_occ"],
                                   spot_radius=it["spot_radius"], lyot_frac=lyot, m_det=m_det, du_det=it["du_det"])
        ref_f = coronagraph.lyot_fields(pupils[b], p)["det"]
        assert abs(peak[b] / ref_peak - 1) < 1e-12
        mask = coronagraph.dark_hole_mask(m_det, it["du_det"], it["dh_in"], it["dh_out"]) > 0
        i64 = np.abs(got_f[b]) ** 2 / peak[b]                  # the FP64 result; the float32
        err = np.max(np.abs(i64[mask] - ref_i[mask]))          # intensity adds its own rounding
        print(f"FP64 plan item {b}: max |dI| in dark hole {err:.3e}, S {dh[b]:.9e} vs {ref_s:.9e}")
        assert err <= DH_TARGET
        assert np.all(np.abs(got[b] - ref_i) <= 2.0 ** -23 * ref_i + 1e-13)
        assert np.max(np.abs(got_f[b] - ref_f)) < 1e-10 * np.sqrt(ref_peak)
        assert abs(dh[b] - ref_s) <= 1e-9 * ref_s
    with pytest.raises(coro.CoroError):
        plan.gradient(x, peak)
    dh_default = plan.execute(x)                               # peak NULL = 1: unnormalised sums
    np.testing.assert_allclose(dh_default, dh * peak, rtol=1e-12)


def test_lyot_plan_fp64_full_size_meets_darkhole_target(ctx):
    """The full-size Lyot system through the plan at CORO_MFT_FP64: |dI| <= 1e-11 in the dark
    hole, the bar the split-precision plan misses."""
    w = inputs.LyotWorkload()
    pupil = zernike_pupil(w.n, w.npix, w.wavelength_m, w.seed)
    x = torch.from_numpy(pupil).cuda().unsqueeze(0)
    it = dict(m_occ=w.m_occ, du_occ=w.du_occ, spot_radius=w.spot_radius_lamd, du_det=w.du_det,
              dh_in=w.dh_inner, dh_out=w.dh_outer)
    plan = coro.LyotPlan(ctx, n=w.n, npix=w.npix, lyot_frac=w.lyot_frac, m_det=w.m_det, items=[it],
                         precision=coro.MFT_FP64)
    peak = plan.peak(x)
    field = torch.empty((1, w.m_det, w.m_det), dtype=torch.complex128, device="cuda")
    dh = plan.execute(x, peak=peak, field=field)
    ref_i, ref_s, ref_peak = oracle_psf(pupil, w.n, w.npix, it, w.lyot_frac, w.m_det)
    assert abs(peak[0] / ref_peak - 1) < 1e-12
    mask = coronagraph.dark_hole_mask(w.m_det, w.du_det, w.dh_inner, w.dh_outer) > 0
    err = np.max(np.abs(np.abs(field.cpu().numpy()[0][mask]) ** 2 / peak[0] - ref_i[mask]))
    print(f"FP64 plan: max |dI| in the dark hole {err:.3e}, S {dh[0]:.9e} vs {ref_s:.9e}")
    assert err <= DH_TARGET
    assert abs(dh[0] - ref_s) <= 1e-9 * ref_s


def test_lyot_graph_replay_matches_eager(ctx):
    """a10: the graph-replayed execute gives bitwise the eager result, follows new peak values
    (copied outside the graph) and re-captures when the output buffer changes."""
    n, npix, m_det = 128, 120, 96
    items = [dict(m_occ=40, du_occ=0.25, spot_radius=3.0, du_det=0.5, dh_in=4.0, dh_out=16.0),
             dict(m_occ=37, du_occ=0.27, spot_radius=3.0, du_det=0.45, dh_in=4.0, dh_out=16.0)]
    pupils = np.stack([zernike_pupil(n, npix, 550e-9, s, rms=20e-9) for s in range(2)]).astype(np.complex64)
    x = torch.from_numpy(pupils).cuda()
    plan = coro.LyotPlan(ctx, n=n, npix=npix, lyot_frac=0.8, m_det=m_det, items=items, precision=coro.MFT_3XTF32)
    peak = plan.peak(x)
    eager = torch.empty((2, m_det, m_det), dtype=torch.float32, device="cuda")
    dh_eager = plan.execute(x, peak=peak, intensity=eager)
    plan.use_graph(True)
    out = torch.full((2, m_det, m_det), float("nan"), device="cuda")
    for _ in range(3):                                  # capture, then two replays
        out.fill_(float("nan"))
        dh = plan.execute(x, peak=peak, intensity=out)
        assert torch.equal(out, eager)
        assert np.array_equal(dh, dh_eager)
    dh2 = plan.execute(x, peak=2 * np.asarray(peak), intensity=out)     # new normalisation, same graph
    assert torch.allclose(out, eager / 2, rtol=1e-6, atol=0)
    assert np.allclose(dh2, dh_eager / 2, rtol=1e-12)
    other = torch.empty_like(out)
    plan.execute(x, peak=peak, intensity=other)        # new pointer: re-captured
    assert torch.equal(other, eager)
    plan.set_timing(2)
    for _ in range(2):
        other.fill_(float("nan"))
        plan.execute_n(x, 2, peak=peak, intensity=other)
        assert torch.equal(other, eager)
    t = plan.unit_times(2)
    assert t.shape == (2, 6) and np.all(t > 0)
    plan.set_timing(0)
    plan.use_graph(False)


@pytest.mark.slow
@pytest.mark.parametrize("prec", [coro.MFT_3XTF32, coro.MFT_EXT])
def test_broadband_batch_sampled_items(ctx, prec):
    """The benchmarked broadband workload as bench.py runs it -- 21 wavelengths x 8 DM sinc
    probes = 168 items with uneven occulters (235-282 px), three executes replayed as one CUDA
    graph. Sampled items (first, middle, last): the GPU-synthesised pupil (aperture, Zernike
    4-21 and the DM probe OPD as phasors) against the oracle's own pupil, then the PSF of that
    pupil against the oracle's PSF of it, own peaks on both sides."""
    bw = inputs.BroadbandWorkload()
    lw = bw.lyot
    lams = bw.wavelengths()
    lam_b = np.repeat(lams, bw.n_probe)
    B, n, npix, md = len(lam_b), lw.n, lw.npix, lw.m_det
    dx = lw.diam_m / npix
    field = torch.empty((B, n, n), dtype=torch.complex64, device="cuda")
    coro.wavefront_init(ctx, field, 1.0)
    coro.apply_element(ctx, field, dx, lam_b, coro.element(coro.EL_APERTURE, radius=lw.diam_m / 2))
    coro.apply_element(ctx, field, dx, lam_b, coro.element(coro.EL_ZERNIKE, radius=lw.diam_m / 2,
                                                           coeffs=lw.zernike(), j_first=lw.zernike_first))
    probes = bw.probes()
    heights = torch.from_numpy(np.tile(probes, (len(lams), 1, 1)).astype(np.float32)).cuda()
    pitch = lw.diam_m / bw.n_act
    opd = coro.dm_opd(ctx, heights, pitch, pitch, n, dx, 2.0)
    coro.apply_element(ctx, field, dx, lam_b, coro.element(coro.EL_OPD_MAP, opd=opd, flags=coro.ELF_MAP_BATCHED))
    del opd
    r = bw.lambda_c_m / lam_b
    items = [dict(m_occ=int(m), du_occ=lw.du_occ * rr, spot_radius=lw.spot_radius_lamd * rr, du_det=lw.du_det * rr,
                  dh_in=lw.dh_inner * rr, dh_out=lw.dh_outer * rr)
             for m, rr in zip(np.repeat(bw.occulter_sizes(), bw.n_probe), r)]
    plan = coro.LyotPlan(ctx, n=n, npix=npix, lyot_frac=lw.lyot_frac, m_det=md, items=items, precision=prec)
    peak = plan.peak(field)
    inten = torch.empty((B, md, md), dtype=torch.float32, device="cuda")
    plan.use_graph(True)
    plan.execute_n(field, 3, peak=peak, intensity=inten)
    torch.cuda.synchronize()
    zopd = optics.zernike_opd(n, dx, lw.diam_m / 2, lw.zernike(), lw.zernike_first)
    aperture = optics.circular_aperture(n, dx, lw.diam_m / 2)
    for b in (0, B // 2, B - 1):
        it = items[b]
        e = field[b].cpu().numpy().astype(np.complex128)
        dm = optics.dm_opd(n, dx, probes[b % bw.n_probe].astype(np.float32).astype(np.float64), pitch)
        e_ref = aperture * optics.phasor(zopd + dm, lam_b[b])
        pupil_err = np.linalg.norm(e - e_ref) / np.linalg.norm(e_ref)
        ref_i, ref_s, ref_peak = oracle_psf(e, n, npix, it, lw.lyot_frac, md)
        got = inten[b].cpu().numpy()
        mask = coronagraph.dark_hole_mask(md, it["du_det"], it["dh_in"], it["dh_out"]) > 0
        err = np.max(np.abs(got[mask] - ref_i[mask]))
        print(f"prec {prec} item {b} (m_occ {it['m_occ']}): pupil rel L2 {pupil_err:.2e}, "
              f"peak rel {peak[b] / ref_peak - 1:.2e}, max |dI| in dark hole {err:.3e}")
        assert pupil_err < 1e-6
        assert abs(peak[b] / ref_peak - 1) < PEAK_TOL[prec]
        assert err < DH_TOL_FULL[prec]
        assert np.max(np.abs(got - ref_i)) < 1e-5
    plan.use_graph(False)
