"""GPU parity of the differentiable wavefront-control chain against the FP64 oracle: DM
synthesis and its transpose, the Lyot-chain adjoint, and dL/dh of the two-DM system (adjoint
chain vs the oracle's adjoint and vs FP64 central finite differences, h = 1e-3 nm, on 16
seeded actuators). Gradient bar: 1e-3 relative."""
import numpy as np
import pytest
import torch

from oracle import adjoint, coronagraph, optics
from paper_1806_06467_gb300 import coro, inputs, wfc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    c = coro.Context(0)
    yield c
    c.synchronize()


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.complex128) - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("n,dx,na,pitch", [(256, 1.0 / 200, 12, 1.0 / 12), (1024, 0.048 / 1024, 48, 1e-3),
                                           (4096, 0.048 / 1024, 48, 1e-3)])
def test_dm_opd_and_correlate(ctx, n, dx, na, pitch):
    """Gaussian-influence synthesis and its transpose (FWHM one pitch) against the oracle's
    influence matrices: a coarse grid, the 1024^2 pupil of the Lyot workloads and the 4096^2
    grid of the wavefront-control workload (DM over its central 1024 pixels)."""
    h = inputs.dm_heights(5, na, 2)
    ht = torch.from_numpy(h.astype(np.float32)).cuda()
    opd = coro.dm_opd(ctx, ht, pitch, pitch, n, dx, 2.0).cpu().numpy()
    for b in range(2):
        ref = optics.dm_opd(n, dx, h[b].astype(np.float32).astype(np.float64), pitch)
        assert np.max(np.abs(opd[b] - ref)) < 1e-5 * np.max(np.abs(ref))
    w = inputs.rng(3).standard_normal((2, n, n))
    g = coro.dm_correlate(ctx, torch.from_numpy(w.astype(np.float32)).cuda(), dx, na, pitch, pitch, 3.0).cpu().numpy()
    gm = optics.dm_influence_matrix(n, dx, na, pitch)
    for b in range(2):
        ref = 3.0 * gm.T @ w[b].astype(np.float32).astype(np.float64) @ gm
        assert np.max(np.abs(g[b] - ref)) < 1e-5 * np.max(np.abs(ref))


def small_setup(prec=coro.MFT_3XTF32):
    npix, n_f, na = 32, 128, 8
    items = dict(m_occ=20, du_occ=0.35, spot_radius=2.5, du_det=0.5, dh_in=3.0, dh_out=9.0)
    lyot = coronagraph.LyotParams(n=npix, npix=npix, m_occ=20, du_occ=0.35, spot_radius=2.5, lyot_frac=0.8,
                                  m_det=40, du_det=0.5)
    p = adjoint.WfcParams(n_f=n_f, npix=npix, diam_m=0.048, z_m=0.3, n_act=na, lyot=lyot, dh_in=3.0, dh_out=9.0)
    return p, items


@pytest.mark.parametrize("prec", [coro.MFT_3XTF32, coro.MFT_3XBF16])
def test_lyot_adjoint_matches_oracle(ctx, prec):
    p, it = small_setup()
    lp = p.lyot
    e = coronagraph.pupil_field(lp.n, lp.npix, 550e-9, optics.zernike_opd(lp.n, 1 / lp.npix, 0.5,
                                inputs.zernike_coefficients(1, 4, 11, 30e-9), 4)).astype(np.complex64)
    x = torch.from_numpy(e).cuda().unsqueeze(0)
    plan = coro.LyotPlan(ctx, n=lp.n, npix=lp.npix, lyot_frac=lp.lyot_frac, m_det=lp.m_det, items=[it], precision=prec)
    peak = plan.peak(x)
    g, dh = plan.gradient(x, peak)
    e64 = e.astype(np.complex128)
    det = coronagraph.lyot_fields(e64, lp)["det"]
    mask = coronagraph.dark_hole_mask(lp.m_det, lp.du_det, 3.0, 9.0)
    ref = adjoint.lyot_adjoint(mask * det / peak[0], lp)
    err = rel_l2(g.cpu().numpy()[0], ref)
    print(f"prec {prec}: Lyot adjoint rel L2 {err:.3e}")
    assert err < 1e-3
    assert abs(dh[0] / coronagraph.dark_hole_sum(np.abs(det) ** 2 / peak[0], lp.du_det, 3.0, 9.0) - 1) < 1e-3


def make_wfc(ctx, p, it, lams, prec):
    return wfc.WfcPlan(ctx, wavelengths=lams, n_fresnel=p.n_f, diam_m=p.diam_m, npix=p.npix, z_m=p.z_m,
                       n_act=p.n_act, pitch_m=p.pitch, fwhm_m=p.pitch, lyot_frac=p.lyot.lyot_frac,
                       m_det=p.lyot.m_det, items=[it] * len(lams), precision=prec)


def test_wfc_gradient_matches_oracle_and_fd(ctx):
    p, it = small_setup()
    lams = [530e-9, 570e-9]
    h = inputs.dm_heights(7, p.n_act, 2)
    plan = make_wfc(ctx, p, it, lams, coro.MFT_3XTF32)
    peaks = plan.peak()
    ht = torch.from_numpy(h.astype(np.float32)).cuda().requires_grad_(True)
    loss = wfc.dark_hole_loss(ht, plan)
    loss.backward()
    got = ht.grad.cpu().numpy().astype(np.float64)
    h32 = h.astype(np.float32).astype(np.float64)
    ref_loss, ref_grad, ref_peaks = adjoint.broadband_gradient(h32, lams, p)
    np.testing.assert_allclose(peaks, ref_peaks, rtol=1e-5)
    assert abs(loss.item() / ref_loss - 1) < 1e-4
    err = np.linalg.norm(got - ref_grad) / np.linalg.norm(ref_grad)
    print(f"wfc gradient rel L2 vs oracle adjoint {err:.3e}")
    assert err < 1e-3
    # FP64 central differences of the oracle loss on 16 seeded actuators
    d = 1e-12
    picks = inputs.actuator_offsets(11, p.n_act, 16)
    scale = np.abs(ref_grad).max()
    for dm, r, c in picks:
        hp = h32.copy(); hp[dm, r, c] += d
        hm = h32.copy(); hm[dm, r, c] -= d
        fd = sum(adjoint.forward(hp, lam, p, peak=pk)["loss"] - adjoint.forward(hm, lam, p, peak=pk)["loss"]
                 for lam, pk in zip(lams, ref_peaks)) / (2 * d)
        assert abs(got[dm, r, c] - fd) <= 1e-3 * scale, (dm, r, c, got[dm, r, c], fd)


def test_wfc_forward_only_matches_gradient_pass(ctx):
    p, it = small_setup()
    plan = make_wfc(ctx, p, it, [550e-9], coro.MFT_3XTF32)
    h = torch.from_numpy(inputs.dm_heights(2, p.n_act, 2).astype(np.float32)).cuda()
    l0, per0, _ = plan.evaluate(h, want_grad=False)
    l1, per1, g = plan.evaluate(h, want_grad=True)
    assert l0 == pytest.approx(l1, rel=1e-12)
    assert torch.isfinite(g).all()


def full_size_params(w, lam):
    """The oracle's parameters for one wavelength of the 4096^2, 48x48-actuator workload."""
    it = w.item(lam)
    lw = w.lyot
    lyot = coronagraph.LyotParams(n=lw.n, npix=lw.npix, m_occ=it["m_occ"], du_occ=it["du_occ"],
                                  spot_radius=it["spot_radius"], lyot_frac=lw.lyot_frac, m_det=lw.m_det,
                                  du_det=it["du_det"])
    return adjoint.WfcParams(n_f=w.n_fresnel, npix=lw.npix, diam_m=w.diam_m, z_m=w.z_m, n_act=w.n_act, lyot=lyot,
                             dh_in=it["dh_in"], dh_out=it["dh_out"])


def oracle_pool():
    """Spawned FP64 oracle workers, one BLAS thread each (about 2.5 GB per worker at 4096^2)."""
    import multiprocessing as mp
    import os
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(max(1, min(12, (os.cpu_count() or 2) - 2)))
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k)
            else:
                os.environ[k] = v


@pytest.mark.slow
def test_wfc_full_size_gradient(ctx):
    """The full workload: 2 x 48 x 48 heights (uniform +-5 nm), Fresnel 4096^2 over 0.3 m,
    Lyot chain at 11 wavelengths over 525-575 nm (3xTF32). Per-wavelength sums and the summed
    gradient against the FP64 oracle's adjoint; then, at 550 nm alone, the GPU gradient
    against FP64 central differences (h = 1e-3 nm) on 16 seeded actuators."""
    w = inputs.WfcWorkload()
    lw = w.lyot
    lams = list(w.wavelengths())
    h32 = w.heights().astype(np.float32).astype(np.float64)
    ht = torch.from_numpy(h32.astype(np.float32)).cuda()

    def plan_for(ls):
        return wfc.WfcPlan(ctx, wavelengths=ls, n_fresnel=w.n_fresnel, diam_m=w.diam_m, npix=lw.npix, z_m=w.z_m,
                           n_act=w.n_act, pitch_m=w.pitch_m, fwhm_m=w.pitch_m, lyot_frac=lw.lyot_frac,
                           m_det=lw.m_det, items=[w.item(l) for l in ls], precision=coro.MFT_3XTF32)

    plan = plan_for(lams)
    peaks = plan.peak()
    loss, per, grad = plan.evaluate(ht)
    got = grad.cpu().numpy().astype(np.float64)
    plan.close()
    lc = w.lambda_c_m
    plan1 = plan_for([lc])
    _, per1, g1 = plan1.evaluate(ht)
    got1 = g1.cpu().numpy().astype(np.float64)
    plan1.close()

    params = [full_size_params(w, l) for l in lams]
    pc = full_size_params(w, lc)
    picks = w.fd_actuators(16)
    d = 1e-12
    with oracle_pool() as pool:
        ref_peaks = pool.starmap(adjoint.zero_height_peak, [(l, p) for l, p in zip(lams, params)])
        pk_c = ref_peaks[lams.index(lc)] if lc in lams else adjoint.zero_height_peak(lc, pc)
        jobs = [(h32, l, p, None, pk) for l, p, pk in zip(lams, params, ref_peaks)]
        ref = pool.starmap(adjoint.gradient, jobs)
        fd_jobs = []
        for dm, r, c in picks:
            for s in (1.0, -1.0):
                hh = h32.copy()
                hh[dm, r, c] += s * d
                fd_jobs.append((hh, lc, pc, pk_c))
        fd_loss = pool.starmap(adjoint.loss, fd_jobs)
    np.testing.assert_allclose(peaks, ref_peaks, rtol=1e-5)
    ref_per = np.array([r[0] for r in ref])
    ref_grad = sum(r[1] for r in ref)
    per_err = np.max(np.abs(per / ref_per - 1))
    err = np.linalg.norm(got - ref_grad) / np.linalg.norm(ref_grad)
    print(f"full-size wfc: per-wavelength dark-hole sums max rel {per_err:.3e}; gradient rel L2 {err:.3e}")
    assert per_err < 1e-3
    assert err < 1e-3
    fd = (np.array(fd_loss[0::2]) - np.array(fd_loss[1::2])) / (2 * d)
    gp = np.array([got1[dm, r, c] for dm, r, c in picks])
    scale = np.abs(got1).max()
    worst = np.max(np.abs(gp - fd)) / scale
    print(f"full-size wfc at 550 nm: GPU gradient vs FP64 central differences, max |diff| / max |grad| {worst:.3e}")
    assert worst <= 1e-3, list(zip(gp, fd))


def test_wfc_chunked_band_matches_resident(ctx):
    """HBM budget: the same three-wavelength system with all wavelengths resident, two per
    chunk and one per chunk gives the same per-wavelength sums and gradient."""
    p, it = small_setup()
    lams = [530e-9, 550e-9, 570e-9]
    h = torch.from_numpy(inputs.dm_heights(9, p.n_act, 2).astype(np.float32)).cuda()
    out = {}
    for res in (0, 2, 1):
        plan = wfc.WfcPlan(ctx, wavelengths=lams, n_fresnel=p.n_f, diam_m=p.diam_m, npix=p.npix, z_m=p.z_m,
                           n_act=p.n_act, pitch_m=p.pitch, fwhm_m=p.pitch, lyot_frac=p.lyot.lyot_frac,
                           m_det=p.lyot.m_det, items=[it] * 3, precision=coro.MFT_3XTF32, max_resident=res)
        r, chunks = plan.resident()
        assert (r, chunks) == {0: (3, 1), 2: (2, 2), 1: (1, 3)}[res]
        loss, per, g = plan.evaluate(h)
        out[res] = (loss, per, g.cpu().numpy().astype(np.float64), plan.peak())
        plan.close()
    for res in (2, 1):
        np.testing.assert_allclose(out[res][3], out[0][3], rtol=1e-6)
        np.testing.assert_allclose(out[res][1], out[0][1], rtol=1e-6)
        assert np.linalg.norm(out[res][2] - out[0][2]) / np.linalg.norm(out[0][2]) < 1e-6


@pytest.mark.slow
def test_wfc_8192_grid_196_actuators(ctx):
    """The N = 8192 case of Sec. 1.2: 196 x 196 actuators at seven pixels per actuator (a
    1372-pixel pupil), two wavelengths run one per chunk (1.5 GiB of fields resident), against
    the FP64 oracle: per-wavelength dark-hole sums and the summed gradient (adjoint)."""
    nf, na, npix, D, z = 8192, 196, 1372, 0.0784, 0.3
    pitch = D / na
    lams = [540e-9, 560e-9]
    lw = inputs.LyotWorkload(n=npix, npix=npix)

    def item(lam):
        r = 550e-9 / lam
        return dict(m_occ=int(np.rint(lw.m_occ * r)), du_occ=lw.du_occ * r, spot_radius=lw.spot_radius_lamd * r,
                    du_det=lw.du_det * r, dh_in=lw.dh_inner * r, dh_out=lw.dh_outer * r)

    items = [item(l) for l in lams]
    plan = wfc.WfcPlan(ctx, wavelengths=lams, n_fresnel=nf, diam_m=D, npix=npix, z_m=z, n_act=na, pitch_m=pitch,
                       fwhm_m=pitch, lyot_frac=lw.lyot_frac, m_det=lw.m_det, items=items,
                       precision=coro.MFT_3XTF32, max_resident=1)
    assert plan.resident() == (1, 2)
    h32 = inputs.dm_heights(21, na, 2).astype(np.float32).astype(np.float64)
    peaks = plan.peak()
    loss, per, g = plan.evaluate(torch.from_numpy(h32.astype(np.float32)).cuda())
    got = g.cpu().numpy().astype(np.float64)
    plan.close()

    def params(lam, it):
        lyot = coronagraph.LyotParams(n=npix, npix=npix, m_occ=it["m_occ"], du_occ=it["du_occ"],
                                      spot_radius=it["spot_radius"], lyot_frac=lw.lyot_frac, m_det=lw.m_det,
                                      du_det=it["du_det"])
        return adjoint.WfcParams(n_f=nf, npix=npix, diam_m=D, z_m=z, n_act=na, lyot=lyot, dh_in=it["dh_in"],
                                 dh_out=it["dh_out"])

    ps = [params(l, it) for l, it in zip(lams, items)]
    with oracle_pool() as pool:
        ref_peaks = pool.starmap(adjoint.zero_height_peak, list(zip(lams, ps)))
        ref = pool.starmap(adjoint.gradient, [(h32, l, p, None, pk) for l, p, pk in zip(lams, ps, ref_peaks)])
    np.testing.assert_allclose(peaks, ref_peaks, rtol=1e-5)
    ref_per = np.array([r[0] for r in ref])
    ref_grad = ref[0][1] + ref[1][1]
    per_err = np.max(np.abs(per / ref_per - 1))
    err = np.linalg.norm(got - ref_grad) / np.linalg.norm(ref_grad)
    print(f"8192^2 wfc, 196 actuators: dark-hole sums max rel {per_err:.3e}; gradient rel L2 {err:.3e}")
    assert per_err < 1e-3
    assert err < 1e-3


def test_wfc_rejects_negative_budget(ctx):
    p, it = small_setup()
    with pytest.raises(RuntimeError):
        wfc.WfcPlan(ctx, wavelengths=[550e-9], n_fresnel=p.n_f, diam_m=p.diam_m, npix=p.npix, z_m=p.z_m,
                    n_act=p.n_act, pitch_m=p.pitch, fwhm_m=p.pitch, lyot_frac=p.lyot.lyot_frac,
                    m_det=p.lyot.m_det, items=[it], precision=coro.MFT_3XTF32, max_resident=-1)
