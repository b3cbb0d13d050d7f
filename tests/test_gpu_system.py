"""GPU parity: Fresnel systems with the propagation method chosen by a Gaussian pilot beam
(coro_fresnel_system_create; Sec. 1.1 citing Lawrence's angular-spectrum / direct choice)
and the direct hop with z < 0, against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import optics, propagation
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return coro.Context(0)


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def gaussian(n, pitch, wavelength, q):
    r2 = optics.radius_sq_exact(n, pitch)
    return np.exp(1j * np.pi * r2 / (wavelength * q))


@pytest.mark.parametrize("z", [0.37, -0.37])
def test_direct_hop_both_directions(ctx, z):
    """Standalone direct hop: z > 0 (forward DFT) and z < 0 (inverse DFT, natural grid)."""
    n, dx, lam = 256, 2e-5, 633e-9
    e = inputs.random_field((n, n), seed=4) * optics.circular_aperture(n, dx, 0.3 * n * dx)
    x = torch.from_numpy(e.astype(np.complex64)).cuda().unsqueeze(0).contiguous()
    ps = coro.propagate_fresnel(ctx, x, dx, lam, z, coro.FRESNEL_DIRECT)
    ref, du = propagation.direct_fresnel(e, dx, lam, z)
    assert abs(ps[0] - du) < 1e-15 * du
    assert rel_l2(x.cpu().numpy()[0], ref) < 1e-5
    ps2 = coro.propagate_fresnel(ctx, x, ps, lam, -z, coro.FRESNEL_DIRECT)    # and back
    assert abs(ps2[0] - dx) < 1e-15 * dx
    assert rel_l2(x.cpu().numpy()[0], e) < 1e-5


def test_pilot_system_gaussian_through_focus(ctx):
    """Gaussian beam, lens, focus, beyond (outside -> inside -> outside -> outside with a
    backward leg): GPU plan vs the oracle and vs the closed form."""
    n, lam, w0 = 256, 1e-6, 1e-3
    dx = w0 / 20
    q0 = complex(0.0, -np.pi * w0 ** 2 / lam)
    e0 = gaussian(n, dx, lam, q0)
    distances = [0.5, 0.3, 0.2]
    plan = coro.FresnelSystem(ctx, n=n, batch=1, pixelscale=dx, wavelength=lam, beam_radius=w0, distances=distances,
                              elements=[coro.element(coro.EL_LENS, plane=0, focal_length=0.5)])
    flags, legs = plan.info()
    assert flags == [True, False, True, True] and legs == 4
    x = torch.from_numpy(e0.astype(np.complex64)).cuda().unsqueeze(0).contiguous()
    ps = plan.execute(x)
    ref, pitch, rflags, rlegs = propagation.fresnel_system_pilot(e0, dx, lam, w0, [[("lens", 0.5)], [], [], []], distances)
    assert rflags == flags and rlegs == legs
    assert abs(ps[0] - pitch) < 1e-14 * pitch
    assert rel_l2(x.cpu().numpy()[0], ref) < 1e-5
    q = 1.0 / (1.0 / q0 - 1.0 / 0.5)
    amp = 1.0 + 0j
    for d in distances:
        amp *= q / (q + d)
        q = q + d
    assert rel_l2(x.cpu().numpy()[0], amp * gaussian(n, pitch, lam, q)) < 1e-5


def relay_with_foci(n, dx, w):
    """Aperture + PSD surface + lens at the pupil, a field stop at the focus, a collimating
    lens, a Lyot-like stop in the relayed pupil, a final lens to the detector focus."""
    r = 0.5 * n * dx / 2
    maps = [m.astype(np.float32) for m in w.psd_maps()]
    gpu = [coro.element(coro.EL_APERTURE, plane=0, radius=r, obscuration=0.3, n_spiders=4, spider_width=0.02 * r),
           coro.element(coro.EL_LENS, plane=0, focal_length=2.0),
           coro.element(coro.EL_CIRCLE, plane=1, radius=FIELD_STOP),
           coro.element(coro.EL_LENS, plane=2, focal_length=1.5),
           coro.element(coro.EL_CIRCLE, plane=3, radius=0.35 * r),
           coro.element(coro.EL_LENS, plane=3, focal_length=3.0)]
    dist = [2.0, 1.5, 1.5, 3.0]          # focus, collimating lens, relayed pupil, final focus
    return maps, gpu, dist, r


FIELD_STOP = 2.5e-5                      # about 22 lambda/D at the first focus


def test_pilot_system_relay_with_foci_batch(ctx):
    """A five-plane relay (pupil with lens, field-stopped focus, collimating lens, relayed
    pupil with stop and lens, final focus), two wavelengths in one batch (the pilot-beam
    regimes agree), every item against the oracle."""
    n = 512
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=6)
    dx = w.dx
    lams = np.array([540e-9, 560e-9])
    maps, els, dist, r = relay_with_foci(n, dx, w)
    opd = torch.from_numpy(maps[0]).cuda()
    els.append(coro.element(coro.EL_OPD_MAP, plane=0, opd=opd))
    plan = coro.FresnelSystem(ctx, n=n, batch=2, pixelscale=dx, wavelength=lams, beam_radius=r, distances=dist,
                              elements=els, init_uniform=True)
    flags, legs = plan.info()
    x = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    ps = plan.execute(x)
    got = x.cpu().numpy()
    for b, lam in enumerate(lams):
        planes = [[lambda nn, p: optics.circular_aperture(nn, p, r, 0.3, 4, 0.02 * r),
                   lambda nn, p, lam=lam: optics.phasor(maps[0].astype(np.float64), lam), ("lens", 2.0)],
                  [lambda nn, p: optics.circle_stop(nn, p, FIELD_STOP)],
                  [("lens", 1.5)],
                  [lambda nn, p: optics.circle_stop(nn, p, 0.35 * r), ("lens", 3.0)],
                  []]
        ref, pitch, rflags, rlegs = propagation.fresnel_system_pilot(np.ones((n, n), complex), dx, lam, r, planes, dist)
        assert rflags == flags and rlegs == legs
        assert abs(ps[b] - pitch) < 1e-13 * pitch
        err = rel_l2(got[b], ref)
        print(f"item {b}: flags {flags}, direct legs {legs}, final pitch {pitch:.3e}, rel L2 {err:.2e}")
        assert err < 1e-5
    assert flags == [True, False, False, True, False] and legs == 3


def test_pilot_system_regime_disagreement_is_rejected(ctx):
    """Items whose pilot beams fall on different sides of the Rayleigh range: CORO_ENOTIMPL."""
    n, dx, w0 = 128, 1e-4, 2e-3
    lams = np.array([500e-9, 5e-6])                          # z_R = 25 m and 2.5 m
    with pytest.raises(coro.CoroError):
        coro.FresnelSystem(ctx, n=n, batch=2, pixelscale=dx, wavelength=lams, beam_radius=w0, distances=[10.0],
                           elements=[])


def spc_elements(w, maps):
    """GPU elements of the App.-B-shaped system; maps: dict of device tensors for the two masks."""
    els = []
    for p, plane in enumerate(w.layout()):
        for el in plane:
            if el[0] == "aperture":
                els.append(coro.element(coro.EL_APERTURE, plane=p, radius=w.d_prim_m / 2, obscuration=w.obscuration,
                                        n_spiders=w.n_spiders, spider_width=w.spider_width_frac * w.d_prim_m))
            elif el[0] == "lens":
                els.append(coro.element(coro.EL_LENS, plane=p, focal_length=el[1]))
            else:
                els.append(coro.element(coro.EL_OPD_MAP, plane=p, opd=maps["zero"], amplitude=maps[el[0]],
                                        flags=coro.ELF_MAP_BATCHED))
    return els


def spc_oracle(w, lam, pitch_sp, pitch_fpm):
    def ap(nn, p):
        return optics.circular_aperture(nn, p, w.d_prim_m / 2, w.obscuration, w.n_spiders,
                                        w.spider_width_frac * w.d_prim_m)

    def sp(nn, p):
        assert abs(p - pitch_sp) < 1e-13 * p         # the GPU plan chose the same sampling
        return w.shaped_pupil(nn, p)

    def fpm(nn, p):
        assert abs(p - pitch_fpm) < 1e-13 * p
        return w.bowtie(nn, p, lam)

    planes = []
    for plane in w.layout():
        row = []
        for el in plane:
            row.append({"aperture": ap, "shaped_pupil": sp, "fpm": fpm}[el[0]] if el[0] != "lens" else ("lens", el[1]))
        planes.append(row)
    return propagation.fresnel_system_pilot(np.ones((w.n, w.n), complex), w.dx, lam, w.d_prim_m / 2, planes,
                                            w.distances())


def test_spc_shaped_system(ctx):
    """Next row f1: the nine-plane system of App. B's shape (telescope, 20 mm relay, shaped
    pupil, bow-tie focal-plane mask, three foci; seven direct legs) at two wavelengths, with
    the masks generated at the sampling the plan chose, against the oracle."""
    w = inputs.SpcWorkload(npix=128)
    n, lams = w.n, np.array([545e-9, 555e-9])
    maps = {"zero": torch.zeros((2, n, n), device="cuda"), "shaped_pupil": torch.zeros((2, n, n), device="cuda"),
            "fpm": torch.zeros((2, n, n), device="cuda")}
    plan = coro.FresnelSystem(ctx, n=n, batch=2, pixelscale=w.dx, wavelength=lams, beam_radius=w.d_prim_m / 2,
                              distances=w.distances(), elements=spc_elements(w, maps), init_uniform=True)
    p_sp, p_fpm = plan.plane_pitch(4), plan.plane_pitch(6)
    for b, lam in enumerate(lams):
        maps["shaped_pupil"][b] = torch.from_numpy(w.shaped_pupil(n, p_sp[b]))
        maps["fpm"][b] = torch.from_numpy(w.bowtie(n, p_fpm[b], lam))
    flags, legs = plan.info()
    x = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    ps = plan.execute(x)
    got = x.cpu().numpy()
    for b, lam in enumerate(lams):
        ref, pitch, rflags, rlegs = spc_oracle(w, lam, p_sp[b], p_fpm[b])
        assert rflags == flags and rlegs == legs == 7
        assert abs(ps[b] - pitch) < 1e-13 * pitch
        err = rel_l2(got[b], ref)
        print(f"spc item {b}: final pitch {pitch:.3e} m, rel L2 {err:.2e}")
        assert err < 1e-5
