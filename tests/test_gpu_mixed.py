"""GPU parity of the mixed-radix passes (line lengths that are not powers of two: N = 2800 of
Sec. 3.1, N = 4100 = 4 x 1025 of App. B's npix = 1025) against the FP64 oracle, through the
C ABI: centred 2-D DFTs, Fresnel hops, elements and a fused relay plan.

Tolerance: relative L2 error <= 1e-5 for complex64 and <= 1e-12 for complex128 (widened by
the oracle's own rounding of large quadratic phases where a lens is involved)."""
import numpy as np
import pytest
import torch

from oracle import optics, propagation
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu

TOL = {torch.complex64: 1e-5, torch.complex128: 1e-12}


@pytest.fixture(scope="module")
def ctx(lib):
    return coro.Context(0)


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def to_dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda().contiguous()


@pytest.mark.parametrize("n,dtype", [(48, torch.complex64), (100, torch.complex64), (2800, torch.complex64),
                                     (4100, torch.complex64), (96, torch.complex128), (150, torch.complex128),
                                     (1050, torch.complex128)])
def test_centred_dft_mixed(ctx, n, dtype):
    """Radices 16/8/4/2 with 3, 5, 7 and the prime 41 (4100); 150 and 1050 have an odd N/2."""
    batch = 2 if n <= 1050 else 1
    f = inputs.random_field((batch, n, n), seed=n)
    x = to_dev(f, dtype)
    coro.fft2(ctx, x, -1)
    assert rel_l2(x.cpu().numpy(), propagation.centred_dft2(f)) < TOL[dtype]
    coro.fft2(ctx, x, +1)
    assert rel_l2(x.cpu().numpy(), f) < TOL[dtype]


@pytest.mark.parametrize("n,dtype", [(2800, torch.complex64), (1050, torch.complex128)])
def test_angular_spectrum_mixed(ctx, n, dtype):
    dx, lam, z = 2.0 / n, 600e-9, 1.5
    f = inputs.random_field((1, n, n), seed=3)
    x = to_dev(f, dtype)
    coro.propagate_fresnel(ctx, x, dx, lam, z, coro.FRESNEL_AS)
    assert rel_l2(x.cpu().numpy()[0], propagation.angular_spectrum(f[0], dx, lam, z)) < TOL[dtype]


def test_relay_plan_2800(ctx):
    """The six-plane relay at N = 2800 (npix 700) through the fused plan: every pass is a
    mixed-radix kernel, elements (obscured spidered aperture, lenses, PSD surfaces, field
    stop) applied inside the row passes."""
    n, npix = 2800, 700
    w = inputs.RelayWorkload(n=n, npix=npix, seed=5)
    maps = [m.astype(np.float32) for m in w.psd_maps()]
    maps_t = [torch.from_numpy(m).cuda() for m in maps]
    r = w.diam_m / 2
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=r, obscuration=w.obscuration, n_spiders=w.n_spiders,
                        spider_width=w.spider_width_frac * w.diam_m),
           coro.element(coro.EL_LENS, plane=1, focal_length=w.lens1_m),
           coro.element(coro.EL_OPD_MAP, plane=2, opd=maps_t[0]),
           coro.element(coro.EL_LENS, plane=3, focal_length=w.lens2_m),
           coro.element(coro.EL_OPD_MAP, plane=4, opd=maps_t[1]),
           coro.element(coro.EL_CIRCLE, plane=5, radius=w.field_stop_frac * r)]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=els, init_uniform=True)
    assert plan.launch_count == 11
    assert all("_mixed" in plan.pass_kernel(i) for i in range(plan.launch_count))
    assert all(plan.pass_radix(i) == [16, 5, 5, 7] for i in range(plan.launch_count))   # 2800 = 16 x 5 x 5 x 7
    x = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    plan.execute(x)
    lam, dx = w.wavelength_m, w.dx
    oels = [optics.circular_aperture(n, dx, r, w.obscuration, w.n_spiders, w.spider_width_frac * w.diam_m),
            optics.thin_lens(n, dx, lam, w.lens1_m), optics.phasor(maps[0], lam),
            optics.thin_lens(n, dx, lam, w.lens2_m), optics.phasor(maps[1], lam),
            optics.circle_stop(n, dx, w.field_stop_frac * r)]
    ref = propagation.fresnel_chain(np.ones((n, n), complex), dx, lam, oels, list(w.distances()))
    assert rel_l2(x.cpu().numpy()[0], ref) < 1e-5
    # every kernel the tuner chooses from: the shared-memory engine's column widths, 4 columns
    # per 1024-thread block (alone on its SM) and 2 per 512-thread block (two per SM), and the
    # packed-pair engine's row and column kernels (compile-time radix plan, in place)
    kernels = set()
    for rv, cl in ((0, 4), (0, 2), (6, -5), (6, 4), (0, -5)):
        plan.set_pass_kernel(rv, cl)
        kernels |= {plan.pass_kernel(i) for i in range(plan.launch_count)}
        assert all(plan.pass_radix(i) == [16, 5, 5, 7] for i in range(plan.launch_count))
        x.fill_(float("nan"))
        plan.execute(x)
        assert rel_l2(x.cpu().numpy()[0], ref) < 1e-5, (rv, cl)
    assert kernels == {"col_pass_mixed<2800,4>", "col_pass_mixed<2800,2>", "row_pass_mixed<2800>",
                       "col_pass_mixed_pair<2800,2>", "row_pass_mixed_pair<2800>"}
    with pytest.raises(coro.CoroError):
        plan.set_pass_kernel(0, 8)


def test_mixed_pair_engine_4100_both_engines(ctx):
    """N = 4100 = 4 x 5 x 5 x 41 (App. B's npix 1025 x 4): an angular-spectrum hop on the
    packed-pair engine (its default; the prime 41 as an in-place last stage) and on the
    shared-memory engine, against the oracle."""
    n, dx, lam, z = 4100, 2.0 / 4100, 600e-9, 1.5
    f = inputs.random_field((1, n, n), seed=11)
    ref = propagation.angular_spectrum(f[0], dx, lam, z)
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=dx, wavelength=np.array([lam]), distances=[z],
                            methods=[coro.FRESNEL_AS], elements=[])
    seen = set()
    for rv, cl in ((6, -5), (0, 2)):
        plan.set_pass_kernel(rv, cl)
        seen |= {plan.pass_kernel(i) for i in range(plan.launch_count)}
        assert all(plan.pass_radix(i) == [4, 5, 5, 41] for i in range(plan.launch_count))
        x = to_dev(f, torch.complex64)
        plan.execute(x)
        assert rel_l2(x.cpu().numpy()[0], ref) < 1e-5, (rv, cl)
    assert {"row_pass_mixed_pair<4100>", "col_pass_mixed_pair<4100,2>"} <= seen


@pytest.mark.parametrize("n,npix", [(1400, 350), (2800, 700)])
def test_mixed_pair_engine_direct_and_as_hops(ctx, n, npix):
    """The packed-pair mixed-radix kernels (row variant 6, column kernel -5) on a direct hop
    (forward-only column pass) and an angular-spectrum hop on two wavelengths, batch 2, against
    the oracle; 1400 = 8 x 5 x 5 x 7 has a radix-8 stage, 2800 = 16 x 5 x 5 x 7 a radix-16 one."""
    dx = 1.0 / npix
    lams = np.array([500e-9, 600e-9])
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=0.5, obscuration=0.1, n_spiders=4, spider_width=0.02),
           coro.element(coro.EL_LENS, plane=0, focal_length=10.0),
           coro.element(coro.EL_CIRCLE, plane=1, radius=40e-6, flags=coro.ELF_OPAQUE_INSIDE)]
    plan = coro.FresnelPlan(ctx, n=n, batch=2, pixelscale=dx, wavelength=lams, distances=[10.0, 0.05],
                            methods=[coro.FRESNEL_DIRECT, coro.FRESNEL_AS], elements=els, init_uniform=True)
    plan.set_pass_kernel(6, -5)
    names = {plan.pass_kernel(i) for i in range(plan.launch_count)}
    assert names == {f"row_pass_mixed_pair<{n}>", f"col_pass_mixed_pair<{n},2>"}
    x = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    ps = plan.execute(x)
    got = x.cpu().numpy()
    for b in range(2):
        e = optics.circular_aperture(n, dx, 0.5, 0.1, 4, 0.02) * optics.thin_lens(n, dx, lams[b], 10.0)
        e, du = propagation.direct_fresnel(e, dx, lams[b], 10.0)
        e = e * optics.circle_stop(n, du, 40e-6, opaque_inside=True)
        e = propagation.angular_spectrum(e, du, lams[b], 0.05)
        assert abs(ps[b] - du) < 1e-15 * du
        assert rel_l2(got[b], e) < 1e-5


def test_direct_hop_mixed_two_wavelengths(ctx):
    """Lens, direct hop to focus (new pixel scale per item), focal stop, angular-spectrum
    hop, at N = 1100 (4 x 25 x 11) on two wavelengths."""
    n, npix = 1100, 440
    dx = 1.0 / npix
    lams = np.array([500e-9, 600e-9])
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=0.5),
           coro.element(coro.EL_LENS, plane=0, focal_length=10.0),
           coro.element(coro.EL_CIRCLE, plane=1, radius=40e-6, flags=coro.ELF_OPAQUE_INSIDE)]
    plan = coro.FresnelPlan(ctx, n=n, batch=2, pixelscale=dx, wavelength=lams, distances=[10.0, 0.05],
                            methods=[coro.FRESNEL_DIRECT, coro.FRESNEL_AS], elements=els, init_uniform=True)
    x = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    ps = plan.execute(x)
    got = x.cpu().numpy()
    for b in range(2):
        e = optics.circular_aperture(n, dx, 0.5) * optics.thin_lens(n, dx, lams[b], 10.0)
        e, du = propagation.direct_fresnel(e, dx, lams[b], 10.0)
        e = e * optics.circle_stop(n, du, 40e-6, opaque_inside=True)
        e = propagation.angular_spectrum(e, du, lams[b], 0.05)
        assert abs(ps[b] - du) < 1e-15 * du
        assert rel_l2(got[b], e) < 1e-5


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_zernike_and_sine_elements_mixed(ctx, dtype):
    n, dx, lam = 300, 1.0 / 250, 550e-9
    c = inputs.zernike_coefficients(3, 4, 21, 50e-9)
    f = inputs.random_field((1, n, n), seed=4)
    x = to_dev(f, dtype)
    coro.apply_element(ctx, x, dx, lam, coro.element(coro.EL_ZERNIKE, radius=0.5, coeffs=c, j_first=4))
    coro.apply_element(ctx, x, dx, lam, coro.element(coro.EL_SINE, sine_freq=40.0, sine_amplitude=5e-9, axis=0))
    ref = f[0] * optics.phasor(optics.zernike_opd(n, dx, 0.5, c, 4), lam) \
        * optics.phasor(optics.sine_wfe(n, dx, 40.0, 5e-9, axis=1), lam)
    assert rel_l2(x.cpu().numpy()[0], ref) < (1e-6 if dtype == torch.complex64 else TOL[dtype])


@pytest.mark.parametrize("n", [101, 134, 8200])
def test_unsupported_lengths_rejected(ctx, n):
    """Odd N, a prime factor above 61 (134 = 2 x 67) and N above 8192 are refused on the host
    with CORO_ESIZE before any launch."""
    x = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
    with pytest.raises(RuntimeError):
        coro.fft2(ctx, x, -1)
