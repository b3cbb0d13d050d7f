"""GPU parity: matrix Fourier transform (forward and inverse, batched with per-item sampling)
against the FP64 oracle's direct sums, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import coronagraph, propagation
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu

PRECS = [coro.MFT_FP32]


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.complex128) - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def ctx(lib):
    return coro.Context(0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,npix,m", [(64, 50, 40), (128, 128, 96), (256, 200, 130), (100, 90, 37)])
def test_mft_forward(ctx, n, npix, m, prec):
    du = np.array([0.3, 0.45])
    f = inputs.random_field((2, n, n), seed=n + m)
    x = torch.from_numpy(f.astype(np.complex64)).cuda()
    y = coro.propagate_mft(ctx, x, npix, -1, m, du, prec).cpu().numpy()
    for b in range(2):
        assert rel_l2(y[b], propagation.mft(f[b], npix, m, du[b])) < 1e-5


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m,n,npix", [(40, 64, 50), (130, 256, 200), (37, 100, 90)])
def test_mft_inverse(ctx, m, n, npix, prec):
    du = np.array([0.3, 0.2])
    f = inputs.random_field((2, m, m), seed=m)
    x = torch.from_numpy(f.astype(np.complex64)).cuda()
    y = coro.propagate_mft(ctx, x, npix, +1, n, du, prec).cpu().numpy()
    for b in range(2):
        assert rel_l2(y[b], propagation.imft(f[b], npix, n, du[b])) < 1e-5


def test_mft_lyot_sizes(ctx):
    """1024^2 pupil -> 256^2 at 0.05 lambda/D (the occulter plane of the Lyot workload)."""
    w = inputs.LyotWorkload()
    e = coronagraph.pupil_field(w.n, w.npix, w.wavelength_m, None)
    f = e * inputs.random_field(e.shape, seed=2)
    x = torch.from_numpy(f.astype(np.complex64)).cuda().unsqueeze(0)
    y = coro.propagate_mft(ctx, x, w.npix, -1, w.m_occ, w.du_occ).cpu().numpy()[0]
    assert rel_l2(y, propagation.mft(f, w.npix, w.m_occ, w.du_occ)) < 1e-5


@pytest.mark.parametrize("n,npix,m", [(100, 80.0, 64), (256, 128.0, 75)])
def test_mft_fp64_forward_inverse(ctx, n, npix, m):
    """complex128 fields through the FP64 CUDA-core MFT, two items with different focal
    pitches, against the oracle's direct sums."""
    f = inputs.random_field((2, n, n), seed=n + m)
    du = [0.35, 0.41]
    x = torch.from_numpy(f).cuda()
    y = coro.propagate_mft(ctx, x, npix, -1, m, du)
    assert y.dtype == torch.complex128
    for b in range(2):
        assert rel_l2(y[b].cpu().numpy(), propagation.mft(f[b], npix, m, du[b])) < 1e-12
    back = coro.propagate_mft(ctx, y, npix, +1, n, du)
    for b in range(2):
        ref = propagation.imft(propagation.mft(f[b], npix, m, du[b]), npix, n, du[b])
        assert rel_l2(back[b].cpu().numpy(), ref) < 1e-12
    with pytest.raises(RuntimeError):
        coro.propagate_mft(ctx, x, npix, -1, m, du, precision=coro.MFT_3XTF32)   # FP64 only for complex128


def test_airy_config_fp64_end_to_end(ctx):
    """The plain FP64 configuration: a 128-px clear 1 m aperture on 256^2 complex128, lens
    f = 10 m and direct Fresnel 10 m to focus (0.5 lambda/D per pixel), and the FP64 MFT of the
    pupil to 64^2 at 0.5 lambda/D. Both routes against the oracle (1e-12), against the closed
    form (2 J1(pi rho)/(pi rho))^2 within the pixelation bound of the oracle's own pin (3e-3),
    and against each other on the shared 64 x 64 pixels."""
    import scipy.special as sp
    from oracle import optics
    n, npix, lam, fl = 256, 128, 500e-9, 10.0
    dx = 1.0 / npix
    pupil = optics.circular_aperture(n, dx, 0.5).astype(np.complex128)
    x = torch.from_numpy(pupil).cuda().unsqueeze(0)
    det = coro.propagate_mft(ctx, x, float(npix), -1, 64, [0.5])[0].cpu().numpy()
    ref_det = propagation.mft(pupil, npix, 64, 0.5)
    assert rel_l2(det, ref_det) < 1e-12
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=0.5), coro.element(coro.EL_LENS, plane=0, focal_length=fl)]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=dx, wavelength=lam, distances=[fl],
                            methods=[coro.FRESNEL_DIRECT], elements=els, dtype=coro.C128, init_uniform=True)
    foc = torch.empty((1, n, n), dtype=torch.complex128, device="cuda")
    plan.execute(foc)
    ifoc = np.abs(foc.cpu().numpy()[0]) ** 2
    ifoc /= ifoc.max()
    idet = np.abs(det) ** 2
    idet /= idet.max()

    def airy(rho):
        v = np.pi * rho
        out = np.ones_like(v)
        nz = v != 0
        out[nz] = (2 * sp.j1(v[nz]) / v[nz]) ** 2
        return out

    xd, yd = optics.grid(64, 0.5)
    assert np.max(np.abs(idet - airy(np.hypot(xd, yd)))) < 3e-3
    c = n // 2
    np.testing.assert_allclose(ifoc[c - 32:c + 32, c - 32:c + 32], idet, atol=1e-10)


def test_wavefront_axpy_and_its_checks(ctx):
    """y += alpha x in both dtypes; mismatched shapes or dtypes are refused before any launch."""
    for dt, tol in ((torch.complex64, 1e-6), (torch.complex128, 1e-15)):
        x = torch.from_numpy(inputs.random_field((2, 64, 64), seed=1)).to(dt).cuda()
        y0 = torch.from_numpy(inputs.random_field((2, 64, 64), seed=2)).to(dt).cuda()
        y = coro.wavefront_axpy(ctx, -0.75, x, y0.clone())
        ref = (y0 - 0.75 * x).cpu().numpy()
        assert np.max(np.abs(y.cpu().numpy() - ref)) < tol * np.max(np.abs(ref))
    with pytest.raises(RuntimeError):
        coro.wavefront_axpy(ctx, 1.0, torch.zeros((2, 64, 64), dtype=torch.complex64, device="cuda"),
                            torch.zeros((2, 32, 32), dtype=torch.complex64, device="cuda"))
    with pytest.raises(RuntimeError):
        coro.wavefront_axpy(ctx, 1.0, torch.zeros((1, 64, 64), dtype=torch.complex64, device="cuda"),
                            torch.zeros((1, 64, 64), dtype=torch.complex128, device="cuda"))
