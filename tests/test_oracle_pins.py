"""Pins for the FP64 oracle: each test checks the oracle against something other than
itself -- a brute-force sum, a closed form, an invariant, or a textbook special case --
so that a dropped term, a wrong sign or a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import coronagraph, optics, propagation
from paper_1806_06467_gb300 import inputs


# ----------------------------------------------------------------------------- centred DFT

def brute_centred_dft2(f):
    n0, n1 = f.shape
    out = np.zeros_like(f, dtype=np.complex128)
    for k0 in range(n0):
        for k1 in range(n1):
            acc = 0j
            for j0 in range(n0):
                for j1 in range(n1):
                    acc += f[j0, j1] * np.exp(-2j * np.pi * ((j0 - n0 // 2) * (k0 - n0 // 2) / n0
                                                             + (j1 - n1 // 2) * (k1 - n1 // 2) / n1))
            out[k0, k1] = acc
    return out


@pytest.mark.parametrize("n", [4, 8, 16, 12, 18, 30])
def test_centred_dft_matches_brute_force(n):
    """Powers of two and the lengths of the mixed-radix passes (12 = 4 x 3; 18 and 30 have an
    odd N/2, where the per-axis sign (-1)^(N/2) of the checkerboard centring is -1)."""
    f = inputs.random_field((n, n), seed=n)
    np.testing.assert_allclose(propagation.centred_dft2(f), brute_centred_dft2(f),
                               rtol=0, atol=1e-12 * n * n)
    back = propagation.centred_idft2(propagation.centred_dft2(f))
    np.testing.assert_allclose(back, f, rtol=0, atol=1e-13)


def test_centred_dft_impulse_closed_forms():
    n = 32
    f = np.zeros((n, n), complex)
    f[n // 2, n // 2] = 1.0                      # impulse on the axis -> constant spectrum
    np.testing.assert_allclose(propagation.centred_dft2(f), np.ones((n, n)), atol=1e-14)
    f[:] = 0
    f[n // 2, n // 2 + 3] = 1.0                  # offset impulse -> linear phase along x
    k = np.arange(n) - n // 2
    expect = np.exp(-2j * np.pi * 3 * k / n)[None, :].repeat(n, 0)
    np.testing.assert_allclose(propagation.centred_dft2(f), expect, atol=1e-13)


def test_parseval():
    f = inputs.random_field((64, 64), seed=3)
    e0 = np.sum(np.abs(f) ** 2)
    e1 = np.sum(np.abs(propagation.centred_dft2(f)) ** 2) / 64 ** 2
    assert abs(e1 / e0 - 1) < 1e-13
    g = propagation.angular_spectrum(f, 1e-3, 550e-9, 2.3)
    assert abs(np.sum(np.abs(g) ** 2) / e0 - 1) < 1e-12


# ----------------------------------------------------------------------------- angular spectrum

@pytest.mark.parametrize("z_over_zr", [0.3, 1.0, 2.0])
def test_gaussian_beam_closed_form(z_over_zr):
    """exp(-r^2/w0^2) under the paraxial transfer function is the textbook Gaussian beam
    1/(1 + i z/zR) exp(-r^2 / (w0^2 (1 + i z/zR))): waist growth w(z), Gouy phase and
    curvature all follow."""
    n, dx, lam = 256, 1e-3, 633e-9
    w0 = 10 * dx
    zr = np.pi * w0 ** 2 / lam
    z = z_over_zr * zr
    x, y = optics.grid(n, dx)
    r2 = x * x + y * y
    e = propagation.angular_spectrum(np.exp(-r2 / w0 ** 2).astype(complex), dx, lam, z)
    q = 1 + 1j * z / zr
    expect = np.exp(-r2 / (w0 ** 2 * q)) / q
    np.testing.assert_allclose(e, expect, rtol=0, atol=1e-12)
    centre = e[n // 2, n // 2]
    assert abs(abs(centre) - 1 / math.sqrt(1 + z_over_zr ** 2)) < 1e-12     # w0 / w(z)
    assert abs(np.angle(centre) + math.atan(z_over_zr)) < 1e-12             # Gouy phase


def test_round_trip_identity():
    f = inputs.random_field((64, 64), seed=5)
    g = propagation.angular_spectrum(propagation.angular_spectrum(f, 2e-4, 550e-9, 1.7),
                                     2e-4, 550e-9, -1.7)
    np.testing.assert_allclose(g, f, atol=1e-12)
    lens = optics.thin_lens(64, 2e-4, 550e-9, 3.0) * optics.thin_lens(64, 2e-4, 550e-9, -3.0)
    np.testing.assert_allclose(lens, np.ones((64, 64)), atol=1e-12)


def talbot_closed_form(x, a, nu, lam, z, nmax=12):
    """exp(i a sin(2 pi nu x)) = sum_n J_n(a) exp(i n 2 pi nu x) (Jacobi-Anger); each
    harmonic picks up exp(-i pi lambda z (n nu)^2) under the paraxial transfer function."""
    out = np.zeros_like(x, dtype=np.complex128)
    for nn in range(-nmax, nmax + 1):
        out += sp.jv(nn, a) * np.exp(1j * nn * 2 * np.pi * nu * x - 1j * np.pi * lam * z * (nn * nu) ** 2)
    return out


def test_talbot_app_a():
    """App. A: beam radius 2 cm, 0.5 um, npix 256 x oversample 8, 5 nm sine at 500 /m.
    Z_T = 2 p^2 / lambda with p = 1/nu (Eq. 1 read with D/f as the grating period); at
    Z_T/4 the phase grating has become a pure amplitude grating (Fig. 1)."""
    lam, nu, amp = 0.5e-6, 500.0, 5e-9
    diam = 2 * 0.02
    npix, over = 256, 8
    n = npix * over
    dx = diam / npix
    assert abs(n * dx * nu - round(n * dx * nu)) < 1e-9      # 160 whole periods on the grid
    zt = 2 * (1 / nu) ** 2 / lam
    opd = optics.sine_wfe(n, dx, nu, amp)
    e0 = optics.phasor(opd, lam)
    a = 2 * np.pi * amp / lam
    x = optics.coords(n, dx)
    for frac in (0.05, 0.25):
        e = propagation.angular_spectrum(e0, dx, lam, frac * zt)
        expect = talbot_closed_form(x, a, nu, lam, frac * zt)
        np.testing.assert_allclose(e[n // 3], expect, rtol=0, atol=1e-12)
        np.testing.assert_allclose(e[7], expect, rtol=0, atol=1e-12)
    # complete phase-to-amplitude conversion at Z_T/4
    e = propagation.angular_spectrum(e0, dx, lam, 0.25 * zt)[0]
    assert np.max(np.abs(np.angle(e))) < 1e-3 * a
    assert abs((np.abs(e).max() - np.abs(e).min()) / 2 - a) < 0.01 * a


# ----------------------------------------------------------------------------- direct Fresnel

def test_direct_fresnel_matches_brute_force_integral():
    """Q_out . DFT . Q_in with du = lambda z/(N dx) equals the Fresnel convolution integral
    (1/(i lambda z)) sum_x E(x) exp(i pi |u - x|^2 / (lambda z)) dx^2 evaluated directly."""
    n, dx, lam, z = 12, 3e-4, 600e-9, 0.8
    f = inputs.random_field((n, n), seed=11)
    out, du = propagation.direct_fresnel(f, dx, lam, z)
    x = optics.coords(n, dx)
    u = optics.coords(n, du)
    brute = np.zeros((n, n), complex)
    for iv in range(n):
        for iu in range(n):
            d2 = (u[iu] - x[None, :]) ** 2 + (u[iv] - x[:, None]) ** 2
            brute[iv, iu] = np.sum(f * np.exp(1j * np.pi * d2 / (lam * z))) * dx * dx / (1j * lam * z)
    np.testing.assert_allclose(out, brute, rtol=1e-11, atol=1e-11 * np.abs(brute).max())


def test_direct_fresnel_energy():
    f = inputs.random_field((64, 64), seed=2)
    dx = 1e-3
    out, du = propagation.direct_fresnel(f, dx, 550e-9, 3.0)
    assert abs(np.sum(np.abs(out) ** 2) * du * du / (np.sum(np.abs(f) ** 2) * dx * dx) - 1) < 1e-12


def airy(rho):
    v = np.pi * np.asarray(rho, dtype=float)
    out = np.ones_like(v)
    nz = v != 0
    out[nz] = (2 * sp.j1(v[nz]) / v[nz]) ** 2
    return out


def airy_focal_fields(npix):
    n = 2 * npix
    diam, lam, f = 1.0, 500e-9, 10.0
    dx = diam / npix
    e = optics.circular_aperture(n, dx, diam / 2).astype(complex)
    e = e * optics.thin_lens(n, dx, lam, f)
    foc, du = propagation.direct_fresnel(e, dx, lam, f)
    pupil = optics.circular_aperture(n, dx, diam / 2).astype(complex)
    det = propagation.mft(pupil, npix, 64, 0.5)
    return foc, du, det, lam * f / diam


@pytest.mark.parametrize("npix", [64, 128])
def test_airy_pattern(npix):
    """Lens f = 10 m then direct Fresnel 10 m lands on focus at 0.5 lambda/D per pixel, and
    the MFT to 64^2 at 0.5 lambda/D sees the same plane; both follow (2 J1(pi rho)/(pi rho))^2
    up to the pixelation of the disk."""
    foc, du, det, lamd = airy_focal_fields(npix)
    n = foc.shape[0]
    assert abs(du / lamd - 0.5) < 1e-12
    ifoc = np.abs(foc) ** 2
    ifoc /= ifoc.max()
    x, y = optics.grid(n, du / lamd)
    err_f = np.max(np.abs(ifoc - airy(np.hypot(x, y))))
    idet = np.abs(det) ** 2
    idet /= idet.max()
    xd, yd = optics.grid(64, 0.5)
    err_m = np.max(np.abs(idet - airy(np.hypot(xd, yd))))
    bound = 3e-3 if npix == 128 else 8e-3
    assert err_f < bound and err_m < bound
    # the two routes agree on the shared 64 x 64 pixels (same sampling, same centre)
    c = n // 2
    sub = ifoc[c - 32:c + 32, c - 32:c + 32]
    np.testing.assert_allclose(sub, idet, atol=1e-12)


def test_airy_error_falls_with_sampling():
    errs = []
    for npix in (32, 64, 128):
        foc, du, det, lamd = airy_focal_fields(npix)
        i = np.abs(det) ** 2
        i /= i.max()
        xd, yd = optics.grid(64, 0.5)
        errs.append(np.max(np.abs(i - airy(np.hypot(xd, yd)))))
    assert errs[0] > errs[1] > errs[2]


# ----------------------------------------------------------------------------- MFT

@pytest.mark.parametrize("n,npix", [(16, 16), (32, 16), (24, 12)])
def test_mft_complete_grid_is_centred_dft(n, npix):
    """With M = N and dU = npix/N the MFT is the unitary-scaled centred DFT."""
    f = inputs.random_field((n, n), seed=n)
    du = npix / n
    np.testing.assert_allclose(propagation.mft(f, npix, n, du),
                               propagation.centred_dft2(f) / n, atol=1e-12)
    np.testing.assert_allclose(propagation.imft(propagation.mft(f, npix, n, du), npix, n, du),
                               f, atol=1e-12)
    e0 = np.sum(np.abs(f) ** 2)
    assert abs(np.sum(np.abs(propagation.mft(f, npix, n, du)) ** 2) / e0 - 1) < 1e-12


def test_mft_shift_theorem():
    """A pupil tilt of k cycles across D moves the focal field by k lambda/D."""
    n, npix, m, du, k = 32, 32, 40, 0.25, 2
    f = inputs.random_field((n, n), seed=9)
    xx, _ = optics.grid(n, 1.0 / npix)
    tilted = propagation.mft(f * np.exp(2j * np.pi * k * xx), npix, m, du)
    plain = propagation.mft(f, npix, m + 2 * int(k / du), du)
    s = int(k / du)
    np.testing.assert_allclose(tilted, plain[s:s + m, :m], atol=1e-12)


# ----------------------------------------------------------------------------- Lyot chain

def small_lyot(n=32, m_occ=24, du_occ=0.25, spot=2.0, lyot=0.8, m_det=40, du_det=0.5):
    return coronagraph.LyotParams(n=n, npix=n, m_occ=m_occ, du_occ=du_occ, spot_radius=spot,
                                  lyot_frac=lyot, m_det=m_det, du_det=du_det)


def test_lyot_without_spot_is_plain_mft():
    p = small_lyot(spot=-1.0, lyot=2.0)
    e = inputs.random_field((32, 32), seed=4)
    out = coronagraph.lyot_fields(e, p)["det"]
    np.testing.assert_allclose(out, propagation.mft(e, 32, 40, 0.5), atol=1e-12)


def test_lyot_full_spot_on_complete_grid_is_dark():
    """If the occulter plane is the complete grid and the spot covers all of it, Babinet
    subtracts the whole field: E_C = 0."""
    n = 16
    p = coronagraph.LyotParams(n=n, npix=n, m_occ=n, du_occ=1.0, spot_radius=100.0,
                               lyot_frac=2.0, m_det=8, du_det=0.5)
    e = inputs.random_field((n, n), seed=6)
    np.testing.assert_allclose(coronagraph.lyot_fields(e, p)["C"], 0, atol=1e-12)


def test_lyot_psf_symmetry_and_positivity():
    p = small_lyot(n=64, m_occ=32, du_occ=0.25, spot=3.0, m_det=64, du_det=0.5)
    # radius just under D/2 so that every lit pixel has its mirror image on the grid
    e = coronagraph.pupil_field(64, 64, 550e-9, None, radius_frac=0.98)
    i, s, peak = coronagraph.lyot_psf(e, p, 4.0, 12.0)
    assert s >= 0 and peak > 0
    core = i[1:, 1:]
    np.testing.assert_allclose(core, core[::-1, :], atol=1e-14)
    np.testing.assert_allclose(core, core.T, atol=1e-14)
    # the coronagraph removes most of the on-axis light
    assert i.max() < 0.1


# ----------------------------------------------------------------------------- elements

def test_noll_table():
    """Noll (1976) Table 1 ordering for j = 1..21, read from a golden text fixture."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "noll_1976_nm.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for j, n, m in ((int(a), int(b), int(c)) for a, b, c in rows):
        assert optics.noll_to_nm(j) == (n, m), j


def test_zernike_orthonormal_on_fine_disk():
    n = 1024
    x, y = optics.grid(n, 2.0 / n)
    rho = np.hypot(x, y)
    th = np.arctan2(y, x)
    inside = rho <= 1.0
    zs = np.stack([optics.zernike_noll(j, rho, th)[inside] for j in range(1, 22)])
    gram = zs @ zs.T / inside.sum()
    np.testing.assert_allclose(gram, np.eye(21), atol=1e-2)


def test_dm_influence_fwhm_and_linearity():
    n, dx, n_act = 512, 1.0 / 400, 8
    pitch = 1.0 / n_act
    h = np.zeros((n_act, n_act))
    h[3, 4] = 1.0
    s = optics.dm_surface(n, dx, h, pitch)
    xa = (4 - (n_act - 1) / 2) * pitch
    ya = (3 - (n_act - 1) / 2) * pitch
    # the surface is the product of two 1-D Gaussians of FWHM = pitch centred on the actuator
    xs = np.linspace(-pitch, pitch, 4001)
    sigma = pitch / (2 * math.sqrt(2 * math.log(2)))
    half = xs[np.exp(-xs ** 2 / (2 * sigma ** 2)) >= 0.5]
    assert abs((half.max() - half.min()) - pitch) < 1e-3 * pitch
    gm = optics.dm_influence_matrix(n, dx, n_act, pitch)
    jx = np.argmax(gm[:, 4])
    assert abs(optics.coords(n, dx)[jx] - xa) <= dx / 2
    assert abs(s.max() - gm[:, 3].max() * gm[:, 4].max()) < 1e-14
    h2 = inputs.dm_heights(1, n_act, 1)[0]
    np.testing.assert_allclose(optics.dm_surface(n, dx, h + 2 * h2, pitch),
                               s + 2 * optics.dm_surface(n, dx, h2, pitch), atol=1e-15)
    assert abs(ya) > 0


def test_aperture_geometry():
    n, dx = 256, 1.0 / 200
    a = optics.circular_aperture(n, dx, 0.5, obscuration=0.3, n_spiders=4, spider_width=0.01)
    x, y = optics.grid(n, dx)
    r = np.hypot(x, y)
    assert np.all(a[r > 0.5] == 0)
    assert np.all(a[r < 0.15] == 0)
    assert np.all(a[(np.abs(x) < 0.005) | (np.abs(y) < 0.005)] == 0)
    clear = (r <= 0.5) & (r >= 0.15) & (np.abs(x) >= 0.005) & (np.abs(y) >= 0.005)
    assert np.all(a[clear] == 1)
    area = a.sum() * dx * dx
    expect = np.pi * (0.25 - 0.15 ** 2) - 4 * 0.01 * (0.5 - 0.15)
    assert abs(area / expect - 1) < 0.02


# ----------------------------------------------------------------------------- detector masks and normalisation

def lattice_count(r2: int) -> int:
    """Gauss circle count #{(i, j) in Z^2 : i^2 + j^2 <= r2}, row by row with integer square roots."""
    r = math.isqrt(r2)
    return sum(2 * math.isqrt(r2 - i * i) + 1 for i in range(-r, r + 1))


def test_dark_hole_sum_counts_the_annulus():
    """At 0.25 lambda/D per pixel the 6-20 lambda/D annulus is 24 <= |(i', j')| <= 80 pixels, both
    bounds inclusive (reading S7): a unit intensity sums to the lattice-point count, and r^2 as
    the intensity to the integer sum of i'^2 + j'^2 over those points."""
    m, du = 512, 0.25
    s = coronagraph.dark_hole_sum(np.ones((m, m)), du, 6.0, 20.0)
    assert s == lattice_count(80 * 80) - lattice_count(24 * 24 - 1)
    assert abs(s / (math.pi * (80 ** 2 - 24 ** 2)) - 1) < 1e-3      # the annulus area in pixels
    k = np.arange(m) - m // 2
    r2 = (k[None, :] ** 2 + k[:, None] ** 2).astype(float)
    brute = sum(i * i + j * j for i in range(-80, 81) for j in range(-80, 81)
                if 576 <= i * i + j * j <= 6400)
    assert coronagraph.dark_hole_sum(r2, du, 6.0, 20.0) == brute


def test_lyot_stop_radius_is_half_frac_of_d():
    """lyot_frac is a fraction of the pupil DIAMETER's half: at npix = 128 and frac = 0.75 the
    stop passes |(i', j')| <= 48 pixels."""
    stop = coronagraph.lyot_stop(160, 128, 0.75)
    assert stop.sum() == lattice_count(48 * 48)
    assert stop[80, 80 + 48] == 1 and stop[80, 80 + 49] == 0


@pytest.mark.parametrize("lyot_frac,r_px", [(1.0, 32), (0.75, 24)])
def test_peak_intensity_of_clear_disk(lyot_frac, r_px):
    """Without the occulter the on-axis detector field is s * (sum of the lit pupil samples), every
    phase factor being 1 at U = 0, and no pixel can exceed it: peak = (dU/npix * N_lit)^2."""
    n, npix = 80, 64
    p = coronagraph.LyotParams(n=n, npix=npix, m_occ=32, du_occ=0.25, spot_radius=2.0,
                               lyot_frac=lyot_frac, m_det=48, du_det=0.5)
    e = coronagraph.pupil_field(n, npix, 550e-9, None)
    n_lit = lattice_count(r_px * r_px)
    assert abs(coronagraph.peak_intensity(e, p) / (0.5 / npix * n_lit) ** 2 - 1) < 1e-13


# ----------------------------------------------------------------------------- Zernike OPD maps

# Noll (1976) Table 1, unit-RMS forms written out (rho = r/R, theta from +x towards +y)
NOLL_CLOSED = {
    4: lambda r, t: math.sqrt(3) * (2 * r ** 2 - 1),
    5: lambda r, t: math.sqrt(6) * r ** 2 * np.sin(2 * t),
    6: lambda r, t: math.sqrt(6) * r ** 2 * np.cos(2 * t),
    7: lambda r, t: math.sqrt(8) * (3 * r ** 3 - 2 * r) * np.sin(t),
    8: lambda r, t: math.sqrt(8) * (3 * r ** 3 - 2 * r) * np.cos(t),
    11: lambda r, t: math.sqrt(5) * (6 * r ** 4 - 6 * r ** 2 + 1),
}


@pytest.mark.parametrize("j", sorted(NOLL_CLOSED))
def test_zernike_opd_single_term_closed_form(j):
    """One coefficient: c Z_j(r/R, theta) inside r <= R (R = 0.37 m on a 1 cm grid, so rho is not
    a grid ratio), exactly zero outside."""
    n, dx, radius, c = 96, 0.01, 0.37, 3e-9
    opd = optics.zernike_opd(n, dx, radius, np.array([c]), j)
    for (iy, ix) in [(48, 48), (48, 70), (20, 55), (60, 31), (75, 70), (48, 48 + 37)]:
        x, y = (ix - 48) * dx, (iy - 48) * dx
        r = math.hypot(x, y)
        expect = c * NOLL_CLOSED[j](r / radius, math.atan2(y, x)) if r * r <= radius * radius else 0.0
        assert abs(opd[iy, ix] - expect) < 1e-12 * c, (iy, ix)
    k = np.arange(n) - 48
    outside = (k[None, :] ** 2 + k[:, None] ** 2) * dx * dx > radius * radius
    assert np.all(opd[outside] == 0.0)


def test_zernike_opd_composes_consecutive_terms():
    """Coefficients c_0.. belong to Noll indices j_first, j_first + 1, ...: the map is their sum."""
    n, dx, radius = 64, 0.02, 0.55
    cs = np.array([1e-9, -2e-9, 0.5e-9])
    opd = optics.zernike_opd(n, dx, radius, cs, 5)
    x, y = optics.grid(n, dx)
    r, t = np.hypot(x, y) / radius, np.arctan2(y, x)
    expect = sum(c * NOLL_CLOSED[5 + i](r, t) for i, c in enumerate(cs))
    expect[r > 1] = 0.0
    np.testing.assert_allclose(opd, expect, rtol=0, atol=1e-20)


def test_focal_mask_spot_count():
    """The occulting spot covers rho <= 5 lambda/D inclusive: at 0.25 lambda/D per pixel, the
    lattice points within 20 pixels."""
    spot = coronagraph.focal_mask(64, 0.25, 5.0)
    assert spot.sum() == lattice_count(400)
    assert spot[32, 52] == 1 and spot[32, 53] == 0


def test_fresnel_chain_composes_hops():
    """Transfer functions multiply: bare planes z1 then z2 equal one hop z1 + z2; an element
    applied at a plane acts on the field that arrives there."""
    n, dx, lam = 64, 2e-4, 600e-9
    f = inputs.random_field((n, n), seed=21)
    two = propagation.fresnel_chain(f, dx, lam, [None, None, None], [0.7, 1.1])
    one = propagation.angular_spectrum(f, dx, lam, 1.8)
    np.testing.assert_allclose(two, one, atol=1e-12)
    a = optics.circular_aperture(n, dx, 20 * dx).astype(complex)
    chained = propagation.fresnel_chain(f, dx, lam, [None, a, None], [0.7, 1.1])
    manual = propagation.angular_spectrum(a * propagation.angular_spectrum(f, dx, lam, 0.7), dx, lam, 1.1)
    np.testing.assert_allclose(chained, manual, atol=1e-12)
