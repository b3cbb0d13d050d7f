"""Pins of the oracle's pilot-beam Fresnel system (automatic angular-spectrum / direct hops,
Sec. 1.1 citing Lawrence's method) and of the direct hop for z < 0 (CPU only)."""
import numpy as np
import pytest

from oracle import optics, propagation


def gaussian(n, pitch, wavelength, q):
    """exp(i pi r^2 / (lambda q)): a Gaussian beam under the kernel exp(+i pi r^2/(lambda z))
    (q = z - z_waist - i pi w0^2 / lambda)."""
    r2 = optics.radius_sq_exact(n, pitch)
    return np.exp(1j * np.pi * r2 / (wavelength * q))


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_direct_hop_round_trip_negative_z():
    """Direct hop by z then by -z (the inverse DFT on the natural grid) is the identity."""
    n, dx, lam, z = 128, 2e-5, 633e-9, 0.37
    rng = np.random.default_rng(3)
    e = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) * optics.circular_aperture(n, dx, 0.3 * n * dx)
    e1, du = propagation.direct_fresnel(e, dx, lam, z)
    e2, dx2 = propagation.direct_fresnel(e1, du, lam, -z)
    assert abs(dx2 - dx) < 1e-15 * dx
    assert rel_l2(e2, e) < 1e-12


def test_direct_hop_negative_z_is_gaussian_backwards():
    """A Gaussian beam propagated backwards by a direct hop matches the closed form on the
    natural (non-mirrored) grid: checked with an off-axis tilt, which a mirrored grid fails."""
    n, lam = 256, 1e-6
    w0, dx = 1e-3, 5e-5
    q0 = complex(0.0, -np.pi * w0 ** 2 / lam)
    x, _ = optics.grid(n, dx)
    tilt = np.exp(2j * np.pi * x * 2000.0)                 # 2000 cycles/m along x
    z = -0.8
    e1, du = propagation.direct_fresnel(gaussian(n, dx, lam, q0) * tilt, dx, lam, z)
    u, v = optics.grid(n, du)
    # Fresnel diffraction of a tilted Gaussian: the beam walks by lambda z f_x and keeps the tilt
    shift = lam * z * 2000.0
    qz = q0 + z
    ref = (q0 / qz) * np.exp(1j * np.pi * ((u - shift) ** 2 + v ** 2) / (lam * qz)) \
        * np.exp(2j * np.pi * 2000.0 * u) * np.exp(-1j * np.pi * lam * z * 2000.0 ** 2)
    assert rel_l2(e1, ref) < 1e-9


def pilot_gaussian_system():
    n, lam, w0 = 256, 1e-6, 1e-3
    dx = w0 / 20
    planes = [[("lens", 0.5)], [], [], []]
    distances = [0.5, 0.3, 0.2]
    return n, lam, w0, dx, planes, distances


def test_pilot_system_gaussian_closed_form():
    """A Gaussian beam through a lens, across its focus and beyond: the pilot-beam system
    (outside -> inside -> outside -> outside, including a backward leg) reproduces the closed
    form A exp(i pi r^2/(lambda q)) with q += d, 1/q -= 1/f, A *= q/(q + d)."""
    n, lam, w0, dx, planes, distances = pilot_gaussian_system()
    q = complex(0.0, -np.pi * w0 ** 2 / lam)
    e0 = gaussian(n, dx, lam, q)
    for k in range(1, len(planes) + 1):
        got, pitch, flags, legs = propagation.fresnel_system_pilot(e0, dx, lam, w0, planes[:k], distances[:k - 1])
        qq, amp = q, 1.0 + 0j
        qq = 1.0 / (1.0 / qq - 1.0 / 0.5)
        for d in distances[:k - 1]:
            amp *= qq / (qq + d)
            qq = qq + d
        ref = amp * gaussian(n, pitch, lam, qq)
        assert rel_l2(got, ref) < 1e-9, (k, rel_l2(got, ref))
    assert flags == [True, False, True, True] and legs == 4


def test_pilot_system_energy():
    """Every hop (angular spectrum and both direct legs) conserves sum |E|^2 pitch^2."""
    n, lam, w0, dx, planes, distances = pilot_gaussian_system()
    rng = np.random.default_rng(5)
    e0 = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) * optics.circular_aperture(n, dx, 8 * dx)
    e0 = e0 * gaussian(n, dx, lam, complex(0, -np.pi * (4 * dx) ** 2 / lam))
    got, pitch, _, _ = propagation.fresnel_system_pilot(e0, dx, lam, w0, planes, distances)
    e_in = np.sum(np.abs(e0) ** 2) * dx * dx
    e_out = np.sum(np.abs(got) ** 2) * pitch * pitch
    assert abs(e_out / e_in - 1) < 1e-12


def test_pilot_system_all_inside_is_plain_angular_spectrum():
    """A beam that never leaves its Rayleigh range: the system is a plain angular-spectrum
    chain at constant pitch."""
    n, lam, dx = 128, 550e-9, 1e-4
    w0 = 40 * dx                                           # z_R = 93 m
    rng = np.random.default_rng(7)
    opd = rng.normal(size=(n, n)) * 20e-9
    aperture = lambda nn, p: optics.circular_aperture(nn, p, 30 * dx)
    phase = lambda nn, p: optics.phasor(opd, lam)
    planes = [[aperture], [phase], []]
    distances = [3.0, 5.0]
    e0 = np.ones((n, n), complex)
    got, pitch, flags, legs = propagation.fresnel_system_pilot(e0, dx, lam, w0, planes, distances)
    ref = propagation.angular_spectrum(e0 * aperture(n, dx), dx, lam, 3.0)
    ref = propagation.angular_spectrum(ref * phase(n, dx), dx, lam, 5.0)
    assert pitch == dx and flags == [False, False, False] and legs == 0
    assert rel_l2(got, ref) < 1e-13


@pytest.mark.parametrize("npix", [64, 128])
def test_pilot_system_airy_at_focus(npix):
    """Circular aperture behind a lens, observed at the focal plane through the pilot-beam
    system (a direct leg): intensity vs (2 J1(v)/v)^2 to the pixelated-disk level."""
    from scipy.special import j1
    n, lam, f, diam = 4 * npix, 500e-9, 10.0, 1.0
    dx = diam / npix
    planes = [[lambda nn, p: optics.circular_aperture(nn, p, diam / 2), ("lens", f)], []]
    got, pitch, flags, legs = propagation.fresnel_system_pilot(np.ones((n, n), complex), dx, lam, diam / 2,
                                                               planes, [f])
    assert legs >= 1 and flags[1] is False
    i = np.abs(got) ** 2
    i /= i.max()
    x, y = optics.grid(n, pitch)
    v = np.pi * diam * np.hypot(x, y) / (lam * f)
    airy = np.where(v > 0, (2 * j1(np.where(v > 0, v, 1)) / np.where(v > 0, v, 1)) ** 2, 1.0)
    core = v < 10
    assert np.max(np.abs(i[core] - airy[core])) < (3e-3 if npix == 128 else 6e-3)
