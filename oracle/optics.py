"""Sampling grid and optical elements in FP64 (oracle; test infrastructure only).

Conventions (the paper states none of these; see the readings list in the design notes):
pixel centres are x_j = (j - N/2) dx, so the optical axis sits on pixel N/2; arrays are
[y][x]; masks are binary and sampled at pixel centres (r <= R transmits).
"""
from __future__ import annotations

import math

import numpy as np


def coords(n: int, dx: float) -> np.ndarray:
    """1-D pixel-centre coordinates (j - n/2) * dx."""
    return (np.arange(n, dtype=np.float64) - n // 2) * dx


def grid(n: int, dx: float) -> tuple[np.ndarray, np.ndarray]:
    """2-D coordinate arrays (x, y), each [n][n], row index = y."""
    c = coords(n, dx)
    return c[None, :].repeat(n, 0), c[:, None].repeat(n, 1)


def radius_sq_exact(n: int, dx: float) -> np.ndarray:
    """r^2 = (i'^2 + j'^2) * (dx * dx), with i' = i - n/2 and the integer sum exact (Sec. 2.3:
    the quadratic phase argument is large, so it is formed from exact integers). Every binary
    mask below is the FP64 predicate r^2 <= R * R on this array."""
    k = np.arange(n, dtype=np.int64) - n // 2
    k2 = (k[None, :] ** 2 + k[:, None] ** 2).astype(np.float64)
    return k2 * (dx * dx)


def circular_aperture(n: int, dx: float, radius: float, obscuration: float = 0.0,
                      n_spiders: int = 0, spider_width: float = 0.0) -> np.ndarray:
    """Binary pupil (App. A ``CircularAperture``): transmits r <= radius, blocks r < eps*radius
    (central obscuration), and blocks the vanes |x| < w/2 or |y| < w/2 when spiders are on
    (four vanes in a '+' through the centre)."""
    x, y = grid(n, dx)
    r2 = radius_sq_exact(n, dx)
    a = (r2 <= radius * radius).astype(np.float64)
    if obscuration > 0.0:
        ro = obscuration * radius
        a[r2 < ro * ro] = 0.0
    if n_spiders:
        if n_spiders != 4:
            raise ValueError("only the four-vane '+' spider is defined")
        half = spider_width / 2.0
        a[(np.abs(x) < half) | (np.abs(y) < half)] = 0.0
    return a


def circle_stop(n: int, pitch: float, radius: float, opaque_inside: bool = False) -> np.ndarray:
    """Circular stop on a grid of the given pitch: transmits r <= radius (a field or Lyot stop),
    or, with ``opaque_inside``, blocks r <= radius (an occulting spot). A negative radius
    is an empty disk."""
    inside = (radius_sq_exact(n, pitch) <= radius * radius) & (radius >= 0.0)
    return (~inside if opaque_inside else inside).astype(np.float64)


def thin_lens(n: int, dx: float, wavelength: float, focal_length: float) -> np.ndarray:
    """Thin-lens transmission exp(-i pi r^2 / (lambda f)) (Sec. 1.1, Goodman Eq. 5-10; the
    quadratic phase factor of Eq. 2 with the constant read as pi/lambda)."""
    r2 = radius_sq_exact(n, dx)
    return np.exp(-1j * np.pi * r2 / (wavelength * focal_length))


def phasor(opd_m: np.ndarray, wavelength: float, amplitude: np.ndarray | None = None) -> np.ndarray:
    """Element phasor A exp(2 pi i OPD / lambda) (Eq. 3, read with the OPD in the numerator)."""
    p = np.exp(2j * np.pi * np.asarray(opd_m, dtype=np.float64) / wavelength)
    if amplitude is not None:
        p = p * np.asarray(amplitude, dtype=np.float64)
    return p


def sine_wfe(n: int, dx: float, spatial_freq: float, amplitude: float,
             axis: int = 1) -> np.ndarray:
    """Sine-wave OPD map (App. A ``SineWaveWFE``): amplitude * sin(2 pi nu x) along x (axis 1)
    or y (axis 0)."""
    x, y = grid(n, dx)
    t = x if axis == 1 else y
    return amplitude * np.sin(2 * np.pi * spatial_freq * t)


# ---------------------------------------------------------------------------- Zernike


def noll_to_nm(j: int) -> tuple[int, int]:
    """Noll index j >= 1 to (n, m); m > 0 is the cosine term, m < 0 the sine term.

    Noll (1976) ordering: radial order n ascending, |m| ascending within an order, and
    for m != 0 the pair (cos, sin) occupies two consecutive indices with the even index
    taking the cosine.
    """
    if j < 1:
        raise ValueError("Noll index starts at 1")
    count = 0
    n = 0
    while True:
        for am in range(n % 2, n + 1, 2):
            if am == 0:
                count += 1
                if count == j:
                    return n, 0
            else:
                first, second = count + 1, count + 2
                count += 2
                if j in (first, second):
                    return (n, am) if j % 2 == 0 else (n, -am)
        n += 1


def zernike_radial(n: int, m: int, rho: np.ndarray) -> np.ndarray:
    """R_n^|m|(rho) = sum_k (-1)^k (n-k)! / (k! ((n+|m|)/2-k)! ((n-|m|)/2-k)!) rho^(n-2k)."""
    am = abs(m)
    out = np.zeros_like(rho)
    for k in range((n - am) // 2 + 1):
        c = ((-1) ** k * math.factorial(n - k)
             / (math.factorial(k) * math.factorial((n + am) // 2 - k)
                * math.factorial((n - am) // 2 - k)))
        out = out + c * rho ** (n - 2 * k)
    return out


def zernike_noll(j: int, rho: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Unit-RMS Zernike polynomial Z_j over the unit disk (Noll normalisation)."""
    n, m = noll_to_nm(j)
    r = zernike_radial(n, m, rho)
    if m == 0:
        return math.sqrt(n + 1) * r
    norm = math.sqrt(2 * (n + 1))
    if m > 0:
        return norm * r * np.cos(m * theta)
    return norm * r * np.sin(-m * theta)


def zernike_opd(n: int, dx: float, radius: float, coeffs_m: np.ndarray,
                j_first: int) -> np.ndarray:
    """OPD = sum_j c_j Z_j(r/R, theta) inside the disk r <= R, zero outside."""
    x, y = grid(n, dx)
    rho = np.hypot(x, y) / radius
    theta = np.arctan2(y, x)
    opd = np.zeros((n, n))
    for i, c in enumerate(coeffs_m):
        opd += c * zernike_noll(j_first + i, rho, theta)
    opd[radius_sq_exact(n, dx) > radius * radius] = 0.0
    return opd


# ---------------------------------------------------------------------------- DM


def dm_influence_matrix(n: int, dx: float, n_act: int, pitch: float) -> np.ndarray:
    """G[j, a] = exp(-(x_j - x_a)^2 / (2 sigma^2)): 1-D Gaussian influence with FWHM = one
    pitch, actuator centres x_a = (a - (n_act-1)/2) * pitch."""
    sigma = pitch / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    x = coords(n, dx)
    xa = (np.arange(n_act) - (n_act - 1) / 2.0) * pitch
    d = x[:, None] - xa[None, :]
    return np.exp(-d * d / (2.0 * sigma * sigma))


def dm_surface(n: int, dx: float, heights_m: np.ndarray, pitch: float) -> np.ndarray:
    """DM surface s(x, y) = sum_{b,a} h[b,a] g(x - x_a) g(y - y_b) = G h G^T ([y][x])."""
    g = dm_influence_matrix(n, dx, heights_m.shape[-1], pitch)
    return g @ heights_m @ g.T


def dm_opd(n: int, dx: float, heights_m: np.ndarray, pitch: float) -> np.ndarray:
    """Reflected OPD = 2 x surface."""
    return 2.0 * dm_surface(n, dx, heights_m, pitch)
