"""Fresnel and Fraunhofer propagators in FP64 (oracle; test infrastructure only).

* Centred DFT: F[k] = sum_j f[j] exp(-2 pi i (j - N/2)(k - N/2) / N), inverse with 1/N per
  axis, one axis after the other through the textbook radix-2 FFT of ``oracle.fft`` (direct
  sums on the odd factor of N).
* Angular spectrum (Sec. 1.1, Lawrence Eqs. 82-89 cited, paraxial transfer function):
  E(z) = IDFT2[ H . DFT2[E] ], H = exp(-i pi lambda z (fx^2 + fy^2)), piston dropped.
* Direct Fresnel (Sec. 1.1, with the quadratic phase factor of Eq. 2 read as
  exp(i pi r^2 / (lambda z))): E'(u) = 1/(i lambda z) Q(u) dx^2 DFT2[Q(x) E(x)],
  output pitch du = |lambda z / (N dx)|; the inverse DFT for z < 0.
* Pilot-beam system (Lawrence's method as cited in Sec. 1.1): fresnel_system_pilot.
* Matrix Fourier transform (Sec. 1.1 and Sec. 2.3, the "matrix DFT" of Soummer et al.):
  E'[v,u] = s sum_{i,j} E[i,j] exp(-+2 pi i (X_j U_u + Y_i V_v)), X in units of D, U in
  lambda/D, s = dU / npix.
"""
from __future__ import annotations

import numpy as np

from . import fft, optics


def centred_dft2(e: np.ndarray) -> np.ndarray:
    """Centred 2-D DFT over the last two axes (no normalisation): rows, then columns."""
    return fft.centred_dft(fft.centred_dft(e, -1, -1), -2, -1)


def centred_idft2(e: np.ndarray) -> np.ndarray:
    """Centred 2-D inverse DFT over the last two axes (1/N per axis)."""
    n0, n1 = e.shape[-2], e.shape[-1]
    return fft.centred_dft(fft.centred_dft(e, -1, +1), -2, +1) / (n0 * n1)


def freqs(n: int, dx: float) -> np.ndarray:
    """Centred spatial frequencies f_k = (k - N/2) / (N dx)."""
    return (np.arange(n, dtype=np.float64) - n // 2) / (n * dx)


def transfer_function(n: int, dx: float, wavelength: float, z: float) -> np.ndarray:
    """Paraxial angular-spectrum transfer function exp(-i pi lambda z (fx^2 + fy^2)).

    The frequency offsets are exact integers k' = k - N/2, so the argument is formed as
    pi lambda z (kx'^2 + ky'^2) / (N dx)^2.
    """
    k = np.arange(n, dtype=np.int64) - n // 2
    k2 = (k[None, :] ** 2 + k[:, None] ** 2).astype(np.float64)
    return np.exp(-1j * np.pi * wavelength * z * k2 / (n * dx) ** 2)


def angular_spectrum(e: np.ndarray, dx: float, wavelength: float, z: float) -> np.ndarray:
    """Plane-to-plane angular-spectrum hop at constant pixel scale."""
    h = transfer_function(e.shape[-1], dx, wavelength, z)
    return centred_idft2(h * centred_dft2(e))


def quadratic_phase(n: int, pitch: float, wavelength: float, z: float) -> np.ndarray:
    """Quadratic phase factor exp(i pi r^2 / (lambda z)) (Eq. 2 with the pi/lambda restored)."""
    r2 = optics.radius_sq_exact(n, pitch)
    return np.exp(1j * np.pi * r2 / (wavelength * z))


def direct_fresnel(e: np.ndarray, dx: float, wavelength: float, z: float,
                   q_in: bool = True, q_out: bool = True) -> tuple[np.ndarray, float]:
    """Single-FFT (direct) Fresnel hop; returns (field, output pitch du = |lambda z / (N dx)|).

    The Fresnel kernel exp(-2 pi i x u / (lambda z)) on the grids x_j = (j - N/2) dx and
    u_k = (k - N/2) du is exp(-+ 2 pi i j' k' / N) for z >< 0: the forward DFT, or the
    unnormalised inverse DFT (N^2 times centred_idft2) for z < 0. q_in / q_out drop the input
    or output quadratic phase (hops from / to a pilot-beam waist, see fresnel_system_pilot).
    """
    n = e.shape[-1]
    du = abs(wavelength * z / (n * dx))
    a = e * quadratic_phase(n, dx, wavelength, z) if q_in else e
    inner = centred_dft2(a) if z > 0 else (n * n) * centred_idft2(a)
    out = inner * (dx * dx / (1j * wavelength * z))
    if q_out:
        out = out * quadratic_phase(n, du, wavelength, z)
    return out, du


def mft_matrix(m: int, du: float, n: int, npix: float, sign: int) -> np.ndarray:
    """A[u, j] = exp(sign 2 pi i X_j U_u), X_j = (j - n/2)/npix (units of D),
    U_u = (u - m/2) du (units of lambda/D)."""
    x = (np.arange(n, dtype=np.float64) - n // 2) / npix
    u = (np.arange(m, dtype=np.float64) - m // 2) * du
    return np.exp(sign * 2j * np.pi * np.outer(u, x))


def mft(e: np.ndarray, npix: float, m: int, du: float) -> np.ndarray:
    """Forward MFT pupil -> focal plane: E' = s Ay E Ax^T with s = du / npix."""
    n = e.shape[-1]
    a = mft_matrix(m, du, n, npix, -1)
    return (du / npix) * (a @ e @ a.T)


def imft(e: np.ndarray, npix: float, n: int, du: float) -> np.ndarray:
    """Inverse MFT focal plane (pitch du in lambda/D, width m) -> pupil of n pixels with npix
    pixels across D: E[i,j] = s sum E'[v,u] exp(+2 pi i (X_j U_u + Y_i V_v)), s = du/npix."""
    m = e.shape[-1]
    a = mft_matrix(m, du, n, npix, +1)   # [m][n]
    return (du / npix) * (a.T @ e @ a)


def fresnel_chain(e0: np.ndarray, dx: float, wavelength: float, elements: list,
                  distances: list) -> np.ndarray:
    """Plane-by-plane system: apply element 0, hop distances[0], apply element 1, ...

    ``elements`` are complex transmission arrays (or None for a bare plane); angular
    spectrum hops keep the pixel scale (App. B prescription style: add_optic(optic, distance)).
    """
    e = e0.astype(np.complex128)
    for i, el in enumerate(elements):
        if el is not None:
            e = e * el
        if i < len(distances):
            e = angular_spectrum(e, dx, wavelength, distances[i])
    return e


def fresnel_system_pilot(e0: np.ndarray, dx: float, wavelength: float, beam_radius: float,
                         planes: list, distances: list) -> tuple[np.ndarray, float, list, int]:
    """Fresnel system with the method chosen by a Gaussian pilot beam (Sec. 1.1: the angular-
    spectrum / direct choice of Lawrence's method; reading R17).

    planes[p] is a list of elements at plane p: ("lens", f) for a thin lens, or a function
    (n, pitch) -> array multiplied onto the field. The pilot beam starts with its waist
    beam_radius at plane 0; its complex parameter q (Gaussian exp(i pi r^2 / (lambda q)) under
    the kernel of direct_fresnel) moves as q += d over a distance d and 1/q -= 1/f at a lens.
    A plane with |Re q| < |Im q| is inside the Rayleigh range and holds the field itself;
    otherwise it holds the field times exp(-i pi r^2 / (lambda R)), R = Re q, the distance from
    the pilot waist. Between planes: inside -> inside angular spectrum; inside -> outside
    angular spectrum to the waist, then direct Fresnel without output phase; outside -> inside
    direct Fresnel without input phase to the waist, then angular spectrum; outside -> outside
    both direct legs. Returns (field at the last plane, pitch, per-plane outside flags, number
    of direct legs).
    """
    n = e0.shape[-1]
    e = np.array(e0, dtype=np.complex128)
    pitch = float(dx)
    q = complex(0.0, -np.pi * beam_radius ** 2 / wavelength)

    def is_inside(qq: complex) -> bool:
        return abs(qq.real) < abs(qq.imag)

    def reference(radius: float) -> np.ndarray:          # exp(i pi r^2 / (lambda R))
        return quadratic_phase(n, pitch, wavelength, radius)

    outside = False
    flags, legs = [], 0
    for p, plane in enumerate(planes):
        lenses = [el[1] for el in plane if isinstance(el, tuple) and el[0] == "lens"]
        for el in plane:
            if not (isinstance(el, tuple) and el[0] == "lens"):
                e = e * el(n, pitch)
        if lenses:
            if outside:
                e = e * reference(q.real)                 # back to the field itself
            for f in lenses:
                e = e * optics.thin_lens(n, pitch, wavelength, f)
                q = 1.0 / (1.0 / q - 1.0 / f)
            outside = not is_inside(q)
            if outside:
                e = e / reference(q.real)
        flags.append(outside)
        if p == len(planes) - 1:
            if outside:
                e = e * reference(q.real)
            break
        d = distances[p]
        qb = q + d
        in_a, in_b = not outside, is_inside(qb)
        if in_a and in_b:
            e = angular_spectrum(e, pitch, wavelength, d)
        elif in_a:
            if -q.real != 0.0:
                e = angular_spectrum(e, pitch, wavelength, -q.real)
            e, pitch = direct_fresnel(e, pitch, wavelength, qb.real, q_in=True, q_out=False)
            legs += 1
        elif in_b:
            e, pitch = direct_fresnel(e, pitch, wavelength, -q.real, q_in=False, q_out=True)
            legs += 1
            if qb.real != 0.0:
                e = angular_spectrum(e, pitch, wavelength, qb.real)
        else:
            e, pitch = direct_fresnel(e, pitch, wavelength, -q.real, q_in=False, q_out=True)
            e, pitch = direct_fresnel(e, pitch, wavelength, qb.real, q_in=True, q_out=False)
            legs += 2
        q = qb
        outside = not in_b
    return e, pitch, flags, legs
