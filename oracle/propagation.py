"""Fresnel and Fraunhofer propagators in FP64 (oracle; test infrastructure only).

* Centred DFT: F[k] = sum_j f[j] exp(-2 pi i (j - N/2)(k - N/2) / N), inverse with 1/N per
  axis. Written as fftshift(fft(ifftshift(.))) -- a library FFT used as a step.
* Angular spectrum (Sec. 1.1, Lawrence Eqs. 82-89 cited, paraxial transfer function):
  E(z) = IDFT2[ H . DFT2[E] ], H = exp(-i pi lambda z (fx^2 + fy^2)), piston dropped.
* Direct Fresnel (Sec. 1.1, with the quadratic phase factor of Eq. 2 read as
  exp(i pi r^2 / (lambda z))): E'(u) = 1/(i lambda z) Q(u) dx^2 DFT2[Q(x) E(x)],
  output pitch du = lambda z / (N dx).
* Matrix Fourier transform (Sec. 1.1 and Sec. 2.3, the "matrix DFT" of Soummer et al.):
  E'[v,u] = s sum_{i,j} E[i,j] exp(-+2 pi i (X_j U_u + Y_i V_v)), X in units of D, U in
  lambda/D, s = dU / npix.
"""
from __future__ import annotations

import numpy as np

from . import optics


def centred_dft2(e: np.ndarray) -> np.ndarray:
    """Centred 2-D DFT over the last two axes (no normalisation)."""
    ax = (-2, -1)
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(e, axes=ax), axes=ax), axes=ax)


def centred_idft2(e: np.ndarray) -> np.ndarray:
    """Centred 2-D inverse DFT over the last two axes (1/N^2 normalisation)."""
    ax = (-2, -1)
    return np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(e, axes=ax), axes=ax), axes=ax)


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


def direct_fresnel(e: np.ndarray, dx: float, wavelength: float, z: float) -> tuple[np.ndarray, float]:
    """Single-FFT (direct) Fresnel hop; returns (field, output pitch du = lambda z / (N dx))."""
    n = e.shape[-1]
    du = wavelength * z / (n * dx)
    inner = centred_dft2(e * quadratic_phase(n, dx, wavelength, z))
    out = quadratic_phase(n, du, wavelength, z) * inner * (dx * dx / (1j * wavelength * z))
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
