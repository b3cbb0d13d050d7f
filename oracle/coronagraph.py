"""Semi-analytic Lyot coronagraph, detector intensity and dark-hole sums in FP64
(oracle; test infrastructure only).

The paper (Sec. 1.1) names the Soummer et al. semi-analytic method -- MFTs of modest
arrays around a small focal-plane mask -- without writing it out. Its Babinet form is:

    E_B = MFT(E_A; M_occ, dU_occ)                    pupil -> occulter
    E_C = E_A - MFT^-1(spot . E_B)                    occulter -> Lyot (spot = 1 on the mask)
    E_D = E_C . Lyot stop
    E_det = MFT(E_D; M_det, dU_det)                   Lyot -> detector

Intensities are normalised by the peak of the same chain with the occulter removed.
The dark hole is the annulus r_in <= rho <= r_out (lambda/D, inclusive).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import optics, propagation


@dataclasses.dataclass
class LyotParams:
    n: int
    npix: float
    m_occ: int
    du_occ: float
    spot_radius: float       # lambda/D
    lyot_frac: float         # of the pupil radius
    m_det: int
    du_det: float


def focal_mask(m: int, du: float, radius: float) -> np.ndarray:
    """1 on the occulting spot (rho <= radius in lambda/D), 0 elsewhere."""
    return optics.circle_stop(m, du, radius, opaque_inside=False)


def lyot_stop(n: int, npix: float, frac: float) -> np.ndarray:
    """Lyot stop transmitting r <= frac * D/2 on the pupil grid (pitch 1/npix in D units)."""
    return optics.circle_stop(n, 1.0 / npix, 0.5 * frac)


def lyot_fields(e_pupil: np.ndarray, p: LyotParams, occulter: bool = True) -> dict:
    """All intermediate planes of the Babinet Lyot chain for one wavelength."""
    e_b = propagation.mft(e_pupil, p.npix, p.m_occ, p.du_occ)
    if occulter:
        spot = focal_mask(p.m_occ, p.du_occ, p.spot_radius)
        e_c = e_pupil - propagation.imft(spot * e_b, p.npix, p.n, p.du_occ)
    else:
        e_c = e_pupil.astype(np.complex128)
    e_d = e_c * lyot_stop(p.n, p.npix, p.lyot_frac)
    e_det = propagation.mft(e_d, p.npix, p.m_det, p.du_det)
    return {"B": e_b, "C": e_c, "D": e_d, "det": e_det}


def intensity(e: np.ndarray, norm: float = 1.0) -> np.ndarray:
    return (e.real ** 2 + e.imag ** 2) / norm


def peak_intensity(e_pupil: np.ndarray, p: LyotParams) -> float:
    """Normalisation: max |E_det|^2 with the occulter removed (Lyot stop kept)."""
    return float(intensity(lyot_fields(e_pupil, p, occulter=False)["det"]).max())


def dark_hole_mask(m: int, du: float, r_in: float, r_out: float) -> np.ndarray:
    r2 = optics.radius_sq_exact(m, du)
    return ((r2 >= r_in * r_in) & (r2 <= r_out * r_out)).astype(np.float64)


def dark_hole_sum(i_norm: np.ndarray, du: float, r_in: float, r_out: float) -> float:
    """S = sum of the normalised intensity over the dark-hole annulus."""
    return float(np.sum(i_norm * dark_hole_mask(i_norm.shape[-1], du, r_in, r_out)))


def lyot_psf(e_pupil: np.ndarray, p: LyotParams, r_in: float, r_out: float,
             peak: float | None = None) -> tuple[np.ndarray, float, float]:
    """Normalised detector intensity, dark-hole sum and the peak used."""
    if peak is None:
        peak = peak_intensity(e_pupil, p)
    i_norm = intensity(lyot_fields(e_pupil, p)["det"], peak)
    return i_norm, dark_hole_sum(i_norm, p.du_det, r_in, r_out), peak


def pupil_field(n: int, npix: float, wavelength: float, opd_m: np.ndarray | None,
                radius_frac: float = 1.0) -> np.ndarray:
    """Clear circular pupil (radius D/2 on a grid of pitch D/npix, D = 1) times the phasor of
    an OPD map."""
    a = optics.circular_aperture(n, 1.0 / npix, 0.5 * radius_frac)
    if opd_m is None:
        return a.astype(np.complex128)
    return a * optics.phasor(opd_m, wavelength)
