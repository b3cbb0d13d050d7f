"""Wavefront-control model and its hand-derived adjoint in FP64 (oracle; test
infrastructure only).

Model (one wavelength): a clear pupil carrying DM1 sits on an N_f x N_f Fresnel grid,
the field hops +z to DM2, takes DM2's phase, hops -z back to the pupil-conjugate plane,
the central n x n is cut out and sent through the Babinet Lyot chain. The loss is the
summed normalised dark-hole intensity L = sum_lambda sum_{pix in DH} |E_det|^2 / I_peak,
with I_peak computed once at zero DM heights and held fixed.

Gradient convention: for a real loss, G = dL/d conj(E) so that dL = 2 Re sum conj(G) dE.
Linear maps pass G through their conjugate transposes (MFT^H = inverse MFT with the same
pitch and scale; AS(z)^H = AS(-z); masks are real). At a phase element
E_out = E_in exp(i phi): dL/dphi = 2 Im(G conj(E_out)) and G_in = exp(-i phi) G_out.
With OPD = 2 x surface and phi = 2 pi OPD / lambda, dL/dh = (4 pi / lambda) G^T (dL/dphi) G.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import coronagraph, optics, propagation


@dataclasses.dataclass
class WfcParams:
    n_f: int                  # Fresnel grid
    npix: int                 # pupil pixels across D (also the Lyot-chain pupil array size)
    diam_m: float
    z_m: float                # DM1 -> DM2 distance
    n_act: int
    lyot: coronagraph.LyotParams
    dh_in: float
    dh_out: float

    @property
    def dx(self) -> float:
        return self.diam_m / self.npix

    @property
    def pitch(self) -> float:
        return self.diam_m / self.n_act


def crop(e: np.ndarray, n: int) -> np.ndarray:
    c = e.shape[-1] // 2
    return e[..., c - n // 2:c + n // 2, c - n // 2:c + n // 2]


def pad(e: np.ndarray, n_f: int) -> np.ndarray:
    """Adjoint of ``crop``: embed in the centre of zeros."""
    n = e.shape[-1]
    out = np.zeros(e.shape[:-2] + (n_f, n_f), dtype=np.complex128)
    c = n_f // 2
    out[..., c - n // 2:c + n // 2, c - n // 2:c + n // 2] = e
    return out


def forward(h: np.ndarray, wavelength: float, p: WfcParams, static_opd: np.ndarray | None = None,
            peak: float | None = None) -> dict:
    """Forward model for one wavelength; keeps every plane for the adjoint."""
    dx = p.dx
    ap = optics.circular_aperture(p.n_f, dx, 0.5 * p.diam_m)
    opd1 = optics.dm_opd(p.n_f, dx, h[0], p.pitch)
    if static_opd is not None:
        opd1 = opd1 + static_opd
    e0 = ap * optics.phasor(opd1, wavelength)
    e1 = propagation.angular_spectrum(e0, dx, wavelength, p.z_m)
    ph2 = optics.phasor(optics.dm_opd(p.n_f, dx, h[1], p.pitch), wavelength)
    e2 = e1 * ph2
    e3 = propagation.angular_spectrum(e2, dx, wavelength, -p.z_m)
    e_a = crop(e3, p.npix)
    planes = coronagraph.lyot_fields(e_a, p.lyot)
    if peak is None:
        peak = coronagraph.peak_intensity(e_a, p.lyot)
    mask = coronagraph.dark_hole_mask(p.lyot.m_det, p.lyot.du_det, p.dh_in, p.dh_out)
    loss = float(np.sum(mask * coronagraph.intensity(planes["det"], peak)))
    return dict(e0=e0, e1=e1, e2=e2, ph2=ph2, e3=e3, e_a=e_a, planes=planes, peak=peak,
                mask=mask, loss=loss)


def loss(h: np.ndarray, wavelength: float, p: WfcParams, peak: float) -> float:
    """The loss alone (what a central difference needs), for process pools."""
    return forward(h, wavelength, p, peak=peak)["loss"]


def zero_height_peak(wavelength: float, p: WfcParams) -> float:
    """The normalisation peak: the system with both DMs flat."""
    return forward(np.zeros((2, p.n_act, p.n_act)), wavelength, p)["peak"]


def lyot_adjoint(g_det: np.ndarray, p: coronagraph.LyotParams) -> np.ndarray:
    """Conjugate transpose of the Babinet Lyot chain: detector gradient -> pupil gradient."""
    g_d = propagation.imft(g_det, p.npix, p.n, p.du_det)              # MFT_3^H
    g_c = g_d * coronagraph.lyot_stop(p.n, p.npix, p.lyot_frac)
    spot = coronagraph.focal_mask(p.m_occ, p.du_occ, p.spot_radius)
    inner = propagation.mft(g_c, p.npix, p.m_occ, p.du_occ)            # IMFT_2^H
    return g_c - propagation.imft(spot * inner, p.npix, p.n, p.du_occ)  # MFT_1^H


def gradient(h: np.ndarray, wavelength: float, p: WfcParams, static_opd: np.ndarray | None = None,
             peak: float | None = None) -> tuple[float, np.ndarray]:
    """Loss and dL/dh ([2][n_act][n_act], per metre of surface) for one wavelength."""
    f = forward(h, wavelength, p, static_opd, peak)
    g_det = f["mask"] * f["planes"]["det"] / f["peak"]
    g_a = lyot_adjoint(g_det, p.lyot)
    g3 = pad(g_a, p.n_f)
    g2 = propagation.angular_spectrum(g3, p.dx, wavelength, p.z_m)     # AS(-z)^H
    dphi2 = 2.0 * np.imag(g2 * np.conj(f["e2"]))
    g1 = np.conj(f["ph2"]) * g2
    g0 = propagation.angular_spectrum(g1, p.dx, wavelength, -p.z_m)    # AS(z)^H
    dphi1 = 2.0 * np.imag(g0 * np.conj(f["e0"]))
    gm = optics.dm_influence_matrix(p.n_f, p.dx, p.n_act, p.pitch)
    scale = 4.0 * np.pi / wavelength
    grad = np.stack([scale * (gm.T @ dphi1 @ gm), scale * (gm.T @ dphi2 @ gm)])
    return f["loss"], grad


def broadband_gradient(h: np.ndarray, wavelengths, p: WfcParams,
                       static_opd: np.ndarray | None = None, peaks=None):
    """Sum of losses and gradients over wavelengths; peaks default to the h = 0 values."""
    if peaks is None:
        zero = np.zeros_like(h)
        peaks = [forward(zero, lam, p, static_opd)["peak"] for lam in wavelengths]
    total = 0.0
    grad = np.zeros_like(h)
    for lam, pk in zip(wavelengths, peaks):
        l, g = gradient(h, lam, p, static_opd, pk)
        total += l
        grad += g
    return total, grad, list(peaks)
