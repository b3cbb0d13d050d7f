"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only draws numbers and packs workload parameters. It holds none of the
propagation arithmetic (no element masks, no phase factors, no transforms of the field),
so that the GPU path and the FP64 oracle stay independent of each other and meet only
here, at their inputs.

Workloads (all synthetic; the paper's own benchmark system needs optics data files that
are not available, so inputs of the same shape stand in for it):

* ``talbot``      -- App. A: 2 cm beam radius, 0.5 um, npix 256, oversample 8, a sine phase
                     grating of 5 nm amplitude at 500 cycles/m.
* ``airy``        -- 128-px clear 1 m aperture padded to 256^2 (complex128), 500 nm,
                     lens f = 10 m, direct Fresnel 10 m to focus, MFT to 64^2 at 0.5 lambda/D.
* ``relay``       -- 1024-px pupil padded to 2048^2 / 4096^2 (complex64), 550 nm, six planes
                     (obscured + spidered aperture, lens 5 m, PSD surface, lens 2 m, PSD
                     surface, field stop), five hops of 0.5-5 m drawn from the seed
                     (Sec. 1.2: N of 2048 or 4096; about ten optics and 19 FFTs per
                     wavelength for the paper's example system).
* ``lyot``        -- classical Lyot coronagraph: 1024^2 pupil, Zernike 4-21 at 5 nm RMS,
                     MFT to 256^2 occulter at 0.05 lambda/D with a 5 lambda/D spot, MFT back
                     to the 1024^2 Lyot plane (stop 80 % of D), MFT to 512^2 at 0.25 lambda/D.
* ``broadband``   -- the Lyot system at 21 wavelengths over 500-600 nm x 8 DM probes.
* ``wfc``         -- two 48x48 DMs 0.3 m apart (Fresnel 4096^2), Lyot chain at 11 wavelengths.
* ``spc``         -- the shape of App. B's shaped-pupil coronagraph system: a 2.37 m f/7.8
                     telescope, a 20 mm relay beam, four f/20 relay optics, a shaped pupil and a
                     bow-tie focal-plane mask, nine planes through three foci. The two masks are
                     binary amplitude maps standing in for the App. B mask files (not available):
                     like the PSD surfaces they are inputs, generated here at a pitch the caller
                     gives and passed to both paths.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ----------------------------------------------------------------------------------------
# random draws
# ----------------------------------------------------------------------------------------


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator; identical streams on x86-64 and aarch64."""
    return np.random.default_rng(seed)


def random_field(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    """Complex Gaussian test field (unit variance per component)."""
    g = rng(seed)
    re = g.standard_normal(shape)
    im = g.standard_normal(shape)
    return (re + 1j * im).astype(dtype)


def hop_distances(seed: int, n_hops: int, lo: float = 0.5, hi: float = 5.0) -> np.ndarray:
    """Propagation distances in metres, uniform in [lo, hi)."""
    return rng(seed).uniform(lo, hi, size=n_hops)


def psd_surface(n: int, seed: int, exponent: float = -3.0, rms_m: float = 20e-9) -> np.ndarray:
    """Power-law PSD surface map (metres of OPD), float64 [n][n].

    White complex Gaussian noise shaped by |f|^(exponent/2) (so the PSD goes as
    |f|^exponent), the zero-frequency term removed, real part taken, then scaled to
    ``rms_m`` RMS over the whole map. Input synthesis only.
    """
    g = rng(seed)
    white = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    k = np.fft.fftfreq(n)
    kr = np.hypot(k[None, :], k[:, None])
    shape = np.zeros_like(kr)
    nz = kr > 0
    shape[nz] = kr[nz] ** (exponent / 2.0)
    surf = np.fft.ifft2(white * shape).real
    surf -= surf.mean()
    surf *= rms_m / math.sqrt(np.mean(surf * surf))
    return surf


def zernike_coefficients(seed: int, j_first: int = 4, j_last: int = 21,
                         rms_m: float = 5e-9) -> np.ndarray:
    """Normal coefficients for Noll terms j_first..j_last, scaled so sqrt(sum c^2) = rms_m."""
    c = rng(seed).standard_normal(j_last - j_first + 1)
    return c * (rms_m / math.sqrt(float(np.sum(c * c))))


def dm_heights(seed: int, n_act: int = 48, n_dm: int = 2, amp_m: float = 5e-9) -> np.ndarray:
    """DM actuator heights (metres of surface), uniform in [-amp, amp), [n_dm][n_act][n_act]."""
    return rng(seed).uniform(-amp_m, amp_m, size=(n_dm, n_act, n_act))


def sinc_probes(n_act: int = 48, n_probe: int = 8, amp_m: float = 10e-9,
                width_act: float = 2.0, cycles: float = 13.0) -> np.ndarray:
    """Sinc probe commands [n_probe][n_act][n_act] (metres of surface).

    Probe p is amp * sinc(a/w) * sinc(b/w) * cos(2 pi cycles a / n_act + p pi/4), where a, b
    are actuator offsets from the grid centre in actuator pitches. These are DM *commands*
    (inputs); the influence-function synthesis is part of the method.
    """
    a = np.arange(n_act) - (n_act - 1) / 2.0
    sx = np.sinc(a / width_act)
    out = np.empty((n_probe, n_act, n_act))
    for p in range(n_probe):
        carrier = np.cos(2 * np.pi * cycles * a / n_act + p * np.pi / 4)
        out[p] = amp_m * np.outer(sx, sx * carrier)
    return out


def actuator_offsets(seed: int, n_act: int, count: int) -> np.ndarray:
    """Distinct (dm, row, col) actuator picks for finite-difference checks, [count][3]."""
    g = rng(seed)
    flat = g.choice(2 * n_act * n_act, size=count, replace=False)
    dm = flat // (n_act * n_act)
    rem = flat % (n_act * n_act)
    return np.stack([dm, rem // n_act, rem % n_act], axis=1)


# ----------------------------------------------------------------------------------------
# workload parameter sets
# ----------------------------------------------------------------------------------------


@dataclasses.dataclass
class RelayWorkload:
    """Six-plane Fresnel relay (complex64); element order along the beam."""
    n: int = 4096
    npix: int = 1024
    diam_m: float = 1.0
    wavelength_m: float = 550e-9
    obscuration: float = 0.3          # fraction of the radius
    n_spiders: int = 4
    spider_width_frac: float = 0.01   # of D
    lens1_m: float = 5.0
    lens2_m: float = 2.0
    field_stop_frac: float = 0.9      # of the pupil radius
    psd_rms_m: float = 20e-9
    seed: int = 0
    batch: int = 1

    @property
    def dx(self) -> float:
        return self.diam_m / self.npix

    def distances(self) -> np.ndarray:
        return hop_distances(self.seed, 5)

    def psd_maps(self) -> tuple[np.ndarray, np.ndarray]:
        return (psd_surface(self.n, 1000 + 2 * self.seed, rms_m=self.psd_rms_m),
                psd_surface(self.n, 1001 + 2 * self.seed, rms_m=self.psd_rms_m))


@dataclasses.dataclass
class LyotWorkload:
    """Classical Lyot coronagraph (semi-analytic, MFT based)."""
    n: int = 1024                # pupil array = pupil diameter in pixels
    npix: int = 1024
    diam_m: float = 1.0
    wavelength_m: float = 550e-9
    zernike_first: int = 4
    zernike_last: int = 21
    zernike_rms_m: float = 5e-9
    m_occ: int = 256
    du_occ: float = 0.05         # lambda/D per pixel at the occulter
    spot_radius_lamd: float = 5.0
    lyot_frac: float = 0.8       # Lyot stop radius / pupil radius
    m_det: int = 512
    du_det: float = 0.25         # lambda/D per pixel at the detector
    dh_inner: float = 6.0
    dh_outer: float = 20.0
    seed: int = 0

    def zernike(self) -> np.ndarray:
        return zernike_coefficients(self.seed, self.zernike_first, self.zernike_last,
                                    self.zernike_rms_m)


@dataclasses.dataclass
class BroadbandWorkload:
    """Lyot system over a band x DM probes; uneven occulter sizes per wavelength."""
    lyot: LyotWorkload = dataclasses.field(default_factory=LyotWorkload)
    n_lambda: int = 21
    lambda_lo_m: float = 500e-9
    lambda_hi_m: float = 600e-9
    lambda_c_m: float = 550e-9
    n_probe: int = 8
    n_act: int = 48

    def wavelengths(self) -> np.ndarray:
        return np.linspace(self.lambda_lo_m, self.lambda_hi_m, self.n_lambda)

    def occulter_sizes(self) -> np.ndarray:
        """Per-wavelength occulter width: fixed angular pitch 0.05 lambda_c/D over the same
        12.8 lambda_c/D field, so M = round(256 lambda_c / lambda)."""
        return np.rint(self.lyot.m_occ * self.lambda_c_m / self.wavelengths()).astype(np.int64)

    def probes(self) -> np.ndarray:
        return sinc_probes(self.n_act, self.n_probe)


@dataclasses.dataclass
class WfcWorkload:
    """Two-DM wavefront control: 48x48 Gaussian-influence DMs (FWHM one pitch) over a 48 mm
    pupil, DM2 0.3 m from DM1 on a Fresnel grid of n_fresnel^2, then the Lyot system at
    n_lambda wavelengths over 525-575 nm. The focal-plane masks are fixed in lambda_c/D, so
    each wavelength's item scales by lambda_c / lambda (uneven occulter sizes)."""
    lyot: LyotWorkload = dataclasses.field(default_factory=LyotWorkload)
    n_fresnel: int = 4096
    diam_m: float = 0.048
    z_m: float = 0.3
    n_act: int = 48
    act_amp_m: float = 5e-9
    n_lambda: int = 11
    lambda_lo_m: float = 525e-9
    lambda_hi_m: float = 575e-9
    lambda_c_m: float = 550e-9
    seed: int = 0

    @property
    def pitch_m(self) -> float:
        return self.diam_m / self.n_act

    def wavelengths(self) -> np.ndarray:
        return np.linspace(self.lambda_lo_m, self.lambda_hi_m, self.n_lambda)

    def heights(self) -> np.ndarray:
        return dm_heights(self.seed, self.n_act, 2, self.act_amp_m)

    def item(self, wavelength: float) -> dict:
        """One wavelength's Lyot item (occulter, spot, detector pitch, dark hole in lambda/D)."""
        lw, r = self.lyot, self.lambda_c_m / wavelength
        return dict(m_occ=int(np.rint(lw.m_occ * r)), du_occ=lw.du_occ * r, spot_radius=lw.spot_radius_lamd * r,
                    du_det=lw.du_det * r, dh_in=lw.dh_inner * r, dh_out=lw.dh_outer * r)

    def fd_actuators(self, count: int = 16) -> np.ndarray:
        return actuator_offsets(self.seed + 11, self.n_act, count)


@dataclasses.dataclass
class SpcWorkload:
    """Optical system of App. B's shape (its prescription: primary f/7.8 of 2.37 m, a secondary
    that collimates a 20 mm beam, f/20 relay optics); masks are stand-ins (see module doc)."""
    npix: int = 256
    oversample: int = 4
    wavelength_m: float = 550e-9
    d_prim_m: float = 2.37
    f_ratio_prim: float = 7.8
    d_relay_m: float = 0.02
    f_ratio_relay: float = 20.0
    obscuration: float = 0.3
    n_spiders: int = 4
    spider_width_frac: float = 0.01
    bowtie_inner_lamd: float = 2.5
    bowtie_outer_lamd: float = 9.0
    bowtie_half_angle_deg: float = 32.5
    n_rings: int = 6
    seed: int = 0

    @property
    def n(self) -> int:
        return self.npix * self.oversample

    @property
    def dx(self) -> float:
        return self.d_prim_m / self.npix

    @property
    def f_pri(self) -> float:
        return self.f_ratio_prim * self.d_prim_m

    @property
    def f_m2(self) -> float:
        return self.f_pri * self.d_relay_m / self.d_prim_m

    @property
    def f_m3(self) -> float:
        return self.f_ratio_relay * self.d_relay_m

    def layout(self) -> list:
        """Per plane, what sits there: ("aperture",), ("lens", f), ("shaped_pupil",), ("fpm",)."""
        f3 = self.f_m3
        return [[("aperture",), ("lens", self.f_pri)], [("lens", self.f_m2)], [("lens", f3)], [("lens", f3)],
                [("shaped_pupil",)], [("lens", f3)], [("fpm",)], [("lens", f3)], []]

    def distances(self) -> list:
        f3 = self.f_m3
        return [self.f_pri + self.f_m2, self.f_m2 + f3, 2 * f3, f3, f3, f3, 2 * f3, 2 * f3]

    def shaped_pupil(self, n: int, pitch: float) -> np.ndarray:
        """Binary concentric-ring amplitude mask over the relayed 20 mm pupil: ring edges drawn
        from the seed, alternately open and closed, closed inside the obscuration."""
        r_pup = 0.5 * self.d_relay_m
        edges = np.sort(rng(self.seed + 500).uniform(self.obscuration, 1.0, 2 * self.n_rings - 1)) * r_pup
        k = np.arange(n, dtype=np.float64) - n // 2
        r = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2) * pitch
        zone = np.searchsorted(edges, r)                   # 0 .. 2 n_rings - 1
        m = (zone % 2 == 0) & (r >= self.obscuration * r_pup) & (r <= r_pup)
        return m.astype(np.float32)

    def bowtie(self, n: int, pitch: float, wavelength: float) -> np.ndarray:
        """Bow-tie focal-plane mask: open for inner <= r <= outer (lambda/D of the f/20 relay
        beam) within +-half_angle of the x axis on both sides."""
        lamd = wavelength * self.f_ratio_relay
        k = np.arange(n, dtype=np.float64) - n // 2
        x, y = k[None, :] * pitch, k[:, None] * pitch
        r = np.hypot(x, y)
        wedge = np.abs(y) <= np.tan(np.radians(self.bowtie_half_angle_deg)) * np.abs(x)
        m = (r >= self.bowtie_inner_lamd * lamd) & (r <= self.bowtie_outer_lamd * lamd) & wedge
        return m.astype(np.float32)


def configs_summary() -> dict:
    return {"relay": dataclasses.asdict(RelayWorkload()),
            "lyot": dataclasses.asdict(LyotWorkload())}
