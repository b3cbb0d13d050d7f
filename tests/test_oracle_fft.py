"""Pins for the oracle's textbook FFT (radix-2 Cooley-Tukey with direct sums on the odd factor)
against the DFT's definition: brute-force sums, closed forms of impulses and pure tones,
Parseval's identity, the inverse, and (on a few lines at N = 4096 only) numpy's library FFT.
"""
import cmath

import numpy as np
import pytest

from oracle import fft, propagation
from paper_1806_06467_gb300 import inputs


def brute_dft(f, sign=-1):
    """F[k] = sum_j f[j] exp(sign 2 pi i j k / N), one term at a time."""
    n = len(f)
    return np.array([sum(f[j] * cmath.exp(sign * 2j * cmath.pi * j * k / n) for j in range(n))
                     for k in range(n)])


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 6, 12, 18, 30, 48, 100, 150, 3, 7])
def test_fft_matches_brute_force(n):
    f = inputs.random_field((n,), seed=100 + n)
    ref = brute_dft(f)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(fft.dft(f) - ref).max() < 1e-13 * scale * max(1, np.log2(n))
    assert np.abs(fft.dft_direct(f) - ref).max() < 1e-13 * scale * n
    assert np.abs(fft.dft(f, +1) - brute_dft(f, +1)).max() < 1e-13 * scale * max(1, np.log2(n))


@pytest.mark.parametrize("n", [4096, 2800, 4100])
def test_fft_closed_forms_at_grid_sizes(n):
    """Impulse at j0 -> exp(-2 pi i j0 k / N); the tone exp(2 pi i k0 j / N) -> N delta(k - k0);
    a constant -> N delta(k). The grid sizes of the relay (4096) and of the mixed-radix passes
    (2800 = 16 x 175, 4100 = 4 x 1025)."""
    k = np.arange(n)
    j0, k0 = 37, 1234 % n
    f = np.zeros(n, complex)
    f[j0] = 1.0
    expect = np.exp(-2j * np.pi * ((j0 * k) % n) / n)
    assert np.abs(fft.dft(f) - expect).max() < 1e-12
    tone = np.exp(2j * np.pi * ((k0 * k) % n) / n)
    spec = fft.dft(tone)
    delta = np.zeros(n)
    delta[k0] = n
    assert np.abs(spec - delta).max() < 1e-9
    assert np.abs(fft.dft(np.ones(n)) - np.eye(1, n, 0)[0] * n).max() < 1e-9


@pytest.mark.parametrize("n", [4096, 4100])
def test_fft_parseval_and_inverse(n):
    f = inputs.random_field((3, n), seed=n)
    g = fft.dft(f)
    assert abs(np.sum(np.abs(g) ** 2) / (n * np.sum(np.abs(f) ** 2)) - 1) < 1e-13
    np.testing.assert_allclose(fft.dft(g, +1) / n, f, rtol=0, atol=1e-12)


def test_fft_cross_check_library_4096():
    """A library FFT as an outside check on a few lines of the relay's grid size."""
    f = inputs.random_field((4, 4096), seed=7)
    ref = np.fft.fft(f)
    assert np.abs(fft.dft(f) - ref).max() < 1e-11 * np.abs(ref).max()


def test_centred_dft_shift_theorem_4100():
    """Centred DFT of a field shifted by s pixels = the spectrum times exp(-2 pi i s k'/N)."""
    n, s = 4100, 5
    f = inputs.random_field((2, n), seed=3)
    kc = np.arange(n) - n // 2
    a = fft.centred_dft(np.roll(f, s, axis=-1))
    b = fft.centred_dft(f) * np.exp(-2j * np.pi * s * kc / n)
    assert np.abs(a - b).max() < 1e-10 * np.abs(b).max()


def test_centred_dft2_separable_axes():
    """The 2-D transform is rows then columns: a product field f(y) g(x) maps to F(v) G(u)."""
    n = 64
    fy = inputs.random_field((n,), seed=1)
    gx = inputs.random_field((n,), seed=2)
    two_d = propagation.centred_dft2(np.outer(fy, gx))
    np.testing.assert_allclose(two_d, np.outer(fft.centred_dft(fy), fft.centred_dft(gx)), atol=1e-11)
