"""Textbook discrete Fourier transforms in FP64 (oracle; test infrastructure only).

The paper (Sec. 1.2, Sec. 2.2) spends most of a Fresnel system's time in 2-D FFTs and hands them
to FFT libraries; what those libraries compute is the plain DFT

    F[k] = sum_{j=0}^{N-1} f[j] exp(-2 pi i j k / N),        inverse with +i and 1/N.

This module computes it two ways, both written out here:

* ``dft_direct``   -- the O(N^2) sum itself, as a matrix with the exponent j*k reduced modulo N in
                      exact integer arithmetic before the FP64 exponential.
* ``dft``          -- the iterative radix-2 decimation-in-time Cooley-Tukey FFT (Cooley & Tukey
                      1965; any numerical-methods text): for N = 2^a the input is put into
                      bit-reversed order and a stages of butterflies follow,

                          X[k]     = E[k] + W_{2L}^k O[k]
                          X[k + L] = E[k] - W_{2L}^k O[k],      W_{2L} = exp(-2 pi i / (2L)),

                      with the half-length L doubling from 1 to N/2. For N = 2^a * m with m odd
                      (the non-power-of-two grids of Sec. 3.1, N = 2800, and App. B's npix = 1025
                      padded to N = 4100), the bit reversal acts on the 2^a interleaved
                      subsequences x[r + 2^a t], each of length m is first transformed by the direct
                      sum, and the same butterflies combine them with L running from m to N/2.

Both act along the last axis and vectorise over the leading ones. A library FFT is NOT used here;
the tests cross-check ``dft`` against the brute-force sum, closed forms and, at N = 4096 on a
few lines, numpy's FFT.
"""
from __future__ import annotations

import numpy as np


def _bit_reverse(r: np.ndarray, bits: int) -> np.ndarray:
    out = np.zeros_like(r)
    for b in range(bits):
        out |= ((r >> b) & 1) << (bits - 1 - b)
    return out


def dft_matrix(n: int, sign: int = -1) -> np.ndarray:
    """W[k, j] = exp(sign 2 pi i (j k mod n) / n), the exponent reduced in integers."""
    j = np.arange(n, dtype=np.int64)
    jk = np.outer(j, j) % n
    return np.exp(sign * 2j * np.pi * jk.astype(np.float64) / n)


def dft_direct(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """O(N^2) DFT along the last axis (unnormalised, either sign)."""
    x = np.asarray(x, dtype=np.complex128)
    return x @ dft_matrix(x.shape[-1], sign).T


def dft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Iterative radix-2 DIT FFT along the last axis (unnormalised, either sign); direct sums of
    length m on the odd factor of N. The lines are independent; large batches are transformed
    a few dozen lines at a time (the same arithmetic per line, in cache)."""
    x = np.asarray(x, dtype=np.complex128)
    lines = x.reshape(-1, x.shape[-1]) if x.ndim > 1 else x.reshape(1, -1)
    chunk = max(1, (1 << 19) // max(1, x.shape[-1]))     # about 8 MB of lines at a time
    if lines.shape[0] > chunk:
        out = np.empty_like(lines)
        for i in range(0, lines.shape[0], chunk):
            out[i:i + chunk] = _dft_lines(lines[i:i + chunk], sign)
        return out.reshape(x.shape)
    return _dft_lines(lines, sign).reshape(x.shape)


def _dft_lines(x: np.ndarray, sign: int) -> np.ndarray:
    n = x.shape[-1]
    a = 0
    while n % (2 << a) == 0:
        a += 1
    p, m = 1 << a, n >> a                               # n = p * m, m odd
    lead = x.shape[:-1]
    # subsequence r is x[r + p t], t = 0..m-1; it enters block position bitrev(r)
    sub = x.reshape(lead + (m, p))                      # sub[..., t, r] = x[t p + r]
    sub = np.swapaxes(sub, -1, -2)                      # [..., r, t]
    if m > 1:
        sub = sub @ dft_matrix(m, sign).T               # length-m DFT of every subsequence
    order = _bit_reverse(np.arange(p), a)
    y = np.ascontiguousarray(sub[..., order, :]).reshape(lead + (n,))
    half = m                                            # L: length of the transforms being combined
    while half < n:
        k = np.arange(half, dtype=np.float64)
        w = np.exp(sign * 1j * np.pi * k / half)        # W_{2L}^k
        v = y.reshape(lead + (n // (2 * half), 2, half))  # [..., group, E or O, k]
        o = v[..., 1, :] * w
        v[..., 1, :] = v[..., 0, :] - o
        v[..., 0, :] += o
        half *= 2
    return y


def dft_axis(x: np.ndarray, axis: int, sign: int = -1) -> np.ndarray:
    """``dft`` along any axis."""
    y = np.ascontiguousarray(np.moveaxis(x, axis, -1))
    return np.moveaxis(dft(y, sign), -1, axis)


def centred_dft(x: np.ndarray, axis: int = -1, sign: int = -1) -> np.ndarray:
    """Centred DFT F[k] = sum_j f[j] exp(sign 2 pi i (j - N/2)(k - N/2) / N) along one axis, N
    even: the index shift j -> j - N/2 is a rotation of the input by N/2 and likewise of the
    output (the fftshift of the paper's Sec. 2.4 is this rotation)."""
    n = x.shape[axis]
    if n % 2:
        raise ValueError("centred DFT needs an even length")
    y = np.roll(x, -(n // 2), axis=axis)
    y = dft_axis(y, axis, sign)
    return np.roll(y, n // 2, axis=axis)
