"""GPU parity: matrix Fourier transform (forward and inverse, batched with per-item sampling)
against the FP64 oracle's direct sums, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import coronagraph, propagation
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu

PRECS = [coro.MFT_FP32]


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.complex128) - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def ctx(lib):
    return coro.Context(0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,npix,m", [(64, 50, 40), (128, 128, 96), (256, 200, 130), (100, 90, 37)])
def test_mft_forward(ctx, n, npix, m, prec):
    du = np.array([0.3, 0.45])
    f = inputs.random_field((2, n, n), seed=n + m)
    x = torch.from_numpy(f.astype(np.complex64)).cuda()
    y = coro.propagate_mft(ctx, x, npix, -1, m, du, prec).cpu().numpy()
    for b in range(2):
        assert rel_l2(y[b], propagation.mft(f[b], npix, m, du[b])) < 1e-5


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m,n,npix", [(40, 64, 50), (130, 256, 200), (37, 100, 90)])
def test_mft_inverse(ctx, m, n, npix, prec):
    du = np.array([0.3, 0.2])
    f = inputs.random_field((2, m, m), seed=m)
    x = torch.from_numpy(f.astype(np.complex64)).cuda()
    y = coro.propagate_mft(ctx, x, npix, +1, n, du, prec).cpu().numpy()
    for b in range(2):
        assert rel_l2(y[b], propagation.imft(f[b], npix, n, du[b])) < 1e-5


def test_mft_lyot_sizes(ctx):
    """1024^2 pupil -> 256^2 at 0.05 lambda/D (the occulter plane of the Lyot workload)."""
    w = inputs.LyotWorkload()
    e = coronagraph.pupil_field(w.n, w.npix, w.wavelength_m, None)
    f = e * inputs.random_field(e.shape, seed=2)
    x = torch.from_numpy(f.astype(np.complex64)).cuda().unsqueeze(0)
    y = coro.propagate_mft(ctx, x, w.npix, -1, w.m_occ, w.du_occ).cpu().numpy()[0]
    assert rel_l2(y, propagation.mft(f, w.npix, w.m_occ, w.du_occ)) < 1e-5
