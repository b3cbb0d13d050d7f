"""GPU parity of the tensor-core MFTs (tcgen05) against the FP64 oracle's direct sums.

Bars (relative L2 over the output field), the same at every size:
* 3xTF32 (hi*hi + hi*lo + lo*hi, FP32 accumulate, every 16-element K slice drained to FP32
  registers): 1e-5, the FP32-path bar. The operands keep ~22 bits and the accumulator truncates
  inside a slice; measured on GB300 5.1e-7 ... 6.5e-7 on every case below.
* 3xBF16: the operands keep ~16 bits; measured 5.1e-6 ... 5.7e-6; held at 1.2e-5, about twice
  the largest.
* EXT (four exact 8-bit BF16 slices, two-float accumulation): measured 3.4e-8 ... 3.8e-8, the
  rounding of the complex64 result; held at 1e-7.
The per-result error is printed."""
import numpy as np
import pytest
import torch

from oracle import propagation
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu

TOL = {coro.MFT_3XTF32: 1e-5, coro.MFT_3XBF16: 1.2e-5, coro.MFT_EXT: 1e-7}
PRECS = [coro.MFT_3XTF32, coro.MFT_3XBF16, coro.MFT_EXT]


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.complex128) - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def ctx(lib):
    c = coro.Context(0)
    yield c
    c.synchronize()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,npix,m", [(64, 50, 40), (256, 200, 130), (100, 90, 37), (1024, 1024, 256)])
def test_tc_mft_forward(ctx, n, npix, m, prec):
    du = np.array([0.3, 0.05 if n == 1024 else 0.45])
    f = inputs.random_field((2, n, n), seed=n + m)
    x = torch.from_numpy(f.astype(np.complex64)).cuda()
    y = coro.propagate_mft(ctx, x, npix, -1, m, du, prec).cpu().numpy()
    ctx.synchronize()
    for b in range(2):
        err = rel_l2(y[b], propagation.mft(f[b], npix, m, du[b]))
        print(f"prec {prec} n {n} m {m} item {b}: rel L2 {err:.3e}")
        assert err < TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m,n,npix", [(40, 64, 50), (130, 256, 200), (256, 1024, 1024)])
def test_tc_mft_inverse(ctx, m, n, npix, prec):
    du = np.array([0.3, 0.2])
    f = inputs.random_field((2, m, m), seed=m)
    x = torch.from_numpy(f.astype(np.complex64)).cuda()
    y = coro.propagate_mft(ctx, x, npix, +1, n, du, prec).cpu().numpy()
    ctx.synchronize()
    for b in range(2):
        err = rel_l2(y[b], propagation.imft(f[b], npix, n, du[b]))
        print(f"prec {prec} m {m} n {n} item {b}: rel L2 {err:.3e}")
        assert err < TOL[prec]


def test_ext_mft_degenerate_inputs(ctx):
    """Extended precision on inputs that stress its per-group scaling: an all-zero field (every
    scaling group empty) gives exact zeros; a centred impulse gives the constant s * v exactly
    (X_j = 0 there, every basis entry 1); a field whose rows span twelve decades keeps the
    oracle's answer to the complex64 rounding of the output."""
    n, npix, m, du = 96, 80, 40, 0.3
    z = torch.zeros((1, n, n), dtype=torch.complex64, device="cuda")
    y = coro.propagate_mft(ctx, z, npix, -1, m, [du], coro.MFT_EXT)
    assert torch.count_nonzero(y).item() == 0
    v = 0.7 - 0.2j
    f = np.zeros((1, n, n), np.complex64)
    f[0, n // 2, n // 2] = v
    y = coro.propagate_mft(ctx, torch.from_numpy(f).cuda(), npix, -1, m, [du], coro.MFT_EXT).cpu().numpy()
    expect = np.complex64(complex(np.complex64(v)) * du / npix)
    assert np.max(np.abs(y - expect)) <= 2.0 ** -23 * abs(expect)
    g = inputs.random_field((1, n, n), seed=77)
    g = g * (10.0 ** np.linspace(-6, 6, n))[None, :, None]
    x = torch.from_numpy(g.astype(np.complex64)).cuda()
    y = coro.propagate_mft(ctx, x, npix, -1, m, [du], coro.MFT_EXT).cpu().numpy()
    err = rel_l2(y[0], propagation.mft(g[0].astype(np.complex64).astype(np.complex128), npix, m, du))
    print(f"EXT twelve-decade rows: rel L2 {err:.3e}")
    assert err < TOL[coro.MFT_EXT]
