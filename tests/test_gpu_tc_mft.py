"""GPU parity of the split-precision tensor-core MFT (tcgen05, 3xTF32 and 3xBF16, FP32
accumulate) against the FP64 oracle's direct sums.

Tolerances (relative L2 over the output field). Operand splitting: 3xTF32 keeps ~22
significant bits per product (dropped lo*lo term 2^-22), 3xBF16 ~16 bits (2^-16). On top,
the tensor-core FP32 accumulator rounds every update of a K = 8 (TF32) / 16 (BF16) slice
product, six updates per slice for the complex split product, each up to one FP32 ulp of the
running sum with a common sign, so the relative error can grow linearly in K: about
2^-23 * 6/8 * K ~ 9e-8 K for a chain of two GEMMs. The bar is max(1e-5, 6e-8 K) for TF32 and
max(1e-4, 6e-8 K) for BF16, K the longest inner length; the per-result error is printed."""
import numpy as np
import pytest
import torch

from oracle import propagation
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu

TOL = {coro.MFT_3XTF32: 1e-5, coro.MFT_3XBF16: 1e-4}


def tol(prec, k):
    return max(TOL[prec], 6e-8 * k)


def rel_l2(got, ref):
    return float(np.linalg.norm(np.asarray(got, np.complex128) - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def ctx(lib):
    c = coro.Context(0)
    yield c
    c.synchronize()


@pytest.mark.parametrize("prec", [coro.MFT_3XTF32, coro.MFT_3XBF16])
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
        assert err < tol(prec, n)


@pytest.mark.parametrize("prec", [coro.MFT_3XTF32, coro.MFT_3XBF16])
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
        assert err < tol(prec, m)
