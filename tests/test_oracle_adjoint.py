"""Pins for the oracle's hand-derived adjoint: dot-product identities per operator and
central finite differences of the loss (both independent of the adjoint's own algebra)."""
import numpy as np
import pytest

from oracle import adjoint, coronagraph, propagation
from paper_1806_06467_gb300 import inputs


def inner(a, b):
    return np.vdot(a, b)      # sum conj(a) b


def small_params(n_f=96, npix=32):
    lyot = coronagraph.LyotParams(n=npix, npix=npix, m_occ=20, du_occ=0.35, spot_radius=2.5,
                                  lyot_frac=0.8, m_det=40, du_det=0.5)
    return adjoint.WfcParams(n_f=n_f, npix=npix, diam_m=0.048, z_m=0.3, n_act=8, lyot=lyot,
                             dh_in=3.0, dh_out=9.0)


def test_dot_product_mft_and_imft():
    x = inputs.random_field((24, 24), seed=1)
    y = inputs.random_field((18, 18), seed=2)
    fx = propagation.mft(x, 20, 18, 0.3)
    assert abs(inner(fx, y) - inner(x, propagation.imft(y, 20, 24, 0.3))) < 1e-12 * abs(inner(fx, y))


def test_dot_product_angular_spectrum():
    x = inputs.random_field((32, 32), seed=3)
    y = inputs.random_field((32, 32), seed=4)
    ax = propagation.angular_spectrum(x, 1e-4, 600e-9, 0.7)
    aty = propagation.angular_spectrum(y, 1e-4, 600e-9, -0.7)
    assert abs(inner(ax, y) - inner(x, aty)) < 1e-12 * abs(inner(ax, y))


def test_dot_product_lyot_chain():
    p = small_params().lyot
    x = inputs.random_field((p.n, p.n), seed=5)
    y = inputs.random_field((p.m_det, p.m_det), seed=6)
    lx = coronagraph.lyot_fields(x, p)["det"]
    lty = adjoint.lyot_adjoint(y, p)
    assert abs(inner(lx, y) - inner(x, lty)) < 1e-12 * abs(inner(lx, y))


def test_dot_product_crop_pad():
    x = inputs.random_field((40, 40), seed=7)
    y = inputs.random_field((16, 16), seed=8)
    assert abs(inner(adjoint.crop(x, 16), y) - inner(x, adjoint.pad(y, 40))) < 1e-12


@pytest.mark.parametrize("lam", [525e-9, 575e-9])
def test_gradient_matches_central_differences(lam):
    """dL/dh from the adjoint vs (L(h + d) - L(h - d)) / 2d with d = 1e-3 nm."""
    p = small_params()
    h = inputs.dm_heights(3, p.n_act, 2)
    peak = adjoint.forward(np.zeros_like(h), lam, p)["peak"]
    loss, grad = adjoint.gradient(h, lam, p, peak=peak)
    d = 1e-12
    picks = inputs.actuator_offsets(4, p.n_act, 6)
    for dm, r, c in picks:
        hp = h.copy(); hp[dm, r, c] += d
        hm = h.copy(); hm[dm, r, c] -= d
        fd = (adjoint.forward(hp, lam, p, peak=peak)["loss"]
              - adjoint.forward(hm, lam, p, peak=peak)["loss"]) / (2 * d)
        assert abs(grad[dm, r, c] - fd) <= 1e-6 * np.abs(grad).max(), (dm, r, c)


def test_broadband_gradient_is_sum():
    p = small_params(n_f=64, npix=32)
    h = inputs.dm_heights(9, p.n_act, 2)
    lams = [530e-9, 560e-9]
    total, grad, peaks = adjoint.broadband_gradient(h, lams, p)
    l0, g0 = adjoint.gradient(h, lams[0], p, peak=peaks[0])
    l1, g1 = adjoint.gradient(h, lams[1], p, peak=peaks[1])
    assert abs(total - l0 - l1) < 1e-15 * abs(total) + 1e-30
    np.testing.assert_allclose(grad, g0 + g1, rtol=1e-14, atol=0)
