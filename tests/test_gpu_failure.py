"""Failure detection without a GPU fault: a bounded device-side wait that nothing completes
expires, raises the context's error flag, and the context stays usable."""
import numpy as np
import pytest
import torch

from oracle import optics, propagation
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return coro.Context(0)


def test_expired_wait_is_reported_and_context_survives(ctx):
    ctx.synchronize()                                  # clean state
    ctx.lib.check(ctx.lib.coro_selftest_wait_timeout(ctx.handle, 1000))
    with pytest.raises(coro.CoroError) as ei:
        ctx.synchronize()
    assert ei.value.status == coro.ETIMEOUT
    ctx.synchronize()                                  # the flag was cleared
    # the context still propagates correctly
    n, dx, lam = 256, 1.0 / 128, 550e-9
    e = inputs.random_field((n, n), seed=9) * optics.circular_aperture(n, dx, 0.5)
    x = torch.from_numpy(e.astype(np.complex64)).cuda().unsqueeze(0).contiguous()
    coro.propagate_fresnel(ctx, x, dx, lam, 2.0, coro.FRESNEL_AS)
    ctx.synchronize()
    ref = propagation.angular_spectrum(e, dx, lam, 2.0)
    got = x.cpu().numpy()[0].astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_selftest_rejects_bad_bounds(ctx):
    with pytest.raises(coro.CoroError):
        ctx.lib.check(ctx.lib.coro_selftest_wait_timeout(ctx.handle, 0))
