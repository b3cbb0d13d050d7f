"""The allocation-free dark-hole sum (for callers that cannot allocate device memory while
they run) against the ordinary coro_darkhole_sum and against the FP64 oracle's dark-hole sum,
through the C ABI, on two calls in a row, for complex64 and complex128 fields, on torch's
current stream and on a stream of its own.

This file is collected last so that a run stopping at its first failure has already run
everything else; it also passes alone in a fresh process.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from oracle import coronagraph
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("own_stream", [False, True])
def test_noalloc_darkhole_matches_allocating_path_and_oracle(lib, dtype, own_stream):
    ctx = coro.Context(0)
    batch, n, du = 5, 512, np.array([0.25, 0.3, 0.2, 0.25, 0.5])
    norm = np.array([1.0, 2.5, 0.5, 3.0, 7.0])
    stream = torch.cuda.Stream() if own_stream else None
    for call in range(2):          # the shared scratch keeps the previous call's sums
        f = inputs.random_field((batch, n, n), seed=40 + call).astype(dtype)
        x = torch.from_numpy(f).cuda()
        ref = coro.darkhole_sum(ctx, x, du, 6.0, 20.0, norm)
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                got = coro.darkhole_sum_noalloc(x, du, 6.0, 20.0, norm, stream=stream)
        else:
            got = coro.darkhole_sum_noalloc(x, du, 6.0, 20.0, norm)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
        f64 = f.astype(np.complex128)
        oracle = [coronagraph.dark_hole_sum(coronagraph.intensity(f64[b], norm[b]), du[b], 6.0, 20.0)
                  for b in range(batch)]
        np.testing.assert_allclose(got, oracle, rtol=1e-10, atol=0)
        assert np.all(got > 0)


def test_noalloc_rejects_batch_over_limit(lib):
    x = torch.zeros((1, 32, 32), dtype=torch.complex64, device="cuda")
    w = coro.WF(x)
    w.s.batch = 1025                     # beyond CORO_NOALLOC_MAX_BATCH; rejected on the host
    du = (ct.c_double * 1025)(*([0.25] * 1025))
    out = (ct.c_double * 1025)()
    st = lib.coro_darkhole_sum_noalloc(ct.byref(w.s), du, 6.0, 20.0, None, None, out)
    assert st == coro.ESIZE
    assert b"1024" in lib.coro_last_error()


def test_noalloc_rejects_field_on_another_device(lib):
    """A field on device 1 while device 0 is current is rejected on the host (needs two GPUs)."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    x = torch.ones((1, 64, 64), dtype=torch.complex64, device="cuda:1")
    w = coro.WF(x)
    du = (ct.c_double * 1)(0.25)
    out = (ct.c_double * 1)()
    with torch.cuda.device(0):
        st = lib.coro_darkhole_sum_noalloc(ct.byref(w.s), du, 6.0, 20.0, None, None, out)
    assert st == coro.EINVAL
    assert b"device" in lib.coro_last_error()
