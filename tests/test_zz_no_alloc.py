"""The allocation-free dark-hole sum (for callers that cannot allocate device memory while
they run) against the ordinary coro_darkhole_sum, through the C ABI, on two calls in a row.

This file is collected last so that a run stopping at its first failure has already run
everything else; it also passes alone in a fresh process.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu


def test_noalloc_darkhole_matches_allocating_path(lib):
    ctx = coro.Context(0)
    batch, n, du = 5, 512, np.array([0.25, 0.3, 0.2, 0.25, 0.5])
    norm = np.array([1.0, 2.5, 0.5, 3.0, 7.0])
    for call in range(2):          # the shared scratch keeps the previous call's sums
        f = inputs.random_field((batch, n, n), seed=40 + call)
        x = torch.from_numpy(f.astype(np.complex64)).cuda()
        ref = coro.darkhole_sum(ctx, x, du, 6.0, 20.0, norm)
        got = coro.darkhole_sum_noalloc(x, du, 6.0, 20.0, norm)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
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
