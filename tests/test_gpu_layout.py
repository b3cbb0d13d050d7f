"""GPU parity: the alternating plane layout of the fused Fresnel plan (a column pass writes its
result transposed into a plan-owned plane, the next row pass reads it back column-wise) against
the FP64 oracle and against the natural in-place layout, through the C ABI.

Tolerance: relative L2 <= 1e-5 against the oracle (complex64), and <= 1e-6 between the two
layouts (the same FP32 arithmetic in another kernel family: rounding order only).
"""
import numpy as np
import pytest
import torch

from paper_1806_06467_gb300 import coro, inputs
from test_gpu_fresnel import rel_l2, relay_elements, relay_oracle, relay_oracle_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(lib):
    return coro.Context(0)


def relay_plan(ctx, w, maps_t, batch=1, wavelengths=None, extra=None):
    els = relay_elements(w, maps_t) if extra is None else extra
    return coro.FresnelPlan(ctx, n=w.n, batch=batch, pixelscale=w.dx,
                            wavelength=w.wavelength_m if wavelengths is None else wavelengths,
                            distances=list(w.distances()), elements=els, init_uniform=True)


def names(plan):
    return [plan.pass_kernel(i) for i in range(plan.launch_count)]


@pytest.mark.parametrize("n", [1024, 2048, 4096])
def test_alternating_layout_relay(ctx, n):
    """Six-plane relay on both layouts: the oracle's field to 1e-5 (1024, 2048; 4096 against
    the natural layout only), the layouts within 1e-6 of each other, and the kernels each
    layout reports."""
    w = inputs.RelayWorkload(n=n, npix=n // 2 if n < 4096 else 1024, seed=5)
    maps = [m.astype(np.float32) for m in w.psd_maps()]
    maps_t = [torch.from_numpy(m).cuda() for m in maps]
    plan = relay_plan(ctx, w, maps_t)
    out = {}
    for alt in (True, False):
        plan.set_layout(alt)
        assert plan.layout == alt
        k = names(plan)
        assert any("_pair_t" in x for x in k) == alt, k
        x = torch.full((1, n, n), float("nan"), dtype=torch.complex64, device="cuda")
        plan.execute(x)
        out[alt] = x.cpu().numpy()[0]
    d = rel_l2(out[True], out[False].astype(np.complex128))
    print(f"n {n}: alternating vs natural rel L2 {d:.2e}")
    assert d < 1e-6
    if n < 4096:
        ref = relay_oracle(w, maps)
        assert rel_l2(out[True], ref) < 1e-5


def test_alternating_layout_batch_of_wavelengths(ctx):
    """Two items at different wavelengths (item offsets in the transposed plane and its TMA
    boxes) at 4096^2: alternating equals natural per item."""
    n = 4096
    w = inputs.RelayWorkload(n=n, npix=1024, seed=6)
    maps_t = [torch.from_numpy(m.astype(np.float32)).cuda() for m in w.psd_maps()]
    plan = relay_plan(ctx, w, maps_t, batch=2, wavelengths=[550e-9, 610e-9])
    res = {}
    for alt in (True, False):
        plan.set_layout(alt)
        x = torch.full((2, n, n), float("nan"), dtype=torch.complex64, device="cuda")
        plan.execute(x)
        res[alt] = x.cpu().numpy()
    for b in range(2):
        d = rel_l2(res[True][b], res[False][b].astype(np.complex128))
        assert d < 1e-6, (b, d)
    assert rel_l2(res[True][0], res[True][1].astype(np.complex128)) > 1e-3   # the items differ


def test_alternating_layout_checkpoints_and_taps(ctx):
    """Checkpoints and the phase-gradient tap inside row passes that read the transposed
    plane: stored planes match the oracle's per-plane fields, as on the natural layout."""
    n = 1024
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=4)
    maps = [m.astype(np.float32) for m in w.psd_maps()]
    maps_t = [torch.from_numpy(m).cuda() for m in maps]
    cps = [torch.zeros((1, n, n), dtype=torch.complex64, device="cuda") for _ in range(3)]
    tap = torch.zeros((1, n, n), dtype=torch.float32, device="cuda")
    g = torch.from_numpy(np.exp(1j * np.linspace(0, 3, n * n)).reshape(1, n, n).astype(np.complex64)).cuda()
    els = relay_elements(w, maps_t)
    els = [els[0], els[1],
           coro.element(coro.EL_CHECKPOINT, plane=2, store=cps[0]), els[2], els[3],
           coro.element(coro.EL_PHASE_GRAD, plane=4, store=tap, ref=g, scalar=1.0),
           els[4], coro.element(coro.EL_CHECKPOINT, plane=4, store=cps[1]), els[5],
           coro.element(coro.EL_CHECKPOINT, plane=5, store=cps[2])]
    plan = relay_plan(ctx, w, maps_t, extra=els)
    ref = relay_oracle_planes(w, maps)
    want = [ref[2][0], ref[4][1], ref[5][1]]
    got = {}
    for alt in (True, False):
        plan.set_layout(alt)
        for c in cps:
            c.fill_(float("nan"))
        tap.fill_(float("nan"))
        x = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
        plan.execute(x)
        for i, (c, r) in enumerate(zip(cps, want)):
            assert rel_l2(c.cpu().numpy()[0], r) < 1e-5, (alt, i)
        assert torch.equal(cps[2], x)
        got[alt] = tap.cpu().numpy()[0].astype(np.float64)
    assert np.all(np.isfinite(got[True]))
    assert np.linalg.norm(got[True] - got[False]) <= 1e-5 * np.linalg.norm(got[False])


def test_alternating_layout_graph_and_ranges(ctx):
    """Graph replay on the alternating layout is bitwise the eager result; execute_range runs
    every pass in place (natural layout), so the ranges in order agree to rounding; switching
    layouts or kernels resets the plan as documented."""
    n = 1024
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=7)
    maps_t = [torch.from_numpy(m.astype(np.float32)).cuda() for m in w.psd_maps()]
    plan = relay_plan(ctx, w, maps_t)
    plan.set_layout(True)
    eager = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    plan.execute(eager)
    plan.use_graph(True)
    x = torch.empty_like(eager)
    for _ in range(3):
        x.fill_(float("nan"))
        plan.execute(x)
        assert torch.equal(x, eager)
    plan.use_graph(False)
    y = torch.empty_like(eager)
    for i in range(plan.launch_count):
        plan.execute_range(y, i, 1)
    assert rel_l2(y.cpu().numpy()[0], eager.cpu().numpy()[0].astype(np.complex128)) < 1e-6
    plan.set_pass_kernel(1, 0)
    assert not plan.layout and not any("_pair_t" in k for k in names(plan))


def test_alternating_layout_refused_where_unsupported(ctx):
    """complex128 plans and sizes outside 1024-4096 have no alternating layout: CORO_ENOTIMPL
    and the plan stays on the natural layout."""
    for n, dtype in ((512, coro.C64), (1024, coro.C128)):
        w = inputs.RelayWorkload(n=n, npix=n // 2, seed=8)
        maps_t = [torch.from_numpy(m.astype(np.float32)).cuda() for m in w.psd_maps()]
        plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                                distances=list(w.distances()), elements=relay_elements(w, maps_t),
                                init_uniform=True, dtype=dtype)
        with pytest.raises(coro.CoroError):
            plan.set_layout(True)
        assert not plan.layout


def test_plan_tuning_leaves_caller_buffers_alone(ctx):
    """The plan-time tuner (kernel candidates, row variants over every pass, layouts) runs on
    a scratch field with the checkpoint and tap elements left out: buffers those elements
    write keep their contents until the first execute."""
    n = 1024
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=9)
    maps_t = [torch.from_numpy(m.astype(np.float32)).cuda() for m in w.psd_maps()]
    cp = torch.full((1, n, n), 7.0 + 3.0j, dtype=torch.complex64, device="cuda")
    tap = torch.full((1, n, n), -5.0, dtype=torch.float32, device="cuda")
    els = relay_elements(w, maps_t)
    els = els[:3] + [coro.element(coro.EL_CHECKPOINT, plane=2, store=cp),
                     coro.element(coro.EL_PHASE_GRAD, plane=3, store=tap, scalar=1.0)] + els[3:]
    plan = relay_plan(ctx, w, maps_t, extra=els)
    torch.cuda.synchronize()
    assert bool((cp == (7.0 + 3.0j)).all()) and bool((tap == -5.0).all())
    x = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    plan.execute(x)
    assert not bool((cp == (7.0 + 3.0j)).any()) and bool(torch.isfinite(tap).all())


def test_copy_tuning(ctx):
    """A second plan of the same system takes the first one's kernels and layout; plans of
    another size or pass sequence are refused and left unchanged."""
    n = 1024
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=10)
    maps_t = [torch.from_numpy(m.astype(np.float32)).cuda() for m in w.psd_maps()]
    a = relay_plan(ctx, w, maps_t)
    b = relay_plan(ctx, w, maps_t)
    a.set_pass_kernel(2, -1)                             # units rows, persistent columns
    a.set_layout(True)
    b.copy_tuning(a)
    assert names(b) == names(a) and b.layout
    x, y = (torch.empty((1, n, n), dtype=torch.complex64, device="cuda") for _ in range(2))
    a.execute(x)
    b.execute(y)
    assert torch.equal(x, y)
    a.set_layout(False)
    b.copy_tuning(a)
    assert names(b) == names(a) and not b.layout
    w2 = inputs.RelayWorkload(n=2048, npix=1024, seed=10)
    maps2 = [torch.from_numpy(m.astype(np.float32)).cuda() for m in w2.psd_maps()]
    c = relay_plan(ctx, w2, maps2)
    before = names(c)
    with pytest.raises(coro.CoroError):
        c.copy_tuning(a)
    assert names(c) == before


def test_pass_flops(ctx):
    """FFT arithmetic per pass: two line transforms in every column pass and interior row pass,
    one in the first (uniform start, forward only) and the last (inverse only) row pass."""
    n = 1024
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=11)
    maps_t = [torch.from_numpy(m.astype(np.float32)).cuda() for m in w.psd_maps()]
    plan = relay_plan(ctx, w, maps_t)
    one = 5.0 * n * np.log2(n) * n
    f = [plan.pass_flops(i) for i in range(plan.launch_count)]
    assert f[0] == one and f[-1] == one
    assert all(x == 2 * one for x in f[1:-1])
