"""GPU parity: centred 2-D DFT, Fresnel hops, elements and the fused Fresnel plan against
the FP64 oracle, element by element, through the C ABI.

Tolerance: relative L2 field error <= 1e-5 for complex64 and <= 1e-12 for complex128. Binary
masks are compared exactly (which samples are zeroed).
"""
import numpy as np
import pytest
import torch

from oracle import optics, propagation
from paper_1806_06467_gb300 import coro, inputs

pytestmark = pytest.mark.gpu

TOL = {torch.complex64: 1e-5, torch.complex128: 1e-12}
EPS64 = np.finfo(np.float64).eps


def tol(dtype, phase_max=0.0):
    """complex64: 1e-5. complex128: 1e-12, widened by the rounding the FP64 oracle itself
    commits when it evaluates a quadratic phase of magnitude phase_max (Sec. 2.3: these
    arguments reach 1e6-1e7 rad), i.e. a few eps * |phase|."""
    if dtype == torch.complex64:
        return TOL[dtype]
    return TOL[dtype] + 8 * EPS64 * phase_max


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def to_dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda().contiguous()


@pytest.fixture(scope="module")
def ctx(lib):
    return coro.Context(0)


SIZES = [32, 64, 128, 256, 512, 1024, 2048]


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("n", SIZES)
def test_centred_dft_forward_inverse(ctx, n, dtype):
    batch = 2
    f = inputs.random_field((batch, n, n), seed=n)
    x = to_dev(f, dtype)
    coro.fft2(ctx, x, -1)
    ref = propagation.centred_dft2(f)
    assert rel_l2(x.cpu().numpy(), ref) < TOL[dtype]
    coro.fft2(ctx, x, +1)
    assert rel_l2(x.cpu().numpy(), f) < TOL[dtype]


@pytest.mark.parametrize("n", [4096, 8192])
def test_centred_dft_large(ctx, n):
    f = inputs.random_field((1, n, n), seed=7)
    x = to_dev(f, torch.complex64)
    coro.fft2(ctx, x, -1)
    assert rel_l2(x.cpu().numpy(), propagation.centred_dft2(f)) < 1e-5


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("n", [64, 256, 1024])
def test_angular_spectrum_hop(ctx, n, dtype):
    lams = np.array([500e-9, 600e-9])
    dxs = np.array([1.0 / 200, 1.3 / 200])
    f = inputs.random_field((2, n, n), seed=3 * n)
    x = to_dev(f, dtype)
    ps = coro.propagate_fresnel(ctx, x, dxs, lams, 2.7, coro.FRESNEL_AS)
    np.testing.assert_array_equal(ps, dxs)
    got = x.cpu().numpy()
    for b in range(2):
        ref = propagation.angular_spectrum(f[b], dxs[b], lams[b], 2.7)
        assert rel_l2(got[b], ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("n", [64, 512])
def test_direct_fresnel_hop(ctx, n, dtype):
    lams = np.array([500e-9, 550e-9])
    dx = 1.0 / 128
    f = inputs.random_field((2, n, n), seed=5 * n)
    x = to_dev(f, dtype)
    ps = coro.propagate_fresnel(ctx, x, dx, lams, -3.5, coro.FRESNEL_DIRECT)
    got = x.cpu().numpy()
    for b in range(2):
        ref, du = propagation.direct_fresnel(f[b], dx, lams[b], -3.5)
        assert abs(ps[b] - abs(du)) < 1e-15 * abs(du)
        r2max = 2 * (n / 2) ** 2 * max(dx, abs(du)) ** 2
        assert rel_l2(got[b], ref) < tol(dtype, np.pi * r2max / (lams[b] * 3.5))


def apply(ctx, n, dtype, el, dx=1.0 / 300, lam=550e-9, batch=1, seed=0):
    f = inputs.random_field((batch, n, n), seed=seed)
    x = to_dev(f, dtype)
    coro.apply_element(ctx, x, dx, lam, el)
    return f, x.cpu().numpy()


@pytest.mark.parametrize("n", [256, 1024])
def test_aperture_mask_exact(ctx, n):
    dx = 1.0 / (n // 2 - 1)   # a pitch with no exact binary representation
    el = coro.element(coro.EL_APERTURE, radius=0.5, obscuration=0.3, n_spiders=4, spider_width=0.01)
    f, got = apply(ctx, n, torch.complex64, el, dx=dx)
    mask = optics.circular_aperture(n, dx, 0.5, 0.3, 4, 0.01)
    np.testing.assert_array_equal(got[0] == 0, mask == 0)
    np.testing.assert_array_equal(got[0][mask == 1], f[0][mask == 1].astype(np.complex64))


@pytest.mark.parametrize("opaque", [False, True])
def test_circle_stop_exact(ctx, opaque):
    n, dx = 512, 1.0 / 200
    el = coro.element(coro.EL_CIRCLE, radius=0.45, flags=coro.ELF_OPAQUE_INSIDE if opaque else 0)
    f, got = apply(ctx, n, torch.complex64, el, dx=dx)
    mask = optics.circle_stop(n, dx, 0.45, opaque_inside=opaque)
    np.testing.assert_array_equal(got[0] == 0, mask == 0)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_lens(ctx, dtype):
    n, dx, lam, fl = 1024, 1.0 / 400, 550e-9, 5.0
    f, got = apply(ctx, n, dtype, coro.element(coro.EL_LENS, focal_length=fl), dx=dx, lam=lam)
    ref = f[0] * optics.thin_lens(n, dx, lam, fl)
    phase_max = np.pi * 2 * (n / 2 * dx) ** 2 / (lam * fl)
    assert rel_l2(got[0], ref) < (2e-7 if dtype == torch.complex64 else tol(dtype, phase_max))


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_opd_map_and_amplitude(ctx, dtype):
    n, lam = 256, 600e-9
    opd = inputs.psd_surface(n, 4) * 10
    amp = inputs.rng(2).uniform(0.5, 1.0, (n, n))
    opd_t = torch.from_numpy(opd.astype(np.float32)).cuda()
    amp_t = torch.from_numpy(amp.astype(np.float32)).cuda()
    el = coro.element(coro.EL_OPD_MAP, opd=opd_t, amplitude=amp_t)
    f, got = apply(ctx, n, dtype, el, lam=lam)
    ref = f[0] * optics.phasor(opd.astype(np.float32), lam, amp.astype(np.float32))
    assert rel_l2(got[0], ref) < (1e-6 if dtype == torch.complex64 else TOL[dtype])


def test_opd_map_batched(ctx):
    n, lams = 128, np.array([500e-9, 700e-9, 650e-9])
    opd = np.stack([inputs.psd_surface(n, s) for s in range(3)]).astype(np.float32)
    el = coro.element(coro.EL_OPD_MAP, opd=torch.from_numpy(opd).cuda(), flags=coro.ELF_MAP_BATCHED)
    f = inputs.random_field((3, n, n), seed=1)
    x = to_dev(f, torch.complex64)
    coro.apply_element(ctx, x, 1e-3, lams, el)
    got = x.cpu().numpy()
    for b in range(3):
        assert rel_l2(got[b], f[b] * optics.phasor(opd[b], lams[b])) < 1e-6


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_zernike(ctx, dtype):
    n, dx, lam = 512, 1.0 / 500, 550e-9
    c = inputs.zernike_coefficients(3, 4, 21, 50e-9)
    el = coro.element(coro.EL_ZERNIKE, radius=0.5, coeffs=c, j_first=4)
    f, got = apply(ctx, n, dtype, el, dx=dx, lam=lam)
    ref = f[0] * optics.phasor(optics.zernike_opd(n, dx, 0.5, c, 4), lam)
    assert rel_l2(got[0], ref) < (1e-6 if dtype == torch.complex64 else TOL[dtype])


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
@pytest.mark.parametrize("axis", [0, 1])
def test_sine_wfe(ctx, axis, dtype):
    n, dx, lam = 2048, 0.04 / 256, 0.5e-6
    el = coro.element(coro.EL_SINE, sine_freq=500.0, sine_amplitude=5e-9, axis=axis)
    f, got = apply(ctx, n, dtype, el, dx=dx, lam=lam)
    ref = f[0] * optics.phasor(optics.sine_wfe(n, dx, 500.0, 5e-9, axis=1 if axis == 0 else 0), lam)
    assert rel_l2(got[0], ref) < (1e-6 if dtype == torch.complex64 else TOL[dtype])


def test_scalar_and_init(ctx):
    x = torch.empty((2, 64, 64), dtype=torch.complex64, device="cuda")
    coro.wavefront_init(ctx, x, 1.0)
    coro.apply_element(ctx, x, 1e-3, 5e-7, coro.element(coro.EL_SCALAR, scalar=0.25))
    assert torch.all(x == 0.25)
    f, got = apply(ctx, 64, torch.complex128, coro.element(coro.EL_SCALAR, scalar=0.1))
    assert rel_l2(got[0], f[0] * 0.1) < 1e-15                 # 0.1 is not a float: FP64 scalar


# ------------------------------------------------------------------------------ fused plan

def relay_elements(w, maps):
    r = w.diam_m / 2
    return [
        coro.element(coro.EL_APERTURE, plane=0, radius=r, obscuration=w.obscuration,
                     n_spiders=w.n_spiders, spider_width=w.spider_width_frac * w.diam_m),
        coro.element(coro.EL_LENS, plane=1, focal_length=w.lens1_m),
        coro.element(coro.EL_OPD_MAP, plane=2, opd=maps[0]),
        coro.element(coro.EL_LENS, plane=3, focal_length=w.lens2_m),
        coro.element(coro.EL_OPD_MAP, plane=4, opd=maps[1]),
        coro.element(coro.EL_CIRCLE, plane=5, radius=w.field_stop_frac * r),
    ]


def relay_oracle(w, maps_np):
    n, dx, lam = w.n, w.dx, w.wavelength_m
    r = w.diam_m / 2
    els = [optics.circular_aperture(n, dx, r, w.obscuration, w.n_spiders, w.spider_width_frac * w.diam_m),
           optics.thin_lens(n, dx, lam, w.lens1_m),
           optics.phasor(maps_np[0], lam),
           optics.thin_lens(n, dx, lam, w.lens2_m),
           optics.phasor(maps_np[1], lam),
           optics.circle_stop(n, dx, w.field_stop_frac * r)]
    return propagation.fresnel_chain(np.ones((n, n), complex), dx, lam, els, list(w.distances()))


@pytest.mark.parametrize("n", [256, 2048])
def test_relay_chain_plan(ctx, n):
    """Six-plane relay (obscured spidered aperture, two lenses, two PSD surfaces, field
    stop), five angular-spectrum hops of 0.5-5 m, fused into 11 passes."""
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=1)
    maps = [m.astype(np.float32) for m in w.psd_maps()]
    maps_t = [torch.from_numpy(m).cuda() for m in maps]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=relay_elements(w, maps_t),
                            init_uniform=True)
    assert plan.launch_count == 11
    x = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    plan.execute(x)
    ref = relay_oracle(w, maps)
    assert rel_l2(x.cpu().numpy()[0], ref) < 1e-5


@pytest.mark.slow
def test_relay_chain_plan_4096(ctx):
    """The full-size relay at 4096^2 (the benchmarked configuration), whole field."""
    w = inputs.RelayWorkload(n=4096, npix=1024, seed=0)
    maps = [m.astype(np.float32) for m in w.psd_maps()]
    maps_t = [torch.from_numpy(m).cuda() for m in maps]
    plan = coro.FresnelPlan(ctx, n=4096, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=relay_elements(w, maps_t),
                            init_uniform=True)
    x = torch.empty((1, 4096, 4096), dtype=torch.complex64, device="cuda")
    plan.execute(x)
    ref = relay_oracle(w, maps)
    assert rel_l2(x.cpu().numpy()[0], ref) < 1e-5


def test_relay_graph_replay_matches_eager(ctx):
    """a10: the relay plan replayed as one CUDA graph gives bitwise the eager result, for the
    captured field and after a re-capture on a new field."""
    n = 512
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=3)
    maps = [torch.from_numpy(m.astype(np.float32)).cuda() for m in w.psd_maps()]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=relay_elements(w, maps), init_uniform=True)
    eager = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    plan.execute(eager)
    plan.use_graph(True)
    x = torch.empty_like(eager)
    for _ in range(3):
        x.fill_(float("nan"))
        plan.execute(x)
        assert torch.equal(x, eager)
    y = torch.empty_like(eager)
    plan.execute(y)
    assert torch.equal(y, eager)
    # K executes in one graph with per-pass events recorded inside it
    plan.set_timing(3)
    for _ in range(2):                                  # capture, then replay
        y.fill_(float("nan"))
        plan.execute_n(y, 3)
        assert torch.equal(y, eager)                    # the plan starts from a uniform field
    t = plan.unit_times(3)
    assert t.shape == (3, plan.launch_count) and np.all(t > 0)
    plan.set_timing(0)
    plan.use_graph(False)
    plan.execute_n(y, 2)                                # eager path of execute_n
    assert torch.equal(y, eager)


KERNEL_CHOICES = {
    # n: (row variants, column kernels) the complex64 plan offers
    1024: ([0, 1, 2, 3, 5], [16, 8, -1, -2, -3, -4, -7, -8]),
    2048: ([0, 1, 2, 3, 5], [8, 4, -1, -2, -3, -4, -7, -8]),
    4096: ([0, 1, 2, 3, 5], [4, 2, -1, -2, -3, -4, -7, -8]),
}


def _relay_all_kernels(ctx, n, npix, seed):
    w = inputs.RelayWorkload(n=n, npix=npix, seed=seed)
    maps = [m.astype(np.float32) for m in w.psd_maps()]
    maps_t = [torch.from_numpy(m).cuda() for m in maps]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=relay_elements(w, maps_t),
                            init_uniform=True)
    ref = relay_oracle(w, maps)
    rows, cols = KERNEL_CHOICES[n]
    x = torch.empty((1, n, n), dtype=torch.complex64, device="cuda")
    seen = set()
    # every row kernel with one column kernel, every column kernel with one row kernel
    combos = [(rv, cols[0]) for rv in rows] + [(rows[0], cl) for cl in cols[1:]]
    r16 = {1024: [16, 16, 4], 2048: [16, 16, 8], 4096: [16, 16, 16]}[n]
    r8 = {1024: [8, 8, 8, 2], 2048: [8, 8, 8, 4], 4096: [8, 8, 8, 8]}[n]
    for rv, cl in combos:
        plan.set_pass_kernel(rv, cl)
        names = {plan.pass_kernel(i) for i in range(plan.launch_count)}
        seen |= names
        for i in range(plan.launch_count):            # the FFT factorisation each pass runs
            row, _ = plan.pass_info(i)
            assert plan.pass_radix(i) == (r8 if (rv == 5 if row else cl == -8) else r16), (rv, cl, i)
        x.fill_(float("nan"))
        plan.execute(x)
        err = rel_l2(x.cpu().numpy()[0], ref)
        assert err < 1e-5, (rv, cl, sorted(names), err)
    with pytest.raises(RuntimeError):
        plan.set_pass_kernel(4, 0)                     # the transposed-input row kernel is not a choice
    with pytest.raises(RuntimeError):
        plan.set_pass_kernel(0, 3)
    return seen


@pytest.mark.parametrize("n", [1024, 2048])
def test_relay_every_pass_kernel(ctx, n):
    """Every row and column kernel the plan can pick (per-group, persistent, unit-pipelined,
    packed pairs, wide, quad, and the radix-8 shared-memory engine: a second factorisation of
    the power-of-two lengths) gives the oracle's relay to 1e-5 relative L2, and reports its
    radix sequence."""
    seen = _relay_all_kernels(ctx, n, n // 2, seed=2)
    assert any("_units" in k for k in seen) and any("_persistent" in k for k in seen)


@pytest.mark.slow
def test_relay_every_pass_kernel_4096(ctx):
    """The same at 4096^2, the benchmarked size (one oracle run, nine kernel pairs)."""
    seen = _relay_all_kernels(ctx, 4096, 1024, seed=0)
    assert "row_pass_units<4096>" in seen and "col_pass_units<4096,2>" in seen and "col_pass_pair<4096,2>" in seen
    assert "col_pass_wide<4096,4>" in seen and "row_pass_pair<4096>" in seen and "col_pass_quad<4096,4>" in seen
    assert "row_pass_mixed_r8<4096>" in seen and any(k.startswith("col_pass_mixed_r8<4096,") for k in seen)


def relay_oracle_planes(w, maps_np):
    """The relay's field at every plane: (before, after) the plane's element."""
    n, dx, lam = w.n, w.dx, w.wavelength_m
    r = w.diam_m / 2
    els = [optics.circular_aperture(n, dx, r, w.obscuration, w.n_spiders, w.spider_width_frac * w.diam_m),
           optics.thin_lens(n, dx, lam, w.lens1_m),
           optics.phasor(maps_np[0], lam),
           optics.thin_lens(n, dx, lam, w.lens2_m),
           optics.phasor(maps_np[1], lam),
           optics.circle_stop(n, dx, w.field_stop_frac * r)]
    e = np.ones((n, n), complex)
    out = []
    for p, z in enumerate(list(w.distances()) + [None]):
        before = e
        e = e * els[p]
        out.append((before, e))
        if z is not None:
            e = propagation.angular_spectrum(e, dx, lam, z)
    return out


@pytest.mark.parametrize("n,dtype", [(256, torch.complex128), (1024, torch.complex64)])
def test_checkpoint_elements(ctx, n, dtype):
    """Per-plane checkpoints inside the fused relay plan: after the aperture (first row pass),
    before and after a PSD surface (mid-chain row passes, whose field carries the fftshift
    sign), after the field stop (last pass: equal to the output). Every row kernel."""
    w = inputs.RelayWorkload(n=n, npix=n // 2, seed=4)
    maps = [m.astype(np.float32) for m in w.psd_maps()]
    maps_t = [torch.from_numpy(m).cuda() for m in maps]
    cps = [torch.zeros((1, n, n), dtype=dtype, device="cuda") for _ in range(4)]
    els = relay_elements(w, maps_t)
    els = [els[0], coro.element(coro.EL_CHECKPOINT, plane=0, store=cps[0]), els[1],
           coro.element(coro.EL_CHECKPOINT, plane=2, store=cps[1]), els[2], els[3], els[4],
           coro.element(coro.EL_CHECKPOINT, plane=4, store=cps[2]), els[5],
           coro.element(coro.EL_CHECKPOINT, plane=5, store=cps[3])]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=w.dx, wavelength=w.wavelength_m,
                            distances=list(w.distances()), elements=els, init_uniform=True,
                            dtype=coro.C128 if dtype == torch.complex128 else coro.C64)
    assert plan.launch_count == 11
    ref = relay_oracle_planes(w, maps)
    want = [ref[0][1], ref[2][0], ref[4][1], ref[5][1]]
    x = torch.empty((1, n, n), dtype=dtype, device="cuda")
    r_max = np.sqrt(2) * (n / 2) * w.dx                  # the lenses' largest quadratic phase
    bound = tol(dtype, np.pi * r_max ** 2 / (w.wavelength_m * min(w.lens1_m, w.lens2_m)))
    rows = KERNEL_CHOICES[n][0] if n in KERNEL_CHOICES and dtype == torch.complex64 else [None]
    for rv in rows:
        if rv is not None:
            plan.set_pass_kernel(rv, 0)
        for c in cps:
            c.fill_(float("nan"))
        plan.execute(x)
        for i, (c, r) in enumerate(zip(cps, want)):
            err = rel_l2(c.cpu().numpy()[0], r)
            assert err < bound, (rv, i, err)
        assert torch.equal(cps[3], x)


@pytest.mark.parametrize("n,dtype", [(256, torch.complex128), (1024, torch.complex64)])
def test_phase_grad_tap(ctx, n, dtype):
    """The adjoint tap (scalar / lambda_b) 2 Im(G conj(E)) inside a plan, mid-chain (after an
    angular-spectrum hop: the row pass holds the fftshift sign) and at the last plane, on two
    wavelengths, against the oracle's fields; every row kernel for complex64."""
    lams = np.array([530e-9, 570e-9])
    dx, z, scal = 2e-3 / n * 4, 0.05, 4 * np.pi
    f0 = inputs.random_field((2, n, n), seed=21)
    ref = inputs.random_field((2, n, n), seed=22)
    cdt = coro.C128 if dtype == torch.complex128 else coro.C64
    x = to_dev(f0, dtype)
    ref_t = to_dev(ref, dtype)
    out = [torch.zeros((2, n, n), dtype=torch.float32, device="cuda") for _ in range(2)]
    els = [coro.element(coro.EL_PHASE_GRAD, plane=1, scalar=scal, ref=ref_t, store=out[0]),
           coro.element(coro.EL_PHASE_GRAD, plane=2, scalar=scal, ref=ref_t, store=out[1])]
    plan = coro.FresnelPlan(ctx, n=n, batch=2, pixelscale=dx, wavelength=lams, distances=[z, -0.5 * z],
                            elements=els, dtype=cdt)
    want = []
    for b in range(2):
        g1 = propagation.angular_spectrum(f0[b], dx, lams[b], z)
        g2 = propagation.angular_spectrum(g1, dx, lams[b], -0.5 * z)
        want.append([scal / lams[b] * 2 * np.imag(g * np.conj(ref[b])) for g in (g1, g2)])
    rows = KERNEL_CHOICES[n][0] if dtype == torch.complex64 else [None]
    for rv in rows:
        if rv is not None:
            plan.set_pass_kernel(rv, 0)
        y = x.clone()
        for o in out:
            o.fill_(float("nan"))
        plan.execute(y)
        for k in range(2):
            got = out[k].cpu().numpy()
            for b in range(2):
                w = want[b][k]
                err = np.linalg.norm(got[b] - w) / np.linalg.norm(w)
                assert err < 1e-5, (rv, k, b, err)             # the map is written in float


def test_phase_grad_tap_unit_reference(ctx):
    """With no reference field the tap writes (scalar / lambda) 2 Im(field), here after an
    angular-spectrum hop (the last plane of the plan, fftshift sign pending)."""
    n, lam, dx, z = 512, 600e-9, 2e-5, 0.03
    f0 = inputs.random_field((1, n, n), seed=31)
    x = to_dev(f0, torch.complex64)
    out = torch.zeros((1, n, n), dtype=torch.float32, device="cuda")
    els = [coro.element(coro.EL_PHASE_GRAD, plane=1, scalar=2.0, store=out)]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=dx, wavelength=lam, distances=[z], elements=els)
    plan.execute(x)
    g = propagation.angular_spectrum(f0[0], dx, lam, z)
    want = 2.0 / lam * 2 * np.imag(g)
    got = out.cpu().numpy()[0]
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5
    assert rel_l2(x.cpu().numpy()[0], g) < 1e-5                # the field itself passes unchanged


def test_checkpoint_after_direct_hop_and_apply(ctx):
    """A checkpoint at the focal plane of a direct hop (natural layout, new pixel scale), on
    two wavelengths; coro_apply_element with a checkpoint copies the field."""
    n, npix = 256, 128
    dx = 1.0 / npix
    lams = np.array([500e-9, 600e-9])
    cp = torch.zeros((2, n, n), dtype=torch.complex64, device="cuda")
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=0.5),
           coro.element(coro.EL_LENS, plane=0, focal_length=10.0),
           coro.element(coro.EL_CHECKPOINT, plane=1, store=cp),
           coro.element(coro.EL_CIRCLE, plane=1, radius=40e-6, flags=coro.ELF_OPAQUE_INSIDE)]
    plan = coro.FresnelPlan(ctx, n=n, batch=2, pixelscale=dx, wavelength=lams, distances=[10.0, 0.05],
                            methods=[coro.FRESNEL_DIRECT, coro.FRESNEL_AS], elements=els, init_uniform=True)
    x = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    plan.execute(x)
    got = cp.cpu().numpy()
    for b in range(2):
        e = optics.circular_aperture(n, dx, 0.5) * optics.thin_lens(n, dx, lams[b], 10.0)
        e, _ = propagation.direct_fresnel(e, dx, lams[b], 10.0)
        assert rel_l2(got[b], e) < 1e-5
    y = to_dev(inputs.random_field((2, n, n), seed=9), torch.complex64)
    out = torch.zeros_like(y)
    coro.apply_element(ctx, y, dx, lams, coro.element(coro.EL_CHECKPOINT, store=out))
    assert torch.equal(out, y)


def test_mixed_plan_direct_then_as(ctx):
    """Lens, direct hop to focus, focal stop, angular-spectrum hop, on a batch of two
    wavelengths (the direct hop changes the pixel scale per item)."""
    n, npix = 256, 128
    dx = 1.0 / npix
    lams = np.array([500e-9, 600e-9])
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=0.5),
           coro.element(coro.EL_LENS, plane=0, focal_length=10.0),
           coro.element(coro.EL_CIRCLE, plane=1, radius=40e-6, flags=coro.ELF_OPAQUE_INSIDE)]
    plan = coro.FresnelPlan(ctx, n=n, batch=2, pixelscale=dx, wavelength=lams, distances=[10.0, 0.05],
                            methods=[coro.FRESNEL_DIRECT, coro.FRESNEL_AS], elements=els, init_uniform=True)
    x = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    ps = plan.execute(x)
    got = x.cpu().numpy()
    for b in range(2):
        e = optics.circular_aperture(n, dx, 0.5) * optics.thin_lens(n, dx, lams[b], 10.0)
        e, du = propagation.direct_fresnel(e, dx, lams[b], 10.0)
        e = e * optics.circle_stop(n, du, 40e-6, opaque_inside=True)
        e = propagation.angular_spectrum(e, du, lams[b], 0.05)
        assert abs(ps[b] - du) < 1e-15 * du
        assert rel_l2(got[b], e) < 1e-5


@pytest.mark.parametrize("col", [0, -1, -7])
def test_direct_hop_column_kernels_2048(ctx, col):
    """A direct (single-transform) hop followed by an angular-spectrum hop at 2048^2 on two
    wavelengths, with the default column kernel, the persistent one and the quad one (their
    forward-only form for the direct hop)."""
    n, npix = 2048, 512
    dx = 1.0 / npix
    lams = np.array([500e-9, 600e-9])
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=0.5),
           coro.element(coro.EL_LENS, plane=0, focal_length=10.0),
           coro.element(coro.EL_CIRCLE, plane=1, radius=40e-6, flags=coro.ELF_OPAQUE_INSIDE)]
    plan = coro.FresnelPlan(ctx, n=n, batch=2, pixelscale=dx, wavelength=lams, distances=[10.0, 0.05],
                            methods=[coro.FRESNEL_DIRECT, coro.FRESNEL_AS], elements=els, init_uniform=True)
    plan.set_pass_kernel(3, col)
    x = torch.empty((2, n, n), dtype=torch.complex64, device="cuda")
    plan.execute(x)
    got = x.cpu().numpy()
    for b in range(2):
        e = optics.circular_aperture(n, dx, 0.5) * optics.thin_lens(n, dx, lams[b], 10.0)
        e, du = propagation.direct_fresnel(e, dx, lams[b], 10.0)
        e = e * optics.circle_stop(n, du, 40e-6, opaque_inside=True)
        e = propagation.angular_spectrum(e, du, lams[b], 0.05)
        assert rel_l2(got[b], e) < 1e-5


def test_airy_fp64_direct(ctx):
    """128-px 1 m aperture on 256^2 complex128, lens 10 m, direct Fresnel 10 m to focus."""
    n, npix, lam = 256, 128, 500e-9
    dx = 1.0 / npix
    els = [coro.element(coro.EL_APERTURE, plane=0, radius=0.5),
           coro.element(coro.EL_LENS, plane=0, focal_length=10.0)]
    plan = coro.FresnelPlan(ctx, n=n, batch=1, pixelscale=dx, wavelength=lam, distances=[10.0],
                            methods=[coro.FRESNEL_DIRECT], elements=els, dtype=coro.C128, init_uniform=True)
    x = torch.empty((1, n, n), dtype=torch.complex128, device="cuda")
    ps = plan.execute(x)
    e = optics.circular_aperture(n, dx, 0.5) * optics.thin_lens(n, dx, lam, 10.0)
    ref, du = propagation.direct_fresnel(e, dx, lam, 10.0)
    assert abs(ps[0] / (lam * 10.0) - 0.5) < 1e-14
    phase_max = np.pi * 2 * (n / 2 * du) ** 2 / (lam * 10.0)
    assert rel_l2(x.cpu().numpy()[0], ref) < tol(torch.complex128, phase_max)


# ------------------------------------------------------------------------------ reductions

def test_intensity_and_darkhole(ctx):
    du = 0.25
    f = inputs.random_field((3, 256, 256), seed=12)
    x = to_dev(f, torch.complex64)
    norm = np.array([2.0, 3.0, 5.0])
    i = coro.intensity(ctx, x, norm).cpu().numpy()
    f32 = f.astype(np.complex64).astype(np.complex128)
    for b in range(3):
        ref = np.abs(f32[b]) ** 2 / norm[b]
        np.testing.assert_allclose(i[b], ref, rtol=2e-7)
    s = coro.darkhole_sum(ctx, x, du, 6.0, 20.0, norm)
    from oracle import coronagraph
    for b in range(3):
        ref = coronagraph.dark_hole_sum(np.abs(f32[b]) ** 2 / norm[b], du, 6.0, 20.0)
        assert abs(s[b] - ref) < 1e-12 * ref
