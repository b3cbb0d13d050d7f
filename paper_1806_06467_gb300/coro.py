"""Thin Python binding of libcoro's C ABI (include/coro.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. PyTorch supplies device memory and the stream. If ``libcoro.so`` has not been built
the import of the library raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
import weakref
from typing import Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcoro.so")

# status codes
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTIMPL, ESIZE = 0, -1, -2, -3, -4, -5, -6
C64, C128 = 0, 1
EL_APERTURE, EL_CIRCLE, EL_LENS, EL_OPD_MAP, EL_ZERNIKE, EL_SINE, EL_SCALAR, EL_CHECKPOINT, EL_PHASE_GRAD = \
    1, 2, 3, 4, 5, 6, 7, 8, 9
ELF_OPAQUE_INSIDE, ELF_MAP_BATCHED = 1, 2
FRESNEL_AS, FRESNEL_DIRECT = 0, 1
PLAN_INIT_UNIFORM = 1
MFT_FP32, MFT_3XTF32, MFT_3XBF16, MFT_FP64, MFT_EXT = 0, 1, 2, 3, 4


class CoroError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libcoro status {status}: {msg}")
        self.status = status


class Wavefront(ct.Structure):
    _fields_ = [("data", ct.c_void_p), ("dtype", ct.c_int), ("batch", ct.c_int), ("n", ct.c_int),
                ("pixelscale", ct.POINTER(ct.c_double)), ("wavelength", ct.POINTER(ct.c_double))]


class Element(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("flags", ct.c_int), ("plane", ct.c_int), ("n_spiders", ct.c_int),
                ("radius", ct.c_double), ("obscuration", ct.c_double), ("spider_width", ct.c_double),
                ("focal_length", ct.c_double), ("opd", ct.c_void_p), ("amplitude", ct.c_void_p),
                ("coeffs", ct.POINTER(ct.c_double)), ("j_first", ct.c_int), ("n_coeffs", ct.c_int),
                ("sine_freq", ct.c_double), ("sine_amplitude", ct.c_double), ("axis", ct.c_int),
                ("scalar", ct.c_double), ("store", ct.c_void_p), ("ref", ct.c_void_p)]


class FresnelDesc(ct.Structure):
    _fields_ = [("dtype", ct.c_int), ("batch", ct.c_int), ("n", ct.c_int),
                ("pixelscale", ct.POINTER(ct.c_double)), ("wavelength", ct.POINTER(ct.c_double)),
                ("n_planes", ct.c_int), ("distance", ct.POINTER(ct.c_double)), ("method", ct.POINTER(ct.c_int)),
                ("n_elements", ct.c_int), ("elements", ct.POINTER(Element)), ("flags", ct.c_int)]


class FresnelSystemDesc(ct.Structure):
    _fields_ = [("dtype", ct.c_int), ("batch", ct.c_int), ("n", ct.c_int),
                ("pixelscale", ct.POINTER(ct.c_double)), ("wavelength", ct.POINTER(ct.c_double)),
                ("beam_radius", ct.c_double), ("n_planes", ct.c_int), ("distance", ct.POINTER(ct.c_double)),
                ("n_elements", ct.c_int), ("elements", ct.POINTER(Element)), ("flags", ct.c_int)]


class LyotItem(ct.Structure):
    _fields_ = [("m_occ", ct.c_int), ("du_occ", ct.c_double), ("spot_radius", ct.c_double),
                ("du_det", ct.c_double), ("dh_in", ct.c_double), ("dh_out", ct.c_double)]


class LyotDesc(ct.Structure):
    _fields_ = [("batch", ct.c_int), ("n", ct.c_int), ("npix", ct.c_double), ("lyot_frac", ct.c_double),
                ("m_det", ct.c_int), ("items", ct.POINTER(LyotItem)), ("precision", ct.c_int)]


class WfcDesc(ct.Structure):
    _fields_ = [("batch", ct.c_int), ("wavelength", ct.POINTER(ct.c_double)), ("n_fresnel", ct.c_int),
                ("diam_m", ct.c_double), ("npix", ct.c_int), ("z_m", ct.c_double), ("n_act", ct.c_int),
                ("act_pitch_m", ct.c_double), ("act_fwhm_m", ct.c_double), ("lyot_frac", ct.c_double),
                ("m_det", ct.c_int), ("items", ct.POINTER(LyotItem)), ("precision", ct.c_int),
                ("max_resident", ct.c_int)]


_P = ct.c_void_p
_SIGS = {
    "coro_lyot_plan_set_pupil_layout": (ct.c_int, [_P, ct.c_int, ct.c_longlong]),
    "coro_lyot_plan_gradient": (ct.c_int, [_P, _P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), _P, ct.c_int,
                                           ct.c_longlong]),
    "coro_wfc_plan_create": (ct.c_int, [_P, ct.POINTER(WfcDesc), ct.POINTER(_P)]),
    "coro_wfc_plan_peak": (ct.c_int, [_P, ct.POINTER(ct.c_double)]),
    "coro_wfc_plan_resident": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "coro_wfc_plan_evaluate": (ct.c_int, [_P, _P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), _P]),
    "coro_dm_opd": (ct.c_int, [_P, _P, ct.c_int, ct.c_int, ct.c_double, ct.c_double, ct.c_int, ct.c_double,
                               ct.c_double, _P]),
    "coro_dm_correlate": (ct.c_int, [_P, _P, ct.c_int, ct.c_int, ct.c_double, ct.c_int, ct.c_double,
                                     ct.c_double, ct.c_double, _P]),
    "coro_lyot_plan_create": (ct.c_int, [_P, ct.POINTER(LyotDesc), ct.POINTER(_P)]),
    "coro_lyot_plan_execute": (ct.c_int, [_P, _P, ct.POINTER(ct.c_double), _P, _P, ct.POINTER(ct.c_double)]),
    "coro_lyot_plan_peak": (ct.c_int, [_P, _P, ct.POINTER(ct.c_double)]),
    "coro_lyot_plan_execute_range": (ct.c_int, [_P, _P, ct.POINTER(ct.c_double), _P, _P, ct.c_int, ct.c_int]),
    "coro_lyot_plan_flops": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]),
    "coro_lyot_plan_gemm_tile": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "coro_fresnel_plan_pass_radix": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int), ct.c_int, ct.POINTER(ct.c_int)]),
    "coro_lyot_plan_set_gemm_tile": (ct.c_int, [_P, ct.c_int]),
    "coro_version": (ct.c_int, []),
    "coro_last_error": (ct.c_char_p, []),
    "coro_ctx_create": (ct.c_int, [ct.c_int, _P, ct.POINTER(_P)]),
    "coro_ctx_destroy": (ct.c_int, [_P]),
    "coro_ctx_set_stream": (ct.c_int, [_P, _P]),
    "coro_ctx_synchronize": (ct.c_int, [_P]),
    "coro_wavefront_init": (ct.c_int, [_P, ct.POINTER(Wavefront), ct.c_double]),
    "coro_wavefront_axpy": (ct.c_int, [_P, ct.c_double, ct.POINTER(Wavefront), ct.POINTER(Wavefront)]),
    "coro_apply_element": (ct.c_int, [_P, ct.POINTER(Wavefront), ct.POINTER(Element)]),
    "coro_propagate_fresnel": (ct.c_int, [_P, ct.POINTER(Wavefront), ct.c_double, ct.c_int]),
    "coro_fft2": (ct.c_int, [_P, ct.POINTER(Wavefront), ct.c_int]),
    "coro_fresnel_plan_create": (ct.c_int, [_P, ct.POINTER(FresnelDesc), ct.POINTER(_P)]),
    "coro_fresnel_system_create": (ct.c_int, [_P, ct.POINTER(FresnelSystemDesc), ct.POINTER(_P)]),
    "coro_fresnel_system_info": (ct.c_int, [_P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "coro_fresnel_system_pitch": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_double)]),
    "coro_fresnel_plan_execute": (ct.c_int, [_P, _P, ct.POINTER(ct.c_double)]),
    "coro_plan_launch_count": (ct.c_int, [_P, ct.POINTER(ct.c_int)]),
    "coro_fresnel_plan_execute_range": (ct.c_int, [_P, _P, ct.c_int, ct.c_int]),
    "coro_fresnel_plan_pass_info": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_double)]),
    "coro_fresnel_plan_pass_flops": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_double)]),
    "coro_fresnel_plan_pass_kernel": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]),
    "coro_fresnel_plan_set_pass_kernel": (ct.c_int, [_P, ct.c_int, ct.c_int]),
    "coro_fresnel_plan_set_layout": (ct.c_int, [_P, ct.c_int]),
    "coro_fresnel_plan_layout": (ct.c_int, [_P, ct.POINTER(ct.c_int)]),
    "coro_fresnel_plan_copy_tuning": (ct.c_int, [_P, _P]),
    "coro_selftest_wait_timeout": (ct.c_int, [_P, ct.c_int]),
    "coro_plan_set_timing": (ct.c_int, [_P, ct.c_int]),
    "coro_plan_unit_times": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_float)]),
    "coro_fresnel_plan_execute_n": (ct.c_int, [_P, _P, ct.c_int]),
    "coro_lyot_plan_execute_n": (ct.c_int, [_P, _P, ct.POINTER(ct.c_double), _P, _P, ct.c_int]),
    "coro_plan_set_graph": (ct.c_int, [_P, ct.c_int]),
    "coro_plan_destroy": (ct.c_int, [_P]),
    "coro_propagate_mft": (ct.c_int, [_P, ct.POINTER(Wavefront), ct.c_double, ct.c_int, ct.c_int,
                                      ct.POINTER(ct.c_double), ct.c_int, ct.POINTER(Wavefront)]),
    "coro_intensity": (ct.c_int, [_P, ct.POINTER(Wavefront), ct.POINTER(ct.c_double), _P]),
    "coro_darkhole_sum": (ct.c_int, [_P, ct.POINTER(Wavefront), ct.POINTER(ct.c_double), ct.c_double,
                                     ct.c_double, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]),
    "coro_darkhole_sum_noalloc": (ct.c_int, [ct.POINTER(Wavefront), ct.POINTER(ct.c_double), ct.c_double,
                                             ct.c_double, ct.POINTER(ct.c_double), _P, ct.POINTER(ct.c_double)]),
}


def declared_symbols() -> list[str]:
    return sorted(_SIGS)


class Library:
    """The loaded libcoro.so with typed entry points."""
    _inst: "Library | None" = None

    def __init__(self, path: str = LIB_PATH):
        if not os.path.exists(path):
            raise RuntimeError(f"libcoro is not built ({path} missing): run __graft_entry__.build()")
        self.path = path
        self.dll = ct.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(self.dll, name)
            fn.restype = res
            fn.argtypes = args

    @classmethod
    def get(cls) -> "Library":
        if cls._inst is None:
            cls._inst = cls()
        return cls._inst

    def check(self, status: int):
        if status != OK:
            raise CoroError(status, self.dll.coro_last_error().decode())

    def __getattr__(self, name):
        return getattr(self.dll, name)


def _dbl(values) -> ct.Array:
    arr = np.ascontiguousarray(np.asarray(values, dtype=np.float64).ravel())
    return (ct.c_double * len(arr))(*arr.tolist())


class Context:
    """coro_ctx bound to a CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = Library.get()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ct.c_void_p()
        self.lib.check(self.lib.coro_ctx_create(device, ct.c_void_p(stream.cuda_stream), ct.byref(h)))
        self.handle = h
        self._plans = weakref.WeakSet()

    def _track(self, plan):
        self._plans.add(plan)

    def close(self):
        """Destroy every plan made on this context, then the context itself."""
        for plan in list(getattr(self, "_plans", ())):
            plan.close()
        if getattr(self, "handle", None):
            self.lib.coro_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        self.lib.check(self.lib.coro_ctx_synchronize(self.handle))


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise TypeError(f"field must be complex64 or complex128, got {t.dtype}")


class WF:
    """Keeps a Wavefront struct and its host arrays alive. field: [batch][n][n] CUDA tensor."""

    def __init__(self, field, pixelscale: Sequence[float] | float | None = None,
                 wavelength: Sequence[float] | float | None = None):
        if field.dim() == 2:
            field = field.unsqueeze(0)
        if not field.is_cuda or not field.is_contiguous():
            raise ValueError("field must be a contiguous CUDA tensor")
        self.field = field
        b, n0, n1 = field.shape
        if n0 != n1:
            raise ValueError("field must be square")
        ps = np.broadcast_to(np.asarray(1.0 if pixelscale is None else pixelscale, float), (b,))
        lam = np.broadcast_to(np.asarray(1.0 if wavelength is None else wavelength, float), (b,))
        self._ps = _dbl(ps)
        self._lam = _dbl(lam)
        self.s = Wavefront(field.data_ptr(), _dtype_code(field), b, n0, self._ps, self._lam)

    @property
    def pixelscale(self) -> np.ndarray:
        return np.array(self._ps[:])


def element(kind: int, plane: int = 0, **kw) -> Element:
    """Build a coro_element; keyword names follow the C struct (coeffs as a sequence)."""
    e = Element()
    e.kind = kind
    e.plane = plane
    keep = []
    for k, v in kw.items():
        if k == "coeffs":
            arr = _dbl(v)
            keep.append(arr)
            e.coeffs = arr
            e.n_coeffs = len(arr)
        elif k in ("opd", "amplitude", "store", "ref"):
            if v is not None:
                keep.append(v)
                setattr(e, k, v.data_ptr())
        else:
            setattr(e, k, v)
    e._keep = keep
    return e


def wavefront_init(ctx: Context, field, amplitude: float = 1.0):
    w = WF(field)
    ctx.lib.check(ctx.lib.coro_wavefront_init(ctx.handle, ct.byref(w.s), amplitude))


def apply_element(ctx: Context, field, pixelscale, wavelength, el: Element):
    w = WF(field, pixelscale, wavelength)
    ctx.lib.check(ctx.lib.coro_apply_element(ctx.handle, ct.byref(w.s), ct.byref(el)))


def propagate_fresnel(ctx: Context, field, pixelscale, wavelength, z: float, method: int = FRESNEL_AS) -> np.ndarray:
    """In-place hop; returns the new per-item pixel scale."""
    w = WF(field, pixelscale, wavelength)
    ctx.lib.check(ctx.lib.coro_propagate_fresnel(ctx.handle, ct.byref(w.s), z, method))
    return w.pixelscale


def fft2(ctx: Context, field, direction: int = -1):
    w = WF(field)
    ctx.lib.check(ctx.lib.coro_fft2(ctx.handle, ct.byref(w.s), direction))


def wavefront_axpy(ctx: Context, alpha: float, x, y):
    """y += alpha x (two device fields of the same dtype and shape)."""
    wx, wy = WF(x), WF(y)
    ctx.lib.check(ctx.lib.coro_wavefront_axpy(ctx.handle, float(alpha), ct.byref(wx.s), ct.byref(wy.s)))
    return y


def propagate_mft(ctx: Context, field, npix: float, direction: int, m: int, du, precision: int | None = None,
                  out=None):
    """precision: MFT_FP32 / MFT_3XTF32 / MFT_3XBF16 / MFT_EXT for complex64 fields, MFT_FP64 for complex128
    (the default follows the field's dtype: FP32 CUDA cores or FP64)."""
    import torch
    if precision is None:
        precision = MFT_FP64 if field.dtype == torch.complex128 else MFT_FP32
    w = WF(field)
    b = w.s.batch
    if out is None:
        out = torch.empty((b, m, m), dtype=field.dtype, device=field.device)
    wo = WF(out)
    du_arr = _dbl(np.broadcast_to(np.asarray(du, float), (b,)))
    ctx.lib.check(ctx.lib.coro_propagate_mft(ctx.handle, ct.byref(w.s), npix, direction, m, du_arr,
                                             precision, ct.byref(wo.s)))
    return out


def intensity(ctx: Context, field, norm=None, out=None):
    import torch
    w = WF(field)
    if out is None:
        out = torch.empty(w.field.shape, dtype=torch.float32, device=field.device)
    nrm = None if norm is None else _dbl(np.broadcast_to(np.asarray(norm, float), (w.s.batch,)))
    ctx.lib.check(ctx.lib.coro_intensity(ctx.handle, ct.byref(w.s), nrm, ct.c_void_p(out.data_ptr())))
    return out


def darkhole_sum(ctx: Context, field, du, r_in: float, r_out: float, norm=None) -> np.ndarray:
    w = WF(field)
    b = w.s.batch
    du_arr = _dbl(np.broadcast_to(np.asarray(du, float), (b,)))
    nrm = None if norm is None else _dbl(np.broadcast_to(np.asarray(norm, float), (b,)))
    out = (ct.c_double * b)()
    ctx.lib.check(ctx.lib.coro_darkhole_sum(ctx.handle, ct.byref(w.s), du_arr, r_in, r_out, nrm, out))
    return np.array(out[:])


def darkhole_sum_noalloc(field, du, r_in: float, r_out: float, norm=None, stream=None) -> np.ndarray:
    """coro_darkhole_sum_noalloc: same sums as darkhole_sum, with no device allocation (for
    callers that must not allocate while they run). Runs with the field's device current, on
    torch's current stream of that device unless one is given; calls that overlap on the GPU
    race (one shared scratch array)."""
    import torch
    lib = Library.get()
    w = WF(field)
    b = w.s.batch
    du_arr = _dbl(np.broadcast_to(np.asarray(du, float), (b,)))
    nrm = None if norm is None else _dbl(np.broadcast_to(np.asarray(norm, float), (b,)))
    out = (ct.c_double * b)()
    with torch.cuda.device(field.device):
        if stream is None:
            stream = torch.cuda.current_stream(field.device)
        lib.check(lib.coro_darkhole_sum_noalloc(ct.byref(w.s), du_arr, r_in, r_out, nrm,
                                                ct.c_void_p(stream.cuda_stream), out))
    return np.array(out[:])


def dm_opd(ctx: Context, heights, pitch: float, fwhm: float, n: int, pixelscale: float, scale: float = 2.0,
           out=None):
    """heights: CUDA float32 [batch][na][na] (metres) -> OPD map [batch][n][n]."""
    import torch
    b, na, _ = heights.shape
    if out is None:
        out = torch.empty((b, n, n), dtype=torch.float32, device=heights.device)
    ctx.lib.check(ctx.lib.coro_dm_opd(ctx.handle, ct.c_void_p(heights.data_ptr()), b, na, pitch, fwhm, n,
                                      pixelscale, scale, ct.c_void_p(out.data_ptr())))
    return out


def dm_correlate(ctx: Context, w, pixelscale: float, na: int, pitch: float, fwhm: float, scale: float = 1.0,
                 out=None):
    """w: CUDA float32 [batch][n][n] -> [batch][na][na] (transpose of dm_opd)."""
    import torch
    b, n, _ = w.shape
    if out is None:
        out = torch.empty((b, na, na), dtype=torch.float32, device=w.device)
    ctx.lib.check(ctx.lib.coro_dm_correlate(ctx.handle, ct.c_void_p(w.data_ptr()), b, n, pixelscale, na, pitch,
                                            fwhm, scale, ct.c_void_p(out.data_ptr())))
    return out


class LyotPlan:
    """Batched semi-analytic Lyot coronagraph (coro_lyot_plan_*). items: sequence of dicts with
    m_occ, du_occ, spot_radius, du_det, dh_in, dh_out (lambda/D units)."""

    def __init__(self, ctx: Context, *, n: int, npix: float, lyot_frac: float, m_det: int, items,
                 precision: int = MFT_3XTF32):
        self.ctx = ctx
        self.batch = len(items)
        self.n, self.m_det = n, m_det
        self._items = (LyotItem * self.batch)(*[LyotItem(**it) for it in items])
        d = LyotDesc(self.batch, n, npix, lyot_frac, m_det, self._items, precision)
        h = ct.c_void_p()
        ctx.lib.check(ctx.lib.coro_lyot_plan_create(ctx.handle, ct.byref(d), ct.byref(h)))
        self.handle = h
        ctx._track(self)

    def peak(self, pupil) -> np.ndarray:
        out = (ct.c_double * self.batch)()
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_peak(self.handle, ct.c_void_p(pupil.data_ptr()), out))
        return np.array(out[:])

    def execute(self, pupil, peak=None, intensity=None, field=None, want_dh: bool = True):
        """Returns the dark-hole sums (host) when want_dh; fills intensity / field if given."""
        pk = None if peak is None else _dbl(np.broadcast_to(np.asarray(peak, float), (self.batch,)))
        dh = (ct.c_double * self.batch)() if want_dh else None
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_execute(
            self.handle, ct.c_void_p(pupil.data_ptr()), pk,
            None if intensity is None else ct.c_void_p(intensity.data_ptr()),
            None if field is None else ct.c_void_p(field.data_ptr()), dh))
        return np.array(dh[:]) if want_dh else None

    timing_units = 6

    def execute_n(self, pupil, times: int, peak=None, intensity=None, field=None):
        """`times` executes back to back (coro_lyot_plan_execute_n)."""
        pk = None if peak is None else _dbl(np.broadcast_to(np.asarray(peak, float), (self.batch,)))
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_execute_n(
            self.handle, ct.c_void_p(pupil.data_ptr()), pk,
            None if intensity is None else ct.c_void_p(intensity.data_ptr()),
            None if field is None else ct.c_void_p(field.data_ptr()), times))

    def set_pupil_layout(self, ld: int, bstride: int):
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_set_pupil_layout(self.handle, ld, bstride))

    def gradient(self, pupil, peak, grad_out=None, grad_ld: int | None = None, grad_bstride: int | None = None):
        """dS/dconj(E_A) per item (complex64 [batch][n][n] unless a strided window is given) and the
        dark-hole sums."""
        import torch
        if grad_out is None:
            grad_out = torch.empty((self.batch, self.n, self.n), dtype=torch.complex64, device=pupil.device)
            grad_ld, grad_bstride = self.n, self.n * self.n
        dh = (ct.c_double * self.batch)()
        pk = _dbl(np.broadcast_to(np.asarray(peak, float), (self.batch,)))
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_gradient(
            self.handle, ct.c_void_p(pupil.data_ptr()), pk, dh, ct.c_void_p(grad_out.data_ptr()), grad_ld, grad_bstride))
        return grad_out, np.array(dh[:])

    def execute_range(self, pupil, first: int, count: int = 1, peak=None, intensity=None, field=None):
        pk = None if peak is None else _dbl(np.broadcast_to(np.asarray(peak, float), (self.batch,)))
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_execute_range(
            self.handle, ct.c_void_p(pupil.data_ptr()), pk,
            None if intensity is None else ct.c_void_p(intensity.data_ptr()),
            None if field is None else ct.c_void_p(field.data_ptr()), first, count))

    def gemm_tile(self) -> tuple[int, int]:
        """(rows, complex columns) of the tensor-core GEMM tile the plan runs."""
        m, n = ct.c_int(), ct.c_int()
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_gemm_tile(self.handle, ct.byref(m), ct.byref(n)))
        return m.value, n.value

    def set_gemm_tile(self, tile_n: int) -> None:
        """Override the tuned tile width (EXT: 64 or 32)."""
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_set_gemm_tile(self.handle, tile_n))

    def flops(self) -> tuple[float, float]:
        """(useful, issued) tensor flops of one execute (coro_lyot_plan_flops)."""
        u, i = ct.c_double(), ct.c_double()
        self.ctx.lib.check(self.ctx.lib.coro_lyot_plan_flops(self.handle, ct.byref(u), ct.byref(i)))
        return u.value, i.value

    def use_graph(self, enable: bool = True) -> None:
        """Replay execute as a CUDA graph (coro_plan_set_graph)."""
        self.ctx.lib.check(self.ctx.lib.coro_plan_set_graph(self.handle, 1 if enable else 0))

    def set_timing(self, steps: int) -> None:
        """Per-unit CUDA-event timing of the next `steps` executes (coro_plan_set_timing)."""
        self.ctx.lib.check(self.ctx.lib.coro_plan_set_timing(self.handle, steps))

    def unit_times(self, steps: int) -> np.ndarray:
        """[steps][units] durations in ms (coro_plan_unit_times)."""
        units = self.timing_units
        buf = (ct.c_float * (steps * units))()
        self.ctx.lib.check(self.ctx.lib.coro_plan_unit_times(self.handle, steps, buf))
        return np.array(buf[:], dtype=np.float64).reshape(steps, units)

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.coro_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FresnelPlan:
    """Fused plane-by-plane Fresnel system (coro_fresnel_plan_*)."""

    def __init__(self, ctx: Context, *, n: int, batch: int, pixelscale, wavelength, distances,
                 elements: Sequence[Element], methods=None, dtype: int = C64, init_uniform: bool = False):
        self.ctx = ctx
        self.batch = batch
        self.n = n
        d = FresnelDesc()
        d.dtype, d.batch, d.n = dtype, batch, n
        self._ps = _dbl(np.broadcast_to(np.asarray(pixelscale, float), (batch,)))
        self._lam = _dbl(np.broadcast_to(np.asarray(wavelength, float), (batch,)))
        d.pixelscale, d.wavelength = self._ps, self._lam
        d.n_planes = len(distances) + 1
        self._dist = _dbl(distances) if len(distances) else None
        d.distance = self._dist
        if methods is not None:
            self._meth = (ct.c_int * len(methods))(*methods)
            d.method = self._meth
        self._els = (Element * max(1, len(elements)))(*elements)
        self._keep = list(elements)
        d.n_elements = len(elements)
        d.elements = self._els
        d.flags = PLAN_INIT_UNIFORM if init_uniform else 0
        h = ct.c_void_p()
        ctx.lib.check(ctx.lib.coro_fresnel_plan_create(ctx.handle, ct.byref(d), ct.byref(h)))
        self.handle = h
        ctx._track(self)

    def use_graph(self, enable: bool = True) -> None:
        """Replay execute as a CUDA graph (coro_plan_set_graph)."""
        self.ctx.lib.check(self.ctx.lib.coro_plan_set_graph(self.handle, 1 if enable else 0))

    def set_timing(self, steps: int) -> None:
        """Per-unit CUDA-event timing of the next `steps` executes (coro_plan_set_timing)."""
        self.ctx.lib.check(self.ctx.lib.coro_plan_set_timing(self.handle, steps))

    def unit_times(self, steps: int) -> np.ndarray:
        """[steps][units] durations in ms (coro_plan_unit_times)."""
        units = self.timing_units
        buf = (ct.c_float * (steps * units))()
        self.ctx.lib.check(self.ctx.lib.coro_plan_unit_times(self.handle, steps, buf))
        return np.array(buf[:], dtype=np.float64).reshape(steps, units)

    def execute(self, field) -> np.ndarray:
        ps = (ct.c_double * self.batch)()
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_execute(self.handle, ct.c_void_p(field.data_ptr()), ps))
        return np.array(ps[:])

    @property
    def timing_units(self) -> int:
        return self.launch_count

    def plane_pitch(self, plane: int) -> np.ndarray:
        """Per-item pixel scale at which plane `plane`'s elements act."""
        buf = (ct.c_double * self.batch)()
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_system_pitch(self.handle, plane, buf))
        return np.array(buf[:])

    def execute_n(self, field, times: int):
        """`times` executes back to back (coro_fresnel_plan_execute_n)."""
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_execute_n(self.handle, ct.c_void_p(field.data_ptr()), times))

    def execute_range(self, field, first: int, count: int = 1):
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_execute_range(
            self.handle, ct.c_void_p(field.data_ptr()), first, count))

    def pass_flops(self, i: int) -> float:
        """FFT arithmetic of pass i (coro_fresnel_plan_pass_flops)."""
        f = ct.c_double()
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_pass_flops(self.handle, i, ct.byref(f)))
        return f.value

    def pass_info(self, i: int) -> tuple[bool, float]:
        """(is_row_pass, algorithmic HBM bytes) of pass i."""
        r, b = ct.c_int(), ct.c_double()
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_pass_info(self.handle, i, ct.byref(r), ct.byref(b)))
        return bool(r.value), b.value

    def pass_kernel(self, i: int) -> str:
        """Name of the kernel pass i launches, e.g. 'col_pass_persistent<4096,2>'."""
        p, w = ct.c_int(), ct.c_int()
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_pass_kernel(self.handle, i, ct.byref(p), ct.byref(w)))
        row, _ = self.pass_info(i)
        kind = "row_pass" if row else "col_pass"
        name = kind + ("_kernel", "_persistent", "_units", "_pair", "_wide", "", "_mixed", "_pair_t", "_quad",
                              "_mixed_pair")[p.value]
        if p.value == 6 and self.n & (self.n - 1) == 0:
            name += "_r8"                               # the shared-memory engine at radix 8
        return f"{name}<{self.n}>" if row else f"{name}<{self.n},{w.value}>"

    def pass_radix(self, i: int) -> list[int]:
        """Radix sequence of pass i's line transforms (coro_fresnel_plan_pass_radix)."""
        buf, k = (ct.c_int * 16)(), ct.c_int()
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_pass_radix(self.handle, i, buf, 16, ct.byref(k)))
        return list(buf[:k.value])

    def set_pass_kernel(self, row_variant: int, col_lines: int) -> None:
        """Override the tuned kernels (row: 0 persistent, 1 per-group, 2 units, 3 packed row
        pairs, 5 shared-memory radix-8 engine, 6 packed-pair mixed-radix engine; column: lines
        per block, -1 persistent TMA, -2 units, -3 packed column pairs, -4 wide four-column
        groups, -5 packed-pair mixed-radix engine, -7 quad four-column strips, -8 shared-memory
        radix-8 engine, 0 default)."""
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_set_pass_kernel(self.handle, row_variant, col_lines))

    def set_layout(self, transposed: bool) -> None:
        """Natural (False) or alternating (True) plane layout between passes
        (coro_fresnel_plan_set_layout)."""
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_set_layout(self.handle, 1 if transposed else 0))

    def copy_tuning(self, other: "FresnelPlan") -> None:
        """Run the kernels and layout `other`'s tuner chose (coro_fresnel_plan_copy_tuning)."""
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_copy_tuning(self.handle, other.handle))

    @property
    def layout(self) -> bool:
        """True when the plan runs on the alternating layout."""
        t = ct.c_int()
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_plan_layout(self.handle, ct.byref(t)))
        return bool(t.value)

    @property
    def launch_count(self) -> int:
        c = ct.c_int()
        self.ctx.lib.check(self.ctx.lib.coro_plan_launch_count(self.handle, ct.byref(c)))
        return c.value

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.coro_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FresnelSystem(FresnelPlan):
    """Fresnel system with the propagation method chosen by a Gaussian pilot beam
    (coro_fresnel_system_create): lenses refocus the pilot beam, planes within its Rayleigh
    range use angular-spectrum hops, others direct hops with spherical references."""

    def __init__(self, ctx: Context, *, n: int, batch: int, pixelscale, wavelength, beam_radius: float,
                 distances, elements: Sequence[Element], dtype: int = C64, init_uniform: bool = False):
        self.ctx = ctx
        self.batch = batch
        self.n = n
        self.n_planes = len(distances) + 1
        d = FresnelSystemDesc()
        d.dtype, d.batch, d.n = dtype, batch, n
        self._ps = _dbl(np.broadcast_to(np.asarray(pixelscale, float), (batch,)))
        self._lam = _dbl(np.broadcast_to(np.asarray(wavelength, float), (batch,)))
        d.pixelscale, d.wavelength = self._ps, self._lam
        d.beam_radius = float(beam_radius)
        d.n_planes = self.n_planes
        self._dist = _dbl(distances) if len(distances) else None
        d.distance = self._dist
        self._els = (Element * max(1, len(elements)))(*elements)
        self._keep = list(elements)
        d.n_elements = len(elements)
        d.elements = self._els
        d.flags = PLAN_INIT_UNIFORM if init_uniform else 0
        h = ct.c_void_p()
        ctx.lib.check(ctx.lib.coro_fresnel_system_create(ctx.handle, ct.byref(d), ct.byref(h)))
        self.handle = h
        ctx._track(self)

    def info(self) -> tuple[list[bool], int]:
        """(per plane: spherical reference?, number of direct sub-hops)."""
        sph = (ct.c_int * self.n_planes)()
        nd = ct.c_int()
        self.ctx.lib.check(self.ctx.lib.coro_fresnel_system_info(self.handle, sph, ct.byref(nd)))
        return [bool(v) for v in sph], nd.value
