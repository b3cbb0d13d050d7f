"""Differentiable wavefront control: summed dark-hole intensity of a two-DM Lyot coronagraph
as a torch.autograd.Function of the DM actuator heights.

The forward pass and the hand-written adjoint both run in libcoro (coro_wfc_plan_evaluate);
this module only marshals arguments. The gradient is produced together with the loss (the
adjoint chain reuses the forward's checkpoints) and handed back in backward().
"""
from __future__ import annotations

import ctypes as ct

import numpy as np
import torch

from . import coro


class WfcPlan:
    """coro_wfc_plan_*: DM1 at the pupil, DM2 a Fresnel hop z away, Lyot chain per wavelength.
    max_resident bounds the wavelengths whose fields are in memory at once (0: as many as fit
    in 70 % of the free device memory); the band then runs in chunks."""

    def __init__(self, ctx: coro.Context, *, wavelengths, n_fresnel: int, diam_m: float, npix: int, z_m: float,
                 n_act: int, pitch_m: float, fwhm_m: float, lyot_frac: float, m_det: int, items,
                 precision: int = coro.MFT_3XTF32, max_resident: int = 0):
        self.ctx = ctx
        self.batch = len(wavelengths)
        self.n_act = n_act
        self._lam = coro._dbl(wavelengths)
        self._items = (coro.LyotItem * self.batch)(*[coro.LyotItem(**it) for it in items])
        d = coro.WfcDesc(self.batch, self._lam, n_fresnel, diam_m, npix, z_m, n_act, pitch_m, fwhm_m, lyot_frac,
                         m_det, self._items, precision, max_resident)
        h = ct.c_void_p()
        ctx.lib.check(ctx.lib.coro_wfc_plan_create(ctx.handle, ct.byref(d), ct.byref(h)))
        self.handle = h
        ctx._track(self)

    def resident(self) -> tuple[int, int]:
        """(wavelengths held in memory at once, chunks the band runs in)."""
        r, c = ct.c_int(), ct.c_int()
        self.ctx.lib.check(self.ctx.lib.coro_wfc_plan_resident(self.handle, ct.byref(r), ct.byref(c)))
        return r.value, c.value

    def peak(self) -> np.ndarray:
        out = (ct.c_double * self.batch)()
        self.ctx.lib.check(self.ctx.lib.coro_wfc_plan_peak(self.handle, out))
        return np.array(out[:])

    def evaluate(self, heights, want_grad: bool = True):
        """heights: CUDA float32 [2][n_act][n_act]. Returns (loss, per-wavelength sums, grad or None)."""
        h = heights.detach().contiguous()
        if h.dtype != torch.float32 or not h.is_cuda or tuple(h.shape) != (2, self.n_act, self.n_act):
            raise ValueError("heights must be a CUDA float32 tensor [2][n_act][n_act]")
        loss = ct.c_double()
        per = (ct.c_double * self.batch)()
        grad = torch.empty_like(h) if want_grad else None
        self.ctx.lib.check(self.ctx.lib.coro_wfc_plan_evaluate(
            self.handle, ct.c_void_p(h.data_ptr()), ct.byref(loss), per,
            None if grad is None else ct.c_void_p(grad.data_ptr())))
        return loss.value, np.array(per[:]), grad

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.coro_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DarkHoleLoss(torch.autograd.Function):
    """L(h) = sum over wavelengths of the normalised dark-hole intensity; dL/dh from the
    library's adjoint chain."""

    @staticmethod
    def forward(fctx, heights, plan: WfcPlan):
        loss, _, grad = plan.evaluate(heights, want_grad=heights.requires_grad)
        fctx.save_for_backward(grad if grad is not None else torch.zeros_like(heights))
        return torch.tensor(loss, dtype=torch.float64, device=heights.device)

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return (g.to(grad.dtype) * grad), None


def dark_hole_loss(heights, plan: WfcPlan):
    return DarkHoleLoss.apply(heights, plan)
