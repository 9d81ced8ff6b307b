"""torch.autograd integration of the propagator (FWI objective and gradient).

``AcousticForward`` maps the squared slowness m (and optionally the source
wavelet) to receiver data d = F(m) q (Eq. AS) through ``wp_forward_save``, which
keeps the forward field's snapshots resident in device memory.  Its backward
turns the upstream gradient dL/dd into dL/dm = J^T (dL/dd) with ``wp_backward``
(the adjoint-state gradient of Eq. Grad, recomputing the forward field between
snapshots), and into dL/dq = F^T (dL/dd) with the adjoint propagator (Eq. Adj)
when the wavelet requires a gradient.  eta (the absorbing-layer profile) is an
input of the operator, not a parameter: it receives no gradient.

``misfit`` is J = 1/2 ||d - d_obs||^2 (the library's residual kernel), whose
gradient with respect to d is the residual d - d_obs, so
``misfit(prop(m), d_obs).backward()`` yields dJ/dm.  The propagator's arithmetic
runs in the CUDA library; torch provides device memory, streams and the autograd
graph (and scales the residual by the upstream gradient of J, a scalar).
"""
from __future__ import annotations

import torch

from . import wavprop as W


class _State:
    """Owns a wp_state (snapshots in device memory); frees it when collected."""

    def __init__(self, handle: int):
        self.handle = handle

    def free(self):
        if self.handle:
            W.wp_state_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class AcousticForward(torch.autograd.Function):
    """d = F(m) q for one shot; differentiable in m (and in q)."""

    @staticmethod
    def forward(ctx, m, eta, wavelet, prop):
        grid = prop.grid
        m, eta, wavelet = m.contiguous(), eta.contiguous(), wavelet.contiguous()
        d = torch.empty((grid.nt, len(prop.rec)), device=m.device, dtype=torch.float32)
        ctx.prop = prop
        ctx.save_for_backward(m, eta)
        if ctx.needs_input_grad[0]:
            # keep the snapshots resident only when dL/dm can be asked for
            st = W.wp_forward_save(prop.context.handle, grid, m.detach(), eta.detach(), wavelet.detach(),
                                   prop.src, prop.rec, prop.snap_interval, d)
            ctx.state = _State(st)
        else:
            W.wp_forward_dev(prop.context.handle, grid, m.detach(), eta.detach(), wavelet.detach(), prop.src,
                             prop.rec, d)
            ctx.state = None
        return d

    @staticmethod
    def backward(ctx, grad_d):
        m, eta = ctx.saved_tensors
        prop = ctx.prop
        grad_d = grad_d.contiguous().to(torch.float32)
        grad_m = grad_q = None
        if ctx.needs_input_grad[0]:
            grad_m = torch.empty_like(m)
            W.wp_backward(ctx.state.handle, grad_d, grad_m)
        if ctx.needs_input_grad[2]:
            grad_q = torch.empty((prop.grid.nt, len(prop.src)), device=m.device, dtype=torch.float32)
            W.wp_adjoint_dev(prop.context.handle, prop.grid, m.detach(), eta.detach(), grad_d, prop.rec, prop.src,
                             grad_q)
        return grad_m, None, grad_q, None


class AcousticPropagator:
    """One acquisition geometry on one grid: call it with (m, eta, wavelet).

    shape, spacing, origin use the C order of the fields ((nz, ny, nx) / (nz, nx));
    src and rec are (npoints, ndim) coordinates in the same order; snap_interval
    is the number of steps between resident forward snapshots.
    """

    def __init__(self, shape, spacing, origin, space_order, dt, nt, src, rec, snap_interval=10,
                 context: W.Context | None = None, device: int = 0):
        import numpy as np
        self.grid = W.Grid(tuple(shape), tuple(spacing), tuple(origin), int(space_order), float(dt), int(nt))
        self.src = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, len(shape)))
        self.rec = np.ascontiguousarray(np.asarray(rec, dtype=np.float64).reshape(-1, len(shape)))
        self.snap_interval = int(snap_interval)
        self.context = context if context is not None else W.Context(device)

    def __call__(self, m, eta, wavelet):
        return AcousticForward.apply(m, eta, wavelet, self)


_misfit_contexts: dict = {}


def _misfit_context(device) -> W.Context:
    """One small library context per device for the misfit kernel (created on first use)."""
    idx = device.index if device.index is not None else torch.cuda.current_device()
    c = _misfit_contexts.get(idx)
    if c is None:
        c = _misfit_contexts[idx] = W.Context(idx)
    return c


class Misfit(torch.autograd.Function):
    """J = 1/2 ||d - d_obs||^2 (Eq. AS) by the library's residual kernel (r = d - d_obs
    and the sum of r^2 in double, fixed order); dJ/dd = r, dJ/dd_obs = -r."""

    @staticmethod
    def forward(ctx, d, d_obs):
        d = d.detach().contiguous()
        d_obs = d_obs.detach().contiguous()
        r = torch.empty_like(d)
        J = W.wp_misfit_dev(_misfit_context(d.device).handle, d, d_obs, r)
        ctx.save_for_backward(r)
        return torch.tensor(J, dtype=torch.float64, device=d.device)

    @staticmethod
    def backward(ctx, g):
        (r,) = ctx.saved_tensors
        gr = (r * g.to(r.dtype)) if g is not None else r
        return gr, -gr


def misfit(d, d_obs):
    """J = 1/2 ||d - d_obs||^2 (Eq. AS) as a float64 scalar tensor; differentiable in d
    (and d_obs)."""
    return Misfit.apply(d, d_obs)
