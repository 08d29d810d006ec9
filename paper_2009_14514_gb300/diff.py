"""Differentiable WCSPH rollout behind torch.autograd.Function (binding of rts_diff_*).

The rollout (global constant stepping at dt_b, the Serna predictor-corrector and the WCSPH
physics of the library) and its adjoint both run in librts; this module only marshals
arguments.  ``rollout(engine, v0, B, alpha)`` returns the final positions and densities
(x_T, rho_T) as tensors whose backward gives d/dv0 (per particle), d/dB and d/dalpha.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import rts


class DiffEngine:
    """One differentiable rollout setup: scene, number of steps, checkpoint interval."""

    def __init__(self, params: dict, x0, xb, n_steps: int, ckpt_every: int = 10, stream=None):
        P = rts.make_params(params)
        n, nb = int(x0.shape[0]), int(xb.shape[0])
        x0 = rts._f32(x0, n)
        xb = rts._f32(xb, nb)
        h = C.c_void_p()
        st = rts.lib().rts_diff_create(C.byref(P), n, rts._ptr(x0), nb, rts._ptr(xb), int(n_steps),
                                        int(ckpt_every), rts._stream(stream), C.byref(h))
        if st != rts.RTS_OK:
            msg = rts.lib().rts_last_error(None)
            raise rts.RtsError(st, "rts_diff_create", msg.decode() if msg else "")
        self.handle = h
        self.n = n
        self.n_steps = int(n_steps)
        self.ckpt_every = int(ckpt_every)

    def _check(self, st, what):
        if st != rts.RTS_OK:
            msg = rts.lib().rts_diff_last_error(self.handle)
            raise rts.RtsError(st, what, msg.decode() if msg else "")

    def forward(self, v0: torch.Tensor, B: float, alpha: float):
        v0 = v0.detach().contiguous().to(torch.float32)
        dev = v0.device
        x = torch.empty((self.n, 3), dtype=torch.float32, device=dev)
        rho = torch.empty((self.n,), dtype=torch.float32, device=dev)
        st = rts.lib().rts_diff_forward(self.handle, rts._ptr(v0), C.c_float(B), C.c_float(alpha),
                                        rts._ptr(x), rts._ptr(rho))
        self._check(st, "rts_diff_forward")
        return x, rho

    def backward(self, gx, grho):
        dev = gx.device if gx is not None else grho.device
        gx = None if gx is None else gx.detach().contiguous().to(torch.float32)
        grho = None if grho is None else grho.detach().contiguous().to(torch.float32)
        gv = torch.empty((self.n, 3), dtype=torch.float32, device=dev)
        gB, ga = C.c_double(0.0), C.c_double(0.0)
        st = rts.lib().rts_diff_backward(self.handle, rts._ptr(gx), rts._ptr(grho), rts._ptr(gv),
                                         C.byref(gB), C.byref(ga))
        self._check(st, "rts_diff_backward")
        return gv, gB.value, ga.value

    def close(self):
        if self.handle:
            rts.lib().rts_diff_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v0, B, alpha, engine):
        x, rho = engine.forward(v0, float(B), float(alpha))
        ctx.engine = engine
        ctx.pdtype = (B.dtype, B.device) if torch.is_tensor(B) else (torch.float64, v0.device)
        return x, rho

    @staticmethod
    def backward(ctx, gx, grho):
        gv, gB, ga = ctx.engine.backward(gx, grho)
        dt, dev = ctx.pdtype
        return gv, torch.tensor(gB, dtype=dt, device=dev), torch.tensor(ga, dtype=dt, device=dev), None


def rollout(engine: DiffEngine, v0: torch.Tensor, B, alpha):
    """(x_T, rho_T) of the rollout; differentiable in v0, B and alpha (tensors)."""
    return _Rollout.apply(v0, B, alpha, engine)


def centroid_density_loss(x, rho, target, rho0=1000.0):
    """|mean(x_T) - target|^2 + mean |rho_T - rho0| / rho0 (torch, differentiable)."""
    c = x.mean(0) - torch.as_tensor(target, dtype=x.dtype, device=x.device)
    return (c * c).sum() + (rho - rho0).abs().mean() / rho0
