"""Receiver misfit J(c^2, g) and its gradient as a torch.autograd.Function.

c^2 and the spatial factor g of the source f = g(x) s(t) are nodal fields on
the uniform grid of level jp of the domain box; the solver samples c^2 at cell
centres and g at the nodes of every component level by multilinear
interpolation of those fields (host-side data preparation, as for any
problem).  The forward pass solves every component of Eq. (19), evaluates
J = 1/2 sum_s w_s sum_r (u^CF(x_r, t_s) - d[s, r])^2 and, in the same call,
the gradient by one adjoint solve per component (st_misfit_gradient); the
backward pass scales the stored gradient by the incoming one.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .st import ST_FP64, Solver


def nodal_interpolant(values: np.ndarray, d: int, lo, hi, jp: int):
    """Multilinear interpolant of the (2^jp+1)^d nodal values (x fastest) on the box, as a callback."""
    values = np.asarray(values, dtype=np.float64)
    Np = 1 << jp
    lo = np.asarray(lo[:d], dtype=np.float64)
    h = (np.asarray(hi[:d], dtype=np.float64) - lo) / Np

    def f(pts):
        pts = np.asarray(pts, dtype=np.float64)
        t = (pts - lo) / h
        c = np.clip(np.floor(t).astype(np.int64), 0, Np - 1)
        fr = t - c
        out = np.zeros(len(pts))
        for e in range(1 << d):
            w = np.ones(len(pts))
            idx = np.zeros(len(pts), dtype=np.int64)
            st = 1
            for k in range(d):
                b = (e >> k) & 1
                w = w * (fr[:, k] if b else 1.0 - fr[:, k])
                idx = idx + (c[:, k] + b) * st
                st *= Np + 1
            out += w * values[idx]
        return out
    return f


def problem_with(base, c2_nodal, g_nodal, s, jp):
    """base with c^2 and f = g(x) s(t) given by nodal values on the level-jp grid (u0 = v0 = 0)."""
    d = base.d
    return dataclasses.replace(base, c2=nodal_interpolant(c2_nodal, d, base.lo, base.hi, jp),
                               terms=[(nodal_interpolant(g_nodal, d, base.lo, base.hi, jp), s)],
                               f_general=None, u0=None, v0=None)


class ReceiverMisfit(torch.autograd.Function):
    """J(c2_nodal, g_nodal) for fixed receivers, observations and levels."""

    @staticmethod
    def forward(ctx, c2_nodal, g_nodal, base, s, jp, receivers, jt_star, d_obs, precision=ST_FP64):
        p = problem_with(base, c2_nodal.detach().cpu().numpy(), g_nodal.detach().cpu().numpy(), s, jp)
        with Solver(p, precision=precision) as solver:
            solver.solve(-1)
            J, dc2, dg, _ = solver.misfit_gradient(jt_star, receivers, d_obs, jp)
        ctx.save_for_backward(dc2.to(c2_nodal.device, c2_nodal.dtype), dg.to(g_nodal.device, g_nodal.dtype))
        return torch.tensor(J, dtype=c2_nodal.dtype, device=c2_nodal.device)

    @staticmethod
    def backward(ctx, grad_J):
        dc2, dg = ctx.saved_tensors
        return grad_J * dc2, grad_J * dg, None, None, None, None, None, None, None


def receiver_misfit(c2_nodal, g_nodal, base, s, jp, receivers, jt_star, d_obs, precision=ST_FP64):
    return ReceiverMisfit.apply(c2_nodal, g_nodal, base, s, jp, receivers, jt_star, d_obs, precision)


def observations(base, c2_nodal, g_nodal, s, jp, receivers, jt_star, precision=ST_FP64):
    """u^CF at the receivers for the given parameters (synthetic data), (times, receivers) on the GPU."""
    p = problem_with(base, np.asarray(c2_nodal), np.asarray(g_nodal), s, jp)
    with Solver(p, precision=precision) as solver:
        solver.solve(-1)
        return solver.receiver_values(jt_star, receivers).clone()
