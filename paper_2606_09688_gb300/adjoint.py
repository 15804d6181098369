"""Receiver misfit J(c^2, g) and its gradient as a torch.autograd.Function.

c^2 and the spatial factor g of the source f = g(x) s(t) are nodal fields on
the uniform grid of level jp of the domain box.  They are passed to the
library as nodal arrays (st_problem.c2_nodal / g_nodal); the library samples
them (c^2 at cell centres, g at the nodes of every component level) by
multilinear interpolation and takes the gradient through the transpose of the
same interpolation.  The forward pass solves every component of Eq. (19),
evaluates J = 1/2 sum_s w_s sum_r (u^CF(x_r, t_s) - d[s, r])^2 and, in the same
call, the gradient by one adjoint solve per component (st_misfit_gradient);
the backward pass scales the stored gradient by the incoming one.  This module
only marshals arguments.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .st import ST_FP64, Solver


def problem_with(base, s):
    """base with f = g(x) s(t) (g given by nodal values at solver set-up), u0 = v0 = 0."""
    return dataclasses.replace(base, c2=None, terms=[(None, s)], f_general=None, u0=None, v0=None)


def nodal_solver(base, c2_nodal, g_nodal, s, jp, precision=ST_FP64):
    """A Solver for base with c^2 and g given by nodal values on the level-jp grid."""
    return Solver(problem_with(base, s), precision=precision, c2_nodal=np.asarray(c2_nodal, dtype=np.float64),
                  g_nodal=np.asarray(g_nodal, dtype=np.float64), param_level=jp)


class ReceiverMisfit(torch.autograd.Function):
    """J(c2_nodal, g_nodal) for fixed receivers, observations and levels."""

    @staticmethod
    def forward(ctx, c2_nodal, g_nodal, base, s, jp, receivers, jt_star, d_obs, precision=ST_FP64):
        with nodal_solver(base, c2_nodal.detach().cpu().numpy(), g_nodal.detach().cpu().numpy(), s, jp,
                          precision) as solver:
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
    with nodal_solver(base, c2_nodal, g_nodal, s, jp, precision) as solver:
        solver.solve(-1)
        return solver.receiver_values(jt_star, receivers).clone()
