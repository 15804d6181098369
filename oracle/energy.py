"""Energy of the combined solution (Section 6.3):

    E(s; v) = 1/2 ( ||d_t v(., s)||^2_{L^2(Omega)} + ||c grad v(., s)||^2_{L^2(Omega)} ).

For v = u^CF_J (Eq. (19)) the integrands are evaluated exactly: every
component is Q1 in space (its gradient is the derivative of the multilinear
interpolant of its nodal values, the lifting u0 included) and a quadratic
spline in time (its time derivative is the B-spline derivative), summed with
the +-1 coefficients.  The integral over Omega is taken by tensor Gauss
quadrature on the cells of an evaluation level jq that is at least as fine as
every component's spatial level, so every integrand is a polynomial on each
cell and 3 points per direction integrate it exactly.  c^2 is sampled at the
centres of the level-jq cells (cellwise constant, as in the discretisation).
"""
import numpy as np

from . import space, timebasis


def _gauss_cells(problem, jq, npts=3):
    """Gauss points (n, d) and weights of every cell of level jq, and the cell of each point."""
    d = problem.d
    xg, wg = np.polynomial.legendre.leggauss(npts)
    N, h = space.grid(d, problem.lo, problem.hi, jq)
    cells = space.cell_centres(d, problem.lo, problem.hi, jq)
    offs = np.stack(np.meshgrid(*([xg] * d), indexing="ij"), axis=-1).reshape(-1, d)
    wloc = np.prod(np.stack(np.meshgrid(*([wg] * d), indexing="ij"), axis=-1).reshape(-1, d), axis=1)
    pts = (cells[:, None, :] + 0.5 * offs[None, :, :] * h[None, None, :]).reshape(-1, d)
    w = np.tile(wloc, len(cells)) * np.prod(h) / (2 ** d)
    cell_of = np.repeat(np.arange(len(cells)), len(wloc))
    return pts, w, cells, cell_of


def component_derivatives(problem, jx, jt, U, pts, times):
    """(d_t u_k, grad u_k) of one component at the points and times:
    shapes (len(times), len(pts)) and (len(times), len(pts), d)."""
    from .solve import _nodal, all_node_values
    N_t = 1 << jt
    pt = getattr(problem, "pt", 2)
    P0 = timebasis.psi(np.asarray(times, dtype=np.float64), N_t, problem.T, 0, pt)
    P1 = timebasis.psi(np.asarray(times, dtype=np.float64), N_t, problem.T, 1, pt)
    lift = _nodal(problem.u0, space.node_coords(problem.d, problem.lo, problem.hi, jx))
    dt = np.zeros((len(times), len(pts)))
    gr = np.zeros((len(times), len(pts), problem.d))
    for s in range(len(times)):
        dt[s] = space.interpolate_nodal(all_node_values(problem, jx, P1[s] @ U), problem.d, problem.lo, problem.hi,
                                        jx, pts)
        vals = all_node_values(problem, jx, P0[s] @ U) + lift
        gr[s] = space.interpolate_nodal_grad(vals, problem.d, problem.lo, problem.hi, jx, pts)
    return dt, gr


def energy_cf(problem, comps, sols, jq, times):
    """E(t; u^CF) at the given times, evaluation level jq >= every component's spatial level."""
    pts, w, cells, cell_of = _gauss_cells(problem, jq)
    c2 = np.asarray(problem.c2(cells), dtype=np.float64)[cell_of]
    dt = np.zeros((len(times), len(pts)))
    gr = np.zeros((len(times), len(pts), problem.d))
    for (jx, jt, c), U in zip(comps, sols):
        a, b = component_derivatives(problem, jx, jt, U, pts, times)
        dt += c * a
        gr += c * b
    return 0.5 * (np.sum(w[None, :] * dt ** 2, axis=1) + np.sum(w[None, :] * c2[None, :] * np.sum(gr ** 2, axis=2),
                                                               axis=1))


def energy_of(problem, dt_fn, grad_fn, jq, times, npts=5):
    """E(t; v) of a function given by callables dt_fn(x, t) -> (n,), grad_fn(x, t) -> (n, d),
    by Gauss quadrature with npts points per direction on the level-jq cells."""
    pts, w, cells, cell_of = _gauss_cells(problem, jq, npts)
    c2 = np.asarray(problem.c2(cells), dtype=np.float64)[cell_of]
    out = np.zeros(len(times))
    for s, t in enumerate(times):
        a = dt_fn(pts, t)
        g = grad_fn(pts, t)
        out[s] = 0.5 * (np.sum(w * a ** 2) + np.sum(w * c2 * np.sum(g ** 2, axis=1)))
    return out
