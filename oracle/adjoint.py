"""Gradient of a receiver misfit with respect to c^2 and the source factor,
through the adjoint of each component's Galerkin system (Eq. (9), Eq. (30)).

TEST INFRASTRUCTURE ONLY: imported by tests/ and bench.py's baseline legs.

Objective.  Receivers x_r, the target times t_s = s T / 2^jt* (s = 0..2^jt*)
with trapezoid weights w_s, observations d[s, r]:

    J = 1/2 sum_s w_s sum_r (u^CF(x_r, t_s) - d[s, r])^2,   u^CF of Eq. (19).

Parameters.  c^2 and the spatial factor g of a separable source f = g(x) s(t)
are given by nodal values on a uniform parameter grid of level jp ((2^jp+1)^d
nodes); the method sees c^2 at cell centres and g at the nodes of each
component's level, both by multilinear interpolation of the nodal values
(linear maps P_k and Q_k).

Gradient.  For component k, S_k U_k = F_k with S_k = A (x) M + B (x) K(c2),
K(c2) = sum_e c2_e K_e (K_e the unit-coefficient element stiffness).  J depends
on U_k through G_k = dJ/dU_k = c_k E_k^T (w * e) (E_k: evaluation at the
receivers, e the misfit).  With the adjoint state S_k^T L_k = G_k:

    dJ/dc2_e  = - L_k^T (B (x) K_e) U_k          (per cell of level jx_k)
    dJ/d(I_k g) = M_load^T sum_i b_k[i] L_k[i]    (b_k[i] = (s, psi_i')_e)

then chained through P_k^T, Q_k^T onto the parameter grid and summed over k.
u0 = v0 = 0 is assumed (the lifting would add terms; the configuration has
none).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import combination, space, timebasis, timemats
from . import solve as osolve


def interp_matrix(d, lo, hi, jp, pts):
    """Sparse matrix of multilinear interpolation from the (2^jp+1)^d nodal
    values of level jp (all nodes, x fastest) to the points."""
    N, h = space.grid(d, lo, hi, jp)
    nn = N + 1
    rows, cols, vals = [], [], []
    idx, frac = [], []
    for k in range(d):
        s = (pts[:, k] - lo[k]) / h[k]
        c = np.clip(np.floor(s).astype(np.int64), 0, N - 1)
        idx.append(c)
        frac.append(s - c)
    for c in range(1 << d):
        w = np.ones(len(pts))
        g = np.zeros(len(pts), dtype=np.int64)
        stride = 1
        for k in range(d):
            b = (c >> k) & 1
            w = w * (frac[k] if b else (1.0 - frac[k]))
            g = g + (idx[k] + b) * stride
            stride *= nn
        rows.append(np.arange(len(pts)))
        cols.append(g)
        vals.append(w)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(len(pts), nn ** d))


def nodal_function(values, d, lo, hi, jp):
    """The multilinear interpolant of nodal values, as a callable on points."""
    values = np.asarray(values, dtype=np.float64)
    return lambda pts: interp_matrix(d, lo, hi, jp, np.asarray(pts, dtype=np.float64)) @ values


def with_parameters(problem, c2_nodal, g_nodal, s, jp):
    """A copy of problem with c^2 and the source f = g(x) s(t) given by nodal values."""
    import dataclasses
    d, lo, hi = problem.d, problem.lo, problem.hi
    return dataclasses.replace(problem, c2=nodal_function(c2_nodal, d, lo, hi, jp),
                               terms=[(nodal_function(g_nodal, d, lo, hi, jp), s)], f_general=None,
                               u0=None, v0=None)


def target_times(problem, jt_star):
    """t_s and trapezoid weights w_s on the uniform target times."""
    n = 1 << jt_star
    t = np.linspace(0.0, problem.T, n + 1)
    w = np.full(n + 1, problem.T / n)
    w[0] *= 0.5
    w[-1] *= 0.5
    return t, w


def receiver_values(problem, comps, sols, receivers, jt_star):
    """u^CF(x_r, t_s), shape (2^jt*+1, n_receivers)."""
    t, _ = target_times(problem, jt_star)
    return osolve.combine(problem, comps, sols, receivers, t)


def objective(problem, comps, sols, receivers, jt_star, d_obs):
    """J and the misfit e[s, r]."""
    _, w = target_times(problem, jt_star)
    e = receiver_values(problem, comps, sols, receivers, jt_star) - d_obs
    return 0.5 * float(np.sum(w[:, None] * e * e)), e


def _interior_eval(problem, jx, receivers):
    """E_x: receivers x interior nodes of level jx (Q1 evaluation of interior values)."""
    E = interp_matrix(problem.d, problem.lo, problem.hi, jx, receivers)
    inner = np.nonzero(space.interior_mask(problem.d, jx))[0]
    return E[:, inner]


def _cell_corners(d, jx):
    """Global (all-node) index of the 2^d corners of every cell, cells x-fastest."""
    N = 1 << jx
    nn = N + 1
    cells = np.stack(np.meshgrid(*([np.arange(N)] * d), indexing="ij")[::-1], axis=-1).reshape(-1, d)
    corner = np.zeros((len(cells), 1 << d), dtype=np.int64)
    for c in range(1 << d):
        g = np.zeros(len(cells), dtype=np.int64)
        stride = 1
        for k in range(d):
            g += (cells[:, k] + ((c >> k) & 1)) * stride
            stride *= nn
        corner[:, c] = g
    return corner


def adjoint_state(problem, jx, jt, G):
    """L with (A^T (x) M + B^T (x) K) vec(L) = vec(G), time-major like U."""
    S = osolve.system_matrix(problem, jx, jt)
    L = spl.spsolve(S.T.tocsc(), G.ravel())
    return np.asarray(L).reshape(G.shape)


def gradient(problem, c2_nodal, g_nodal, s, jp, receivers, jt_star, d_obs):
    """J, dJ/dc2_nodal and dJ/dg_nodal (both on the (2^jp+1)^d parameter grid)."""
    p = with_parameters(problem, c2_nodal, g_nodal, s, jp)
    d, lo, hi, T = p.d, p.lo, p.hi, p.T
    comps = combination.components(p.J, p.mx, p.mt)
    sols = [osolve.solve_component(p, jx, jt) for jx, jt, _ in comps]
    J, e = objective(p, comps, sols, receivers, jt_star, d_obs)
    t, w = target_times(p, jt_star)
    gc2 = np.zeros(len(c2_nodal))
    gg = np.zeros(len(g_nodal))
    for (jx, jt, c), U in zip(comps, sols):
        Pt = timebasis.psi(t, 1 << jt, T, 0)                     # (n_times, n_t)
        Ex = _interior_eval(p, jx, receivers)                     # (n_recv, N_int)
        G = c * (Pt.T @ (w[:, None] * e)) @ Ex.toarray()          # dJ/dU_k, (n_t, N_int)
        L = adjoint_state(p, jx, jt, G)
        A, B = timemats.time_matrices(jt, T)
        Z = B @ U                                                 # sum_j B[i, j] U[j]
        inner = np.nonzero(space.interior_mask(d, jx))[0]
        N, h = space.grid(d, lo, hi, jx)
        nall = (N + 1) ** d
        L_all = np.zeros((L.shape[0], nall))
        Z_all = np.zeros((L.shape[0], nall))
        L_all[:, inner] = L
        Z_all[:, inner] = Z
        corner = _cell_corners(d, jx)
        _, Ke = space.element_matrices(d, h)
        gcell = -np.einsum("icp,pq,icq->c", L_all[:, corner], Ke, Z_all[:, corner])
        P = interp_matrix(d, lo, hi, jp, space.cell_centres(d, lo, hi, jx))
        gc2 += P.T @ gcell
        sm = space.space_matrices(p, jx)
        b = timemats.load_separable(s, jt, T)
        gI = sm["M_load"].T @ (b @ L)                             # dJ/d(I_k g), all nodes
        Q = interp_matrix(d, lo, hi, jp, space.node_coords(d, lo, hi, jx))
        gg += Q.T @ gI
    return J, gc2, gg


def objective_at(problem, c2_nodal, g_nodal, s, jp, receivers, jt_star, d_obs):
    """J for the given parameters (forward solves only), for finite differences."""
    p = with_parameters(problem, c2_nodal, g_nodal, s, jp)
    comps = combination.components(p.J, p.mx, p.mt)
    sols = [osolve.solve_component(p, jx, jt) for jx, jt, _ in comps]
    return objective(p, comps, sols, receivers, jt_star, d_obs)[0]
