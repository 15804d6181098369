"""Pins for the oracle's Q1 spatial matrices (CPU only)."""
import numpy as np
import pytest

import st_workloads as W
from oracle import space


@pytest.mark.parametrize("d", [1, 2, 3])
def test_mass_total_is_measure_and_constants_in_kernel(d):
    lo, hi = (0.0,) * d, (1.0, 2.0, 0.5)[:d]
    jx = 2
    c2 = np.random.default_rng(d).uniform(0.5, 3.0, size=(1 << jx) ** d)
    M, K = space.assemble_full(d, lo, hi, jx, c2)
    assert M.sum() == pytest.approx(np.prod(np.subtract(hi, lo)), rel=1e-14)   # sum (phi_a, phi_b) = |Omega|
    assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-12                      # grad 1 = 0


@pytest.mark.parametrize("jx", [2, 4, 6])
def test_1d_generalised_eigenvalues_closed_form(jx):
    """For c = 1 in 1D the eigenvalues of M^{-1} K are (6/h^2)(1 - cos th)/(2 + cos th),
    th = k pi h, k = 1..N-1 (discrete sine modes)."""
    p = W.standing_wave(1, 2 * jx, jx)
    sm = space.space_matrices(p, jx)
    N = 1 << jx
    h = 1.0 / N
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(sm["M"].toarray(), sm["K"].toarray())).real)
    th = np.arange(1, N) * np.pi * h
    assert np.allclose(ev, np.sort(6 / h ** 2 * (1 - np.cos(th)) / (2 + np.cos(th))), rtol=1e-10)


def test_stiffness_is_weighted_dirichlet_form_2d():
    """x^T K x = int c^2 |grad(I x)|^2, evaluated pointwise at 3x3 Gauss points of
    every cell from the bilinear interpolant (not from element matrices)."""
    d, jx = 2, 3
    p = W.layered_2d(2 * jx, jx)
    N = 1 << jx
    h = 1.0 / N
    c2 = p.c2(space.cell_centres(d, p.lo, p.hi, jx))
    M, K = space.assemble_full(d, p.lo, p.hi, jx, c2)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((N + 1) ** 2)
    X = x.reshape(N + 1, N + 1)                # [iy, ix]
    g, wg = np.polynomial.legendre.leggauss(3)
    e = 0.0
    m = 0.0
    for cy in range(N):
        for cx in range(N):
            v00, v10, v01, v11 = X[cy, cx], X[cy, cx + 1], X[cy + 1, cx], X[cy + 1, cx + 1]
            for a, wa in zip(g, wg):
                for b, wb in zip(g, wg):
                    s, t = 0.5 * (a + 1), 0.5 * (b + 1)
                    ux = ((v10 - v00) * (1 - t) + (v11 - v01) * t) / h
                    uy = ((v01 - v00) * (1 - s) + (v11 - v10) * s) / h
                    u = v00 * (1 - s) * (1 - t) + v10 * s * (1 - t) + v01 * (1 - s) * t + v11 * s * t
                    wq = wa * wb * 0.25 * h * h
                    e += wq * c2[cy * N + cx] * (ux * ux + uy * uy)
                    m += wq * u * u
    assert x @ (K @ x) == pytest.approx(e, rel=1e-12)
    assert x @ (M @ x) == pytest.approx(m, rel=1e-12)


def test_1d_stiffness_of_parabola_interpolant():
    """In 1D, (K I u)_a = -h u'' for u = x(1-x): K I u = 2 M 1 on interior rows."""
    p = W.standing_wave(1, 8, 4)
    sm = space.space_matrices(p, 4)
    x = space.node_coords(1, p.lo, p.hi, 4)[:, 0]
    u = x * (1 - x)
    assert np.allclose(sm["K_load"] @ u, 2 * (sm["M_load"] @ np.ones_like(u)), atol=1e-13)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_interpolation_reproduces_multilinear(d):
    lo, hi = (-1.0,) * d, (1.0, 2.0, 3.0)[:d]
    jx = 2
    nodes = space.node_coords(d, lo, hi, jx)
    coef = np.array([0.3, -1.2, 0.7])[:d]
    f = lambda X: 1.5 + X @ coef + (np.prod(X, axis=1) if d > 1 else 0.0)
    pts = np.random.default_rng(1).uniform(lo, hi, size=(50, d))
    assert np.allclose(space.interpolate_nodal(f(nodes), d, lo, hi, jx, pts), f(pts), atol=1e-12)
