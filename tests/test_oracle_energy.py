"""Pins of the oracle's energy functional E(s; v) of Section 6.3.

* The Q1 gradient evaluation against central differences of the interpolant.
* The functional on closed forms: the standing wave u = sin(pi x) cos(pi t)
  (c = 1) has E = pi^2/4 at every t; the travelling wave of Section 6.3 has a
  constant energy (no source, Dirichlet data), equal to the t = 0 value.
* E(t; u^CF) by the exact derivative route against an independent route: finite
  differences in t and x of the combined solution evaluated pointwise.
* Convergence: the relative energy error of u^CF on the travelling wave decreases
  under refinement and stays bounded over [0, T].
"""
import dataclasses

import numpy as np
import pytest

import st_workloads as W
from oracle import energy, solve as osolve, space


def test_q1_gradient_matches_central_differences():
    p = W.layered_2d(6, 2)
    rng = np.random.default_rng(0)
    jx = 3
    vals = rng.standard_normal(((1 << jx) + 1) ** 2)
    pts = rng.uniform(0.05, 0.95, size=(50, 2))
    g = space.interpolate_nodal_grad(vals, 2, p.lo, p.hi, jx, pts)
    eps = 1e-6
    for k in range(2):
        e = np.zeros(2)
        e[k] = eps
        fd = (space.interpolate_nodal(vals, 2, p.lo, p.hi, jx, pts + e) -
              space.interpolate_nodal(vals, 2, p.lo, p.hi, jx, pts - e)) / (2 * eps)
        assert np.max(np.abs(fd - g[:, k])) < 1e-6 * max(1.0, np.max(np.abs(g[:, k])))


def test_energy_of_closed_forms():
    sw = W.standing_wave(1, 6, 1)
    t = np.linspace(0.0, 1.0, 7)
    E = energy.energy_of(sw, lambda x, s: -np.pi * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * s),
                         lambda x, s: (np.pi * np.cos(np.pi * x[:, 0]) * np.cos(np.pi * s))[:, None], 4, t)
    assert np.max(np.abs(E - np.pi ** 2 / 4)) < 1e-10
    tw = W.travelling_wave(4)
    Et = energy.energy_of(tw, tw.exact_dt, tw.exact_grad, 8, np.linspace(0.0, 1.0, 9))
    assert np.max(np.abs(Et - Et[0])) < 1e-10 * Et[0]


def test_energy_of_the_combination_against_finite_differences():
    p = W.travelling_wave(3)
    comps, sols = osolve.solve_all(p)
    jq = max(jx for jx, _, _ in comps)
    times = np.array([0.13, 0.47, 0.87])   # off the time knots (central differences of a C^1 spline)
    E = energy.energy_cf(p, comps, sols, jq, times)
    # independent route: u^CF pointwise, derivatives by central differences on a fine Gauss set
    xg, wg = np.polynomial.legendre.leggauss(3)
    N, h = space.grid(1, p.lo, p.hi, jq)
    cells = space.cell_centres(1, p.lo, p.hi, jq)
    pts = (cells[:, None, 0] + 0.5 * xg[None, :] * h[0]).reshape(-1, 1)
    w = np.tile(wg * 0.5 * h[0], len(cells))
    et, ex = 1e-5, 1e-7
    for s, t in enumerate(times):
        u = lambda x, tt: osolve.combine(p, comps, sols, x, np.array([tt]))[0]
        dt = (u(pts, t + et) - u(pts, t - et)) / (2 * et)
        dx = (u(pts + ex, t) - u(pts - ex, t)) / (2 * ex)
        Efd = 0.5 * np.sum(w * (dt ** 2 + 0.64 * dx ** 2))
        assert abs(Efd - E[s]) < 1e-6 * E[s], (t, Efd, E[s])


def test_energy_error_of_the_combination_decreases_and_stays_bounded():
    times = np.linspace(0.0, 1.0, 41)
    errs = []
    for J in (3, 4, 5):
        p = W.travelling_wave(J)
        comps, sols = osolve.solve_all(p)
        jq = max(jx for jx, _, _ in comps)
        E = energy.energy_cf(p, comps, sols, jq, times)
        Eex = energy.energy_of(p, p.exact_dt, p.exact_grad, jq + 2, times[:1])[0]
        errs.append(np.abs(E - Eex) / Eex)
    assert np.max(errs[2]) < np.max(errs[1]) < np.max(errs[0])
    assert np.max(errs[2]) < 0.05


@pytest.mark.parametrize("pt", [3, 4])
def test_energy_error_with_higher_time_degree_decreases(pt):
    """The same energy study with time splines of degree 3 and 4 (maximal regularity):
    the relative error of E(t; u^CF) against the conserved exact energy falls with
    the level and stays small, as for quadratic splines."""
    times = np.linspace(0.0, 1.0, 21)
    errs = []
    for J in (3, 4, 5):
        base = W.travelling_wave(J)
        p = dataclasses.replace(base, pt=pt)
        comps, sols = osolve.solve_all(p)
        jq = max(jx for jx, _, _ in comps)
        E = energy.energy_cf(p, comps, sols, jq, times)
        Eex = energy.energy_of(p, base.exact_dt, base.exact_grad, jq + 2, times[:1])[0]
        errs.append(np.max(np.abs(E - Eex) / Eex))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 0.05, errs
