"""Pins of the oracle's relative L^2(Q_T) error (oracle/solve.l2_error_qt), the
measure of the convergence and coarsest-mesh studies of Section 6.

Functions that lie in a component's discrete space (Q1 hats in space times a
quadratic spline in time that vanishes at t = 0) are represented exactly by
coefficient arrays written out from the B-spline polar form (blossom): for the
quadratic B-spline B_i with knots t_i..t_{i+3}, t^2 has coefficient
t_{i+1} t_{i+2} and t has (t_{i+1} + t_{i+2}) / 2.  An approximation that
differs from the exact solution by a second such function then has a relative
error fixed by one-dimensional integrals (hat norms, the moments of t), so a
wrong space or time weight, a wrong interval length or a wrong T fails here.
"""
import numpy as np

import st_workloads as W
from oracle import solve


def _knots(N, T):
    return np.concatenate([[0.0, 0.0], np.linspace(0.0, T, N + 1), [T, T]])


def _coef_t2(N, T):
    t = _knots(N, T)
    return np.array([t[i + 1] * t[i + 2] for i in range(1, N + 2)])      # B_1 .. B_{N+1}


def _coef_t(N, T):
    t = _knots(N, T)
    return np.array([0.5 * (t[i + 1] + t[i + 2]) for i in range(1, N + 2)])


def _problem(d, hi, T, exact):
    return W.Problem(d=d, lo=(0.0,) * d, hi=hi, T=T, c2=lambda x: np.ones(len(x)), J=0, mx=2, mt=2,
                     exact=exact, name="l2_pin")


def _hat(x, centre, width):
    return np.maximum(0.0, 1.0 - np.abs(x - centre) / width)


def test_exactly_represented_function_has_zero_error():
    T = 1.0
    p = _problem(1, (1.0,), T, lambda x, t: _hat(x[:, 0], 0.5, 0.25) * t ** 2)
    space = np.array([0.0, 1.0, 0.0])                       # hat at x = 1/2 on the level-2 grid
    U = np.outer(_coef_t2(4, T), space)
    assert solve.l2_error_qt(p, [(2, 2, 1)], [U], 3, 3) < 1e-14


def test_space_perturbation_gives_the_hat_norm_ratio():
    """approx - exact = delta psi(x) t^2 with psi and phi hats of equal width: error = delta."""
    T, delta = 1.0, 0.03
    p = _problem(1, (1.0,), T, lambda x, t: _hat(x[:, 0], 0.5, 0.25) * t ** 2)
    U = np.outer(_coef_t2(4, T), np.array([delta, 1.0, 0.0]))
    assert abs(solve.l2_error_qt(p, [(2, 2, 1)], [U], 3, 3) - delta) < 1e-13


def test_time_perturbation_gives_the_moment_ratio_for_T_not_one():
    """approx - exact = eps phi(x) t on (0, T): error = eps sqrt(int t^2 / int t^4) = eps sqrt(5 / (3 T^2))."""
    T, eps = 2.0, 0.05
    p = _problem(1, (1.0,), T, lambda x, t: _hat(x[:, 0], 0.5, 0.25) * t ** 2)
    U = np.outer(_coef_t2(4, T) + eps * _coef_t(4, T), np.array([0.0, 1.0, 0.0]))
    want = eps * np.sqrt(5.0 / (3.0 * T ** 2))
    assert abs(solve.l2_error_qt(p, [(2, 2, 1)], [U], 3, 4) - want) < 1e-13 * want / eps


def test_two_dimensional_box_and_combination_of_components():
    """2D box (0,2) x (0,1): exact phi(x) phi(y) t^2 split over two components whose
    coefficients (+1 and -1) add up to it plus eps phi(x) phi(y) t: error eps sqrt(5/3)."""
    T, eps = 1.0, 0.02
    hx, hy = 0.5, 0.25                                       # level-2 cells of the box
    p = _problem(2, (2.0, 1.0), T,
                 lambda x, t: _hat(x[:, 0], 1.0, hx) * _hat(x[:, 1], 0.5, hy) * t ** 2)
    node = np.zeros(9)
    node[4] = 1.0                                            # interior node (1, 1) = (x = 1, y = 1/2)
    full = np.outer(_coef_t2(4, T) + eps * _coef_t(4, T), node)
    half = 0.5 * full
    # u^CF = 1.5 * full - 0.5 * full (two copies of the same component, coefficients +1, -1)
    err = solve.l2_error_qt(p, [(2, 2, 1), (2, 2, -1)], [1.5 * full, half], 3, 3)
    assert abs(err - eps * np.sqrt(5.0 / 3.0)) < 1e-13
