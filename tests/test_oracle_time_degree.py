"""Pins for the oracle's time splines of degree p_t = 3, 4 with maximal regularity
C^{p_t - 1} (the conjectured cases of Table "validity"), next to p_t = 2.

Each check compares against something the oracle does not compute itself: the
truncated-power closed form of the uniform cardinal B-spline, Marsden's identity
(the coefficients of t^k are the blossoms e_k(t_{i+1}..t_{i+p}) / C(p, k)),
finite differences, continuity of the derivatives up to order p - 1 at the
knots, the identity of Eq. (3) under an independent 20-point rule, exact
reproduction of ODE solutions t^k (k <= p) that lie in V_t (Eq. (10)), and the
O(h^2) convergence of the combined solution (p_x = 1 bounds the rate).
"""
import math
from itertools import combinations

import numpy as np
import pytest

import st_workloads as W
from oracle import combination, solve, timebasis, timemats

T = 1.0
DEGREES = [2, 3, 4]


def cardinal(s, p):
    """Uniform cardinal B-spline of degree p on knots 0..p+1:
    (1/p!) sum_j (-1)^j C(p+1, j) (s - j)_+^p."""
    s = np.asarray(s, dtype=float)
    out = np.zeros_like(s)
    for j in range(p + 2):
        out += (-1) ** j * math.comb(p + 1, j) * np.maximum(s - j, 0.0) ** p
    out /= math.factorial(p)
    return np.where((s >= 0) & (s <= p + 1), out, 0.0)


def blossom_coefficients(N, Tf, p, k):
    """Coefficients of t^k in the B-spline basis B_0 .. B_{N+p-1} (Marsden's identity)."""
    kv = timebasis.knots(N, Tf, p)
    c = []
    for i in range(N + p):
        tau = kv[i + 1:i + p + 1]
        e = sum(np.prod(sub) for sub in combinations(tau, k)) if k > 0 else 1.0
        c.append(e / math.comb(p, k))
    return np.array(c)


@pytest.mark.parametrize("p", DEGREES)
@pytest.mark.parametrize("N", [4, 8])
def test_partition_of_unity_and_monomial_reproduction(p, N):
    t = np.linspace(0, T, 401)
    B = timebasis.bsplines(t, N, T, 0, p)
    assert B.shape[1] == N + p
    assert np.allclose(B.sum(axis=1), 1.0, atol=1e-14)
    for k in range(1, p + 1):
        assert np.allclose(B @ blossom_coefficients(N, T, p, k), t ** k, atol=1e-13), k


@pytest.mark.parametrize("p", DEGREES)
def test_interior_splines_match_the_truncated_power_form(p):
    N = 8
    h = T / N
    t = np.linspace(0, T, 1201)
    B = timebasis.bsplines(t, N, T, 0, p)
    # B_i for p <= i <= N - 1 has the simple knots (i - p) h .. (i + 1) h
    for i in range(p, N):
        assert np.allclose(B[:, i], cardinal(t / h - (i - p), p), atol=1e-13), i


@pytest.mark.parametrize("p", [3, 4])
def test_derivatives_against_finite_differences_and_continuity(p):
    N = 8
    h = T / N
    t = (np.arange(N)[:, None] * h + np.array([0.23, 0.5, 0.81])[None, :] * h).ravel()
    e = 1e-5
    Bf = lambda s: timebasis.bsplines(s, N, T, 0, p)
    d1 = (Bf(t + e) - Bf(t - e)) / (2 * e)
    d2 = (Bf(t + e) - 2 * Bf(t) + Bf(t - e)) / e ** 2
    assert np.allclose(timebasis.bsplines(t, N, T, 1, p), d1, atol=1e-7 * N ** 3)
    assert np.allclose(timebasis.bsplines(t, N, T, 2, p), d2, atol=1e-3 * N ** 2)
    # maximal regularity: B and B', B'' (p >= 3) continuous across the interior knots
    knots = np.arange(1, N) * h
    for deriv in (0, 1, 2):
        left = timebasis.bsplines(knots - 1e-9, N, T, deriv, p)
        right = timebasis.bsplines(knots + 1e-9, N, T, deriv, p)
        assert np.allclose(left, right, atol=1e-6 * N ** (deriv + 1)), deriv


@pytest.mark.parametrize("p", DEGREES)
@pytest.mark.parametrize("jt", [1, 3, 5])
def test_basis_vanishes_at_zero_and_dimension(p, jt):
    N = 1 << jt
    P = timebasis.psi(np.array([0.0]), N, T, 0, p)
    assert np.all(P == 0.0)
    # dim V_jt = N (p - r) + r with r = p - 1 (Section 3.2)
    assert P.shape[1] == N * (p - (p - 1)) + (p - 1) == timebasis.n_time_dofs(jt, p) \
        == combination.time_dofs(jt, p)


def _weighted_norm2(w, N, Tf, order=20):
    x, wq = np.polynomial.legendre.leggauss(order)
    h = Tf / N
    t = (np.arange(N)[:, None] * h + (x[None, :] + 1) * 0.5 * h).ravel()
    ww = np.tile(wq * 0.5 * h, N) * np.exp(-t / Tf)
    return np.sum(ww * w(t) ** 2)


@pytest.mark.parametrize("p", [3, 4])
@pytest.mark.parametrize("jt,Tf", [(2, 1.0), (3, 2.5)])
def test_energy_identity_eq3(p, jt, Tf):
    """Eq. (3): c^T B c = ||w||_e^2 / (2T) + w(T)^2 / (2e) and
    c^T A c = ||w'||_e^2 / (2T) + w'(T)^2 / (2e) + w'(0)^2 / 2 for w = sum c_i psi_i."""
    N = 1 << jt
    A, B = timemats.time_matrices(jt, Tf, p)
    rng = np.random.default_rng(10 * p + jt)
    for _ in range(3):
        c = rng.standard_normal(timebasis.n_time_dofs(jt, p))
        w = lambda t: timebasis.psi(t, N, Tf, 0, p) @ c
        dw = lambda t: timebasis.psi(t, N, Tf, 1, p) @ c
        wT, dwT, dw0 = w(np.array([Tf]))[0], dw(np.array([Tf]))[0], dw(np.array([0.0]))[0]
        assert c @ B @ c == pytest.approx(_weighted_norm2(w, N, Tf) / (2 * Tf) + wT ** 2 / (2 * np.e), rel=1e-12)
        assert c @ A @ c == pytest.approx(_weighted_norm2(dw, N, Tf) / (2 * Tf) + dwT ** 2 / (2 * np.e)
                                          + 0.5 * dw0 ** 2, rel=1e-12)


@pytest.mark.parametrize("p", [3, 4])
def test_symmetric_parts_positive_definite(p):
    """Proof of Prop. 1 holds for any C^1 time space: positive definite symmetric parts."""
    for jt in (1, 3, 5):
        A, B = timemats.time_matrices(jt, T, p)
        assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
        assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


@pytest.mark.parametrize("p", [3, 4])
@pytest.mark.parametrize("mu", [0.0, 3.7, 250.0])
def test_ode_solutions_t_to_the_k_are_reproduced(p, mu):
    """(A + mu B) c = b, b[i] = (f, psi_i')_e + v0 psi_i'(0), is the Galerkin method of
    Eq. (10) for q'' + mu q = f, q(0) = 0, q'(0) = v0; q = t^k (k <= p) lies in V_t, so its
    blossom coefficients (B_0's, zero, dropped) come back exactly."""
    jt = 3
    A, B = timemats.time_matrices(jt, T, p)
    d0 = timemats.dpsi_at_zero(jt, T, p)
    for k in range(1, p + 1):
        f = lambda t, k=k: (k * (k - 1) * t ** (k - 2) if k >= 2 else 0.0 * t) + mu * t ** k
        b = timemats.load_separable(f, jt, T, p) + (1.0 if k == 1 else 0.0) * d0
        want = blossom_coefficients(1 << jt, T, p, k)
        assert abs(want[0]) < 1e-15
        assert np.allclose(np.linalg.solve(A + mu * B, b), want[1:], atol=1e-10), k


@pytest.mark.parametrize("p", [3, 4])
def test_combination_converges_at_second_order(p):
    """u^CF of the 1D standing wave with time splines of degree p: the L^2(Q_T) error
    falls by about 4 per level (p_x = 1 bounds the rate at h^2, Theorem 1)."""
    errs = []
    for n in (5, 6, 7):
        base = W.standing_wave(1, n, 1)
        prob = W.Problem(**{**base.__dict__, "pt": p})
        comps, sols = solve.solve_all(prob)
        errs.append(solve.l2_error_qt(prob, comps, sols, prob.mx + prob.J, prob.mt + prob.J))
    rates = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(r > 3.0 for r in rates), (errs, rates)
