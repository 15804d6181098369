"""Pins for the oracle's time basis and time matrices (CPU only).

Each check compares against something the oracle does not compute itself:
textbook closed forms of uniform quadratic B-splines, polynomial reproduction,
finite differences, the identity of Eq. (3), and exact reproduction of ODE
solutions that lie in the discrete space (Galerkin property, Eq. (10)).
"""
import numpy as np
import pytest

from oracle import timebasis, timemats

T = 1.0


def cardinal_quadratic(s):
    """Uniform quadratic B-spline on knots 0,1,2,3 (textbook closed form)."""
    s = np.asarray(s, dtype=float)
    out = np.zeros_like(s)
    a = (s >= 0) & (s < 1)
    b = (s >= 1) & (s < 2)
    c = (s >= 2) & (s <= 3)
    out[a] = 0.5 * s[a] ** 2
    out[b] = 0.5 * (-2 * s[b] ** 2 + 6 * s[b] - 3)
    out[c] = 0.5 * (3 - s[c]) ** 2
    return out


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_partition_of_unity_and_reproduction(N):
    t = np.linspace(0, T, 401)
    B = timebasis.bsplines(t, N, T)
    assert np.allclose(B.sum(axis=1), 1.0, atol=1e-14)
    kv = timebasis.knots(N, T)
    # quadratic splines reproduce t (Greville abscissae) and t^2 (products of inner knots)
    greville = 0.5 * (kv[1:N + 3] + kv[2:N + 4])
    assert np.allclose(B @ greville, t, atol=1e-14)
    assert np.allclose(B @ (kv[1:N + 3] * kv[2:N + 4]), t * t, atol=1e-14)


@pytest.mark.parametrize("N", [4, 8])
def test_interior_splines_match_cardinal_closed_form(N):
    h = T / N
    t = np.linspace(0, T, 1001)
    B = timebasis.bsplines(t, N, T)
    # B_i for 2 <= i <= N-1 is the cardinal spline shifted to start at knot (i-2) h
    for i in range(2, N):
        assert np.allclose(B[:, i], cardinal_quadratic(t / h - (i - 2)), atol=1e-13)


@pytest.mark.parametrize("N", [4, 8])
def test_derivatives_against_finite_differences(N):
    h = T / N
    # points away from knots so that B'' (piecewise constant) is well defined
    t = (np.arange(N)[:, None] * h + np.array([0.21, 0.5, 0.83])[None, :] * h).ravel()
    e = 1e-6
    B = lambda s: timebasis.bsplines(s, N, T)
    d1 = (B(t + e) - B(t - e)) / (2 * e)
    d2 = (B(t + e) - 2 * B(t) + B(t - e)) / e ** 2
    assert np.allclose(timebasis.bsplines(t, N, T, 1), d1, atol=1e-6 * N)
    assert np.allclose(timebasis.bsplines(t, N, T, 2), d2, rtol=1e-3, atol=1e-2 * N * N)


@pytest.mark.parametrize("jt", [1, 2, 3, 5])
def test_basis_vanishes_at_zero_and_dimension(jt):
    N = 1 << jt
    P = timebasis.psi(np.array([0.0]), N, T)
    assert np.all(P == 0.0)
    # dim V_jt = N (p - r) + r with p = 2, r = 1 (Section 3.2)
    assert P.shape[1] == N * (2 - 1) + 1 == timebasis.n_time_dofs(jt)


def _weighted_norm2(w, N, T, order=20):
    """int_0^T w(t)^2 exp(-t/T) dt by a 20-point rule per interval (independent of the 8-point one)."""
    x, wq = np.polynomial.legendre.leggauss(order)
    h = T / N
    t = (np.arange(N)[:, None] * h + (x[None, :] + 1) * 0.5 * h).ravel()
    ww = np.tile(wq * 0.5 * h, N) * np.exp(-t / T)
    return np.sum(ww * w(t) ** 2)


@pytest.mark.parametrize("jt,Tf", [(2, 1.0), (4, 1.0), (3, 2.5)])
def test_energy_identity_eq3(jt, Tf):
    """Eq. (3) for w = sum c_i psi_i (w(0) = 0) gives
    c^T B c = ||w||_e^2 / (2T) + w(T)^2 / (2e) and, applied to w',
    c^T A c = ||w'||_e^2 / (2T) + w'(T)^2 / (2e) + w'(0)^2 / 2."""
    N = 1 << jt
    A, B = timemats.time_matrices(jt, Tf)
    rng = np.random.default_rng(jt)
    for _ in range(4):
        c = rng.standard_normal(N + 1)
        w = lambda t: timebasis.psi(t, N, Tf) @ c
        dw = lambda t: timebasis.psi(t, N, Tf, 1) @ c
        wT = w(np.array([Tf]))[0]
        dwT = dw(np.array([Tf]))[0]
        dw0 = dw(np.array([0.0]))[0]
        rhs_b = _weighted_norm2(w, N, Tf) / (2 * Tf) + wT ** 2 / (2 * np.e)
        rhs_a = _weighted_norm2(dw, N, Tf) / (2 * Tf) + dwT ** 2 / (2 * np.e) + 0.5 * dw0 ** 2
        assert c @ B @ c == pytest.approx(rhs_b, rel=1e-12)
        assert c @ A @ c == pytest.approx(rhs_a, rel=1e-12)


@pytest.mark.parametrize("jt", [1, 3, 6])
def test_symmetric_parts_positive_definite(jt):
    """Proof of Prop. 1: A and B have positive definite symmetric parts."""
    A, B = timemats.time_matrices(jt, T)
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


@pytest.mark.parametrize("jt", [1, 2, 4])
@pytest.mark.parametrize("mu", [0.0, 3.7, 250.0])
def test_ode_solutions_in_the_space_are_reproduced(jt, mu):
    """The time scheme for one spatial eigenmode, (A + mu B) c = b with
    b[i] = (f, psi_i')_e + v0 psi_i'(0), is the Galerkin method of Eq. (10)
    for q'' + mu q = f, q(0) = 0, q'(0) = v0.  When q lies in V_jt (q = t, t^2)
    its coefficients must be returned exactly.  This fixes the orientation of
    A and B (test index first) and the penalty term."""
    N = 1 << jt
    A, B = timemats.time_matrices(jt, T)
    kv = timebasis.knots(N, T)
    greville = 0.5 * (kv[1:N + 3] + kv[2:N + 4])[1:]        # coefficients of t (B_0 has weight 0)
    blossom = (kv[1:N + 3] * kv[2:N + 4])[1:]                # coefficients of t^2
    d0 = timemats.dpsi_at_zero(jt, T)
    # q = t: f = mu t, v0 = 1
    b = timemats.load_separable(lambda t: mu * t, jt, T) + d0
    assert np.allclose(np.linalg.solve(A + mu * B, b), greville, atol=1e-11)
    # q = t^2: f = 2 + mu t^2, v0 = 0
    b = timemats.load_separable(lambda t: 2 + mu * t * t, jt, T)
    assert np.allclose(np.linalg.solve(A + mu * B, b), blossom, atol=1e-11)
