"""Pins for the oracle's component solve and combination (CPU only)."""
import os

import numpy as np
import pytest

import st_workloads as W
from oracle import combination, solve, space

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_component_set_matches_worked_example():
    """Section 6.1 figure of meshes: Omega_T = (-1,1) x (0,1), h0 = 1/2, J = 3."""
    rows = np.loadtxt(os.path.join(GOLDEN, "meshes_ex1_J3.txt"), dtype=int)
    p = W.e1_vanishing(3)
    comps = combination.components(p.J, p.mx, p.mt)
    got = sorted(((1 << jx), (1 << jt), c) for jx, jt, c in comps)
    want = sorted(tuple(r) for r in rows if r[2] != 0)
    assert got == want
    full = [tuple(r) for r in rows if r[2] == 0][0]
    assert (1 << (p.mx + p.J), 1 << (p.mt + p.J)) == full[:2]


@pytest.mark.parametrize("J", [0, 1, 4, 9])
def test_coefficients_sum_to_one_and_count(J):
    comps = combination.components(J, 2, 3)
    assert len(comps) == 2 * J + 1                   # 2J+1 solves (Section 3.1)
    assert sum(c for _, _, c in comps) == 1


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("J", [1, 3, 6])
def test_dof_count_closed_forms(d, J):
    """Section 3.2: with dim ~ 2^{d jx} 2^{jt}, the sum over the component set equals
    2^J (J + 1 + J/2) for d = 1 and
    (1 - 2^{(d-1)(J+1)}) / (1 - 2^{d-1}) (2^J + 2^{J-d}) - 2^{J-d} for d = 2, 3."""
    comps = combination.components(J, 0, 0)
    approx = sum(2.0 ** (d * jx + jt) for jx, jt, _ in comps)
    if d == 1:
        closed = 2.0 ** J * (J + 1 + J / 2)
    else:
        closed = (1 - 2.0 ** ((d - 1) * (J + 1))) / (1 - 2.0 ** (d - 1)) * (2.0 ** J + 2.0 ** (J - d)) - 2.0 ** (J - d)
    assert approx == pytest.approx(closed, rel=1e-14)


def test_dof_counts_of_workloads():
    """Exact N^sparse_DoFs: 1D formula (N_jx (p-r) + r - 1)(N_jt (p-r) + r) with
    p_x = 1, r_x = 0, p_t = 2, r_t = 1 and its d-dimensional Q1 analogue."""
    assert combination.sparse_dofs(1, 4, 1, 1) == 439
    assert combination.sparse_dofs(2, 8, 2, 2) == 12_099_257
    assert combination.sparse_dofs(3, 4, 3, 3) == 26_823_511
    for jx, jt in [(3, 2), (5, 1)]:
        assert combination.space_dofs(1, jx) * combination.time_dofs(jt) == \
            ((1 << jx) * 1 + 0 - 1) * ((1 << jt) * 1 + 1)


@pytest.mark.parametrize("d,jx,jt", [(1, 3, 3), (2, 2, 2), (2, 3, 1)])
def test_galerkin_reproduces_discrete_solution(d, jx, jt):
    """Eq. (10): P reproduces discrete functions, so F := S U* gives back U*.
    Dense numpy solve as an independent check of the sparse solvers."""
    p = W.standing_wave(d, 2 * max(jx, jt), max(jx, jt))
    S = solve.system_matrix(p, jx, jt)
    nt = (1 << jt) + 1
    Ustar = np.random.default_rng(0).standard_normal((nt, S.shape[0] // nt))
    F = (S @ Ustar.ravel()).reshape(Ustar.shape)
    for method in ("lu", "schur"):
        assert np.allclose(solve.solve_component(p, jx, jt, F=F, method=method), Ustar, atol=1e-10)
    assert np.allclose(np.linalg.solve(S.toarray(), F.ravel()).reshape(Ustar.shape), Ustar, atol=1e-10)


def test_level_zero_combination_is_the_full_grid_solution():
    """J = 0: Eq. (19) has a single term, u^CF = P_{m,m} u."""
    p = W.standing_wave(1, 6, 3)
    comps, sols = solve.solve_all(p)
    assert comps == [(3, 3, 1)]
    pts, times = solve.target_grid(p, 4, 4)
    direct = solve.evaluate_component(p, 3, 3, solve.solve_component(p, 3, 3), pts, times)
    assert np.array_equal(solve.combine(p, comps, sols, pts, times), direct)


def test_detail_identity_eq21():
    """Eq. (21): u^CF_J = sum_{jx + jt <= J} Delta^P_{jx,jt} u, Delta^P from Eq. (20),
    and Eq. (21bis) for P_{J,J} u, checked by brute force on target values (J = 2)."""
    p = W.e2_variable_speed(2)
    J = p.J
    pts, times = solve.target_grid(p, p.mx + J, p.mt + J)
    P = {}
    for a in range(-1, J + 1):
        for b in range(-1, J + 1):
            if a < 0 or b < 0:
                P[a, b] = 0.0
            else:
                U = solve.solve_component(p, p.mx + a, p.mt + b)
                P[a, b] = solve.evaluate_component(p, p.mx + a, p.mt + b, U, pts, times)
    delta = lambda a, b: (P[a, b] - P[a - 1, b]) - (P[a, b - 1] - P[a - 1, b - 1])
    comps, sols = solve.solve_all(p)
    ucf = solve.combine(p, comps, sols, pts, times)
    s21 = sum(delta(a, b) for a in range(J + 1) for b in range(J + 1) if a + b <= J)
    assert np.allclose(ucf, s21, atol=1e-12)
    full = sum(delta(a, b) for a in range(J + 1) for b in range(J + 1))
    assert np.allclose(full, P[J, J], atol=1e-12)


def test_initial_value_is_the_interpolant():
    """psi_i(0) = 0 for every basis function, so u_k(x, 0) = I_jx u0 and
    u^CF(., 0) = sum_k c_k I_{jx,k} u0; at the nodes of the coarsest spatial grid all
    interpolants agree with u0 and the coefficients sum to 1."""
    p = W.standing_wave(2, 6, 2)
    comps, sols = solve.solve_all(p)
    pts = space.node_coords(2, p.lo, p.hi, p.mx)
    v = solve.combine(p, comps, sols, pts, np.array([0.0]))[0]
    assert np.allclose(v, p.u0(pts), atol=1e-14)


def _slopes(errs):
    e = np.asarray(errs)
    return np.log2(e[:-1] / e[1:])


def test_convergence_rate_standing_wave_1d():
    """Eq. (18) and Theorem 1 with p_x = 1, p_t = 2: O(h^2) for FG and SG (no log factor)."""
    fg, sg = [], []
    for n in (4, 5, 6, 7):
        p = W.standing_wave(1, n, 1)
        comps, sols = solve.solve_all(p)
        jf = p.mx + p.J
        sg.append(solve.l2_error_qt(p, comps, sols, jf, jf))
        fg.append(solve.l2_error_qt(p, [(jf, jf, 1)], [solve.solve_component(p, jf, jf)], jf, jf))
    assert np.all(np.abs(_slopes(fg) - 2) < 0.15), fg
    assert np.all(np.abs(_slopes(sg) - 2) < 0.15), sg


def test_convergence_rate_vanishing_example_e1():
    """Section 6.1 exact solution (vanishing conditions hold): SG rate 2 with Q1 x S^2_1."""
    errs = []
    for J in (2, 3, 4, 5):
        p = W.e1_vanishing(J)
        comps, sols = solve.solve_all(p)
        errs.append(solve.l2_error_qt(p, comps, sols, p.mx + J, p.mt + J))
    assert np.all(np.abs(_slopes(errs) - 2) < 0.15), errs


def test_convergence_rate_variable_speed_e2():
    """Section 6.2 (c^2 = 1 + x, u0, v0 != 0, non-separable f): SG rate 2."""
    errs = []
    for J in (2, 3, 4, 5):
        p = W.e2_variable_speed(J)
        comps, sols = solve.solve_all(p)
        errs.append(solve.l2_error_qt(p, comps, sols, p.mx + J, p.mt + J))
    assert np.all(np.abs(_slopes(errs) - 2) < 0.15), errs


def test_convergence_rate_standing_wave_2d():
    errs = []
    for n in (4, 5, 6):
        p = W.standing_wave(2, n, 1)
        comps, sols = solve.solve_all(p)
        jf = p.mx + p.J
        errs.append(solve.l2_error_qt(p, comps, sols, jf, jf, npts=2, ntpts=3))
    assert np.all(np.abs(_slopes(errs) - 2) < 0.3), errs
