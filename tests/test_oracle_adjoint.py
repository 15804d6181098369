"""Pins of the oracle's receiver-misfit gradient (adjoint of Eq. (9)).

The adjoint state solves the transposed space-time system; the gradient
formulas follow from differentiating S_k U_k = F_k (Eq. (30)).  Pinned by the
transposition identity <S^-T G, F> = <G, S^-1 F> and by central finite
differences of J itself (forward solves only) along seeded directions.
"""
import numpy as np

import st_workloads as W
from oracle import adjoint as A
from oracle import solve as S


def _tiny(seed=3):
    st = W.inverse_2d(n=4, m=1, jp=2, n_receivers=5, seed=seed)
    p_obs = A.with_parameters(st.base, st.c2_obs_nodal, st.g_nodal, st.s, st.jp)
    comps, sols = S.solve_all(p_obs)
    t, _ = A.target_times(p_obs, st.jt_star)
    d_obs = S.combine(p_obs, comps, sols, st.receivers, t)
    return st, d_obs


def test_adjoint_state_solves_the_transposed_system():
    st, _ = _tiny()
    p = A.with_parameters(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp)
    rng = np.random.default_rng(0)
    for jx, jt in ((2, 2), (3, 1), (1, 3)):
        Sm = S.system_matrix(p, jx, jt)
        n = Sm.shape[0]
        nt = (1 << jt) + 1
        G = rng.standard_normal((nt, n // nt))
        F = rng.standard_normal((nt, n // nt))
        L = A.adjoint_state(p, jx, jt, G)
        U = S.solve_component(p, jx, jt, F=F)
        assert abs(np.sum(L * F) - np.sum(G * U)) <= 1e-10 * np.sqrt(np.sum(L * L) * np.sum(F * F))
        # and S^T L = G directly
        assert np.linalg.norm(Sm.T @ L.ravel() - G.ravel()) <= 1e-10 * np.linalg.norm(G)


def test_gradient_matches_central_differences():
    st, d_obs = _tiny()
    J, gc, gg = A.gradient(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp, st.receivers, st.jt_star, d_obs)
    assert J > 0
    rng = np.random.default_rng(11)
    for _ in range(4):
        for which in ("c2", "g"):
            v = rng.standard_normal(len(st.c2_nodal))
            h = 1e-4 if which == "c2" else 1e-3
            def J_at(eps):
                c2 = st.c2_nodal + (eps * v if which == "c2" else 0.0)
                g = st.g_nodal + (eps * v if which == "g" else 0.0)
                return A.objective_at(st.base, c2, g, st.s, st.jp, st.receivers, st.jt_star, d_obs)
            fd = (J_at(h) - J_at(-h)) / (2 * h)
            an = float(v @ (gc if which == "c2" else gg))
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * J), (which, fd, an)


def test_gradient_vanishes_at_the_data_parameters():
    """With observations made by the same parameters, J = 0 and so is its gradient."""
    st, _ = _tiny()
    p = A.with_parameters(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp)
    comps, sols = S.solve_all(p)
    t, _ = A.target_times(p, st.jt_star)
    d_same = S.combine(p, comps, sols, st.receivers, t)
    J, gc, gg = A.gradient(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp, st.receivers, st.jt_star, d_same)
    assert J < 1e-25
    assert np.max(np.abs(gc)) < 1e-12 and np.max(np.abs(gg)) < 1e-12
