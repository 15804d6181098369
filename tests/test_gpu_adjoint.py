"""GPU tests of the receiver misfit and its adjoint gradient (st_misfit_gradient).

Parity with the oracle's adjoint (oracle/adjoint.py, itself pinned by finite
differences) on small problems, central finite differences of the GPU's own
J along 20 seeded directions on the differentiation configuration (d = 2,
n = 10, m = 2, 65 x 65 nodal c^2 and g, 32 receivers on y = 0.9), the
FP32 + refinement path against the FP64 path, and the autograd wrapper.
"""
import dataclasses

import numpy as np
import pytest

import st_workloads as W
from oracle import adjoint as OA
from oracle import solve as osolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09688_gb300 import build
    build.build(force=False)


def _oracle_obs(st):
    p = OA.with_parameters(st.base, st.c2_obs_nodal, st.g_nodal, st.s, st.jp)
    comps, sols = osolve.solve_all(p, method="schur")
    t, _ = OA.target_times(p, st.jt_star)
    return osolve.combine(p, comps, sols, st.receivers, t)


@pytest.mark.parametrize("n,m,jp,nrec", [(4, 1, 2, 5), (6, 1, 3, 8), (7, 2, 4, 12)])
def test_misfit_and_gradient_match_the_oracle(n, m, jp, nrec):
    import torch
    from paper_2606_09688_gb300 import ST_FP64
    from paper_2606_09688_gb300.adjoint import nodal_solver
    st = W.inverse_2d(n=n, m=m, jp=jp, n_receivers=nrec, seed=n)
    d_obs = _oracle_obs(st)
    J0, gc0, gg0 = OA.gradient(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp, st.receivers, st.jt_star, d_obs)
    with nodal_solver(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp, ST_FP64) as s:
        s.solve(-1)
        vals = s.receiver_values(st.jt_star, st.receivers).cpu().numpy()
        J, gc, gg, info = s.misfit_gradient(st.jt_star, st.receivers, torch.from_numpy(d_obs).cuda(), st.jp)
    pa = OA.with_parameters(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp)
    comps, sols = osolve.solve_all(pa, method="schur")
    t, _ = OA.target_times(pa, st.jt_star)
    ref_vals = osolve.combine(pa, comps, sols, st.receivers, t)
    assert np.max(np.abs(vals - ref_vals)) <= 1e-10 * np.max(np.abs(ref_vals))
    assert abs(J - J0) <= 1e-9 * J0
    gc, gg = gc.cpu().numpy(), gg.cpu().numpy()
    assert np.linalg.norm(gc - gc0) <= 1e-8 * np.linalg.norm(gc0), np.linalg.norm(gc - gc0) / np.linalg.norm(gc0)
    assert np.linalg.norm(gg - gg0) <= 1e-8 * np.linalg.norm(gg0), np.linalg.norm(gg - gg0) / np.linalg.norm(gg0)
    assert info.status == 0


def _diff_setup():
    import torch
    from paper_2606_09688_gb300.adjoint import observations
    st = W.inverse_2d()                                  # n = 10, m = 2, 65 x 65 nodal fields, 32 receivers
    d_obs = observations(st.base, st.c2_obs_nodal, st.g_nodal, st.s, st.jp, st.receivers, st.jt_star)
    return st, d_obs


def test_gradient_matches_central_differences_on_20_directions():
    from paper_2606_09688_gb300 import ST_FP64
    from paper_2606_09688_gb300.adjoint import nodal_solver
    st, d_obs = _diff_setup()

    def J_and_grad(c2, g, grad=False):
        with nodal_solver(st.base, c2, g, st.s, st.jp, ST_FP64) as s:
            s.solve(-1)
            J, gc, gg, _ = s.misfit_gradient(st.jt_star, st.receivers, d_obs, st.jp)
        return (J, gc.cpu().numpy(), gg.cpu().numpy()) if grad else J

    J, gc, gg = J_and_grad(st.c2_nodal, st.g_nodal, grad=True)
    assert J > 0
    rng = np.random.default_rng(2024)
    worst = 0.0
    for k in range(20):
        vc = rng.standard_normal(len(gc))
        vg = rng.standard_normal(len(gg))
        vc /= np.max(np.abs(vc))
        vg /= np.max(np.abs(vg))
        h = 1e-4
        Jp = J_and_grad(st.c2_nodal + h * vc, st.g_nodal + h * vg)
        Jm = J_and_grad(st.c2_nodal - h * vc, st.g_nodal - h * vg)
        fd = (Jp - Jm) / (2 * h)
        an = float(vc @ gc + vg @ gg)
        rel = abs(fd - an) / max(abs(an), 1e-12)
        worst = max(worst, rel)
        assert rel <= 1e-5, (k, fd, an, rel)
    print("central differences: worst relative deviation %.2e over 20 directions" % worst)


def test_fp32_refinement_gradient_matches_fp64():
    from paper_2606_09688_gb300 import ST_FP32_IR, ST_FP64
    from paper_2606_09688_gb300.adjoint import nodal_solver
    st, d_obs = _diff_setup()
    out = {}
    for prec in (ST_FP64, ST_FP32_IR):
        with nodal_solver(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp, prec) as s:
            s.solve(-1)
            out[prec] = s.misfit_gradient(st.jt_star, st.receivers, d_obs, st.jp)
    J64, gc64, gg64, _ = out[ST_FP64]
    J32, gc32, gg32, _ = out[ST_FP32_IR]
    assert abs(J32 - J64) <= 1e-8 * J64
    assert float((gc32 - gc64).norm() / gc64.norm()) <= 1e-8
    assert float((gg32 - gg64).norm() / gg64.norm()) <= 1e-8


def test_autograd_function_returns_the_adjoint_gradient():
    import torch
    from paper_2606_09688_gb300.adjoint import receiver_misfit
    st = W.inverse_2d(n=6, m=1, jp=3, n_receivers=8, seed=1)
    d_obs = torch.from_numpy(_oracle_obs(st)).cuda()
    c2 = torch.tensor(st.c2_nodal, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(st.g_nodal, dtype=torch.float64, requires_grad=True)
    J = receiver_misfit(c2, g, st.base, st.s, st.jp, st.receivers, st.jt_star, d_obs)
    Jv = float(J.detach())
    (3.0 * J).backward()
    J0, gc0, gg0 = OA.gradient(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp, st.receivers, st.jt_star,
                               d_obs.cpu().numpy())
    assert abs(Jv - J0) <= 1e-9 * J0
    assert np.linalg.norm(c2.grad.numpy() - 3.0 * gc0) <= 1e-8 * np.linalg.norm(3.0 * gc0)
    assert np.linalg.norm(g.grad.numpy() - 3.0 * gg0) <= 1e-8 * np.linalg.norm(3.0 * gg0)


def test_misfit_gradient_argument_errors():
    import torch
    from paper_2606_09688_gb300 import Solver, StError
    from paper_2606_09688_gb300 import st as B
    st = W.inverse_2d(n=4, m=1, jp=2, n_receivers=3)
    from paper_2606_09688_gb300.adjoint import nodal_solver, problem_with
    d = torch.zeros(((1 << st.jt_star) + 1, 3), dtype=torch.float64, device="cuda")
    with nodal_solver(st.base, st.c2_nodal, st.g_nodal, st.s, st.jp) as s:
        with pytest.raises(StError) as e:
            s.misfit_gradient(st.jt_star, st.receivers, d, st.jp)
        assert e.value.code == B.ST_ERR_STATE                 # not solved yet
        s.solve(-1)
        with pytest.raises(StError) as e:
            s.misfit_gradient(st.jt_star, st.receivers + 2.0, d, st.jp)
        assert e.value.code == B.ST_ERR_ARG                   # receivers outside the box
        with pytest.raises(StError) as e:
            s.misfit_gradient(st.jt_star, st.receivers, d, st.jp + 1)
        assert e.value.code == B.ST_ERR_ARG                   # another parameter level than the problem's
    # c^2 from a callback: the gradient with respect to nodal values is refused
    with Solver(dataclasses.replace(problem_with(st.base, st.s), c2=st.base.c2, terms=st.base.terms or
                                    [(lambda x: np.ones(len(x)), st.s)])) as s:
        s.solve(-1)
        with pytest.raises(StError) as e:
            s.misfit_gradient(st.jt_star, st.receivers, d, st.jp)
        assert e.value.code == B.ST_ERR_STATE
    q = W.standing_wave(2, 4, 1)                              # u0 != 0
    with Solver(q) as s:
        s.solve(-1)
        d2 = torch.zeros(((1 << 3) + 1, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(StError) as e:
            s.misfit_gradient(3, st.receivers, d2, 2)
        assert e.value.code == B.ST_ERR_ARG
