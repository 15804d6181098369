"""GPU energy of the combined solution (st_energy, Section 6.3) against the oracle.

E(t; u^CF) = 1/2 (||d_t u^CF||^2 + ||c grad u^CF||^2) on the travelling wave of
Section 6.3 (c = 4/5 on (-1, 1)) at 800 equispaced instants of [0, T], as in
the paper's figure, and on the 2D layered medium (cellwise c^2 in {1, 4}).
Tolerances as for the combined solution: 1e-10 relative (FP64 path), 1e-8
(FP32 + FP64 refinement).  The relative energy error against the exact
solution's (constant) energy stays bounded over [0, T] and decreases with J.
"""
import numpy as np
import pytest

import st_workloads as W
from oracle import energy, solve as osolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09688_gb300 import build
    build.build(force=False)


def _gpu_energy(p, prec, times):
    from paper_2606_09688_gb300 import Solver
    with Solver(p, precision=prec) as s:
        s.solve(-1)
        return s.energy(times)


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_travelling_wave_800_instants(prec):
    p = W.travelling_wave(5)
    times = np.linspace(0.0, 1.0, 800)
    got = _gpu_energy(p, prec, times)
    comps, sols = osolve.solve_all(p)
    jq = max(jx for jx, _, _ in comps)
    ref = energy.energy_cf(p, comps, sols, jq, times)
    tol = 1e-10 if prec == 0 else 1e-8
    assert np.max(np.abs(got - ref)) <= tol * np.max(ref)
    e_exact = energy.energy_of(p, p.exact_dt, p.exact_grad, jq + 2, times[:1])[0]
    err = np.abs(got - e_exact) / e_exact
    assert np.max(err) < 0.05


def test_energy_error_decreases_with_the_level():
    times = np.linspace(0.0, 1.0, 200)
    worst = []
    for J in (3, 4, 5, 6):
        p = W.travelling_wave(J)
        got = _gpu_energy(p, 0, times)
        jq = p.mx + p.J
        e_exact = energy.energy_of(p, p.exact_dt, p.exact_grad, jq + 2, times[:1])[0]
        worst.append(np.max(np.abs(got - e_exact)) / e_exact)
    assert all(b < a for a, b in zip(worst, worst[1:])), worst


def test_energy_layered_medium_2d():
    p = W.layered_2d(8, 2)
    times = np.linspace(0.0, 1.0, 21)
    got = _gpu_energy(p, 0, times)
    comps, sols = osolve.solve_all(p, method="schur")
    jq = max(jx for jx, _, _ in comps)
    ref = energy.energy_cf(p, comps, sols, jq, times)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(ref)


def test_energy_argument_errors():
    from paper_2606_09688_gb300 import Solver, StError
    from paper_2606_09688_gb300 import st as B
    p = W.travelling_wave(3)
    with Solver(p) as s:
        with pytest.raises(StError) as e:
            s.energy([0.5])
        assert e.value.code == B.ST_ERR_STATE
        s.solve(-1)
        with pytest.raises(StError) as e:
            s.energy([1.5])
        assert e.value.code == B.ST_ERR_ARG
        with pytest.raises(StError) as e:
            s.energy([0.5], jx_eval=2)
        assert e.value.code == B.ST_ERR_ARG


def test_coarsest_mesh_study_of_section_6_3():
    """Section 6.3, h0 study: three sequences with coarsest meshes h0 = 2^-1, 2^-2, 2^-3 and
    the same finest meshes.  For the travelling wave, the relative L^2(Q_T) error of the
    GPU's combined solution (the oracle's quadrature applied to the GPU's component
    arrays) decreases at every finest mesh as h0 is refined, and with h0 = 2^-3 it
    converges at the O(h^2) rate of Theorem 1 (error ratio near 4 per level)."""
    from paper_2606_09688_gb300 import ST_FP64, Solver
    errs = {}
    for h0 in (1, 2, 3):
        for finest in (4, 5, 6):
            J = finest - h0
            p = W.travelling_wave(J, h0_level=h0)
            with Solver(p, precision=ST_FP64) as s:
                s.solve(-1)
                infos = s.components()
                sols = [s.coeffs(k) for k in range(len(infos))]
            comps = [(ci.jx, ci.jt, ci.coef) for ci in infos]
            errs[(h0, finest)] = osolve.l2_error_qt(p, comps, sols, p.mx + p.J, p.mt + p.J)
    for finest in (4, 5, 6):
        assert errs[(3, finest)] < errs[(2, finest)] < errs[(1, finest)], errs
    assert 3.0 < errs[(3, 5)] / errs[(3, 6)] < 5.0, errs
