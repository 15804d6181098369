"""GPU parity at the configurations' full sizes and on a general box.

* 3D random medium with the configuration's coarsest level m = 3 (Eq. (19)
  components (3+a, 3+J-a)): element-wise oracle parity of the combined target
  at n = 7; at n = 8 sampled target values against values the oracle wrote
  once (tests/golden/make_fullsize_samples.py); at n = 9 and 10 (largest
  component (7,3): 127^3 x 9) the normwise backward error of every component
  under the oracle's own definition of S and F, including (3,7) whose 129 time
  unknowns sit at the time/space-eigenbasis switch, plus sampled target values
  against the oracle's evaluation of Eq. (19) from the GPU's component arrays.
* A 2D problem on a non-square, non-unit box with T != 1 and non-zero u0, v0
  and source: element-wise parity in both precisions.

Tolerances: 1e-10 (FP64 path) and 1e-8 (FP32 + FP64 refinement) relative l2
for forward comparisons.  Backward errors are taken in the 1-norm with the
exact ||S||_1; the solver's own stopping rule uses the 2-norm with an upper
bound of ||S||_2, so the test sets the solver's target explicitly (tol) and
allows a factor 10 between the two norms' figures.
"""
import os
import sys

import numpy as np
import pytest

import st_workloads as W
from oracle import solve as osolve

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_fullsize_samples as golden  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-8
BE_TOL = 1e-13          # solver target backward error passed explicitly


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09688_gb300 import build
    build.build(force=False)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _elementwise(p, prec, target):
    from paper_2606_09688_gb300 import Solver
    with Solver(p, precision=prec) as s:
        info = s.solve(-1)
        out = s.combine(*target).cpu().numpy()
        coeffs = [s.coeffs(k) for k in range(s.num_components)]
        infos = s.components()
    comps, sols = osolve.solve_all(p, method="schur")
    assert [(c.jx, c.jt, c.coef) for c in infos] == comps
    pts, times = osolve.target_grid(p, *target)
    ref = osolve.combine(p, comps, sols, pts, times)
    tol = TOL64 if prec == 0 else TOL32
    assert info.status == 0
    assert _rel(out, ref) < tol, (p.name, _rel(out, ref))
    for (jx, jt, _), U, Uo in zip(comps, coeffs, sols):
        assert _rel(U, Uo) < 10 * tol, ((jx, jt), _rel(U, Uo))


@pytest.mark.parametrize("prec", [0, 1])
def test_anisotropic_box_final_time_1p7(prec):
    """Box (-0.5,1.5) x (0,0.75), T = 1.7, variable c^2, u0, v0 and f non-zero,
    n = 8, m = 2: the (6,2) and (5,2) grids go through multigrid-preconditioned COCG
    with unequal mesh widths; the others are direct."""
    _elementwise(W.anisotropic_2d(8, 2), prec, (6, 6))


@pytest.mark.parametrize("prec", [0, 1])
def test_random_medium_3d_n7_m3_elementwise(prec):
    """3D random medium, coarsest level 3 as in the configuration, n = 7 (the
    (4,3) component is the 15^3 grid, half bandwidth 241, solved directly)."""
    _elementwise(W.random_medium_3d(7, 3), prec, (4, 4))


@pytest.mark.parametrize("name,prec", [("random_medium_3d_n8_m3", 0), ("random_medium_3d_n8_m3", 1)])
def test_random_medium_3d_m3_sampled_against_oracle_fixture(name, prec):
    """n = 8 (target (5,5); the (5,3) component is the 31^3 grid solved directly):
    64 x 16 sampled target values against the oracle's Schur-route solution of every
    component, written once by tests/golden/make_fullsize_samples.py (a sparse LU of
    the 31^3 complex system takes the oracle about half a minute per time mode)."""
    import torch
    from paper_2606_09688_gb300 import Solver
    factory, target = golden.FIXTURES[name][0], golden.FIXTURES[name][1]
    pi, si, ref = golden.read(name)
    with Solver(factory(), precision=prec) as s:
        out, info = s.solve_combine(*target)
        got = out[torch.as_tensor(si, device=out.device)][:, torch.as_tensor(pi, device=out.device)].cpu().numpy()
    assert info.status == 0
    tol = TOL64 if prec == 0 else TOL32
    assert _rel(got, ref) < tol, _rel(got, ref)


@pytest.mark.parametrize("n", [9, 10])
def test_random_medium_3d_m3_every_component_backward_error(n):
    """The 3D configuration at full size (n = 10, m = 3, 9 components, 26.8 M
    space-time DOFs, largest (7,3) = 127^3 x 9) and at n = 9 (largest (6,3) =
    63^3 x 9, whose direct solve by the oracle's sparse LU would take about an
    hour per time mode), FP32 bulk + FP64 refinement, through st_solve_combine
    with target (n-3, n-3): (a) every component's normwise backward error under
    the oracle's S and F; (b) 32 x 8 sampled target values against the oracle's
    evaluation of Eq. (19) from the GPU's component arrays."""
    import torch
    from paper_2606_09688_gb300 import ST_FP32_IR, Solver
    from oracle import space
    p = W.random_medium_3d(n, 3)
    target = (n - 3, n - 3)
    rng = np.random.default_rng(n)
    pts, times = osolve.target_grid(p, *target)
    pi = np.sort(rng.choice(len(pts), 32, replace=False))
    si = np.sort(rng.choice(len(times), 8, replace=False))
    with Solver(p, precision=ST_FP32_IR, tol=BE_TOL) as s:
        out, info = s.solve_combine(*target)
        got = out[torch.as_tensor(si, device=out.device)][:, torch.as_tensor(pi, device=out.device)].cpu().numpy()
        del out
        infos = s.components()
        coeffs = [s.coeffs(k) for k in range(len(infos))]
    assert info.status == 0
    assert n != 10 or (3, 7) in [(ci.jx, ci.jt) for ci in infos]
    ref = sum(ci.coef * osolve.evaluate_component(p, ci.jx, ci.jt, U, pts[pi], times[si])
              for ci, U in zip(infos, coeffs))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    worst = {}
    for ci, U in zip(infos, coeffs):
        sm = space.space_matrices(p, ci.jx)
        worst[(ci.jx, ci.jt)] = osolve.backward_error(p, ci.jx, ci.jt, U, sm=sm)
        del sm
    assert max(worst.values()) < 10 * BE_TOL, worst
