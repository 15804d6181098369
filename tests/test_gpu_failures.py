"""Failure detection on the GPU, in forms that fault, trap or hang nothing.

* Iteration limits: an inner Krylov limit of one iteration, and a refinement
  limit of one sweep with a backward-error target one FP32 sweep cannot reach,
  give ST_ERR_NOT_CONVERGED.
* Device memory: a per-handle allocation cap below what st_setup needs gives
  ST_ERR_OOM (the allocation fails on the host side, as a real one would).
* Bounded waits: with the test-only option that withholds the first
  factor-row copy of the single-warp banded solve, its copy wait (shortened to
  200,000 cycles) runs out, the kernel records the fact, lets its other copy
  land and returns; the solve reports ST_ERR_TIMEOUT.  Nothing is left in
  flight, and the context stays usable: the same problem solved afterwards
  matches the oracle.
* Bad data: c^2 that is NaN somewhere is refused at set-up (ST_ERR_ARG); a
  source whose values are NaN makes the COCG status words report a non-finite
  value, and the solve returns ST_ERR_NUMERIC (host-driven loop and graph
  solves alike), after which a clean handle solves normally.
"""
import numpy as np
import pytest

import st_workloads as W
from oracle import solve as osolve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09688_gb300 import build
    build.build(force=False)


def _component(s, jx, jt):
    return next(k for k, ci in enumerate(s.components()) if (ci.jx, ci.jt) == (jx, jt))


@pytest.mark.parametrize("device_loop", [0, 4])
def test_inner_iteration_limit_reports_not_converged(device_loop):
    from paper_2606_09688_gb300 import Solver, StError
    from paper_2606_09688_gb300 import st as B
    # grids above 500 unknowns go through multigrid-preconditioned COCG; with graph
    # solves the modes' status words are read by the device-side stopping test
    with Solver(W.layered_2d(8, 2), max_direct_rows=500, max_iter=1, device_loop=device_loop) as s:
        with pytest.raises(StError) as e:
            s.solve(_component(s, 6, 2))
        assert e.value.code == B.ST_ERR_NOT_CONVERGED
        assert "iteration limit" in str(e.value)


@pytest.mark.parametrize("device_loop", [0, 4])
def test_refinement_sweep_limit_reports_not_converged(device_loop):
    from paper_2606_09688_gb300 import ST_FP32_IR, Solver, StError
    from paper_2606_09688_gb300 import st as B
    # with graph solves the sweep limit is applied by the device-side stopping test
    with Solver(W.layered_2d(8, 2), precision=ST_FP32_IR, max_sweeps=1, tol=1e-15,
                device_loop=device_loop) as s:
        with pytest.raises(StError) as e:
            s.solve(_component(s, 6, 2))
        assert e.value.code == B.ST_ERR_NOT_CONVERGED


def test_allocation_cap_reports_oom_and_a_sufficient_cap_solves():
    from paper_2606_09688_gb300 import Solver, StError
    from paper_2606_09688_gb300 import st as B
    p = W.layered_2d(8, 2)
    with pytest.raises(StError) as e:
        Solver(p, mem_cap_bytes=1 << 20)
    assert e.value.code == B.ST_ERR_OOM
    with Solver(p, mem_cap_bytes=8 << 30) as s:
        assert s.solve(-1).status == 0


@pytest.mark.parametrize("device_loop", [0, 4])
def test_bounded_copy_wait_runs_out_and_context_stays_usable(device_loop):
    from paper_2606_09688_gb300 import Solver, StError
    from paper_2606_09688_gb300 import st as B
    p = W.standing_wave(3, 6, 2)          # (4,2): 15^3 grid, half bandwidth 241, solved directly
    # with graph solves the timeout flag is read by the device-side stopping test
    with Solver(p, wait_cycles=200000, inject_stall=1, device_loop=device_loop) as s:
        k = _component(s, 4, 2)
        with pytest.raises(StError) as e:
            s.solve(k)
        assert e.value.code == B.ST_ERR_TIMEOUT
        # a component on another kernel (the blocked solve, bands up to 128) is unaffected
        assert s.solve(_component(s, 3, 3)).status == 0
    with Solver(p) as s:
        s.solve(-1)
        out = s.combine(4, 4).cpu().numpy()
    comps, sols = osolve.solve_all(p, method="schur")
    pts, times = osolve.target_grid(p, 4, 4)
    ref = osolve.combine(p, comps, sols, pts, times)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-10


def test_nan_speed_is_refused_at_setup():
    from paper_2606_09688_gb300 import Solver, StError
    from paper_2606_09688_gb300 import st as B
    p = W.layered_2d(6, 2)
    bad = W.Problem(**{**p.__dict__, "c2": lambda x: np.where(x[:, 0] > 0.7, np.nan, 1.0)})
    with pytest.raises(StError) as e:
        Solver(bad)
    assert e.value.code == B.ST_ERR_ARG


@pytest.mark.parametrize("device_loop", [0, 4])
def test_nan_source_reports_numeric_error_and_context_stays_usable(device_loop):
    from paper_2606_09688_gb300 import Solver, StError
    from paper_2606_09688_gb300 import st as B
    p = W.layered_2d(8, 2)
    g, s_t = p.terms[0]
    bad = W.Problem(**{**p.__dict__, "terms": [(lambda x: g(x) * np.nan, s_t)]})
    with Solver(bad, max_direct_rows=500, device_loop=device_loop) as s:
        with pytest.raises(StError) as e:
            s.solve(_component(s, 6, 2))           # a multigrid component
        assert e.value.code == B.ST_ERR_NUMERIC
    with Solver(p, max_direct_rows=500, device_loop=device_loop) as s:
        assert s.solve(_component(s, 6, 2)).status == 0
