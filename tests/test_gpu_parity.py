"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: the plain FP64 path must match the oracle's combined solution to
1e-10 relative l2 on the target grid; the FP32 + FP64-refinement path to 1e-8.
Component coefficient arrays are compared too (same scale).
"""
import numpy as np
import pytest

import st_workloads as W
from oracle import solve as osolve

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09688_gb300 import build
    build.build(force=False)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _run(p, precision, target, method="lu", check_components=True, tol=None):
    from paper_2606_09688_gb300 import Solver
    jxs, jts = target
    with Solver(p, precision=precision) as s:
        info = s.solve(-1)
        out = s.combine(jxs, jts).cpu().numpy()
        coeffs = [s.coeffs(k) for k in range(s.num_components)] if check_components else None
        comps_info = s.components()
    comps, sols = osolve.solve_all(p, method=method)
    assert [(c.jx, c.jt, c.coef) for c in comps_info] == comps
    pts, times = osolve.target_grid(p, jxs, jts)
    ref = osolve.combine(p, comps, sols, pts, times)
    tol = tol or (TOL64 if precision == 0 else TOL32)
    err = _rel(out, ref)
    assert err < tol, (p.name, err, info.rel_residual)
    if check_components:
        for (jx, jt, c), U, Uo in zip(comps, coeffs, sols):
            if np.linalg.norm(Uo) > 0:
                assert _rel(U, Uo) < 10 * tol, (jx, jt, _rel(U, Uo))
    return err, info


@pytest.mark.parametrize("prec", [0, 1])
def test_standing_wave_1d_level6(prec):
    """The 1D configuration: c = 1, f = 0, u0 = sin(pi x), n = 6, m = 1 (9 components)."""
    p = W.standing_wave(1, 6, 1)
    _run(p, prec, (5, 5))
    _run(p, prec, (6, 6))     # target finer than every component
    _run(p, prec, (3, 2))     # target coarser than most components


@pytest.mark.parametrize("prec", [0, 1])
def test_variable_speed_general_source_1d(prec):
    """Section 6.2 data: c^2 = 1 + x, u0 and v0 non-zero, non-separable f."""
    _run(W.e2_variable_speed(4), prec, (5, 5))


def test_vanishing_example_1d_domain_minus1_1():
    _run(W.e1_vanishing(4), 0, (6, 5))


def test_space_eigenbasis_components_1d():
    """n = 11, m = 1: components with 2^jt + 1 > 129 time unknowns use the
    spatial eigenbasis with banded time solves.  Their systems are
    ill-conditioned (the oracle's own sparse-LU solution of the (1,10)
    component leaves a relative residual of 6.6e-10, i.e. cond(S) eps ~ 1e-9),
    so two correct FP64 solvers agree only to that level: tolerance 2e-9."""
    _run(W.standing_wave(1, 11, 1), 0, (8, 8), check_components=True, tol=2e-9)


def test_single_component_level_zero():
    p = W.standing_wave(2, 6, 3)
    err, _ = _run(p, 0, (3, 3))


@pytest.mark.parametrize("prec", [0, 1])
def test_standing_wave_2d(prec):
    _run(W.standing_wave(2, 7, 2), prec, (5, 5))


@pytest.mark.parametrize("prec", [0, 1])
def test_layered_medium_2d_multigrid(prec):
    """The 2D layered medium at n = 8, m = 2: the (6,2) and (5,2) components
    (more than 1024 spatial unknowns) go through COCG with the multigrid
    V-cycle; the others are direct."""
    _run(W.layered_2d(8, 2), prec, (6, 6))


def test_layered_medium_2d_level9_fp64_direct_127():
    """n = 9: the (7,2) component (127^2 grid, half bandwidth 128) is solved by the
    banded direct method; in FP64 each mode spreads over four warps."""
    _run(W.layered_2d(9, 2), 0, (7, 7), method="schur")


def test_layered_medium_2d_level10():
    """n = 10: (8,2) 255^2 x 5 with a 4-level V-cycle; (2,8) with the space eigenbasis."""
    _run(W.layered_2d(10, 2), 1, (8, 8), method="schur", check_components=False)



@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_layered_n12_sampled_targets_and_backward_errors(prec):
    """The bench's workload at full size (layered 2D medium, n = 12, m = 2: 17 components,
    12.1 M space-time DOFs, target (10,10) of 1.08 G values) through st_solve_combine as the
    bench runs it.  (a) Target values at sampled nodes and times equal the oracle's own
    evaluation of Eq. (19) from the GPU's component arrays (independent of the combination
    kernel); (b) they match the oracle's own Schur-route solution of every component at
    64 x 16 sampled target values (fixture written by tests/golden/make_fullsize_samples.py);
    (c) the normwise backward error of every one of the 17 components, with S and F defined
    by the oracle, is below 10x the solver's target (set explicitly: the oracle's figure
    uses the 1-norm and the exact ||S||_1, the solver's the 2-norm and a bound of ||S||_2)."""
    import os
    import sys
    import torch
    from paper_2606_09688_gb300 import Solver
    from oracle import space
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_fullsize_samples as golden
    be_tol = 1e-13
    p = W.layered_2d(12, 2)
    target = (10, 10)
    rng = np.random.default_rng(12)
    pts, times = osolve.target_grid(p, *target)
    pi = np.sort(rng.choice(len(pts), 48, replace=False))
    si = np.sort(rng.choice(len(times), 12, replace=False))
    gpi, gsi, gref = golden.read("layered_2d_n12_m2")
    with Solver(p, precision=prec, tol=be_tol) as s:
        out, info = s.solve_combine(*target)
        got = out[torch.as_tensor(si, device=out.device)][:, torch.as_tensor(pi, device=out.device)].cpu().numpy()
        ggot = out[torch.as_tensor(gsi, device=out.device)][:, torch.as_tensor(gpi, device=out.device)].cpu().numpy()
        del out
        infos = s.components()
        coeffs = [s.coeffs(k) for k in range(len(infos))]
    assert info.status == 0
    ref = sum(ci.coef * osolve.evaluate_component(p, ci.jx, ci.jt, U, pts[pi], times[si])
              for ci, U in zip(infos, coeffs))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert _rel(ggot, gref) < (TOL64 if prec == 0 else TOL32), _rel(ggot, gref)
    worst = {}
    for ci, U in zip(infos, coeffs):
        worst[(ci.jx, ci.jt)] = osolve.backward_error(p, ci.jx, ci.jt, U, sm=space.space_matrices(p, ci.jx))
    assert len(worst) == 17 and max(worst.values()) < 10 * be_tol, worst


@pytest.mark.parametrize("prec", [0, 1])
def test_standing_wave_3d(prec):
    _run(W.standing_wave(3, 6, 2), prec, (4, 4))


def test_random_medium_3d_small():
    _run(W.random_medium_3d(6, 2, seed=3), 1, (4, 4))


@pytest.mark.parametrize("prec", [0, 1])
def test_random_medium_3d_31cubed_direct_backward_error(prec):
    """The 31^3 grid (band 993) is solved by the banded direct method; checked by
    the oracle's own assembly of S and F: the normwise backward error of the
    GPU's coefficient array is at the refinement target."""
    import scipy.sparse.linalg as spl
    from paper_2606_09688_gb300 import Solver
    p = W.random_medium_3d(7, 2, seed=3)
    with Solver(p, precision=prec) as s:
        infos = s.components()
        k = next(i for i, ci in enumerate(infos) if ci.jx == 5)
        s.solve(k)
        U = s.coeffs(k)
    jx, jt = infos[k].jx, infos[k].jt
    S = osolve.system_matrix(p, jx, jt)
    F = osolve.rhs(p, jx, jt)
    R = F.ravel() - S @ U.ravel()
    snorm = spl.norm(S, 1)
    eta = np.linalg.norm(R, 1) / (snorm * np.linalg.norm(U.ravel(), 1) + np.linalg.norm(F.ravel(), 1))
    assert eta < 1e-13, eta


def test_errors_are_reported():
    from paper_2606_09688_gb300 import Solver, StError
    from paper_2606_09688_gb300 import st as B
    bad = W.standing_wave(2, 6, 2)
    bad.c2 = lambda x: -np.ones(len(x))
    with pytest.raises(StError) as e:
        Solver(bad)
    assert e.value.code == B.ST_ERR_ARG
    boom = W.standing_wave(1, 4, 1)

    def raises(x):
        raise ValueError("data")
    boom.u0 = raises
    with pytest.raises(StError) as e:
        Solver(boom)
    assert e.value.code == B.ST_ERR_CALLBACK
    with Solver(W.standing_wave(1, 4, 1)) as s:
        with pytest.raises(StError) as e:
            s.combine(3, 3)
        assert e.value.code == B.ST_ERR_STATE
        with pytest.raises(StError) as e:
            s.solve(99)
        assert e.value.code == B.ST_ERR_ARG


def test_combine_subset_parts_add_up_to_the_combination():
    """Sharded combination (st_combine_subset): the parts of the ranks of an
    LPT partition sum to st_combine's result and to the oracle's."""
    from paper_2606_09688_gb300 import Solver, StError, shard
    from paper_2606_09688_gb300 import st as B
    p = W.layered_2d(8, 2)
    target = (6, 6)
    with Solver(p, precision=0) as s:
        with pytest.raises(StError) as e:
            s.combine_subset(*target, [0])
        assert e.value.code == B.ST_ERR_STATE          # component 0 not solved yet
        s.solve(-1)
        full = s.combine(*target).cpu().numpy()
        parts = shard.partition(shard.component_costs(s), 3)
        acc = sum(s.combine_subset(*target, ks).cpu().numpy() for ks in parts if ks)
        for bad in ([0, 0], [99], [-1]):
            with pytest.raises(StError) as e:
                s.combine_subset(*target, bad)
            assert e.value.code == B.ST_ERR_ARG
    assert np.max(np.abs(acc - full)) <= 1e-13 * np.max(np.abs(full))
    comps, sols = osolve.solve_all(p, method="schur")
    pts, times = osolve.target_grid(p, *target)
    assert _rel(acc, osolve.combine(p, comps, sols, pts, times)) < TOL64


def test_solve_batch_matches_separate_solves():
    """st_solve_batch over several instances gives each instance's own solution."""
    from paper_2606_09688_gb300 import ST_FP32_IR, Solver, StError, solve_batch
    probs = W.batch_instances(count=4, seed=5, levels=(6, 7, 8))
    solvers = [Solver(p, precision=ST_FP32_IR) for p in probs]
    try:
        info = solve_batch(solvers, max_threads=8)
        assert info.status == 0
        for p, s in zip(probs, solvers):
            J = p.J + 2 * p.mx
            tgt = (J - p.mx, J - p.mx)
            out = s.combine(*tgt).cpu().numpy()
            comps, sols = osolve.solve_all(p, method="schur")
            pts, times = osolve.target_grid(p, *tgt)
            assert _rel(out, osolve.combine(p, comps, sols, pts, times)) < TOL32
        with pytest.raises(StError):
            solve_batch([solvers[0], solvers[0]])
    finally:
        for s in solvers:
            s.close()


def test_autotuned_launch_shapes_keep_the_results():
    """Multigrid on a 127^2 grid (direct limit lowered so that it is not solved
    directly): with the built-in shapes, the autotuned shapes, and every 2D key
    pinned to the shared-memory tile kernel and then to the column-streaming
    kernel, the combination matches the oracle."""
    from paper_2606_09688_gb300 import ST_FP32_IR, ST_FP64, Solver, StError
    from paper_2606_09688_gb300.st import set_tuned_shape, tuned_shapes
    p = W.layered_2d(9, 2)
    target = (7, 7)
    comps, sols = osolve.solve_all(p, method="schur")
    pts, times = osolve.target_grid(p, *target)
    ref = osolve.combine(p, comps, sols, pts, times)

    def run(prec, tune):
        with Solver(p, precision=prec, max_direct_rows=4096, autotune=tune) as s:
            s.solve(-1)
            return s.combine(*target).cpu().numpy()
    for prec in (ST_FP64, ST_FP32_IR):
        tol = TOL64 if prec == ST_FP64 else TOL32
        assert _rel(run(prec, -1), ref) < tol
        assert _rel(run(prec, 1), ref) < tol
    shapes = tuned_shapes()
    assert any(e["nodes"] == 127 * 127 for e in shapes)
    for e in shapes:
        assert e["modes_per_thread"] in (1, 2, 3, 4) and e["block"] in (0, 64, 128, 256, 512)
        assert e["modes_per_thread"] != 3 or e["block"] == 64
    for kernel in (0, 64):        # the shared-memory tile kernel, then the column-streaming kernel
        pinned = 0
        for e in shapes:
            if e["d"] == 2 and e["op"] != 3:
                mq = 2 if (kernel == 0 and e["modes_per_thread"] == 3) else e["modes_per_thread"]
                set_tuned_shape(dict(e, block=kernel, modes_per_thread=mq))
                pinned += 1
        assert pinned > 0
        for prec in (ST_FP64, ST_FP32_IR):
            assert _rel(run(prec, -1), ref) < (TOL64 if prec == ST_FP64 else TOL32), kernel
    with pytest.raises(StError):
        set_tuned_shape(dict(shapes[0], modes_per_thread=3, block=128))


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_combine_overlapped_matches_separate_calls(prec):
    """st_solve_combine (combination levels enqueued as their components finish)
    gives the same target values as st_solve_component + st_combine, and the oracle's."""
    from paper_2606_09688_gb300 import Solver
    p = W.layered_2d(9, 2)
    target = (7, 7)
    with Solver(p, precision=prec) as s:
        out, info = s.solve_combine(*target)
        a = out.cpu().numpy()
        s.solve(-1)
        b = s.combine(*target).cpu().numpy()
        a2 = s.solve_combine(*target)[0].cpu().numpy()       # second call on the same handle
    assert info.status == 0
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    assert np.max(np.abs(a2 - b)) <= 1e-12 * np.max(np.abs(b))
    comps, sols = osolve.solve_all(p, method="schur")
    pts, times = osolve.target_grid(p, *target)
    assert _rel(a, osolve.combine(p, comps, sols, pts, times)) < (TOL64 if prec == 0 else TOL32)


@pytest.mark.parametrize("prec", [0, 1])
def test_back_to_back_solve_combine_calls_overlap_correctly(prec):
    """Consecutive st_solve_combine calls on one handle, with no synchronisation in
    between, overlap the next call's solves with the previous call's combination
    levels (the levels read pair copies of the components, double-buffered).  Three
    queued calls with different targets and outputs give exactly the targets of
    separate, synchronised calls."""
    import torch
    from paper_2606_09688_gb300 import Solver
    p = W.layered_2d(9, 2)
    targets = [(7, 7), (6, 5), (7, 7), (5, 6)]
    with Solver(p, precision=prec) as s:
        ref = []
        for t in targets:
            out, info = s.solve_combine(*t)
            assert info.status == 0
            ref.append(out.cpu().numpy())
            s.solve(0)                 # another call in between: the next one starts afresh
        outs = [s.solve_combine(*t, sync=False)[0] for t in targets]
        torch.cuda.synchronize()
        got = [o.cpu().numpy() for o in outs]
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


GRAPH_CASES = [
    # (workload, precision, COCG iterations per convergence test, direct limit, target)
    ("layered_2d_n8_multigrid", 0, 4, 500, (6, 6)),
    ("layered_2d_n8_multigrid", 1, 8, 500, (6, 6)),
    ("layered_2d_n8_direct", 1, 4, 0, (6, 6)),
    ("standing_wave_1d_n11_space_eigenbasis", 0, 4, 0, (8, 8)),
]


def _graph_problem(name):
    if name.startswith("layered_2d_n8"):
        return W.layered_2d(8, 2)
    return W.standing_wave(1, 11, 1)


@pytest.mark.parametrize("name,prec,body,max_direct,target", GRAPH_CASES)
def test_graph_solves_match_the_oracle(name, prec, body, max_direct, target):
    """Every forward solve as one CUDA graph (st_options.device_loop): refinement sweeps
    in a WHILE node with the backward-error test on the device, each sweep's COCG loop
    in a nested WHILE node.  Multigrid, direct and space-eigenbasis components give the
    oracle's combined targets (1e-10 FP64 / 1e-8 FP32 + IR; 2e-9 where the space
    eigenbasis is used, as for the host-driven path) and reach the backward-error target."""
    from paper_2606_09688_gb300 import Solver
    p = _graph_problem(name)
    kw = {"max_direct_rows": max_direct} if max_direct else {}
    with Solver(p, precision=prec, device_loop=body, **kw) as s:
        info = s.solve(-1)
        out = s.combine(*target).cpu().numpy()
        methods = {ci.method for ci in s.components()}
    assert info.status == 0 and info.sweeps >= 1 and info.backward_error <= 1e-13
    if "multigrid" in name:
        assert info.max_inner_iters > 0
    if "space_eigenbasis" in name:
        assert 1 in methods
    comps, sols = osolve.solve_all(p, method="schur")
    pts, times = osolve.target_grid(p, *target)
    ref = osolve.combine(p, comps, sols, pts, times)
    tol = 2e-9 if "space_eigenbasis" in name else (TOL64 if prec == 0 else TOL32)
    assert _rel(out, ref) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_solves_equal_host_driven_solves_bitwise(prec):
    """With 4 COCG iterations per convergence test the graph runs the same kernels in
    the same order as the host-driven loop (which checks every 4 iterations), so the
    component arrays, sweeps and backward errors are identical."""
    from paper_2606_09688_gb300 import Solver
    p = W.layered_2d(8, 2)
    res = []
    for body in (0, 4):
        with Solver(p, precision=prec, max_direct_rows=500, device_loop=body, autotune=-1) as s:
            info = s.solve(-1)
            res.append((info, [s.coeffs(k) for k in range(s.num_components)]))
    (i0, u0), (i1, u1) = res
    assert i0.sweeps == i1.sweeps and i0.backward_error == i1.backward_error
    for a, b in zip(u0, u1):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("body", [0, 4])
def test_repeated_solves_are_bit_reproducible(body):
    """The reductions (COCG dot products, norms, the combination) are deterministic:
    two st_solve_combine calls on one handle give bit-identical targets."""
    from paper_2606_09688_gb300 import ST_FP32_IR, Solver
    with Solver(W.layered_2d(9, 2), precision=ST_FP32_IR, device_loop=body) as s:
        a = s.solve_combine(7, 7)[0].cpu().numpy()
        s.solve(0)
        b = s.solve_combine(7, 7)[0].cpu().numpy()
    assert np.array_equal(a, b)


def test_graph_batch_of_32_instances_matches_the_oracle():
    """st_solve_batch with graph solves: the components of 32 instances (levels 6-8,
    uneven sizes) are enqueued from one thread, largest first, with one host
    synchronisation for the batch; every instance's combined target matches the
    oracle (FP32 + IR, 1e-8)."""
    from paper_2606_09688_gb300 import ST_FP32_IR, Solver, solve_batch
    probs = W.batch_instances(count=32, seed=7, levels=(6, 7, 8))
    solvers = [Solver(p, precision=ST_FP32_IR, device_loop=4) for p in probs]
    try:
        info = solve_batch(solvers)
        assert info.status == 0 and info.backward_error <= 1e-13
        for p, s in zip(probs, solvers):
            tgt = (p.J + p.mx, p.J + p.mx)
            out = s.combine(*tgt).cpu().numpy()
            comps, sols = osolve.solve_all(p, method="schur")
            pts, times = osolve.target_grid(p, *tgt)
            assert _rel(out, osolve.combine(p, comps, sols, pts, times)) < TOL32, p.name
    finally:
        for s in solvers:
            s.close()


@pytest.mark.parametrize("body", [0, 4])
def test_tight_target_takes_later_sweeps_with_adaptive_inner_tolerance(body):
    """A backward-error target of 1e-15 needs a second FP64 sweep on the multigrid
    components; that sweep solves only to the tolerance the remaining reduction needs
    (next_inner_tol), on the host-driven loop and in graph solves, and still reaches
    (or stagnates within 1e3 of) the target with the oracle's combined solution."""
    from paper_2606_09688_gb300 import ST_FP64, Solver
    p = W.layered_2d(8, 2)
    with Solver(p, precision=ST_FP64, max_direct_rows=500, tol=1e-15, device_loop=body) as s:
        info = s.solve(-1)
        out = s.combine(6, 6).cpu().numpy()
    assert info.status == 0 and info.sweeps >= 2 and info.backward_error < 1e-14
    comps, sols = osolve.solve_all(p, method="schur")
    pts, times = osolve.target_grid(p, 6, 6)
    assert _rel(out, osolve.combine(p, comps, sols, pts, times)) < TOL64
