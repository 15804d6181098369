"""Component sharding over ranks (host logic), on CPU with the gloo backend.

Each rank solves and combines only its share of the components; one
sum-reduction gives the full combination of Eq. (19) on every rank.  The
per-component work here is done by the oracle (CPU, FP64) behind the same
interface as the GPU solver (components(), solve(k), combine_subset(...)), so
the partition and the collective run exactly as in a multi-GPU run.
"""
import os
import socket
from types import SimpleNamespace

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import st_workloads as W
from paper_2606_09688_gb300 import shard


def test_partition_covers_every_component_once_and_balances():
    rng = np.random.default_rng(7)
    for n in (1, 5, 17, 31):
        costs = rng.integers(1, 10_000_000, size=n).astype(float)
        for world in (1, 2, 3, 4, 8):
            parts = shard.partition(costs, world)
            assert len(parts) == world
            flat = sorted(k for p in parts for k in p)
            assert flat == list(range(n))
            loads = [sum(costs[k] for k in p) for p in parts]
            # any greedy list schedule: makespan <= mean load + largest job
            assert max(loads) <= costs.sum() / world + costs.max() + 1e-6
    # LPT is within 4/3 of the optimal makespan (Graham 1969): brute force on small sets
    import itertools
    for trial in range(20):
        costs = rng.integers(1, 100, size=7).astype(float)
        for world in (2, 3):
            best = min(max(sum(costs[k] for k in range(7) if a[k] == r) for r in range(world))
                       for a in itertools.product(range(world), repeat=7))
            parts = shard.partition(costs, world)
            lpt = max(sum(costs[k] for k in p) for p in parts)
            assert lpt <= (4.0 / 3.0) * best + 1e-9
    # same input, same partition (every rank computes it independently)
    c = [5.0, 5.0, 3.0, 3.0, 2.0]
    assert shard.partition(c, 2) == shard.partition(list(c), 2)
    with pytest.raises(ValueError):
        shard.partition(c, 0)


class OracleSolver:
    """The oracle behind the solver interface that shard.sharded_combine uses."""

    def __init__(self, problem):
        from oracle import combination
        self.problem = problem
        self.comps = combination.components(problem.J, problem.mx, problem.mt)
        self.sols = {}

    def components(self):
        from oracle import combination
        d = self.problem.d
        return [SimpleNamespace(jx=jx, jt=jt, coef=c, n_space=combination.space_dofs(d, jx),
                                n_time=combination.time_dofs(jt)) for jx, jt, c in self.comps]

    def solve(self, k, sync=True):
        from oracle import solve as S
        jx, jt, _ = self.comps[k]
        self.sols[k] = S.solve_component(self.problem, jx, jt)

    def combine_subset(self, jx_star, jt_star, ks, out):
        from oracle import solve as S
        pts, times = S.target_grid(self.problem, jx_star, jt_star)
        val = S.combine(self.problem, [self.comps[k] for k in ks], [self.sols[k] for k in ks], pts, times)
        out.copy_(torch.from_numpy(val))
        return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, target, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = W.e2_variable_speed(5)
        solver = OracleSolver(p)
        nts, nsp = (1 << target[1]) + 1, ((1 << target[0]) + 1) ** p.d
        out = torch.zeros((nts, nsp), dtype=torch.float64)
        shard.sharded_combine(solver, target[0], target[1], out, rank, world)
        mine = shard.partition(shard.component_costs(solver), world)[rank]
        results[rank] = (out.numpy().copy(), sorted(solver.sols))
        assert sorted(solver.sols) == mine
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_sharded_combination_gloo_matches_the_full_sum(world):
    from oracle import solve as S
    target = (4, 4)
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), target, results), nprocs=world,
                       start_method="spawn", join=True)
    p = W.e2_variable_speed(5)
    comps, sols = S.solve_all(p)
    pts, times = S.target_grid(p, *target)
    full = S.combine(p, comps, sols, pts, times)
    owned = []
    for r in range(world):
        got, ks = results[r]
        owned += ks
        assert np.max(np.abs(got - full)) <= 1e-13 * np.max(np.abs(full))
    assert sorted(owned) == list(range(len(comps)))   # every component solved by exactly one rank


class FailingSolver(OracleSolver):
    """A solver whose first solve raises (a failed component on one rank)."""

    def solve(self, k, sync=True):
        raise RuntimeError("component solve failed on this rank")


def _rank_main_failing(rank, world, port, results):
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    p = W.e2_variable_speed(3)
    solver = FailingSolver(p) if rank == 1 else OracleSolver(p)
    out = torch.zeros(((1 << 3) + 1, (1 << 3) + 1), dtype=torch.float64)
    try:
        shard.sharded_combine(solver, 3, 3, out, rank, world)
        results[rank] = "completed"
    except Exception as e:  # the failing rank's own error, or the collective's on the others
        results[rank] = "error: " + type(e).__name__
        if rank == 1:
            raise          # the failed rank leaves (process exit code != 0)
    finally:
        if rank == 0:
            try:
                dist.destroy_process_group()
            except Exception:
                pass


def test_a_failed_rank_is_detected_by_the_others():
    """Rank 1 fails before the sum-reduction of the sharded combination; rank 0 does not
    hang in the collective: the collective ends with an error (peer gone or timeout)."""
    import time
    world = 2
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    t0 = time.time()
    ctx = mp.start_processes(_rank_main_failing, args=(world, _free_port(), results), nprocs=world,
                             start_method="spawn", join=False)
    for p in ctx.processes:
        p.join(timeout=120)
    codes = [p.exitcode for p in ctx.processes]
    for p in ctx.processes:
        if p.is_alive():
            p.kill()
    assert codes[1] not in (0, None)                      # the failed rank exited with an error
    assert codes[0] == 0 and results[0].startswith("error")  # the other rank saw the failure and returned
    assert time.time() - t0 < 120
