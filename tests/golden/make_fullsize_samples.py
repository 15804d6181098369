"""Writes the sampled target values of the full-size parity tests.

For each workload below it solves every component of Eq. (19) with the
oracle's exact Schur-in-time route (complex Schur form of B^-1 A, one sparse
LU per time mode), evaluates the combination at a seeded sample of target
nodes and times (all nodes' indices drawn without replacement), and writes a
text fixture: the sampled node indices, time indices and the values
u^CF(x_p, t_s), one row per sampled time.

It calls only ``oracle`` and ``st_workloads``.  Run from the repository root:
    python tests/golden/make_fullsize_samples.py [name ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import st_workloads as W  # noqa: E402
from oracle import combination, solve as osolve  # noqa: E402

# name: (problem factory, target (jx*, jt*), sampled nodes, sampled times, seed)
FIXTURES = {
    "layered_2d_n12_m2": (lambda: W.layered_2d(12, 2), (10, 10), 64, 16, 1201),
    "random_medium_3d_n8_m3": (lambda: W.random_medium_3d(8, 3), (5, 5), 64, 16, 803),
}


def sample_indices(p, target, n_pts, n_times, seed):
    """Seeded node and time indices of the target grid (sorted)."""
    rng = np.random.default_rng(seed)
    nsp = ((1 << target[0]) + 1) ** p.d
    nts = (1 << target[1]) + 1
    return (np.sort(rng.choice(nsp, n_pts, replace=False)), np.sort(rng.choice(nts, n_times, replace=False)))


def write(name):
    factory, target, n_pts, n_times, seed = FIXTURES[name]
    p = factory()
    pi, si = sample_indices(p, target, n_pts, n_times, seed)
    pts, times = osolve.target_grid(p, *target)
    comps = combination.components(p.J, p.mx, p.mt)
    vals = np.zeros((len(si), len(pi)))
    t0 = time.time()
    for jx, jt, c in comps:
        U = osolve.solve_component(p, jx, jt, method="schur")
        vals += c * osolve.evaluate_component(p, jx, jt, U, pts[pi], times[si])
        print(f"{name}: ({jx},{jt}) done at {time.time() - t0:.0f} s", flush=True)
    path = os.path.join(HERE, f"{name}_samples.txt")
    with open(path, "w") as f:
        f.write(f"# Oracle values of u^CF (Eq. (19)) at sampled target nodes, workload {name}, "
                f"target ({target[0]},{target[1]}), seed {seed}.\n")
        f.write("# Written by tests/golden/make_fullsize_samples.py (oracle Schur-in-time solves only).\n")
        f.write("# Line 3: node indices; line 4: time indices; then one line of values per sampled time.\n")
        f.write(" ".join(str(int(i)) for i in pi) + "\n")
        f.write(" ".join(str(int(i)) for i in si) + "\n")
        for row in vals:
            f.write(" ".join(f"{v:.17e}" for v in row) + "\n")
    print(path)


def read(name):
    """(node indices, time indices, values[time, node]) of a fixture."""
    path = os.path.join(HERE, f"{name}_samples.txt")
    rows = [ln for ln in open(path) if not ln.startswith("#")]
    pi = np.array(rows[0].split(), dtype=np.int64)
    si = np.array(rows[1].split(), dtype=np.int64)
    vals = np.array([r.split() for r in rows[2:]], dtype=np.float64)
    return pi, si, vals


if __name__ == "__main__":
    for n in (sys.argv[1:] or sorted(FIXTURES)):
        write(n)
