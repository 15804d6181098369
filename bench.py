#!/usr/bin/env python3
"""Throughput benchmark of the space-time sparse-grid wave solver.

One step = the whole hot path on one problem instance: every component of
the combination formula solved (right-hand side, time transforms, spatial mode
solves, FP64 refinement) and the +-1 combination evaluated on the nodal target
grid.  Metric: space-time DOFs/s, DOFs = sum over components of
dim V_jx x dim V_jt (the sparse DoF count of Section 3.2), device-timed with
CUDA events on the solver's stream.  Inputs are resident in HBM after setup;
the 8.6 GB combination output written every step is larger than L2, so each
step starts with a cold L2.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun every rank solves its own instance (independent problems,
weak scaling, no collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

if "--impl" in sys.argv and "reference" in sys.argv:
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import st_workloads as W  # noqa: E402

WORKLOADS = {
    # name: (problem factory, target (jx*, jt*), description)
    "layered_2d_n12": (lambda: W.layered_2d(12, 2), (10, 10),
                       "d=2, c^2 in {1,4} (layer at y=0.5), Gaussian x Ricker source, n=12, m=2, 17 components"),
    "layered_2d_n12_t6": (lambda: W.layered_2d(12, 2), (6, 6),
                          "the layered 2D workload with a (6,6) target grid (profiling the solves)"),
    "layered_2d_n10": (lambda: W.layered_2d(10, 2), (8, 8),
                       "d=2, layered c^2, Gaussian x Ricker source, n=10, m=2, 13 components (profiling size)"),
    "standing_wave_1d_n6": (lambda: W.standing_wave(1, 6, 1), (5, 5),
                            "d=1, c=1, u0=sin(pi x), n=6, m=1, 9 components"),
    "random_medium_3d_n10": (lambda: W.random_medium_3d(10, 3), (7, 7),
                             "d=3, c^2=clip(exp(16-mode field),0.25,4), u0=prod sin, n=10, m=3, 9 components"),
}
METRIC = "space-time DOFs/s (all components, device-timed) + HBM roofline %, FP32+IR vs FP64"
HBM_FALLBACK = 6800.0
FP64_PEAK_GFLOPS = 1250.0      # nominal dense FP64 rate of GB300
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.07   # SMs x FP32 lanes x 2 flop x max SM GHz
FP64_CLASSES = {"combine_level", "st_residual_fp64", "norm_fp64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="layered_2d_n12", choices=sorted(WORKLOADS) + ["batch64"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32ir"],
                    help="precision of the headline value; the other one is reported beside it")
    ap.add_argument("--skip", default="", help="comma list of: other,profile,e2e,cpu")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="inner Krylov tolerance per refinement sweep (0 = library default)")
    ap.add_argument("--max-direct-rows", type=int, default=0,
                    help="largest spatial grid solved by the banded direct method (0 = library default)")
    ap.add_argument("--only-component", type=int, default=-1,
                    help="profiling aid: each step solves only this component (no combination)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_FALLBACK)), "measured"
    return HBM_FALLBACK, "fallback"


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, bus_id=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if bus_id:
            mine = [r for r in rows if bus_id.lower() in r[1].lower()]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- oracle sample
def oracle_sample(workload, dof_cap=300000):
    """Oracle (CPU, FP64) on a bounded sample of the workload: every component
    with at most dof_cap space-time DOFs, each by the oracle's exact
    Schur-in-time route (complex Schur form of B^-1 A, one sparse LU per time
    mode).  Returns (dofs, seconds, list of components)."""
    from oracle import combination, solve as osolve
    p = WORKLOADS[workload][0]()
    comps = combination.components(p.J, p.mx, p.mt)
    sample = [(jx, jt, c) for jx, jt, c in comps
              if combination.space_dofs(p.d, jx) * combination.time_dofs(jt) <= dof_cap]
    t0 = time.perf_counter()
    dofs = 0
    for jx, jt, c in sample:
        U = osolve.solve_component(p, jx, jt, method="schur")
        dofs += U.size
    return dofs, time.perf_counter() - t0, sample


def _oracle_component(args):
    workload, jx, jt = args
    from oracle import solve as osolve
    p = WORKLOADS[workload][0]()
    return osolve.solve_component(p, jx, jt, method="schur").size


def oracle_sample_parallel(workload, workers, dof_cap=300000):
    """The same sample as oracle_sample, its components spread over a pool of
    single-threaded worker processes (largest first); the pool is started and
    warmed before the clock starts.  Returns (dofs, seconds, components)."""
    import concurrent.futures as cf
    import multiprocessing as mpc
    from oracle import combination
    p = WORKLOADS[workload][0]()
    comps = combination.components(p.J, p.mx, p.mt)
    sample = [(jx, jt, c) for jx, jt, c in comps
              if combination.space_dofs(p.d, jx) * combination.time_dofs(jt) <= dof_cap]
    order = sorted(sample, key=lambda t: -combination.space_dofs(p.d, t[0]) * combination.time_dofs(t[1]))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mpc.get_context("spawn")) as ex:
        list(ex.map(_oracle_component, [(workload, 1, 0)] * workers))  # start-up and imports, untimed
        t0 = time.perf_counter()
        dofs = sum(ex.map(_oracle_component, [(workload, jx, jt) for jx, jt, _ in order]))
        secs = time.perf_counter() - t0
    return dofs, secs, sample


def cpu_baseline(workload):
    """The oracle on this host: one thread, and all cores (one single-threaded
    worker process per core, components spread over them)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cores = os.cpu_count() or 1
    code = ("import json,sys; sys.path.insert(0, %r); import bench; d,s,c = bench.oracle_sample(%r); "
            "dp,sp,_ = bench.oracle_sample_parallel(%r, %d); print(json.dumps([d, s, c, dp, sp]))"
            % (ROOT, workload, workload, cores))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": "DOFs/s", "cores": cores, "kind": "oracle", "sample": "failed: " + r.stderr[-200:]}
    dofs, secs, comps, dofs_p, secs_p = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": dofs_p / secs_p, "unit": "DOFs/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(comps)} smallest components (<= 300000 DOFs each, {dofs} DOFs) of the same workload, "
                      f"oracle Schur-in-time sparse LU solves spread over {cores} single-threaded processes, "
                      f"{secs_p:.1f} s; combination not included",
            "one_thread": {"value": dofs / secs, "cores": 1, "seconds": secs}}


def run_reference(args):
    """The oracle on this host's cores (one single-threaded worker process per
    core, the sample's components spread over them, largest first), each step
    one bounded sample of the workload; rank 0 only."""
    import concurrent.futures as cf
    import multiprocessing as mpc
    from oracle import combination
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    p = WORKLOADS[args.workload][0]()
    comps = combination.components(p.J, p.mx, p.mt)
    sample = [(jx, jt, c) for jx, jt, c in comps
              if combination.space_dofs(p.d, jx) * combination.time_dofs(jt) <= 300000]
    order = sorted(sample, key=lambda t: -combination.space_dofs(p.d, t[0]) * combination.time_dofs(t[1]))
    tasks = [(args.workload, jx, jt) for jx, jt, _ in order]
    t = []
    dofs = 0
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mpc.get_context("spawn")) as ex:
        list(ex.map(_oracle_component, [(args.workload, 1, 0)] * cores))  # start-up and imports
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            dofs = sum(ex.map(_oracle_component, tasks))
            if step >= args.warmup:
                t.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(t))
    value = dofs / (ms / 1e3)
    desc = (f"{len(sample)} smallest components (<= 300000 DOFs each, {dofs} DOFs) of {args.workload}, "
            f"oracle Schur-in-time sparse LU solves spread over {cores} single-threaded processes; "
            "combination not included")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOFs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload][2]},
            "cpu_baseline": {"value": value, "unit": "DOFs/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "DOFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours
def csrc_hash(files=None):
    """Hash of CUDA/C++ sources of the library (all of them, or the listed
    files): a changed kernel invalidates its ncu numbers."""
    src = os.path.join(ROOT, "paper_2606_09688_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(files if files is not None else os.listdir(src)):
        with open(os.path.join(src, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()


def traffic_for(kclass, precision):
    """DRAM bytes per launch of a kernel class ("<precision>:<class>@<unknowns>")
    from the committed ncu summary, or None when the source files that define
    the kernel have changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get("bytes_per_launch", {}).get(f"{precision}:{kclass}")
    if not e or not e.get("sources") or e.get("sha256") != csrc_hash(e["sources"]):
        return None
    return e.get("bytes")


def timed_steps(solver, out, target, steps, stream, torch, only=-1):
    jx, jt = target
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        if only >= 0:
            solver.solve(only, sync=False)
            continue
        solver.solve_combine(jx, jt, out, sync=False)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / steps


def roofline(stats, hbm, hbm_src, precision):
    if not stats:
        return None
    top = max(stats, key=lambda s: s["ms"])
    gbs = top["bytes"] / (top["ms"] * 1e6)
    gflops = top["flops"] / (top["ms"] * 1e6)
    # the combination and the refinement residual compute in FP64 on both paths
    fp64_kernel = precision == "fp64" or top["name"].split("@")[0] in FP64_CLASSES
    alu_peak = FP64_PEAK_GFLOPS if fp64_kernel else FP32_PEAK_GFLOPS
    fh, fa = gbs / hbm, gflops / alu_peak
    tr = traffic_for(top["name"], precision)
    if fa > fh:
        src = ("derived: GB300 nominal dense FP64 1.25 TFLOP/s" if fp64_kernel else
               "derived: GB300 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz")
        r = {"bound": "alu", "achieved": gflops / 1e3, "peak": alu_peak / 1e3, "unit": "TFLOP/s", "frac": fa,
             "peak_source": src}
    else:
        r = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": fh,
             "peak_source": f"{hbm_src} MEASURED_PEAKS.json hbm_gbs"}
    r.update({"traffic": tr, "kernel": top["name"], "launches": top["launches"],
              "ms_per_launch": top["ms"] / top["launches"], "bytes_per_launch": top["bytes"] / top["launches"],
              "share_of_profiled_time": top["ms"] / sum(s["ms"] for s in stats),
              "achieved_gbs": gbs, "achieved_gflops": gflops})
    return r


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2606_09688_gb300 import ST_FP32_IR, ST_FP64, Solver
    from paper_2606_09688_gb300 import build as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build(force=False)
    skip = set(filter(None, args.skip.split(",")))
    factory, target, desc = WORKLOADS[args.workload]
    problem = factory()
    stream = torch.cuda.Stream(device=dev)
    hbm, hbm_src = peaks()
    nsp = ((1 << target[0]) + 1) ** problem.d
    nts = (1 << target[1]) + 1
    out = torch.empty((nts, nsp), dtype=torch.float64, device=dev)
    # pinned host buffer for the end-to-end measurement, allocated once up front
    host_out = None if "e2e" in skip else torch.empty((nts, nsp), dtype=torch.float64, pin_memory=True)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def maxall(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    results = {}
    precs = [args.precision] + ([] if "other" in skip else [p for p in ("fp64", "fp32ir") if p != args.precision])
    for prec in precs:
        code = ST_FP64 if prec == "fp64" else ST_FP32_IR
        with torch.cuda.stream(stream):
            t0 = time.perf_counter()
            solver = Solver(problem, precision=code, stream=stream, inner_tol=args.inner_tol,
                            max_direct_rows=args.max_direct_rows)
            setup_s = time.perf_counter() - t0
            dofs = solver.total_dofs
            for _ in range(args.warmup):
                if args.only_component < 0:
                    solver.solve_combine(target[0], target[1], out, sync=False)
                else:
                    solver.solve(args.only_component, sync=False)
            if args.only_component < 0:
                _, info = solver.solve_combine(target[0], target[1], out, sync=True)
            else:
                info = solver.solve(args.only_component, sync=True)
            barrier()
            l0 = solver.kernel_launches
            clocks = Clocks()
            if prec == args.precision:
                clocks.start()
            ms = timed_steps(solver, out, target, args.steps, stream, torch, args.only_component)
            launches = (solver.kernel_launches - l0) // args.steps
            ck = clocks.stop(getattr(torch.cuda.get_device_properties(dev), "pci_bus_id", None)) \
                if prec == args.precision else None
            barrier()
            ms = maxall(ms)
            stats = None
            comp_ms = None
            if "profile" not in skip:
                solver.profile(True)
                solver.solve(args.only_component, sync=False)
                if args.only_component < 0:
                    solver.combine(target[0], target[1], out)
                stats = solver.profile_read()
                solver.profile(False)
                # each component alone (what bounds the step when they overlap)
                comp_ms = []
                for k, ci in enumerate(solver.components()):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    solver.solve(k, sync=False)
                    b.record(stream)
                    b.synchronize()
                    comp_ms.append({"jx": ci.jx, "jt": ci.jt, "method": ci.method, "modes": ci.n_modes,
                                    "ms": a.elapsed_time(b)})
            results[prec] = dict(ms=ms, value=dofs * world / (ms / 1e3), dofs=dofs, setup_s=setup_s,
                                 launches=launches, clocks=ck, stats=stats, comp_ms=comp_ms,
                                 sweeps=info.sweeps, inner_iters=info.max_inner_iters,
                                 backward_error=info.backward_error, rel_residual=info.rel_residual,
                                 solver=solver)
    head = results[args.precision]
    # end to end through the public API with host buffers: setup from the host
    # data (callbacks, uploads), solve, combine, copy the target grid to pinned host memory
    e2e = None
    if "e2e" not in skip:
        for r in results.values():
            r["solver"].close()
        code = ST_FP64 if args.precision == "fp64" else ST_FP32_IR
        e2e_steps = max(1, min(args.steps, 2))
        # one untimed pass first: the pinned output buffer's pages are mapped
        # for the GPU on its first copy
        with torch.cuda.stream(stream):
            s = Solver(problem, precision=code, stream=stream, inner_tol=args.inner_tol,
                            max_direct_rows=args.max_direct_rows)
            s.solve_combine(target[0], target[1], out, sync=False)
            host_out.copy_(out, non_blocking=True)
            stream.synchronize()
            s.close()
        barrier()
        t0 = time.perf_counter()
        h2d = d2h = 0
        phase = [0.0, 0.0, 0.0, 0.0]  # setup, solve + combine, copy to host, release
        for _ in range(e2e_steps):
            with torch.cuda.stream(stream):
                ta = time.perf_counter()
                s = Solver(problem, precision=code, stream=stream, inner_tol=args.inner_tol,
                            max_direct_rows=args.max_direct_rows)
                tb = time.perf_counter()
                s.solve_combine(target[0], target[1], out, sync=False)
                stream.synchronize()
                tc = time.perf_counter()
                host_out.copy_(out, non_blocking=True)
                stream.synchronize()
                td = time.perf_counter()
                a, b = s.transfer_bytes()
                h2d += a
                d2h += b + host_out.numel() * 8
                s.close()
                te = time.perf_counter()
                for k, dt in enumerate((tb - ta, tc - tb, td - tc, te - td)):
                    phase[k] += dt / e2e_steps
        e2e_s = maxall((time.perf_counter() - t0) / e2e_steps)
        e2e = {"value": head["dofs"] * world / e2e_s, "unit": "DOFs/s", "h2d_bytes_per_step": h2d // e2e_steps,
               "d2h_bytes_per_step": d2h // e2e_steps, "s_per_step": e2e_s,
               "includes": "st_setup from host callbacks + solve + combine + target grid copied to pinned host",
               "phases_s": {"setup": phase[0], "solve_combine": phase[1], "copy_to_host": phase[2],
                            "release": phase[3]}}
    if rank != 0:
        return
    cpu = None if "cpu" in skip else cpu_baseline(args.workload)
    rl = roofline(head["stats"], hbm, hbm_src, args.precision)
    line = {
        "metric": METRIC, "value": head["value"], "unit": "DOFs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded recipe of the workload; no dataset)",
        "config": {"workload": args.workload, "desc": desc, "target": list(target), "precision": args.precision,
                   "space_time_dofs": head["dofs"], "l2": "each step writes the 8.6 GB target grid (> L2)",
                   "parallelism": f"{world} independent instance(s), one per GPU"},
        "gpu_launches": head["launches"], "clocks": head["clocks"], "roofline": rl, "cpu_baseline": cpu, "e2e": e2e,
        "setup_s": head["setup_s"], "sweeps": head["sweeps"], "inner_iters": head["inner_iters"],
        "backward_error": head["backward_error"],
    }
    for prec, r in results.items():
        if prec == args.precision:
            continue
        line[prec] = {"value": r["value"], "ms_per_step": r["ms"], "setup_s": r["setup_s"],
                      "gpu_launches": r["launches"], "sweeps": r["sweeps"], "inner_iters": r["inner_iters"],
                      "backward_error": r["backward_error"], "roofline": roofline(r["stats"], hbm, hbm_src, prec)}
    line["kernels"] = {prec: r["stats"] for prec, r in results.items()}
    line["components_alone_ms"] = {prec: r["comp_ms"] for prec, r in results.items()}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Batching configuration: 64 independent 2D instances (levels n in 8..12,
    random smooth c^2 in [0.5, 2] with a jump, random Gaussian sources), all
    components of all instances solved together by st_solve_batch.  Value =
    space-time DOFs of all instances per second of the batch solve (combination
    excluded: each instance's own target grid would total ~120 GB)."""
    import torch
    from paper_2606_09688_gb300 import ST_FP32_IR, ST_FP64, Solver, solve_batch
    torch.cuda.set_device(0)
    code = ST_FP64 if args.precision == "fp64" else ST_FP32_IR
    probs = W.batch_instances(64)
    t0 = time.perf_counter()
    solvers = [Solver(p, precision=code, inner_tol=args.inner_tol, max_direct_rows=args.max_direct_rows)
               for p in probs]
    setup_s = time.perf_counter() - t0
    dofs = sum(s.total_dofs for s in solvers)
    for _ in range(args.warmup):
        solve_batch(solvers)
    torch.cuda.synchronize()
    times = []
    info = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        info = solve_batch(solvers)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    levels = {}
    for p in probs:
        levels[p.J + 2 * p.mx] = levels.get(p.J + 2 * p.mx, 0) + 1
    line = {"metric": METRIC, "value": dofs / (ms / 1e3), "unit": "DOFs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if code == ST_FP64 else "f32+f64", "data": "synthetic",
            "config": {"workload": "batch64", "instances": len(probs), "levels_n": levels, "space_time_dofs": dofs,
                       "timing": "host wall clock around st_solve_batch (blocking, all streams synchronised)",
                       "combination": "excluded"},
            "setup_s": setup_s, "sweeps": info.sweeps, "inner_iters": info.max_inner_iters,
            "backward_error": info.backward_error}
    for s in solvers:
        s.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
