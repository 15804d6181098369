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
FP64_NOMINAL_GFLOPS = 1250.0      # nominal dense FP64 rate of GB300 (used only if the probe fails)
FP32_NOMINAL_GFLOPS = 152 * 128 * 2 * 2.07   # SMs x FP32 lanes x 2 flop x max SM GHz
FP64_CLASSES = {"st_residual_fp64", "norm_fp64"}
DS_CLASSES = {"combine_level"}      # double-single arithmetic on the FP32 pipe in both precisions


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="layered_2d_n12", choices=sorted(WORKLOADS) + ["batch64"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32ir"],
                    help="precision of the headline value; the other one is reported beside it")
    ap.add_argument("--skip", default="", help="comma list of: other,profile,e2e,cpu,cfg3,batch64")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="inner Krylov tolerance per refinement sweep (0 = library default)")
    ap.add_argument("--max-direct-rows", type=int, default=0,
                    help="largest spatial grid solved by the banded direct method (0 = library default)")
    ap.add_argument("--only-component", type=int, default=-1,
                    help="profiling aid: each step solves only this component (no combination)")
    ap.add_argument("--target", default="",
                    help="profiling aid: target levels 'jx,jt' in place of the workload's")
    ap.add_argument("--device-loop", type=int, default=None, choices=[0, 4, 8, 16],
                    help="every solve as one CUDA graph, k COCG iterations per device-side convergence test "
                         "(0 = host-driven solves; default: 0 for a single instance, 4 for the batch)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_FALLBACK)), "measured"
    return HBM_FALLBACK, "fallback"


def alu_peaks():
    """FP64 and FP32 FMA rates of this device measured by st_probe_fma (GFLOP/s),
    the denominators of the "alu" roofline fractions; nominal figures only if
    the probe fails."""
    from paper_2606_09688_gb300.st import probe_fma
    out = {}
    for name, prec, nominal in (("fp64", 0, FP64_NOMINAL_GFLOPS), ("fp32", 1, FP32_NOMINAL_GFLOPS)):
        try:
            probe_fma(prec, 256)
            out[name] = (max(probe_fma(prec, 4096) for _ in range(3)), "measured by st_probe_fma")
        except Exception as e:  # reported in the line's peak_source
            out[name] = (nominal, f"nominal (probe failed: {str(e)[:60]})")
    return out


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
            "sample_short": f"{len(comps)} smallest components ({dofs} DOFs), solves only",
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


def roofline(stats, hbm, hbm_src, precision, alu):
    """Roofline entry of the kernel class with the largest summed event time:
    achieved = its algorithmic bytes (or flops) / its event time, against the
    measured HBM copy rate or the measured FMA rate of its arithmetic type,
    whichever bounds it by the algorithmic count."""
    if not stats:
        return None
    top = max(stats, key=lambda s: s["ms"])
    gbs = top["bytes"] / (top["ms"] * 1e6)
    gflops = top["flops"] / (top["ms"] * 1e6)
    # the refinement residual and its norms compute in FP64 on both paths (the
    # combination computes in double-single arithmetic, on the FP32 pipe)
    cls = top["name"].split("@")[0]
    fp64_kernel = cls in FP64_CLASSES or (precision == "fp64" and cls not in DS_CLASSES)
    alu_peak, alu_src = alu["fp64" if fp64_kernel else "fp32"]
    fh, fa = gbs / hbm, gflops / alu_peak
    tr = traffic_for(top["name"], precision)
    if fa > fh:
        r = {"bound": "alu", "achieved": gflops / 1e3, "peak": alu_peak / 1e3, "unit": "TFLOP/s", "frac": fa,
             "peak_source": ("FP64" if fp64_kernel else "FP32") + " FMA rate " + alu_src}
    else:
        r = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": fh,
             "peak_source": f"{hbm_src} MEASURED_PEAKS.json hbm_gbs"}
    r.update({"traffic": tr, "kernel": top["name"], "launches": top["launches"],
              "ms_per_launch": top["ms"] / top["launches"], "bytes_per_launch": top["bytes"] / top["launches"],
              "share_of_profiled_time": top["ms"] / sum(s["ms"] for s in stats),
              "achieved_gbs": gbs, "achieved_gflops": gflops, "hbm_frac": fh})
    return r


def measure(solver, target, steps, warmup, stream, torch, barrier, maxall, only=-1, clocks=False, profile=True):
    """Warm-up, then `steps` device-timed steps of one solver; optionally the
    nvidia-smi clock record of the timed region, a per-kernel-class profile pass
    and each component timed alone."""
    out = solver._bench_out
    for _ in range(warmup):
        if only < 0:
            solver.solve_combine(target[0], target[1], out, sync=False)
        else:
            solver.solve(only, sync=False)
    if only < 0:
        _, info = solver.solve_combine(target[0], target[1], out, sync=True)
    else:
        info = solver.solve(only, sync=True)
    barrier()
    l0 = solver.kernel_launches
    ck = Clocks() if clocks else None
    if ck:
        ck.start()
    ms = timed_steps(solver, out, target, steps, stream, torch, only)
    launches = (solver.kernel_launches - l0) // steps
    ck = ck.stop(getattr(torch.cuda.get_device_properties(out.device), "pci_bus_id", None)) if ck else None
    barrier()
    ms = maxall(ms)
    stats = comp_ms = None
    if profile:
        solver.profile(True)
        solver.solve(only, sync=False)
        if only < 0:
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
    return dict(ms=ms, launches=launches, clocks=ck, stats=stats, comp_ms=comp_ms, sweeps=info.sweeps,
                inner_iters=info.max_inner_iters, backward_error=info.backward_error,
                rel_residual=info.rel_residual)


def compact_roofline(r):
    """The roofline keys of the JSON line (the full entry goes to the detail file)."""
    if r is None:
        return None
    out = {k: r[k] for k in ("bound", "unit", "traffic", "kernel") if k in r}
    for k in ("achieved", "peak", "frac"):
        out[k] = sig(r[k])
    return out


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
    if args.target:
        target = tuple(int(v) for v in args.target.split(","))
    problem = factory()
    stream = torch.cuda.Stream(device=dev)
    hbm, hbm_src = peaks()
    with torch.cuda.stream(stream):
        alu = alu_peaks()
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
                            max_direct_rows=args.max_direct_rows, device_loop=args.device_loop or 0)
            setup_s = time.perf_counter() - t0
            solver._bench_out = out
            r = measure(solver, target, args.steps, args.warmup, stream, torch, barrier, maxall,
                        only=args.only_component, clocks=(prec == args.precision), profile="profile" not in skip)
            r.update(value=solver.total_dofs * world / (r["ms"] / 1e3), dofs=solver.total_dofs, setup_s=setup_s,
                     solver=solver)
            results[prec] = r
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
               "phases_s": {k: round(v, 4) for k, v in zip(("setup", "solve_combine", "copy_to_host", "release"),
                                                           phase)}}
    for r in results.values():
        r["solver"].close()
    del out, host_out
    torch.cuda.empty_cache()

    # the other single-GPU configurations, compact: the 3D random medium (FP32 + FP64
    # refinement, its stated precision) and the 64-instance batch
    subs = {}
    if "cfg3" not in skip and args.only_component < 0:
        subs["cfg3"] = sub_3d(args, stream, torch, barrier, maxall, hbm, hbm_src, alu, world)
    if "batch64" not in skip and world == 1:
        subs["batch64"] = batch_measure(args, steps=2, warmup=1, compact=True)
    if rank != 0:
        return
    cpu = None if "cpu" in skip else cpu_baseline(args.workload)
    rl = roofline(head["stats"], hbm, hbm_src, args.precision, alu)
    ck = head["clocks"] or {}
    line = {
        "metric": METRIC, "value": sig(head["value"]), "unit": "DOFs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sig(head["ms"]), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "target": list(target), "dofs": head["dofs"],
                   "l2": "target grid written each step > L2", "device_loop": args.device_loop or 0},
        "gpu_launches": head["launches"],
        "clocks": {"sm_mhz": ck.get("sm_mhz"), "sm_max_mhz": ck.get("sm_max_mhz"), "reasons": ck.get("reasons")},
        "roofline": compact_roofline(rl),
        "cpu_baseline": None if cpu is None else {
            "value": sig(cpu["value"]), "unit": cpu["unit"], "cores": cpu["cores"], "kind": "oracle",
            "sample": cpu["sample_short"]},
        "e2e": None if e2e is None else {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step",
                                                            "d2h_bytes_per_step")},
        "backward_error": sig(head["backward_error"], 2), "sweeps": head["sweeps"], "inner_iters": head["inner_iters"],
    }
    if line["e2e"]:
        line["e2e"]["value"] = sig(line["e2e"]["value"])
    for prec, r in results.items():
        if prec == args.precision:
            continue
        rr = roofline(r["stats"], hbm, hbm_src, prec, alu)
        line[prec] = {"value": sig(r["value"]), "ms_per_step": sig(r["ms"]), "backward_error": sig(r["backward_error"], 2),
                      "sweeps": r["sweeps"], "inner_iters": r["inner_iters"],
                      "roofline_frac": sig(rr["frac"], 3) if rr else None}
    for name, sub in subs.items():
        line[name] = {"value": sig(sub["value"]), "ms_per_step": sig(sub["ms_per_step"]),
                      "backward_error": sig(sub["backward_error"], 2)}
    detail = {"line": line, "setup_s": {p: r["setup_s"] for p, r in results.items()},
              "roofline_full": {p: roofline(r["stats"], hbm, hbm_src, p, alu) for p, r in results.items()},
              "kernels": {p: r["stats"] for p, r in results.items()},
              "components_alone_ms": {p: r["comp_ms"] for p, r in results.items()},
              "cpu_baseline": cpu, "e2e": e2e, "alu_peaks": alu, "subresults": subs,
              "clocks": head["clocks"], "launches": {p: r["launches"] for p, r in results.items()}}
    try:
        from paper_2606_09688_gb300.st import tuned_shapes
        detail["tuned_shapes"] = tuned_shapes()
    except Exception as e:  # diagnostics only
        detail["tuned_shapes"] = str(e)
    write_detail(detail)
    print(json.dumps(line, separators=(",", ":")), flush=True)


def sig(x, digits=4):
    """x rounded to `digits` significant figures (None stays None)."""
    if x is None:
        return None
    return float(f"{x:.{digits}g}")


def write_detail(detail):
    """Per-kernel tables and per-component times beside the JSON line (the
    line itself stays short enough to be read whole)."""
    d = os.path.join(ROOT, "gpurun_out")
    try:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "bench_detail.json"), "w") as f:
            json.dump(detail, f, indent=1, default=str)
    except OSError as e:
        print(f"bench: detail not written: {e}", file=sys.stderr)


def sub_3d(args, stream, torch, barrier, maxall, hbm, hbm_src, alu, world):
    """The 3D random-medium configuration (n = 10, m = 3, target (7,7)) in its
    stated precision, FP32 bulk with FP64 refinement: compact figures."""
    from paper_2606_09688_gb300 import ST_FP32_IR, Solver
    factory, target, _ = WORKLOADS["random_medium_3d_n10"]
    problem = factory()
    out = torch.empty(((1 << target[1]) + 1, ((1 << target[0]) + 1) ** 3), dtype=torch.float64,
                      device=torch.cuda.current_device())
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        solver = Solver(problem, precision=ST_FP32_IR, stream=stream)
        setup_s = time.perf_counter() - t0
        solver._bench_out = out
        r = measure(solver, target, min(args.steps, 5), 2, stream, torch, barrier, maxall, profile=True)
        dofs = solver.total_dofs
        solver.close()
    del out
    torch.cuda.empty_cache()
    rl = roofline(r["stats"], hbm, hbm_src, "fp32ir", alu)
    return {"workload": "random_medium_3d_n10", "precision": "fp32ir", "target": list(target),
            "space_time_dofs": dofs, "value": dofs * world / (r["ms"] / 1e3), "ms_per_step": r["ms"],
            "steps": min(args.steps, 5), "warmup": 2, "backward_error": r["backward_error"],
            "setup_s": round(setup_s, 2), "gpu_launches": r["launches"], "roofline": compact_roofline(rl)}


def batch_measure(args, steps, warmup, compact=False):
    """Batching configuration: 64 independent 2D instances (levels n in 8..12,
    random smooth c^2 in [0.5, 2] with a jump, random Gaussian sources), all
    components of all instances solved together by st_solve_batch.  Value =
    space-time DOFs of all instances per second of the batch solve (combination
    excluded: each instance's own target grid would total ~120 GB)."""
    import torch
    from paper_2606_09688_gb300 import ST_FP32_IR, ST_FP64, Solver, solve_batch
    code = ST_FP64 if (args.precision == "fp64" and not compact) else ST_FP32_IR
    probs = W.batch_instances(64)
    t0 = time.perf_counter()
    dl = 4 if args.device_loop is None else args.device_loop
    solvers = [Solver(p, precision=code, inner_tol=args.inner_tol, max_direct_rows=args.max_direct_rows,
                      device_loop=dl) for p in probs]
    setup_s = time.perf_counter() - t0
    dofs = sum(s.total_dofs for s in solvers)
    for _ in range(warmup):
        solve_batch(solvers)
    torch.cuda.synchronize()
    times = []
    info = None
    for _ in range(steps):
        t0 = time.perf_counter()
        info = solve_batch(solvers)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    levels = {}
    for p in probs:
        levels[p.J + 2 * p.mx] = levels.get(p.J + 2 * p.mx, 0) + 1
    for s in solvers:
        s.close()
    torch.cuda.empty_cache()
    res = {"value": dofs / (ms / 1e3), "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "precision": "fp64" if code == ST_FP64 else "fp32ir", "instances": len(probs), "space_time_dofs": dofs,
           "backward_error": info.backward_error, "setup_s": round(setup_s, 2),
           "timing": "host wall clock around st_solve_batch (blocking)",
           "solves": f"one CUDA graph per component, {dl} COCG iterations per device test, one host sync per batch"
           if dl else "host-driven"}
    if compact:
        return res
    res["levels_n"] = levels
    return res


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    r = batch_measure(args, args.steps, args.warmup)
    line = {"metric": METRIC, "value": r["value"], "unit": "DOFs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if r["precision"] == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "batch64", "instances": r["instances"], "levels_n": r["levels_n"],
                       "space_time_dofs": r["space_time_dofs"], "timing": r["timing"], "combination": "excluded"},
            "setup_s": r["setup_s"], "backward_error": r["backward_error"]}
    print(json.dumps(line, separators=(",", ":")), flush=True)


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
