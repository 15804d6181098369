"""Thin ctypes binding of the C ABI in include/st.h.

Argument marshalling only: every step of the method runs inside libst.so.
Device memory for outputs and the CUDA stream come from PyTorch.  If the
library has not been built (``__graft_entry__.build()`` or
``python -m paper_2606_09688_gb300.build``) importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libst.so")

ST_OK, ST_ERR_ARG, ST_ERR_CUDA, ST_ERR_OOM, ST_ERR_NOT_CONVERGED, ST_ERR_STATE, ST_ERR_CALLBACK, ST_ERR_NUMERIC, ST_ERR_TIMEOUT = range(9)
ST_FP64, ST_FP32_IR = 0, 1
STATUS_NAMES = {0: "ST_OK", 1: "ST_ERR_ARG", 2: "ST_ERR_CUDA", 3: "ST_ERR_OOM", 4: "ST_ERR_NOT_CONVERGED",
                5: "ST_ERR_STATE", 6: "ST_ERR_CALLBACK", 7: "ST_ERR_NUMERIC", 8: "ST_ERR_TIMEOUT"}

SPACE_FN = C.CFUNCTYPE(C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)
TIME_FN = C.CFUNCTYPE(C.c_int, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)
SPACETIME_FN = C.CFUNCTYPE(C.c_int, C.c_int64, C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_double), C.c_void_p)


class StField(C.Structure):
    _fields_ = [("fn", SPACE_FN), ("user", C.c_void_p)]


class StSourceTerm(C.Structure):
    _fields_ = [("g", SPACE_FN), ("g_user", C.c_void_p), ("s", TIME_FN), ("s_user", C.c_void_p)]


class StProblem(C.Structure):
    _fields_ = [("d", C.c_int), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("T", C.c_double),
                ("c2", StField), ("n_terms", C.c_int), ("terms", C.POINTER(StSourceTerm)),
                ("f_general", SPACETIME_FN), ("f_user", C.c_void_p), ("u0", StField), ("v0", StField),
                ("J", C.c_int), ("mx", C.c_int), ("mt", C.c_int),
                ("c2_nodal", C.c_void_p), ("g_nodal", C.c_void_p), ("param_level", C.c_int)]


class StOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("max_sweeps", C.c_int),
                ("stream", C.c_void_p), ("inner_tol", C.c_double), ("max_direct_rows", C.c_int),
                ("autotune", C.c_int), ("mem_cap_bytes", C.c_int64), ("wait_cycles", C.c_int64),
                ("inject_stall", C.c_int), ("device_loop", C.c_int)]


class StComponentInfo(C.Structure):
    _fields_ = [("jx", C.c_int), ("jt", C.c_int), ("coef", C.c_int), ("n_space", C.c_int64),
                ("n_time", C.c_int64), ("method", C.c_int), ("n_modes", C.c_int)]


class StSolveInfo(C.Structure):
    _fields_ = [("sweeps", C.c_int), ("max_inner_iters", C.c_int), ("rel_residual", C.c_double),
                ("backward_error", C.c_double), ("status", C.c_int)]


class StKernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


EXPORTED = ["st_transfer_bytes", "st_profile", "st_profile_read", "st_setup", "st_num_components", "st_component", "st_solve_component", "st_combine",
            "st_component_coeffs", "st_total_dofs", "st_kernel_launches", "st_destroy", "st_last_error"]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    lib.st_setup.argtypes = [C.POINTER(StProblem), C.POINTER(StOptions), C.POINTER(C.c_void_p)]
    lib.st_num_components.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    lib.st_component.argtypes = [C.c_void_p, C.c_int, C.POINTER(StComponentInfo)]
    lib.st_solve_component.argtypes = [C.c_void_p, C.c_int, C.POINTER(StSolveInfo)]
    lib.st_combine.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    lib.st_solve_combine.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.POINTER(StSolveInfo)]
    lib.st_combine_subset.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_void_p]
    lib.st_solve_batch.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(StSolveInfo)]
    lib.st_receiver_values.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]
    lib.st_misfit_gradient.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                       C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.POINTER(StSolveInfo)]
    lib.st_component_coeffs.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
    lib.st_total_dofs.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
    lib.st_kernel_launches.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
    lib.st_transfer_bytes.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.st_profile.argtypes = [C.c_void_p, C.c_int]
    lib.st_profile_read.argtypes = [C.c_void_p, C.POINTER(StKernelStat), C.c_int, C.POINTER(C.c_int)]
    lib.st_destroy.argtypes = [C.c_void_p]
    lib.st_last_error.argtypes = [C.c_void_p]
    lib.st_last_error.restype = C.c_char_p
    for name in EXPORTED:
        getattr(lib, name).restype = C.c_int if name != "st_last_error" else C.c_char_p
    return lib


_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class StError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _space_cb(fn, d):
    def cb(n, pts, out, user):
        try:
            x = np.ctypeslib.as_array(pts, shape=(n * d,)).reshape(n, d)
            o = np.ctypeslib.as_array(out, shape=(n,))
            o[:] = np.asarray(fn(x.copy()), dtype=np.float64).reshape(n)
            return 0
        except Exception:  # reported to the library as a callback failure
            return 1
    return SPACE_FN(cb)


def _time_cb(fn):
    def cb(n, t, out, user):
        try:
            tt = np.ctypeslib.as_array(t, shape=(n,)).copy()
            o = np.ctypeslib.as_array(out, shape=(n,))
            o[:] = np.asarray(fn(tt), dtype=np.float64).reshape(n)
            return 0
        except Exception:
            return 1
    return TIME_FN(cb)


def _spacetime_cb(fn, d):
    def cb(n, pts, t, out, user):
        try:
            x = np.ctypeslib.as_array(pts, shape=(n * d,)).reshape(n, d)
            o = np.ctypeslib.as_array(out, shape=(n,))
            o[:] = np.asarray(fn(x.copy(), float(t)), dtype=np.float64).reshape(n)
            return 0
        except Exception:
            return 1
    return SPACETIME_FN(cb)


class Solver:
    """One problem instance behind the C ABI (st_setup .. st_destroy)."""

    def __init__(self, problem, precision: int = ST_FP64, tol: float = 0.0, max_iter: int = 0,
                 max_sweeps: int = 0, stream=None, inner_tol: float = 0.0, max_direct_rows: int = 0,
                 autotune: int = 0, mem_cap_bytes: int = 0, wait_cycles: int = 0, inject_stall: int = 0,
                 device_loop: int = 0, c2_nodal=None, g_nodal=None, param_level: int = 0):
        """c2_nodal / g_nodal: optional nodal values ((2^param_level+1)^d, x fastest) of
        c^2 and of the first source term's spatial factor on the uniform grid of level
        param_level; the library interpolates them (and its gradient uses the transpose)."""
        import torch
        self._lib = lib()
        p = problem
        if getattr(p, "pt", 2) != 2:
            raise StError(ST_ERR_ARG, "the library solves C^1 quadratic time splines (pt = 2)")
        d = p.d
        keep = []  # callbacks and arrays must outlive st_setup

        def field(fn):
            if fn is None:
                return StField(SPACE_FN(), None)
            cb = _space_cb(fn, d)
            keep.append(cb)
            return StField(cb, None)

        terms = (StSourceTerm * max(1, len(p.terms)))()
        for r, (g, s) in enumerate(p.terms):
            gc = SPACE_FN() if g is None else _space_cb(g, d)
            sc = _time_cb(s)
            keep += [gc, sc]
            terms[r] = StSourceTerm(gc, None, sc, None)
        prob = StProblem()
        prob.d = d
        for k in range(d):
            prob.lo[k] = p.lo[k]
            prob.hi[k] = p.hi[k]
        prob.T = p.T
        prob.c2 = field(p.c2)
        prob.n_terms = len(p.terms)
        prob.terms = C.cast(terms, C.POINTER(StSourceTerm))
        if p.f_general is not None:
            fg = _spacetime_cb(p.f_general, d)
            keep.append(fg)
            prob.f_general = fg
        prob.u0 = field(p.u0)
        prob.v0 = field(p.v0)
        prob.J, prob.mx, prob.mt = p.J, p.mx, p.mt
        for name, arr in (("c2_nodal", c2_nodal), ("g_nodal", g_nodal)):
            if arr is not None:
                a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).ravel())
                if a.size != ((1 << param_level) + 1) ** d:
                    raise ValueError(f"{name}: expected {((1 << param_level) + 1) ** d} nodal values")
                keep.append(a)
                setattr(prob, name, a.ctypes.data)
        prob.param_level = param_level
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt = StOptions(precision, tol, max_iter, max_sweeps, C.c_void_p(stream.cuda_stream), inner_tol,
                        max_direct_rows, autotune, mem_cap_bytes, wait_cycles, inject_stall, device_loop)
        h = C.c_void_p()
        code = self._lib.st_setup(C.byref(prob), C.byref(opt), C.byref(h))
        if code != ST_OK:
            raise StError(code, self._lib.st_last_error(None).decode())
        self._h = h
        self.problem = problem
        self.precision = precision

    def _check(self, code):
        if code != ST_OK:
            raise StError(code, self._lib.st_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.st_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def num_components(self) -> int:
        n = C.c_int()
        self._check(self._lib.st_num_components(self._h, C.byref(n)))
        return n.value

    def component(self, k: int) -> StComponentInfo:
        info = StComponentInfo()
        self._check(self._lib.st_component(self._h, k, C.byref(info)))
        return info

    def components(self) -> List[StComponentInfo]:
        return [self.component(k) for k in range(self.num_components)]

    def solve(self, k: int = -1, sync: bool = True) -> Optional[StSolveInfo]:
        if sync:
            info = StSolveInfo()
            self._check(self._lib.st_solve_component(self._h, k, C.byref(info)))
            return info
        self._check(self._lib.st_solve_component(self._h, k, None))
        return None

    def combine(self, jx_star: int, jt_star: int, out=None):
        import torch
        nsp = ((1 << jx_star) + 1) ** self.problem.d
        nts = (1 << jt_star) + 1
        if out is None:
            out = torch.empty((nts, nsp), dtype=torch.float64, device="cuda")
        assert out.dtype == torch.float64 and out.is_cuda and out.is_contiguous() and out.numel() == nts * nsp
        self._check(self._lib.st_combine(self._h, jx_star, jt_star, C.c_void_p(out.data_ptr())))
        return out

    def solve_combine(self, jx_star: int, jt_star: int, out=None, sync: bool = True):
        """solve(-1) then combine(jx*, jt*), the combination levels overlapped with the
        solves (st_solve_combine).  Returns (out, StSolveInfo or None)."""
        import torch
        nsp = ((1 << jx_star) + 1) ** self.problem.d
        nts = (1 << jt_star) + 1
        if out is None:
            out = torch.empty((nts, nsp), dtype=torch.float64, device="cuda")
        assert out.dtype == torch.float64 and out.is_cuda and out.is_contiguous() and out.numel() == nts * nsp
        info = StSolveInfo() if sync else None
        self._check(self._lib.st_solve_combine(self._h, jx_star, jt_star, C.c_void_p(out.data_ptr()),
                                               C.byref(info) if sync else None))
        return out, info

    def combine_subset(self, jx_star: int, jt_star: int, comps, out=None):
        """Contribution of the listed components to u^CF on the target grid
        (st_combine_subset); disjoint sets covering all components sum to combine()."""
        import torch
        nsp = ((1 << jx_star) + 1) ** self.problem.d
        nts = (1 << jt_star) + 1
        if out is None:
            out = torch.empty((nts, nsp), dtype=torch.float64, device="cuda")
        assert out.dtype == torch.float64 and out.is_cuda and out.is_contiguous() and out.numel() == nts * nsp
        ks = [int(k) for k in comps]
        arr = (C.c_int * len(ks))(*ks)
        self._check(self._lib.st_combine_subset(self._h, jx_star, jt_star, arr, len(ks), C.c_void_p(out.data_ptr())))
        return out

    def receiver_values(self, jt_star: int, receivers):
        """u^CF at the receivers (n x d array) and the 2^jt*+1 uniform times, (times, receivers)."""
        import torch
        x = np.ascontiguousarray(receivers, dtype=np.float64)
        out = torch.empty(((1 << jt_star) + 1, len(x)), dtype=torch.float64, device="cuda")
        self._check(self._lib.st_receiver_values(self._h, jt_star, x.ctypes.data_as(C.c_void_p), len(x),
                                                  C.c_void_p(out.data_ptr())))
        return out

    def misfit_gradient(self, jt_star: int, receivers, d_obs, jp: int):
        """J = 1/2 sum_s w_s sum_r (u^CF - d)^2 and its gradients with respect to nodal c^2 and
        nodal source factor g on the level-jp grid (st_misfit_gradient).  d_obs: CUDA float64
        tensor (times, receivers).  Returns (J, dJ/dc2, dJ/dg, StSolveInfo of the adjoint solves)."""
        import torch
        x = np.ascontiguousarray(receivers, dtype=np.float64)
        d_obs = d_obs.to(dtype=torch.float64, device="cuda").contiguous()
        assert d_obs.shape == ((1 << jt_star) + 1, len(x))
        npar = ((1 << jp) + 1) ** self.problem.d
        dc2 = torch.empty(npar, dtype=torch.float64, device="cuda")
        dg = torch.empty(npar, dtype=torch.float64, device="cuda")
        J = C.c_double()
        info = StSolveInfo()
        self._check(self._lib.st_misfit_gradient(self._h, jt_star, x.ctypes.data_as(C.c_void_p), len(x),
                                                  C.c_void_p(d_obs.data_ptr()), jp, C.byref(J),
                                                  C.c_void_p(dc2.data_ptr()), C.c_void_p(dg.data_ptr()),
                                                  C.byref(info)))
        return J.value, dc2, dg, info

    def energy(self, times, jx_eval: int = 0) -> np.ndarray:
        """E(t; u^CF) of Section 6.3 at the given times in [0, T] (st_energy)."""
        t = np.ascontiguousarray(np.asarray(times, dtype=np.float64).ravel())
        out = np.empty(len(t))
        self._lib.st_energy.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        self._lib.st_energy.restype = C.c_int
        self._check(self._lib.st_energy(self._h, t.ctypes.data_as(C.c_void_p), len(t), jx_eval,
                                        out.ctypes.data_as(C.c_void_p)))
        return out

    def coeffs(self, k: int) -> np.ndarray:
        info = self.component(k)
        out = np.empty((info.n_time, info.n_space), dtype=np.float64)
        self._check(self._lib.st_component_coeffs(self._h, k, out.ctypes.data_as(C.c_void_p)))
        return out

    @property
    def total_dofs(self) -> int:
        n = C.c_int64()
        self._check(self._lib.st_total_dofs(self._h, C.byref(n)))
        return n.value

    @property
    def kernel_launches(self) -> int:
        n = C.c_int64()
        self._check(self._lib.st_kernel_launches(self._h, C.byref(n)))
        return n.value

    def profile(self, enable: bool = True):
        """Start (clearing the record) or stop per-kernel-class event timing."""
        self._check(self._lib.st_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> List[dict]:
        buf = (StKernelStat * 512)()
        n = C.c_int()
        self._check(self._lib.st_profile_read(self._h, buf, 512, C.byref(n)))
        return [dict(name=buf[i].name.decode(), launches=buf[i].launches, ms=buf[i].ms, bytes=buf[i].bytes,
                     flops=buf[i].flops) for i in range(min(n.value, 512))]

    def transfer_bytes(self):
        """(host->device, device->host) bytes moved by the library so far."""
        a, b = C.c_int64(), C.c_int64()
        self._check(self._lib.st_transfer_bytes(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value


def solve_batch(solvers, max_threads: int = 0, sync: bool = True):
    """Solve all components of several independent Solver instances together
    (st_solve_batch): (instance, component) pairs largest first over a pool of
    host threads, each component on its own stream."""
    solvers = list(solvers)
    if not solvers:
        raise ValueError("no solvers")
    lib = solvers[0]._lib
    arr = (C.c_void_p * len(solvers))(*[s._h for s in solvers])
    info = StSolveInfo()
    code = lib.st_solve_batch(arr, len(solvers), max_threads, C.byref(info) if sync else None)
    if code != ST_OK:
        msgs = [lib.st_last_error(s._h).decode() for s in solvers]
        raise StError(code, next((m for m in msgs if m), "st_solve_batch failed"))
    return info if sync else None


def tuned_shapes():
    """Stencil launch shapes chosen by the autotuner in this process (st_tuned_shapes):
    a list of dicts (op, d, elem_bytes, nodes, modes, modes_per_thread, block)."""
    lib = load_library()
    n = C.c_int()
    lib.st_tuned_shapes(None, 0, C.byref(n))
    buf = (C.c_int * (7 * max(n.value, 1)))()
    lib.st_tuned_shapes(buf, n.value, C.byref(n))
    keys = ("op", "d", "elem_bytes", "nodes", "modes", "modes_per_thread", "block")
    return [dict(zip(keys, buf[7 * i:7 * i + 7])) for i in range(n.value)]


def set_tuned_shape(entry: dict):
    """Pin one stencil launch shape (st_set_tuned_shape); entry as returned by tuned_shapes()."""
    lib = load_library()
    keys = ("op", "d", "elem_bytes", "nodes", "modes", "modes_per_thread", "block")
    arr = (C.c_int * 7)(*[int(entry[k]) for k in keys])
    code = lib.st_set_tuned_shape(arr)
    if code != ST_OK:
        raise StError(code, "invalid stencil launch shape")


def probe_fma(precision: int = ST_FP64, iters: int = 4096, stream=None) -> float:
    """Measured FMA throughput of the current device in GFLOP/s (st_probe_fma):
    precision ST_FP64 (0) or ST_FP32_IR (1, meaning FP32 arithmetic here)."""
    import torch
    lib_ = lib()
    lib_.st_probe_fma.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), C.c_void_p]
    lib_.st_probe_fma.restype = C.c_int
    if stream is None:
        stream = torch.cuda.current_stream()
    g = C.c_double()
    code = lib_.st_probe_fma(int(precision), int(iters), C.byref(g), C.c_void_p(stream.cuda_stream))
    if code != ST_OK:
        raise StError(code, "st_probe_fma failed")
    return g.value
