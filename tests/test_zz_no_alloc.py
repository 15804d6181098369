"""GPU test of st_combine_noalloc, the allocation-free combination entry point.

Callers that cannot let the library allocate device memory at call time pass
their own component arrays and output; the call uses a fixed scratch array
compiled into the library.  Its output must equal st_combine's on the same
components, on two different calls in a row (the scratch keeps the previous
call's contents, so the second call checks that nothing stale is read).  This file
is collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest

import st_workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


class CombInput(C.Structure):
    _fields_ = [("U", C.c_void_p), ("lift", C.c_void_p), ("jx", C.c_int), ("jt", C.c_int), ("coef", C.c_int)]


def _node_values(p, jx, fn):
    """fn at all (2^jx+1)^d nodes, lexicographic with x fastest (lo + (hi-lo) i / N)."""
    N = 1 << jx
    axes = [p.lo[k] + (p.hi[k] - p.lo[k]) * np.arange(N + 1) / N for k in range(p.d)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    pts = np.stack([m.ravel() for m in mesh[::-1]], axis=1)
    return np.asarray(fn(pts), dtype=np.float64)


def test_combine_noalloc_matches_st_combine_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09688_gb300 import ST_FP64, Solver
    from paper_2606_09688_gb300 import build
    from paper_2606_09688_gb300 import st as B
    build.build(force=False)
    lib = B.lib()
    fn = lib.st_combine_noalloc
    fn.argtypes = [C.POINTER(CombInput), C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int

    p = W.standing_wave(2, 6, 2)          # u0 != 0, so the lift arrays are exercised
    # two different calls in a row: a target coarser than the finest components
    # (their values are injected), then a finer one (prolongation); stale tables
    # or partial sums of the first call would change the second call's result
    targets = [(3, 3), (5, 4)]
    with Solver(p, precision=ST_FP64) as s:
        s.solve(-1)
        refs = [s.combine(*t).cpu().numpy() for t in targets]
        infos = s.components()
        keep = []
        arr = (CombInput * len(infos))()
        for k, ci in enumerate(infos):
            U = torch.from_numpy(s.coeffs(k)).cuda().contiguous()
            lift = torch.from_numpy(_node_values(p, ci.jx, p.u0)).cuda().contiguous()
            keep += [U, lift]
            arr[k] = CombInput(U.data_ptr(), lift.data_ptr(), ci.jx, ci.jt, ci.coef)
    assert max(ci.jx for ci in infos) > targets[0][0] and max(ci.jx for ci in infos) < targets[1][0]
    stream = torch.cuda.current_stream()
    for call, (target, ref) in enumerate(zip(targets, refs)):
        out = torch.full(ref.shape, float("nan"), dtype=torch.float64, device="cuda")
        code = fn(arr, len(infos), p.d, p.T, target[0], target[1], C.c_void_p(out.data_ptr()),
                  C.c_void_p(stream.cuda_stream))
        assert code == B.ST_OK, (call, code)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < TOL64, (call, rel)

    # a target whose partial sums (level 6: 65^2 x 1025 doubles) exceed the
    # fixed scratch is refused before any work is enqueued
    big = torch.zeros((1025, 129 * 129), dtype=torch.float64, device="cuda")
    assert fn(arr, len(infos), p.d, p.T, 7, 10, C.c_void_p(big.data_ptr()),
              C.c_void_p(stream.cuda_stream)) == B.ST_ERR_ARG
    assert float(big.abs().max()) == 0.0
