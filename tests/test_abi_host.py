"""CPU tests of the C ABI library: it builds, loads, exports every declared
symbol, and its host-side setup math matches the oracle (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest
import scipy.linalg as sla

import st_workloads as W
from oracle import combination, space, timemats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_09688_gb300 import build
    path = build.build(force=False)
    L = C.CDLL(path)
    L.st_host_time_matrices.argtypes = [C.c_int, C.c_double] + [C.c_void_p] * 4
    L.st_host_time_matrices_p.argtypes = [C.c_int, C.c_double, C.c_int] + [C.c_void_p] * 4
    L.st_host_time_eig_p.argtypes = [C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int), C.c_void_p,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.st_host_time_eig.argtypes = [C.c_int, C.c_double, C.POINTER(C.c_int), C.c_void_p, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]
    L.st_host_components.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p]
    L.st_host_sym_gen_eig.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return L


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def test_every_declared_symbol_is_exported(lib):
    names = set()
    for hdr in ("st.h", "st_host.h", "st_probe.h"):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(st_\w+)\s*\(", text))
    assert len(names) >= 14
    for n in sorted(names):
        assert hasattr(lib, n), n


@pytest.mark.parametrize("jt,T", [(0, 1.0), (1, 1.0), (3, 1.0), (5, 2.5), (7, 1.0)])
def test_time_matrices_match_oracle(lib, jt, T):
    nt = (1 << jt) + 1
    A, B = np.zeros((nt, nt)), np.zeros((nt, nt))
    g1, d0 = np.zeros(nt), np.zeros(nt)
    assert lib.st_host_time_matrices(jt, T, _ptr(A), _ptr(B), _ptr(g1), _ptr(d0)) == 0
    Ao, Bo = timemats.time_matrices(jt, T)
    assert np.allclose(A, Ao, rtol=1e-13, atol=1e-13 * np.abs(Ao).max())
    assert np.allclose(B, Bo, rtol=1e-13, atol=1e-13 * np.abs(Bo).max())
    assert np.allclose(g1, timemats.load_one(jt, T), atol=1e-14)
    assert np.allclose(d0, timemats.dpsi_at_zero(jt, T), atol=1e-12)


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("jt,T", [(0, 1.0), (2, 1.0), (4, 2.5), (6, 1.0)])
def test_degree_p_time_matrices_match_oracle(lib, p, jt, T):
    """The library's host set-up math for time splines of degree p (maximal
    regularity) against the oracle's (Cox-de Boor on the whole knot vector, pinned in
    tests/test_oracle_time_degree.py); p = 2 also equals the quadratic routine."""
    nt = (1 << jt) + p - 1
    A, B = np.zeros((nt, nt)), np.zeros((nt, nt))
    g1, d0 = np.zeros(nt), np.zeros(nt)
    assert lib.st_host_time_matrices_p(jt, T, p, _ptr(A), _ptr(B), _ptr(g1), _ptr(d0)) == 0
    Ao, Bo = timemats.time_matrices(jt, T, p)
    assert np.allclose(A, Ao, rtol=1e-13, atol=1e-13 * np.abs(Ao).max())
    assert np.allclose(B, Bo, rtol=1e-13, atol=1e-13 * np.abs(Bo).max())
    assert np.allclose(g1, timemats.load_one(jt, T, p), atol=1e-14)
    assert np.allclose(d0, timemats.dpsi_at_zero(jt, T, p), atol=1e-12)
    if p == 2:
        A2, B2 = np.zeros((nt, nt)), np.zeros((nt, nt))
        assert lib.st_host_time_matrices(jt, T, _ptr(A2), _ptr(B2), None, None) == 0
        assert np.allclose(A, A2, rtol=1e-14, atol=1e-14 * np.abs(A2).max())
        assert np.allclose(B, B2, rtol=1e-14, atol=1e-14 * np.abs(B2).max())
    A1 = np.zeros((nt, nt))
    for bad in ((jt, T, 1), (jt, T, 5), (jt, -1.0, p), (15, T, p)):
        assert lib.st_host_time_matrices_p(bad[0], bad[1], bad[2], _ptr(A1), _ptr(A1), None, None) == 1


@pytest.mark.parametrize("J,mx,mt", [(0, 1, 1), (3, 2, 1), (8, 2, 2)])
def test_component_list_matches_oracle(lib, J, mx, mt):
    out = np.zeros(3 * (2 * J + 1), dtype=np.int32)
    assert lib.st_host_components(J, mx, mt, _ptr(out)) == 0
    assert [tuple(r) for r in out.reshape(-1, 3)] == combination.components(J, mx, mt)


@pytest.mark.parametrize("jt", [1, 2, 4, 6])
def test_time_eigenvalues_match_numpy(lib, jt):
    nt = (1 << jt) + 1
    lam = np.zeros(2 * nt)
    nsel, cond, res = C.c_int(), C.c_double(), C.c_double()
    assert lib.st_host_time_eig(jt, 1.0, C.byref(nsel), _ptr(lam), C.byref(cond), C.byref(res)) == 0
    got = lam[:2 * nsel.value].reshape(-1, 2)
    got = got[:, 0] + 1j * got[:, 1]
    A, B = timemats.time_matrices(jt, 1.0)
    ref = np.linalg.eigvals(np.linalg.solve(B, A))
    full = np.concatenate([got, np.conj(got[np.abs(got.imag) > 0])])
    assert len(full) == nt
    scale = np.abs(ref).max()
    for z in ref:
        assert np.min(np.abs(full - z)) < 1e-9 * scale
    assert res.value < 1e-12
    assert cond.value < 1e7


@pytest.mark.parametrize("p", [3, 4])
@pytest.mark.parametrize("jt", [1, 3, 5])
def test_degree_p_time_eigenvalues_match_numpy(lib, p, jt):
    """The time eigenbasis of the degree-p splines: every eigenvalue of B^{-1} A of the
    oracle's matrices, one of each conjugate pair kept, small residual.  The eigenvalues
    are only determined to about cond(V) eps ||C|| (Bauer-Fike), so the tolerance grows
    with the routine's condition estimate (3e8 for p = 4 at jt = 5)."""
    nt = (1 << jt) + p - 1
    lam = np.zeros(2 * nt)
    nsel, cond, res = C.c_int(), C.c_double(), C.c_double()
    assert lib.st_host_time_eig_p(jt, 1.0, p, C.byref(nsel), _ptr(lam), C.byref(cond), C.byref(res)) == 0
    got = lam[:2 * nsel.value].reshape(-1, 2)
    got = got[:, 0] + 1j * got[:, 1]
    A, B = timemats.time_matrices(jt, 1.0, p)
    ref = np.linalg.eigvals(np.linalg.solve(B, A))
    full = np.concatenate([got, np.conj(got[np.abs(got.imag) > 0])])
    assert len(full) == nt
    tol = max(1e-9, 100 * cond.value * np.finfo(float).eps) * np.abs(ref).max()
    for z in ref:
        assert np.min(np.abs(full - z)) < tol
    assert res.value < 1e-12
    assert lib.st_host_time_eig_p(jt, 1.0, 5, C.byref(nsel), _ptr(lam), None, None) == 1


def test_generalised_symmetric_eig_matches_scipy(lib):
    p = W.layered_2d(6, 3)
    sm = space.space_matrices(p, 3)
    K, M = sm["K"].toarray(), sm["M"].toarray()
    n = K.shape[0]
    mu, Phi = np.zeros(n), np.zeros((n, n))
    assert lib.st_host_sym_gen_eig(n, _ptr(np.ascontiguousarray(K)), _ptr(np.ascontiguousarray(M)),
                                   _ptr(mu), _ptr(Phi)) == 0
    assert np.allclose(np.sort(mu), sla.eigh(K, M, eigvals_only=True), rtol=1e-10)
    assert np.allclose(Phi.T @ M @ Phi, np.eye(n), atol=1e-10)
    assert np.allclose(Phi.T @ K @ Phi, np.diag(mu), atol=1e-8 * mu.max())


def test_setup_rejects_bad_arguments_without_touching_the_gpu():
    from paper_2606_09688_gb300 import st as B
    L = B.lib()
    prob = B.StProblem()
    prob.d = 4
    h = C.c_void_p()
    assert L.st_setup(C.byref(prob), None, C.byref(h)) == B.ST_ERR_ARG
    assert b"d must be" in L.st_last_error(None)
    prob.d = 2
    prob.hi[0] = prob.hi[1] = 1.0
    prob.T = 1.0
    prob.mx = 1
    assert L.st_setup(C.byref(prob), None, C.byref(h)) == B.ST_ERR_ARG   # no c^2 callback
    assert h.value is None


def test_setup_rejects_bad_tolerances_without_touching_the_gpu():
    from paper_2606_09688_gb300 import st as B
    L = B.lib()
    prob = B.StProblem()
    prob.d = 1
    prob.hi[0] = 1.0
    prob.T = 1.0
    prob.J = 2
    prob.mx = 1
    prob.mt = 1

    def c2(n, x, out, user):
        for i in range(n):
            out[i] = 1.0
        return 0
    cb = B.SPACE_FN(c2)
    prob.c2.fn = cb
    h = C.c_void_p()
    for tol, inner in ((-1e-3, 0.0), (1.5, 0.0), (0.0, -1.0), (0.0, 1.0), (0.0, float("nan"))):
        opt = B.StOptions(B.ST_FP64, tol, 0, 0, None, inner, 0, 0)
        assert L.st_setup(C.byref(prob), C.byref(opt), C.byref(h)) == B.ST_ERR_ARG
        assert b"tolerances" in L.st_last_error(None)
        assert h.value is None


def test_sym_gen_eig_on_a_2d_q1_pencil_with_variable_coefficient():
    """Generalised eigenproblem of a 15^2-node Q1 stiffness (variable diagonal
    scaling) and mass: eigenvalues against LAPACK, M-orthonormal eigenvectors
    that diagonalise K."""
    import scipy.linalg as sla
    from paper_2606_09688_gb300 import st as B
    lib = B.lib()
    n1 = 15
    n = n1 * n1
    h = 1.0 / (n1 + 1)
    T = np.diag(2 * np.ones(n1)) - np.diag(np.ones(n1 - 1), 1) - np.diag(np.ones(n1 - 1), -1)
    M1 = (h / 6) * (np.diag(4 * np.ones(n1)) + np.diag(np.ones(n1 - 1), 1) + np.diag(np.ones(n1 - 1), -1))
    K = np.kron(T / h, M1) + np.kron(M1, T / h)
    M = np.kron(M1, M1)
    D = np.diag(np.random.default_rng(0).uniform(0.5, 2.0, n))
    K = D @ K @ D
    mu = np.zeros(n)
    Phi = np.zeros((n, n))
    assert lib.st_host_sym_gen_eig(n, _ptr(np.ascontiguousarray(K)), _ptr(np.ascontiguousarray(M)),
                                   _ptr(mu), _ptr(Phi)) == 0
    ref = sla.eigh(K, M, eigvals_only=True)
    assert np.max(np.abs(np.sort(mu) - ref) / np.abs(ref)) < 1e-11
    assert np.max(np.abs(Phi.T @ M @ Phi - np.eye(n))) < 1e-12
    assert np.max(np.abs(Phi.T @ K @ Phi - np.diag(mu))) < 1e-12 * mu.max()


def test_setup_rejects_bad_solver_options_without_touching_the_gpu():
    from paper_2606_09688_gb300 import st as B
    L = B.lib()
    prob = B.StProblem()
    prob.d = 1
    prob.hi[0] = 1.0
    prob.T = 1.0
    prob.J = 2
    prob.mx = 1
    prob.mt = 1

    def c2(n, x, out, user):
        for i in range(n):
            out[i] = 1.0
        return 0
    cb = B.SPACE_FN(c2)
    prob.c2.fn = cb
    h = C.c_void_p()
    for max_direct, autotune, msg in ((-1, 0, b"max_direct_rows"), (0, 2, b"autotune"), (0, -2, b"autotune")):
        opt = B.StOptions(B.ST_FP64, 0.0, 0, 0, None, 0.0, max_direct, autotune)
        assert L.st_setup(C.byref(prob), C.byref(opt), C.byref(h)) == B.ST_ERR_ARG
        assert msg in L.st_last_error(None)
        assert h.value is None
    for cap, wait, stall in ((-1, 0, 0), (0, -5, 0), (0, 0, 2), (0, 0, -1)):
        opt = B.StOptions(B.ST_FP64, 0.0, 0, 0, None, 0.0, 0, 0, cap, wait, stall)
        assert L.st_setup(C.byref(prob), C.byref(opt), C.byref(h)) == B.ST_ERR_ARG
        assert b"inject_stall" in L.st_last_error(None)
        assert h.value is None
    for loop in (-1, 3, 32):
        opt = B.StOptions(B.ST_FP64, 0.0, 0, 0, None, 0.0, 0, 0, 0, 0, 0, loop)
        assert L.st_setup(C.byref(prob), C.byref(opt), C.byref(h)) == B.ST_ERR_ARG
        assert b"device_loop" in L.st_last_error(None)


def test_tuned_shape_pinning_validates_the_shape():
    from paper_2606_09688_gb300 import StError
    from paper_2606_09688_gb300.st import set_tuned_shape, tuned_shapes
    good = dict(op=2, d=2, elem_bytes=4, nodes=12345, modes=3, modes_per_thread=2, block=0)
    set_tuned_shape(good)
    assert good in tuned_shapes()
    set_tuned_shape(dict(good, block=64))
    assert dict(good, block=64) in tuned_shapes()
    set_tuned_shape(dict(good, block=64, modes_per_thread=3))   # three modes per thread: column kernel only
    assert dict(good, block=64, modes_per_thread=3) in tuned_shapes()
    for bad in (dict(good, modes_per_thread=3), dict(good, block=96), dict(good, d=3, block=0),
                dict(good, d=3, block=64), dict(good, op=3, block=64),
                dict(good, op=3, block=0), dict(good, d=3, modes_per_thread=4, block=256),
                dict(good, elem_bytes=2), dict(good, nodes=0)):
        with pytest.raises(StError):
            set_tuned_shape(bad)
