"""Pins of the oracle's matrix-free residual and norm of the space-time matrix
(used for backward errors of components too large to assemble): both must
equal what the assembled (A (x) M + B (x) K) of Eq. (30) gives."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import st_workloads as W
from oracle import solve as osolve


CASES = [(W.e2_variable_speed(3), 3, 4), (W.layered_2d(6, 2), 3, 2), (W.layered_2d(6, 2), 2, 3),
         (W.random_medium_3d(6, 2, seed=1), 2, 2)]


@pytest.mark.parametrize("p,jx,jt", CASES)
def test_apply_system_equals_assembled_product(p, jx, jt):
    S = osolve.system_matrix(p, jx, jt)
    F = osolve.rhs(p, jx, jt)
    U = np.random.default_rng(jx * 10 + jt).standard_normal(F.shape)
    ref = (S @ U.ravel()).reshape(F.shape)
    got = osolve.apply_system(p, jx, jt, U)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("p,jx,jt", CASES)
def test_system_norm1_equals_assembled_norm(p, jx, jt):
    S = osolve.system_matrix(p, jx, jt)
    assert osolve.system_norm1(p, jx, jt) == pytest.approx(spl.norm(S, 1), rel=1e-13)


def test_backward_error_separates_exact_from_perturbed_solutions():
    p = W.layered_2d(6, 2)
    jx, jt = 3, 2
    U = osolve.solve_component(p, jx, jt)
    assert osolve.backward_error(p, jx, jt, U) < 1e-15
    Up = U * (1 + 1e-7 * np.random.default_rng(0).standard_normal(U.shape))
    eta = osolve.backward_error(p, jx, jt, Up)
    assert 1e-10 < eta < 1e-6
