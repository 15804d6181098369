"""Time matrices and time load vectors (proof of Prop. 1 in Section 4.1; Eq. (9)).

With test functions psi_i' (the time derivative of the test function in
Eq. (6)) and the weighted product (u, v)_{L^2_e} = int_0^T u v exp(-t/T) dt of
the Notation section:

    A[i, j] = (psi_j'', psi_i')_e + psi_j'(0) psi_i'(0)
    B[i, j] = (psi_j,   psi_i')_e

The right-hand side of Eq. (9) with w = phi_a(x) psi_i(t) needs
    (s, psi_i')_e   for each time factor s of the source,
    psi_i'(0)       for the v0 term,
    (1, psi_i')_e   for the u0 term (u0 is constant in time).

All integrals use 8-point Gauss-Legendre per knot interval: the integrands are
(piecewise) polynomials times exp(-t/T) (or a smooth source factor), so the
rule is exact to rounding for the matrices.
"""
import numpy as np

from .timebasis import psi

GAUSS_POINTS = 8


def quadrature(N: int, T: float):
    """Gauss-Legendre nodes and weights on every interval of the uniform mesh."""
    x, w = np.polynomial.legendre.leggauss(GAUSS_POINTS)
    h = T / N
    t = (np.arange(N)[:, None] * h + (x[None, :] + 1.0) * 0.5 * h).ravel()
    wt = np.tile(w * 0.5 * h, N)
    return t, wt


def time_matrices(jt: int, T: float, p: int = 2):
    """(A, B) of size n_t x n_t for level jt (2^jt intervals), splines of degree p."""
    N = 1 << jt
    t, wt = quadrature(N, T)
    we = wt * np.exp(-t / T)
    P = psi(t, N, T, 0, p)
    P1 = psi(t, N, T, 1, p)
    P2 = psi(t, N, T, 2, p)
    A = P1.T @ (we[:, None] * P2)          # A[i, j] = sum_q we psi_i'(t_q) psi_j''(t_q)
    B = P1.T @ (we[:, None] * P)
    d0 = psi(np.array([0.0]), N, T, 1, p)[0]
    A = A + np.outer(d0, d0)
    return A, B


def load_separable(s, jt: int, T: float, p: int = 2) -> np.ndarray:
    """b[i] = (s, psi_i')_e for a time factor s(t)."""
    N = 1 << jt
    t, wt = quadrature(N, T)
    return psi(t, N, T, 1, p).T @ (wt * np.exp(-t / T) * s(t))


def load_one(jt: int, T: float, p: int = 2) -> np.ndarray:
    """g[i] = (1, psi_i')_e."""
    return load_separable(lambda t: np.ones_like(t), jt, T, p)


def dpsi_at_zero(jt: int, T: float, p: int = 2) -> np.ndarray:
    """psi_i'(0)."""
    return psi(np.array([0.0]), 1 << jt, T, 1, p)[0]


def quadrature_rows(jt: int, T: float, p: int = 2):
    """Quadrature times t_q and the matrix Q[i, q] = w_q exp(-t_q/T) psi_i'(t_q),
    so that (f(x, .), psi_i')_e = sum_q Q[i, q] f(x, t_q) for a general source."""
    N = 1 << jt
    t, wt = quadrature(N, T)
    return t, (psi(t, N, T, 1, p) * (wt * np.exp(-t / T))[:, None]).T
