"""Quadratic C^1 B-splines on a uniform mesh of (0, T) (the time space V_jt).

Section 2.2 requires V_jt to lie in H^2_{0,.}(0,T) (Notation: w(0) = 0), and
Remark 1 / Table 1 name C^1 splines of even degree as the proven case; the
lowest such degree is 2 (maximal regularity for degree 2, and the degree paired
with p_x = 1 in Remark "Necessity").  The dimension formula of Section 3.2,
N_t (p_t - r_t) + r_t with p_t = 2, r_t = 1, gives n_t = N_t + 1.

Basis: open uniform knot vector with N intervals, B-splines B_0 .. B_{N+1} by the
Cox-de Boor recursion; B_0 is the only one with B(0) != 0 and is dropped, so
psi_i = B_i for i = 1 .. N+1.
"""
import numpy as np


def knots(N: int, T: float) -> np.ndarray:
    """Open uniform knot vector of degree 2: 0,0,0,h,2h,...,T,T,T."""
    inner = np.linspace(0.0, T, N + 1)
    return np.concatenate([[0.0, 0.0], inner, [T, T]])


def _span(t: np.ndarray, N: int, T: float) -> np.ndarray:
    """Index of the knot interval [k h, (k+1) h) holding t (the last one closed)."""
    k = np.floor(np.asarray(t, dtype=np.float64) / (T / N)).astype(np.int64)
    return np.clip(k, 0, N - 1)


def bsplines(t, N: int, T: float, deriv: int = 0) -> np.ndarray:
    """Values (deriv=0), first or second derivatives of all N+2 quadratic B-splines.

    Returns an array of shape (len(t), N+2).  The Cox-de Boor recursion is taken
    literally: degree-0 indicators, then degree 1 and 2 by the two-term
    recursion, derivatives by the standard B-spline derivative formula
    B'_{i,p} = p/(t_{i+p}-t_i) B_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) B_{i+1,p-1}.
    """
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    kv = knots(N, T)
    nk = len(kv)
    # degree 0: indicator of [kv[i], kv[i+1]); use the span so t = T is included
    B0 = np.zeros((len(t), nk - 1))
    B0[np.arange(len(t)), _span(t, N, T) + 2] = 1.0

    def raise_degree(Bp, p):
        out = np.zeros((len(t), nk - 1 - p))
        for i in range(nk - 1 - p):
            d1 = kv[i + p] - kv[i]
            d2 = kv[i + p + 1] - kv[i + 1]
            if d1 > 0:
                out[:, i] += (t - kv[i]) / d1 * Bp[:, i]
            if d2 > 0:
                out[:, i] += (kv[i + p + 1] - t) / d2 * Bp[:, i + 1]
        return out

    def differentiate(Bp, p):
        out = np.zeros((len(t), nk - 1 - p))
        for i in range(nk - 1 - p):
            d1 = kv[i + p] - kv[i]
            d2 = kv[i + p + 1] - kv[i + 1]
            if d1 > 0:
                out[:, i] += p / d1 * Bp[:, i]
            if d2 > 0:
                out[:, i] -= p / d2 * Bp[:, i + 1]
        return out

    B1 = raise_degree(B0, 1)
    if deriv == 0:
        return raise_degree(B1, 2)
    if deriv == 1:
        return differentiate(B1, 2)
    if deriv == 2:
        # B''_{i,2} = 2/(t_{i+2}-t_i) B'_{i,1} - 2/(t_{i+3}-t_{i+1}) B'_{i+1,1}
        return differentiate(differentiate(B0, 1), 2)
    raise ValueError("deriv must be 0, 1 or 2")


def psi(t, N: int, T: float, deriv: int = 0) -> np.ndarray:
    """The basis of V_jt: B_1 .. B_{N+1} (B_0 removed), shape (len(t), N+1)."""
    return bsplines(t, N, T, deriv)[:, 1:]


def n_time_dofs(jt: int) -> int:
    """dim V_jt = N_t (p_t - r_t) + r_t with N_t = 2^jt, p_t = 2, r_t = 1."""
    return (1 << jt) + 1
