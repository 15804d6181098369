"""B-splines of maximal regularity on a uniform mesh of (0, T) (the time space V_jt).

Section 2.2 requires V_jt to lie in H^2_{0,.}(0,T) (Notation: w(0) = 0).  The
default is degree p = 2 (C^1 quadratics), the case Remark 1 / Table 1 prove
(C^1 splines of even degree); degrees 3 and 4 with maximal regularity
(C^{p-1}) are the conjectured cases of the same table.  The dimension formula
of Section 3.2, N_t (p_t - r_t) + r_t with r_t = p_t - 1, gives n_t = N_t + p - 1.

Basis: open uniform knot vector of degree p with N intervals (p + 1 copies of
0 and of T), B-splines B_0 .. B_{N+p-1} by the Cox-de Boor recursion; B_0 is the
only one with B(0) != 0 and is dropped, so psi_i = B_i for i = 1 .. N+p-1.
"""
import numpy as np


def knots(N: int, T: float, p: int = 2) -> np.ndarray:
    """Open uniform knot vector of degree p: p extra copies of 0 and of T around 0, h, ..., T."""
    inner = np.linspace(0.0, T, N + 1)
    return np.concatenate([np.zeros(p), inner, np.full(p, T)])


def _span(t: np.ndarray, N: int, T: float) -> np.ndarray:
    """Index of the knot interval [k h, (k+1) h) holding t (the last one closed)."""
    k = np.floor(np.asarray(t, dtype=np.float64) / (T / N)).astype(np.int64)
    return np.clip(k, 0, N - 1)


def bsplines(t, N: int, T: float, deriv: int = 0, p: int = 2) -> np.ndarray:
    """Values (deriv=0), first or second derivatives of all N+p B-splines of degree p >= 2.

    Returns an array of shape (len(t), N+p).  The Cox-de Boor recursion is taken
    literally: degree-0 indicators, then degrees 1 .. p by the two-term
    recursion, derivatives by the standard B-spline derivative formula
    B'_{i,q} = q/(t_{i+q}-t_i) B_{i,q-1} - q/(t_{i+q+1}-t_{i+1}) B_{i+1,q-1}.
    """
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    kv = knots(N, T, p)
    nk = len(kv)
    # degree 0: indicator of [kv[i], kv[i+1]); use the span so t = T is included
    B0 = np.zeros((len(t), nk - 1))
    B0[np.arange(len(t)), _span(t, N, T) + p] = 1.0

    def raise_degree(Bp, q):
        out = np.zeros((len(t), nk - 1 - q))
        for i in range(nk - 1 - q):
            d1 = kv[i + q] - kv[i]
            d2 = kv[i + q + 1] - kv[i + 1]
            if d1 > 0:
                out[:, i] += (t - kv[i]) / d1 * Bp[:, i]
            if d2 > 0:
                out[:, i] += (kv[i + q + 1] - t) / d2 * Bp[:, i + 1]
        return out

    def differentiate(Bp, q):
        out = np.zeros((len(t), nk - 1 - q))
        for i in range(nk - 1 - q):
            d1 = kv[i + q] - kv[i]
            d2 = kv[i + q + 1] - kv[i + 1]
            if d1 > 0:
                out[:, i] += q / d1 * Bp[:, i]
            if d2 > 0:
                out[:, i] -= q / d2 * Bp[:, i + 1]
        return out

    if p < 2:
        raise ValueError("degree p must be at least 2 (V_t must lie in H^2)")
    B = [B0]
    for q in range(1, p + 1):
        B.append(raise_degree(B[-1], q))
    if deriv == 0:
        return B[p]
    if deriv == 1:
        return differentiate(B[p - 1], p)
    if deriv == 2:
        # B''_{i,p} = p/(t_{i+p}-t_i) B'_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) B'_{i+1,p-1}
        return differentiate(differentiate(B[p - 2], p - 1), p)
    raise ValueError("deriv must be 0, 1 or 2")


def psi(t, N: int, T: float, deriv: int = 0, p: int = 2) -> np.ndarray:
    """The basis of V_jt: B_1 .. B_{N+p-1} (B_0 removed), shape (len(t), N+p-1)."""
    return bsplines(t, N, T, deriv, p)[:, 1:]


def n_time_dofs(jt: int, p: int = 2) -> int:
    """dim V_jt = N_t (p_t - r_t) + r_t with N_t = 2^jt and maximal regularity r_t = p_t - 1."""
    return (1 << jt) + p - 1
