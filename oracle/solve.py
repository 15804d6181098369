"""One component's Galerkin system, its solution, and the combination sum.

Eq. (9) on V_jx (x) V_jt, with u = sum_j u_j(x) psi_j(t) and the test function
phi_a(x) psi_i(t), is the linear system of Eq. (30) discretised in space:

    sum_j A[i,j] (M u_j)_a + B[i,j] (K u_j)_a = F[i,a],
    i.e.  (A (x) M + B (x) K) vec(U) = vec(F),  U[j, a] = u_j at interior node a.

Right-hand side of Eq. (9), with f = sum_r g_r(x) s_r(t) + f_general(x, t) and the
data replaced by Q1 nodal interpolants I(.) at level jx:

    F[i,a] = sum_r (s_r, psi_i')_e (M I g_r)_a + sum_q Q[i,q] (M I f(., t_q))_a
             + psi_i'(0) (M I v0)_a - (1, psi_i')_e (K I u0)_a.

The weak solution is the discrete w plus u0 (Section 2.1); the lifting uses
I_jx u0.  The combination value at a target node is sum_k c_k u_k(x, t),
Eq. (19), summed in the fixed component order.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import combination, space, timebasis, timemats


def _pt(problem):
    """Spline degree p_t of the time space (2 unless the problem states another)."""
    return getattr(problem, "pt", 2)


def _nodal(fn, pts):
    return np.zeros(len(pts)) if fn is None else np.asarray(fn(pts), dtype=np.float64)


def rhs(problem, jx, jt, sm=None):
    """F of shape (n_t, N_x), time-major."""
    sm = sm or space.space_matrices(problem, jx)
    pts = space.node_coords(problem.d, problem.lo, problem.hi, jx)
    T = problem.T
    pt = _pt(problem)
    nt = timebasis.n_time_dofs(jt, pt)
    F = np.zeros((nt, len(sm["inner"])))
    for g, s in problem.terms:
        F += np.outer(timemats.load_separable(s, jt, T, pt), sm["M_load"] @ _nodal(g, pts))
    if problem.f_general is not None:
        tq, Q = timemats.quadrature_rows(jt, T, pt)
        for q, tt in enumerate(tq):
            F += np.outer(Q[:, q], sm["M_load"] @ _nodal(lambda x: problem.f_general(x, tt), pts))
    if problem.v0 is not None:
        F += np.outer(timemats.dpsi_at_zero(jt, T, pt), sm["M_load"] @ _nodal(problem.v0, pts))
    if problem.u0 is not None:
        F -= np.outer(timemats.load_one(jt, T, pt), sm["K_load"] @ _nodal(problem.u0, pts))
    return F


def system_matrix(problem, jx, jt, sm=None):
    sm = sm or space.space_matrices(problem, jx)
    A, B = timemats.time_matrices(jt, problem.T, _pt(problem))
    return (sp.kron(sp.csr_matrix(A), sm["M"]) + sp.kron(sp.csr_matrix(B), sm["K"])).tocsc()


def apply_system(problem, jx, jt, U, sm=None):
    """(A (x) M + B (x) K) vec(U) without assembling the space-time matrix.

    With U of shape (n_t, N_x) stored time-major, row i of the product is
    sum_j A[i,j] M u_j + B[i,j] K u_j (Eq. (30)), i.e. A U M^T + B U K^T in
    matrix form; M and K are symmetric.  Returns shape (n_t, N_x)."""
    sm = sm or space.space_matrices(problem, jx)
    A, B = timemats.time_matrices(jt, problem.T, _pt(problem))
    UM = (sm["M"] @ U.T).T
    UK = (sm["K"] @ U.T).T
    return A @ UM + B @ UK


def system_norm1(problem, jx, jt, sm=None):
    """||A (x) M + B (x) K||_1 (largest absolute column sum) without assembling it.

    Column (j, b) holds the blocks A[i,j] M[:, b] + B[i,j] K[:, b] for every
    time row i, so its absolute sum is sum_i colsum|A[i,j] M + B[i,j] K|[b]."""
    sm = sm or space.space_matrices(problem, jx)
    A, B = timemats.time_matrices(jt, problem.T, _pt(problem))
    M, K = sm["M"].tocsr(), sm["K"].tocsr()
    M.sort_indices()
    K.sort_indices()
    # M and K come from the same element connectivity; when their stored
    # patterns agree the blocks are formed on the value arrays directly
    same = np.array_equal(M.indptr, K.indptr) and np.array_equal(M.indices, K.indices)
    nt, n = A.shape[0], M.shape[1]
    best = 0.0
    for j in range(nt):
        col = np.zeros(n)
        for i in range(nt):
            if A[i, j] == 0.0 and B[i, j] == 0.0:
                continue
            if same:
                col += np.bincount(M.indices, weights=np.abs(A[i, j] * M.data + B[i, j] * K.data), minlength=n)
            else:
                col += np.asarray(abs(A[i, j] * M + B[i, j] * K).sum(axis=0)).ravel()
        best = max(best, float(col.max()))
    return best


def backward_error(problem, jx, jt, U, F=None, sm=None):
    """Normwise backward error ||F - S U||_1 / (||S||_1 ||U||_1 + ||F||_1) of a
    coefficient array U for component (jx, jt), S and F as defined above."""
    sm = sm or space.space_matrices(problem, jx)
    if F is None:
        F = rhs(problem, jx, jt, sm)
    R = F - apply_system(problem, jx, jt, U, sm)
    return float(np.abs(R).sum() / (system_norm1(problem, jx, jt, sm) * np.abs(U).sum() + np.abs(F).sum()))


def solve_component(problem, jx, jt, F=None, method="lu"):
    """Solve (A (x) M + B (x) K) U = F exactly (up to rounding).

    method="lu": sparse LU of the assembled space-time matrix.
    method="schur": complex Schur form B^{-1}A = Q R Q^H (Q unitary), then the
    triangular recurrence (R_qq M + K) z_q = g_q - sum_{l>q} R_ql M z_l with
    G = Q^H B^{-1} F, each mode by sparse LU, and U = Re(Q Z).  Same solution,
    used where the space-time LU is too large.
    """
    sm = space.space_matrices(problem, jx)
    if F is None:
        F = rhs(problem, jx, jt, sm)
    nt, nx = F.shape
    if method == "lu":
        S = system_matrix(problem, jx, jt, sm)
        return spl.splu(S).solve(F.ravel()).reshape(nt, nx)
    if method == "schur":
        A, B = timemats.time_matrices(jt, problem.T, _pt(problem))
        R, Q = sla.schur(np.linalg.solve(B, A).astype(complex), output="complex")
        G = Q.conj().T @ np.linalg.solve(B, F)
        M = sm["M"].astype(complex)
        K = sm["K"].astype(complex)
        Z = np.zeros((nt, nx), dtype=complex)
        for q in range(nt - 1, -1, -1):
            rhs_q = G[q].copy()
            if q + 1 < nt:
                rhs_q -= M @ (R[q, q + 1:] @ Z[q + 1:])
            Z[q] = spl.splu((R[q, q] * M + K).tocsc()).solve(rhs_q)
        return np.real(Q @ Z)
    raise ValueError(method)


def all_node_values(problem, jx, interior_values):
    """Embed interior values into all (N+1)^d nodes (zero Dirichlet data)."""
    full = np.zeros(((1 << jx) + 1) ** problem.d)
    full[space.interior_mask(problem.d, jx)] = interior_values
    return full


def evaluate_component(problem, jx, jt, U, pts, times):
    """u_k(x, t) = sum_i psi_i(t) (I W_i)(x) + (I_jx u0)(x) on the tensor set pts x times.
    Returns shape (len(times), len(pts))."""
    N_t = 1 << jt
    Pt = timebasis.psi(np.asarray(times, dtype=np.float64), N_t, problem.T, 0, _pt(problem))
    Wt = Pt @ U                                   # (n_times, N_x interior)
    lift = _nodal(problem.u0, space.node_coords(problem.d, problem.lo, problem.hi, jx))
    out = np.zeros((len(times), len(pts)))
    for s in range(len(times)):
        vals = all_node_values(problem, jx, Wt[s]) + lift
        out[s] = space.interpolate_nodal(vals, problem.d, problem.lo, problem.hi, jx, pts)
    return out


def target_grid(problem, jx_star, jt_star):
    """Nodal target: all (2^jx*+1)^d spatial nodes (boundary included) and the
    2^jt*+1 uniform times of [0, T] (0 and T included)."""
    pts = space.node_coords(problem.d, problem.lo, problem.hi, jx_star)
    times = np.linspace(0.0, problem.T, (1 << jt_star) + 1)
    return pts, times


def solve_all(problem, method="lu"):
    """Coefficient arrays U_k of every component of Eq. (19), in component order."""
    comps = combination.components(problem.J, problem.mx, problem.mt)
    return comps, [solve_component(problem, jx, jt, method=method) for jx, jt, _ in comps]


def combine(problem, comps, sols, pts, times):
    """u^CF_J = sum_k c_k u_k at the points, Eq. (19); fixed component order."""
    out = np.zeros((len(times), len(pts)))
    for (jx, jt, c), U in zip(comps, sols):
        out += c * evaluate_component(problem, jx, jt, U, pts, times)
    return out


def l2_error_qt(problem, comps, sols, jx_q, jt_q, npts=3, ntpts=4):
    """Relative L^2(Q_T) error of u^CF against problem.exact, by tensor Gauss
    quadrature on the uniform (jx_q, jt_q) space-time mesh."""
    d = problem.d
    xg, wg = np.polynomial.legendre.leggauss(npts)
    tg, wtg = np.polynomial.legendre.leggauss(ntpts)
    N, h = space.grid(d, problem.lo, problem.hi, jx_q)
    cells = space.cell_centres(d, problem.lo, problem.hi, jx_q)
    offs = np.stack(np.meshgrid(*([xg] * d), indexing="ij"), axis=-1).reshape(-1, d)
    wloc = np.prod(np.stack(np.meshgrid(*([wg] * d), indexing="ij"), axis=-1).reshape(-1, d), axis=1)
    pts = (cells[:, None, :] + 0.5 * offs[None, :, :] * h[None, None, :]).reshape(-1, d)
    wx = np.tile(wloc, len(cells)) * np.prod(h) / (2 ** d)
    Nt = 1 << jt_q
    ht = problem.T / Nt
    times = (np.arange(Nt)[:, None] * ht + (tg[None, :] + 1) * 0.5 * ht).ravel()
    wt = np.tile(wtg * 0.5 * ht, Nt)
    approx = combine(problem, comps, sols, pts, times)
    exact = np.stack([problem.exact(pts, t) for t in times])
    W = wt[:, None] * wx[None, :]
    return np.sqrt(np.sum(W * (approx - exact) ** 2) / np.sum(W * exact ** 2))
