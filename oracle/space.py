"""Q1 finite elements on a uniform tensor grid of a box (Section 3.2, Eq. (44)).

Level jx means N = 2^jx cells per direction, h_k = (hi_k - lo_k)/N.  Nodes are
numbered lexicographically with the first coordinate fastest.  The spatial
space V_jx is the span of the hat functions of the interior nodes (homogeneous
Dirichlet condition of Eq. (1)); dim = (N - 1)^d.

Element matrices on a cell are tensor products of the 1D ones,
    M1 = h/6 [[2, 1], [1, 2]],   K1 = 1/h [[1, -1], [-1, 1]],
    M_e = M1 (x) M1 (x) ...,     K_e = sum_k (M1 (x) .. K1 (in direction k) .. M1),
and K collects c^2_e K_e with c^2 constant on each cell (its value at the cell
centre): K = the matrix of (c^2 grad u, grad v), M of (u, v).
"""
import itertools

import numpy as np
import scipy.sparse as sp


def grid(d, lo, hi, jx):
    N = 1 << jx
    h = np.array([(hi[k] - lo[k]) / N for k in range(d)])
    return N, h


def node_coords(d, lo, hi, jx):
    """All (N+1)^d nodes, lexicographic with x_0 fastest; shape ((N+1)^d, d)."""
    N, h = grid(d, lo, hi, jx)
    axes = [lo[k] + h[k] * np.arange(N + 1) for k in range(d)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")          # slowest first
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


def interior_mask(d, jx):
    N = 1 << jx
    idx = np.meshgrid(*([np.arange(N + 1)] * d), indexing="ij")
    m = np.ones(idx[0].shape, dtype=bool)
    for a in idx:
        m &= (a > 0) & (a < N)
    return m.ravel()


def cell_centres(d, lo, hi, jx):
    """Centres of the N^d cells, lexicographic with x_0 fastest."""
    N, h = grid(d, lo, hi, jx)
    axes = [lo[k] + h[k] * (np.arange(N) + 0.5) for k in range(d)]
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


def element_matrices(d, h):
    """Local mass and unit-coefficient stiffness matrices of one cell, 2^d x 2^d.
    Local corner index c has bit k set when the corner is at the upper end in direction k."""
    M1 = [hk / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]]) for hk in h]
    K1 = [1.0 / hk * np.array([[1.0, -1.0], [-1.0, 1.0]]) for hk in h]
    nc = 1 << d
    Me = np.zeros((nc, nc))
    Ke = np.zeros((nc, nc))
    for a in range(nc):
        for b in range(nc):
            bits_a = [(a >> k) & 1 for k in range(d)]
            bits_b = [(b >> k) & 1 for k in range(d)]
            m = 1.0
            for k in range(d):
                m *= M1[k][bits_a[k], bits_b[k]]
            Me[a, b] = m
            s = 0.0
            for k in range(d):
                term = 1.0
                for l in range(d):
                    mat = K1[l] if l == k else M1[l]
                    term *= mat[bits_a[l], bits_b[l]]
                s += term
            Ke[a, b] = s
    return Me, Ke


def assemble_full(d, lo, hi, jx, c2_cell):
    """Mass and stiffness on ALL nodes (boundary included), as CSR matrices."""
    N, h = grid(d, lo, hi, jx)
    Me, Ke = element_matrices(d, h)
    nn = N + 1
    cells = np.stack(np.meshgrid(*([np.arange(N)] * d), indexing="ij")[::-1], axis=-1).reshape(-1, d)
    # global node of local corner c of each cell
    corner = np.zeros((len(cells), 1 << d), dtype=np.int64)
    for c in range(1 << d):
        g = np.zeros(len(cells), dtype=np.int64)
        stride = 1
        for k in range(d):
            g += (cells[:, k] + ((c >> k) & 1)) * stride
            stride *= nn
        corner[:, c] = g
    rows = np.repeat(corner, 1 << d, axis=1).ravel()
    cols = np.tile(corner, (1, 1 << d)).ravel()
    vm = np.tile(Me.ravel(), len(cells))
    vk = (c2_cell[:, None] * Ke.ravel()[None, :]).ravel()
    n = nn ** d
    M = sp.csr_matrix((vm, (rows, cols)), shape=(n, n))
    K = sp.csr_matrix((vk, (rows, cols)), shape=(n, n))
    return M, K


def space_matrices(problem, jx):
    """Interior-by-interior M, K plus the interior-by-all blocks used for data loads."""
    d = problem.d
    c2 = np.asarray(problem.c2(cell_centres(d, problem.lo, problem.hi, jx)), dtype=np.float64)
    Mf, Kf = assemble_full(d, problem.lo, problem.hi, jx, c2)
    inner = np.nonzero(interior_mask(d, jx))[0]
    return dict(M=Mf[inner][:, inner].tocsr(), K=Kf[inner][:, inner].tocsr(),
                M_load=Mf[inner].tocsr(), K_load=Kf[inner].tocsr(), inner=inner, c2=c2)


def interpolate_nodal(values_all, d, lo, hi, jx, pts):
    """Evaluate the Q1 function with the given values on all (N+1)^d nodes at points pts."""
    N, h = grid(d, lo, hi, jx)
    nn = N + 1
    vals = np.zeros(len(pts))
    idx = []
    frac = []
    for k in range(d):
        s = (pts[:, k] - lo[k]) / h[k]
        c = np.clip(np.floor(s).astype(np.int64), 0, N - 1)
        idx.append(c)
        frac.append(s - c)
    for c in range(1 << d):
        w = np.ones(len(pts))
        g = np.zeros(len(pts), dtype=np.int64)
        stride = 1
        for k in range(d):
            b = (c >> k) & 1
            w *= frac[k] if b else (1.0 - frac[k])
            g += (idx[k] + b) * stride
            stride *= nn
        vals += w * values_all[g]
    return vals


def interpolate_nodal_grad(values_all, d, lo, hi, jx, pts):
    """Gradient (n, d) at the points of the Q1 function with the given values on all
    (N+1)^d nodes: the derivative of the multilinear interpolant in each direction
    (inside the cell holding the point)."""
    N, h = grid(d, lo, hi, jx)
    nn = N + 1
    idx, frac = [], []
    for k in range(d):
        s = (pts[:, k] - lo[k]) / h[k]
        c = np.clip(np.floor(s).astype(np.int64), 0, N - 1)
        idx.append(c)
        frac.append(s - c)
    g = np.zeros((len(pts), d))
    for c in range(1 << d):
        node = np.zeros(len(pts), dtype=np.int64)
        stride = 1
        for k in range(d):
            node += (idx[k] + ((c >> k) & 1)) * stride
            stride *= nn
        v = values_all[node]
        for k in range(d):
            w = np.ones(len(pts))
            for l in range(d):
                b = (c >> l) & 1
                if l == k:
                    w *= (1.0 if b else -1.0) / h[k]
                else:
                    w *= frac[l] if b else (1.0 - frac[l])
            g[:, k] += w * v
    return g
