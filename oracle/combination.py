"""Index set and coefficients of the combination formula, Eq. (19), and the DoF
count of Section 3.2.

u^CF_J = sum_{a=0}^{J} (P_{a, J-a} - P_{a-1, J-a}) u  with P_{-1, .} = 0.
Spatial and temporal levels are offset by the coarsest levels (mx, mt): the
paper's level a corresponds to 2^(mx+a) spatial cells per direction and
2^(mt+b) time intervals.
"""


def components(J: int, mx: int, mt: int):
    """List of (j_x, j_t, coefficient): the +1 terms for a = 0..J, then the -1 terms
    for a = 1..J, each by increasing spatial level."""
    plus = [(mx + a, mt + J - a, +1) for a in range(J + 1)]
    minus = [(mx + a - 1, mt + J - a, -1) for a in range(1, J + 1)]
    return plus + minus


def space_dofs(d: int, jx: int) -> int:
    """dim V_jx for Q1 with homogeneous Dirichlet data: (2^jx - 1)^d."""
    return ((1 << jx) - 1) ** d


def time_dofs(jt: int, p: int = 2) -> int:
    """dim V_jt for splines of degree p and maximal regularity with w(0) = 0: 2^jt + p - 1."""
    return (1 << jt) + p - 1


def sparse_dofs(d: int, J: int, mx: int, mt: int) -> int:
    """N^sparse_DoFs of Section 3.2: the sum of the dimensions of the 2J+1 systems."""
    return sum(space_dofs(d, jx) * time_dofs(jt) for jx, jt, _ in components(J, mx, mt))
