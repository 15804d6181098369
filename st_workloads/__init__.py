"""Seeded synthetic problem data for the space-time sparse-grid wave solver.

This module only *describes* problems of the form of Eq. (1) (domain, final
time, wave speed c^2, source f, initial data u0, v0, combination levels).  It
holds none of the method's arithmetic: no basis functions, no matrices, no
quadrature, no solves.  Both the CPU oracle and the CUDA path read the same
Problem objects, so that both discretise exactly the same data.

Every field is a vectorised Python callable:

* ``c2(x)``, ``u0(x)``, ``v0(x)``, ``g(x)``: ``x`` is an ``(n, d)`` float64 array
  of points, the result an ``(n,)`` float64 array.
* ``s(t)``: ``t`` is an ``(n,)`` array of times, the result ``(n,)``.
* ``f(x, t)``: points ``(n, d)`` and one scalar time, result ``(n,)``.

The source is ``f(x,t) = sum_r g_r(x) s_r(t) + f_general(x,t)``.

Combination levels follow Eq. (19) of Section 3.1, with the coarsest mesh
widths written as minimum levels: a level ``j`` means ``2**j`` uniform cells per
direction on the box (space) or on ``(0,T)`` (time).  Components are
``(mx + a, mt + J - a)`` for ``a = 0..J`` (+1) and ``(mx + a - 1, mt + J - a)`` for
``a = 1..J`` (-1).  The level pair ``(n, m)`` used by the workload recipes means
``J = n - 2m`` and ``mx = mt = m``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

SpaceFn = Callable[[np.ndarray], np.ndarray]
TimeFn = Callable[[np.ndarray], np.ndarray]
SpaceTimeFn = Callable[[np.ndarray, float], np.ndarray]


@dataclass
class Problem:
    """One instance of the wave problem, Eq. (1), plus its combination levels."""

    d: int
    lo: Tuple[float, ...]
    hi: Tuple[float, ...]
    T: float
    c2: SpaceFn
    J: int                      # combination level J of Eq. (19)
    mx: int                     # coarsest spatial level (2**mx cells per direction)
    mt: int                     # coarsest temporal level (2**mt intervals on (0,T))
    terms: List[Tuple[SpaceFn, TimeFn]] = field(default_factory=list)
    f_general: Optional[SpaceTimeFn] = None
    u0: Optional[SpaceFn] = None
    v0: Optional[SpaceFn] = None
    exact: Optional[SpaceTimeFn] = None   # closed-form solution, when known
    name: str = ""
    pt: int = 2                 # degree of the time splines (maximal regularity C^{pt-1})

    @property
    def finest(self) -> Tuple[int, int]:
        """Finest (space, time) level reached by the combination."""
        return self.mx + self.J, self.mt + self.J


def levels_nm(n: int, m: int) -> dict:
    """Translate the (n, m) level pair into (J, mx, mt)."""
    if n < 2 * m:
        raise ValueError("level n must be at least 2m")
    return dict(J=n - 2 * m, mx=m, mt=m)


def _prod_sin(x: np.ndarray) -> np.ndarray:
    return np.prod(np.sin(np.pi * x), axis=1)


# ---------------------------------------------------------------- closed forms
def standing_wave(d: int, n: int, m: int) -> Problem:
    """u = prod_i sin(pi x_i) cos(pi t) on (0,1)^d, c = 1, T = 1.

    u_tt = -pi^2 u and -Lap u = d pi^2 u, so f = (d-1) pi^2 prod sin(pi x_i) cos(pi t)
    (zero for d = 1); u0 = prod sin(pi x_i), v0 = 0.
    """
    terms = []
    if d > 1:
        terms.append((lambda x: (d - 1) * np.pi ** 2 * _prod_sin(x),
                      lambda t: np.cos(np.pi * t)))
    return Problem(d=d, lo=(0.0,) * d, hi=(1.0,) * d, T=1.0,
                   c2=lambda x: np.ones(len(x)), terms=terms,
                   u0=_prod_sin, v0=None,
                   exact=lambda x, t: _prod_sin(x) * np.cos(np.pi * t),
                   name=f"standing_wave_d{d}", **levels_nm(n, m))


def e1_vanishing(J: int, T: float = 1.0) -> Problem:
    """Section 6.1: Omega = (-1,1), c = 1, u0 = v0 = 0,
    u = t^6 sin(pi x) sin^2(5 pi t / 4); h0 = 1/2 in space (4 cells) and time (2 intervals).

    With phi(t) = t^6 sin^2(w t), w = 5 pi / 4, the source is
    f = sin(pi x) (phi'' + pi^2 phi), where
    phi'' = 15 t^4 (1 - cos 2wt) + 12 w t^5 sin 2wt + 2 w^2 t^6 cos 2wt.
    """
    w = 5.0 * np.pi / 4.0

    def phi(t):
        return t ** 6 * np.sin(w * t) ** 2

    def phi2(t):
        return (15 * t ** 4 * (1 - np.cos(2 * w * t)) + 12 * w * t ** 5 * np.sin(2 * w * t)
                + 2 * w ** 2 * t ** 6 * np.cos(2 * w * t))

    return Problem(d=1, lo=(-1.0,), hi=(1.0,), T=T, c2=lambda x: np.ones(len(x)),
                   terms=[(lambda x: np.sin(np.pi * x[:, 0]),
                           lambda t: phi2(t) + np.pi ** 2 * phi(t))],
                   exact=lambda x, t: np.sin(np.pi * x[:, 0]) * phi(t),
                   J=J, mx=2, mt=1, name="e1_vanishing")


def e2_variable_speed(J: int) -> Problem:
    """Section 6.2: Omega = (0,1), T = 1, c^2 = 1 + x, u = exp(xt) x (1 - x).

    u0 = x(1-x), v0 = x^2 (1-x), and f = u_tt - d/dx((1+x) u_x) is not separable:
    f = e^{xt} [x^3(1-x) - (t x(1-x) + 1 - 2x) - (1+x)(t^2 x(1-x) + 2t(1-2x) - 2)].
    """
    def f(x, t):
        x = x[:, 0]
        p = x * (1 - x)
        return np.exp(x * t) * (x * x * p - (t * p + 1 - 2 * x)
                                - (1 + x) * (t * t * p + 2 * t * (1 - 2 * x) - 2))

    return Problem(d=1, lo=(0.0,), hi=(1.0,), T=1.0, c2=lambda x: 1.0 + x[:, 0],
                   f_general=f, u0=lambda x: x[:, 0] * (1 - x[:, 0]),
                   v0=lambda x: x[:, 0] ** 2 * (1 - x[:, 0]),
                   exact=lambda x, t: np.exp(x[:, 0] * t) * x[:, 0] * (1 - x[:, 0]),
                   J=J, mx=1, mt=1, name="e2_variable_speed")


def travelling_wave(J: int, h0_level: int = 1) -> Problem:
    """Section 6.3: Omega = (-1,1), T = 1, c = 4/5, f = 0,
    u = w(x - ct) - w(2 - x - ct) with w(s) = exp(-16 (s - 0.6)^2): a pulse moving
    right and reflecting off x = 1 (u(1, t) = 0 exactly; |u(-1, t)| <= 1e-17).
    u0 = w(x) - w(2 - x), v0 = -c w'(x) + c w'(2 - x).  Coarsest mesh h0 = 2^-h0_level
    relative to the interval length 2 in space and to T in time (levels mx = h0_level + 1,
    mt = h0_level)."""
    c = 0.8

    def w(sv):
        return np.exp(-16.0 * (sv - 0.6) ** 2)

    def dw(sv):
        return -32.0 * (sv - 0.6) * w(sv)

    def exact(x, t):
        x = x[:, 0]
        return w(x - c * t) - w(2.0 - x - c * t)

    p = Problem(d=1, lo=(-1.0,), hi=(1.0,), T=1.0, c2=lambda x: np.full(len(x), c * c),
                u0=lambda x: w(x[:, 0]) - w(2.0 - x[:, 0]),
                v0=lambda x: -c * dw(x[:, 0]) + c * dw(2.0 - x[:, 0]),
                exact=exact, J=J, mx=h0_level + 1, mt=h0_level, name=f"travelling_wave_J{J}")
    p.exact_dt = lambda x, t: -c * dw(x[:, 0] - c * t) + c * dw(2.0 - x[:, 0] - c * t)
    p.exact_grad = lambda x, t: (dw(x[:, 0] - c * t) + dw(2.0 - x[:, 0] - c * t))[:, None]
    return p


# ------------------------------------------------------- workload recipes
def ricker(fp: float = 8.0, t0: Optional[float] = None) -> TimeFn:
    """Ricker wavelet (1 - 2 pi^2 fp^2 (t-t0)^2) exp(-pi^2 fp^2 (t-t0)^2), t0 = 1/fp."""
    t0 = 1.0 / fp if t0 is None else t0

    def s(t):
        a = (np.pi * fp * (np.asarray(t) - t0)) ** 2
        return (1.0 - 2.0 * a) * np.exp(-a)
    return s


def gaussian(centre: Sequence[float], sigma: float = 0.05) -> SpaceFn:
    c = np.asarray(centre, dtype=np.float64)

    def g(x):
        r2 = np.sum((x - c) ** 2, axis=1)
        return np.exp(-r2 / (2.0 * sigma * sigma))
    return g


def layered_2d(n: int = 12, m: int = 2) -> Problem:
    """d = 2, c^2 = 1 (y < 0.5) and 4 (y >= 0.5); u0 = v0 = 0;
    f = Gaussian(sigma 0.05, centre (0.3, 0.5)) x Ricker(peak frequency 8, t0 = 1/8)."""
    return Problem(d=2, lo=(0.0, 0.0), hi=(1.0, 1.0), T=1.0,
                   c2=lambda x: np.where(x[:, 1] < 0.5, 1.0, 4.0),
                   terms=[(gaussian((0.3, 0.5)), ricker(8.0))],
                   name=f"layered_2d_n{n}", **levels_nm(n, m))


def anisotropic_2d(n: int = 8, m: int = 2) -> Problem:
    """d = 2 on the non-square box (-0.5, 1.5) x (0, 0.75) (cells 2.67 times wider
    than tall), final time T = 1.7; c^2 = 1 + 0.5 sin(2 x) cos(3 y) + 0.8 [y > 0.4];
    u0 = a smooth bump vanishing on the boundary, v0 = 0.5 u0 (x + 0.5);
    f = Gaussian(sigma 0.1, centre (0.6, 0.3)) x Ricker(peak frequency 3, t0 = 1/3)."""
    lo, hi = (-0.5, 0.0), (1.5, 0.75)

    def bump(x):
        s = (x - np.asarray(lo)) / (np.asarray(hi) - np.asarray(lo))
        return np.prod(np.sin(np.pi * s), axis=1) * np.exp(-((x[:, 0] - 0.3) ** 2))

    return Problem(d=2, lo=lo, hi=hi, T=1.7,
                   c2=lambda x: 1.0 + 0.5 * np.sin(2 * x[:, 0]) * np.cos(3 * x[:, 1]) + 0.8 * (x[:, 1] > 0.4),
                   terms=[(gaussian((0.6, 0.3), 0.1), ricker(3.0))],
                   u0=bump, v0=lambda x: 0.5 * bump(x) * (x[:, 0] + 0.5),
                   name=f"anisotropic_2d_n{n}", **levels_nm(n, m))


def random_fourier_c2(d: int, seed: int, n_modes: int = 16, amp: float = 0.35,
                      kmax: int = 4, lo: float = 0.25, hi: float = 4.0) -> SpaceFn:
    """c^2 = clip(exp(g), lo, hi), g = sum_k a_k cos(2 pi kappa_k . x + phi_k),
    kappa_k uniform integers in [-kmax, kmax]^d without 0, a_k ~ N(0, amp^2),
    phi_k ~ U[0, 2 pi); numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    kap = []
    while len(kap) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=d)
        if np.any(k != 0):
            kap.append(k)
    kap = np.asarray(kap, dtype=np.float64)
    a = rng.normal(0.0, amp, size=n_modes)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)

    def c2(x):
        g = np.cos(2.0 * np.pi * (x @ kap.T) + ph) @ a
        return np.clip(np.exp(g), lo, hi)
    return c2


def random_medium_3d(n: int = 10, m: int = 3, seed: int = 0) -> Problem:
    """d = 3, c^2 = clip(exp(16-mode random Fourier field), 0.25, 4);
    u0 = prod sin(pi x_i), v0 = f = 0."""
    return Problem(d=3, lo=(0.0,) * 3, hi=(1.0,) * 3, T=1.0,
                   c2=random_fourier_c2(3, seed), u0=_prod_sin,
                   name=f"random_medium_3d_n{n}", **levels_nm(n, m))


def batch_instances(count: int = 64, seed: int = 0, levels: Sequence[int] = (8, 9, 10, 11, 12),
                    m: int = 2) -> List[Problem]:
    """Independent d = 2 instances: smooth random c^2 in [0.5, 2] with a seeded
    horizontal jump, a Gaussian source at a random centre in [0.2, 0.8]^2 times a
    Ricker wavelet, level n drawn uniformly from ``levels``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(levels))
        smooth = random_fourier_c2(2, int(rng.integers(1 << 31)), n_modes=8, amp=0.25,
                                   kmax=3, lo=0.5, hi=2.0)
        yj = float(rng.uniform(0.3, 0.7))
        jump = float(rng.uniform(1.0, 1.6))

        def c2(x, smooth=smooth, yj=yj, jump=jump):
            return np.clip(smooth(x) * np.where(x[:, 1] < yj, 1.0, jump), 0.5, 2.0)
        centre = rng.uniform(0.2, 0.8, size=2)
        out.append(Problem(d=2, lo=(0.0, 0.0), hi=(1.0, 1.0), T=1.0, c2=c2,
                           terms=[(gaussian(centre), ricker(8.0))],
                           name=f"batch_{i}_n{n}", **levels_nm(n, m)))
    return out



@dataclass
class InverseSetup:
    """Inputs of the receiver-misfit gradient: a base problem (box, T, levels),
    c^2 and the source's spatial factor as nodal values on the uniform
    parameter grid of level jp, the source's time factor, receivers, the target
    time level of the misfit, and c^2 of the synthetic observations."""
    base: Problem
    jp: int
    c2_nodal: np.ndarray
    g_nodal: np.ndarray
    s: TimeFn
    receivers: np.ndarray
    jt_star: int
    c2_obs_nodal: np.ndarray


def param_nodes(d: int, jp: int) -> np.ndarray:
    """All (2^jp+1)^d nodes of the unit box, x fastest."""
    ax = np.linspace(0.0, 1.0, (1 << jp) + 1)
    mesh = np.meshgrid(*([ax] * d), indexing="ij")[::-1]
    return np.stack([m.ravel() for m in mesh], axis=1)


def smooth_field(d: int, seed: int, lo: float = 0.5, hi: float = 2.0, n_modes: int = 6,
                 kmax: int = 2) -> SpaceFn:
    """lo + (hi - lo) (1 + tanh(g)) / 2 with g = sum_k a_k cos(2 pi kappa_k . x + phi_k),
    kappa_k integers in [-kmax, kmax]^d without 0, a_k ~ N(0, 1); default_rng(seed)."""
    rng = np.random.default_rng(seed)
    kap = []
    while len(kap) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=d)
        if np.any(k != 0):
            kap.append(k)
    kap = np.asarray(kap, dtype=np.float64)
    a = rng.normal(0.0, 1.0, size=n_modes)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)

    def f(x):
        g = np.cos(2.0 * np.pi * (x @ kap.T) + ph) @ a
        return lo + (hi - lo) * 0.5 * (1.0 + np.tanh(g))
    return f


def inverse_2d(n: int = 10, m: int = 2, jp: int = 6, n_receivers: int = 32, seed: int = 0) -> InverseSetup:
    """d = 2 receiver-misfit setup: c^2 a seeded smooth field in [0.5, 2] on the
    (2^jp+1)^2 nodes; source Gaussian (sigma 0.05, centre (0.3, 0.5)) x Ricker
    (f_p 8); receivers (r + 1/2)/n_receivers, 0.9); observations from c^2 times
    (1 + 0.2 exp(-|x - (0.6, 0.7)|^2 / 0.02)); misfit on target times of level n - m."""
    base = Problem(d=2, lo=(0.0, 0.0), hi=(1.0, 1.0), T=1.0, c2=lambda x: np.ones(len(x)),
                   name=f"inverse_2d_n{n}", **levels_nm(n, m))
    x = param_nodes(2, jp)
    c2 = smooth_field(2, seed)(x)
    bump = 1.0 + 0.2 * np.exp(-np.sum((x - np.array([0.6, 0.7])) ** 2, axis=1) / 0.02)
    rec = np.stack([(np.arange(n_receivers) + 0.5) / n_receivers, np.full(n_receivers, 0.9)], axis=1)
    return InverseSetup(base=base, jp=jp, c2_nodal=c2, g_nodal=gaussian((0.3, 0.5))(x), s=ricker(8.0),
                        receivers=rec, jt_star=n - m, c2_obs_nodal=c2 * bump)
