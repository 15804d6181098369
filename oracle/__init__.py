"""Plain, slow, FP64 CPU oracle for the space-time sparse-grid wave solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It computes the plain definition of the method, step by step, with no
blocking, fusion or reordering:

* ``timebasis``  quadratic C^1 B-splines in time with the first one removed
  (the space V_jt of Section 2.2; w(0) = 0 by H^2_{0,.}, Notation).
* ``timemats``   the 1D time matrices A_jt, B_jt of the proof of Prop. 1
  (Section 4.1), with the exponential weight of the Notation section, and the
  time load vectors of the right-hand side of Eq. (9).
* ``space``      Q1 finite elements on the uniform tensor grid (mass M and
  stiffness K with cellwise c^2, Eq. (44) and Section 3.2), nodal interpolation.
* ``combination`` the index set and coefficients of Eq. (19) and the DoF count
  of Section 3.2.
* ``solve``      assembly of (A (x) M + B (x) K) U = F for one component
  (Eq. (9) written as Eq. (30)), sparse direct solve, lifting by u0
  (Section 2.1), evaluation on target nodes and the +-1 sum of Eq. (19).

Readings where the paper leaves freedom (all shared with the CUDA path by
definition, never by code): time degree 2 with C^1 regularity; data u0, v0 and
the spatial factors of f replaced by their Q1 nodal interpolants at the
component's spatial level; time integrals by 8-point Gauss-Legendre per knot
interval; c^2 sampled at cell centres (cellwise constant).

Parity pins live in ``tests/test_oracle_*.py`` (closed forms, invariants,
Eq. (3), Eq. (10) reproduction, Eq. (19)-(21) identities, convergence rates).
"""
