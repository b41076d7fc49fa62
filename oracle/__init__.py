"""CPU oracle for the multigroup S_N tensor-train transport step (TEST INFRASTRUCTURE).

This package is the independent, slow, obviously-correct FP64 reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and its ``--impl reference`` arm) may import
or execute anything here.  The product path never calls it, and it shares no code
with the CUDA path: the only common inputs are the seeded raw arrays produced by
``paper_2602_00290_gb300.workloads``.

Modules
-------
quadrature  angular quadrature sets (Sec. 4 preamble; Gauss-Legendre mu for the slab)
planck      group emission coefficients epsilon_f(T), Eqs. (Ttoeps1)-(Ttoeps2)
problem     derived per-row coefficients of the operator-split update, Eq. (discRTsource)
dense       dense full-grid FP64 S_N stepper (plain C with OpenMP, loaded by ctypes)
naive_tt    explicit-sum TT arithmetic and SVD-based rounding (numpy / LAPACK)
naive_tt_nux  the same step in the split topology [Z(nu x)][y][theta][phi] (Sec. 5.2)

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, invariants, brute force); none is marked "parity unpinned".
"""
