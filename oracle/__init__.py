"""CPU oracle for the short-characteristics formal solution and Jacobi ALI.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the method of Davis, Stone & Jiang (2012), "A Radiation Transfer Solver for
Athena using Short Characteristics": the angle quadrature (Sec. 3.2), the
short-characteristics formal solution with linear interpolation (Sec. 3.3,
Eq. 20 and the linear upwind-face interpolants), the discrete moments J, H, K
(Eqs. 17-19), the diagonal Lambda operator and the Jacobi ALI update
(Sec. 3.4, Eq. 24) with the convergence test (Eq. 25), and the integral-form
heating rate (Sec. 4).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The CUDA library
never calls it and shares no code with it.

Parity status of each function is listed in ``oracle/README`` style in the
module docstrings: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, invariants or brute force.
"""
