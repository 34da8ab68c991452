"""Oracle: a plain, slow FP64 CPU restatement of the paper's method.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package. The
library's product path never calls it and shares no code with it.

Pearson, Porcelli, Stoll, "Interior point methods and preconditioning for
PDE-constrained optimization problems involving sparsity terms" (2018):

* ``fem``    -- Q1 Galerkin matrices L (stiffness, or convection-diffusion with
               SUPG) and M, the lumped D and D_M = diag(M) (Section 2).
* ``qp``     -- the quadratic program (pb_fe_lin) in (y, z = [w; v]) with its
               bounds z_a, z_b (Section 2).
* ``ipm``    -- Algorithm A.1 (Appendix) with the reduced Newton system
               (NewtonSystem, Section 3) solved by a sparse direct solver,
               the multiplier steps (zupdate1-4), step lengths and the
               feasibility / complementarity measures (prdu), (gap).
* ``brute``  -- the discrete problem (pb_fe)+(boxvector) solved directly by
               cyclic coordinate descent on tiny grids (plain definition).
* ``linear_kkt`` -- the beta = 0, inactive-box optimum from one linear solve.
* ``blocks`` -- dense block matrices of Section 4 (A, B, S, the Schur formula
               (Schur), the matching approximation (SchurApprox) with M-hat,
               the 2x2 z-block approximation, Chebyshev semi-iteration) for
               checking preconditioner algebra on tiny grids.
"""
