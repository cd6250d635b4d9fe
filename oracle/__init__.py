"""CPU FP64 oracle for the space-time least-squares heat-equation solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
CUDA library never calls it and shares no code with it.

What it computes (Montardini, Negri, Sangalli, Tani, arXiv:1809.10026):

* ``bspline``  -- open uniform knots and the Cox-de Boor recursion (Sec. 2.1).
* ``spaces``   -- 1D Galerkin matrices of the reduced bases (Sec. 2.2, 4.1, 4.2).
* ``system``   -- the system matrix A, both by direct quadrature of the
                  least-squares form (Eq. a-form) and as the Kronecker sum of
                  Eq. A_kron; the load vector F (Sec. 3.2).
* ``fd``       -- the preconditioner P (Eq. preconditioner) and its fast
                  diagonalization solve (Algorithm 1).
* ``solve``    -- direct solve and a textbook (flexible) preconditioned CG.
* ``lifting``  -- the non-zero initial datum lifting (Sec. 3.1) and the adjoint
                  gradient of a quadratic loss.
* ``norms``    -- V0, L2 and H1 errors by Gauss quadrature (Sec. 3.4, 5.1).

Everything is plain numpy/scipy in float64, written for checkability, not
speed.  Parity status of each function is stated in its module docstring.
"""
