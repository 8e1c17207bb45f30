"""Plain FP64 CPU oracle for the 1D two-level-atom CRD polarized transfer
problem of Benedusi, Janett, Belluzzi & Krause (2021), "Numerical solutions to
linear transfer problems of polarized radiation II. Krylov methods and
matrix-free implementation".

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is written to be read against the paper, not to be fast: numpy arrays
stand in for the loops over rays, and a loop over heights carries the depth
recurrence.  It shares no code with the CUDA path; both only read the seeded
inputs of ``rt_workloads``.

Modules
  grids    -- Gauss-Legendre angles, Voigt profile, spectral weights (Sect. 3.1, 4.1)
  formal   -- formal solvers: DELO-linear, implicit Euler, trapezoidal (Eq. 9-10)
  transfer -- T, Lambda, J, the sigma-form (Eq. 18) and I-form (Eq. 19)
              operators, right-hand sides, Jacobi diagonals, assembly and the
              exact LU solution (Algorithm 1, Sect. 3.3, Sect. 4.4)
  krylov   -- textbook GMRES(m), BiCGSTAB, CGS and Richardson (Sect. 2)
  stationary -- SOR and SSOR preconditioners of the assembled sigma-form
              matrix (Sect. 2.3, with the readings that reproduce Tables 4-5)

Parity status of each function is stated in its docstring; every function is
pinned by ``tests/test_oracle_*.py`` except where a docstring says
"parity unpinned".
"""
