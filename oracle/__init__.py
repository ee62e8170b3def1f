"""CPU oracle for the three-grid IOFD Helmholtz solver -- TEST INFRASTRUCTURE.

A plain, slow, complex128 NumPy/SciPy restatement of the method of
"A Massively Parallel Three-Grid Preconditioner for the High-Frequency
Helmholtz Equation" (Fu, Wang, Zhao): the IOFD operator of Sec. 2, the
three-grid preconditioner of Sec. 3 / Algorithm 1 and the outer FGMRES.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU
library (``paper_2608_22946_gb300``); the only common inputs are the seeded
workloads of ``hz_workloads`` and the IOFD coefficient table file, which is
an input of the method (the paper takes it from Stolk 2016).

Modules:
  iofd       -- PML, velocity extension, level grids, IOFD row coefficients,
                matrix-free A, B, Q and their adjoints, an independent
                Kronecker-assembled sparse builder, point sources.
  threegrid  -- transfers, damped Jacobi, GMRES / FGMRES cycles, the shifted
                V-cycle, the 2h Krylov solve, the fine smoother, Algorithm 1,
                the outer FGMRES solve.
  gradient   -- receiver misfit and adjoint-state gradient with respect to
                the squared slowness m = 1/c^2.

Parity status: every function is pinned by a ``-m "not gpu"`` test (closed
forms, symbols, brute force, sparse direct solves, dot tests, finite
differences) except the PC-call counts of the full solver, which depend on
the unpublished IOFD tables: parity unpinned for those counts only.
"""
