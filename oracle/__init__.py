"""Plain FP64 CPU oracle for the immersed Newmark IMEX method (arXiv 2310.14712).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_2310_14712_gb300``); the two meet only in
the seeded input generator ``paper_2310_14712_gb300/workloads.py``, which holds
none of the method's arithmetic, and the oracle does not even import that: the
callers hand it plain arrays.

Every function follows a stated passage of the paper, with assembled
``scipy.sparse`` matrices and a library sparse LU as the direct solver, exactly
as the paper's own 2D study does (Sec. "Numerical examples", 2D perforated
plate: "scipy.sparse.linalg.splu").  There is no blocking, fusion or
reordering beyond what the paper states, so the code can be read against it.

Modules
-------
basis        GLL / Gauss-Legendre points, Lagrange basis (Sec. Spatial discretization)
geometry     holes, physical-point test, cell classification (Sec. Spatial discretization, FCM)
discretize   spacetree quadrature, element matrices, assembly, partition
             (Eqs. Mglobal, K, f; Sec. Partitioning, Eqs. MStructure..f_xStructure)
integrators  CDM, trapezoidal Newmark and Newmark IMEX on an assembled system
             (Sec. Time integration, Eqs. Newmark1/2, CDMstep, CDMacc,
             Figs. implicitNewmark and TrapCDMIMEX)
sources      source time functions and spatial bell (Eqs. ft, fx; Ricker)
pipeline     setup + run of one workload (the four steps put together)

Parity status of each function is listed in its module header.  Everything
here is pinned by a ``-m "not gpu"`` test except where a header says
"parity unpinned".
"""
