"""Plain, slow FP64 CPU oracle for the HT / CP explicit time step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run anything
in this package.  The CUDA library never links, imports or calls it, and it shares
no code with the CUDA path (the seeded input generators in
``paper_1803_10270_gb300.inputs`` are the only module both sides read).

Modules
- ``tree``     balanced and linear (tensor-train) dimension trees (Section 2.2, eqs. HTD / coreT)
- ``fullgrid`` full-grid finite-difference RK2 / AB2 steppers for small grids
- ``jacobi``   one-sided (Hestenes) Jacobi SVD, written out
- ``ht``       hierarchical Tucker tensors: full conversion, operator application
               (eq. Lz, Section 3.2), orthogonalisation and root-to-leaves HSVD truncation,
               RK2 / HEUN2 / AB2 steps
- ``cp``       canonical tensors and ALS (eqs. functional-SSE, als, SSYSTEM, A^{ln}_{jhp})
- ``problems`` the operators' 1-D factors: constant- and variable-coefficient advection
               (Table tab:ordering0), the linearised kinetic operator (Table tab:ordering)
- ``cn_als``   the implicit Crank-Nicolson step solved by CP-ALS (Section 3.3, eqs. ALS2 /
               ML / MR; Gauss-Seidel and the damped-Jacobi variant of Appendix B)

Every function names the passage it follows.  Parity status of each function is
listed at the top of its module; a function no independent check pins says
"parity unpinned".
"""
