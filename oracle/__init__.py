"""FP64 CPU oracle for the field-split GMG-preconditioned FGMRES FSI solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline and reference legs) may import this package.
It shares no code with the CUDA library: it imports only numpy, scipy and the
seeded problem generator ``paper_1909_13201_gb300.inputs`` (problem data, no
solver arithmetic).

Modules, each citing the passage of the paper it follows:
  fem       Q2/Q1 reference-element integrals (Gauss rule)      Sec. 2.2, Q2 spaces
  mesh      level hierarchy, materials, node classes, J2 dofs    Sec. 3.2 (J2), Sec. 3.3
  assemble  linearised monolithic operator in J2 order          Eqs. kinsld-cntfld, matrix_J2
  transfer  prolongation P2 and equation-aware restriction R2   Sec. 3.3
  fsasm     field-split additive Schwarz smoother (AS1, AS2)     Sec. 3.2, FS / AS1 / AS2
  gmg       V-cycle with damped Richardson smoothing            Sec. 3.2
  fgmres    restarted flexible GMRES, CGS2, Givens              Sec. 3.2 (outer Krylov)
  adjoint   transposed solve and gradients                      (extension; no paper passage)
"""
