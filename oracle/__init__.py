"""CPU FP64 oracle for the power-series H-matrix EFIE (and CFIE) solve (arXiv 2109.04129).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, NumPy float64
statement of the method, written from the paper, used to check the GPU library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The GPU library never calls into it and shares no
code with it; the only common inputs are the meshes and incidence angles from
``hm_workloads``.

Modules, in the order the method uses them:

  quadrature   7-point degree-5 triangle rule
  potentials   closed-form integrals of 1/R, rho/R and (r-r')/R^3 over a triangle
  rwg          RWG basis on a triangle mesh                  (Sec. II)
  efie         EFIE Galerkin entries and plane-wave RHS      (Eq. 1-3, 9)
  mfie         MFIE and CFIE entries and RHS                 (Eq. 4-8)
  octree       octree clusters, admissibility, block tree   (Eq. 10, 13)
  aca          partially pivoted ACA + recompression        (Eq. 11-12)
  hmatrix      near/far block store and its products        (Eq. 13)
  scaling      Schur-complement scaling coefficients        (Eq. 14-29)
  series       two-term (or n-term) power series            (Eq. 30-45)
  nonsym       non-symmetric H-matrix, left and right scaling
               coefficients and series for the CFIE         (Eq. 8, 14-36)
  rcs          radiation integral, RCS, Mie series           (Sec. V)
  export       writer of the neutral block file the GPU library imports
  cefie        plain-C statement of the EFIE entry (fast fills for large meshes)
  study_leaf_size  series accuracy against the leaf size  (Sec. V-A, Fig. 4)
  study_fill       near-field and scaling-coefficient memory against N
  study_mixed_error  precision model of the mixed path (not in the paper)
               (the three studies run from the command line; they are not
               steps of the method)

Parity status of every function is listed in its module docstring; functions
without an independent pin say "parity unpinned".
"""
