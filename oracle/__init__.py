"""CPU oracle for the FMM-accelerated Helmholtz BEM (Gumerov & Duraiswami,
"Fast multipole accelerated boundary element methods for room acoustics").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the test suite, the package's ``smoke()`` self-check and the
``cpu_baseline`` / reference leg of ``bench.py`` may call it.  It is a plain,
slow, obviously-correct FP64 restatement of what the GPU path computes, written
in numpy/scipy, and shares no code with the CUDA sources.

Modules
  geometry   element centroids, normals, areas, Gauss rules on triangles
  integrals  closed-form flat-triangle integrals of 1/R, grad(1/R), solid angle
  bem        dense collocation matrices L, M, L', the Eq. (dbem4) system, RHS
  fgmres     flexible GMRES in FP64
  images     image-source sums, Eq. (an2)
  sph        spherical basis functions, coaxial recursions (Sec. 3.3.1),
             rotation blocks, composed translations
  octree     uniform octree, U/V interaction lists
  fmmops     per-box P2M / L2P operators (definitions)
  fmm        a plain FMM matvec assembled from the pieces above
"""
