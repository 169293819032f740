"""FP64 CPU oracle of the pixel-aligned occupancy field, its hierarchical
surface localization and the mesh-free render (Li et al., arXiv 2007.13988,
Sec. 3.1 Eq. 1-2 and Sec. 3.2 Eq. 3).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the CUDA path computes.  Only the test-suite, the package's
smoke check and the benchmark's CPU-baseline leg may import it; the library
and its Python binding never do.  It shares no code with the CUDA path: it
reads the generator's arrays (float32 inputs, promoted to float64 here) and
nothing else.

Modules
-------
field     Eq. 1 / Eq. 2: projection, bilinear sampling Phi, the MLPs, and the
          analytic capsule occupancy used to pin the localization.
localize  Sec. 3.2 "Octree-based Robust Surface Localization": dense
          (brute-force) evaluation and the coarse-to-fine algorithm.
render    Sec. 3.2 "Mesh-free Rendering": first 0.5 crossing per pixel ray,
          surface point, Eq. 3 colour.
metrics   IoU, Chamfer distance in voxels, PSNR.

Parity pins live in tests/test_oracle_*.py.  Unpinned parts are named in each
module's header.
"""
