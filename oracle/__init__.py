"""Oracle: a plain, slow, FP64 CPU statement of the space-time predictor of
ADER-DG for Biot's poroelastic equations (Wolf et al., "An Efficient ADER-DG
Local Time Stepping Scheme for 3D HPC Simulation of Seismic Waves in
Poroelastic Media").

This package is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import it.  It shares no code
with the CUDA library and never imports it; the two paths meet only through
the seeded input generator, which holds none of the method's arithmetic.

Module map (each function cites the passage of the paper it restates):
  material   -- material parameters -> Jacobians A, B, C and source matrix E
                (Section "Governing equations", Eq. poroelastic-wave, Eq. biot-dynamic)
  basis      -- Dubiner basis on the reference tetrahedron in exact rational
                arithmetic, mass and stiffness matrices (Section "Spatial
                discretisation"; matrices of Section "Space-Time predictor")
  timebasis  -- shifted-Legendre time basis and the time matrices W, w, S, K^tau
  geometry   -- affine element map, reference Jacobians A*, B*, C*, CFL step
  predictor  -- the predictor system Y Q = r (Eq. stp-lineq) solved by dense LU,
                and Algorithms 1, 2 and 3 written as plain loops
  flops      -- the operation / storage model of Table flop-count
"""
