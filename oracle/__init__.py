"""FP64 CPU oracle for the MI-DELBM per-timestep fluid-particle step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, numpy restatement of
what the method computes (arXiv 2209.10411, Sec. 2.1 Eq. 1 and Sec. 2.3), used
to check the CUDA path.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import it.  The product path (the C-ABI library and its
Python binding) never imports, calls or links anything in here, and nothing in
here imports the product package: the two share no code, no tables and no
constants.

Arithmetic is float64, except where floating point decides an integer that
the kernels decide in FP32 (the convex-hull test and the draws of the shape
fitting, the solid test of the shape descriptors): there the oracle takes the
same decision in FP32 with the same single roundings, and says so.  Each
function names the passage of the paper it follows; where the paper is silent or ambiguous the reading taken is stated in
the function's docstring (the full list of readings, numbered A1..A27, is kept
with the design notes).

Modules
  d3q19     lattice velocities, weights, opposite directions
  lbm       equilibrium, moments, BGK collide (+ Guo forcing), pull streaming
            with halfway bounce-back walls, one bulk step
  metaball  field f, gradient, Hessian; quaternion -> rotation; solid flags;
            mass properties by grid quadrature
  coupling  boundary links and wall fraction q, refill of uncovered nodes,
            interpolated bounce-back, Galilean-invariant momentum exchange,
            one coupled LBM step
  contact   broad phase, Newton-Raphson closest points (pair and wall),
            spring-dashpot forces
  dem       rigid-body update
  step      the whole coupled step in the order flag -> links -> LBM -> DEM
  mlp       learned Newton guess: features, the MLP, its loss and AdamW
  gs        Gradient Search refinement of a metaball model (Algorithm 2)
  ga        Genetic Algorithm capture of a contour (Algorithm 1)
  shape     sphericity, nominal and projected-area diameters, Corey shape
            factor of a metaball model (Sec. 3)

Parity status: every function is pinned by a test under tests/ that checks it
against something other than itself (closed forms, invariants, brute force,
published generator outputs).  The FP16/BF16 storage error and the gain of the
learned Newton guess are measured numbers, not functions of this package.
"""
