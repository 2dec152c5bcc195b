"""Reference oracle for the diffuse-interface finite-volume step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 CPU
restatement (PyTorch CPU tensor ops) of the explicit step of Wallis, Barton &
Nikiforakis, "A Diffuse Interface Model of Reactive-fluids and
Solid-dynamics" (arXiv 2009.14555), Sections 2-3 and Appendices A-B.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark may import
it; the CUDA library never does, and it shares no code with it.

Modules:
  closures        equations of state, mixture rules, strain, stress (Sec. 2.2-2.3, App. B)
  reconstruction  MUSCL, THINC, BVD, Youngs normal (Sec. 3.1, App. A)
  riemann         HLLD-type elastic Riemann solver (Sec. 3.1; a reading of the
                  unprinted HLLD of Barton 2019, from the jump conditions)
  scheme          ghost cells, spatial operator, RK3, CFL, plastic and reactive
                  updates (Arrhenius or k sqrt(lam) rate), cylindrical
                  geometric source (Sec. 3, 3.1-3.3, 4.1)
  hancock         single-stage MUSCL-Hancock form of the hyperbolic update
  adjoint         reverse mode of the step (PyTorch autograd through the above)

Pins live in tests/test_oracle_*.py: exact Riemann solutions, closed forms,
invariants, convergence orders and brute-force checks, one or more per
function.  Whole 2D runs (shock-disc, reactive plate) have no closed form; on
top of their functions' pins they are checked through conservation,
boundedness and symmetry.
"""
from .scheme import (run, step, spatial_operator, cfl_dt, cfl_rate, plastic_update,  # noqa: F401
                     reaction_update, prim_from_array, cons_from_array, cons_to_array,
                     prim_to_array, grid_of, fill_ghosts, NG)
from .closures import prim_to_cons, cons_to_prim, hencky_dev  # noqa: F401
