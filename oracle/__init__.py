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
  riemann         HLLC-type elastic Riemann solver (Sec. 3.1; reading of the
                  unprinted HLLD of Barton 2019)
  scheme          ghost cells, spatial operator, RK3, CFL, plastic and reactive
                  updates (Sec. 3, 3.1-3.3)

Parity pins live in tests/test_oracle_*.py.  Functions without an independent
pin are listed as "parity unpinned" there and in the design notes: the full 2D
shock-disc and reactive-plate dynamics (checked only through conservation,
boundedness and symmetry).
"""
from .scheme import (run, step, spatial_operator, cfl_dt, cfl_rate, plastic_update,  # noqa: F401
                     reaction_update, prim_from_array, cons_from_array, cons_to_array,
                     prim_to_array, grid_of, fill_ghosts, NG)
from .closures import prim_to_cons, cons_to_prim, hencky_dev  # noqa: F401
