"""Parity at full problem sizes, in the launch configuration the benchmark uses.

The oracle cannot step a 2048 x 1024 grid in seconds, so each check runs the
GPU on the full grid and the oracle on sampled windows of the same seeded
input: one step needs a margin of 9 cells (3 stages x 3 ghost layers), the
window edges inside the domain get transmissive ghosts (which only disturb the
margin), and edges on the domain boundary keep the real boundary condition.
Both sides take the oracle's CFL time step of the full grid (pointwise, cheap).
Batched problems are checked on a sample of whole problems.
"""
import numpy as np
import pytest
import torch

from oracle import closures as OC
from oracle import scheme as OS
from paper_2009_14555_gb300 import workloads as W
from paper_2009_14555_gb300.solver import Solver
from tests.parity_util import cons_l1

pytestmark = pytest.mark.gpu
M = 9  # margin cells for one step


def full_dt(wl, patch):
    q = OC.prim_to_cons(OS.prim_from_array(patch.prim, wl.dim, wl.reactive), wl.materials)
    return OS.cfl_dt(q, OS.grid_of(patch, wl.dim), wl.materials, wl.cfl)


def oracle_window(wl, patch, j0, j1, i0, i1, dt):
    ny, nx = patch.prim.shape[1:]
    a, b = max(j0 - M, 0), min(j1 + M, ny)
    c, d = max(i0 - M, 0), min(i1 + M, nx)
    sub = W.Patch(nx=d - c, ny=b - a, dx=patch.dx, dy=patch.dy,
                  bc=(patch.bc[0] if c == 0 else W.BC_TRANSMISSIVE,
                      patch.bc[1] if d == nx else W.BC_TRANSMISSIVE,
                      patch.bc[2] if a == 0 else W.BC_TRANSMISSIVE,
                      patch.bc[3] if b == ny else W.BC_TRANSMISSIVE),
                  prim=patch.prim[:, a:b, c:d])
    q = OC.prim_to_cons(OS.prim_from_array(sub.prim, wl.dim, wl.reactive), wl.materials)
    q, _ = OS.step(q, OS.grid_of(sub, wl.dim), wl.materials, dict(cfl=wl.cfl, thinc=wl.thinc), dt)
    out = OS.cons_to_array(q, wl.dim, wl.reactive).numpy()
    return out[:, j0 - a:j1 - a, i0 - c:i1 - c]


def run_full(wl, dt, precision):
    s = Solver.from_workload(wl, precision=precision)
    s.set_prim([p.prim for p in wl.patches])
    s.step_fixed_dt(1, dt)
    rc, _, _ = s.check()
    assert rc == 0
    out = s.get_arrays()
    s.close()
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_bulk", 1e-4)])
def test_reactive_plate_2048x1024_sampled(precision, tol):
    wl = W.reactive_plate_2d()  # the benchmark workload (THINC on)
    p = wl.patches[0]
    dt = full_dt(wl, p)
    g = run_full(wl, dt, precision)[0]
    windows = [(300, 316, 1016, 1032),   # hot spot
               (196, 212, 500, 516),     # plate surface
               (0, 12, 0, 12),           # domain corner: two boundaries
               (1012, 1024, 2036, 2048),  # opposite corner
               (600, 616, 1700, 1716)]   # far field
    for (j0, j1, i0, i1) in windows:
        o = oracle_window(wl, p, j0, j1, i0, i1, dt)
        err = cons_l1(wl, g[:, j0:j1, i0:i1], o)
        assert err.max() <= tol, ((j0, i0), err)


def test_shock_disc_512_sampled():
    wl = W.shock_disc_2d(512)
    p = wl.patches[0]
    dt = full_dt(wl, p)
    g = run_full(wl, dt, "fp64")[0]
    for (j0, j1, i0, i1) in [(120, 136, 120, 136), (250, 262, 140, 156), (0, 10, 500, 512)]:
        o = oracle_window(wl, p, j0, j1, i0, i1, dt)
        err = cons_l1(wl, g[:, j0:j1, i0:i1], o)
        assert err.max() <= 1e-10, ((j0, i0), err)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_bulk", 5e-3)])
def test_batched_4096_sampled_problems(precision, tol):
    wl = W.batched_riemann_1d()  # 4096 problems, 256-4096 cells each
    dts = np.array([full_dt(wl, p) for p in wl.patches])
    s = Solver.from_workload(wl, precision=precision)
    s.set_prim([p.prim for p in wl.patches])
    s.step_fixed_dt(2, dts)
    assert s.check()[0] == 0
    g = s.get_arrays()
    s.close()
    rng = np.random.default_rng(7)
    for k in rng.choice(len(wl.patches), 12, replace=False):
        p = wl.patches[k]
        o, _ = OS.run(p.prim, 1, wl.materials, OS.grid_of(p, 1), dict(cfl=wl.cfl, thinc=False), 2,
                      [dts[k]] * 2)
        err = cons_l1(wl, g[k], o.numpy())
        assert err.max() <= tol, (k, p.nx, err)
