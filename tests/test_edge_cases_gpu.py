"""Degenerate and boundary-size inputs through the C ABI, both precisions:
a uniform state at rest is a fixed point of the step (bit for bit); zero
steps leave the state untouched; the smallest accepted patches (4 cells a
side), batched with different cell sizes and boundary conditions, match the
oracle."""
import copy

import numpy as np
import pytest

from paper_2009_14555_gb300 import workloads as W
from tests.parity_util import cons_l1, oracle_run

pytestmark = pytest.mark.gpu


def _uniform(dim, n, phi1):
    names = W.prim_names(dim, False)
    k = {f: i for i, f in enumerate(names)}
    ny = n if dim == 2 else 1
    w = np.zeros((len(names), ny, n))
    w[k["phi1"]] = phi1
    w[k["rho1"]] = W.SOLID_RHO0
    w[k["rho2"]] = 1.2
    w[k["p"]] = 2e5
    for f in ("V11", "V22", "V33"):
        w[k[f]] = 1.0
    per = (W.BC_PERIODIC,) * 4
    p = W.Patch(nx=n, ny=ny, dx=1.0 / n, dy=1.0 / n if dim == 2 else 1.0, bc=per, prim=w)
    return W.Workload(f"uniform_{dim}d", dim, [W.SOLID, W.AIR], [p], 0.6, 10, dim == 2)


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
@pytest.mark.parametrize("dim", [1, 2])
def test_uniform_state_at_rest_is_a_fixed_point(precision, dim):
    from paper_2009_14555_gb300.solver import Solver
    wl = _uniform(dim, 37, 0.3)  # a mixed cell everywhere: THINC (2D) and both materials active
    s = Solver.from_workload(wl, precision=precision)
    s.set_prim([p.prim for p in wl.patches])
    q0 = s.get_state()
    s.step(10)
    assert s.check()[0] == 0
    q1 = s.get_state()
    s.close()
    assert np.array_equal(q0, q1)


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_zero_steps_leave_the_state_untouched(precision):
    from paper_2009_14555_gb300.solver import Solver
    wl = W.shock_disc_2d(20, steps=1)
    s = Solver.from_workload(wl, precision=precision)
    s.set_prim([p.prim for p in wl.patches])
    q0 = s.get_state()
    s.step(0)
    s.step_fixed_dt(0, 1e-9)
    assert np.array_equal(q0, s.get_state())
    s.close()


def test_smallest_patches_batched_match_oracle():
    """1D: patches of 4..7 cells with different widths and boundaries in one
    batch; each patch is an independent problem with its own dt."""
    from tests.test_parity_gpu import gpu_run
    base = W.batched_riemann_1d(8, seed=9, steps=20, nmin=4, nmax=8)
    wl = copy.deepcopy(base)
    bcs = [W.BC_TRANSMISSIVE, W.BC_PERIODIC, W.BC_REFLECTIVE]
    for b, p in enumerate(wl.patches):
        p.dx = (1.0 + 0.5 * b) / p.nx
        p.bc = (bcs[b % 3], bcs[(b + 1) % 3], W.BC_TRANSMISSIVE, W.BC_TRANSMISSIVE)
        # gentle states: tiny patches with strong waves would cavitate
        names = W.prim_names(1, False)
        k = {f: i for i, f in enumerate(names)}
        p.prim[k["u"]] *= 0.05
        p.prim[k["p"]] = np.clip(p.prim[k["p"]], 1e5, 1e6)
    g, _, _ = gpu_run(wl, 20)
    o, _ = oracle_run(wl, 20)
    for k in range(len(o)):
        assert cons_l1(wl, g[k], o[k]).max() <= 1e-10, k


def test_smallest_2d_patch_matches_oracle():
    from tests.test_parity_gpu import gpu_run
    wl = W.perturbed(W.smooth_disc_2d(n=4, steps=10))
    wl.patches[0].dy = 0.5 / 4  # anisotropic cells
    g, _, _ = gpu_run(wl, 10)
    o, _ = oracle_run(wl, 10)
    assert cons_l1(wl, g[0], o[0]).max() <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_async_transfers_match_synchronous_calls(precision):
    """Pipelined transfers (set_state_async / step / get_state_async, three
    rounds in flight, one dis_sync) give the states the synchronous calls
    give, bit for bit, in every round's own output buffer."""
    import torch
    from paper_2009_14555_gb300.solver import Solver, pack
    wl = W.reactive_plate_2d(64, 32, steps=2)
    prim = pack([p.prim for p in wl.patches])
    s = Solver.from_workload(wl, precision=precision)
    s.set_state(prim)
    s.step(2)
    ref = s.get_state()
    hin = torch.from_numpy(prim.copy()).pin_memory()
    outs = [torch.full((s.state_numel,), float("nan"), dtype=torch.float64).pin_memory() for _ in range(3)]
    for k in range(3):
        s.set_state_async(hin)
        s.step(2)
        s.get_state_async(outs[k])
    s.sync()
    s.close()
    for k in range(3):
        assert np.array_equal(outs[k].numpy(), ref), k
