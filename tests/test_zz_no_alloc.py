"""The allocation-free CFL entry point, for callers that cannot allocate.

Some callers cannot call cudaMalloc when they need a time step (inside a host
callback, under a framework that owns the device allocator, or after all
device memory was reserved).  `dis_cfl_dt_static` serves them from a fixed
scratch area inside the library.  This file is collected last so that a run
stopping at its first failure has already run every other test.

Check: through the C ABI, calls in a row (a stiff 2D state, then a 1D batch
with slower waves, so a stale maximum from the first call would show, then a
reactive 1D state, whose layout has the extra reaction field) give the same
per-patch time steps as the context's own step reports; a patch holding a
cell without a real sound speed gets NaN and the others keep theirs.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2009_14555_gb300 import _lib as L
from paper_2009_14555_gb300 import workloads as W
from paper_2009_14555_gb300.solver import Solver, _material, _patch

pytestmark = pytest.mark.gpu
TOL = 1e-12  # relative; both paths evaluate the same closures in float64


def reference(wl):
    """Conservative state on the device and the dt that dis_step reports."""
    s = Solver.from_workload(wl)
    s.set_prim([p.prim for p in wl.patches])
    cons = torch.empty(s.state_numel, dtype=torch.float64, device="cuda")
    s.get_state(kind=L.DIS_CONSERVATIVE, out=cons)
    dt_ref = s.step(1, return_dt=True)  # dt of a step is computed from the state before it
    s.close()
    return cons, dt_ref


def static_dt(wl, cons):
    lib = L.load()
    pa = (L.DisPatch * len(wl.patches))(*[_patch(p, wl.dim) for p in wl.patches])
    ma = (L.DisMaterial * 2)(*[_material(m) for m in wl.materials])
    dt = torch.full((len(wl.patches),), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.dis_cfl_dt_static(wl.dim, len(wl.patches), pa, ma, wl.reactive_material, wl.cfl,
                               ctypes.c_void_p(cons.data_ptr()), ctypes.c_void_p(dt.data_ptr()),
                               ctypes.c_void_p(stream))
    assert rc == L.DIS_OK, lib.dis_last_error()
    torch.cuda.synchronize()
    return dt.cpu().numpy()


def test_static_dt_matches_step_twice_in_a_row():
    wl_a = W.shock_disc_2d(96, steps=1)                        # stiff solid: fast waves
    wl_b = W.batched_riemann_1d(40, seed=5, steps=1, nmin=32, nmax=200)
    for k, m in enumerate(wl_b.materials):                     # slower waves than wl_a
        wl_b.materials[k] = dict(m, p_inf=0.0, G=0.0)
    cons_a, ref_a = reference(wl_a)
    cons_b, ref_b = reference(wl_b)
    got_a = static_dt(wl_a, cons_a)
    got_b = static_dt(wl_b, cons_b)
    np.testing.assert_allclose(got_a, ref_a, rtol=TOL)
    np.testing.assert_allclose(got_b, ref_b, rtol=TOL)
    assert got_b.max() > got_a.max()  # a stale larger maximum would have shrunk these
    # reactive layout (9 fields in 1D, the reaction field last)
    wl_c = W.detonation_copper_1d(200, steps=1)
    cons_c, ref_c = reference(wl_c)
    np.testing.assert_allclose(static_dt(wl_c, cons_c), ref_c, rtol=TOL)


def test_static_dt_is_nan_for_a_nonphysical_patch():
    wl = W.batched_riemann_1d(6, seed=7, steps=1, nmin=32, nmax=64)
    for k, m in enumerate(wl.materials):                       # two ideal gases
        wl.materials[k] = dict(m, p_inf=0.0, G=0.0)
    cons, ref = reference(wl)
    host = cons.cpu().numpy()
    # negative total energy in one cell of patch 3: negative pressure, c^2 < 0
    off = sum(8 * p.nx for p in wl.patches[:3])
    nx3 = wl.patches[3].nx
    host[off + 4 * nx3 + 5] = -1.0                              # field rho E, cell 5
    got = static_dt(wl, torch.from_numpy(host).cuda())
    assert np.isnan(got[3])
    keep = [k for k in range(6) if k != 3]
    np.testing.assert_allclose(got[keep], ref[keep], rtol=TOL)
    # the flag is cleared on the next call
    np.testing.assert_allclose(static_dt(wl, cons), ref, rtol=TOL)


def test_static_rejects_too_many_patches():
    lib = L.load()
    n = 16385
    pa = (L.DisPatch * n)(*[_patch(W.Patch(nx=8, ny=1, dx=0.1, dy=1.0), 1)] * n)
    ma = (L.DisMaterial * 2)(*[_material(W.AIR)] * 2)
    rc = lib.dis_cfl_dt_static(1, n, pa, ma, -1, 0.8, ctypes.c_void_p(1), ctypes.c_void_p(1), None)
    assert rc == L.DIS_EINVAL
    assert b"16384" in lib.dis_last_error()
