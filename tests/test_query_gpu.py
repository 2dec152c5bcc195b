"""dis_query and the per-patch state calls through the C ABI.

dis_query: the device-reduced totals equal the host sums of the packed
conservative state times the cell volume; on a periodic domain mass, momentum
and energy stay constant over the steps (to round-off in float64, to float32
rounding in FP32-bulk), the reported dt range is the one the step returns,
the byte count is the algorithmic state traffic of the call and the kernel
time is positive.  Per-patch calls: setting one patch changes only that
patch; a context steps once every patch holds a state.
"""
import numpy as np
import pytest

from paper_2009_14555_gb300 import _lib as L
from paper_2009_14555_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _host_totals(wl, cons):
    names = W.cons_names(wl.dim, wl.reactive)
    k = {n: i for i, n in enumerate(names)}
    p = wl.patches[0]
    vol = p.dx * p.dy
    a = cons.reshape(len(names), -1)
    return dict(mass=[a[k["ar1"]].sum() * vol, a[k["ar2"]].sum() * vol],
                momentum=[a[k["mx"]].sum() * vol, a[k["my"]].sum() * vol if "my" in k else 0.0],
                energy=a[k["E"]].sum() * vol, phi_min=a[k["phi1"]].min(), phi_max=a[k["phi1"]].max())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32_bulk", 2e-6)])
def test_query_totals_conserved_on_a_periodic_domain(precision, tol):
    from paper_2009_14555_gb300.solver import Solver
    wl = W.smooth_disc_2d(n=48, steps=20, u0=200.0)
    s = Solver.from_workload(wl, precision=precision)
    s.set_prim([p.prim for p in wl.patches])
    q0 = s.query()
    h0 = _host_totals(wl, s.get_state())
    for key in ("mass", "momentum"):
        np.testing.assert_allclose(q0[key], h0[key], rtol=1e-12, atol=1e-12 * abs(h0["energy"]))
    np.testing.assert_allclose(q0["energy"], h0["energy"], rtol=1e-12)
    assert q0["phi_min"] == h0["phi_min"] and q0["phi_max"] == h0["phi_max"]
    assert q0["steps"] == 0 and q0["dt_min"] == 0.0
    dt = s.step(20, return_dt=True)
    q1 = s.query()
    assert q1["status"] == L.DIS_OK and q1["bad_patch"] == -1
    assert q1["steps"] == 20 and q1["kernel_ms"] > 0
    assert q1["dt_min"] == dt.min() and q1["dt_max"] == dt.max()
    nf = len(W.cons_names(wl.dim, wl.reactive))
    per_cell = 8 * nf if precision == "fp64" else 4 * (nf + 1)
    assert q1["bytes"] == 2 * per_cell * wl.cells * 20
    scale = abs(q0["energy"])
    for l in (0, 1):
        assert abs(q1["mass"][l] - q0["mass"][l]) <= tol * abs(q0["mass"][l])
    ref = np.sqrt(abs(q0["energy"]) * (q0["mass"][0] + q0["mass"][1]))  # momentum scale ~ rho c
    for d in (0, 1):
        assert abs(q1["momentum"][d] - q0["momentum"][d]) <= tol * ref
    assert abs(q1["energy"] - q0["energy"]) <= tol * scale
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_per_patch_state_set_and_get(precision):
    from paper_2009_14555_gb300.solver import Solver
    wl = W.batched_riemann_1d(3, seed=9, steps=5, nmin=40, nmax=90)
    shapes = [p.prim.shape for p in wl.patches]
    s = Solver.from_workload(wl, precision=precision)
    # a context without every patch set does not step
    s.set_patch(0, wl.patches[0].prim)
    s.set_patch(2, wl.patches[2].prim)
    with pytest.raises(RuntimeError):
        s.step(1)
    s.set_patch(1, wl.patches[1].prim)
    whole = s.get_arrays()
    # the same as the whole-state call
    ref = Solver.from_workload(wl, precision=precision)
    ref.set_prim([p.prim for p in wl.patches])
    for a, b in zip(whole, ref.get_arrays()):
        np.testing.assert_array_equal(a, b)
    # replace patch 1 only (mirrored, pressure x 1.5); the others are untouched
    new1 = wl.patches[1].prim[:, :, ::-1].copy()
    names = W.prim_names(wl.dim, wl.reactive)
    new1[names.index("u")] *= -1.0
    new1[names.index("p")] *= 1.5
    s.set_patch(1, new1)
    ref1 = Solver.from_workload(wl, precision=precision)
    ref1.set_prim([wl.patches[0].prim, new1, wl.patches[2].prim])
    for k in range(3):
        np.testing.assert_array_equal(s.get_patch(k, whole[k].shape), ref1.get_arrays()[k])
    # primitive export of one patch
    np.testing.assert_array_equal(s.get_patch(1, shapes[1], kind=L.DIS_PRIMITIVE),
                                  ref1.get_arrays(kind=L.DIS_PRIMITIVE)[1])
    # stepping after per-patch loads matches the whole-state load (same
    # kernels: the FP32-bulk variant and schedule are fixed)
    if precision == "fp32_bulk":
        for x in (s, ref1):
            x.set_variant(0)
            x.set_schedule(0)
    s.step(5)
    ref1.step(5)
    for a, b in zip(s.get_arrays(), ref1.get_arrays()):
        np.testing.assert_array_equal(a, b)
    for x in (s, ref, ref1):
        x.close()
