"""The FP32-bulk MUSCL-Hancock step (one fused kernel per step) against the
float64 oracle's MUSCL-Hancock form (oracle/hancock.py), through the C ABI,
at the FP32-bulk bars of tests/test_fp32_bulk_gpu.py: per-field relative L1
1e-4, 5e-3 for the partial densities.

The step reads the state and writes the other buffer of a pair, so the tests
also cover odd and even step counts, captured steps of both buffer parities,
state access between calls, and the persistent 1D batch form.
"""
import numpy as np
import pytest

from paper_2009_14555_gb300 import workloads as W
from tests.parity_util import cons_l1, oracle_run
from tests.test_fp32_bulk_gpu import RESULTS, TOL32, TOL32_PARTIAL, check32

pytestmark = pytest.mark.gpu


def _hancock(wl):
    wl.scheme = "hancock"
    return wl


def _bars(wl):
    names = W.cons_names(wl.dim, wl.reactive)
    return names, np.array([TOL32_PARTIAL if n in ("ar1", "ar2", "arl") else TOL32 for n in names])


def test_hancock32_1d_solid_gas():
    check32("hancock_1d_solid_gas_1000_100steps", _hancock(W.solid_gas_1d(1000, steps=100)), 100)


def test_hancock32_2d_shock_disc():
    wl = W.shock_disc_2d(48, steps=40, shock_x=0.27)
    wl.thinc = False
    check32("hancock_2d_shock_disc_48_40steps", _hancock(wl), 40)


def test_hancock32_2d_shock_disc_thinc():
    check32("hancock_2d_shock_disc_thinc_48_40steps",
            _hancock(W.shock_disc_2d(48, steps=40, shock_x=0.27)), 40)


def test_hancock32_2d_reactive_plate():
    check32("hancock_2d_reactive_plate_64x32_20steps", _hancock(W.reactive_plate_2d(64, 32, steps=20)), 20)


def test_hancock32_water_air_thinc():
    water = W.material(4.4, p_inf=6e8)
    wl = W.riemann_1d(257, dict(mat=0, rho=1000.0, u=0.0, p=1e9, rho2=50.0),
                      dict(mat=1, rho=50.0, u=0.0, p=1e5, rho1=1000.0), x_int=0.7, cfl=0.6,
                      thinc=True, materials=[water, W.AIR])
    check32("hancock_1d_water_air_thinc_257_100steps", _hancock(wl), 100)


def test_hancock32_vanleer_reactive_plate():
    wl = _hancock(W.reactive_plate_2d(64, 32, steps=12))
    wl.limiter = "vanleer"
    check32("hancock_2d_reactive_plate_vanleer_64x32_12steps", wl, 12)


def test_hancock32_romenskii_copper_air():
    wl = W.riemann_1d(400, dict(mat=0, rho=8930.0, u=500.0, p=1e5), dict(mat=1, rho=1.2, u=0.0, p=1e5),
                      materials=[W.COPPER_ROMENSKII, W.AIR], steps=60, name="1d_romenskii_copper_air_400")
    check32("hancock_1d_romenskii_copper_air_400_60steps", _hancock(wl), 60)


@pytest.mark.parametrize("variant", range(3))
def test_hancock32_every_2d_variant(variant):
    """Every tile shape on a patch whose sides are multiples of no tile."""
    from paper_2009_14555_gb300.solver import Solver
    wl = _hancock(W.reactive_plate_2d(45, 23, steps=12))
    s = Solver.from_workload(wl, precision="fp32_bulk")
    with pytest.raises(RuntimeError):
        s.set_variant(3)
    s.set_variant(variant)
    s.set_prim([p.prim for p in wl.patches])
    for _ in range(12):
        s.step(1)
    rc, bp, bc = s.check()
    assert rc == 0, (bp, bc)
    g = s.get_arrays()
    s.close()
    o, _ = oracle_run(wl, 12)
    err = cons_l1(wl, g[0], o[0])
    names, bars = _bars(wl)
    RESULTS[f"hancock_2d_reactive_plate_45x23_12steps_variant{variant}"] = dict(steps=12, l1=err.tolist())
    assert (err <= bars).all(), dict(zip(names, err))


def test_hancock32_step_counts_and_buffer_parity():
    """5 steps in one call, as 3 + 2, and as 1 + 1 + 1 + 1 + 1 give the
    bit-identical state (the same kernels on the same data, captured once per
    buffer parity); the state read between calls, dis_query and a per-patch
    load after an odd number of steps see the current buffer."""
    from paper_2009_14555_gb300.solver import Solver
    wl = _hancock(W.reactive_plate_2d(64, 32, steps=5))
    prim = [p.prim for p in wl.patches]
    out = []
    for split in ((5,), (3, 2), (1, 1, 1, 1, 1)):
        s = Solver.from_workload(wl, precision="fp32_bulk")
        s.set_variant(2)
        s.set_prim(prim)
        for n in split:
            s.step(n)
        out.append(s.get_state())
        q = s.query()
        assert q["steps"] == 5 and q["status"] == 0
        nf = len(W.cons_names(2, True))
        vol = wl.patches[0].dx * wl.patches[0].dy
        e = out[-1].reshape(nf, -1)[W.cons_names(2, True).index("E")].sum() * vol
        np.testing.assert_allclose(q["energy"], e, rtol=1e-12)
        s.close()
    for o in out[1:]:
        np.testing.assert_array_equal(o, out[0])
    # a state loaded after an odd number of steps is the one the next step reads
    s = Solver.from_workload(wl, precision="fp32_bulk")
    s.set_variant(2)
    s.set_prim(prim)
    s.step(3)
    s.set_patch(0, prim[0])
    s.step(5)
    np.testing.assert_array_equal(s.get_state(), out[0])
    s.close()


def test_hancock32_batch_schedules():
    """The persistent batch form (all steps of a call in one launch) against
    the per-step launches (float32 rounding: the two are compiled separately)
    and the oracle bar, with an odd step count per call."""
    from paper_2009_14555_gb300.solver import Solver
    wl = _hancock(W.batched_riemann_1d(30, seed=6, steps=31, nmin=16, nmax=1200))
    prims = [p.prim for p in wl.patches]
    runs = {}
    for sched in (0, 1):
        s = Solver.from_workload(wl, precision="fp32_bulk")
        s.set_variant(1)
        s.set_schedule(sched)
        s.set_prim(prims)
        s.step(11)
        s.step(20)
        assert s.schedule()[0] == sched
        rc, bp, bc = s.check()
        assert rc == 0, (bp, bc)
        runs[sched] = (s.get_state(), s.get_arrays())
        s.close()
    nf = len(W.cons_names(wl.dim, wl.reactive))
    a, b = runs[0][0].reshape(nf, -1), runs[1][0].reshape(nf, -1)
    rel = np.abs(a - b).max(axis=1) / np.abs(a).max(axis=1)
    RESULTS["hancock_1d_batch_30_schedules_max_rel_diff"] = rel.tolist()
    assert rel.max() <= 1e-5, rel
    o, _ = oracle_run(wl, 31)
    names, bars = _bars(wl)
    worst = np.zeros(len(names))
    for k in range(len(o)):
        worst = np.maximum(worst, cons_l1(wl, runs[1][1][k], o[k]))
    RESULTS["hancock_1d_batch_30_31steps_persistent"] = dict(steps=31, l1=worst.tolist())
    assert (worst <= bars).all(), dict(zip(names, worst))


def test_hancock32_matches_float64_hancock():
    """FP32-bulk and float64 MUSCL-Hancock on the reactive plate (THINC on):
    the two precisions of one scheme agree to the FP32-bulk bar."""
    from tests.test_parity_gpu import gpu_run
    wl = _hancock(W.reactive_plate_2d(96, 48, steps=30))
    g32, _, _ = gpu_run(wl, 30, precision="fp32_bulk")
    g64, _, _ = gpu_run(wl, 30, precision="fp64")
    err = cons_l1(wl, g32[0], g64[0])
    names, bars = _bars(wl)
    RESULTS["hancock_2d_reactive_plate_96x48_30steps_fp32_vs_fp64"] = err.tolist()
    assert (err <= bars).all(), dict(zip(names, err))
