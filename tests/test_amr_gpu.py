"""The structured AMR hierarchy (dis_amr_*; Section 3, the AMR platform
paragraph; Section 4.2 flagging) against the oracle's hierarchy
(oracle/amr.py) through the C ABI, float64: the same levels and blocks (the
cell masks of every level equal), the same level-0 time steps (rtol 1e-12),
and every owned cell of every level at the parity bar (the R19 metric of
tests/parity_util.py over the owned cells: per-field relative L1 1e-10,
element-wise 1e-8).  Cases with THINC next to the stiff solid take the bars
max(1e-10, 10 x the oracle's one-ulp spread) for the fields and
max(1e-12, 10 x that spread) for the time steps: one-ulp input
perturbations flip THINC-BVD choices of the oracle itself, which moves its
fields and, through the CFL rate, its time steps.
"""
import numpy as np
import pytest
import torch

from oracle import amr as A
from oracle import closures as C
from oracle import scheme as S
from paper_2009_14555_gb300 import workloads as W
from tests.parity_util import cons_l1, cons_max, record

pytestmark = pytest.mark.gpu
TOL, TOL_MAX = 1e-10, 1e-8


def _oracle(wl, **kw):
    p = wl.patches[0]
    q = C.prim_to_cons(S.prim_from_array(p.prim, wl.dim, wl.reactive), wl.materials)
    return A.Hierarchy(q, S.grid_of(p, wl.dim, wl.geometry), wl.materials,
                       dict(cfl=wl.cfl, thinc=wl.thinc, scheme=wl.scheme), **kw)


def _gpu(wl, **kw):
    from paper_2009_14555_gb300.solver import AmrSolver
    s = AmrSolver(wl, max_levels=kw["max_level"], block=kw["block"], eps=kw["eps"], buffer=kw.get("buffer", 2),
                  regrid_every=kw.get("regrid_every", 4))
    s.set_prim(wl.patches[0].prim)
    return s


def _spread(wl, steps, o, odts, **kw):
    """Per-field L1 (R19 metric, owned cells) between the oracle hierarchy and
    the oracle hierarchy on inputs perturbed by one ulp (random sign), and
    the largest relative difference of their level-0 time steps."""
    import copy
    rng = np.random.default_rng(123)
    wp = copy.deepcopy(wl)
    for p in wp.patches:
        p.prim = p.prim * (1 + np.sign(rng.standard_normal(p.prim.shape)) * 2.0 ** -52)
    op = _oracle(wp, **kw)
    pdts = [op.step() for _ in range(steps)]
    dt_spread = float(np.max(np.abs(np.asarray(pdts) / np.asarray(odts) - 1.0)))
    out = []
    for l in range(min(op.n_levels(), o.n_levels())):
        act = (o.active[l] & op.active[l]).numpy().reshape(-1)
        a = np.asarray(S.cons_to_array(o.q[l], wl.dim, wl.reactive)).reshape(-1, act.size)[:, act]
        b = np.asarray(S.cons_to_array(op.q[l], wl.dim, wl.reactive)).reshape(-1, act.size)[:, act]
        out.append(cons_l1(wl, b, a))
    return np.max(out, axis=0), dt_spread


def compare(wl, steps, name, calibrate=False, **kw):
    o = _oracle(wl, **kw)
    g = _gpu(wl, **kw)
    n, counts = g.levels()
    assert n == o.n_levels(), (n, o.n_levels())
    odts = [o.step() for _ in range(steps)]
    gdts = g.step(steps)
    rc = g.check()
    assert rc[0] == 0, rc
    dt_bar = 1e-12
    if calibrate:  # the level-0 dt moves with the THINC-BVD choices too
        spread, dt_spread = _spread(wl, steps, o, odts, **kw)
        dt_bar = max(1e-12, 10.0 * dt_spread)
    np.testing.assert_allclose(gdts, odts, rtol=dt_bar)
    n, counts = g.levels()
    assert n == o.n_levels(), (n, o.n_levels())
    errs, maxs = [], []
    for l in range(n):
        ga, act = g.get_level(l)
        assert np.array_equal(act, o.active[l].numpy()), f"level {l} blocks differ"
        oa = np.asarray(S.cons_to_array(o.q[l], wl.dim, wl.reactive))
        ga = ga.reshape(ga.shape[0], -1)[:, act.reshape(-1)]
        oa = oa.reshape(oa.shape[0], -1)[:, act.reshape(-1)]
        errs.append(cons_l1(wl, ga, oa))
        maxs.append(cons_max(wl, ga, oa))
    err = np.max(errs, axis=0)
    emax = np.max(maxs, axis=0)
    g.close()
    if calibrate:
        bar = np.maximum(TOL, 10.0 * spread)
        dt_err = float(np.max(np.abs(np.asarray(gdts) / np.asarray(odts) - 1.0)))
        record(name, steps=steps, l1=err, max_rel=emax, levels=int(n), blocks=counts, oracle_spread_l1=spread,
               bar=bar, dt_rel_err=dt_err, oracle_dt_spread=dt_spread)
        assert (err <= bar).all(), (err, spread)
        return o
    record(name, steps=steps, l1=err, max_rel=emax, levels=int(n), blocks=counts)
    assert err.max() <= TOL, err
    assert emax.max() <= TOL_MAX, emax
    return o


def test_amr_1d_solid_gas_three_levels():
    compare(W.solid_gas_1d(128, steps=8), 8, "amr_1d_solid_gas_128_3levels_8",
            max_level=3, block=8, eps=0.05, regrid_every=2)


def test_amr_1d_periodic():
    wl = W.solid_gas_1d(64, steps=8)
    wl.patches[0].bc = [S.BC_PERIODIC] * 4
    compare(wl, 8, "amr_1d_periodic_64_3levels_8", max_level=3, block=8, eps=0.05, regrid_every=2)


def test_amr_2d_shock_disc():
    wl = W.shock_disc_2d(64, steps=6, shock_x=0.3)
    wl.thinc = False
    compare(wl, 6, "amr_2d_shock_disc_64_2levels_6", max_level=2, block=8, eps=0.3, regrid_every=2)


def test_amr_2d_shock_disc_three_levels():
    wl = W.shock_disc_2d(64, steps=4, shock_x=0.3)
    wl.thinc = False
    compare(wl, 4, "amr_2d_shock_disc_64_3levels_4", max_level=3, block=8, eps=0.3, regrid_every=2)


def test_amr_2d_shock_disc_thinc():
    """THINC with the shock starting at the disc's edge: the one-ulp
    differences of the initial conversion flip a THINC-BVD choice in the
    first step (the oracle's own one-ulp spread shows it), so the bar is
    max(1e-10, 10 x that spread), as for the single-grid THINC cases."""
    wl = W.shock_disc_2d(64, steps=4, shock_x=0.3)
    compare(wl, 4, "amr_2d_shock_disc_thinc_64_2levels_4", calibrate=True, max_level=2, block=8, eps=0.3,
            regrid_every=2)


def test_amr_1d_cylinder_core():
    """Cylindrical geometry (Section 3, cylindrical symmetry) with the axis
    at x = 0 (reflective): air at 5e6 Pa implodes onto a solid core; every
    level takes the geometric source at its own cell-centre radii."""
    compare(W.cylinder_core_1d(128, steps=8), 8, "amr_1d_cylinder_core_128_3levels_8",
            max_level=3, block=8, eps=0.05, regrid_every=2)


def test_amr_1d_off_axis_annulus():
    """An annulus r in [0.25, 1.25] (reflective inner wall): the blocks'
    radii start from the domain's x0."""
    compare(W.cylinder_core_1d(128, steps=8, x0=0.25, r_core=0.5), 8, "amr_1d_annulus_128_3levels_8",
            max_level=3, block=8, eps=0.05, regrid_every=2)


def test_amr_2d_sphere_shock_rz():
    """(r, z): the shock meets the solid sphere on the axis in the first
    steps, so the refined blocks carry radial motion (geometric source) next
    to the reflective axis."""
    wl = W.sphere_shock_rz(64, steps=6, thinc=False, shock_z=0.29)
    compare(wl, 6, "amr_2d_sphere_shock_rz_64_2levels_6", max_level=2, block=8, eps=0.3, regrid_every=2)


def test_amr_2d_sphere_shock_rz_thinc():
    """The same with THINC: bar 1e-10 or 10 x the oracle's one-ulp spread
    (THINC next to the stiff solid)."""
    wl = W.sphere_shock_rz(64, steps=6, thinc=True, shock_z=0.29)
    compare(wl, 6, "amr_2d_sphere_shock_rz_thinc_64_2levels_6", calibrate=True, max_level=2, block=8, eps=0.3,
            regrid_every=2)


def test_amr_2d_reactive_plate():
    wl = W.reactive_plate_2d(64, 32, steps=4)
    compare(wl, 4, "amr_2d_reactive_plate_64x32_2levels_4", max_level=2, block=8, eps=0.2, regrid_every=2)


def test_amr_detonation_section_4_1():
    """The one-dimensional test of Section 4.1 in the paper's AMR setting (a
    base grid and two more levels of ratio 2): the generic explosive (two
    closures, the Appendix B root finder) against Romenskii copper, THINC on;
    200 base cells (the paper: 1000), 30 level-0 steps; bar 1e-10 or 10 x the
    oracle's one-ulp spread."""
    wl = W.detonation_copper_1d(200, steps=30, explosive="generic")
    compare(wl, 30, "amr_detonation_generic_200_3levels_30", calibrate=True, max_level=3, block=8, eps=0.1,
            regrid_every=2)


def test_amr_conservation_periodic_2d():
    """Composite totals of the conservative rows on a periodic domain stay
    constant to round-off (refluxing and average-down on the GPU)."""
    from paper_2009_14555_gb300.solver import AmrSolver
    wl = W.smooth_disc_2d(n=64, steps=1, u0=150.0)
    g = AmrSolver(wl, max_levels=2, block=8, eps=0.5, buffer=0, regrid_every=2)
    g.set_prim(wl.patches[0].prim)
    n, counts = g.levels()
    assert n == 2 and 0 < counts[1] < 64
    t0 = g.totals()
    g.step(6)
    t1 = g.totals()
    names = W.cons_names(2, False)
    for k in ("ar1", "ar2", "mx", "my", "E"):
        i = names.index(k)
        scale = max(abs(t0[i]), abs(t0[names.index("E")]) * 1e-6)
        assert abs(t1[i] - t0[i]) <= 1e-13 * scale, (k, t0[i], t1[i])
    g.close()


def test_amr_full_refinement_is_the_fine_grid():
    """Every block refined: level 1 steps exactly as the uniform grid of twice
    the resolution (the same kernels on the same data, dt_0 / 2 per step)."""
    from paper_2009_14555_gb300.solver import AmrSolver, Solver
    wl = W.solid_gas_1d(64, steps=4)
    g = AmrSolver(wl, max_levels=2, block=8, eps=-1.0, regrid_every=0)
    g.set_prim(wl.patches[0].prim)
    q1, act = g.get_level(1)
    assert act.all()
    fw = W.solid_gas_1d(128, steps=4)
    f = Solver.from_workload(fw)
    f.set_state(q1.reshape(-1), kind=0)
    dts = g.step(4)
    for dt in dts:
        f.step_fixed_dt(2, np.array([dt / 2]))
    out = f.get_arrays()[0]
    q1, _ = g.get_level(1)
    np.testing.assert_array_equal(q1.reshape(out.shape), out)
    f.close()
    g.close()


# --- the single-stage MUSCL-Hancock update in the hierarchy ----------------
def _hancock(wl):
    wl.scheme = "hancock"
    return wl


def test_amr_1d_solid_gas_hancock():
    """MUSCL-Hancock levels (one stage: ghost cells at the start of each
    step, registers of weight 1), three levels with regrids."""
    compare(_hancock(W.solid_gas_1d(128, steps=8)), 8, "amr_1d_solid_gas_hancock_128_3levels_8",
            max_level=3, block=8, eps=0.05, regrid_every=2)


def test_amr_2d_shock_disc_hancock():
    wl = _hancock(W.shock_disc_2d(64, steps=6, shock_x=0.3))
    wl.thinc = False
    compare(wl, 6, "amr_2d_shock_disc_hancock_64_2levels_6", max_level=2, block=8, eps=0.3, regrid_every=2)


def test_amr_2d_shock_disc_hancock_thinc():
    """With THINC (the shock at the disc's edge): bar 1e-10 or 10 x the
    oracle's one-ulp spread."""
    wl = _hancock(W.shock_disc_2d(64, steps=4, shock_x=0.3))
    compare(wl, 4, "amr_2d_shock_disc_hancock_thinc_64_2levels_4", calibrate=True, max_level=2, block=8, eps=0.3,
            regrid_every=2)


def test_amr_conservation_periodic_2d_hancock():
    """MUSCL-Hancock: composite totals on a periodic domain to round-off."""
    from paper_2009_14555_gb300.solver import AmrSolver
    wl = _hancock(W.smooth_disc_2d(n=64, steps=1, u0=150.0))
    g = AmrSolver(wl, max_levels=2, block=8, eps=0.5, buffer=0, regrid_every=2)
    g.set_prim(wl.patches[0].prim)
    n, counts = g.levels()
    assert n == 2 and 0 < counts[1] < 64
    t0 = g.totals()
    g.step(6)
    t1 = g.totals()
    names = W.cons_names(2, False)
    for k in ("ar1", "ar2", "mx", "my", "E"):
        i = names.index(k)
        scale = max(abs(t0[i]), abs(t0[names.index("E")]) * 1e-6)
        assert abs(t1[i] - t0[i]) <= 1e-13 * scale, (k, t0[i], t1[i])
    g.close()
