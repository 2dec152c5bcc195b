"""Pins of the oracle's structured AMR (oracle/amr.py; Section 3, the AMR
platform paragraph; Section 4.2, difference-based flagging)."""
import numpy as np
import torch

from oracle import amr as A
from oracle import closures as C
from oracle import scheme as S
from paper_2009_14555_gb300 import workloads as W


def _cons(wl):
    p = wl.patches[0]
    return C.prim_to_cons(S.prim_from_array(p.prim, wl.dim, wl.reactive), wl.materials), S.grid_of(p, wl.dim)


def _opts(wl):
    return dict(cfl=wl.cfl, thinc=wl.thinc, scheme="rk3")


def _same(a, b, rtol=0.0):
    for k in a:
        if rtol == 0.0:
            assert torch.equal(a[k], b[k]), k
        else:
            torch.testing.assert_close(a[k], b[k], rtol=rtol, atol=0.0)


def test_one_level_is_the_plain_step():
    wl = W.solid_gas_1d(96, steps=6)
    q, g = _cons(wl)
    h = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=1, block=8)
    for _ in range(6):
        dt = h.step()
        q, dt_ref = S.step(q, g, wl.materials, _opts(wl))
        assert dt == float(dt_ref)
    _same(h.q[0], q)


def test_full_refinement_is_the_fine_grid():
    """Every cell tagged: level 1 covers the domain, so it evolves as the
    uniform grid of twice the resolution (two steps of dt_0 / 2 per level-0
    step, from the interpolated initial state) and level 0 is its average."""
    wl = W.solid_gas_1d(64, steps=4)
    q, g = _cons(wl)
    h = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=2, block=8, eps=-1.0)
    assert bool(h.active[1].all())
    qf = A.interp_fine(q, g)
    gf = dict(g, dx=g["dx"] / 2)
    for _ in range(4):
        dt = h.step()
        for _ in range(2):
            qf, _ = S.step(qf, gf, wl.materials, _opts(wl), dt=dt / 2)
    _same(h.q[1], qf)
    _same(h.q[0], A.average_down(qf, 1))


def test_interpolation_is_conservative_and_limited():
    """The children's mean is the parent; a linear profile is reproduced; no
    new extrema next to a step."""
    x = torch.arange(8, dtype=torch.float64)
    g = dict(dim=1, dx=1.0, dy=1.0, bc=(0, 0, 0, 0))
    q = {"phi1": (2.0 * x + 1.0)[None, :]}
    f = A.interp_fine(q, g)["phi1"][0]
    torch.testing.assert_close(f[2:-2], (2.0 * (torch.arange(16, dtype=torch.float64) / 2 - 0.25) + 1.0)[2:-2])
    torch.testing.assert_close(0.5 * (f[0::2] + f[1::2]), q["phi1"][0])
    step = {"phi1": torch.where(x < 4, 1.0, 0.0).to(torch.float64)[None, :]}
    fs = A.interp_fine(step, g)["phi1"]
    assert float(fs.max()) == 1.0 and float(fs.min()) == 0.0
    g2 = dict(dim=2, dx=1.0, dy=1.0, bc=(0, 0, 0, 0))
    r = torch.rand(6, 8, dtype=torch.float64, generator=torch.Generator().manual_seed(3))
    f2 = A.interp_fine({"E": r}, g2)["E"]
    torch.testing.assert_close(A.average_down({"E": f2}, 2)["E"], r, rtol=1e-15, atol=1e-15)


def test_tags_follow_the_fractional_change():
    """Section 4.2: a cell and its neighbour are tagged when a variable's
    fractional change between them exceeds eps."""
    wl = W.riemann_1d(32, dict(mat=1, rho=1.2, u=0.0, p=1e5), dict(mat=1, rho=1.2, u=0.0, p=1.05e5),
                      materials=[W.AIR, W.AIR], steps=1)
    q, _ = _cons(wl)
    t = A.tags(q, wl.materials, 1, eps=0.1)
    assert not bool(t.any())  # 5 % pressure change: below 10 %
    t = A.tags(q, wl.materials, 1, eps=0.01)
    assert t[0].nonzero().flatten().tolist() == [15, 16]
    d = A._dilate(t, 2, 1)
    assert d[0].nonzero().flatten().tolist() == [13, 14, 15, 16, 17, 18]


def test_nesting_and_regrid():
    """Level 2 lies inside level 1 with a margin of one block of level 1
    cells; a moving feature is followed by the refined region."""
    wl = W.solid_gas_1d(128, steps=1)
    q, g = _cons(wl)
    h = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=3, block=8, eps=0.05, regrid_every=2)
    assert h.n_levels() == 3
    for _ in range(4):
        h.step()
    a1 = A._block_all(h.active[1], 8, 1)[0]
    a2 = A._block_any(h.active[2], 16, 1)[0]  # level-1 blocks (8 cells) refined at level 2
    for i in np.nonzero(a2.numpy())[0]:
        for j in (i - 1, i, i + 1):
            assert j < 0 or j >= len(a1) or bool(a1[j])
    # the interface (solid|gas) lies inside the finest level
    phi = h.q[2]["phi1"][0]
    mixed = (phi > 0.01) & (phi < 0.99) & h.active[2][0]
    assert bool(mixed.any())


def _periodic_case(dim):
    if dim == 1:
        wl = W.riemann_1d(64, dict(mat=0, rho=8000.0, u=100.0, p=1e8), dict(mat=1, rho=1.2, u=0.0, p=1e5),
                          bc=(W.BC_PERIODIC,) * 2 if hasattr(W, "BC_PERIODIC") else (1, 1), steps=1)
    else:
        wl = W.smooth_disc_2d(n=32, steps=1, u0=150.0)
    return wl


def test_conservation_across_levels_1d_periodic():
    """Periodic domain, a refined region that moves: the composite totals of
    the conservative rows stay constant to round-off (refluxing and
    average-down), through regrids."""
    wl = W.solid_gas_1d(64, steps=1)
    p = wl.patches[0]
    p.bc = [S.BC_PERIODIC, S.BC_PERIODIC, S.BC_PERIODIC, S.BC_PERIODIC]
    q, g = _cons(wl)
    h = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=3, block=8, eps=0.05, regrid_every=2)
    assert h.n_levels() >= 2
    t0 = h.composite_totals()
    for _ in range(8):
        h.step()
    t1 = h.composite_totals()
    for k in ("ar1", "ar2", "mom", "E"):
        scale = float(t0[k].abs().max()) or 1.0
        err = float((t1[k] - t0[k]).abs().max()) / scale
        assert err < 1e-13, (k, err)


def test_conservation_across_levels_2d_periodic():
    """The same in 2D: the refined ring around the disc (tags of a 50 %
    change, the disc's partial densities) meets the coarse level on all
    sides."""
    wl = W.smooth_disc_2d(n=64, steps=1, u0=150.0)
    q, g = _cons(wl)
    h = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=2, block=8, eps=0.5, buffer=0, regrid_every=2)
    assert h.n_levels() == 2 and not bool(h.active[1].all())
    t0 = h.composite_totals()
    for _ in range(4):
        h.step()
    t1 = h.composite_totals()
    for k in ("ar1", "ar2", "mom", "E"):
        scale = float(t0[k].abs().max()) or 1.0
        err = float((t1[k] - t0[k]).abs().max()) / scale
        assert err < 1e-13, (k, err)


def test_uniform_state_stays_uniform():
    """Free stream across coarse-fine boundaries: a uniform moving state with
    a forced partial refinement stays exactly uniform."""
    wl = W.riemann_1d(64, dict(mat=1, rho=1.2, u=50.0, p=1e5), dict(mat=1, rho=1.2, u=50.0, p=1e5),
                      materials=[W.AIR, W.AIR], steps=1)
    q, g = _cons(wl)

    def force(l, grid, shape):
        m = torch.zeros(shape, dtype=torch.bool)
        m[..., 20:40] = True
        return m

    h = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=2, block=8, eps=1e9, extra_tags=force)
    assert h.n_levels() == 2 and not bool(h.active[1].all())
    for _ in range(5):
        h.step()
    for l in range(2):
        for k, v in h.q[l].items():
            a = v[h.active[l]]
            assert float((a - a[0]).abs().max()) == 0.0, (l, k)


def test_refined_interface_is_closer_to_the_fine_grid():
    """A solid|gas problem: the two-level solution on its refined cells is
    closer to the uniform fine-grid solution than the uniform coarse grid is
    (measured on the pressure averaged to the coarse cells)."""
    wl = W.solid_gas_1d(64, steps=1)
    q, g = _cons(wl)
    opts = _opts(wl)
    h = A.Hierarchy(q, g, wl.materials, opts, max_level=2, block=8, eps=0.02, regrid_every=1)
    qc = q
    qf = A.interp_fine(q, g)
    gf = dict(g, dx=g["dx"] / 2)
    for _ in range(12):
        dt = h.step()
        qc, _ = S.step(qc, g, wl.materials, opts, dt=dt)
        for _ in range(2):
            qf, _ = S.step(qf, gf, wl.materials, opts, dt=dt / 2)
    ref = A.average_down(qf, 1)
    cov = h.active[1].reshape(1, -1, 2).any(-1)
    e_amr = float((h.q[0]["E"] - ref["E"])[cov].abs().sum())
    e_coarse = float((qc["E"] - ref["E"])[cov].abs().sum())
    assert e_amr < 0.5 * e_coarse, (e_amr, e_coarse)


def _cons_geo(wl):
    p = wl.patches[0]
    return (C.prim_to_cons(S.prim_from_array(p.prim, wl.dim, wl.reactive), wl.materials),
            S.grid_of(p, wl.dim, wl.geometry))


def test_one_level_is_the_plain_step_cylindrical():
    """Cylindrical geometry (x = r on [0, 1] with the axis at x = 0): a single
    level is the single-grid cylindrical step, geometric source included."""
    wl = W.cylinder_core_1d(96, steps=5)
    q, g = _cons_geo(wl)
    assert g["geometry"] == "cyl"
    h = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=1, block=8)
    for _ in range(5):
        dt = h.step()
        q, dt_ref = S.step(q, g, wl.materials, _opts(wl))
        assert dt == float(dt_ref)
    _same(h.q[0], q)


def _full_refinement_cyl(wl, steps):
    q, g = _cons_geo(wl)
    h = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=2, block=8, eps=-1.0)
    assert bool(h.active[1].all())
    qf = A.interp_fine(q, g)
    gf = dict(g, dx=g["dx"] / 2, dy=g["dy"] / 2 if wl.dim == 2 else g["dy"])
    for _ in range(steps):
        dt = h.step()
        for _ in range(2):
            qf, _ = S.step(qf, gf, wl.materials, _opts(wl), dt=dt / 2)
    _same(h.q[1], qf)
    _same(h.q[0], A.average_down(qf, wl.dim))
    return h


def test_full_refinement_is_the_fine_grid_cylindrical_1d():
    """Every cell refined: level 1 evolves as the uniform cylindrical grid of
    twice the resolution, so its geometric source is taken at the fine
    cell-centre radii (i + 1/2) dx / 2, and level 0 is its average."""
    h = _full_refinement_cyl(W.cylinder_core_1d(64, steps=4), 4)
    # the geometric source acts: the same hierarchy in planar geometry differs
    wl = W.cylinder_core_1d(64, steps=4)
    wl.geometry = "planar"
    q, g = _cons_geo(wl)
    hp = A.Hierarchy(q, g, wl.materials, _opts(wl), max_level=2, block=8, eps=-1.0)
    for _ in range(4):
        hp.step()
    assert not torch.equal(hp.q[1]["mom"], h.q[1]["mom"])


def test_full_refinement_is_the_fine_grid_cylindrical_2d():
    """The same in (r, z): the shock-sphere problem on 16 x 32 cells."""
    _full_refinement_cyl(W.sphere_shock_rz(32, steps=2, thinc=False), 2)


# --- the single-stage MUSCL-Hancock update in the hierarchy ----------------
def _hopts(wl):
    return dict(cfl=wl.cfl, thinc=wl.thinc, scheme="hancock")


def test_one_level_is_the_plain_step_hancock():
    """MUSCL-Hancock: a single level is the single-grid MUSCL-Hancock step."""
    wl = W.solid_gas_1d(96, steps=6)
    q, g = _cons(wl)
    h = A.Hierarchy(q, g, wl.materials, _hopts(wl), max_level=1, block=8)
    for _ in range(6):
        dt = h.step()
        q, dt_ref = S.step(q, g, wl.materials, _hopts(wl))
        assert dt == float(dt_ref)
    _same(h.q[0], q)


def test_full_refinement_is_the_fine_grid_hancock():
    """MUSCL-Hancock, every cell refined (1D solid|gas and the 2D
    shock-disc with THINC): level 1 is the uniform fine grid bit for bit."""
    for wl, steps in ((W.solid_gas_1d(64, steps=4), 4), (W.shock_disc_2d(32, steps=2, shock_x=0.3), 2)):
        q, g = _cons(wl)
        h = A.Hierarchy(q, g, wl.materials, _hopts(wl), max_level=2, block=8, eps=-1.0)
        assert bool(h.active[1].all())
        qf = A.interp_fine(q, g)
        gf = dict(g, dx=g["dx"] / 2, dy=g["dy"] / 2 if wl.dim == 2 else g["dy"])
        for _ in range(steps):
            dt = h.step()
            for _ in range(2):
                qf, _ = S.step(qf, gf, wl.materials, _hopts(wl), dt=dt / 2)
        _same(h.q[1], qf)
        _same(h.q[0], A.average_down(qf, wl.dim))


def test_conservation_across_levels_hancock():
    """MUSCL-Hancock on periodic domains: the composite totals stay constant
    to round-off through regrids (1D, three levels) and across a refined
    ring (2D): the registers hold the corrector's fluxes."""
    wl = W.solid_gas_1d(64, steps=1)
    wl.patches[0].bc = [S.BC_PERIODIC] * 4
    cases = [(wl, dict(max_level=3, block=8, eps=0.05, regrid_every=2), 8),
             (W.smooth_disc_2d(n=64, steps=1, u0=150.0), dict(max_level=2, block=8, eps=0.5, buffer=0,
                                                               regrid_every=2), 4)]
    for wl, kw, steps in cases:
        q, g = _cons(wl)
        h = A.Hierarchy(q, g, wl.materials, _hopts(wl), **kw)
        assert h.n_levels() >= 2 and not bool(h.active[1].all())
        t0 = h.composite_totals()
        for _ in range(steps):
            h.step()
        t1 = h.composite_totals()
        for k in ("ar1", "ar2", "mom", "E"):
            scale = float(t0[k].abs().max()) or 1.0
            err = float((t1[k] - t0[k]).abs().max()) / scale
            assert err < 1e-13, (wl.name, k, err)


def test_uniform_state_stays_uniform_hancock():
    """MUSCL-Hancock free stream across coarse-fine boundaries."""
    wl = W.riemann_1d(64, dict(mat=1, rho=1.2, u=50.0, p=1e5), dict(mat=1, rho=1.2, u=50.0, p=1e5),
                      materials=[W.AIR, W.AIR], steps=1)
    q, g = _cons(wl)

    def force(l, grid, shape):
        m = torch.zeros(shape, dtype=torch.bool)
        m[..., 20:40] = True
        return m

    h = A.Hierarchy(q, g, wl.materials, _hopts(wl), max_level=2, block=8, eps=1e9, extra_tags=force)
    assert h.n_levels() == 2 and not bool(h.active[1].all())
    for _ in range(5):
        h.step()
    for l in range(2):
        for k, v in h.q[l].items():
            a = v[h.active[l]]
            assert float((a - a[0]).abs().max()) == 0.0, (l, k)
