"""Pins of the oracle's single-stage MUSCL-Hancock update (oracle/hancock.py)
against closed forms and invariants: the textbook MUSCL-Hancock formula for
linear advection (1D and unsplit 2D), exact Riemann solutions, discrete
conservation on periodic domains, uniform pressure and velocity across an
interface, and second-order convergence on a smooth problem."""
import math

import numpy as np
import pytest
import torch

from oracle import closures as C
from oracle import scheme as S
from paper_2009_14555_gb300 import workloads as W
from tests import exact_riemann as X
from tests.test_oracle_scheme import GAS, _periodic, totals

GAS2 = W.material(1.67)


def run(wl, steps=None, t_end=None, dt=None, thinc=None):
    p = wl.patches[0]
    grid = S.grid_of(p, wl.dim)
    opts = dict(cfl=wl.cfl, thinc=wl.thinc if thinc is None else thinc, scheme="hancock")
    q = C.prim_to_cons(S.prim_from_array(p.prim, wl.dim, wl.reactive), wl.materials)
    t, n = 0.0, 0
    while True:
        if steps is not None and n >= steps:
            break
        dtn = dt if dt is not None else S.cfl_dt(q, grid, wl.materials, opts["cfl"])
        if t_end is not None:
            if t >= t_end - 1e-15:
                break
            dtn = min(dtn, t_end - t)
        q, dtn = S.step(q, grid, wl.materials, opts, dtn)
        t += dtn
        n += 1
    return q, t


def minmod(a, b):
    return np.where(a * b > 0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def test_linear_advection_1d_matches_textbook_formula():
    """Uniform u > 0 and p, two gases of different gamma and density, smooth
    phi1: one step equals phi_i - nu (f_i - f_{i-1}), f_i = phi_i + (1 - nu) s_i / 2
    (Toro Sec. 14.4, upwind face value of the evolved edge state)."""
    n, u, dt = 50, 3.0, 0.1 / 50
    wl = _periodic(W.riemann_1d(n, dict(mat=0, rho=1.0, u=u, p=1.0), dict(mat=0, rho=1.0, u=u, p=1.0),
                                materials=[GAS, GAS2]))
    xc = (np.arange(n) + 0.5) / n
    prim = wl.patches[0].prim
    prim[0, 0] = 0.5 + 0.4 * np.tanh((xc - 0.5) / 0.08)
    prim[1, 0], prim[2, 0] = 1.0, 3.0
    q, _ = run(wl, steps=1, dt=dt)
    phi = prim[0, 0]
    nu = u * dt * n
    s = minmod(phi - np.roll(phi, 1), np.roll(phi, -1) - phi)
    f = phi + 0.5 * (1 - nu) * s
    ex = phi - nu * (f - np.roll(f, 1))
    assert np.abs(q["phi1"][0].numpy() - ex).max() < 1e-13
    w = C.cons_to_prim(q, wl.materials)
    assert (w["p"] - 1.0).abs().max().item() < 1e-13
    assert (w["u"][..., 0] - u).abs().max().item() < 1e-13 * u


def test_linear_advection_2d_unsplit_formula():
    """Uniform (u, v) = (2, 1): every edge state moves by the unsplit predictor
    -(nu_x s_x + nu_y s_y) / 2, so the x face value is
    phi + s_x / 2 - (nu_x s_x + nu_y s_y) / 2 and the y face value
    phi + s_y / 2 - (nu_x s_x + nu_y s_y) / 2."""
    n, u, v = 24, 2.0, 1.0
    wl = _periodic(W.shock_disc_2d(n, steps=1, shock_x=-1.0))
    wl.materials = [GAS, GAS2]
    wl.thinc = False
    prim = wl.patches[0].prim
    xc = (np.arange(n) + 0.5) / n
    X_, Y_ = np.meshgrid(xc, xc)
    prim[0] = 0.5 + 0.3 * np.sin(2 * np.pi * X_) * np.cos(2 * np.pi * Y_)
    prim[1], prim[2], prim[3], prim[4], prim[5] = 1.0, 2.0, u, v, 1.0
    prim[6], prim[7], prim[8], prim[9], prim[10] = 1.0, 0.0, 0.0, 1.0, 1.0
    dt = 0.2 / (n * (u + v))
    q, _ = run(wl, steps=1, dt=dt)
    phi = prim[0]
    nx_, ny_ = u * dt * n, v * dt * n
    sx = minmod(phi - np.roll(phi, 1, 1), np.roll(phi, -1, 1) - phi)
    sy = minmod(phi - np.roll(phi, 1, 0), np.roll(phi, -1, 0) - phi)
    corr = 0.5 * (nx_ * sx + ny_ * sy)
    fx = phi + 0.5 * sx - corr
    fy = phi + 0.5 * sy - corr
    ex = phi - nx_ * (fx - np.roll(fx, 1, 1)) - ny_ * (fy - np.roll(fy, 1, 0))
    assert np.abs(q["phi1"].numpy() - ex).max() < 1e-13


def test_sod_shock_tube_matches_exact():
    L = dict(rho=1.0, u=0.0, p=1.0, gamma=1.4, pinf=0.0)
    R = dict(rho=0.125, u=0.0, p=0.1, gamma=1.4, pinf=0.0)
    errs = []
    for n in (100, 200):
        wl = W.riemann_1d(n, dict(mat=0, rho=1.0, u=0.0, p=1.0), dict(mat=1, rho=0.125, u=0.0, p=0.1),
                          cfl=0.8, materials=[GAS, GAS])
        q, t = run(wl, t_end=0.2)
        w = C.cons_to_prim(q, wl.materials)
        xc = (np.arange(n) + 0.5) / n
        ex = X.sample(L, R, (xc - 0.5) / t)
        rho = (q["ar1"] + q["ar2"])[0].numpy()
        errs.append(np.abs(rho - ex[0]).mean())
        if n == 200:
            ps, us = X.star(L, R)
            mid = (xc > 0.55) & (xc < 0.62)
            assert np.allclose(w["p"][0].numpy()[mid], ps, rtol=5e-3)
            assert np.allclose(w["u"][0, :, 0].numpy()[mid], us, rtol=5e-3)
    assert errs[1] < 0.7 * errs[0]
    assert errs[1] < 6e-3


@pytest.mark.parametrize("thinc", [False, True])
def test_conservation_periodic_1d(thinc):
    wl = _periodic(W.riemann_1d(64, dict(mat=0, rho=8000.0, u=30.0, p=1e5),
                                dict(mat=1, rho=1.2, u=30.0, p=1e5), cfl=0.8))
    wl.patches[0].prim[4, 0, 40:50] = 3e5
    wl.patches[0].prim[3, 0, 10:20] = 60.0
    q0 = C.prim_to_cons(S.prim_from_array(wl.patches[0].prim, 1, False), wl.materials)
    q, _ = run(wl, steps=40, thinc=thinc)
    a, b = totals(q0), totals(q)
    for k in ("ar1", "ar2", "mx", "E"):
        scale = abs(a["ar1"]) * 500.0 if k == "mx" else abs(a[k])
        assert abs(a[k] - b[k]) / scale < 1e-13, k


def test_conservation_periodic_2d_thinc():
    wl = _periodic(W.shock_disc_2d(24, steps=10))
    q0 = C.prim_to_cons(S.prim_from_array(wl.patches[0].prim, 2, False), wl.materials)
    q, _ = run(wl, steps=10)
    a, b = totals(q0), totals(q)
    ref_mom = (a["ar1"] + a["ar2"]) * 500.0
    for k in ("ar1", "ar2", "E"):
        assert abs(a[k] - b[k]) / abs(a[k]) < 1e-13, k
    for k in ("mx", "my"):
        assert abs(a[k] - b[k]) / ref_mom < 1e-13, k


def test_abgrall_solid_gas():
    wl = _periodic(W.riemann_1d(60, dict(mat=0, rho=8000.0, u=120.0, p=1e5),
                                dict(mat=1, rho=1.2, u=120.0, p=1e5)))
    q, _ = run(wl, steps=60, thinc=False)
    w = C.cons_to_prim(q, wl.materials)
    assert (w["p"] - 1e5).abs().max().item() / 1e5 < 1e-8
    assert (w["u"][..., 0] - 120.0).abs().max().item() / 120.0 < 1e-12


def test_second_order_smooth_advection():
    """phi1 = 0.5 + 0.4 sin(2 pi x) at u = 1, dt proportional to dx: L1 error
    order >= 1.8 (space and time together)."""
    errs = []
    for n in (32, 64, 128):
        wl = _periodic(W.riemann_1d(n, dict(mat=0, rho=1.0, u=1.0, p=1.0),
                                    dict(mat=0, rho=1.0, u=1.0, p=1.0), materials=[GAS, GAS]))
        xc = (np.arange(n) + 0.5) / n
        wl.patches[0].prim[0, 0] = 0.5 + 0.4 * np.sin(2 * np.pi * xc)
        q, t = run(wl, t_end=0.25, dt=0.4 / n)
        ex = 0.5 + 0.4 * np.sin(2 * np.pi * (xc - t))
        errs.append(np.abs(q["phi1"][0].numpy() - ex).mean())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert orders[-1] >= 1.8, orders


def test_solid_impact_gas_shock_matches_piston():
    """Config-0 solid|gas impact: phi1 stays in [0, 1] and the air ahead of the
    solid carries the exact piston-shock pressure for the contact velocity."""
    n = 200
    wl = W.solid_gas_1d(n, steps=400)
    q, t = run(wl, steps=400)
    assert q["phi1"].min().item() >= -1e-12 and q["phi1"].max().item() <= 1 + 1e-12
    w = C.cons_to_prim(q, wl.materials)
    xc = (np.arange(n) + 0.5) / n
    xint = xc[np.argmin(np.abs(q["phi1"][0].numpy() - 0.5))]
    ug = w["u"][0, :, 0].numpy()
    shock_at = xc[np.argmax(ug < 250.0)]
    ustar = ug[(xc > xint + 3.0 / n) & (xc < shock_at - 3.0 / n)].mean()
    A, B = 2 / (2.4 * 1.2), 0.4 / 2.4 * 1e5
    lo, hi = 1e5, 1e7
    for _ in range(200):  # gas shock relation u*(p*) of a piston at u*
        mid = 0.5 * (lo + hi)
        if (mid - 1e5) * math.sqrt(A / (mid + B)) > ustar:
            hi = mid
        else:
            lo = mid
    pstar = 0.5 * (lo + hi)
    S_sh = math.sqrt(1.4 * 1e5 / 1.2) * math.sqrt(2.4 / 2.8 * pstar / 1e5 + 0.4 / 2.8)
    gas_zone = (xc > xint + 3.0 / n) & (xc < 0.5 + S_sh * t - 3.0 / n)
    assert gas_zone.sum() >= 4
    assert np.allclose(w["p"][0].numpy()[gas_zone], pstar, rtol=2e-2)
    assert 450.0 < ustar < 500.0
