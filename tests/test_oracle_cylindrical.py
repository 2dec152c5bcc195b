"""Pins of the oracle's cylindrical (axisymmetric, x = r, y = z) geometric
source term (oracle.scheme.geometric_source_terms / spatial_operator):

  * homologous expansion u_r = a r of a uniform gas with V = I: every
    component of D equals its closed form (mass 2 a rho, radial momentum
    3 rho a^2 r, energy from the exact face fluxes, V_rr and V_thth -a/3,
    V_zz 2a/3: the unimodular stretch of F = diag(e^{at}, e^{at}, 1));
  * a strained solid at rest: radial momentum D = (sigma_thth - sigma_rr)/r;
  * a radially symmetric gas pulse computed in 2D Cartesian (x, y) and in
    (r, z) with no z dependence give the same radial pressure profile to the
    grid error.
"""
import math

import numpy as np
import torch

from oracle import closures as C
from oracle import scheme as S
from paper_2009_14555_gb300 import workloads as W

F64 = torch.float64
GAS = W.material(1.4)


def _state(nx, ny, x0, dx, prim_fn, mats):
    wl = W.riemann_1d(4, dict(mat=0, rho=1.0, u=0.0, p=1.0), dict(mat=0, rho=1.0, u=0.0, p=1.0),
                      materials=mats)
    p = W.Patch(nx=nx, ny=ny, dx=dx, dy=dx, x0=x0,
                bc=(W.BC_TRANSMISSIVE, W.BC_TRANSMISSIVE, W.BC_PERIODIC, W.BC_PERIODIC))
    xc = x0 + (np.arange(nx) + 0.5) * dx
    prim = np.zeros((11, ny, nx))
    prim_fn(prim, np.broadcast_to(xc[None, :], (ny, nx)))
    return p, C.prim_to_cons(S.prim_from_array(prim, 2, False), mats), xc


def test_homologous_expansion_closed_forms():
    a, rho, p0 = 50.0, 2.0, 3.0e5
    nx, ny, x0, dx = 24, 4, 0.2, 0.01

    def fill(prim, X):
        prim[0] = 1.0 - 1e-8
        prim[1], prim[2], prim[3], prim[5] = rho, rho, a * X, p0
        prim[6], prim[9], prim[10] = 1.0, 1.0, 1.0

    patch, q, xc = _state(nx, ny, x0, dx, fill, [GAS, GAS])
    grid = S.grid_of(patch, 2, "cyl")
    D = S.spatial_operator(q, grid, [GAS, GAS], False)
    sl = slice(3, nx - 3)  # away from the transmissive edges
    r = xc[sl]
    rp, rm = r + 0.5 * dx, r - 0.5 * dx
    arho = q["ar1"][0, sl].numpy() + q["ar2"][0, sl].numpy()
    np.testing.assert_allclose(D["ar1"][0, sl].numpy() + D["ar2"][0, sl].numpy(), 2 * a * arho, rtol=1e-12)
    np.testing.assert_allclose(D["mom"][0, sl, 0].numpy(), 3 * rho * a * a * r, rtol=1e-11)
    np.testing.assert_allclose(D["mom"][0, sl, 1].numpy(), 0.0, atol=1e-9 * rho * a * a)
    rhoe = p0 / 0.4

    def H(x):  # energy flux (rho E + p) u at radius x
        return (rhoe + 0.5 * rho * (a * x) ** 2 + p0) * a * x

    DE = (H(rp) - H(rm)) / dx + H(r) / r
    np.testing.assert_allclose(D["E"][0, sl].numpy(), DE, rtol=1e-11)
    V = D["V"][0, sl]
    np.testing.assert_allclose(V[:, 0, 0].numpy(), -a / 3, rtol=1e-10)
    np.testing.assert_allclose(V[:, 2, 2].numpy(), -a / 3, rtol=1e-10)
    np.testing.assert_allclose(V[:, 1, 1].numpy(), 2 * a / 3, rtol=1e-10)
    assert V[:, 0, 1].abs().max().item() < 1e-10 * a and V[:, 1, 0].abs().max().item() < 1e-10 * a
    assert D["phi1"][0, sl].abs().max().item() < 1e-12 * a


def test_strained_solid_at_rest_radial_force():
    """Uniform V = diag(1.001, 1, 0.999) in the config-0 solid at rest: the
    flux differences vanish and the radial momentum D is (s_thth - s_rr) / r."""
    nx, ny, x0, dx = 16, 4, 0.5, 0.01

    def fill(prim, X):
        prim[0] = 1.0 - 1e-8
        prim[1], prim[2], prim[5] = 8000.0, 1.2, 1e5
        prim[6], prim[9], prim[10] = 1.001, 1.0, 0.999

    mats = [W.SOLID, W.AIR]
    patch, q, xc = _state(nx, ny, x0, dx, fill, mats)
    grid = S.grid_of(patch, 2, "cyl")
    D = S.spatial_operator(q, grid, mats, False)
    w = C.cons_to_prim(q, mats)
    devH, J2 = C.hencky_dev(w["V"])
    _, Gm, _, _ = C.mixture_props(C.phases(w["phi1"]), [w["rho1"], w["rho2"]], w["p"], J2, mats, None)
    sig = C.stress(w["p"], Gm, devH)
    sl = slice(3, nx - 3)
    expect = ((sig[0, sl, 2, 2] - sig[0, sl, 0, 0]) / torch.as_tensor(xc[sl])).numpy()
    assert abs(expect).min() > 1e6  # a real force: sigma_thth - sigma_rr ~ 2 G (H_thth - H_rr)
    np.testing.assert_allclose(D["mom"][0, sl, 0].numpy(), expect, rtol=1e-9)
    assert D["ar1"][0, sl].abs().max().item() == 0.0


def _pulse(r):
    return 1e5 * (1.0 + 0.5 * np.exp(-(r / 0.15) ** 2))


def test_cylindrical_pulse_matches_cartesian_2d():
    """A smooth radially symmetric pressure pulse in air: (r, z) with no z
    dependence (reflective axis) against the 2D Cartesian quarter plane
    (reflective walls on both axes), same cell size; radial pressure
    profiles agree to 1 % of the pulse amplitude after the pulse has moved
    about a third of its width."""
    n, dx = 40, 1.0 / 80
    mats = [GAS, GAS]
    t_end = 0.3 * 0.15 / math.sqrt(1.4e5 / 1.2)

    def run(patch, q, grid):
        t = 0.0
        while t < t_end - 1e-15:
            dt = min(S.cfl_dt(q, grid, mats, 0.4), t_end - t)
            q, _ = S.step(q, grid, mats, dict(cfl=0.4, thinc=False), dt)
            t += dt
        return C.cons_to_prim(q, mats)["p"]

    # (r, z): 40 radial cells, 4 periodic axial cells
    pc = W.Patch(nx=n, ny=4, dx=dx, dy=dx, x0=0.0,
                 bc=(W.BC_REFLECTIVE, W.BC_TRANSMISSIVE, W.BC_PERIODIC, W.BC_PERIODIC))
    rc = (np.arange(n) + 0.5) * dx
    prim_rz = np.zeros((11, 4, n))
    prim_rz[0], prim_rz[1], prim_rz[2] = 0.5, 1.2, 1.2
    prim_rz[5] = _pulse(rc)[None, :]
    prim_rz[6], prim_rz[9], prim_rz[10] = 1.0, 1.0, 1.0
    q_rz = C.prim_to_cons(S.prim_from_array(prim_rz, 2, False), mats)
    pcyl = run(pc, q_rz, S.grid_of(pc, 2, "cyl"))[0].numpy()
    # Cartesian quarter plane
    pq = W.Patch(nx=n, ny=n, dx=dx, dy=dx,
                 bc=(W.BC_REFLECTIVE, W.BC_TRANSMISSIVE, W.BC_REFLECTIVE, W.BC_TRANSMISSIVE))
    X, Y = np.meshgrid(rc, rc)
    prim = np.zeros((11, n, n))
    prim[0], prim[1], prim[2] = 0.5, 1.2, 1.2
    prim[5] = _pulse(np.sqrt(X * X + Y * Y))
    prim[6], prim[9], prim[10] = 1.0, 1.0, 1.0
    pcar = run(pq, C.prim_to_cons(S.prim_from_array(prim, 2, False), mats), S.grid_of(pq, 2)).numpy()
    # the Cartesian pressure on the ring of radius r: mean of the cells whose
    # centre lies within half a cell of r
    R = np.sqrt(X * X + Y * Y).ravel()
    ring = np.array([pcar.ravel()[np.abs(R - r) < 0.5 * dx].mean() for r in rc[:30]])
    err = np.abs(pcyl[:30] - ring).max() / 0.5e5
    assert err < 2e-2, err
    # and the geometry matters: the same (r, z) run without s_g differs clearly
    pplan = run(pc, q_rz, S.grid_of(pc, 2))[0].numpy()
    assert np.abs(pplan[:30] - ring).max() / 0.5e5 > 5 * err
