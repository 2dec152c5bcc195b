"""Pins of the oracle's reverse mode (PyTorch autograd through the float64
oracle, oracle/adjoint.py) against central finite differences of the oracle
forward run, on smooth inputs with the time steps held at their recorded
values.  This ties the reference gradient of the adjoint parity tests to
something other than itself."""
import numpy as np
import pytest
import torch

from oracle import adjoint as OA
from paper_2009_14555_gb300 import workloads as W


def _grads(wl, steps, material, qbar=None):
    p = wl.patches[0]
    opts = dict(cfl=wl.cfl, thinc=wl.thinc)
    theta = torch.tensor([m[k] for m in wl.materials for k in OA.PARAM_KEYS], dtype=torch.float64,
                         requires_grad=True)
    w = torch.tensor(p.prim, dtype=torch.float64, requires_grad=True)
    J, _, dts = OA.rollout(w, "prim", wl.dim, OA.with_params(wl.materials, theta), p, opts, steps, material,
                           qbar)
    J.backward()

    def J_at(wv, th):
        with torch.no_grad():
            return float(OA.rollout(wv, "prim", wl.dim, OA.with_params(wl.materials, th), p, opts, steps,
                                    material, qbar, dts=dts)[0])

    return w.grad, theta.grad, J_at, torch.tensor(p.prim, dtype=torch.float64), theta.detach().clone()


def test_oracle_reverse_mode_vs_fd_state_and_elastoplastic_params():
    wl = W.smooth_disc_2d(n=10, steps=4, sigma_y=4e7)
    gw, gth, J_at, w0, th0 = _grads(wl, 4, 0)
    assert torch.isfinite(gw).all() and torch.isfinite(gth).all()
    k = {n: i for i, n in enumerate(W.prim_names(2, False))}
    d = torch.zeros_like(w0)
    d[k["rho1"]] = w0[k["rho1"]] * torch.linspace(-1, 1, 100, dtype=torch.float64).reshape(10, 10)
    d[k["u"]] = 10.0
    d[k["p"]] = 1e3
    eps = 1e-6
    fd = (J_at(w0 + eps * d, th0) - J_at(w0 - eps * d, th0)) / (2 * eps)
    an = float((gw * d).sum())
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    for kk in (0, 1):  # shear modulus and yield stress of the solid
        h = 1e-5 * float(th0[kk])
        e = torch.zeros_like(th0)
        e[kk] = h
        fdk = (J_at(w0, th0 + e) - J_at(w0, th0 - e)) / (2 * h)
        assert abs(fdk - float(gth[kk])) <= 1e-6 * abs(float(gth[kk])), (kk, fdk, float(gth[kk]))


def test_oracle_reverse_mode_vs_fd_heat_release():
    # a fast reaction (A = 1e9 /s) so that the products' heat release shows
    # within three steps; objective: final reaction-progress density (Q
    # raises the recovered pressure, hence the temperature and the rate)
    wl = W.reactive_plate_2d(nx=12, ny=6, steps=3, A=1e9)
    names = W.prim_names(2, True)
    qbar = np.zeros_like(wl.patches[0].prim)
    qbar[names.index("lam")] = 1.0  # slot of phi_y rho_y lam
    gw, gth, J_at, w0, th0 = _grads(wl, 3, -1, qbar)
    kq = 5  # Q of material 2 (the reactive gas)
    h = 1e-5 * float(th0[kq])
    e = torch.zeros_like(th0)
    e[kq] = h
    fdk = (J_at(w0, th0 + e) - J_at(w0, th0 - e)) / (2 * h)
    assert float(gth[kq]) != 0.0
    assert abs(fdk - float(gth[kq])) <= 1e-6 * abs(float(gth[kq])), (fdk, float(gth[kq]))


def test_oracle_perfect_plasticity_is_radial_return():
    """The closed-form return min(J*, J_Y) of the oracle's plastic update
    equals the bisection of the relaxation objective with a large finite rate
    (the chi0 -> infinity limit of Section 3.2)."""
    from oracle import scheme as OS
    from oracle.closures import prim_to_cons
    wl = W.smooth_disc_2d(n=8, steps=1, sigma_y=4e7)
    p = wl.patches[0]
    q = prim_to_cons(OS.prim_from_array(p.prim, 2, False), wl.materials)
    # strain the solid: stretch V by 2 % along x with a 1 % shear
    V = q["V"].clone()
    V[..., 0, 0] = 1.02
    V[..., 0, 1] = 0.01
    q = dict(q, V=V)
    dt = 1e-6
    a = OS.plastic_update(q, wl.materials, dt)
    mats_rate = [dict(m) for m in wl.materials]
    mats_rate[0]["plastic"] = 2
    mats_rate[0]["chi0"] = 1e300
    b = OS.plastic_update(q, mats_rate, dt, iters=200)
    assert torch.allclose(a["V"], b["V"], rtol=1e-13, atol=1e-14)
    assert not torch.allclose(a["V"], V)  # the state yielded


def test_oracle_reverse_mode_vs_fd_romenskii():
    """The same pin with the solid on the Romenskii form (Section 2.3:
    G(rho) = G_0 (rho / rho_0)^(beta + 1) in the stress, the sound speed and
    the yield strain): state direction, G_0 and sigma_y of the solid.  This
    is the reference of the GPU adjoint of Romenskii contexts."""
    wl = W.smooth_disc_2d(n=10, steps=4, sigma_y=4e7)
    cu = dict(W.COPPER_ROMENSKII, plastic=1, sigma_y=4e7)
    wl.materials = [cu, wl.materials[1]]
    k = {n: i for i, n in enumerate(W.prim_names(2, False))}
    p = wl.patches[0]
    p.prim[k["rho1"]] *= cu["rho0"] / W.SOLID_RHO0
    gw, gth, J_at, w0, th0 = _grads(wl, 4, 0)
    assert torch.isfinite(gw).all() and torch.isfinite(gth).all()
    d = torch.zeros_like(w0)
    d[k["rho1"]] = w0[k["rho1"]] * torch.linspace(-1, 1, 100, dtype=torch.float64).reshape(10, 10)
    d[k["u"]] = 10.0
    d[k["p"]] = 1e3
    eps = 1e-6
    fd = (J_at(w0 + eps * d, th0) - J_at(w0 - eps * d, th0)) / (2 * eps)
    an = float((gw * d).sum())
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    for kk in (0, 1):  # G_0 and yield stress of the copper
        assert float(gth[kk]) != 0.0
        h = 1e-5 * float(th0[kk])
        e = torch.zeros_like(th0)
        e[kk] = h
        fdk = (J_at(w0, th0 + e) - J_at(w0, th0 - e)) / (2 * h)
        assert abs(fdk - float(gth[kk])) <= 1e-6 * abs(float(gth[kk])), (kk, fdk, float(gth[kk]))


def test_oracle_reverse_mode_vs_fd_two_fluids():
    """Two fluids (LX-17 reactant on its JWL form expanding into air): the
    mixture shear modulus is zero at every face, where the HLLD-type solver
    drops its shear waves; the reverse mode stays finite there and matches
    central differences along a state direction."""
    wl = W.perturbed(W.riemann_1d(40, dict(mat=0, rho=1905.0, u=0.0, p=1e9), dict(mat=1, rho=1.2, u=0.0, p=1e5),
                                  materials=[W.LX17_REACTANT_JWL, W.AIR], steps=3), seed=33)
    gw, gth, J_at, w0, th0 = _grads(wl, 3, 0)
    assert torch.isfinite(gw).all() and torch.isfinite(gth).all()
    k = {n: i for i, n in enumerate(W.prim_names(1, False))}
    d = torch.zeros_like(w0)
    d[k["rho1"]] = w0[k["rho1"]] * torch.linspace(-1, 1, 40, dtype=torch.float64).reshape(1, 40)
    d[k["p"]] = 1e5
    eps = 1e-6
    fd = (J_at(w0 + eps * d, th0) - J_at(w0 - eps * d, th0)) / (2 * eps)
    an = float((gw * d).sum())
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
