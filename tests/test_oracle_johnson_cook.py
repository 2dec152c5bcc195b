"""Pins of the oracle's Johnson-Cook plasticity (Section 2.3.2, Section 3.2).

  * temperature: T0 on the reference state, T0 (rho/rho0)^Gamma along the
    reference curve (the Debye temperature of a constant Grueneisen
    coefficient), and dE/dT = C_V at fixed density through the energy closure;
  * the relaxation root against the closed form of the objective with a
    constant yield stress (Lambert W), over three decades of dt chi0;
  * the rate-independent limit c3 -> 0 with linear hardening against the
    closed-form return J = (c1 + c2 (eps_p + J*)) / (sqrt(6) G + c2);
  * thermal softening: the c3 -> 0 return onto the softened yield surface,
    and full relaxation at the melting temperature;
  * the step changes no conserved row and only raises eps_p;
  * a symmetric copper-copper impact keeps its contact at half the flyer
    speed and leaves a plastic strain that grows with the impact speed.
"""
import math

import numpy as np
import pytest
import torch

from oracle import closures as C
from oracle import scheme as S
from paper_2009_14555_gb300 import workloads as W

F64 = torch.float64
AIR = W.material(1.4)
CU = W.COPPER_JC


def _cu(**kw):
    m = dict(CU)
    m.update(kw)
    return m


def _cell(m, s, dT=-1.0, rho=8930.0, eps0=0.0):
    """One almost pure copper cell with stretch V = diag(s, 1/s, 1) (so J* is
    set by s), at the pressure that puts its temperature dT above the
    reference-curve temperature (dT < 0 keeps it below T0: no softening)."""
    s = torch.as_tensor(s, dtype=F64).reshape(-1)
    n = s.numel()
    z = torch.zeros(n, dtype=F64)
    V = torch.zeros(n, 3, 3, dtype=F64)
    V[:, 0, 0] = s
    V[:, 1, 1] = 1.0 / s
    V[:, 2, 2] = 1.0
    _, J2 = C.hencky_dev(V)
    r = z + rho
    Gam = C.Gamma(m)
    p = C.p_ref(m, r, J2) + r * Gam * m["cv"] * dT
    phi = 1.0 - 1e-8
    w = dict(phi1=z + phi, rho1=r, rho2=z + 1.2, u=torch.zeros(n, 3, dtype=F64), p=p, V=V, lam=z + eps0)
    q = C.prim_to_cons(w, [m, AIR])
    return q, J2.sqrt()


def _deps(q, m, dt):
    out = S.plastic_update(q, [m, AIR], dt)
    return (out["arl"] - q["arl"]) / q["ar1"], out


def test_temperature_reference_curve_and_heat_capacity():
    m = CU
    r = torch.tensor([8930.0, 8930.0 * 1.3, 8930.0 * 0.9], dtype=F64)
    J2 = torch.tensor([0.0, 1e-4, 3e-5], dtype=F64)
    # on the reference curve (p = p_ref) the temperature is T0 (rho/rho0)^Gamma, Gamma = 2
    T = C.jc_temperature(m, r, C.p_ref(m, r, J2), J2)
    assert torch.allclose(T, 298.0 * (r / 8930.0) ** 2, rtol=1e-14, atol=0)
    # Gamma = d ln theta_D / d ln rho along it (the sign of the Grueneisen relation)
    h = 1e-6
    lo = C.jc_temperature(m, r * (1 - h), C.p_ref(m, r * (1 - h), J2), J2)
    hi = C.jc_temperature(m, r * (1 + h), C.p_ref(m, r * (1 + h), J2), J2)
    assert torch.allclose((hi.log() - lo.log()) / (math.log1p(h) - math.log1p(-h)), torch.full_like(r, 2.0),
                          rtol=1e-8)
    # at fixed density the specific energy of the closure rises by C_V per kelvin
    p1 = torch.tensor([1e9, 2e10, 5e8], dtype=F64)
    p2 = p1 + 3e9
    dE = C.material_energy(m, r, p2, J2) - C.material_energy(m, r, p1, J2)
    dTm = C.jc_temperature(m, r, p2, J2) - C.jc_temperature(m, r, p1, J2)
    assert torch.allclose(dE / dTm, torch.full_like(r, m["cv"]), rtol=1e-12)


@pytest.mark.parametrize("dtchi", [1e-9, 1e-7, 1e-5])
def test_rate_root_is_the_lambert_w_closed_form(dtchi):
    """With c2 = 0 and T below T0 the objective J - J* + dt chi0
    exp((J/J_Y - 1)/c3) = 0, J_Y = c1 / (sqrt 6 G(rho)), solves as
    J* - J = a W(K/a), a = c3 J_Y, K = dt chi0 exp((J*/J_Y - 1)/c3)."""
    from scipy.special import lambertw
    m = _cu(jc_c2=0.0)
    s = np.linspace(1.002, 1.008, 7)
    q, Js = _cell(m, s)
    G = C.shear_modulus(m, torch.tensor(8930.0, dtype=F64)).item()
    JY = m["sigma_y"] / (math.sqrt(6.0) * G)
    dt = dtchi / m["chi0"]
    deps, _ = _deps(q, m, dt)
    a = m["jc_c3"] * JY
    K = dtchi * np.exp((Js.numpy() / JY - 1.0) / m["jc_c3"])
    x = a * np.real(lambertw(K / a))
    assert (Js.numpy() > JY).any() and (Js.numpy() < JY).any()
    np.testing.assert_allclose(deps.numpy(), x, rtol=1e-9, atol=1e-18)


def test_rate_independent_limit_with_hardening():
    """c3 -> 0: the stress returns onto the hardened yield surface,
    sqrt 6 G J = c1 + c2 (eps0 + J* - J), n = 1, so
    J = (c1 + c2 (eps0 + J*)) / (sqrt 6 G + c2)."""
    m = _cu(jc_c3=1e-7)
    s = np.linspace(1.004, 1.02, 5)
    eps0 = 0.03
    q, Js = _cell(m, s, eps0=eps0)
    G = C.shear_modulus(m, torch.tensor(8930.0, dtype=F64)).item()
    deps, _ = _deps(q, m, 1e-7)
    J = Js.numpy() - deps.numpy()
    Jc = (m["sigma_y"] + m["jc_c2"] * (eps0 + Js.numpy())) / (math.sqrt(6.0) * G + m["jc_c2"])
    np.testing.assert_allclose(J, Jc, rtol=5e-5)
    # hardening lifts the return above the unhardened yield strain
    assert (J > m["sigma_y"] / (math.sqrt(6.0) * G) * (1 + 1e-3)).all()


def test_thermal_softening_and_melt():
    m = _cu(jc_c2=0.0, jc_c3=1e-7)
    G = C.shear_modulus(m, torch.tensor(8930.0, dtype=F64)).item()
    s = np.linspace(1.004, 1.01, 4)
    # halfway to the melting temperature: sigma_Y = c1 (1 - 0.5^m)
    q, Js = _cell(m, s, dT=0.5 * (m["jc_Tmelt"] - m["jc_T0"]))
    deps, _ = _deps(q, m, 1e-7)
    J = Js.numpy() - deps.numpy()
    Jc = m["sigma_y"] * (1.0 - 0.5 ** m["jc_m"]) / (math.sqrt(6.0) * G)
    np.testing.assert_allclose(J, Jc, rtol=5e-5)
    # at the melting temperature nothing holds the shear strain
    q, Js = _cell(m, s, dT=m["jc_Tmelt"] - m["jc_T0"] + 1.0)
    deps, out = _deps(q, m, 1e-7)
    np.testing.assert_allclose(deps.numpy(), Js.numpy(), rtol=1e-12)
    _, J2 = C.hencky_dev(out["V"])
    assert (J2.sqrt() < 1e-9 * Js).all()


def test_step_keeps_conserved_rows_and_raises_eps():
    m = CU
    q, Js = _cell(m, np.linspace(1.0, 1.02, 9), dT=40.0, eps0=0.1)
    deps, out = _deps(q, m, 2e-8)
    for k in ("phi1", "ar1", "ar2", "E"):
        assert torch.equal(out[k], q[k]), k
    assert torch.equal(out["mom"], q["mom"])
    assert (deps >= 0).all() and (deps <= Js).all()
    assert deps[0] == 0 and deps[-1] > 0


def _flyer(u, n=200, steps=120):
    wl = W.jc_flyer_1d(n, steps=steps, u_flyer=u)
    p = wl.patches[0]
    q = C.prim_to_cons(S.prim_from_array(p.prim, 1, True), wl.materials)
    grid = S.grid_of(p, 1)
    for _ in range(steps):
        q, _ = S.step(q, grid, wl.materials, dict(cfl=wl.cfl, thinc=wl.thinc))
    return C.cons_to_prim(q, wl.materials)


def test_symmetric_impact_contact_speed_and_plastic_strain():
    """Copper on copper: the contact moves at half the flyer speed (momentum
    and symmetry), the shocked copper flows plastically (eps_p > 0 behind
    both shocks, none ahead of them), and a faster flyer leaves more plastic
    strain (ahead of the waves, eps_p stays at the floor of the rate law)."""
    w = _flyer(876.0)
    x = (np.arange(200) + 0.5) * 0.04 / 200
    u = w["u"][0, :, 0].numpy()
    eps = w["lam"][0].numpy()
    mid = (x > 0.0085) & (x < 0.0115)
    assert np.abs(u[mid] - 438.0).max() < 0.02 * 438.0
    assert eps[mid].min() > 1e-3
    far = x > 0.025
    # ahead of the waves only the rate's floor chi0 exp(-1/c3) acts
    assert np.abs(eps[far & (w["phi1"][0].numpy() > 0.5)]).max() < 1e-12
    w2 = _flyer(1300.0)
    assert w2["lam"][0].numpy()[mid].mean() > 1.2 * eps[mid].mean()
