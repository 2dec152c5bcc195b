"""Pins of the oracle's mixed-cell closures against what the discrete system
does, not against the oracle's own formulas.

  * Mixture sound speed (Section 2.2 mixture rules; reading R4, the frozen
    form c^2 = sum Y_l c_l^2 / Gamma_l / sum phi_l / Gamma_l): a small pressure
    pulse in a uniform 50/50 mixture at rest splits into two acoustic waves;
    the velocity centroid of the right-moving one travels at the speed of the
    discrete system.  The Riemann solver's wave-speed estimates only set the
    dissipation, so the speed that is measured comes from the pressure
    function (Appendix B) and the stress, not from the c^2 formula under
    test.  Cases: water|air (c^2 alone), two elastic solids (c_L^2 =
    c^2 + 4/3 G_mix / rho), solid|air (reading R14: the fluid relaxes fully,
    so the mixed cell keeps no shear stiffness and the pulse runs at c).
  * The non-hyperbolic face fallback (reading R10'): a face whose
    THINC-steepened state has c_L^2 <= 0 takes the cell-centre state on that
    side, and only on that side.
  * The phi/Gamma weighting of the relaxed strain norm J* (Section 3.2,
    equation for the mixture J*): hand-computed values in 50/50 cells.
"""
import math

import numpy as np
import torch

from oracle import closures as C
from oracle import scheme as S
from oracle.riemann import hllc
from paper_2009_14555_gb300 import workloads as W

F64 = torch.float64

WATER = W.material(4.4, p_inf=6e8)
AIR = W.material(1.4)
SOLID_A = W.material(4.0, p_inf=6e10, G=5e10)             # elastic, no plasticity
SOLID_B = W.material(3.0, p_inf=4.55e10, G=3.94e10)       # elastic, no plasticity


def _pulse_speed(mats, phi1, rho1, rho2, p0, amp, n=400, travel=0.25):
    """Velocity centroid speed of the right-moving half of a Gaussian pressure
    pulse (width 0.02, centre 0.5) on a periodic [0, 1] line, and the oracle's
    c^2, c_L^2 of the undisturbed mixture."""
    w, k = W._blank(1, False, 1, n)
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    w[k["phi1"], 0] = phi1
    w[k["rho1"], 0] = rho1
    w[k["rho2"], 0] = rho2
    w[k["p"], 0] = p0 * (1 + amp * np.exp(-((xc - 0.5) / 0.02) ** 2))
    patch = W.Patch(nx=n, ny=1, dx=dx, dy=1.0, bc=(1, 1, 0, 0), prim=w)
    grid = S.grid_of(patch, 1)
    q = C.prim_to_cons(S.prim_from_array(w, 1, False), mats)
    w0 = C.cons_to_prim(q, mats)
    _, J2 = C.hencky_dev(w0["V"])
    _, _, c2, cL2 = C.mixture_props(C.phases(w0["phi1"]), [w0["rho1"], w0["rho2"]], w0["p"], J2, mats, None)
    c2, cL2 = float(c2[0, 0]), float(cL2[0, 0])
    t_end = travel / math.sqrt(cL2)
    t = 0.0
    while t < t_end - 1e-15:
        dt = min(S.cfl_dt(q, grid, mats, 0.5), t_end - t)
        q, dt = S.step(q, grid, mats, dict(cfl=0.5, thinc=False), dt)
        t += dt
    u = C.cons_to_prim(q, mats)["u"][0, :, 0].numpy()
    right = xc > 0.5
    x_c = (u[right] * xc[right]).sum() / u[right].sum()
    return (x_c - 0.5) / t, c2, cL2


def _frozen_c2(parts):
    """sum Y_l c_l^2 / Gamma_l / sum phi_l / Gamma_l and the printed variant
    with phi_l Y_l in the numerator, from textbook stiffened-gas phase speeds
    c_l^2 = gamma_l (p + p_inf,l) / rho_l; parts = [(phi, rho, gamma, p_inf)]."""
    rho = sum(ph * r for ph, r, _, _ in parts)
    num = sum((ph * r / rho) * g * (1e5 + pi) / r / (g - 1) for ph, r, g, pi in parts)
    garbled = sum(ph * (ph * r / rho) * g * (1e5 + pi) / r / (g - 1) for ph, r, g, pi in parts)
    xi = sum(ph / (g - 1) for ph, _, g, _ in parts)
    return num / xi, garbled / xi


def test_mixture_sound_speed_water_air_pulse():
    speed, c2, cL2 = _pulse_speed([WATER, AIR], 0.5, 1000.0, 1.2, 1e5, 0.1)
    assert cL2 == c2  # no shear modulus
    r4, garbled = _frozen_c2([(0.5, 1000.0, 4.4, 6e8), (0.5, 1.2, 1.4, 0.0)])
    assert abs(c2 / r4 - 1) < 1e-12
    # the measured speed is the frozen (Allaire) speed; the printed phi*Y
    # numerator would give a speed lower by a factor ~sqrt(2)
    assert abs(speed / math.sqrt(c2) - 1) < 1e-3, (speed, math.sqrt(c2))
    assert abs(speed / math.sqrt(garbled) - 1) > 0.2


def test_mixture_longitudinal_speed_two_elastic_solids_pulse():
    speed, c2, cL2 = _pulse_speed([SOLID_A, SOLID_B], 0.5, 8000.0, 8930.0, 1e5, 1000.0)
    r4, garbled = _frozen_c2([(0.5, 8000.0, 4.0, 6e10), (0.5, 8930.0, 3.0, 4.55e10)])
    assert abs(c2 / r4 - 1) < 1e-9  # the strain of the undisturbed state is zero
    # G_mix = sum phi_l G_l / Gamma_l / sum phi_l / Gamma_l (Section 2.2)
    Gm = (0.5 * 5e10 / 3.0 + 0.5 * 3.94e10 / 2.0) / (0.5 / 3.0 + 0.5 / 2.0)
    assert abs(cL2 / (r4 + 4.0 / 3.0 * Gm / 8465.0) - 1) < 1e-9
    assert abs(speed / math.sqrt(cL2) - 1) < 1e-3, (speed, math.sqrt(cL2))
    assert abs(speed / math.sqrt(c2) - 1) > 0.1          # the shear stiffness is felt
    assert abs(speed / math.sqrt(garbled + 4.0 / 3.0 * Gm / 8465.0) - 1) > 0.1


def test_fluid_relaxation_removes_mixed_cell_shear_stiffness():
    """Reading R14 (a fluid's J*_l = 0) in a 50/50 solid|air cell: the
    mixture J* keeps only (phi_s/Gamma_s) / (sum phi/Gamma) = 0.118 of the
    strain each step, so the pulse runs at the hydrodynamic c, not c_L.  (With
    the fluid contributing J*_l = J^star instead, no strain would relax and the
    pulse would run at c_L = 3003 m/s.)"""
    speed, c2, cL2 = _pulse_speed([W.SOLID, AIR], 0.5, 8000.0, 1.2, 1e5, 10.0)
    assert abs(speed / math.sqrt(c2) - 1) < 1e-3, (speed, math.sqrt(c2))
    assert abs(speed / math.sqrt(cL2) - 1) > 0.1


def _line(cells):
    """Primitive components of a 1D line from (phi1, rho1, rho2, u, p) tuples."""
    a = torch.tensor(cells, dtype=F64).T
    z = torch.zeros(len(cells), dtype=F64)
    one = torch.ones(len(cells), dtype=F64)
    c = dict(phi1=a[0], rho1=a[1], rho2=a[2], ux=a[3], uy=z, p=a[4],
             V11=one, V12=z, V21=z, V22=one, V33=one)
    return {k: v[None, :] for k, v in c.items()}


def _state(phi1, rho1, rho2, u, p):
    t = lambda x: torch.tensor([[x]], dtype=F64)  # noqa: E731
    z = torch.zeros(1, 1, 3, dtype=F64)
    z[..., 0] = u
    return dict(phi1=t(phi1), rho1=t(rho1), rho2=t(rho2), u=z, p=t(p),
                V=torch.eye(3, dtype=F64).expand(1, 1, 3, 3).clone())


def _cL2(phi1, rho1, rho2, p, mats):
    ph = torch.tensor([phi1], dtype=F64)
    _, _, _, cL2 = C.mixture_props([ph, 1 - ph], [torch.tensor([rho1], dtype=F64),
                                                  torch.tensor([rho2], dtype=F64)],
                                   torch.tensor([p], dtype=F64), torch.zeros(1, dtype=F64), mats, None)
    return float(cL2[0])


def test_non_hyperbolic_face_falls_back_to_the_cell_centre_on_that_side():
    """A solid in tension (p = -5e8 Pa) next to dense air at 1e5 Pa.  The mixed
    cell (phi_s = 0.2) is hyperbolic, but its THINC edge towards the air is
    air-dominated at the solid's negative pressure: c_L^2 < 0.  That face
    must use the mixed cell's centre state on the left and the air cell's own
    reconstructed state (u = 5 m/s: minmod of the slopes 10, 10) on the right."""
    mats = [W.SOLID, AIR]
    eps = 1e-8
    cells = [(1 - eps, 8000.0, 100.0, 0.0, -5e8)] * 4 + [(0.2, 8000.0, 100.0, 0.0, -5e8)] + \
            [(eps, 8000.0, 100.0, 10.0 * (k + 1), 1e5) for k in range(4)]
    n = len(cells) - 2 * S.NG
    F, phi_f, u_f, V_f = S._sweep(_line(cells), None, 0, n, mats, True)
    # face f is between cells NG-1+f and NG+f: the mixed cell is cell 4, so the
    # face between it and the first air cell is f = 4 - NG + 1
    f = 4 - S.NG + 1
    assert _cL2(0.2, 8000.0, 100.0, -5e8, mats) > 0          # the mixed cell is hyperbolic
    assert _cL2(eps, 8000.0, 100.0, 5e4, mats) > 0           # so is the air
    # the THINC edge of the mixed cell towards the air is air-dominated
    # (phi_s = 0.0115), and such a state is not hyperbolic at -5e8 Pa
    from oracle.reconstruction import thinc_faces
    phl = torch.tensor([[1 - eps, 1 - eps, 0.2, eps, eps]], dtype=F64)
    _, tR, mixed = thinc_faces(phl, torch.full_like(phl, 2.51))
    assert bool(mixed[0, 2]) and abs(float(tR[0, 2]) - 0.0115) < 1e-4
    assert _cL2(float(tR[0, 2]), 8000.0, 100.0, -5e8, mats) < 0
    want = hllc(_state(0.2, 8000.0, 100.0, 0.0, -5e8), _state(eps, 8000.0, 100.0, 5.0, 1e5), 0, mats)
    centre = hllc(_state(0.2, 8000.0, 100.0, 0.0, -5e8), _state(eps, 8000.0, 100.0, 10.0, 1e5), 0, mats)
    for k in F:
        assert torch.allclose(F[k][0, f], want[0][k][0, 0], rtol=1e-13, atol=0), k
    assert torch.allclose(u_f[0, f], want[2][0, 0], rtol=1e-13, atol=1e-12)
    # the right side kept its reconstruction (u = 5, not the centre's 10)
    assert not torch.allclose(F["E"][0, f], centre[0]["E"][0, 0], rtol=1e-6)
    # every flux of the line is finite (no NaN from a non-hyperbolic state)
    for k in F:
        assert torch.isfinite(F[k]).all(), k


def _shear_V(J):
    """Stretch diag(e^s, e^-s, 1) whose Bazant strain norm is J:
    B = diag(e^2s, e^-2s, 1), 1/4 (B - B^-1) = diag(sinh 2s, -sinh 2s, 0) / 2,
    already deviatoric, so J = sinh(2s) / sqrt(2)."""
    s = 0.5 * math.asinh(math.sqrt(2.0) * J)
    V = torch.diag(torch.tensor([math.exp(s), math.exp(-s), 1.0], dtype=F64))
    return V[None, None]


def _relaxed_J(mats, phi1, J):
    """Strain norm after the plastic step of a cell at rest, read back from
    the Pade form V_ii = (1 + h_i / 2) / (1 - h_i / 2) of the result."""
    V = _shear_V(J)
    z = torch.zeros(1, 1, dtype=F64)
    q = dict(phi1=z + phi1, ar1=z + phi1 * 8000.0, ar2=z + (1 - phi1) * 8000.0,
             mom=torch.zeros(1, 1, 3, dtype=F64), E=z + 1e9, V=V)
    Vn = S.plastic_update(q, mats, 1e-9)["V"][0, 0]
    d = torch.diagonal(Vn)
    h = 2.0 * (d - 1.0) / (d + 1.0)
    assert abs(float(Vn[0, 1])) < 1e-15 and abs(float(h.sum())) < 1e-12
    return float(torch.sqrt((h * h).sum()))


def test_plastic_mixture_J_is_phi_over_Gamma_weighted():
    """Section 3.2: J* = sum (phi_l / Gamma_l) J*_l / sum phi_l / Gamma_l.
    Two perfectly plastic solids, 50/50, both past yield at J^star = 0.01:
      A: Gamma 3,   J_Y = 4e8 / (sqrt 6 * 5e10) = 3.265986e-3
      B: Gamma 1.5, J_Y = 3e8 / (sqrt 6 * 3e10) = 4.082483e-3
      J* = (1/6 * 3.265986e-3 + 1/3 * 4.082483e-3) / (1/2) = 3.810317e-3
    (a phi-only weighting would give 3.674235e-3)."""
    A = W.material(4.0, p_inf=6e10, G=5e10, plastic=1, sigma_y=4e8)
    B = W.material(2.5, p_inf=1e10, G=3e10, plastic=1, sigma_y=3e8)
    got = _relaxed_J([A, B], 0.5, 0.01)
    assert abs(got / 3.810317e-3 - 1) < 1e-6, got
    assert abs(got / 3.674235e-3 - 1) > 1e-2


def test_plastic_mixed_solid_air_cell_keeps_the_solid_share_of_its_yield_strain():
    """Reading R14 in a 50/50 solid|air cell past yield: the air's J*_l = 0
    with weight 0.5 / 0.4, the solid's J_Y = 3.265986e-3 with weight 0.5 / 3:
      J* = (1/6 * 3.265986e-3) / (1/6 + 5/4) = 3.842337e-4.
    Below yield (J^star = 1e-3) the same weights keep 0.117647 of the strain."""
    got = _relaxed_J([W.SOLID, AIR], 0.5, 0.01)
    assert abs(got / 3.842337e-4 - 1) < 1e-6, got
    got = _relaxed_J([W.SOLID, AIR], 0.5, 1e-3)
    assert abs(got / 1.17647059e-4 - 1) < 1e-6, got


def test_romenskii_copper_longitudinal_speed_pulse():
    """A small pressure pulse in Romenskii copper at rest (Section 2.3 closure,
    the Section 4.1 table) runs at the closed-form longitudinal speed
    sqrt((K0 + 4/3 G0) / rho0) = 4600.6 m/s of the cold curve at rho0."""
    cu = W.COPPER_ROMENSKII
    speed, c2, cL2 = _pulse_speed([cu, cu], 0.5, 8930.0, 8930.0, 1e5, 1000.0)
    exact = math.sqrt((136.5e9 + 4.0 / 3.0 * 39.4e9) / 8930.0)
    assert abs(math.sqrt(cL2) / exact - 1) < 1e-6
    assert abs(speed / exact - 1) < 1e-3, (speed, exact)
