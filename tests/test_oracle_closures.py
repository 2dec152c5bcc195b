"""Pins of the oracle's closures, reconstruction and Riemann solver.

Each check compares the oracle with something other than itself: textbook
special cases (ideal and stiffened gas), numerical derivatives, exact matrix
functions, quadrature of the THINC profile, and the invariance of the flux
under a mirror of the frame.
"""
import math

import numpy as np
import pytest
import torch

from oracle import closures as C
from oracle import reconstruction as Rc
from oracle import riemann as Rm
from paper_2009_14555_gb300 import workloads as W

F64 = torch.float64
GAS = W.material(1.4)
WATER = W.material(4.4, p_inf=6e8)
SOLID = W.SOLID


def t(x):
    return torch.as_tensor(x, dtype=F64)


def rand_stretch(n, amp, gen):
    """Random plane-strain stretch near I (unimodular not required)."""
    V = torch.eye(3, dtype=F64).repeat(n, 1, 1)
    V[:, :2, :2] += amp * torch.randn(n, 2, 2, generator=gen, dtype=F64)
    V[:, 2, 2] += amp * torch.randn(n, generator=gen, dtype=F64)
    return V


def test_ideal_gas_pressure_is_textbook():
    rho, u, p = t([1.0, 0.125, 3.0]), t([0.0, 2.0, -1.0]), t([1.0, 0.1, 7.0])
    phi1 = t([1e-6, 0.5, 1 - 1e-6])
    w = dict(phi1=phi1, rho1=rho, rho2=rho, u=torch.stack([u, 0 * u, 0 * u], -1), p=p,
             V=torch.eye(3, dtype=F64).repeat(3, 1, 1))
    q = C.prim_to_cons(w, [GAS, GAS])
    # textbook: E = p/(gamma-1) + rho u^2/2
    assert torch.allclose(q["E"], p / 0.4 + 0.5 * rho * u * u, rtol=1e-14)
    assert torch.allclose(C.cons_to_prim(q, [GAS, GAS])["p"], p, rtol=1e-13)


def test_stiffened_gas_pressure_and_sound_speed_textbook():
    rho, p = t([1000.0, 1100.0]), t([1e5, 3e9])
    e = (p + WATER["gamma"] * WATER["p_inf"]) / ((WATER["gamma"] - 1) * rho)  # textbook SG
    J2 = torch.zeros_like(rho)
    phis = [torch.ones_like(rho), torch.zeros_like(rho)]
    pp = C.mixture_pressure(phis, [rho, rho], rho * e, J2, [WATER, GAS])
    assert torch.allclose(pp, p, rtol=1e-12)
    c2 = C.material_sound_speed2(WATER, rho, p, J2)
    assert torch.allclose(c2, WATER["gamma"] * (p + WATER["p_inf"]) / rho, rtol=1e-13)


@pytest.mark.parametrize("J2v", [0.0, 1e-4, 4e-3])
def test_sound_speed_is_isentropic_derivative(J2v):
    """c^2 = (dp/drho)_s at fixed strain: central differences along de = p/rho^2 drho."""
    rho0, p0 = 8000.0, 2e8
    J2 = t([J2v])
    phis = [t([1.0]), t([0.0])]
    mats = [SOLID, GAS]

    def p_of(rho, e):
        return C.mixture_pressure(phis, [t([rho]), t([1.0])], t([rho * e]), J2, mats).item()

    e0 = C.material_energy(SOLID, t([rho0]), t([p0]), J2).item()
    h = 1e-3
    # second-order isentrope step: de/drho = p/rho^2
    ep = e0 + p0 / rho0 ** 2 * h
    em = e0 - p0 / rho0 ** 2 * h
    num = (p_of(rho0 + h, ep) - p_of(rho0 - h, em)) / (2 * h)
    c2 = C.material_sound_speed2(SOLID, t([rho0]), t([p0]), J2).item()
    assert abs(num - c2) / c2 < 1e-6


def test_reactive_closure_textbook():
    """Pure reactive ideal gas: p = (gamma-1)(rho e + (1-lam) rho Q), c^2 = gamma p / rho."""
    gas = W.material(1.4, reactive=1, Q=2e6, cv=717.5, A=1.0, T_act=1.0)
    rho, p, lam = t([1.2, 0.4]), t([1e5, 2e6]), t([1.0, 0.3])
    w = dict(phi1=t([1e-12, 1e-12]), rho1=t([8000.0, 8000.0]), rho2=rho,
             u=torch.zeros(2, 3, dtype=F64), p=p, V=torch.eye(3, dtype=F64).repeat(2, 1, 1),
             lam=lam)
    q = C.prim_to_cons(w, [GAS, gas])
    rhoe_th = (q["E"] + (1 - lam) * rho * gas["Q"])  # thermal part for the pure gas
    assert torch.allclose(0.4 * rhoe_th, p, rtol=1e-9)
    c2 = C.material_sound_speed2(gas, rho, p, torch.zeros(2, dtype=F64), lam)
    assert torch.allclose(c2, 1.4 * p / rho, rtol=1e-13)


def test_mixture_pressure_equilibrium_all_fractions():
    """Any phi with a common pressure recovers that pressure (Abgrall)."""
    phi = t(np.linspace(1e-6, 1 - 1e-6, 11))
    n = len(phi)
    w = dict(phi1=phi, rho1=torch.full((n,), 8000.0, dtype=F64), rho2=torch.full((n,), 1.2, dtype=F64),
             u=torch.zeros(n, 3, dtype=F64), p=torch.full((n,), 1e5, dtype=F64),
             V=torch.eye(3, dtype=F64).repeat(n, 1, 1))
    q = C.prim_to_cons(w, [SOLID, GAS])
    assert torch.allclose(C.cons_to_prim(q, [SOLID, GAS])["p"], w["p"], rtol=1e-9)


@pytest.mark.parametrize("sym", [True, False])
def test_bazant_strain_third_order(sym):
    """dev(H) ~ log V for symmetric unimodular V with error O(|H|^3) (Section 3.2)."""
    gen = torch.Generator().manual_seed(0)
    A = torch.randn(3, 3, generator=gen, dtype=F64)
    A = 0.5 * (A + A.T) if sym else A
    A[2, :2] = 0
    A[:2, 2] = 0
    A = A - torch.trace(A) / 3 * torch.eye(3, dtype=F64)
    errs, jerrs = [], []
    for h in (0.02, 0.01):
        Hx = h * 0.5 * (A + A.T)
        V = torch.linalg.matrix_exp(Hx)  # exact symmetric stretch with log = Hx
        if not sym:
            # a rotation on the left does not change V V^T when V is replaced by V R^T
            R = torch.linalg.matrix_exp(h * 0.5 * (A - A.T))
            V = V @ R.T
        devH, J2 = C.hencky_dev(V[None])
        errs.append((devH[0] - Hx).abs().max().item())
        jerrs.append(abs(J2.item() - (Hx * Hx).sum().item()))
    assert 6.0 < errs[0] / errs[1] < 10.0      # dev(H) error O(h^3)
    assert 12.0 < jerrs[0] / jerrs[1] < 20.0   # J^2 error O(h^4)


def test_minmod_and_muscl():
    x = t(np.arange(8.0))
    wL, wR = Rc.muscl_faces(2 * x + 1)
    assert torch.allclose(wL[1:-1], 2 * x[1:-1], rtol=0, atol=1e-15)
    assert torch.allclose(wR[1:-1], 2 * x[1:-1] + 2, rtol=0, atol=1e-15)
    peak = t([0.0, 1.0, 3.0, 1.0, 0.0])
    wL, wR = Rc.muscl_faces(peak)
    assert wL[2] == 3.0 and wR[2] == 3.0
    assert Rc.minmod(t(-2.0), t(-1.0)) == -1.0 and Rc.minmod(t(2.0), t(-1.0)) == 0.0


@pytest.mark.parametrize("beta", [2.51, 0.5, 1.7])
def test_thinc_edges_conserve_cell_average(beta):
    """The tanh profile through the THINC edge values has cell average q_i (App. A)."""
    gen = np.random.default_rng(1)
    for _ in range(20):
        qm, qp = gen.uniform(0, 1, 2)
        lo, hi = min(qm, qp), max(qm, qp)
        qc = lo + (hi - lo) * gen.uniform(0.05, 0.95)
        q = t([qm, qc, qp])
        qL, qR, mixed = Rc.thinc_faces(q, torch.full((3,), beta, dtype=F64))
        assert bool(mixed[1])
        qmin, jump, th = lo, hi - lo, math.copysign(1.0, qp - qm)
        # invert the left edge value for the interface position x0: q_L = qmin + jump/2 (1 + th tanh(-beta x0))
        tl = ((qL[1].item() - qmin) / (jump / 2) - 1) / th
        x0 = -math.atanh(tl) / beta
        xs = (np.arange(20000) + 0.5) / 20000
        prof = qmin + jump / 2 * (1 + th * np.tanh(beta * (xs - x0)))
        assert abs(prof.mean() - qc) < 1e-9
        right = qmin + jump / 2 * (1 + th * math.tanh(beta * (1 - x0)))
        assert abs(right - qR[1].item()) < 1e-12


def test_thinc_mixed_cell_test():
    beta = torch.full((3,), 2.51, dtype=F64)
    _, _, m = Rc.thinc_faces(t([0.0, 0.5, 0.4]), beta)  # not monotone
    assert not bool(m[1])
    _, _, m = Rc.thinc_faces(t([0.0, 1e-7, 1.0]), beta)  # C below delta
    assert not bool(m[1])


def test_bvd_prefers_thinc_at_a_step_and_muscl_on_a_ramp():
    step = t([0.0, 0.0, 0.0, 0.0, 0.5, 1.0, 1.0, 1.0, 1.0])
    ramp = t(np.linspace(0, 1, 9))
    for prof, expect_thinc in ((step, True), (ramp, False)):
        mL, mR = Rc.muscl_faces(prof)
        tL, tR, mixed = Rc.thinc_faces(prof, torch.full_like(prof, 2.51))
        L, R = Rc.bvd_select(mL, mR, tL, tR, mixed)
        used_thinc = bool(mixed[4]) and (L[4] != mL[4]).item()
        assert used_thinc == expect_thinc


def test_youngs_normal_of_a_plane():
    ny, nx = 6, 7
    yy, xx = torch.meshgrid(t(np.arange(ny)), t(np.arange(nx)), indexing="ij")
    phi = 0.3 * xx * 0.5 - 0.2 * yy * 2.0
    anx, any_ = Rc.youngs_abs_normal(phi, 0.5, 2.0)
    gx, gy = 0.3, 0.2  # physical gradient components
    assert torch.allclose(anx[1:-1, 1:-1], torch.full((ny - 2, nx - 2), gx / math.hypot(gx, gy), dtype=F64))
    assert torch.allclose(any_[1:-1, 1:-1], torch.full((ny - 2, nx - 2), gy / math.hypot(gx, gy), dtype=F64))


def _prim_batch(n, gen, solid=True):
    phi = t(np.random.default_rng(2).uniform(0.1, 0.9, n))
    return dict(phi1=phi, rho1=8000 * (1 + 0.1 * torch.rand(n, generator=gen, dtype=F64)),
                rho2=1.2 * (1 + torch.rand(n, generator=gen, dtype=F64)),
                u=100 * torch.randn(n, 3, generator=gen, dtype=F64) * t([1, 1, 0]),
                p=1e5 + 1e8 * torch.rand(n, generator=gen, dtype=F64),
                V=rand_stretch(n, 0.01 if solid else 0.0, gen))


@pytest.mark.parametrize("d", [0, 1])
def test_hllc_consistency(d):
    """Equal left and right states: the flux is the physical flux (Section 3)."""
    gen = torch.Generator().manual_seed(3)
    w = _prim_batch(16, gen)
    F, phi_f, u_f, V_f = Rm.hllc(w, w, d, [SOLID, GAS])
    s = Rm.face_state(w, [SOLID, GAS])
    Fp = Rm.physical_flux(s, d)
    for k in Fp:
        assert torch.allclose(F[k], Fp[k], rtol=1e-12, atol=1e-6)
    assert torch.equal(phi_f, w["phi1"])
    assert torch.allclose(u_f, w["u"]) and torch.allclose(V_f, w["V"])


def test_hllc_mirror_symmetry():
    """Mirroring x -> -x maps the flux of (L, R) to minus the mirrored flux of (R', L')."""
    gen = torch.Generator().manual_seed(4)
    wl, wr = _prim_batch(16, gen), _prim_batch(16, gen)
    P = torch.diag(t([-1.0, 1.0, 1.0]))

    def mirror(w):
        m = dict(w)
        m["u"] = w["u"] @ P
        m["V"] = P @ w["V"] @ P
        return m

    F, phi_f, u_f, V_f = Rm.hllc(wl, wr, 0, [SOLID, GAS])
    Fm, phi_m, u_m, V_m = Rm.hllc(mirror(wr), mirror(wl), 0, [SOLID, GAS])
    for k in ("ar1", "ar2", "E"):
        assert torch.allclose(F[k], -Fm[k], rtol=1e-10, atol=1e-3)
    # momentum is odd under the mirror in its x component and the flux direction flips
    assert torch.allclose(F["mom"], -(Fm["mom"] @ P), rtol=1e-10, atol=1e-3)
    assert torch.allclose(u_f, u_m @ P, rtol=1e-12, atol=1e-9)
    assert torch.allclose(V_f, P @ V_m @ P, rtol=1e-12, atol=1e-12)


def test_hllc_star_stretch_keeps_determinant():
    gen = torch.Generator().manual_seed(5)
    wl, wr = _prim_batch(32, gen), _prim_batch(32, gen)
    wr["u"][:, 0] -= 300.0  # compressive
    _, _, _, V_f = Rm.hllc(wl, wr, 0, [SOLID, GAS])
    detL, detR = torch.linalg.det(wl["V"]), torch.linalg.det(wr["V"])
    dv = torch.linalg.det(V_f)
    assert torch.all(torch.minimum((dv - detL).abs(), (dv - detR).abs()) < 1e-12)


@pytest.mark.parametrize("d", [0, 1])
def test_hllc_star_states_satisfy_rankine_hugoniot(d):
    """Each HLLC star state obeys S_K (Q* - Q_K) = F(Q*) - F(Q_K) for mass,
    momentum and energy (the jump conditions it is built from)."""
    gen = torch.Generator().manual_seed(11)
    wl, wr = _prim_batch(32, gen), _prim_batch(32, gen)
    wr["u"][:, d] -= 200.0
    mats = [SOLID, GAS]
    L, R = Rm.face_state(wl, mats), Rm.face_state(wr, mats)
    unL, unR = L["u"][..., d], R["u"][..., d]
    SL = torch.minimum(unL - L["cL"], unR - R["cL"])
    SR = torch.maximum(unL + L["cL"], unR + R["cL"])
    mL, mR = L["rho"] * (SL - unL), R["rho"] * (SR - unR)
    Sst = (L["sigma"][..., d, d] - R["sigma"][..., d, d] + mL * unL - mR * unR) / (mL - mR)
    for K, S in ((L, SL), (R, SR)):
        Q, us, _ = Rm.star_state(K, S, Sst, d)
        un = K["u"][..., d]
        m = K["rho"] * (S - un)
        sig_n = K["sigma"][..., :, d].clone()
        sig_s = sig_n.clone()
        sig_s[..., d] = sig_n[..., d] - m * (Sst - un)
        F = Rm.physical_flux(K, d)
        Fs = dict(ar1=Q["ar1"] * Sst, ar2=Q["ar2"] * Sst,
                  mom=Q["mom"] * Sst[..., None] - sig_s,
                  E=Q["E"] * Sst - (us * sig_s).sum(-1))
        for k in ("ar1", "ar2", "mom", "E"):
            Sk = S[..., None] if Q[k].dim() > S.dim() else S
            res = Sk * (Q[k] - K[k]) - (Fs[k] - F[k])
            scale = F[k].abs() + (Sk * K[k]).abs() + 1.0
            assert (res.abs() / scale).max().item() < 1e-12, k


def _hlld_parts(wl, wr, d, mats):
    """Recompute the HLLD pieces the oracle uses (for jump-condition pins)."""
    L, R = Rm.face_state(wl, mats), Rm.face_state(wr, mats)
    unL, unR = L["u"][..., d], R["u"][..., d]
    SL = torch.minimum(unL - L["cL"], unR - R["cL"])
    SR = torch.maximum(unL + L["cL"], unR + R["cL"])
    mL, mR = L["rho"] * (SL - unL), R["rho"] * (SR - unR)
    Sst = (L["sigma"][..., d, d] - R["sigma"][..., d, d] + mL * unL - mR * unR) / (mL - mR)
    return L, R, SL, SR, Sst


@pytest.mark.parametrize("d", [0, 1])
def test_hlld_shear_jumps_satisfy_rankine_hugoniot(d):
    """Across each shear wave S*_K: S*_K (Q** - Q*) = F(Q**) - F(Q*), and the
    tangential velocity and traction of the two double-star states agree."""
    gen = torch.Generator().manual_seed(12)
    wl, wr = _prim_batch(32, gen), _prim_batch(32, gen)
    t = 1 - d
    wr["u"][:, t] += 80.0  # shear
    mats = [SOLID, SOLID]
    L, R, SL, SR, Sst = _hlld_parts(wl, wr, d, mats)
    tm = torch.ones(3, dtype=F64)
    tm[d] = 0.0
    Qs, us, Vs, cs = {}, {}, {}, {}
    for side, K, S in (("L", L, SL), ("R", R, SR)):
        Qs[side], us[side], Vs[side] = Rm.star_state(K, S, Sst, d)
        cs[side] = torch.sqrt(K["Gm"] / (Qs[side]["ar1"] + Qs[side]["ar2"]))
    Z = {k: (Qs[k]["ar1"] + Qs[k]["ar2"]) * cs[k] for k in "LR"}
    st = {k: K["sigma"][..., :, d] * tm for k, K in (("L", L), ("R", R))}
    ut = {k: K["u"] * tm for k, K in (("L", L), ("R", R))}
    ut2 = (Z["L"][..., None] * ut["L"] + Z["R"][..., None] * ut["R"] + st["R"] - st["L"]) / (Z["L"] + Z["R"])[..., None]
    st2 = st["L"] + Z["L"][..., None] * (ut2 - ut["L"])
    st2R = st["R"] - Z["R"][..., None] * (ut2 - ut["R"])
    assert torch.allclose(st2, st2R, rtol=1e-12, atol=1e-3)  # common traction at the contact
    for side, K, sgn in (("L", L, -1.0), ("R", R, 1.0)):
        Ssh = Sst + sgn * cs[side]
        Q2, u2, V2 = Rm.shear_state(K, Qs[side], us[side], Vs[side], Ssh, Sst, ut2, st2, d)
        m = K["rho"] * ((SL if side == "L" else SR) - K["u"][..., d])
        snn_s = K["sigma"][..., d, d] - m * (Sst - K["u"][..., d])
        trac_s = st[side].clone()
        trac_s[..., d] = snn_s
        trac_2 = st2.clone()
        trac_2[..., d] = snn_s

        def flux(Q, u, trac):
            return dict(ar1=Q["ar1"] * Sst, mom=Q["mom"] * Sst[..., None] - trac,
                        E=Q["E"] * Sst - (u * trac).sum(-1))
        F1, F2 = flux(Qs[side], us[side], trac_s), flux(Q2, u2, trac_2)
        for k in ("ar1", "mom", "E"):
            Sk = Ssh[..., None] if Q2[k].dim() > Ssh.dim() else Ssh
            res = Sk * (Q2[k] - Qs[side][k]) - (F2[k] - F1[k])
            scale = F1[k].abs() + (Sk * Qs[side][k]).abs() + 1.0
            assert (res.abs() / scale).max().item() < 1e-12, (side, k)
        assert torch.allclose(torch.linalg.det(V2), torch.linalg.det(Vs[side]), rtol=1e-13)


def test_hlld_flux_continuous_across_stationary_contact():
    """Mirror-symmetric states give S* = 0; the double-star fluxes from both
    sides coincide, so the tie rule does not matter."""
    gen = torch.Generator().manual_seed(13)
    w = _prim_batch(16, gen)
    w["u"][:, 0] = 150.0
    P = torch.diag(t([-1.0, 1.0, 1.0]))
    m = dict(w)
    m["u"] = w["u"] @ P
    m["V"] = P @ w["V"] @ P
    F, _, u_f, _ = Rm.hllc(w, m, 0, [SOLID, GAS])
    Fm, _, _, _ = Rm.hllc(w, m, 0, [SOLID, GAS])
    assert torch.allclose(u_f[..., 0], torch.zeros(16, dtype=F64), atol=1e-9)
    assert F["ar1"].abs().max().item() < 1e-6 * (w["rho1"] * 150).max().item()


def test_reflective_wall_face_takes_the_left_star_state():
    """At a reflective wall the two face states are exact mirror images
    (u_n, V12, V21 negated).  The contact speed's numerator then cancels
    exactly, S* = 0 (as -0.0), and the tie rule S* >= 0 picks the left
    (x-low side) star state: u_face has a zero normal component, and V12 of
    the face is the left star value, which is minus the right one."""
    gen = torch.Generator().manual_seed(12)
    w = _prim_batch(16, gen, solid=True)
    w["u"][:, 0] += 50.0 * torch.sign(w["u"][:, 0])  # flow into / out of the wall
    P = torch.diag(t([-1.0, 1.0, 1.0]))
    m = dict(w)
    m["u"] = w["u"] @ P
    m["V"] = P @ w["V"] @ P
    F, phi_f, u_f, V_f = Rm.hllc(m, w, 0, [SOLID, GAS])
    assert torch.all(u_f[:, 0] == 0.0)
    # moving the right state by +-1e-7 m/s puts S* just right or left of the
    # face: the exact tie takes the limit from the S* > 0 side (left star state)
    wp, wm = dict(w), dict(w)
    wp["u"] = w["u"] + t([1e-7, 0.0, 0.0])
    wm["u"] = w["u"] - t([1e-7, 0.0, 0.0])
    _, _, up, Vp = Rm.hllc(m, wp, 0, [SOLID, GAS])
    _, _, um, Vm = Rm.hllc(m, wm, 0, [SOLID, GAS])
    assert torch.all(up[:, 0] > 0) and torch.all(um[:, 0] < 0)
    assert torch.allclose(V_f, Vp, rtol=1e-6, atol=1e-12)
    assert torch.allclose(V_f[:, 0, 1], -Vm[:, 0, 1], rtol=1e-6, atol=1e-12)
    assert torch.all(V_f[:, 0, 1].abs() > 1e-8)


# ---- Romenskii and JWL reference curves (Section 2.3) ----------------------
CU = W.COPPER_ROMENSKII
LX = W.LX17_REACTANT_JWL


@pytest.mark.parametrize("m", [CU, LX], ids=["romenskii", "jwl"])
@pytest.mark.parametrize("J2v", [0.0, 2e-4])
def test_reference_pressure_is_rho2_dE_ref(m, J2v):
    """p_ref = rho^2 dE_ref/drho (Section 2.3), by central differences of the
    reference energy, and the closed-form derivatives used by the sound speed."""
    J2 = t([J2v])
    for x in (0.8, 1.0, 1.15, 1.4):
        rho = m["rho0"] * x
        h = rho * 1e-6
        dE = (C.e_ref(m, t([rho + h]), J2) - C.e_ref(m, t([rho - h]), J2)).item() / (2 * h)
        pr = C.p_ref(m, t([rho]), J2).item()
        assert abs(rho * rho * dE - pr) <= 1e-6 * max(abs(pr), 1e5), (x, rho * rho * dE, pr)
        dp = (C.p_ref(m, t([rho + h]), J2) - C.p_ref(m, t([rho - h]), J2)).item() / (2 * h)
        assert abs(dp - C.dp_ref_drho(m, t([rho]), J2).item()) <= 1e-6 * abs(dp) + 1e-3
        assert abs(dE - C.de_ref_drho(m, t([rho]), J2).item()) <= 1e-6 * abs(dE) + 1e-9


def test_romenskii_copper_at_reference_density():
    """At rho0 the cold curves vanish, the bulk sound speed is K0 / rho0 and the
    shear modulus is G0; G scales as (rho / rho0)^(beta + 1) = x^4."""
    r0 = t([CU["rho0"]])
    z = t([0.0])
    assert C.p_ref(CU, r0, z).item() == 0.0 and C.e_ref(CU, r0, z).item() == 0.0
    c2 = C.material_sound_speed2(CU, r0, t([0.0]), z).item()
    assert abs(c2 / (136.5e9 / 8930.0) - 1) < 1e-12
    assert C.shear_modulus(CU, r0).item() == 39.4e9
    assert abs(C.shear_modulus(CU, r0 * 1.1).item() / 39.4e9 - 1.1 ** 4) < 1e-12


def test_jwl_reference_pressure_at_rho0():
    """p_ref(rho0) = A e^(-R1) + B e^(-R2) with the table's LX-17 reactant
    constants: 778.1e11 e^-11.3 - 0.0503e11 e^-1.13 = -6.6212e8 Pa."""
    pr = C.p_ref(LX, t([1905.0]), t([0.0])).item()
    assert abs(pr / (778.1e11 * math.exp(-11.3) - 0.0503e11 * math.exp(-1.13)) - 1) < 1e-12
    assert abs(pr / -6.6212e8 - 1) < 1e-4


@pytest.mark.parametrize("m", [CU, LX], ids=["romenskii", "jwl"])
def test_sound_speed_is_isentropic_derivative_other_families(m):
    """c^2 = (dp/drho)_s along de = p / rho^2 drho for the Romenskii and JWL
    closures (pure material, strained for Romenskii)."""
    rho0, p0 = m["rho0"] * 1.05, 3e9
    J2 = t([1e-4 if m is CU else 0.0])
    phis = [t([1.0]), t([0.0])]
    mats = [m, GAS]

    def p_of(rho, e):
        return C.mixture_pressure(phis, [t([rho]), t([1.0])], t([rho * e]), J2, mats).item()

    e0 = C.material_energy(m, t([rho0]), t([p0]), J2).item()
    h = 1e-3
    num = (p_of(rho0 + h, e0 + p0 / rho0 ** 2 * h) - p_of(rho0 - h, e0 - p0 / rho0 ** 2 * h)) / (2 * h)
    c2 = C.material_sound_speed2(m, t([rho0]), t([p0]), J2).item()
    assert abs(num - c2) / c2 < 1e-6


# ---- Reactive mixture with distinct closures: Appendix B ------------------
EXPL = W.generic_explosive()


def _mix_state(lam, p, rho_y=1600.0, phi_y=1.0 - 1e-8):
    """A cell of copper trace + explosive (primitive), as the oracle's dicts."""
    cu = W.material(3.0, p_inf=136.5e9 / 3.0, G=39.4e9)
    mats = [cu, EXPL]
    one = torch.ones(1, dtype=F64)
    w = dict(phi1=one * (1 - phi_y), rho1=one * 8930.0, rho2=one * rho_y,
             u=torch.zeros(1, 3, dtype=F64), p=one * p, V=torch.eye(3, dtype=F64)[None], lam=one * lam)
    return w, mats


def test_mixture_temperature_equality_and_mixture_rule():
    """At the share s found from the conservative state (bisection), the
    reactant and product temperatures are equal and the component densities
    satisfy the mixture rule 1/rho_y = lam/rho_a + (1 - lam)/rho_b."""
    for lam in (0.05, 0.3, 0.5, 0.9):
        for p in (1e5, 1e9, 2e10):
            w, mats = _mix_state(lam, p)
            q = C.prim_to_cons(w, mats)
            back = C.cons_to_prim(q, mats)
            # the reactant's stiff part gamma p_inf = 4e9 Pa sets the round-off scale
            assert abs(back["p"].item() - p) < 1e-13 * (p + 4e9), (lam, p, back["p"].item())
            s = C.reactant_share(EXPL, torch.tensor(lam, dtype=F64), back["p"]).item()
            ry = 1600.0
            ra, rb = lam * ry / s, (1 - lam) * ry / (1 - s)
            Ta = (p + 4.0 * 1e9) / (ra * 3.0 * 2000.0)
            Tb = (p + 0.0) / (rb * 2.0 * 1000.0)
            assert abs(Ta / Tb - 1) < 1e-10, (lam, p, Ta, Tb)
            assert abs(1 / ry - (lam / ra + (1 - lam) / rb)) < 1e-12 / ry


def test_mixture_share_hand_solution():
    """lam = 0.5 at p = 1 GPa: s = lam G_a Cv_a (p + gb pb) / (...) with
    Gamma_a C_V,a = 3 x 2000 = 6000, Gamma_b C_V,b = 2 x 1000 = 2000,
    p + gamma_a p_inf,a = 5e9, p + gamma_b p_inf,b = 1e9:
    s = 0.5 x 6000 x 1e9 / (0.5 x 6000 x 1e9 + 0.5 x 2000 x 5e9) = 3/8."""
    s = C.reactant_share(EXPL, torch.tensor(0.5, dtype=F64), torch.tensor(1e9, dtype=F64)).item()
    assert abs(s - 0.375) < 1e-15


def test_identical_closures_reduce_to_the_closed_form():
    """Giving the product the reactant's closure explicitly (two-closure path,
    bisection) reproduces the closed-form pressure of identical closures."""
    m1 = W.material(1.4, reactive=1, Q=2e6, cv=717.5, A=1.0, T_act=1.0)
    m2 = dict(m1, prod_gamma=1.4, prod_p_inf=0.0, prod_cv=717.5)
    air = W.AIR
    for lam in (0.2, 0.7):
        one = torch.ones(1, dtype=F64)
        w = dict(phi1=one * 0.3, rho1=one * 1.2, rho2=one * 2.0, u=torch.zeros(1, 3, dtype=F64),
                 p=one * 3e5, V=torch.eye(3, dtype=F64)[None], lam=one * lam)
        q1 = C.prim_to_cons(w, [air, m1])
        q2 = C.prim_to_cons(w, [air, m2])
        assert torch.allclose(q1["E"], q2["E"], rtol=1e-14)
        p2 = C.cons_to_prim(q1, [air, m2])["p"]
        assert abs(p2.item() / 3e5 - 1) < 1e-12


def test_mixture_sound_speed_limits():
    """lam = 1: the reactant's gamma (p + p_inf) / rho; lam = 0: the product's."""
    for lam, g, pi in ((1.0, 4.0, 1e9), (0.0, 3.0, 0.0)):
        c2 = C.material_sound_speed2(EXPL, t([1600.0]), t([2e9]), t([0.0]), t([lam])).item()
        assert abs(c2 / (g * (2e9 + pi) / 1600.0) - 1) < 1e-12
