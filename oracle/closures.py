"""Oracle closures: equations of state, mixture rules, strain and stress.

TEST INFRASTRUCTURE ONLY.  Plain PyTorch CPU float64, written for reading
against the paper, not for speed.  Nothing in the product path imports it.

Cites (Wallis, Barton & Nikiforakis, arXiv 2009.14555):
  * Section 2.2, Eqs. for E_s, J^2, sigma, p, dev(sigma) and the mixture rules
    (phi, rho, rho*E, G, c^2, sigma weighted by phi/Gamma);
  * Section 2.3, Mie-Grueneisen form p = p_ref + rho*Gamma*(E - E_ref) with the
    stiffened-gas reference curves;
  * Section 2.3.1, reactive physical mixture (lambda, Q shift of the product
    reference energy, MiNi16 mixture sound speed);
  * Section 3.2, Bazant approximation of the Hencky strain;
  * Appendix B, pressure function and temperature.

Readings taken where the paper is silent or garbled:
  * sigma = -p I + dev(sigma) (the flux rho u u - sigma needs the minus sign);
  * E = e + |u|^2 / 2;
  * stiffened-gas solid with constant shear modulus G: the shear energy
    G J^2 / rho enters E_ref, so p_ref = -gamma p_inf - G J^2 and
    E_ref = e_inf + G J^2 / rho;
  * mixture sound speed c^2 = sum(Y_l c_l^2 / Gamma_l) / sum(phi_l / Gamma_l)
    (the printed numerator carries a spurious extra phi);
  * dev(H) is taken as dev(1/4 (B - B^-1)) with B = V V^T (explicit deviator);
  * a reactive material has identical ideal-gas reactant and product closures
    (same gamma and C_V), so the temperature equality of Appendix B gives
    rho_alpha = rho_beta = rho_y and the pressure function is closed form;
  * Johnson-Cook solid (Section 2.3.2): its temperature carries the thermal
    energy of Section 2.2, E_t = C_V (T - T0 theta_D(rho)), with the Debye
    temperature theta_D = (rho/rho0)^Gamma of a constant Grueneisen
    coefficient (Gamma = rho theta_D' / theta_D; the printed derivative with
    respect to ln(1/rho) has the opposite sign), and T0 the Johnson-Cook
    reference temperature (298 K); the homologous temperature of the thermal
    softening is clamped to [0, 1].
"""
from __future__ import annotations

import torch

F64 = torch.float64


PLASTIC_NONE, PLASTIC_PERFECT, PLASTIC_IDEAL, PLASTIC_JC = 0, 1, 2, 3


def Gamma(m) -> float:
    """Grueneisen coefficient Gamma = gamma - 1 (Section 2.3, ideal/stiffened gas)."""
    return m["gamma"] - 1.0


def history_material(mats):
    """Index of the material carrying the history row rho_y phi_y alpha_y of
    Section 2.1: the reactive material (alpha = lam, Section 2.3.1) or a
    Johnson-Cook solid (alpha = eps_p, Section 2.3.2); None without one."""
    for i, m in enumerate(mats):
        if m["reactive"] or m["plastic"] == PLASTIC_JC:
            return i
    return None


# ----------------------------------------------------------------------------
# Strain: Section 2.2 (J^2) and Section 3.2 (Bazant approximation).
# ----------------------------------------------------------------------------
def stretch_matrix(V11, V12, V21, V22, V33):
    """Assemble the 3x3 stretch tensor of plane strain (z rows/cols diagonal)."""
    z = torch.zeros_like(V11)
    rows = [torch.stack([V11, V12, z], -1),
            torch.stack([V21, V22, z], -1),
            torch.stack([z, z, V33], -1)]
    return torch.stack(rows, -2)


def dev(M):
    """Matrix deviator dev(M) = M - tr(M)/3 I (footnote of Section 2.2)."""
    tr = torch.diagonal(M, dim1=-2, dim2=-1).sum(-1)
    eye = torch.eye(3, dtype=M.dtype).expand(M.shape)
    return M - (tr / 3.0)[..., None, None] * eye


def hencky_dev(V):
    """dev(H) ~ 1/2 H_B^(1)(V V^T),  H_B^(m)(X) = (X^m - X^-m) / (2m)  (Section 3.2).

    Returns (devH, J2) with J2 = tr(devH devH^T) (Section 2.2).
    """
    B = V @ V.transpose(-1, -2)
    HB1 = 0.5 * (B - torch.linalg.inv(B))
    devH = dev(0.5 * HB1)
    J2 = (devH * devH).sum((-1, -2))
    return devH, J2


# ----------------------------------------------------------------------------
# Reference curves of the Mie-Grueneisen form (Section 2.3, reading above).
#
# Three families (m["eos"]), all with a constant Gamma = gamma - 1:
#   "sg"  stiffened gas (the default): cold pressure -gamma p_inf, cold energy
#         e_inf, constant shear modulus G;
#   "romenskii" (Section 2.3, elastic solids): cold energy
#         K0 / (2 rho0 a^2) ((rho/rho0)^a - 1)^2 and its pressure
#         rho^2 dE_c/drho = (K0 / a) x^(a+1) (x^a - 1), x = rho / rho0, and the
#         shear modulus G(rho) = G0 x^(b+1) (a, b: the exponents alpha-bar,
#         beta-bar; G0 = m["G"]).  Reading: the printed cold energy lacks the
#         square and has rho for rho0, which would give a reference pressure
#         K0 / (2 a) at rho0; this form has zero pressure and bulk modulus K0
#         there;
#   "jwl" (Section 2.3, explosives and products): cold pressure
#         A e^(-R1 rho0/rho) + B e^(-R2 rho0/rho) and cold energy
#         A / (R1 rho0) e^(-R1 rho0/rho) + B / (R2 rho0) e^(-R2 rho0/rho).
# The shear energy G(rho) J2 / rho adds (rho G' - G) J2 to the reference
# pressure (rho^2 times its density derivative).
# ----------------------------------------------------------------------------
def eos_kind(m):
    return m.get("eos", "sg")


def shear_modulus(m, rho):
    """G(rho) of Section 2.3 (constant except for the Romenskii solid)."""
    if eos_kind(m) == "romenskii":
        return m["G"] * (rho / m["rho0"]) ** (m["beta_r"] + 1.0)
    return m["G"] + 0.0 * rho


def _shear_p_factor(m, rho):
    """rho G'(rho) - G(rho) and its density derivative."""
    if eos_kind(m) == "romenskii":
        b = m["beta_r"]
        G = shear_modulus(m, rho)
        return b * G, b * (b + 1.0) * G / rho
    return -m["G"] + 0.0 * rho, 0.0 * rho


def cold_curves(m, rho):
    """(E_c, p_c, dE_c/drho, dp_c/drho) of the cold (J2 = 0) reference curves."""
    kind = eos_kind(m)
    if kind == "romenskii":
        a, K0, r0 = m["alpha_r"], m["K0"], m["rho0"]
        x = rho / r0
        xa = x ** a
        Ec = K0 / (2.0 * r0 * a * a) * (xa - 1.0) ** 2
        pc = K0 / a * x ** (a + 1.0) * (xa - 1.0)
        dpc = K0 / (a * r0) * xa * ((2.0 * a + 1.0) * xa - (a + 1.0))
        return Ec, pc, pc / (rho * rho), dpc
    if kind == "jwl":
        r0 = m["rho0"]
        e1 = m["jwl_A"] * torch.exp(-m["jwl_R1"] * r0 / rho)
        e2 = m["jwl_B"] * torch.exp(-m["jwl_R2"] * r0 / rho)
        Ec = e1 / (m["jwl_R1"] * r0) + e2 / (m["jwl_R2"] * r0)
        pc = e1 + e2
        dpc = (e1 * m["jwl_R1"] + e2 * m["jwl_R2"]) * r0 / (rho * rho)
        return Ec, pc, pc / (rho * rho), dpc
    z = 0.0 * rho
    return m["e_inf"] + z, -m["gamma"] * m["p_inf"] + z, z, z


def p_ref(m, rho, J2):
    return cold_curves(m, rho)[1] + _shear_p_factor(m, rho)[0] * J2


def e_ref(m, rho, J2):
    return cold_curves(m, rho)[0] + shear_modulus(m, rho) * J2 / rho


def dp_ref_drho(m, rho, J2):
    return cold_curves(m, rho)[3] + _shear_p_factor(m, rho)[1] * J2


def de_ref_drho(m, rho, J2):
    return cold_curves(m, rho)[2] + _shear_p_factor(m, rho)[0] * J2 / (rho * rho)


# ----------------------------------------------------------------------------
# Reactive physical mixture with distinct reactant and product closures
# (Section 2.3.1, Appendix B).  Both components are stiffened gases (no shear
# modulus): the reactant takes the material's gamma, p_inf, C_V; the product
# m["prod_gamma"], m["prod_p_inf"], m["prod_cv"] and the heat release Q.  With
# s = lam rho_y / rho_alpha the reactant's share of the mixture's volume
# (the mixture rule 1/rho_y = lam/rho_alpha + (1 - lam)/rho_beta is
# s + (1 - s) = 1), the pressure function of Appendix B depends on the
# densities only through s, and the temperature equality T_alpha = T_beta
# fixes s: in closed form when p is known (primitive variables), by
# bisection on s in [0, 1] with the pressure function otherwise (the paper's
# bisection on rho_alpha, over the bounded variable).  Identical closures give
# s = lam, rho_alpha = rho_beta = rho_y (the closed form of the other reactive
# closure).  Sound speed: the lam-weighted form of Section 2.3.1 with
# (d rho_k / d rho_y)_p = rho_k / rho_y (reading: the paper leaves this
# derivative unstated; this is compression at fixed composition).
# ----------------------------------------------------------------------------
def two_eos(m):
    return bool(m["reactive"]) and ("prod_gamma" in m or "prod_p_inf" in m or "prod_cv" in m)


def _comps(m):
    g_a, pi_a, cv_a = m["gamma"], m["p_inf"], m["cv"]
    return ((g_a, pi_a, cv_a),
            (m.get("prod_gamma", g_a), m.get("prod_p_inf", pi_a), m.get("prod_cv", cv_a)))


def reactant_share(m, lam, p):
    """s of the temperature equality at pressure p (closed form)."""
    (ga, pa, ca), (gb, pb, cb) = _comps(m)
    wa = lam * (ga - 1.0) * ca * (p + gb * pb)
    wb = (1.0 - lam) * (gb - 1.0) * cb * (p + ga * pa)
    return wa / (wa + wb)


def _mix_terms(m, s):
    """(1/Gamma_y, sum_k share_k kappa_k) of the mixture at reactant share s."""
    (ga, pa, ca), (gb, pb, cb) = _comps(m)
    iG = s / (ga - 1.0) + (1.0 - s) / (gb - 1.0)
    kap = s * ga * pa / (ga - 1.0) + (1.0 - s) * gb * pb / (gb - 1.0)
    return iG, kap


def mixture_share(phis, rhos, rhoe, mats, lam, iters=64):
    """Reactant share s of the reactive material from the conservative state:
    bisection of (T_alpha - T_beta) lam (1 - lam) on [0, 1], the pressure from
    the pressure function at each trial s (Appendix B)."""
    y = next(i for i, m in enumerate(mats) if m["reactive"])
    m = mats[y]
    (ga, pa, ca), (gb, pb, cb) = _comps(m)
    num0 = rhoe.clone()
    den0 = torch.zeros_like(rhoe)
    J2 = torch.zeros_like(rhoe)
    for l, (mm, phi, rho) in enumerate(zip(mats, phis, rhos)):
        if l == y:
            continue
        G = Gamma(mm)
        num0 = num0 + phi * rho * (p_ref(mm, rho, J2) / (rho * G) - e_ref(mm, rho, J2))
        den0 = den0 + phi / G
    phy, rhy = phis[y], rhos[y]

    def pressure(s):
        iG, kap = _mix_terms(m, s)
        return (num0 - phy * kap + phy * rhy * (1.0 - lam) * m["Q"]) / (den0 + phy * iG)

    def g(s):
        p = pressure(s)
        return (1.0 - lam) * (gb - 1.0) * cb * (p + ga * pa) * s - lam * (ga - 1.0) * ca * (p + gb * pb) * (1.0 - s)

    lo = torch.zeros_like(rhoe)
    hi = torch.ones_like(rhoe)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        neg = g(mid) < 0
        lo = torch.where(neg, mid, lo)
        hi = torch.where(neg, hi, mid)
    return 0.5 * (lo + hi)


def material_energy(m, rho, p, J2, lam=None):
    """Specific internal energy of one material from the MG form (Section 2.3).

    For a reactive material, E = lam E_alpha + (1 - lam) E_beta with the product
    reference energy shifted by -Q (Section 2.3.1) and rho_alpha = rho_beta = rho
    (identical closures) or the temperature-equality densities (two closures).
    """
    G = Gamma(m)
    if two_eos(m):
        s = reactant_share(m, lam, p)
        iG, kap = _mix_terms(m, s)
        # rho_y E = sum_k share_k (p + gamma_k p_inf,k) / Gamma_k - rho_y (1 - lam) Q
        return (p * iG + kap) / rho - (1.0 - lam) * m["Q"]
    if m["reactive"]:
        e_a = (p - p_ref(m, rho, J2)) / (rho * G) + e_ref(m, rho, J2)
        e_b = (p - p_ref(m, rho, J2)) / (rho * G) + e_ref(m, rho, J2) - m["Q"]
        return lam * e_a + (1.0 - lam) * e_b
    return (p - p_ref(m, rho, J2)) / (rho * G) + e_ref(m, rho, J2)


def mixture_pressure(phis, rhos, rhoe, J2, mats, lam=None):
    """Pressure function of Appendix B (all materials at one pressure).

    p = [rho e + sum_x phi_x rho_x (p_ref,x/(rho_x Gamma_x) - E_ref,x)
               + phi_y rho_y lam (p_ref,a/(rho_a Gamma_a) - E_ref,a)
               + phi_y rho_y (1-lam) (p_ref,b/(rho_b Gamma_b) - E_ref,b)]
        / [sum_x phi_x/Gamma_x + phi_y rho_y lam/(rho_a Gamma_a)
                               + phi_y rho_y (1-lam)/(rho_b Gamma_b)]
    """
    if any(two_eos(m) for m in mats):
        s = mixture_share(phis, rhos, rhoe, mats, lam)
    num = rhoe.clone()
    den = torch.zeros_like(rhoe)
    for m, phi, rho in zip(mats, phis, rhos):
        G = Gamma(m)
        if two_eos(m):
            iG, kap = _mix_terms(m, s)
            num = num - phi * kap + phi * rho * (1.0 - lam) * m["Q"]
            den = den + phi * iG
        elif m["reactive"]:
            ra = rb = rho  # temperature equality with equal Gamma, C_V
            num = num + phi * rho * lam * (p_ref(m, ra, J2) / (ra * G) - e_ref(m, ra, J2))
            num = num + phi * rho * (1 - lam) * (p_ref(m, rb, J2) / (rb * G)
                                                 - (e_ref(m, rb, J2) - m["Q"]))
            den = den + phi * rho * lam / (ra * G) + phi * rho * (1 - lam) / (rb * G)
        else:
            num = num + phi * rho * (p_ref(m, rho, J2) / (rho * G) - e_ref(m, rho, J2))
            den = den + phi / G
    return num / den


def material_sound_speed2(m, rho, p, J2, lam=None):
    """Squared sound speed of one material at fixed strain.

    Inert material: c^2 = (dp/drho)_E + p/rho^2 (dp/dE)_rho of the MG form.
    Reactive mixture: MiNi16 form of Section 2.3.1,
      c^2 = [p/rho^2 - (dE/drho)_p] / (dE/dp)_rho,
    with rho_alpha = rho_beta = rho so (d rho_alpha/d rho)_p = 1.
    """
    G = Gamma(m)
    if two_eos(m):
        s = reactant_share(m, lam, p)
        iG, kap = _mix_terms(m, s)
        # [p + sum_k share_k (p + gamma_k p_inf,k) / Gamma_k] / (rho / Gamma_y)
        return (p + p * iG + kap) / (rho * iG)
    if m["reactive"]:
        dEdp = lam / (rho * G) + (1 - lam) / (rho * G)
        # (dE_k/drho_k)_p for the MG form: -(p - p_ref)/(rho^2 G) + dp_ref/drho/(... ) terms
        dEa = (-(p - p_ref(m, rho, J2)) / (rho * rho * G)
               - dp_ref_drho(m, rho, J2) / (rho * G) + de_ref_drho(m, rho, J2))
        dEb = dEa
        dEdrho = lam * dEa * 1.0 + (1 - lam) * dEb * 1.0
        return (p / (rho * rho) - dEdrho) / dEdp
    dpdrho = dp_ref_drho(m, rho, J2) + (p - p_ref(m, rho, J2)) / rho - rho * G * de_ref_drho(m, rho, J2)
    dpde = rho * G
    return dpdrho + p / (rho * rho) * dpde


def temperature(m, rho, p, J2, lam=None):
    """T = (p - p_ref) / (rho Gamma C_V)  (Appendix B); for two closures the
    common temperature sum_k share_k (p + gamma_k p_inf,k) / (Gamma_k C_V,k) / rho_y."""
    if two_eos(m):
        (ga, pa, ca), (gb, pb, cb) = _comps(m)
        s = reactant_share(m, lam, p)
        return (s * (p + ga * pa) / ((ga - 1.0) * ca) + (1.0 - s) * (p + gb * pb) / ((gb - 1.0) * cb)) / rho
    return (p - p_ref(m, rho, J2)) / (rho * Gamma(m) * m["cv"])


def jc_temperature(m, rho, p, J2):
    """Temperature of a Johnson-Cook (Romenskii) solid at density rho and
    pressure p: E - E_ref = C_V (T - T0 theta_D(rho)) (Section 2.2) with
    E - E_ref = (p - p_ref) / (rho Gamma) (the Mie-Grueneisen form, Section
    2.3) and theta_D = (rho/rho0)^Gamma."""
    return m["jc_T0"] * (rho / m["rho0"]) ** Gamma(m) + (p - p_ref(m, rho, J2)) / (rho * Gamma(m) * m["cv"])


def jc_yield(m, eps_p, T):
    """Johnson-Cook yield stress of Section 2.3.2,
    sigma_Y = (c1 + c2 eps_p^n) (1 - T*^m), T* = (T - T0) / (T_melt - T0)
    clamped to [0, 1] (no softening below T0, no strength above T_melt);
    eps_p^n of max(eps_p, 0).  c1 is the material's sigma_y."""
    Ts = ((T - m["jc_T0"]) / (m["jc_Tmelt"] - m["jc_T0"])).clamp(0.0, 1.0)
    return (m["sigma_y"] + m["jc_c2"] * eps_p.clamp(min=0.0) ** m["jc_n"]) * (1.0 - Ts ** m["jc_m"])


def inv_gamma(m, p=None, lam=None):
    """1 / Gamma of a material in the mixture rules (phi / Gamma weights):
    s / Gamma_alpha + (1 - s) / Gamma_beta for two reactive closures."""
    if two_eos(m):
        return _mix_terms(m, reactant_share(m, lam, p))[0]
    return 1.0 / Gamma(m)


# ----------------------------------------------------------------------------
# Whole-state closures.  A state is a dict of tensors:
#   phi1, rho1, rho2, u (...,3), p, V (...,3,3), lam      (primitive)
#   phi1, ar1, ar2, mom (...,3), E, V (...,3,3), arl      (conservative)
# ----------------------------------------------------------------------------
def phases(phi1):
    return [phi1, 1.0 - phi1]  # Eq. sum phi = 1 (Section 2.2)


def mixture_props(phis, rhos, p, J2, mats, lam):
    """Mixture G, c^2 and longitudinal c_L^2 (Section 2.2 mixture rules)."""
    rho = sum(ph * r for ph, r in zip(phis, rhos))
    ig = [inv_gamma(m, p, lam) for m in mats]
    xi = sum(ph * g for ph, g in zip(phis, ig))
    Gm = sum(ph * shear_modulus(m, r) * g for ph, r, m, g in zip(phis, rhos, mats, ig)) / xi
    c2 = sum((ph * r / rho) * material_sound_speed2(m, r, p, J2, lam) * g
             for ph, r, m, g in zip(phis, rhos, mats, ig)) / xi
    cL2 = c2 + (4.0 / 3.0) * Gm / rho
    return rho, Gm, c2, cL2


def stress(p, Gm, devH):
    """sigma = -p I + 2 G devH (Section 2.2, sign reading above)."""
    eye = torch.eye(3, dtype=p.dtype).expand(devH.shape)
    return -p[..., None, None] * eye + 2.0 * Gm[..., None, None] * devH


def prim_to_cons(w, mats):
    """Conservative state from primitives (MG form solved for E, mixture rules)."""
    phis = phases(w["phi1"])
    rhos = [w["rho1"], w["rho2"]]
    devH, J2 = hencky_dev(w["V"])
    rho = phis[0] * rhos[0] + phis[1] * rhos[1]
    rhoe = sum(ph * r * material_energy(m, r, w["p"], J2, w.get("lam"))
               for ph, r, m in zip(phis, rhos, mats))
    ke = 0.5 * rho * (w["u"] * w["u"]).sum(-1)
    q = dict(phi1=w["phi1"], ar1=phis[0] * rhos[0], ar2=phis[1] * rhos[1],
             mom=rho[..., None] * w["u"], E=rhoe + ke, V=w["V"])
    if "lam" in w:
        y = history_material(mats)
        q["arl"] = q["ar1" if y == 0 else "ar2"] * w["lam"]
    return q


def cons_to_prim(q, mats):
    """Primitives from the conservative state (pressure function of Appendix B)."""
    phis = phases(q["phi1"])
    ars = [q["ar1"], q["ar2"]]
    rhos = [ars[0] / phis[0], ars[1] / phis[1]]
    rho = ars[0] + ars[1]
    u = q["mom"] / rho[..., None]
    rhoe = q["E"] - 0.5 * rho * (u * u).sum(-1)
    devH, J2 = hencky_dev(q["V"])
    lam = None
    if "arl" in q:
        y = history_material(mats)
        lam = q["arl"] / ars[y]
    p = mixture_pressure(phis, rhos, rhoe, J2, mats, lam)
    w = dict(phi1=q["phi1"], rho1=rhos[0], rho2=rhos[1], u=u, p=p, V=q["V"])
    if lam is not None:
        w["lam"] = lam
    return w
