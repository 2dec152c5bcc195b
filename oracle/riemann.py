"""Oracle Riemann solver: HLLD-type flux for the elastic diffuse-interface system.

TEST INFRASTRUCTURE ONLY (plain PyTorch CPU float64).

The paper (Section 3.1) uses the HLLD solver of Barton (2019), whose formulas
it does not print.  The reading taken here is an HLLD-type solver with five
waves (two longitudinal, two shear, one contact), written from the
Rankine-Hugoniot conditions of the conservative part of the system (vector
form of Section 3).  Without the shear waves (an HLLC-type solver) elastic
shear modes of a 2D solid get no dissipation and grow without bound.
Longitudinal waves and the contact:

  * wave speeds: Davis bounds with the longitudinal sound speed c_L;
  * contact speed S* from continuity of the normal traction sigma_nn
    (HLLC with p replaced by -sigma_nn);
  * star state of side K: density ratio r = (S_K - u_nK)/(S_K - S*); partial
    densities scaled by r, phi unchanged, u* = u_K with its normal component
    replaced by S*, sigma*_n from the normal-momentum jump, energy from the
    energy jump E*(S_K - S*) = E_K (S_K - u_nK) + u_K.sigma_n,K - u*.sigma*_n,
    and the stretch tensor from the kinematic jump of a planar
    wave, V* = det(F_w)^(-1/3) F_w V_K with F_w = I + (u_K - u*) n^T/(S_K - u_nK);
Shear waves at S*_L = S* - c_s,L and S*_R = S* + c_s,R, c_s^2 = G_mix / rho*
(star densities): across them u_n, sigma_nn and the densities stay, while the
tangential velocity and traction meet a common value across the contact,
from the shear impedances Z_K = rho*_K c_s,K:
    u_t** = (Z_L u_t,L + Z_R u_t,R + s_t,R - s_t,L) / (Z_L + Z_R),
    s_t** = s_t,L + Z_L (u_t** - u_t,L)    (s_t = tangential traction),
the energy from its jump E** (S*_K - S*) = E* (S*_K - S*) - (u_t** s_t** - u_t,K s_t,K),
and V** = (I + w e_t n^T) V* with w = (u_t,K - u_t**) / (S*_K - S*)
(a shear jump keeps the determinant).  With Z_L + Z_R = 0 (two fluids) the
shear waves and the contact coincide and the solver is HLLC.

Conservative fields take the nested HLL jumps F*_K = F_K + S_K (Q*_K - Q_K),
F**_K = F*_K + S*_K (Q**_K - Q*_K); phi and V take the flux of the state
found at x/t = 0, which also supplies the face velocity and stretch used by
the non-conservative terms.

Tie rule at x/t = 0: S_L >= 0 -> L; else S*_L >= 0 -> *L; else S* >= 0 -> **L;
else S*_R >= 0 -> **R; else S_R >= 0 -> *R; else R.  (The ** fluxes are
continuous across S* = 0.)
"""
from __future__ import annotations

import torch

from .closures import history_material, hencky_dev, mixture_props, phases, stress, material_energy

CONS_KEYS = ("ar1", "ar2", "mom", "E", "arl")


def face_state(w, mats):
    """Everything the flux needs from one reconstructed primitive state."""
    phis = phases(w["phi1"])
    rhos = [w["rho1"], w["rho2"]]
    devH, J2 = hencky_dev(w["V"])
    lam = w.get("lam")
    rho, Gm, c2, cL2 = mixture_props(phis, rhos, w["p"], J2, mats, lam)
    rhoe = sum(ph * r * material_energy(m, r, w["p"], J2, lam)
               for ph, r, m in zip(phis, rhos, mats))
    s = dict(phi1=w["phi1"], rho=rho, u=w["u"], V=w["V"], Gm=Gm,
             ar1=phis[0] * rhos[0], ar2=phis[1] * rhos[1],
             mom=rho[..., None] * w["u"],
             E=rhoe + 0.5 * rho * (w["u"] * w["u"]).sum(-1),
             sigma=stress(w["p"], Gm, devH), cL=torch.sqrt(cL2))
    if lam is not None:
        y = history_material(mats)
        s["arl"] = s["ar1" if y == 0 else "ar2"] * lam
    return s


def physical_flux(s, d):
    """Conservative flux along axis d: (ar u_d, rho u u_d - sigma_{.d},
    E u_d - u_i sigma_{id}, arl u_d)."""
    un = s["u"][..., d]
    sig_n = s["sigma"][..., :, d]
    F = dict(ar1=s["ar1"] * un, ar2=s["ar2"] * un,
             mom=s["mom"] * un[..., None] - sig_n,
             E=s["E"] * un - (s["u"] * sig_n).sum(-1))
    if "arl" in s:
        F["arl"] = s["arl"] * un
    return F


def star_state(s, S, Sst, d):
    un = s["u"][..., d]
    m = s["rho"] * (S - un)
    r = (S - un) / (S - Sst)
    ustar = s["u"].clone()
    ustar[..., d] = Sst
    sig_n = s["sigma"][..., :, d]
    sig_n_star = sig_n.clone()
    sig_n_star[..., d] = sig_n[..., d] - m * (Sst - un)
    # energy jump across the wave: S (E* - E) = (E* S* - u*.sigma*_n) - (E u_n - u.sigma_n)
    Estar = (s["E"] * (S - un) + (s["u"] * sig_n).sum(-1)
             - (ustar * sig_n_star).sum(-1)) / (S - Sst)
    n = torch.zeros_like(s["u"])
    n[..., d] = 1.0
    eye = torch.eye(3, dtype=un.dtype).expand(s["V"].shape)
    Fw = eye + (s["u"] - ustar)[..., :, None] * n[..., None, :] / (S - un)[..., None, None]
    Vstar = torch.linalg.det(Fw).pow(-1.0 / 3.0)[..., None, None] * (Fw @ s["V"])
    Q = dict(ar1=r * s["ar1"], ar2=r * s["ar2"], mom=(r * s["rho"])[..., None] * ustar,
             E=Estar)
    if "arl" in s:
        Q["arl"] = r * s["arl"]
    return Q, ustar, Vstar


def shear_state(K, Qs, us, Vs, S_sh, Sst, ut2, st2, d):
    """Double-star state of side K across its shear wave at speed S_sh."""
    tmask = torch.ones(3, dtype=ut2.dtype)
    tmask[d] = 0.0
    ut_s = us * tmask                       # tangential velocity of the star state
    sig_n = K["sigma"][..., :, d]
    st_s = sig_n * tmask                    # tangential traction (unchanged across S_K)
    u2 = ut2 + us * (1 - tmask)             # normal component S*, tangential ut2
    dS = S_sh - Sst
    safe = torch.where(dS == 0, torch.ones_like(dS), dS)
    E2 = Qs["E"] - ((ut2 * st2).sum(-1) - (ut_s * st_s).sum(-1)) / safe
    w = (ut_s - ut2) / safe[..., None]      # tangential jump vector
    n = torch.zeros_like(us)
    n[..., d] = 1.0
    eye = torch.eye(3, dtype=us.dtype).expand(Vs.shape)
    V2 = (eye + w[..., :, None] * n[..., None, :]) @ Vs
    rho_s = Qs["ar1"] + Qs["ar2"]
    Q2 = dict(ar1=Qs["ar1"], ar2=Qs["ar2"], mom=rho_s[..., None] * u2, E=E2)
    if "arl" in Qs:
        Q2["arl"] = Qs["arl"]
    return Q2, u2, V2


def hllc(wL, wR, d, mats):
    """HLLD-type flux across faces normal to axis d (see the module text).

    Returns (F, phi_face, u_face, V_face): conservative fluxes (dict), and the
    face state at x/t = 0 used for the phi and V fluxes and the
    non-conservative terms.
    """
    L = face_state(wL, mats)
    R = face_state(wR, mats)
    unL, unR = L["u"][..., d], R["u"][..., d]
    SL = torch.minimum(unL - L["cL"], unR - R["cL"])
    SR = torch.maximum(unL + L["cL"], unR + R["cL"])
    mL = L["rho"] * (SL - unL)
    mR = R["rho"] * (SR - unR)
    snnL = L["sigma"][..., d, d]
    snnR = R["sigma"][..., d, d]
    Sst = (snnL - snnR + mL * unL - mR * unR) / (mL - mR)

    FL, FR = physical_flux(L, d), physical_flux(R, d)
    QsL, usL, VsL = star_state(L, SL, Sst, d)
    QsR, usR, VsR = star_state(R, SR, Sst, d)

    # shear waves in the star regions
    rsL = QsL["ar1"] + QsL["ar2"]
    rsR = QsR["ar1"] + QsR["ar2"]
    # shear wave speeds sqrt(G_mix / rho*); a face between fluids has
    # G_mix = 0, where they vanish and the solver drops the shear waves.
    # There the value is kept but not differentiated (the derivative of sqrt
    # at 0 is unbounded and would turn the reverse mode's zero weights into
    # NaN); every forward value is the plain sqrt(G_mix / rho*).
    def shear_speed(G, r):
        zero = G == 0
        exact = torch.sqrt(G / r).detach()
        safe = torch.sqrt(torch.where(zero, torch.ones_like(r), G / r))
        return torch.where(zero, exact, safe)

    csL = shear_speed(L["Gm"], rsL)
    csR = shear_speed(R["Gm"], rsR)
    ZL, ZR = rsL * csL, rsR * csR
    SsL, SsR = Sst - csL, Sst + csR
    tmask = torch.ones(3, dtype=unL.dtype)
    tmask[d] = 0.0
    utL, utR = L["u"] * tmask, R["u"] * tmask
    stL, stR = L["sigma"][..., :, d] * tmask, R["sigma"][..., :, d] * tmask
    Zs = ZL + ZR
    shear = Zs > 0
    Zsafe = torch.where(shear, Zs, torch.ones_like(Zs))[..., None]
    ut2 = (ZL[..., None] * utL + ZR[..., None] * utR + stR - stL) / Zsafe
    st2 = stL + ZL[..., None] * (ut2 - utL)
    ut2L = torch.where(shear[..., None], ut2, utL)
    ut2R = torch.where(shear[..., None], ut2, utR)
    st2L = torch.where(shear[..., None], st2, stL)
    st2R = torch.where(shear[..., None], st2, stR)
    Q2L, u2L, V2L = shear_state(L, QsL, usL, VsL, SsL, Sst, ut2L, st2L, d)
    Q2R, u2R, V2R = shear_state(R, QsR, usR, VsR, SsR, Sst, ut2R, st2R, d)

    reg = [SL >= 0]
    reg.append(~reg[0] & (SsL >= 0))
    reg.append(~reg[0] & ~reg[1] & (Sst >= 0))
    reg.append(~reg[0] & ~reg[1] & ~reg[2] & (SsR >= 0))
    reg.append(~reg[0] & ~reg[1] & ~reg[2] & ~reg[3] & (SR >= 0))

    def pick(*vals):
        shape = vals[0].shape

        def ex(mk):
            return mk.reshape(mk.shape + (1,) * (len(shape) - mk.dim()))
        out = vals[5]
        for k in range(4, -1, -1):
            out = torch.where(ex(reg[k]), vals[k], out)
        return out

    def ex(a, like):
        return a.reshape(a.shape + (1,) * (like.dim() - a.dim()))

    F = {}
    for k in FL:
        FsL = FL[k] + ex(SL, FL[k]) * (QsL[k] - L[k])
        FsR = FR[k] + ex(SR, FR[k]) * (QsR[k] - R[k])
        F2L = FsL + ex(SsL, FL[k]) * (Q2L[k] - QsL[k])
        F2R = FsR + ex(SsR, FR[k]) * (Q2R[k] - QsR[k])
        F[k] = pick(FL[k], FsL, F2L, F2R, FsR, FR[k])
    phi_face = pick(L["phi1"], L["phi1"], L["phi1"], R["phi1"], R["phi1"], R["phi1"])
    u_face = pick(L["u"], usL, u2L, u2R, usR, R["u"])
    V_face = pick(L["V"], VsL, V2L, V2R, VsR, R["V"])
    return F, phi_face, u_face, V_face
