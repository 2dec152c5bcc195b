"""Oracle Riemann solver: HLLC-type flux for the elastic diffuse-interface system.

TEST INFRASTRUCTURE ONLY (plain PyTorch CPU float64).

The paper (Section 3.1) uses the HLLD solver of Barton (2019), whose formulas
it does not print.  The reading taken here is an HLLC-type solver with one
contact wave, written from the Rankine-Hugoniot conditions of the conservative
part of the system (vector form of Section 3):

  * wave speeds: Davis bounds with the longitudinal sound speed c_L;
  * contact speed S* from continuity of the normal traction sigma_nn
    (HLLC with p replaced by -sigma_nn);
  * star state of side K: density ratio r = (S_K - u_nK)/(S_K - S*); partial
    densities scaled by r, phi unchanged, u* = u_K with its normal component
    replaced by S*, sigma*_n from the normal-momentum jump, energy from the
    energy jump, and the stretch tensor from the kinematic jump of a planar
    wave, V* = det(F_w)^(-1/3) F_w V_K with F_w = I + (u_K - u*) n^T/(S_K - u_nK);
  * conservative fields take F_K + S_K (Q*_K - Q_K); phi and V take the flux of
    the state found at x/t = 0, which also supplies the face velocity and
    stretch used by the non-conservative terms.

Tie rule at x/t = 0: S_L >= 0 -> left state; else S* >= 0 -> left star;
else S_R >= 0 -> right star; else right state.
"""
from __future__ import annotations

import torch

from .closures import hencky_dev, mixture_props, phases, stress, material_energy

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
    s = dict(phi1=w["phi1"], rho=rho, u=w["u"], V=w["V"],
             ar1=phis[0] * rhos[0], ar2=phis[1] * rhos[1],
             mom=rho[..., None] * w["u"],
             E=rhoe + 0.5 * rho * (w["u"] * w["u"]).sum(-1),
             sigma=stress(w["p"], Gm, devH), cL=torch.sqrt(cL2))
    if lam is not None:
        y = next(i for i, m in enumerate(mats) if m["reactive"])
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
    Estar = (s["E"] * (S - un) - (s["u"] * sig_n).sum(-1)
             + (ustar * sig_n_star).sum(-1)) / (S - Sst)
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


def hllc(wL, wR, d, mats):
    """HLLC-type flux across faces normal to axis d.

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

    reg_L = SL >= 0
    reg_sL = (~reg_L) & (Sst >= 0)
    reg_sR = (~reg_L) & (~reg_sL) & (SR >= 0)

    def pick(a, b, c, e):
        shape = a.shape
        def ex(mk):
            return mk.reshape(mk.shape + (1,) * (len(shape) - mk.dim()))
        return torch.where(ex(reg_L), a, torch.where(ex(reg_sL), b, torch.where(ex(reg_sR), c, e)))

    F = {}
    for k in FL:
        FsL = FL[k] + (SL.reshape(SL.shape + (1,) * (FL[k].dim() - SL.dim())) * (QsL[k] - L[k]))
        FsR = FR[k] + (SR.reshape(SR.shape + (1,) * (FR[k].dim() - SR.dim())) * (QsR[k] - R[k]))
        F[k] = pick(FL[k], FsL, FsR, FR[k])
    phi_face = pick(L["phi1"], L["phi1"], R["phi1"], R["phi1"])
    u_face = pick(L["u"], usL, usR, R["u"])
    V_face = pick(L["V"], VsL, VsR, R["V"])
    return F, phi_face, u_face, V_face
