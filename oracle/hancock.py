"""Oracle single-stage MUSCL-Hancock form of the hyperbolic update.

TEST INFRASTRUCTURE ONLY (plain PyTorch CPU float64, one patch at a time).

The paper integrates the hyperbolic part with three-stage Runge-Kutta
(Section 3.1).  This module is the second-order alternative with a single
Riemann solve per face and step: the predictor-corrector MUSCL-Hancock scheme
(van Leer; Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
Sec. 14.4, conservative-variable form), applied with the reconstruction,
Riemann solver and non-conservative terms of Section 3.1:

  1. edge states: the left and right edge values of every cell along each
     axis d, the MUSCL values of the primitives and the MUSCL-BVD-THINC values
     of phi1 (Appendix A), i.e. the per-cell edge values the Runge-Kutta
     operator feeds to its Riemann problems; an edge state that is not
     hyperbolic (c_L^2 <= 0) is replaced by the cell-centre state;
  2. predictor: every edge state of a cell moves by -dt/2 D_c, where D_c is
     the operator of Section 3.1 evaluated on the cell alone - its own two
     edge states of each axis take the place of the two faces (their physical
     fluxes, their phi, normal velocity and stretch in the phi and V fluxes
     and in the non-conservative terms), with the cell-centre coefficients
     phi_i, V_i, u_i; the same increment for every edge state of the cell
     (unsplit in 2D); an evolved state that is not hyperbolic is replaced by
     the cell-centre state at t^n;
  3. corrector: at each face the Riemann problem between the evolved right
     edge state of the left cell and the evolved left edge state of the
     right cell, and q* = q^n - dt D with D assembled from those face outputs
     exactly as in the Runge-Kutta stages (scheme.operator_from_faces).

For linear advection (uniform velocity u > 0 and pressure) the update of phi1
reduces to the textbook MUSCL-Hancock formula
phi_i - nu [(phi_i + (1 - nu) s_i / 2) - (phi_{i-1} + (1 - nu) s_{i-1} / 2)],
nu = u dt / dx, s the minmod slope.
"""
from __future__ import annotations

import torch

from .closures import cons_to_prim, prim_to_cons
from .reconstruction import bvd_select, muscl_faces, thinc_beta, thinc_faces, youngs_abs_normal
from .riemann import face_state, hllc, physical_flux
from .scheme import NG, _assemble, _components, _hyperbolic, fill_ghosts, operator_from_faces


def _edge_components(comps, absn, thinc, limiter="minmod"):
    """Left and right edge values along the last axis of every primitive
    component (NaN where a cell lacks the neighbours its values need)."""
    L, R = {}, {}
    for k, t in comps.items():
        mL, mR = muscl_faces(t, limiter)
        if k == "phi1" and thinc:
            beta = thinc_beta(absn) if absn is not None else torch.full_like(t, thinc_beta(1.0))
            tL, tR, mixed = thinc_faces(t, beta)
            mL, mR = bvd_select(mL, mR, tL, tR, mixed)
        L[k], R[k] = mL, mR
    return L, R


def _fallback(w, wc, mats):
    """w where hyperbolic, else the cell-centre state wc."""
    ok = _hyperbolic(w, mats)
    out = {}
    for k, t in w.items():
        m = ok.reshape(ok.shape + (1,) * (t.dim() - ok.dim()))
        out[k] = torch.where(m, t, wc[k])
    return out


def _own_faces(w, d, mats):
    """Outputs of a cell's own edge state w on axis d as if it were a face
    state: physical fluxes (Section 3 vector form), phi1, u, V."""
    s = face_state(w, mats)
    return physical_flux(s, d), s["phi1"], s["u"], s["V"]


def hancock_operator(q, grid, mats, thinc, dt, limiter="minmod"):
    """D of the MUSCL-Hancock update (q* = q^n - dt D) for the interior cells."""
    return hancock_operator_padded(q, fill_ghosts(q, grid), grid, mats, thinc, dt, limiter)[0]


def hancock_operator_padded(q, qg, grid, mats, thinc, dt, limiter="minmod"):
    """D of the MUSCL-Hancock update for the interior cells of q, from qg: q
    with NG ghost layers on each side (filled by the caller); also returns
    the face outputs of the corrector along each axis (conservative fluxes,
    face phi, u, V)."""
    ny, nx = q["phi1"].shape
    dim = grid["dim"]
    wg = cons_to_prim(qg, mats)
    comps = _components(wg)
    dims = [0] if dim == 1 else [0, 1]
    hs = [grid["dx"], grid["dy"]]
    if dim == 2 and thinc:
        anx, any_ = youngs_abs_normal(comps["phi1"], grid["dx"], grid["dy"])

    # 1. edge states of every padded cell along each axis
    edges = []
    for d in dims:
        if d == 0:
            L, R = _edge_components(comps, anx if (dim == 2 and thinc) else None, thinc, limiter)
        else:
            L, R = _edge_components({k: t.transpose(0, 1) for k, t in comps.items()},
                                    any_.transpose(0, 1) if thinc else None, thinc, limiter)
            L = {k: t.transpose(0, 1) for k, t in L.items()}
            R = {k: t.transpose(0, 1) for k, t in R.items()}
        edges.append((_fallback(_assemble(L), wg, mats), _fallback(_assemble(R), wg, mats)))

    # 2. predictor: D_c of each cell from its own edge states
    Dc = {k: torch.zeros_like(v) for k, v in qg.items()}
    divu = torch.zeros_like(qg["phi1"])
    beta = torch.zeros_like(qg["mom"])
    for d in dims:
        Fm, phm, um, Vm = _own_faces(edges[d][0], d, mats)
        Fp, php, up, Vp = _own_faces(edges[d][1], d, mats)
        h = hs[d]
        for k in Fp:
            Dc[k] = Dc[k] + (Fp[k] - Fm[k]) / h
        Dc["phi1"] = Dc["phi1"] + (php * up[..., d] - phm * um[..., d]) / h
        divu = divu + (up[..., d] - um[..., d]) / h

        def FV(V, u):
            return V * u[..., d][..., None, None] - V[..., d, :][..., None, :] * u[..., :, None]

        Dc["V"] = Dc["V"] + (FV(Vp, up) - FV(Vm, um)) / h
        beta = beta + (Vp[..., d, :] - Vm[..., d, :]) / h
    uc = qg["mom"] / (qg["ar1"] + qg["ar2"])[..., None]
    Dc["phi1"] = Dc["phi1"] - qg["phi1"] * divu
    Dc["V"] = Dc["V"] - ((2.0 / 3.0) * qg["V"] * divu[..., None, None]
                         - uc[..., :, None] * beta[..., None, :])

    def evolve(w):
        Q = prim_to_cons(w, mats)
        Qt = {k: Q[k] - 0.5 * dt * Dc[k] for k in Q}
        return _fallback(cons_to_prim(Qt, mats), wg, mats)

    evolved = [(evolve(m), evolve(p)) for m, p in edges]

    # 3. corrector: Riemann problems between evolved edge states
    faces = []
    for d in dims:
        wm, wp = evolved[d]
        if d == 0:
            rows = slice(NG, NG + ny) if dim == 2 else slice(0, 1)
            left = {k: t[rows, NG - 1:NG + nx] for k, t in wp.items()}
            right = {k: t[rows, NG:NG + nx + 1] for k, t in wm.items()}
        else:
            cols = slice(NG, NG + nx)
            left = {k: t[NG - 1:NG + ny, cols] for k, t in wp.items()}
            right = {k: t[NG:NG + ny + 1, cols] for k, t in wm.items()}
        faces.append(hllc(left, right, d, mats))
    return operator_from_faces(q, faces, grid), faces
