"""Oracle time step: ghost cells, spatial operator D, SSP-RK3, CFL, sources.

TEST INFRASTRUCTURE ONLY (plain PyTorch CPU float64, one patch at a time).

Cites arXiv 2009.14555:
  * Section 3 (vector form of the system): conservative fluxes, the
    non-conservative terms phi div(u) and (2/3) V div(u) - u_i beta_j;
  * Section 3 (fractional steps): time step a fraction of the largest stable
    step; hyperbolic update first, then plastic, then reactive source;
  * Section 3.1, Eq. for D: flux differences of dimensional sweeps summed,
    minus the non-conservative sources; the three-stage Runge-Kutta scheme;
  * Section 3.2: plastic update (J*, mixture J*, scaled dev(H), first Pade
    approximant, bisection of the objective on [0, J*]);
  * Section 3.3: reactive update with classical RK4;
  * Section 3 (cylindrical symmetry): the geometric source s_g, with x = r and
    y = z (geometric_source_terms), added to the operator of the stages.

Readings: the non-conservative terms use the face velocity and face stretch of
the Riemann solution, with cell-centred coefficients phi_i, V_i, u_i;
the CFL rate of a cell is sum_d (|u_d| + c_L)/dx_d with
c_L^2 = c^2 + 4/3 G/rho; a fluid (G = 0) relaxes fully in the plastic step
(J*_l = 0) so V returns to I; perfect plasticity is the chi0 -> infinity limit
of the ideal-plasticity rate; the reaction rate of the reactive material is
Arrhenius, lam_dot = -A lam exp(-T_act / T), zero where T <= 0, or (rate_law
1) the k sqrt(lam) law of Section 4.1 for the reactant fraction,
lam_dot = -k sqrt(lam) with k = A, switched on where the pressure of the
state the rate is evaluated at exceeds p_ign; sqrt of max(lam, 0), and the
RK4 result is clamped at lam >= 0.
"""
from __future__ import annotations

import math

import torch

from .closures import (PLASTIC_JC, Gamma, cons_to_prim, hencky_dev, history_material, inv_gamma,
                       jc_temperature, jc_yield, mixture_props, phases, prim_to_cons, shear_modulus,
                       stress, temperature, two_eos)
from .reconstruction import (bvd_select, muscl_faces, thinc_beta, thinc_faces,
                             youngs_abs_normal)
from .riemann import hllc

F64 = torch.float64
NG = 3  # ghost layers: the BVD choice at a face reaches three cells out

BC_TRANSMISSIVE, BC_PERIODIC, BC_REFLECTIVE = 0, 1, 2

# primitive scalar components handled by the reconstruction
_UCOMP = {"ux": 0, "uy": 1}
_VCOMP = {"V11": (0, 0), "V12": (0, 1), "V21": (1, 0), "V22": (1, 1), "V33": (2, 2)}


# ----------------------------------------------------------------------------
# Layout conversion between the library's flat arrays and the oracle's dicts.
# ----------------------------------------------------------------------------
def _names(dim, reactive, kind):
    if kind == "prim":
        base = (["phi1", "rho1", "rho2", "u", "p", "V11", "V22", "V33"] if dim == 1 else
                ["phi1", "rho1", "rho2", "u", "v", "p", "V11", "V12", "V21", "V22", "V33"])
        return base + (["lam"] if reactive else [])
    base = (["phi1", "ar1", "ar2", "mx", "E", "V11", "V22", "V33"] if dim == 1 else
            ["phi1", "ar1", "ar2", "mx", "my", "E", "V11", "V12", "V21", "V22", "V33"])
    return base + (["arl"] if reactive else [])


def _vec_mat(f, get):
    z = torch.zeros_like(get("phi1"))
    o = lambda n: f[n] if n in f else z  # noqa: E731
    V = torch.stack([torch.stack([o("V11"), o("V12"), z], -1),
                     torch.stack([o("V21"), o("V22"), z], -1),
                     torch.stack([z, z, o("V33")], -1)], -2)
    return V


def prim_from_array(a, dim, reactive):
    a = torch.as_tensor(a, dtype=F64)
    f = {n: a[k] for k, n in enumerate(_names(dim, reactive, "prim"))}
    z = torch.zeros_like(f["phi1"])
    w = dict(phi1=f["phi1"], rho1=f["rho1"], rho2=f["rho2"],
             u=torch.stack([f["u"], f.get("v", z), z], -1), p=f["p"],
             V=_vec_mat(f, lambda n: f[n]))
    if reactive:
        w["lam"] = f["lam"]
    return w


def cons_from_array(a, dim, reactive):
    a = torch.as_tensor(a, dtype=F64)
    f = {n: a[k] for k, n in enumerate(_names(dim, reactive, "cons"))}
    z = torch.zeros_like(f["phi1"])
    q = dict(phi1=f["phi1"], ar1=f["ar1"], ar2=f["ar2"],
             mom=torch.stack([f["mx"], f.get("my", z), z], -1), E=f["E"],
             V=_vec_mat(f, lambda n: f[n]))
    if reactive:
        q["arl"] = f["arl"]
    return q


def cons_to_array(q, dim, reactive):
    get = dict(phi1=q["phi1"], ar1=q["ar1"], ar2=q["ar2"], mx=q["mom"][..., 0],
               my=q["mom"][..., 1], E=q["E"], V11=q["V"][..., 0, 0], V12=q["V"][..., 0, 1],
               V21=q["V"][..., 1, 0], V22=q["V"][..., 1, 1], V33=q["V"][..., 2, 2])
    if reactive:
        get["arl"] = q["arl"]
    return torch.stack([get[n] for n in _names(dim, reactive, "cons")], 0)


def prim_to_array(w, dim, reactive):
    get = dict(phi1=w["phi1"], rho1=w["rho1"], rho2=w["rho2"], u=w["u"][..., 0],
               v=w["u"][..., 1], p=w["p"], V11=w["V"][..., 0, 0], V12=w["V"][..., 0, 1],
               V21=w["V"][..., 1, 0], V22=w["V"][..., 1, 1], V33=w["V"][..., 2, 2])
    if reactive:
        get["lam"] = w["lam"]
    return torch.stack([get[n] for n in _names(dim, reactive, "prim")], 0)


# ----------------------------------------------------------------------------
# Ghost cells
# ----------------------------------------------------------------------------
def _spatial(t):
    """Number of trailing non-spatial dims of a state entry."""
    return {2: 0, 3: 1, 4: 2}[t.dim()]


def _pad_axis(t, axis, lo_bc, hi_bc, key):
    """Pad spatial axis `axis` (0 = y, 1 = x) of tensor t with NG ghost layers."""
    n = t.shape[axis]

    def take(idx):
        return torch.index_select(t, axis, torch.as_tensor(idx, dtype=torch.long))

    def side(bc, lo):
        if bc == BC_PERIODIC:
            idx = list(range(n - NG, n)) if lo else list(range(NG))
        elif bc == BC_REFLECTIVE:
            idx = list(range(NG - 1, -1, -1)) if lo else list(range(n - 1, n - NG - 1, -1))
        else:
            idx = [0] * NG if lo else [n - 1] * NG
        g = take(idx)
        if bc == BC_REFLECTIVE:
            comp = 1 - axis  # x-wall for spatial axis 1 -> component 0
            if key == "mom":
                g = g.clone()
                g[..., comp] = -g[..., comp]
            elif key == "V":
                P = torch.ones(3, dtype=F64)
                P[comp] = -1.0
                g = g * P[:, None] * P[None, :]
        return g

    return torch.cat([side(lo_bc, True), t, side(hi_bc, False)], axis)


def fill_ghosts(q, grid):
    bc = grid["bc"]
    out = {}
    for k, t in q.items():
        g = _pad_axis(t, 1, bc[0], bc[1], k)
        if grid["dim"] == 2:
            g = _pad_axis(g, 0, bc[2], bc[3], k)
        out[k] = g
    return out


# ----------------------------------------------------------------------------
# Spatial operator D (Section 3.1)
# ----------------------------------------------------------------------------
def _components(w):
    c = dict(phi1=w["phi1"], rho1=w["rho1"], rho2=w["rho2"], ux=w["u"][..., 0],
             uy=w["u"][..., 1], p=w["p"])
    for n, (i, j) in _VCOMP.items():
        c[n] = w["V"][..., i, j]
    if "lam" in w:
        c["lam"] = w["lam"]
    return c


def _assemble(c):
    z = torch.zeros_like(c["phi1"])
    w = dict(phi1=c["phi1"], rho1=c["rho1"], rho2=c["rho2"],
             u=torch.stack([c["ux"], c["uy"], z], -1), p=c["p"],
             V=torch.stack([torch.stack([c["V11"], c["V12"], z], -1),
                            torch.stack([c["V21"], c["V22"], z], -1),
                            torch.stack([z, z, c["V33"]], -1)], -2))
    if "lam" in c:
        w["lam"] = c["lam"]
    return w


def _hyperbolic(w, mats):
    """Mask of states with a positive longitudinal sound speed squared."""
    _, J2 = hencky_dev(w["V"])
    _, _, _, cL2 = mixture_props(phases(w["phi1"]), [w["rho1"], w["rho2"]], w["p"], J2, mats,
                                 w.get("lam"))
    return cL2 > 0


def _sweep(wg, absn, d, n, mats, thinc, limiter="minmod"):
    """Face fluxes along axis d for lines of cells (cells along the last axis).

    wg: primitive components on lines including NG ghosts on each end;
    absn: |n_d| on the same lines (None in 1D).  Returns the HLLC outputs on the
    n + 1 faces of the interior cells.

    Reading: a reconstructed face state that is not hyperbolic (c_L^2 <= 0,
    which THINC sharpening of phi next to a stiff material can produce when
    the gas pressure is negative) is replaced by its cell-centre state
    (first-order fallback on that side of that face).
    """
    L, R, CL, CR = {}, {}, {}, {}
    for k, t in wg.items():
        mL, mR = muscl_faces(t, limiter)
        if k == "phi1" and thinc:
            beta = thinc_beta(absn) if absn is not None else torch.full_like(t, thinc_beta(1.0))
            tL, tR, mixed = thinc_faces(t, beta)
            mL, mR = bvd_select(mL, mR, tL, tR, mixed)
        # face f between cell NG-1+f and NG+f, f = 0..n
        L[k] = mR[..., NG - 1:NG + n]
        R[k] = mL[..., NG:NG + n + 1]
        CL[k] = t[..., NG - 1:NG + n]
        CR[k] = t[..., NG:NG + n + 1]
    wL, wR = _assemble(L), _assemble(R)
    okL, okR = _hyperbolic(wL, mats), _hyperbolic(wR, mats)
    for k in L:
        L[k] = torch.where(okL, L[k], CL[k])
        R[k] = torch.where(okR, R[k], CR[k])
    return hllc(_assemble(L), _assemble(R), d, mats)


def operator_from_faces(q, faces, grid):
    """D of Section 3.1 from the face outputs of each axis.

    faces[d] = (F, phi_f, u_f, V_f) on the faces normal to axis d ((ny, nx+1)
    for d = 0, (ny+1, nx) for d = 1): flux differences, the phi and V fluxes
    of the face state, minus the non-conservative terms with cell-centre
    coefficients phi_i, V_i, u_i of q."""
    hs = [grid["dx"], grid["dy"]]
    D = {k: torch.zeros_like(v) for k, v in q.items()}
    divu = torch.zeros_like(q["phi1"])
    beta = torch.zeros_like(q["mom"])
    Vc = q["V"]
    uc = q["mom"] / (q["ar1"] + q["ar2"])[..., None]
    for d, (F, phi_f, u_f, V_f) in enumerate(faces):

        def diff(t):
            return (t[:, 1:] - t[:, :-1]) if d == 0 else (t[1:, :] - t[:-1, :])

        h = hs[d]
        for k in F:
            D[k] = D[k] + diff(F[k]) / h
        D["phi1"] = D["phi1"] + diff(phi_f * u_f[..., d]) / h
        divu = divu + diff(u_f[..., d]) / h
        # V flux: V_ij u_d - V_dj u_i at the face state
        FV = V_f * u_f[..., d][..., None, None] - V_f[..., d, :][..., None, :] * u_f[..., :, None]
        D["V"] = D["V"] + diff(FV) / h
        beta = beta + diff(V_f[..., d, :]) / h
    D["phi1"] = D["phi1"] - q["phi1"] * divu
    D["V"] = D["V"] - ((2.0 / 3.0) * Vc * divu[..., None, None]
                       - uc[..., :, None] * beta[..., None, :])
    return D


def geometric_source_terms(q, mats):
    """The bracket of the cylindrical geometric source (Section 3, cylindrical
    symmetry): s_g = -(1/r) (0, phi_l rho_l u_r, phi_y rho_y lam u_r,
    rho u_r^2 - sigma_rr + sigma_thth, rho u_z u_r - sigma_rz,
    rho E u_r - (u_r sigma_rr + u_z sigma_zr), V_ij u_r / 3 - delta_{i th} V_ij u_r).
    Axis order: 0 = r (x), 1 = z (y), 2 = theta."""
    w = cons_to_prim(q, mats)
    devH, J2 = hencky_dev(w["V"])
    phis = phases(w["phi1"])
    _, Gm, _, _ = mixture_props(phis, [w["rho1"], w["rho2"]], w["p"], J2, mats, w.get("lam"))
    sig = stress(w["p"], Gm, devH)
    rho = q["ar1"] + q["ar2"]
    ur, uz = w["u"][..., 0], w["u"][..., 1]
    t = {"phi1": torch.zeros_like(q["phi1"]), "ar1": q["ar1"] * ur, "ar2": q["ar2"] * ur}
    if "arl" in q:
        t["arl"] = q["arl"] * ur
    mom = torch.zeros_like(q["mom"])
    mom[..., 0] = rho * ur * ur - sig[..., 0, 0] + sig[..., 2, 2]
    mom[..., 1] = rho * uz * ur - sig[..., 1, 0]
    t["mom"] = mom
    t["E"] = q["E"] * ur - (ur * sig[..., 0, 0] + uz * sig[..., 1, 0])
    factor = torch.tensor([1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0 - 1.0], dtype=F64)
    t["V"] = factor[:, None] * q["V"] * ur[..., None, None]
    return t


def cell_radius(grid, nx):
    """Cell-centre radius r = x0 + (i + 1/2) dx of the interior columns."""
    return grid.get("x0", 0.0) + (torch.arange(nx, dtype=F64) + 0.5) * grid["dx"]


def spatial_operator(q, grid, mats, thinc, limiter="minmod"):
    """D(q) of Section 3.1 for all interior cells of one patch; in cylindrical
    geometry (grid["geometry"] == "cyl", x = r, y = z) minus the geometric
    source s_g."""
    return with_geometric_source(_planar_operator(q, grid, mats, thinc, limiter), q, grid, mats)


def with_geometric_source(D, q, grid, mats):
    """D of the cells of q minus the geometric source s_g = -(1/r) t of
    cylindrical geometry (Section 3, cylindrical symmetry), t the bracket of
    geometric_source_terms, r the cell-centre radius of grid; D itself for a
    planar grid."""
    if grid.get("geometry", "planar") != "cyl":
        return D
    r = cell_radius(grid, q["phi1"].shape[1])[None, :]
    t = geometric_source_terms(q, mats)
    for k in D:
        rr = r.reshape(r.shape + (1,) * (D[k].dim() - 2))
        D[k] = D[k] + t[k] / rr
    return D


def _planar_operator(q, grid, mats, thinc, limiter="minmod"):
    return operator_padded(q, fill_ghosts(q, grid), grid, mats, thinc, limiter)[0]


def operator_padded(q, qg, grid, mats, thinc, limiter="minmod"):
    """D of Section 3.1 (planar) for the interior cells of q, from qg: q with
    NG ghost layers on each side (filled by the caller).  Also returns the
    face outputs of each axis (conservative fluxes, face phi, u, V)."""
    ny, nx = q["phi1"].shape
    wg = cons_to_prim(qg, mats)
    comps = _components(wg)
    dims = [0] if grid["dim"] == 1 else [0, 1]
    if grid["dim"] == 2 and thinc:
        anx, any_ = youngs_abs_normal(comps["phi1"], grid["dx"], grid["dy"])
    faces = []
    for d in dims:
        if d == 0:
            rows = slice(NG, NG + ny) if grid["dim"] == 2 else slice(0, 1)
            lines = {k: t[rows, :] for k, t in comps.items()}
            absn = anx[rows, :] if (grid["dim"] == 2 and thinc) else None
            n = nx
        else:
            lines = {k: t[:, NG:NG + nx].transpose(0, 1) for k, t in comps.items()}
            absn = any_[:, NG:NG + nx].transpose(0, 1) if thinc else None
            n = ny
        F, phi_f, u_f, V_f = _sweep(lines, absn, d, n, mats, thinc, limiter)
        if d == 1:  # back to (ny+1, nx) face layout
            F = {k: v.transpose(0, 1) for k, v in F.items()}
            phi_f, u_f, V_f = phi_f.transpose(0, 1), u_f.transpose(0, 1), V_f.transpose(0, 1)
        faces.append((F, phi_f, u_f, V_f))
    return operator_from_faces(q, faces, grid), faces


# ----------------------------------------------------------------------------
# Time step, RK3, sources
# ----------------------------------------------------------------------------
def cfl_rate(q, grid, mats):
    """Per-cell sum_d (|u_d| + c_L)/dx_d (Section 3: fraction of the stable step)."""
    w = cons_to_prim(q, mats)
    phis = phases(w["phi1"])
    _, J2 = hencky_dev(w["V"])
    _, _, _, cL2 = mixture_props(phis, [w["rho1"], w["rho2"]], w["p"], J2, mats, w.get("lam"))
    cL = torch.sqrt(cL2)
    rate = (w["u"][..., 0].abs() + cL) / grid["dx"]
    if grid["dim"] == 2:
        rate = rate + (w["u"][..., 1].abs() + cL) / grid["dy"]
    return rate


def cfl_dt(q, grid, mats, cfl):
    return cfl / cfl_rate(q, grid, mats).max().item()


def _axpy(a, x, b, y):
    return {k: a * x[k] + b * y[k] for k in x}


def _sqrt0(x):
    """Square root whose derivative at 0 is taken as 0 (a strain norm at zero
    strain is not differentiable; its subgradient 0 is used)."""
    pos = x > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, x, torch.ones_like(x))), torch.zeros_like(x))


def plastic_update(q, mats, dt, iters=64):
    """Section 3.2: J*, per-material relaxed J*, mixture J*, Pade exp.

    Perfect plasticity returns radially onto the yield surface,
    J*_l = min(J*, J_Y) with J_Y = sigma_Y / (sqrt(6) G) (the chi0 -> infinity
    limit of the relaxation objective); a finite rate chi0 solves the objective
    R(J) = J - J* + dt chi(J) by bisection on [0, J*].

    Johnson-Cook (Section 2.3.2): chi = chi0 exp((sqrt(3/2) |dev sigma| /
    sigma_Y(eps_p) - 1) / c3) with |dev sigma| = 2 G J, the objective's plastic
    strain eps_p*(J) = eps_p + (J* - J) (the strain rate chi integrated over
    the step, dt chi = J* - J at the root), and the temperature of the state
    entering the step (frozen during it).  The history row rho_l phi_l eps_p
    then grows by rho_l phi_l (J* - J*_l), the source of its evolution
    equation over the step."""
    phis = phases(q["phi1"])
    devH, J2 = hencky_dev(q["V"])
    Jst = _sqrt0(J2)
    num = torch.zeros_like(Jst)
    den = torch.zeros_like(Jst)
    arl_new = None
    # phi_l / Gamma_l weights (a two-closure reactive mixture: 1 / Gamma_y at
    # the state's own reactant share)
    if any(two_eos(m) for m in mats):
        wq = cons_to_prim(q, mats)
        y = next(i for i, m in enumerate(mats) if m["reactive"])
        lam_q = q["arl"] / q["ar1" if y == 0 else "ar2"]
        igs = [inv_gamma(m, wq["p"], lam_q) for m in mats]
    else:
        igs = [1.0 / Gamma(m) for m in mats]
    for m, ph, ar, ig in zip(mats, phis, (q["ar1"], q["ar2"]), igs):
        # G(rho_l) of the material's own density (constant but for Romenskii)
        Gl = shear_modulus(m, ar / ph)
        if m["G"] == 0.0:
            Jl = torch.zeros_like(Jst)  # fluid: no shear strain survives
        elif m["plastic"] == 1:
            JY = m["sigma_y"] / (math.sqrt(6.0) * Gl)
            Jl = torch.minimum(Jst, JY)
        elif m["plastic"] == 0:
            Jl = Jst
        elif m["plastic"] == PLASTIC_JC:
            w0 = cons_to_prim(q, mats)
            T = jc_temperature(m, ar / ph, w0["p"], J2)
            eps0 = q["arl"] / ar

            def chi_jc(J):
                sY = jc_yield(m, eps0 + (Jst - J), T)
                ratio = math.sqrt(1.5) * 2.0 * Gl * J / torch.where(sY > 0, sY, torch.ones_like(sY))
                rate = m["chi0"] * torch.exp((ratio - 1.0) / m["jc_c3"])
                # no strength left (at or above the melting temperature): the rate is unbounded
                return torch.where(sY > 0, rate, torch.full_like(J, math.inf))

            lo = torch.zeros_like(Jst)
            hi = Jst.clone()
            for _ in range(iters):  # bisection of R(J) = J - J* + dt chi(J, eps_p*(J)) on [0, J*]
                mid = 0.5 * (lo + hi)
                Rm = mid - Jst + dt * chi_jc(mid)
                neg = Rm < 0
                lo = torch.where(neg, mid, lo)
                hi = torch.where(neg, hi, mid)
            Jl = 0.5 * (lo + hi)
            arl_new = q["arl"] + ar * (Jst - Jl)
        else:
            def chi(J):
                # rate-dependent plasticity: chi0 H[sqrt(3/2) |dev sigma| - sigma_Y], |dev sigma| = 2 G J
                on = math.sqrt(1.5) * 2.0 * Gl * J - m["sigma_y"] > 0
                return torch.where(on, torch.full_like(J, m["chi0"]), torch.zeros_like(J))

            lo = torch.zeros_like(Jst)
            hi = Jst.clone()
            for _ in range(iters):  # bisection of R(J) = J - J* + dt chi(J) on [0, J*]
                mid = 0.5 * (lo + hi)
                Rm = mid - Jst + dt * chi(mid)
                neg = Rm < 0
                lo = torch.where(neg, mid, lo)
                hi = torch.where(neg, hi, mid)
            Jl = 0.5 * (lo + hi)
        num = num + ph * ig * Jl
        den = den + ph * ig
    Jnew = num / den
    scale = torch.where(Jst > 0, Jnew / torch.where(Jst > 0, Jst, torch.ones_like(Jst)),
                        torch.zeros_like(Jst))
    Hn = scale[..., None, None] * devH
    eye = torch.eye(3, dtype=F64).expand(Hn.shape)
    Vn = torch.linalg.inv(eye - 0.5 * Hn) @ (eye + 0.5 * Hn)
    out = dict(q)
    out["V"] = Vn
    if arl_new is not None:
        out["arl"] = arl_new
    return out


def reaction_update(q, mats, dt):
    """Section 3.3: RK4 on d(phi rho lam)/dt = phi rho lam_dot, other fields frozen."""
    y = next(i for i, m in enumerate(mats) if m["reactive"])
    m = mats[y]
    ary = q["ar1" if y == 0 else "ar2"]

    law = int(m.get("rate_law", 0))

    def f(arl):
        w = cons_to_prim(dict(q, arl=arl), mats)
        lam = arl / ary
        if law == 1:
            # Section 4.1: lam_dot = -k sqrt(lam) while p > p_ign
            on = (w["p"] > m["p_ign"]) & (lam > 0)
            # (1 in the switched-off cells keeps the reverse mode free of 0 / 0)
            lam_dot = -m["A"] * torch.sqrt(torch.where(on, lam, torch.ones_like(lam)))
            return ary * torch.where(on, lam_dot, torch.zeros_like(lam))
        rho_y = w["rho1" if y == 0 else "rho2"]
        _, J2 = hencky_dev(w["V"])
        T = temperature(m, rho_y, w["p"], J2, lam)
        arr = torch.where(T > 0, torch.exp(-m["T_act"] / torch.where(T > 0, T, torch.ones_like(T))),
                          torch.zeros_like(T))
        return ary * (-m["A"] * lam * arr)

    a0 = q["arl"]
    k1 = f(a0)
    k2 = f(a0 + 0.5 * dt * k1)
    k3 = f(a0 + 0.5 * dt * k2)
    k4 = f(a0 + dt * k3)
    out = dict(q)
    a1 = a0 + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    if law == 1:
        a1 = torch.where(a1 > 0, a1, torch.zeros_like(a1))
    out["arl"] = a1
    return out


def step(q, grid, mats, opts, dt=None):
    """One full time step: CFL dt from q^n, SSP-RK3 hyperbolic update (or,
    with opts["scheme"] == "hancock", the single-stage MUSCL-Hancock update of
    oracle.hancock), then the plastic and reactive source steps (Section 3,
    fractional steps)."""
    if dt is None:
        dt = cfl_dt(q, grid, mats, opts["cfl"])
    th = opts.get("thinc", False)

    def D(x):
        return spatial_operator(x, grid, mats, th, opts.get("limiter", "minmod"))

    if opts.get("scheme", "rk3") == "hancock":
        if grid.get("geometry", "planar") != "planar":
            raise NotImplementedError("the MUSCL-Hancock form is planar only")
        from .hancock import hancock_operator
        qs = _axpy(1.0, q, -dt, hancock_operator(q, grid, mats, th, dt, opts.get("limiter", "minmod")))
    else:
        q1 = _axpy(1.0, q, -dt, D(q))
        q2 = _axpy(1.0, q1, -dt, D(q1))
        q3 = _axpy(0.75, q, 0.25, q2)
        q4 = _axpy(1.0, q3, -dt, D(q3))
        qs = _axpy(1.0 / 3.0, q, 2.0 / 3.0, q4)
    qs = plastic_update(qs, mats, dt)
    if any(m["reactive"] for m in mats):
        qs = reaction_update(qs, mats, dt)
    return qs, dt


def grid_of(patch, dim, geometry="planar"):
    return dict(dim=dim, dx=patch.dx, dy=patch.dy, bc=tuple(patch.bc), x0=getattr(patch, "x0", 0.0),
                geometry=geometry)


def run(prim_array, dim, mats, grid, opts, steps, dt_list=None):
    """Initialise from primitives and take `steps` steps.  Returns (cons array, dts)."""
    reactive = history_material(mats) is not None
    q = prim_to_cons(prim_from_array(prim_array, dim, reactive), mats)
    dts = []
    for s in range(steps):
        q, dt = step(q, grid, mats, opts, None if dt_list is None else dt_list[s])
        dts.append(dt)
    return cons_to_array(q, dim, reactive), dts
