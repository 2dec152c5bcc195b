"""Seeded synthetic workloads shaped like the paper's problems.

This module only lays out geometry, material parameter sets and seeded random
draws.  It holds none of the scheme's arithmetic: no equation of state, no
conversion from primitive to conservative variables, no flux.  Both the oracle
(`oracle/`) and the CUDA path read the *primitive* fields it produces and each
converts them with its own closure code.

Primitive field layout (per cell), matching the state vector of Section 3
(vector form of the system) with two materials, material 1 being the one whose
volume fraction is stored:

    1D : phi1, rho1, rho2, u, p, V11, V22, V33, [lam]
    2D : phi1, rho1, rho2, u, v, p, V11, V12, V21, V22, V33, [lam]

`lam` is the history variable of Section 2.1 carried by one material: the
reaction progress variable of the reactive material (1 = reactant, 0 =
products, Section 2.3.1), or the equivalent plastic strain eps_p of a
Johnson-Cook solid (Section 2.3.2); it is present only when a material carries
one.  Arrays are float64 with shape (nfields, ny, nx) (ny = 1 in 1D).

Materials are plain dicts with the keys
    gamma, p_inf, e_inf, G, plastic (0 none, 1 perfect, 2 rate, 3 Johnson-Cook),
    sigma_y, chi0, reactive (0/1), Q, cv, A, T_act, rate_law, p_ign
(stiffened-gas Mie-Grueneisen closures, Section 2.3; perfect plasticity is the
chi0 -> infinity limit of the ideal-plasticity rate, Section 2.3.2; the rate
parameters only apply to a reactive material: rate_law 0 is the Arrhenius law
with A, T_act, rate_law 1 the k sqrt(lam) law of Section 4.1 with k = A,
switched on above the pressure p_ign), plus the Romenskii, JWL, product-closure
and Johnson-Cook (jc_*) keys of the helpers below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EPS_PHI = 1e-8  # volume fraction given to the absent material in a pure cell

BC_TRANSMISSIVE, BC_PERIODIC, BC_REFLECTIVE = 0, 1, 2

PRIM_1D = ["phi1", "rho1", "rho2", "u", "p", "V11", "V22", "V33"]
PRIM_2D = ["phi1", "rho1", "rho2", "u", "v", "p", "V11", "V12", "V21", "V22", "V33"]
CONS_1D = ["phi1", "ar1", "ar2", "mx", "E", "V11", "V22", "V33"]
CONS_2D = ["phi1", "ar1", "ar2", "mx", "my", "E", "V11", "V12", "V21", "V22", "V33"]


def prim_names(dim: int, reactive: bool) -> list[str]:
    base = PRIM_1D if dim == 1 else PRIM_2D
    return base + (["lam"] if reactive else [])


def cons_names(dim: int, reactive: bool) -> list[str]:
    base = CONS_1D if dim == 1 else CONS_2D
    return base + (["arl"] if reactive else [])


def material(gamma, p_inf=0.0, e_inf=0.0, G=0.0, plastic=0, sigma_y=0.0, chi0=0.0,
             reactive=0, Q=0.0, cv=0.0, A=0.0, T_act=0.0, rate_law=0, p_ign=0.0) -> dict:
    return dict(gamma=float(gamma), p_inf=float(p_inf), e_inf=float(e_inf), G=float(G),
                plastic=int(plastic), sigma_y=float(sigma_y), chi0=float(chi0),
                reactive=int(reactive), Q=float(Q), cv=float(cv), A=float(A),
                T_act=float(T_act), rate_law=int(rate_law), p_ign=float(p_ign))


def romenskii(rho0, K0, G0, Gamma, alpha, beta, plastic=0, sigma_y=0.0) -> dict:
    """Romenskii elastic solid of Section 2.3 (gamma = Gamma + 1)."""
    m = material(Gamma + 1.0, G=G0, plastic=plastic, sigma_y=sigma_y)
    m.update(eos="romenskii", rho0=float(rho0), K0=float(K0), alpha_r=float(alpha), beta_r=float(beta))
    return m


def jwl(rho0, A, B, R1, R2, Gamma, cv=0.0) -> dict:
    """JWL fluid of Section 2.3 (gamma = Gamma + 1; no shear modulus)."""
    m = material(Gamma + 1.0, cv=cv)
    m.update(eos="jwl", rho0=float(rho0), jwl_A=float(A), jwl_B=float(B), jwl_R1=float(R1),
             jwl_R2=float(R2))
    return m


def generic_explosive(A=2.0e6, rate_law=1, p_ign=1.0e8, T_act=0.0) -> dict:
    """The generic multiphase explosive of the paper's table (Section 4.1):
    reactant a stiffened gas (gamma 4, p_inf 1 GPa, C_V 2000), product an ideal
    gas (gamma 3, C_V 1000) with Q = 3.68 MJ/kg; distinct closures, so the
    mixture's component densities come from the temperature equality of
    Appendix B."""
    m = material(4.0, p_inf=1.0e9, reactive=1, Q=3.68e6, cv=2000.0, A=A, T_act=T_act, rate_law=rate_law,
                 p_ign=p_ign)
    m.update(prod_gamma=3.0, prod_p_inf=0.0, prod_cv=1000.0)
    return m


def johnson_cook(m, c1, c2, c3, n, m_exp, T_melt, T0=298.0, chi0=1.0, cv=385.0) -> dict:
    """A Romenskii solid m with the Johnson-Cook plasticity of Section 2.3.2:
    chi = chi0 exp((sqrt(3/2) |dev sigma| / sigma_Y - 1) / c3) with
    sigma_Y = (c1 + c2 eps_p^n)(1 - ((T - T0)/(T_melt - T0))^m_exp).  The
    material then carries the history row rho phi eps_p (the workload's
    reactive_material names it).  chi0 = 1/s, the Johnson-Cook reference strain
    rate, and cv = 385 J/(kg K), copper's specific heat, are not in the
    paper's tables."""
    out = dict(m)
    out.update(plastic=3, sigma_y=float(c1), chi0=float(chi0), cv=float(cv), jc_c2=float(c2),
               jc_c3=float(c3), jc_n=float(n), jc_m=float(m_exp), jc_Tmelt=float(T_melt), jc_T0=float(T0))
    return out


# Copper of the Romenskii table (Section 4.1): rho0 8930, K0 136.5 GPa,
# G0 39.4 GPa, Gamma 2, alpha-bar 1, beta-bar 3.
COPPER_ROMENSKII = romenskii(8930.0, 136.5e9, 39.4e9, 2.0, 1.0, 3.0)
# The same copper with the Johnson-Cook table of the indentation tests
# (Section 4.4): c1 0.4 GPa, c2 0.177 GPa, c3 0.025, n 1, m 1.09, T_melt 1358 K.
COPPER_JC = johnson_cook(COPPER_ROMENSKII, 0.4e9, 0.177e9, 0.025, 1.0, 1.09, 1358.0)
# LX-17 reactant of the JWL table: rho0 1905, A 778.1e11 Pa, B -0.0503e11 Pa,
# R1 11.3, R2 1.13, Gamma 0.8938, C_V 1305.5.
LX17_REACTANT_JWL = jwl(1905.0, 778.1e11, -0.0503e11, 11.3, 1.13, 0.8938, cv=1305.5)


# Solid of the 1D solid|gas problem: stiffened-gas-form hydrostatic EOS,
# constant shear modulus, perfect plasticity with radial return.
SOLID = material(4.0, p_inf=6e10, G=5e10, plastic=1, sigma_y=4e8)
SOLID_RHO0 = 8000.0
AIR = material(1.4)
R_AIR = 287.0


@dataclass
class Patch:
    nx: int
    ny: int
    dx: float
    dy: float
    x0: float = 0.0
    y0: float = 0.0
    bc: tuple = (BC_TRANSMISSIVE,) * 4  # x-low, x-high, y-low, y-high
    prim: np.ndarray | None = None       # (nfields, ny, nx) float64


@dataclass
class Workload:
    name: str
    dim: int
    materials: list
    patches: list
    cfl: float
    steps: int
    thinc: bool
    reactive_material: int = -1          # material carrying the history row (reactive: lam; Johnson-Cook: eps_p), -1 none
    extra: dict = field(default_factory=dict)
    scheme: str = "rk3"                  # hyperbolic update: "rk3" (the paper's) or "hancock"
    geometry: str = "planar"             # "planar" (plane strain) or "cyl" (axisymmetric, x = r, y = z)
    limiter: str = "minmod"              # MUSCL slope limiter: "minmod" or "vanleer"

    @property
    def reactive(self) -> bool:
        return self.reactive_material >= 0

    @property
    def cells(self) -> int:
        return sum(p.nx * p.ny for p in self.patches)


def _blank(dim, reactive, ny, nx):
    names = prim_names(dim, reactive)
    w = np.zeros((len(names), ny, nx))
    idx = {n: k for k, n in enumerate(names)}
    for n in ("V11", "V22", "V33"):
        w[idx[n]] = 1.0
    if reactive:
        w[idx["lam"]] = 1.0
    return w, idx


def _area_fraction_disc(xc, yc, r, x0, y0, dx, dy, nx, ny, sub=8):
    """Fraction of each cell inside a disc, by sub x sub point sampling."""
    off = (np.arange(sub) + 0.5) / sub
    xs = x0 + (np.arange(nx)[:, None] + off[None, :]) * dx   # (nx, sub)
    ys = y0 + (np.arange(ny)[:, None] + off[None, :]) * dy   # (ny, sub)
    dxs = (xs - xc) ** 2
    dys = (ys - yc) ** 2
    inside = (dys[:, None, :, None] + dxs[None, :, None, :]) <= r * r  # ny,nx,sub,sub
    return inside.mean(axis=(2, 3))


def riemann_1d(n: int = 1000, left=None, right=None, x_int: float = 0.5,
               cfl: float = 0.8, steps: int = 500, thinc: bool = False,
               bc=BC_TRANSMISSIVE, materials=None, name="riemann_1d") -> Workload:
    """Two-material 1D Riemann problem on [0, 1].

    `left`/`right` are dicts with keys mat (0 = material 1, 1 = material 2),
    rho, u, p.  Default: the 1D solid|gas impact (solid at 500 m/s into air).
    """
    left = left or dict(mat=0, rho=SOLID_RHO0, u=500.0, p=1e5)
    right = right or dict(mat=1, rho=1.2, u=0.0, p=1e5)
    mats = materials or [SOLID, AIR]
    reactive = any(m["reactive"] for m in mats)
    w, k = _blank(1, reactive, 1, n)
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    for side, mask in ((left, xc < x_int), (right, xc >= x_int)):
        phi1 = 1.0 - EPS_PHI if side["mat"] == 0 else EPS_PHI
        w[k["phi1"], 0, mask] = phi1
        w[k["rho1"], 0, mask] = side.get("rho1", side["rho"])
        w[k["rho2"], 0, mask] = side.get("rho2", side["rho"])
        w[k["u"], 0, mask] = side["u"]
        w[k["p"], 0, mask] = side["p"]
    if left["mat"] == 0 and right["mat"] == 1 and "rho2" not in left:
        # keep the absent phase at the density of the same material across the interface
        w[k["rho2"], 0, xc < x_int] = right["rho"]
        w[k["rho1"], 0, xc >= x_int] = left["rho"]
    rmat = next((i for i, m in enumerate(mats) if m["reactive"]), -1)
    p = Patch(nx=n, ny=1, dx=dx, dy=1.0, bc=(bc, bc, BC_TRANSMISSIVE, BC_TRANSMISSIVE), prim=w)
    return Workload(name, 1, mats, [p], cfl, steps, thinc, rmat)


def solid_gas_1d(n: int = 1000, steps: int = 500) -> Workload:
    """1D solid|gas Riemann problem: 1000 cells, interface 0.5, CFL 0.8, 500 steps."""
    return riemann_1d(n, steps=steps, name=f"1d_solid_gas_{n}")


def mach2_shock_positions():
    """Post-shock state of a Mach-2 shock in air (gamma 1.4) running into (1.2, 1e5, 0)."""
    g, rho1, p1, M = 1.4, 1.2, 1e5, 2.0
    c1 = math.sqrt(g * p1 / rho1)
    rho2 = rho1 * (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = p1 * (1 + 2 * g / (g + 1) * (M * M - 1))
    u2 = M * c1 * (1 - rho1 / rho2)
    return rho2, p2, u2


def shock_disc_2d(n: int = 512, steps: int = 2000, thinc: bool = True,
                  shock_x: float = 0.25, name=None) -> Workload:
    """Mach-2 air shock striking an elastoplastic disc (r 0.1 at (0.4, 0.5)) on [0,1]^2."""
    w, k = _blank(2, False, n, n)
    d = 1.0 / n
    frac = _area_fraction_disc(0.4, 0.5, 0.1, 0.0, 0.0, d, d, n, n)
    w[k["phi1"]] = EPS_PHI + (1 - 2 * EPS_PHI) * frac
    w[k["rho1"]] = SOLID_RHO0
    w[k["rho2"]] = 1.2
    w[k["p"]] = 1e5
    rho2, p2, u2 = mach2_shock_positions()
    xc = (np.arange(n) + 0.5) * d
    post = np.broadcast_to(xc[None, :] < shock_x, (n, n))
    w[k["rho2"]][post] = rho2
    w[k["p"]][post] = p2
    w[k["u"]][post] = u2
    p = Patch(nx=n, ny=n, dx=d, dy=d, prim=w)
    return Workload(name or f"2d_shock_disc_{n}", 2, [SOLID, AIR], [p], 0.6, steps, thinc)


def sphere_shock_rz(n: int = 128, steps: int = 200, thinc: bool = True, shock_z: float = 0.25,
                    name=None) -> Workload:
    """Axisymmetric (x = r, y = z) form of the shock-disc problem: an
    elastoplastic sphere of radius 0.1 centred on the axis at z = 0.4 in air,
    struck by a Mach-2 air shock travelling in +z.  (r, z) in [0, 0.5] x [0, 1],
    n cells per unit length; reflective axis, transmissive elsewhere."""
    nx, ny = n // 2, n
    w, k = _blank(2, False, ny, nx)
    d = 1.0 / n
    frac = _area_fraction_disc(0.0, 0.4, 0.1, 0.0, 0.0, d, d, nx, ny)
    w[k["phi1"]] = EPS_PHI + (1 - 2 * EPS_PHI) * frac
    w[k["rho1"]] = SOLID_RHO0
    w[k["rho2"]] = 1.2
    w[k["p"]] = 1e5
    rho2, p2, u2 = mach2_shock_positions()
    zc = (np.arange(ny) + 0.5) * d
    post = np.broadcast_to(zc[:, None] < shock_z, (ny, nx))
    w[k["rho2"]][post] = rho2
    w[k["p"]][post] = p2
    w[k["v"]][post] = u2
    p = Patch(nx=nx, ny=ny, dx=d, dy=d, x0=0.0,
              bc=(BC_REFLECTIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE), prim=w)
    return Workload(name or f"2d_sphere_shock_rz_{n}", 2, [SOLID, AIR], [p], 0.6, steps, thinc,
                    geometry="cyl")


def cylinder_core_1d(n: int = 400, steps: int = 200, r_core: float = 0.3, x0: float = 0.0,
                     name=None) -> Workload:
    """1D cylindrical (radius only): an elastoplastic core r < r_core at rest
    under 1e5 Pa inside air at 5e6 Pa that implodes onto it; [x0, x0 + 1],
    reflective at the low face (the axis when x0 = 0), transmissive outside."""
    w, k = _blank(1, False, 1, n)
    d = 1.0 / n
    rc = x0 + (np.arange(n) + 0.5) * d
    core = rc < r_core
    w[k["phi1"], 0] = np.where(core, 1.0 - EPS_PHI, EPS_PHI)
    w[k["rho1"], 0] = SOLID_RHO0
    w[k["rho2"], 0] = 1.2
    w[k["p"], 0] = np.where(core, 1e5, 5e6)
    p = Patch(nx=n, ny=1, dx=d, dy=1.0, x0=x0,
              bc=(BC_REFLECTIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE), prim=w)
    return Workload(name or f"1d_cylinder_core_{n}", 1, [SOLID, AIR], [p], 0.8, steps, False,
                    geometry="cyl")


def reactive_plate_2d(nx: int = 2048, ny: int = 1024, steps: int = 1000, seed: int = 2,
                      A: float = 1.0e7, name=None) -> Workload:
    """Premixed reactive air over an elastoplastic plate (y < 0.2) on [0,2]x[0,1].

    Arrhenius single-step A -> B with T_act = 15 T0 and Q = 20 R T0, hot spot of
    radius 0.02 at (1.0, 0.3) at 3 T0, density white noise of amplitude 1e-3.
    """
    rho0, p0, g = 1.2, 1e5, 1.4
    T0 = p0 / (rho0 * R_AIR)
    cv = R_AIR / (g - 1)
    gas = material(g, reactive=1, Q=20 * R_AIR * T0, cv=cv, A=A, T_act=15 * T0)
    w, k = _blank(2, True, ny, nx)
    dx = 2.0 / nx
    dy = 1.0 / ny
    yc = (np.arange(ny) + 0.5) * dy
    # exact fraction of each row below y = 0.2
    ylo = np.arange(ny) * dy
    frac = np.clip((0.2 - ylo) / dy, 0.0, 1.0)
    w[k["phi1"]] = (EPS_PHI + (1 - 2 * EPS_PHI) * frac)[:, None]
    w[k["rho1"]] = SOLID_RHO0
    hot = _area_fraction_disc(1.0, 0.3, 0.02, 0.0, 0.0, dx, dy, nx, ny)
    # hot spot at 3 T0 and ambient pressure: rho = rho0 / 3 (area-weighted specific volume)
    rho_gas = 1.0 / ((1 - hot) / rho0 + hot * 3.0 / rho0)
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, size=(ny, nx))
    gas_cells = (frac < 1.0)[:, None] & np.ones((1, nx), bool)
    rho_gas = np.where(gas_cells, rho_gas * (1 + 1e-3 * xi), rho_gas)
    w[k["rho2"]] = rho_gas
    w[k["p"]] = p0
    w[k["lam"]] = 1.0
    del yc
    p = Patch(nx=nx, ny=ny, dx=dx, dy=dy, prim=w)
    return Workload(name or f"2d_reactive_plate_{nx}x{ny}", 2, [SOLID, gas], [p], 0.6,
                    steps, True, reactive_material=1, extra=dict(T0=T0))


def detonation_copper_1d(n: int = 1000, steps: int = 400, name=None, copper: str = "romenskii",
                         explosive: str = "standin") -> Workload:
    """The shape of the one-dimensional test of Section 4.1 on [0, 0.4] m:
    quiescent elastic copper for x < 0.15, ambient explosive for
    0.15 < x < 0.35, a booster of the same explosive at 1e9 Pa for x > 0.35,
    1e5 Pa elsewhere; the reactant burns at lam_dot = -k sqrt(lam),
    k = 2e6 1/s, once the pressure exceeds 1e8 Pa; CFL 0.9, transmissive ends.

    Copper: the Romenskii solid of the paper's table (rho_0 8930 kg/m^3,
    K_0 136.5 GPa, G_0 39.4 GPa, Gamma 2, alpha 1, beta 3; no plasticity), or
    with copper="stiffened" a stiffened gas of the same rho_0, Gamma,
    gamma p_inf = K_0 and constant G = G_0.  Explosive: explosive="generic"
    is the generic explosive of the paper's table (reactant and product
    stiffened gases with closures of their own, component densities from
    the temperature equality of Appendix B; float64 contexts), the default
    "standin" one ideal gas for reactant and product with the product's
    gamma 3, c_V 1000, Q = 3.68 MJ/kg and the reactant's rho_0 = 1600 kg/m^3
    (every precision and the adjoint accept it).
    """
    copper = (COPPER_ROMENSKII if copper == "romenskii" else material(3.0, p_inf=136.5e9 / 3.0, G=39.4e9))
    expl = (generic_explosive() if explosive == "generic" else
            material(3.0, reactive=1, Q=3.68e6, cv=1000.0, A=2.0e6, rate_law=1, p_ign=1.0e8))
    w, k = _blank(1, True, 1, n)
    dx = 0.4 / n
    xc = (np.arange(n) + 0.5) * dx
    cu = xc < 0.15
    w[k["phi1"], 0] = np.where(cu, 1.0 - EPS_PHI, EPS_PHI)
    w[k["rho1"], 0] = 8930.0
    w[k["rho2"], 0] = 1600.0
    w[k["p"], 0] = np.where(xc > 0.35, 1.0e9, 1.0e5)
    p = Patch(nx=n, ny=1, dx=dx, dy=1.0, prim=w)
    return Workload(name or f"1d_detonation_copper_{n}", 1, [copper, expl], [p], 0.9, steps, True,
                    reactive_material=1)


def jc_flyer_1d(n: int = 400, steps: int = 200, u_flyer: float = 876.0, name=None) -> Workload:
    """Johnson-Cook copper plate impact on [0, 40] mm: a copper flyer
    (x < 10 mm) at u_flyer m/s strikes copper at rest (10 < x < 30 mm), air
    (ideal, gamma 1.4, 1.2 kg/m^3) beyond; 1e5 Pa everywhere, eps_p = 0;
    CFL 0.6, transmissive ends, THINC on."""
    air = material(1.4)
    w, k = _blank(1, True, 1, n)
    dx = 0.04 / n
    xc = (np.arange(n) + 0.5) * dx
    cu = xc < 0.03
    w[k["phi1"], 0] = np.where(cu, 1.0 - EPS_PHI, EPS_PHI)
    w[k["rho1"], 0] = 8930.0
    w[k["rho2"], 0] = 1.2
    w[k["u"], 0] = np.where(xc < 0.01, u_flyer, 0.0)
    w[k["p"], 0] = 1.0e5
    w[k["lam"], 0] = 0.0
    p = Patch(nx=n, ny=1, dx=dx, dy=1.0, prim=w)
    return Workload(name or f"1d_jc_flyer_{n}", 1, [COPPER_JC, air], [p], 0.6, steps, True,
                    reactive_material=0)


def indentation_rz(nr: int = 64, steps: int = 200, radius: float = 4.0e-3, u_drive: float = 876.0,
                   name=None) -> Workload:
    """The shock-driven hemispherical indentation of Section 4.4 in its
    axisymmetric form (x = r, y = z): (r, z) in [0, 6.4] x [0, 32] mm, nr x 5 nr
    square cells; Johnson-Cook copper below z = 20 mm with a hemispherical
    indentation of the given radius centred on the axis at z = 20 mm, air
    (gamma 1.4) above and inside it; the copper below z = 2 mm (14 mm of plate
    under the indentation) moves at u_drive in +z, the driven base; 1e5 Pa,
    eps_p = 0; reflective axis, transmissive elsewhere; CFL 0.6, THINC on.
    Volume fractions are the copper's area share of each cell (8 x 8 point
    sampling)."""
    air = material(1.4)
    nz = 5 * nr
    d = 6.4e-3 / nr
    w, k = _blank(2, True, nz, nr)
    sub = 8
    off = (np.arange(sub) + 0.5) / sub
    rs = (np.arange(nr)[:, None] + off[None, :]) * d          # (nr, sub)
    zs = (np.arange(nz)[:, None] + off[None, :]) * d          # (nz, sub)
    zt = 0.02
    below = zs[:, None, :, None] < zt                          # nz, 1, sub, 1
    inside = (rs[None, :, None, :] ** 2 + (zs[:, None, :, None] - zt) ** 2) < radius * radius
    frac = (below & ~inside).mean(axis=(2, 3))
    w[k["phi1"]] = EPS_PHI + (1 - 2 * EPS_PHI) * frac
    w[k["rho1"]] = 8930.0
    w[k["rho2"]] = 1.2
    w[k["p"]] = 1.0e5
    zc = (np.arange(nz) + 0.5) * d
    w[k["v"]] = np.where(zc < 0.002, u_drive, 0.0)[:, None]
    w[k["lam"]] = 0.0
    p = Patch(nx=nr, ny=nz, dx=d, dy=d, x0=0.0,
              bc=(BC_REFLECTIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE), prim=w)
    return Workload(name or f"2d_indentation_rz_{nr}x{nz}", 2, [COPPER_JC, air], [p], 0.6, steps, True,
                    reactive_material=0, geometry="cyl")


def batched_riemann_1d(n_problems: int = 4096, seed: int = 3, steps: int = 300,
                       nmin: int = 256, nmax: int = 4096, name=None) -> Workload:
    """Many independent two-material 1D Riemann problems of log-uniform size."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_problems))).astype(int)
    patches = []
    for b in range(n_problems):
        n = int(sizes[b])
        sides = []
        for _ in range(2):
            rho = math.exp(rng.uniform(0.0, math.log(1e4)))
            p = math.exp(rng.uniform(math.log(1e5), math.log(1e10)))
            u = rng.uniform(-500.0, 500.0)
            mat = 0 if rng.uniform() < 0.5 else 1
            sides.append(dict(mat=mat, rho=rho, u=u, p=p))
        w, k = _blank(1, False, 1, n)
        dx = 1.0 / n
        xc = (np.arange(n) + 0.5) * dx
        for side, mask in ((sides[0], xc < 0.5), (sides[1], xc >= 0.5)):
            w[k["phi1"], 0, mask] = 1.0 - EPS_PHI if side["mat"] == 0 else EPS_PHI
            w[k["rho1"], 0, mask] = side["rho"]
            w[k["rho2"], 0, mask] = side["rho"]
            w[k["u"], 0, mask] = side["u"]
            w[k["p"], 0, mask] = side["p"]
        patches.append(Patch(nx=n, ny=1, dx=dx, dy=1.0, prim=w))
    return Workload(name or f"1d_batch_{n_problems}", 1, [SOLID, AIR], patches, 0.8,
                    steps, False)


def smooth_disc_2d(n: int = 16, steps: int = 10, u0: float = 100.0, seed: int = 5,
                   sigma_y: float | None = None, name=None) -> Workload:
    """Smooth solid|gas problem for derivative checks on [0, 1]^2 (periodic).

    An elastoplastic disc (radius 0.25 at the centre) with a tanh-profiled
    volume fraction (width 1.5 cells), a Gaussian x-velocity pulse of peak u0
    (width 0.2), and seeded smooth periodic modulations of every other field
    (densities 1 %, pressure 1 %, y velocity 0.1 u0, stretch components 1e-4),
    so that no field is uniform: no shocks, no THINC, no exactly equal
    neighbour differences.  sigma_y overrides the solid's yield stress.
    """
    w, k = _blank(2, False, n, n)
    d = 1.0 / n
    xc = (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(xc, xc)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2)
    phi = 0.5 * (1.0 + np.tanh((0.25 - r) / (1.5 * d)))
    w[k["phi1"]] = EPS_PHI + (1 - 2 * EPS_PHI) * phi
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, size=(8, 2))

    def wave(m):
        return np.sin(2 * np.pi * X + ph[m, 0]) * np.cos(2 * np.pi * Y + ph[m, 1])

    mod = 1.0 + 0.01 * wave(0)
    w[k["rho1"]] = SOLID_RHO0 * mod
    w[k["rho2"]] = 1.2 * mod
    w[k["p"]] = 1e5 * (1.0 + 0.01 * wave(1))
    w[k["u"]] = u0 * np.exp(-r ** 2 / (2 * 0.2 ** 2))
    w[k["v"]] = 0.1 * u0 * wave(2)
    for m, f in enumerate(("V11", "V12", "V21", "V22", "V33")):
        w[k[f]] = w[k[f]] + 1e-4 * wave(3 + m)
    solid = dict(SOLID)
    if sigma_y is not None:
        solid["sigma_y"] = sigma_y
    per = (BC_PERIODIC,) * 4
    p = Patch(nx=n, ny=n, dx=d, dy=d, bc=per, prim=w)
    return Workload(name or f"2d_smooth_disc_{n}", 2, [solid, AIR], [p], 0.6, steps, False)


def perturbed(wl: Workload, seed: int = 11, amp: float = 1e-4) -> Workload:
    """Copy of a workload whose primitive fields carry a seeded cell-wise
    random perturbation of relative size amp (velocities amp x 100 m/s,
    stretch components amp x 1e-2, the volume fraction amp x min(phi, 1 - phi),
    the reactant fraction amp x lam downwards), so that no two neighbouring
    values are equal: limiter, min / max and region choices then have margins
    far above round-off (derivative checks are well posed)."""
    import copy
    out = copy.deepcopy(wl)
    rng = np.random.default_rng(seed)
    k = {n: i for i, n in enumerate(prim_names(wl.dim, wl.reactive))}
    for p in out.patches:
        x = p.prim

        def u():
            return rng.uniform(-1.0, 1.0, size=x.shape[1:])

        phi = x[k["phi1"]]
        x[k["phi1"]] = phi + amp * np.minimum(phi, 1.0 - phi) * u()
        for f in ("rho1", "rho2", "p"):
            x[k[f]] = x[k[f]] * (1.0 + amp * u())
        for f in ("u", "v"):
            if f in k:
                x[k[f]] = x[k[f]] + amp * 100.0 * u()
        for f in ("V11", "V12", "V21", "V22", "V33"):
            if f in k:
                x[k[f]] = x[k[f]] + amp * 1e-2 * u()
        if "lam" in k:
            x[k["lam"]] = x[k["lam"]] * (1.0 - amp * np.abs(u()))
    out.name = wl.name + "_perturbed"
    return out


def adjoint_case_2d(n: int = 256, steps: int = 200, seed: int = 4) -> Workload:
    """256^2 shock-disc problem whose phase densities carry a smooth Gaussian
    perturbation of amplitude 1e-2 (width 0.05, centre seeded within 0.02 of
    the disc centre).  extra["drho_shape"] is the Gaussian, the direction of
    the density-gradient checks.  The shock starts at x = 0.28, next to the
    disc (edge at 0.3): 200 steps last ~8e-5 s, in which a Mach-2 air shock
    travels ~0.05, so the solid is struck within the run."""
    wl = shock_disc_2d(n, steps=steps, shock_x=0.28, name=f"2d_shock_disc_adjoint_{n}")
    rng = np.random.default_rng(seed)
    cx, cy = 0.4 + rng.uniform(-0.02, 0.02), 0.5 + rng.uniform(-0.02, 0.02)
    d = 1.0 / n
    xc = (np.arange(n) + 0.5) * d
    r2 = (xc[None, :] - cx) ** 2 + (xc[:, None] - cy) ** 2
    shape = np.exp(-r2 / (2 * 0.05 ** 2))
    k = {nm: i for i, nm in enumerate(prim_names(2, False))}
    for p in wl.patches:
        p.prim[k["rho1"]] *= 1.0 + 1e-2 * shape
        p.prim[k["rho2"]] *= 1.0 + 1e-2 * shape
    wl.extra["drho_shape"] = shape
    wl.extra["seed"] = seed
    return wl


CONFIGS = {
    "1d_solid_gas": solid_gas_1d,
    "2d_shock_disc": shock_disc_2d,
    "2d_reactive_plate": reactive_plate_2d,
    "1d_batch": batched_riemann_1d,
    "2d_adjoint": adjoint_case_2d,
    "2d_smooth_disc": smooth_disc_2d,
}
