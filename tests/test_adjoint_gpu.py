"""Adjoint of the float64 GPU step (dis_adj_forward / dis_adjoint) against
the oracle's own reverse mode (PyTorch autograd through the float64 CPU
oracle) and against central finite differences.

Inputs: the gradient of a limited scheme is only defined away from its kinks
(minmod at a zero or tied slope, min / max of equal wave speeds, the yield
surface).  The seeded workloads have exactly uniform regions, where every
limiter sits on a kink and a one-ulp difference between two float64 programs
flips the derivative (the oracle's own gradient moves by up to 85 % under
one-ulp input perturbations there).  The parity cases therefore add a seeded
cell-wise perturbation of relative size 1e-4 to every primitive field
(workloads.perturbed), which puts every choice far from its kink.

Parity metric (per field f of the initial-state gradient):
    err_f = max |g_gpu - g_oracle| / max |g_oracle|
Bar: max(1e-8, 10 x the oracle's own spread under one-ulp input
perturbations), the same calibration as the forward THINC parity tests; the
measured spreads are 1e-14 .. 2e-8.  Parameters: same rule.  Finite
differences: 1e-4 relative (central, relative step 1e-6, time steps held at
the recorded values).
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2009_14555_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_record = {}


def _save():
    from tests.parity_util import record_path
    with open(record_path("adjoint_err.json"), "w") as f:
        json.dump(_record, f, indent=1)


def gpu_grad(wl, steps, material, qbar=None, every=3, kind=1, dts=None):
    """GPU J, gradient w.r.t. the initial state (primitive kind=1 or
    conservative kind=0, per patch arrays), parameter gradients and dts."""
    from paper_2009_14555_gb300.solver import Solver, pack, unpack
    s = Solver.from_workload(wl)
    s.set_prim([p.prim for p in wl.patches])
    J, used = s.adj_forward(steps, every=every, material=material, dts=dts)
    rc, bp, bc = s.check()
    assert rc == 0, (bp, bc)
    qN = s.get_arrays()
    qb = None if qbar is None else pack(qbar)
    if qb is not None:
        J = J + float(sum((a * b).sum() for a, b in zip(qbar, qN)))
    g, gp = s.adjoint(qb, 1.0 if material >= 0 else 0.0, kind=kind)
    s.close()
    return J, unpack(g, [p.prim.shape for p in wl.patches]), gp, used


def oracle_grad(wl, steps, material, qbar=None, kind="prim", prim=None):
    from oracle import adjoint as OA
    from oracle import scheme as OS
    from oracle.closures import prim_to_cons
    p = wl.patches[0]
    theta = torch.tensor([m[k] for m in wl.materials for k in OA.PARAM_KEYS], dtype=torch.float64,
                         requires_grad=True)
    w0 = p.prim if prim is None else prim
    if kind == "prim":
        init = torch.tensor(w0, dtype=torch.float64, requires_grad=True)
    else:
        q0 = prim_to_cons(OS.prim_from_array(w0, wl.dim, wl.reactive), wl.materials)
        init = OS.cons_to_array(q0, wl.dim, wl.reactive).detach().clone().requires_grad_(True)
    J, _, dts = OA.rollout(init, kind, wl.dim, OA.with_params(wl.materials, theta), p,
                           dict(cfl=wl.cfl, thinc=wl.thinc, geometry=getattr(wl, "geometry", "planar"),
                                limiter=getattr(wl, "limiter", "minmod")),
                           steps, material,
                           None if qbar is None else qbar[0])
    J.backward()
    return float(J), init.grad.numpy(), theta.grad.numpy(), dts


def field_err(g, o):
    g, o = np.asarray(g), np.asarray(o)
    out = []
    for f in range(o.shape[0]):
        sc = max(np.abs(o[f]).max(), 1e-300)
        out.append(float(np.abs(g[f] - o[f]).max() / sc))
    return out


def param_err(gp, op, mask):
    return [float(abs(gp[k] - op[k]) / max(abs(op[k]), 1e-300)) for k in mask]


def _case(name, wl, steps, material, qbar_seed=None, params=(0, 1), kind="prim"):
    qbar = None
    if qbar_seed is not None:
        rng = np.random.default_rng(qbar_seed)
        # adjoint weights scaled so every field contributes comparably
        sc = np.abs(wl.patches[0].prim).reshape(wl.patches[0].prim.shape[0], -1).max(1)
        qbar = [rng.standard_normal(p.prim.shape) / np.maximum(sc, 1.0)[:, None, None] * 1e-3
                for p in wl.patches]
    Jg, gg, gpg, gdt = gpu_grad(wl, steps, material, qbar, kind=1 if kind == "prim" else 0)
    Jo, go, gpo, odt = oracle_grad(wl, steps, material, qbar, kind)
    # the oracle's own one-ulp spread calibrates the bar
    rng = np.random.default_rng(123)
    p0 = wl.patches[0].prim
    pu = p0 * (1 + np.sign(rng.standard_normal(p0.shape)) * 2.0 ** -52)
    _, gu, gpu_, _ = oracle_grad(wl, steps, material, qbar, kind, prim=pu)
    spread = field_err(gu, go)
    pspread = param_err(gpu_, gpo, params)
    e = field_err(gg[0], go)
    ep = param_err(gpg, gpo, params)
    bar = [max(1e-8, 10 * x) for x in spread]
    pbar = [max(1e-8, 10 * x) for x in pspread]
    _record[name] = dict(J_gpu=Jg, J_oracle=Jo, field_err=e, field_spread=spread, param_err=ep,
                         param_spread=pspread, params_gpu=[float(gpg[k]) for k in params],
                         params_oracle=[float(gpo[k]) for k in params],
                         dt_rel=float(np.max(np.abs(np.asarray(gdt)[:, 0] - np.asarray(odt)) / np.asarray(odt))))
    _save()
    assert abs(Jg - Jo) <= 1e-10 * abs(Jo) + 1e-300, (Jg, Jo)
    assert all(x <= b for x, b in zip(e, bar)), (e, bar)
    assert all(x <= b for x, b in zip(ep, pbar)), (ep, pbar, gpg, gpo)


def test_adjoint_1d_solid_gas_vs_oracle():
    wl = W.perturbed(W.solid_gas_1d(n=100, steps=12))
    _case("1d_solid_gas_100_12", wl, 12, material=0, qbar_seed=1)


def test_adjoint_1d_conservative_vs_oracle():
    wl = W.perturbed(W.solid_gas_1d(n=100, steps=6), seed=12)
    _case("1d_solid_gas_100_6_cons", wl, 6, material=0, qbar_seed=2, kind="cons")


def test_adjoint_2d_shock_disc_vs_oracle():
    wl = W.perturbed(W.shock_disc_2d(n=20, steps=4, thinc=False, shock_x=0.3))
    _case("2d_shock_disc_20_4", wl, 4, material=0, qbar_seed=3)


def _vanleer(wl):
    wl.limiter = "vanleer"
    return wl


def test_adjoint_vanleer_1d_vs_oracle():
    """The van Leer limiter (harmonic slope 2ab / (a + b)) reversed by hand."""
    wl = _vanleer(W.perturbed(W.solid_gas_1d(n=100, steps=12)))
    _case("1d_solid_gas_vanleer_100_12", wl, 12, material=0, qbar_seed=1)


def test_adjoint_vanleer_2d_thinc_vs_oracle():
    wl = _vanleer(W.perturbed(W.shock_disc_2d(n=20, steps=4, thinc=True, shock_x=0.3)))
    _case("2d_shock_disc_vanleer_thinc_20_4", wl, 4, material=0, qbar_seed=4)


def test_adjoint_2d_thinc_vs_oracle():
    wl = W.perturbed(W.shock_disc_2d(n=20, steps=4, thinc=True, shock_x=0.3))
    _case("2d_shock_disc_thinc_20_4", wl, 4, material=0, qbar_seed=4)


def test_adjoint_reactive_vs_oracle():
    # 96 x 48 resolves the hot spot (radius 0.02) so the reaction progresses
    # within 3 steps; the heat release gradient (entry 5) is then not small
    wl = W.perturbed(W.reactive_plate_2d(nx=96, ny=48, steps=3))
    _case("2d_reactive_plate_96x48_3", wl, 3, material=1, qbar_seed=5, params=(0, 1, 5))


def _detonation_partial_burn():
    # the k sqrt(lam) law with its pressure switch (Section 4.1), k lowered to
    # 2e5 1/s so that at 100 cells the booster burns over several steps
    # (partially burnt cells rather than a clamp to lam = 0 in one step)
    wl = W.perturbed(W.detonation_copper_1d(100, steps=8, copper="stiffened"))
    wl.materials[1]["A"] = 2e5
    return wl


def test_adjoint_sqrt_rate_law_vs_oracle():
    _case("1d_detonation_sqrt_law_100_8", _detonation_partial_burn(), 8, material=1, qbar_seed=6,
          params=(0, 5))


def test_adjoint_cylindrical_1d_vs_oracle():
    # implosion onto a solid core in r (the geometric source of Section 3)
    wl = W.perturbed(W.cylinder_core_1d(100, steps=12))
    _case("1d_cylinder_core_100_12", wl, 12, material=0, qbar_seed=7, params=(0,))  # no yield: dJ/dsigma_Y = 0


def _reflective_planar(thinc):
    """Planar 2D case with reflective walls on two sides: the half disc of
    sphere_shock_rz (40 cells per unit length) sits on the x-low wall and the
    Mach-2 shock, started at y = 0.28, strikes it within the first steps; the
    y-high boundary is a reflective wall too."""
    from paper_2009_14555_gb300.workloads import BC_REFLECTIVE, BC_TRANSMISSIVE
    wl = W.sphere_shock_rz(40, steps=4, thinc=thinc, shock_z=0.28)
    wl.geometry = "planar"
    wl.patches[0].bc = (BC_REFLECTIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_REFLECTIVE)
    return W.perturbed(wl, seed=21)


def test_adjoint_2d_reflective_walls_vs_oracle():
    _case("2d_reflective_walls_40_4", _reflective_planar(False), 4, material=0, qbar_seed=8)


def test_adjoint_2d_reflective_walls_thinc_vs_oracle():
    _case("2d_reflective_walls_thinc_40_4", _reflective_planar(True), 4, material=0, qbar_seed=9)


def test_adjoint_cylindrical_2d_vs_oracle():
    """The shock-sphere problem in (r, z): the geometric source of Section 3
    with the reflective axis, the sphere on the axis struck within the run."""
    wl = W.perturbed(W.sphere_shock_rz(40, steps=4, thinc=False, shock_z=0.28), seed=22)
    _case("2d_sphere_shock_rz_40_4", wl, 4, material=0, qbar_seed=10)


def _romenskii_copper(wl, seed):
    """Romenskii copper (the Section 4.1 table) with perfect plasticity at
    sigma_y = 0.4 GPa in place of material 0, perturbed."""
    wl.materials = [dict(W.COPPER_ROMENSKII, plastic=1, sigma_y=0.4e9), W.AIR]
    k = W.prim_names(wl.dim, wl.reactive).index("rho1")
    for p in wl.patches:
        p.prim[k] = 8930.0
    return W.perturbed(wl, seed=seed)


def test_adjoint_romenskii_1d_vs_oracle():
    """Romenskii copper striking air at 500 m/s: the local maps reversed by
    dual numbers through the Romenskii closure (G(rho) = G_0 (rho/rho_0)^(b+1)
    in the stress, the sound speed and the yield strain); parameters G_0 and
    sigma_y of the copper."""
    wl = _romenskii_copper(W.riemann_1d(100, dict(mat=0, rho=8930.0, u=500.0, p=1e5),
                                        dict(mat=1, rho=1.2, u=0.0, p=1e5),
                                        materials=[W.COPPER_ROMENSKII, W.AIR], steps=10), seed=31)
    _case("1d_romenskii_copper_air_100_10", wl, 10, material=0, qbar_seed=11, params=(0, 1))


def test_adjoint_romenskii_detonation_vs_oracle():
    """The k sqrt(lam) detonation driven into Romenskii copper (the Section
    4.1 closures but for the explosive's single closure): reaction and
    Romenskii solid in one reversed step."""
    wl = W.perturbed(W.detonation_copper_1d(100, steps=8, copper="romenskii", explosive="standin"))
    wl.materials[1]["A"] = 2e5
    _case("1d_detonation_romenskii_100_8", wl, 8, material=1, qbar_seed=13, params=(5,))


def test_adjoint_romenskii_2d_vs_oracle():
    """A Romenskii copper disc struck by the Mach-2 air shock (2D)."""
    wl = _romenskii_copper(W.shock_disc_2d(20, steps=4, thinc=False, shock_x=0.28), seed=32)
    _case("2d_romenskii_disc_20_4", wl, 4, material=0, qbar_seed=12, params=(0, 1))


def test_adjoint_smooth_vs_oracle():
    wl = W.perturbed(W.smooth_disc_2d(n=16, steps=8, sigma_y=4e7))
    _case("2d_smooth_disc_16_8", wl, 8, material=0)


def _fd_check(name, wl, steps, material, direction, params, every=4, rel=1e-6, tol=1e-4, qbar=None):
    """Central differences of the GPU objective J + <qbar, q_final> with the
    recorded dts held."""
    from paper_2009_14555_gb300.solver import Solver, pack
    s = Solver.from_workload(wl)
    w0 = pack([p.prim for p in wl.patches])
    qb = None if qbar is None else pack(qbar)
    s.set_state(w0)
    J0, dts = s.adj_forward(steps, every=every, material=material)
    g, gp = s.adjoint(qb, 1.0 if material >= 0 else 0.0, kind=1)
    theta0 = s.params()

    def J_at(w, th):
        s.set_params(th)
        s.set_state(w)
        J, _ = s.adj_forward(steps, every=every, material=material, dts=dts)
        if qb is not None:
            J += float(qb @ s.get_state())
        return J

    rec = {}
    d = pack(direction)
    eps = rel * np.abs(w0).max() / max(np.abs(d).max(), 1e-300)
    fd = (J_at(w0 + eps * d, theta0) - J_at(w0 - eps * d, theta0)) / (2 * eps)
    an = float(g @ d)
    rec["state"] = dict(fd=fd, adjoint=an, rel=abs(fd - an) / abs(an))
    for k in params:
        h = rel * theta0[k]
        e = np.zeros_like(theta0)
        e[k] = h
        fdk = (J_at(w0, theta0 + e) - J_at(w0, theta0 - e)) / (2 * h)
        rec[f"param{k}"] = dict(fd=fdk, adjoint=float(gp[k]), rel=abs(fdk - gp[k]) / abs(gp[k]))
    rec["J"] = J_at(w0, theta0)
    s.close()
    _record[name] = rec
    _save()
    for key, r in rec.items():
        if key != "J":
            assert r["rel"] <= tol, (key, r)


def test_adjoint_fd_smooth():
    wl = W.perturbed(W.smooth_disc_2d(n=32, steps=20, sigma_y=4e7))
    p = wl.patches[0]
    rng = np.random.default_rng(7)
    k = {n: i for i, n in enumerate(W.prim_names(2, False))}
    d = np.zeros_like(p.prim)
    xc = (np.arange(p.nx) + 0.5) * p.dx
    X, Y = np.meshgrid(xc, xc)
    a, b = rng.uniform(0, 2 * np.pi, 2)
    d[k["rho1"]] = p.prim[k["rho1"]] * np.sin(2 * np.pi * X + a)
    d[k["rho2"]] = p.prim[k["rho2"]] * np.sin(2 * np.pi * X + a)
    d[k["u"]] = 10.0 * np.cos(2 * np.pi * Y + b)
    d[k["p"]] = 1e4 * np.sin(2 * np.pi * (X + Y))
    _fd_check("fd_smooth_disc_32_20", wl, 20, 0, [d], params=(0, 1))


def test_adjoint_fd_reactive():
    """Heat release and the gas density against central differences; the
    objective is the final reaction-progress density sum(phi_y rho_y lam)
    (Q raises the recovered pressure, hence the temperature and the rate)."""
    wl = W.perturbed(W.reactive_plate_2d(nx=96, ny=48, steps=6))
    p = wl.patches[0]
    k = {n: i for i, n in enumerate(W.prim_names(2, True))}
    d = np.zeros_like(p.prim)
    d[k["rho2"]] = p.prim[k["rho2"]]
    qbar = np.zeros_like(p.prim)
    qbar[k["lam"]] = 1.0  # slot of phi_y rho_y lam in the conservative layout
    _fd_check("fd_reactive_plate_96x48_6", wl, 6, -1, [d], params=(5,), qbar=[qbar])


def test_adjoint_checkpoint_interval_invariance():
    wl = W.perturbed(W.smooth_disc_2d(n=16, steps=9, sigma_y=4e7))
    from paper_2009_14555_gb300.solver import Solver
    res = []
    for every in (1, 4, 9):
        s = Solver.from_workload(wl)
        s.set_prim([p.prim for p in wl.patches])
        s.adj_forward(9, every=every, material=0)
        res.append(s.adjoint(None, 1.0, kind=1))
        s.close()
    for g, gp in res[1:]:
        assert np.allclose(g, res[0][0], rtol=1e-12, atol=1e-12 * np.abs(res[0][0]).max())
        assert np.allclose(gp, res[0][1], rtol=1e-10, atol=0)


def test_adjoint_fullsize_shock_disc():
    """The 256^2 shock-disc adjoint case: 200 steps, checkpoint every 20,
    gradient of the solid's time-integrated x momentum with respect to the
    initial density field, checked along the seeded Gaussian perturbation by
    central differences (relative steps 1e-4, 1e-5, 1e-6; bar 1e-4 on each);
    forward and reverse times are recorded.  The input carries the 1e-4
    cell-wise perturbation that removes exact ties (uniform regions put every
    limiter on a kink, where finite differences and the adjoint disagree)."""
    import time
    from paper_2009_14555_gb300.solver import Solver, pack
    wl = W.perturbed(W.adjoint_case_2d(256, steps=200))
    p = wl.patches[0]
    k = {n: i for i, n in enumerate(W.prim_names(2, False))}
    d = np.zeros_like(p.prim)
    shape = wl.extra["drho_shape"]
    d[k["rho1"]] = p.prim[k["rho1"]] * shape
    d[k["rho2"]] = p.prim[k["rho2"]] * shape
    s = Solver.from_workload(wl)
    w0 = pack([p.prim])
    s.set_state(w0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J0, dts = s.adj_forward(200, every=20, material=0)
    t1 = time.perf_counter()
    g, gp = s.adjoint(None, 1.0, kind=1)
    t2 = time.perf_counter()
    dd = pack([d])
    an = float(g @ dd)
    rec = dict(J=J0, forward_s=t1 - t0, reverse_s=t2 - t1, dG=float(gp[0]), dsigma_y=float(gp[1]),
               cells=p.nx * p.ny, steps=200)
    for eps in (1e-4, 1e-5, 1e-6):
        def J_at(w):
            s.set_state(w)
            return s.adj_forward(200, every=20, material=0, dts=dts)[0]
        fd = (J_at(w0 + eps * dd) - J_at(w0 - eps * dd)) / (2 * eps)
        rec[f"fd_{eps:g}"] = dict(fd=fd, adjoint=an, rel=abs(fd - an) / abs(an))
    s.close()
    _record["fullsize_shock_disc_256_200"] = rec
    _save()
    assert max(r["rel"] for key, r in rec.items() if key.startswith("fd_")) <= 1e-4, rec


def test_adjoint_of_fp32_bulk_run_matches_float64_adjoint():
    """FP32-bulk forward run with float64 checkpoints and the float64 reverse
    sweep, against the float64 run's adjoint: they differ by the float32
    trajectory error.  Bars: objective 1e-5, parameter gradients 1e-4,
    per-field relative L1 of the state gradient 5e-2 (the stretch-component
    gradients depend on strains of 1e-6 that float32 V keeps to ~6 %; their
    max-norm differences reach 8e-2, the others' 6e-3)."""
    from paper_2009_14555_gb300.solver import Solver
    wl = W.perturbed(W.smooth_disc_2d(n=32, steps=20, sigma_y=4e7))
    res = {}
    for prec in ("fp64", "fp32_bulk"):
        s = Solver.from_workload(wl, precision=prec)
        s.set_prim([p.prim for p in wl.patches])
        J, _ = s.adj_forward(20, every=5, material=0)
        g, gp = s.adjoint(None, 1.0, kind=1)
        s.close()
        res[prec] = (J, g.reshape(wl.patches[0].prim.shape), gp)
    J64, g64, p64 = res["fp64"]
    J32, g32, p32 = res["fp32_bulk"]
    emax = field_err(g32, g64)
    el1 = [float(np.abs(g32[f] - g64[f]).sum() / max(np.abs(g64[f]).sum(), 1e-300)) for f in range(g64.shape[0])]
    ep = param_err(p32, p64, (0, 1))
    _record["fp32_bulk_vs_fp64_adjoint_smooth_disc_32_20"] = dict(J64=J64, J32=J32, field_max_err=emax,
                                                                  field_l1_err=el1, param_err=ep)
    _save()
    assert abs(J32 - J64) <= 1e-5 * abs(J64)
    assert max(ep) <= 1e-4, ep
    assert max(el1) <= 5e-2, el1


@pytest.mark.parametrize("case", ["1d", "2d_thinc", "reactive", "sqrt_law", "vanleer_2d_thinc"])
def test_hand_written_reverses_match_dual_numbers(case):
    """The hand-written reverses of the face Riemann problem (all six regions
    of the HLLD-type solver, shear coupling, wave-speed ties), the face-state
    map, the THINC-BVD edge values, the primitive recovery and the source steps
    (plastic return, RK4 reaction with either rate law) give the gradient of the dual-number
    reference to rounding: measured 1e-15 .. 4.4e-10 per field and parameter
    (the larger values in partial-density and shear-modulus gradients, sums
    with cancellation), 2e-9 for the 3e-13 shear-modulus gradient of the
    detonation case; bar max(1e-9, 10 x the reference's one-ulp spread)."""
    from paper_2009_14555_gb300.solver import Solver
    wl, steps, mat = {
        "1d": (W.perturbed(W.solid_gas_1d(n=100, steps=12)), 12, 0),
        "2d_thinc": (W.perturbed(W.shock_disc_2d(n=20, steps=4, thinc=True, shock_x=0.3)), 4, 0),
        "reactive": (W.perturbed(W.reactive_plate_2d(nx=48, ny=24, steps=3)), 3, 1),
        "sqrt_law": (_detonation_partial_burn(), 8, 1),
        "vanleer_2d_thinc": (_vanleer(W.perturbed(W.shock_disc_2d(n=20, steps=4, thinc=True, shock_x=0.3))), 4, 0),
    }[case]
    rng = np.random.default_rng(123)
    p0 = wl.patches[0].prim
    pu = p0 * (1 + np.sign(rng.standard_normal(p0.shape)) * 2.0 ** -52)
    out = []
    for ref, prim in ((False, p0), (True, p0), (True, pu)):
        s = Solver.from_workload(wl)
        s.adj_reference(ref)
        s.set_prim([prim])
        s.adj_forward(steps, every=3, material=mat)
        rng = np.random.default_rng(8)
        out.append(s.adjoint(rng.standard_normal(s.state_numel) * 1e-3, 1.0, kind=1))
        s.close()
    (g, gp), (gr, gpr), (gu, gpu_) = out
    shape = p0.shape

    def perr(a, b):
        return [abs(x - y) / max(abs(y), 1e-300) if y != 0.0 else abs(x) for x, y in zip(a, b)]

    e = field_err(g.reshape(shape), gr.reshape(shape))
    ep = perr(gp, gpr)
    # the reference form's own spread under one-ulp input perturbations: a
    # parameter gradient that is a sum with heavy cancellation (the copper's
    # shear modulus before any wave reaches it, 3e-13) is only that well defined
    bar = [max(1e-9, 10 * x) for x in field_err(gu.reshape(shape), gr.reshape(shape))]
    pbar = [max(1e-9, 10 * x) for x in perr(gpu_, gpr)]
    _record[f"hand_vs_dual_{case}"] = dict(field_err=e, param_err=ep, field_bar=bar, param_bar=pbar)
    _save()
    assert all(x <= b for x, b in zip(e, bar)), (e, bar)
    assert all(x <= b for x, b in zip(ep, pbar)), (ep, pbar)


def test_autograd_function_matches_library_adjoint():
    """torch.autograd through Rollout equals the direct dis_adjoint call for a
    combined objective J + <c, q_final>."""
    from paper_2009_14555_gb300.autograd import rollout
    from paper_2009_14555_gb300.solver import Solver, pack
    wl = W.perturbed(W.smooth_disc_2d(n=16, steps=6, sigma_y=4e7))
    s = Solver.from_workload(wl)
    w0 = torch.tensor(pack([p.prim for p in wl.patches]), device=s.device, requires_grad=True)
    theta = torch.tensor(s.params(), dtype=torch.float64, requires_grad=True)
    c = torch.linspace(-1e-3, 1e-3, s.state_numel, dtype=torch.float64, device=s.device)
    qN, J = rollout(s, w0, theta, 6, every=2, material=0)
    L_ = J + (c * qN).sum()
    L_.backward()
    s2 = Solver.from_workload(wl)
    s2.set_prim([p.prim for p in wl.patches])
    s2.adj_forward(6, every=2, material=0)
    g, gp = s2.adjoint(c.cpu().numpy(), 1.0, kind=1)
    assert np.allclose(w0.grad.cpu().numpy(), g, rtol=1e-12, atol=1e-12 * np.abs(g).max())
    assert np.allclose(theta.grad.numpy(), gp, rtol=1e-10, atol=0)
    s.close()
    s2.close()
