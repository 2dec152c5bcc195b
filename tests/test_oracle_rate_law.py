"""Pins of the oracle's k sqrt(lam) reaction law (Section 4.1: the reactant
fraction burns at lam_dot = -k sqrt(lam) once the pressure exceeds a switch
value; integrated by RK4 in the reactive step of Section 3.3).

  * closed form: with the switch on, sqrt(lam(t)) = sqrt(lam0) - k t / 2, so
    lam(t) = (sqrt(lam0) - k t / 2)^2 until burn-out; the RK4 steps reach it
    at fourth order, in a cell whose reactive material has phi_y rho_y != 1
    (the rate of phi_y rho_y lam carries the factor phi_y rho_y);
  * burn-out: a step that passes lam = 0 ends at exactly 0, and lam stays 0;
  * the switch: below p_ign nothing changes, above it the closed form holds;
  * only phi_y rho_y lam changes: densities, momentum, energy, V unchanged.
"""
import math

import torch

from oracle import closures as C
from oracle import scheme as S
from paper_2009_14555_gb300 import workloads as W

F64 = torch.float64
GAS = W.material(1.4)
K = 2e6


def _explosive(p_ign=1e8):
    return W.material(3.0, reactive=1, Q=4e6, cv=1000.0, A=K, rate_law=1, p_ign=p_ign)


def _cell(p, lam, phi_y=0.7, rho_y=1600.0):
    """One cell: inert air (material 1) and the explosive (material 2)."""
    t = lambda v: torch.tensor([v], dtype=F64)  # noqa: E731
    w = dict(phi1=t(1.0 - phi_y), rho1=t(1.2), rho2=t(rho_y), u=torch.zeros(1, 3, dtype=F64),
             p=t(p), V=torch.eye(3, dtype=F64)[None], lam=t(lam))
    return w


def _lam(q):
    return (q["arl"] / q["ar2"]).item()


def test_closed_form_fourth_order():
    mats = [GAS, _explosive()]
    q0 = C.prim_to_cons(_cell(1e9, 0.81), mats)
    T_end = 0.6 / K  # sqrt(lam) falls from 0.9 to 0.6
    exact = (0.9 - K * T_end / 2) ** 2
    errs = []
    for m in (4, 8, 16):
        q = dict(q0)
        for _ in range(m):
            q = S.reaction_update(q, mats, T_end / m)
        errs.append(abs(_lam(q) - exact))
    assert errs[2] < 1e-8  # measured 4.3e-9; halving dt divides it by 16
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20


def test_burn_out_clamps_at_zero():
    mats = [GAS, _explosive()]
    q = C.prim_to_cons(_cell(1e9, 0.01), mats)
    dt = 0.5 / K  # one step would take sqrt(lam) from 0.1 to 0.1 - 0.25
    q = S.reaction_update(q, mats, dt)
    assert q["arl"].item() == 0.0
    q = S.reaction_update(q, mats, dt)
    assert q["arl"].item() == 0.0


def test_pressure_switch():
    mats = [GAS, _explosive(p_ign=1e8)]
    q0 = C.prim_to_cons(_cell(5e7, 1.0), mats)
    q = S.reaction_update(q0, mats, 0.1 / K)
    assert torch.equal(q["arl"], q0["arl"])
    # heat release only raises the pressure, so a cell above the switch stays
    # above it: the closed form holds
    q1 = C.prim_to_cons(_cell(2e8, 1.0), mats)
    dt = 0.05 / K
    q = dict(q1)
    for _ in range(4):
        q = S.reaction_update(q, mats, dt)
    assert abs(_lam(q) - (1.0 - K * 4 * dt / 2) ** 2) < 1e-8  # RK4 error 2.3e-9


def test_only_reactant_mass_changes():
    mats = [GAS, _explosive()]
    q0 = C.prim_to_cons(_cell(1e9, 0.5), mats)
    q = S.reaction_update(q0, mats, 0.2 / K)
    for k in q0:
        if k != "arl":
            assert torch.equal(q[k], q0[k]), k
    assert _lam(q) < 0.5
