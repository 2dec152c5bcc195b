"""The detonation-into-copper workload against the values the paper prints
for its one-dimensional test (Section 4.1) and the tables of constants it
uses (tests/golden/detonation_1d_section_4_1.txt).  The copper and the
explosive are stand-ins (a stiffened gas with the Romenskii table's rho_0,
K_0, G_0 and Gamma; one ideal gas for reactant and product with the
product's constants), so the check is on the numbers the stand-ins take from
the paper."""
import os

import numpy as np

from paper_2009_14555_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "detonation_1d_section_4_1.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (s.strip() for s in line.split("=", 1))
                out[k] = float(v)
    return out


def test_detonation_workload_takes_the_printed_values():
    g = _golden()
    n = int(g["cells"])
    wl = W.detonation_copper_1d(n)
    p = wl.patches[0]
    assert p.nx == n and abs(p.nx * p.dx - g["domain_length_m"]) < 1e-15
    assert wl.cfl == g["cfl"]
    copper, expl = wl.materials
    # copper: the Romenskii solid of the table (Gamma = gamma - 1)
    assert copper["eos"] == "romenskii"
    assert abs((copper["gamma"] - 1.0) - g["copper_Gamma"]) < 1e-15
    assert copper["K0"] == g["copper_K0_pa"] and copper["rho0"] == g["copper_rho0"]
    assert copper["alpha_r"] == g["copper_alpha"] and copper["beta_r"] == g["copper_beta"]
    assert copper["G"] == g["copper_G0_pa"] and copper["plastic"] == 0
    # the stiffened stand-in keeps the bulk modulus gamma p_inf = K0
    cs = W.detonation_copper_1d(n, copper="stiffened").materials[0]
    assert abs(cs["gamma"] * cs["p_inf"] - g["copper_K0_pa"]) < 1e-3
    # explosive: the product's constants, the k sqrt(lam) law and its switch
    assert expl["gamma"] == g["explosive_product_gamma"]
    assert expl["cv"] == g["explosive_product_cv"]
    assert expl["Q"] == g["explosive_product_Q"]
    assert expl["rate_law"] == 1 and expl["A"] == g["rate_k_per_s"]
    assert expl["p_ign"] == g["switch_pressure_pa"]
    names = W.prim_names(1, True)
    w = p.prim[:, 0]
    x = (np.arange(n) + 0.5) * p.dx
    cu = x < g["copper_right_m"]
    assert (w[names.index("phi1")][cu] > 0.99).all() and (w[names.index("phi1")][~cu] < 0.01).all()
    assert (w[names.index("rho1")] == g["copper_rho0"]).all()
    assert (w[names.index("rho2")] == g["explosive_reactant_rho0"]).all()
    pr = w[names.index("p")]
    boost = x > g["booster_left_m"]
    assert (pr[boost] == g["booster_pressure_pa"]).all() and (pr[~boost] == g["ambient_pressure_pa"]).all()
    assert (w[names.index("lam")] == 1.0).all() and (w[names.index("u")] == 0.0).all()
