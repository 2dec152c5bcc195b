"""The Romenskii and JWL closure families of Section 2.3 on the GPU, against
the float64 oracle through the C ABI: float64 at the parity bar (per-field
relative L1 1e-10, element-wise 1e-8; THINC cases calibrated by the
oracle's one-ulp spread), FP32-bulk at its float32 bars.

Cases: Romenskii copper (the table of Section 4.1) striking air at 500 m/s
(1D), an elastoplastic Romenskii copper disc struck by a Mach-2 air shock
(2D; yield stress 0.4 GPa as in the rate-stick confiner of Section 4.2), and
an LX-17 reactant on the JWL form (inert) expanding into air.
"""

import numpy as np
import pytest

from paper_2009_14555_gb300 import workloads as W
from tests.test_fp32_bulk_gpu import check32
from tests.test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu

CU = W.COPPER_ROMENSKII
LX = W.LX17_REACTANT_JWL


def _copper_air_1d(n=400, steps=100):
    return W.riemann_1d(n, dict(mat=0, rho=8930.0, u=500.0, p=1e5), dict(mat=1, rho=1.2, u=0.0, p=1e5),
                        materials=[CU, W.AIR], steps=steps, name=f"1d_romenskii_copper_air_{n}")


def _copper_disc_2d(n=40, steps=30, thinc=False):
    wl = W.shock_disc_2d(n, steps=steps, thinc=thinc, shock_x=0.28)
    cu = dict(CU, plastic=1, sigma_y=0.4e9)
    wl.materials = [cu, W.AIR]
    k = W.prim_names(2, False).index("rho1")
    for p in wl.patches:
        p.prim[k] = 8930.0
    wl.name = f"2d_romenskii_disc_{n}" + ("_thinc" if thinc else "")
    return wl


def _jwl_air_1d(n=300, steps=60):
    return W.riemann_1d(n, dict(mat=0, rho=1905.0, u=0.0, p=1e9), dict(mat=1, rho=1.2, u=0.0, p=1e5),
                        materials=[LX, W.AIR], steps=steps, name=f"1d_jwl_lx17_air_{n}")


def test_romenskii_copper_air_1d_fp64():
    assert_parity(_copper_air_1d(), 100)


def test_romenskii_copper_disc_2d_fp64():
    assert_parity(_copper_disc_2d(), 30)


def test_romenskii_copper_disc_2d_thinc_fp64():
    assert_parity(_copper_disc_2d(thinc=True), 30, calibrate=True)


def test_jwl_air_1d_fp64():
    assert_parity(_jwl_air_1d(), 60)


def test_romenskii_copper_air_1d_fp32_bulk():
    check32("1d_romenskii_copper_air_400_100", _copper_air_1d(), 100)


def test_romenskii_copper_disc_2d_fp32_bulk():
    check32("2d_romenskii_disc_40_30", _copper_disc_2d(), 30)


def test_jwl_air_1d_fp32_bulk():
    check32("1d_jwl_lx17_air_300_60", _jwl_air_1d(), 60)


def test_eos_families_hancock_fp64():
    wl = _copper_air_1d(300, 40)
    wl.scheme = "hancock"
    assert_parity(wl, 40, name="1d_romenskii_copper_air_hancock_300_40")


def test_adjoint_refuses_jwl_and_cylindrical_romenskii():
    """The adjoint covers Romenskii solids in planar geometry (their reverse
    by dual numbers, tests/test_adjoint_gpu.py); JWL materials and
    cylindrical Romenskii contexts are refused."""
    from paper_2009_14555_gb300.solver import Solver
    for wl in (_jwl_air_1d(64, 2), _copper_air_1d(64, 2)):
        if wl.materials[0] is CU:
            wl.geometry = "cyl"
        s = Solver.from_workload(wl)
        s.set_prim([wl.patches[0].prim])
        with pytest.raises(RuntimeError):
            s.adj_forward(2, every=1, material=0)
        s.close()


def test_no_alloc_cfl_dt_on_romenskii_state():
    """The allocation-free CFL entry point reads the same closures."""
    from tests.test_zz_no_alloc import reference, static_dt
    wl = _copper_disc_2d(48, 1)
    cons, ref = reference(wl)
    np.testing.assert_allclose(static_dt(wl, cons), ref, rtol=1e-12)


# ---- the generic explosive: reactant and product closures of their own,
# ---- component densities from the temperature equality (Appendix B)
def _generic_detonation(n=200, steps=30):
    return W.detonation_copper_1d(n, steps=steps, explosive="generic",
                                  name=f"1d_detonation_generic_explosive_{n}")


def test_generic_explosive_detonation_fp64():
    """Section 4.1's test with the table's explosive and Romenskii copper:
    booster ignition and the detonation's first 30 steps, strict bar."""
    assert_parity(_generic_detonation(), 30)


def test_generic_explosive_detonation_to_the_copper_fp64():
    """150 steps: the detonation runs into the copper (bar 1e-10 or 10x the
    oracle's one-ulp spread).  Where the detonation meets the copper (steps
    55-70) a discrete choice of the scheme flips under round-off: one-ulp
    perturbations of the input move the oracle's own energy field by
    3e-10 ... 5e-8 (relative L1) depending on the perturbation drawn, so the
    spread is the largest over six perturbations."""
    assert_parity(_generic_detonation(200, 150), 150, calibrate=True, seeds=range(100, 106))


def test_generic_explosive_refused_in_fp32_bulk_and_adjoint():
    from paper_2009_14555_gb300.solver import Solver
    wl = _generic_detonation(64, 2)
    with pytest.raises(RuntimeError):
        Solver.from_workload(wl, precision="fp32_bulk")
    s = Solver.from_workload(wl)
    s.set_prim([wl.patches[0].prim])
    with pytest.raises(RuntimeError):
        s.adj_forward(2, every=1, material=0)
    s.close()
