"""Cylindrical (axisymmetric, x = r, y = z) geometry on the GPU against the
oracle's operator with the Section 3 geometric source, through the C ABI:
float64 at the 1e-10 parity bar (THINC next to the stiff solid: the
self-calibrated bar of tests/test_parity_gpu.py), FP32-bulk at the float32
bars of tests/test_fp32_bulk_gpu.py."""
import numpy as np
import pytest

from paper_2009_14555_gb300 import workloads as W
from tests.parity_util import cons_l1, oracle_run
from tests.test_fp32_bulk_gpu import TOL32, TOL32_PARTIAL, check32
from tests.test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


def test_1d_cylinder_core_implosion():
    assert_parity(W.cylinder_core_1d(300, steps=100), 100)


def test_1d_off_axis_annulus():
    """A patch that does not touch the axis (x0 = 0.5): r from 0.5 to 1.5."""
    assert_parity(W.cylinder_core_1d(200, steps=60, r_core=0.8, x0=0.5), 60)


def test_2d_sphere_shock():
    wl = W.sphere_shock_rz(48, steps=30)
    wl.thinc = False
    assert_parity(wl, 30)


def test_2d_sphere_shock_thinc():
    assert_parity(W.sphere_shock_rz(48, steps=30), 30, calibrate=True)


def test_fp32_cylindrical():
    check32("1d_cylinder_core_300_100steps", W.cylinder_core_1d(300, steps=100), 100)
    wl = W.sphere_shock_rz(48, steps=30)
    wl.thinc = False
    check32("2d_sphere_shock_rz_48_30steps", wl, 30)


def test_homologous_expansion_doubles_the_density_rate():
    """u_r = a r in a uniform gas: the cylindrical continuity equation gives
    d rho / dt = -2 a rho, the planar one -a rho; after a few steps the GPU
    runs show that factor 2 (guards against a silently ignored geometry), and
    the cylindrical run matches the oracle."""
    from tests.test_parity_gpu import gpu_run
    n, a = 100, 40.0
    wl = W.cylinder_core_1d(n, steps=5, r_core=-1.0, x0=0.2)
    prim = wl.patches[0].prim
    rc = 0.2 + (np.arange(n) + 0.5) / n
    prim[0, 0], prim[1, 0], prim[2, 0], prim[3, 0], prim[4, 0] = 1e-8, 1.2, 1.2, a * rc, 1e5
    wl.patches[0].bc = (W.BC_TRANSMISSIVE,) * 4
    g_cyl, _, _ = gpu_run(wl, 5)
    o, _ = oracle_run(wl, 5)
    assert cons_l1(wl, g_cyl[0], o[0]).max() <= 1e-10
    wl.geometry = "planar"
    g_pl, _, _ = gpu_run(wl, 5)
    rho0 = 1.2
    inner = slice(10, n - 10)
    d_cyl = (g_cyl[0][1, 0, inner] + g_cyl[0][2, 0, inner]) - rho0
    d_pl = (g_pl[0][1, 0, inner] + g_pl[0][2, 0, inner]) - rho0
    ratio = d_cyl.mean() / d_pl.mean()
    assert 1.9 < ratio < 2.1, ratio
