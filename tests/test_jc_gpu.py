"""Johnson-Cook plasticity (Section 2.3.2, relaxed as in Section 3.2) on the
GPU against the float64 oracle through the C ABI, at the parity bar
(per-field relative L1 1e-10, element-wise 1e-8; the oracle's one-ulp spread
on these cases is below 3e-13):

  * the copper plate impact (Romenskii copper with the Johnson-Cook table),
    Runge-Kutta and MUSCL-Hancock forms;
  * the shock-driven hemispherical indentation of Section 4.4 in (r, z);
  * the plate impact on the AMR hierarchy (three levels);
  * FP32-bulk contexts and the adjoint refuse Johnson-Cook materials (the
    parameter checks run on the host: tests/test_abi.py).
"""
import pytest

from paper_2009_14555_gb300 import workloads as W
from tests.test_amr_gpu import compare as amr_compare
from tests.test_parity_gpu import assert_parity

pytestmark = pytest.mark.gpu


def test_jc_flyer_1d_fp64():
    assert_parity(W.jc_flyer_1d(200, steps=120), 120)


def test_jc_flyer_1d_hancock_fp64():
    wl = W.jc_flyer_1d(200, steps=120, name="1d_jc_flyer_hancock_200")
    wl.scheme = "hancock"
    assert_parity(wl, 120)


def test_jc_indentation_rz_fp64():
    """The shock from the driven base reaches the indentation (100 steps on
    24 x 120 cells)."""
    assert_parity(W.indentation_rz(24, steps=100), 100)


def test_jc_flyer_amr_three_levels():
    amr_compare(W.jc_flyer_1d(128, steps=24), 24, "amr_jc_flyer_128_3levels_24", max_level=3, block=8,
                eps=0.05, regrid_every=2)


def test_jc_refusals():
    from paper_2009_14555_gb300.solver import Solver
    wl = W.jc_flyer_1d(64, steps=2)
    with pytest.raises(RuntimeError):
        Solver.from_workload(wl, precision="fp32_bulk")
    s = Solver.from_workload(wl)
    s.set_prim([wl.patches[0].prim])
    with pytest.raises(RuntimeError):
        s.adj_forward(2, every=1, material=0)
    s.close()
