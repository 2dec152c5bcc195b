"""The k sqrt(lam) reaction law with its pressure switch (Section 4.1) on the
GPU against the float64 oracle, on the shape of the paper's one-dimensional
detonation test (booster-initiated detonation running into elastic copper,
stand-in stiffened-gas closures).

FP64: bar 1e-10 (per-field relative L1 and dt) over the first 30 steps; over
140 steps, through the detonation's arrival at the copper, max(1e-10, 10 x
the oracle's own one-ulp spread).  FP32-bulk: the float32 bars of the
FP32-bulk tests.  The adjoint cases are in tests/test_adjoint_gpu.py.
"""
import numpy as np
import pytest

from paper_2009_14555_gb300 import workloads as W
from tests.parity_util import oracle_prim, oracle_run
from tests.test_fp32_bulk_gpu import check32
from tests.test_parity_gpu import assert_parity, gpu_run

pytestmark = pytest.mark.gpu


def test_detonation_fp64_strict():
    assert_parity(W.detonation_copper_1d(200, steps=30), 30)


def test_detonation_fp64_into_copper():
    assert_parity(W.detonation_copper_1d(200, steps=140), 140, calibrate=True)


def test_detonation_burns_and_reaches_copper():
    """The GPU run itself: the booster initiates a detonation near the
    ideal-gas Chapman-Jouguet pressure rho0 D^2 / (gamma + 1), D^2 =
    2 (gamma^2 - 1) Q (2.4e10 Pa here), the burnt region has lam = 0 exactly
    (the clamp), and the copper ahead is shocked."""
    wl = W.detonation_copper_1d(200, steps=140)
    _, prim, _ = gpu_run(wl, 140)
    names = W.prim_names(1, True)
    w = prim[0][:, 0]
    lam, p = w[names.index("lam")], w[names.index("p")]
    x = (np.arange(200) + 0.5) * 0.002
    assert (lam[x > 0.2] == 0.0).all()
    assert p[x < 0.15].max() > 1e10
    o, _ = oracle_run(wl, 140)
    op = oracle_prim(wl, o)[0][:, 0]
    # the burnt cells are the oracle's (a cell whose last burning step ends
    # within rounding of lam = 0 may fall either side of the clamp)
    assert ((lam == 0.0) != (op[names.index("lam")] == 0.0)).sum() <= 1


def test_detonation_fp32_bulk():
    check32("1d_detonation_copper_200_60", W.detonation_copper_1d(200, steps=60), 60)
