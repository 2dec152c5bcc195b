"""The C ABI library loads on a machine without a GPU, exports every entry
point that include/dis.h declares, and validates its arguments on the host."""
import ctypes
import os
import re

import pytest

from paper_2009_14555_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_names():
    hdr = open(os.path.join(ROOT, "include", "dis.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(dis_[a-z0-9_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(L.LIB_PATH):
        from paper_2009_14555_gb300 import build
        build.build()
    return L.load()


def test_exports_every_declared_symbol(lib):
    names = header_names()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(L.SIGNATURES), set(names) - set(L.SIGNATURES)


def _patch(nx=16, ny=1):
    return L.DisPatch(nx, ny, 1.0 / nx, 1.0, (ctypes.c_int32 * 4)(0, 0, 0, 0))


def test_create_validates_arguments(lib):
    out = ctypes.c_void_p()
    opts = L.DisOptions(0.8, 0, 0)
    arr = (L.DisPatch * 1)(_patch())
    assert lib.dis_create(3, 1, arr, -1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_EINVAL
    assert b"dim" in lib.dis_last_error()
    bad = L.DisOptions(1.5, 0, 0)
    assert lib.dis_create(1, 1, arr, -1, ctypes.byref(bad), None, ctypes.byref(out)) == L.DIS_EINVAL
    tiny = (L.DisPatch * 1)(_patch(nx=2))
    assert lib.dis_create(1, 1, tiny, -1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_EINVAL
    assert lib.dis_create(1, 0, arr, -1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_EINVAL
    assert lib.dis_create(1, 1, arr, 2, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_EINVAL
    unknown = L.DisOptions(0.8, 0, 0, 7)
    assert lib.dis_create(1, 1, arr, -1, ctypes.byref(unknown), None, ctypes.byref(out)) == L.DIS_EINVAL
    assert b"scheme" in lib.dis_last_error()
    geo = L.DisOptions(0.8, 0, 0, 0, 5)
    assert lib.dis_create(1, 1, arr, -1, ctypes.byref(geo), None, ctypes.byref(out)) == L.DIS_EINVAL
    assert b"geometry" in lib.dis_last_error()
    cyl_h = L.DisOptions(0.8, 0, L.DIS_FP64, L.DIS_HANCOCK, L.DIS_CYLINDRICAL)
    assert lib.dis_create(1, 1, arr, -1, ctypes.byref(cyl_h), None, ctypes.byref(out)) == L.DIS_EINVAL
    cyl = L.DisOptions(0.8, 0, L.DIS_FP64, L.DIS_RK3, L.DIS_CYLINDRICAL)
    neg = (L.DisPatch * 1)(L.DisPatch(16, 1, 1.0 / 16, 1.0, (ctypes.c_int32 * 4)(2, 0, 0, 0), -0.5))
    assert lib.dis_create(1, 1, neg, -1, ctypes.byref(cyl), None, ctypes.byref(out)) == L.DIS_EINVAL
    assert b"x0" in lib.dis_last_error()
    assert lib.dis_create(1, 1, arr, -1, ctypes.byref(cyl), None, ctypes.byref(out)) == L.DIS_OK
    lib.dis_destroy(out)
    cyl_h32 = L.DisOptions(0.8, 0, L.DIS_FP32_BULK, L.DIS_HANCOCK, L.DIS_CYLINDRICAL)
    assert lib.dis_create(1, 1, arr, -1, ctypes.byref(cyl_h32), None, ctypes.byref(out)) == L.DIS_EINVAL
    assert b"cylindrical" in lib.dis_last_error()


def test_hancock_workspace_holds_the_evolved_edge_states(lib):
    """A MUSCL-Hancock context adds 2 x dim x nf planes of the padded cells."""
    out = ctypes.c_void_p()
    arr = (L.DisPatch * 1)(_patch(100))
    sizes = []
    for scheme in (L.DIS_RK3, L.DIS_HANCOCK):
        opts = L.DisOptions(0.8, 0, L.DIS_FP64, scheme)
        assert lib.dis_create(1, 1, arr, -1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_OK
        sizes.append(lib.dis_workspace_bytes(out))
        lib.dis_destroy(out)
    T = (100 + 6 + 31) // 32 * 32
    assert sizes[1] - sizes[0] >= 2 * 1 * 8 * 8 * T


def test_fp32_hancock_workspace_holds_two_state_buffers(lib):
    """FP32-bulk MUSCL-Hancock alternates two state buffers of nf + 1 float
    planes (the Runge-Kutta form holds three)."""
    out = ctypes.c_void_p()
    arr = (L.DisPatch * 1)(_patch(1000))
    sizes = []
    for scheme in (L.DIS_RK3, L.DIS_HANCOCK):
        opts = L.DisOptions(0.8, 0, L.DIS_FP32_BULK, scheme)
        assert lib.dis_create(1, 1, arr, -1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_OK
        sizes.append(lib.dis_workspace_bytes(out))
        lib.dis_destroy(out)
    T = (1000 + 6 + 31) // 32 * 32
    assert sizes[0] - sizes[1] >= 4 * 9 * T


def test_host_side_sizes_and_materials(lib):
    out = ctypes.c_void_p()
    opts = L.DisOptions(0.8, 0, 0)
    arr = (L.DisPatch * 2)(_patch(100), _patch(37))
    assert lib.dis_create(1, 2, arr, -1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_OK
    ctx = out
    assert lib.dis_state_bytes(ctx, 0) == 8 * 8 * 137
    ws = lib.dis_workspace_bytes(ctx)
    assert ws > 3 * 8 * 8 * 137
    gas = L.DisMaterial(1.4, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)
    bad = L.DisMaterial(0.9, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(gas, bad), 2) == L.DIS_EINVAL
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(gas, gas), 1) == L.DIS_EINVAL
    rx = L.DisMaterial(1.4, 0, 0, 0, 0, 0, 0, 1, 1e6, 717.5, 1e7, 4000)
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(gas, rx), 2) == L.DIS_EINVAL  # ctx not reactive
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(gas, gas), 2) == L.DIS_OK
    # stepping before a state exists is refused on the host
    assert lib.dis_step(ctx, 1, None) == L.DIS_ESTATE
    lib.dis_destroy(ctx)


def test_rate_law_validation(lib):
    out = ctypes.c_void_p()
    opts = L.DisOptions(0.9, 0, 0)
    arr = (L.DisPatch * 1)(_patch(64))
    assert lib.dis_create(1, 1, arr, 1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_OK
    ctx = out
    gas = L.DisMaterial(1.4, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)

    def rx(law, p_ign=1e8, A=2e6):
        return L.DisMaterial(3.0, 0, 0, 0, 0, 0, 0, 1, 4e6, 1000.0, A, 0.0, law, p_ign)

    for bad in (rx(2), rx(-1), rx(1, p_ign=float("nan")), rx(1, A=-1.0), rx(1, A=float("inf"))):
        assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(gas, bad), 2) == L.DIS_EINVAL
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(gas, rx(L.DIS_RATE_SQRT)), 2) == L.DIS_OK
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(gas, rx(L.DIS_RATE_ARRHENIUS)), 2) == L.DIS_OK
    lib.dis_destroy(ctx)


def test_johnson_cook_validation(lib):
    """Johnson-Cook plasticity: the history-row material must be the
    Johnson-Cook one, a Romenskii solid with positive rates and exponents and
    T_melt > T0; not reactive; float64 contexts only."""
    from paper_2009_14555_gb300 import workloads as W
    from paper_2009_14555_gb300.solver import _material
    air = _material(W.material(1.4))
    cu = W.COPPER_JC

    def ctx_of(row, precision=0):
        out = ctypes.c_void_p()
        opts = L.DisOptions(0.6, 0, precision)
        arr = (L.DisPatch * 1)(_patch(64))
        assert lib.dis_create(1, 1, arr, row, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_OK
        return out

    ctx = ctx_of(0)
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(_material(cu), air), 2) == L.DIS_OK
    for key, val in (("jc_c3", 0.0), ("jc_n", 0.0), ("jc_m", -1.0), ("chi0", 0.0), ("cv", 0.0),
                     ("jc_Tmelt", 298.0), ("jc_Tmelt", float("inf")), ("jc_c2", -1.0), ("sigma_y", -1.0)):
        assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(_material(dict(cu, **{key: val})), air), 2) \
            == L.DIS_EINVAL, key
    sg = W.material(3.0, p_inf=4.55e10, G=39.4e9)
    sg.update({k: v for k, v in cu.items() if k.startswith("jc_") or k in ("plastic", "sigma_y", "chi0", "cv")})
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(_material(sg), air), 2) == L.DIS_EINVAL
    rx = dict(cu, reactive=1, Q=1e6, cv=385.0)
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(_material(rx), air), 2) == L.DIS_EINVAL
    lib.dis_destroy(ctx)
    for row in (-1, 1):  # the Johnson-Cook material does not carry the row
        ctx = ctx_of(row)
        assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(_material(cu), air), 2) == L.DIS_EINVAL
        lib.dis_destroy(ctx)
    ctx = ctx_of(0, precision=L.DIS_FP32_BULK)
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(_material(cu), air), 2) == L.DIS_EINVAL
    lib.dis_destroy(ctx)


def test_amr_create_validates_arguments(lib):
    """dis_amr_create: float64, SSP-RK3 (planar or cylindrical with x0 >= 0)
    or MUSCL-Hancock (planar), levels 1..4, block >= 4 dividing the domain,
    known boundary kinds (no device work here)."""
    out = ctypes.c_void_p()
    dom = L.DisPatch(64, 1, 1.0 / 64, 1.0, (ctypes.c_int32 * 4)(0, 0, 0, 0))
    opts = L.DisOptions(0.8, 0, L.DIS_FP64, L.DIS_RK3)
    ok = L.DisAmrOptions(3, 8, 0.1, 2, 1.0, 4)
    assert lib.dis_amr_create(1, ctypes.byref(dom), -1, ctypes.byref(opts), ctypes.byref(ok), None,
                              ctypes.byref(out)) == L.DIS_OK
    lib.dis_amr_destroy(out)
    for bad in (L.DisAmrOptions(5, 8, 0.1, 2, 1.0, 4), L.DisAmrOptions(0, 8, 0.1, 2, 1.0, 4),
                L.DisAmrOptions(2, 3, 0.1, 2, 1.0, 4), L.DisAmrOptions(2, 24, 0.1, 2, 1.0, 4),
                L.DisAmrOptions(2, 8, 0.1, -1, 1.0, 4)):
        assert lib.dis_amr_create(1, ctypes.byref(dom), -1, ctypes.byref(opts), ctypes.byref(bad), None,
                                  ctypes.byref(out)) == L.DIS_EINVAL
    hk = L.DisOptions(0.8, 0, L.DIS_FP64, L.DIS_HANCOCK)
    assert lib.dis_amr_create(1, ctypes.byref(dom), -1, ctypes.byref(hk), ctypes.byref(ok), None,
                              ctypes.byref(out)) == L.DIS_OK
    lib.dis_amr_destroy(out)
    for o in (L.DisOptions(0.8, 0, L.DIS_FP32_BULK, L.DIS_RK3), L.DisOptions(0.8, 0, L.DIS_FP64, 5),
              L.DisOptions(0.8, 0, L.DIS_FP64, L.DIS_RK3, 7),
              L.DisOptions(0.8, 0, L.DIS_FP64, L.DIS_HANCOCK, L.DIS_CYLINDRICAL)):
        assert lib.dis_amr_create(1, ctypes.byref(dom), -1, ctypes.byref(o), ctypes.byref(ok), None,
                                  ctypes.byref(out)) == L.DIS_EINVAL
    cyl = L.DisOptions(0.8, 0, L.DIS_FP64, L.DIS_RK3, L.DIS_CYLINDRICAL)
    axis = L.DisPatch(64, 1, 1.0 / 64, 1.0, (ctypes.c_int32 * 4)(L.DIS_BC_REFLECTIVE, 0, 0, 0), 0.0)
    assert lib.dis_amr_create(1, ctypes.byref(axis), -1, ctypes.byref(cyl), ctypes.byref(ok), None,
                              ctypes.byref(out)) == L.DIS_OK
    lib.dis_amr_destroy(out)
    neg = L.DisPatch(64, 1, 1.0 / 64, 1.0, (ctypes.c_int32 * 4)(0, 0, 0, 0), -0.5)
    assert lib.dis_amr_create(1, ctypes.byref(neg), -1, ctypes.byref(cyl), ctypes.byref(ok), None,
                              ctypes.byref(out)) == L.DIS_EINVAL
    assert b"radius" in lib.dis_last_error()
    ext = L.DisPatch(64, 1, 1.0 / 64, 1.0, (ctypes.c_int32 * 4)(L.DIS_BC_EXTERNAL, 0, 0, 0))
    assert lib.dis_amr_create(1, ctypes.byref(ext), -1, ctypes.byref(opts), ctypes.byref(ok), None,
                              ctypes.byref(out)) == L.DIS_EINVAL
    # the external kind is internal to the hierarchy's levels
    arr = (L.DisPatch * 1)(ext)
    assert lib.dis_create(1, 1, arr, -1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_EINVAL
    assert lib.dis_amr_step(None, 1, None) == L.DIS_EINVAL


def test_amr_solver_refuses_without_a_gpu():
    """No CPU fallback: the Python hierarchy needs a CUDA device."""
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2009_14555_gb300 import workloads as W
    from paper_2009_14555_gb300.solver import AmrSolver
    with pytest.raises(RuntimeError):
        AmrSolver(W.solid_gas_1d(64, steps=1))


def test_allocation_and_workspace_failures_are_reported(lib):
    """Fault injection on the host: a caller's workspace one byte too small
    (DIS_ENOMEM), a misaligned one (DIS_EINVAL), and a failed device
    allocation (the machine without a GPU makes cudaMalloc fail: DIS_ENOMEM
    with the CUDA text).  The context stays usable: nothing was loaded, a
    step is refused as out of order, and it is destroyed cleanly."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the device allocation would succeed")
    out = ctypes.c_void_p()
    opts = L.DisOptions(0.8, 0, 0)
    arr = (L.DisPatch * 1)(_patch(64))
    assert lib.dis_create(1, 1, arr, -1, ctypes.byref(opts), None, ctypes.byref(out)) == L.DIS_OK
    ctx = out
    gas = L.DisMaterial(1.4, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)
    assert lib.dis_set_materials(ctx, (L.DisMaterial * 2)(gas, gas), 2) == L.DIS_OK
    need = lib.dis_workspace_bytes(ctx)
    # the pointers are never dereferenced: the size and alignment checks come first
    assert lib.dis_bind_workspace(ctx, ctypes.c_void_p(1 << 20), need - 1) == L.DIS_ENOMEM
    assert b"needed" in lib.dis_last_error()
    assert lib.dis_bind_workspace(ctx, ctypes.c_void_p((1 << 20) + 8), need) == L.DIS_EINVAL
    prim = np.zeros((8, 1, 64))
    prim[0], prim[1], prim[2], prim[4] = 0.5, 1.2, 1.2, 1e5
    prim[5:8] = 1.0
    assert lib.dis_set_state(ctx, L.DIS_PRIMITIVE, ctypes.c_void_p(prim.ctypes.data), 0) == L.DIS_ENOMEM
    assert b"cannot allocate" in lib.dis_last_error()
    assert lib.dis_step(ctx, 1, None) == L.DIS_ESTATE
    lib.dis_destroy(ctx)
