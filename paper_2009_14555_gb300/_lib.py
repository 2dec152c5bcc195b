"""ctypes binding of libdis.so (the C ABI of include/dis.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_longlong, c_size_t, c_void_p, c_char_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdis.so")

DIS_OK, DIS_EINVAL, DIS_ENOMEM, DIS_ECUDA, DIS_ENONPHYSICAL, DIS_ESTATE = 0, -1, -2, -3, -4, -5
DIS_CONSERVATIVE, DIS_PRIMITIVE = 0, 1
DIS_FP64, DIS_FP32_BULK = 0, 1
DIS_RK3, DIS_HANCOCK = 0, 1
DIS_MINMOD, DIS_VANLEER = 0, 1
DIS_EOS_STIFFENED, DIS_EOS_ROMENSKII, DIS_EOS_JWL = 0, 1, 2
DIS_PLANAR, DIS_CYLINDRICAL = 0, 1
DIS_RATE_ARRHENIUS, DIS_RATE_SQRT = 0, 1
DIS_NPARAM = 6  # per material l: G, sigma_y, Q at 3 l + k
DIS_BC_TRANSMISSIVE, DIS_BC_PERIODIC, DIS_BC_REFLECTIVE, DIS_BC_EXTERNAL = 0, 1, 2, 3
DIS_NVARIANTS = 6  # FP32-bulk stage variants: 3 tile shapes x 2 register budgets


class DisStats(ctypes.Structure):
    _fields_ = [("mass", c_double * 2), ("momentum", c_double * 2), ("energy", c_double),
                ("reactant", c_double), ("phi_min", c_double), ("phi_max", c_double),
                ("dt_min", c_double), ("dt_max", c_double), ("kernel_ms", c_double), ("bytes", c_double),
                ("steps", c_longlong), ("launches", c_longlong), ("status", c_int32),
                ("bad_patch", c_int32), ("bad_cell", c_int32)]


class DisMaterial(ctypes.Structure):
    _fields_ = [("gamma", c_double), ("p_inf", c_double), ("e_inf", c_double), ("G", c_double),
                ("plastic", c_int32), ("sigma_y", c_double), ("chi0", c_double),
                ("reactive", c_int32), ("Q", c_double), ("cv", c_double), ("A", c_double),
                ("T_act", c_double), ("rate_law", c_int32), ("p_ign", c_double), ("eos", c_int32),
                ("rho0", c_double), ("K0", c_double), ("alpha", c_double), ("beta", c_double),
                ("jwl_A", c_double), ("jwl_B", c_double), ("jwl_R1", c_double), ("jwl_R2", c_double),
                ("prod_gamma", c_double), ("prod_p_inf", c_double), ("prod_cv", c_double),
                ("jc_c2", c_double), ("jc_c3", c_double), ("jc_n", c_double), ("jc_m", c_double),
                ("jc_Tmelt", c_double), ("jc_T0", c_double)]


class DisPatch(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("dx", c_double), ("dy", c_double),
                ("bc", c_int32 * 4), ("x0", c_double)]


class DisOptions(ctypes.Structure):
    _fields_ = [("cfl", c_double), ("thinc", c_int32), ("precision", c_int32), ("scheme", c_int32),
                ("geometry", c_int32), ("limiter", c_int32)]


class DisAmrOptions(ctypes.Structure):
    _fields_ = [("max_levels", c_int32), ("block", c_int32), ("eps", c_double), ("buffer", c_int32),
                ("u_floor", c_double), ("regrid_every", c_int32)]


class DisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdis error {code}: {msg}")
        self.code = code


# name -> (restype, argtypes); the full exported surface of include/dis.h
SIGNATURES = {
    "dis_create": (c_int, [c_int, c_int, POINTER(DisPatch), c_int, POINTER(DisOptions), c_void_p,
                           POINTER(c_void_p)]),
    "dis_set_materials": (c_int, [c_void_p, POINTER(DisMaterial), c_int]),
    "dis_workspace_bytes": (c_size_t, [c_void_p]),
    "dis_bind_workspace": (c_int, [c_void_p, c_void_p, c_size_t]),
    "dis_set_state": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "dis_get_state": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "dis_step": (c_int, [c_void_p, c_int, c_void_p]),
    "dis_step_fixed_dt": (c_int, [c_void_p, c_int, c_void_p]),
    "dis_check": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int)]),
    "dis_state_bytes": (c_size_t, [c_void_p, c_int]),
    "dis_last_launches": (c_longlong, [c_void_p]),
    "dis_step_timed": (c_int, [c_void_p, c_int, c_void_p]),
    "dis_set_variant": (c_int, [c_void_p, c_int]),
    "dis_set_schedule": (c_int, [c_void_p, c_int]),
    "dis_set_state_async": (c_int, [c_void_p, c_int, c_void_p]),
    "dis_get_state_async": (c_int, [c_void_p, c_int, c_void_p]),
    "dis_sync": (c_int, [c_void_p]),
    "dis_schedule": (c_int, [c_void_p, POINTER(c_int), c_void_p]),
    "dis_tile_choice": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int), c_void_p]),
    "dis_cfl_dt_static": (c_int, [c_int, c_int, POINTER(DisPatch), POINTER(DisMaterial), c_int,
                                   c_double, c_void_p, c_void_p, c_void_p]),
    "dis_adj_forward": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, POINTER(c_double)]),
    "dis_adjoint": (c_int, [c_void_p, c_void_p, c_int, c_double, c_int, c_void_p, c_int, c_void_p,
                            ctypes.c_uint]),
    "dis_adj_reference": (c_int, [c_void_p, c_int]),
    "dis_alu_peaks": (c_int, [c_void_p, POINTER(c_double), POINTER(c_double), c_void_p]),
    "dis_set_patch_state": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int]),
    "dis_get_patch_state": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int]),
    "dis_query": (c_int, [c_void_p, c_void_p]),
    "dis_amr_create": (c_int, [c_int, POINTER(DisPatch), c_int, POINTER(DisOptions), POINTER(DisAmrOptions),
                               c_void_p, POINTER(c_void_p)]),
    "dis_amr_set_materials": (c_int, [c_void_p, POINTER(DisMaterial), c_int]),
    "dis_amr_set_state": (c_int, [c_void_p, c_void_p, c_int]),
    "dis_amr_step": (c_int, [c_void_p, c_int, c_void_p]),
    "dis_amr_levels": (c_int, [c_void_p, POINTER(c_int), c_void_p]),
    "dis_amr_get_level": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "dis_amr_totals": (c_int, [c_void_p, c_void_p]),
    "dis_amr_check": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    "dis_amr_destroy": (None, [c_void_p]),
    "dis_last_error": (c_char_p, []),
    "dis_destroy": (None, [c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libdis.so and declare its signatures (no GPU needed to load)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def check(rc: int):
    if rc != DIS_OK:
        raise DisError(rc, load().dis_last_error().decode())
    return rc


# thin wrappers with the C names
def dis_create(dim, patches, reactive_material, opts, stream):
    lib = load()
    arr = (DisPatch * len(patches))(*patches)
    out = c_void_p()
    check(lib.dis_create(dim, len(patches), arr, reactive_material, ctypes.byref(opts),
                         c_void_p(stream), ctypes.byref(out)))
    return out


def dis_set_materials(ctx, mats):
    arr = (DisMaterial * len(mats))(*mats)
    return check(load().dis_set_materials(ctx, arr, len(mats)))


def dis_workspace_bytes(ctx):
    return load().dis_workspace_bytes(ctx)


def dis_bind_workspace(ctx, ptr, nbytes):
    return check(load().dis_bind_workspace(ctx, c_void_p(ptr), nbytes))


def dis_set_state(ctx, kind, ptr, on_device):
    return check(load().dis_set_state(ctx, kind, c_void_p(ptr), int(on_device)))


def dis_get_state(ctx, kind, ptr, on_device):
    return check(load().dis_get_state(ctx, kind, c_void_p(ptr), int(on_device)))


def dis_set_state_async(ctx, kind, host_ptr):
    return check(load().dis_set_state_async(ctx, kind, c_void_p(host_ptr)))


def dis_get_state_async(ctx, kind, host_ptr):
    return check(load().dis_get_state_async(ctx, kind, c_void_p(host_ptr)))


def dis_sync(ctx):
    return check(load().dis_sync(ctx))


def dis_step(ctx, n, dt_out_ptr=None):
    return check(load().dis_step(ctx, n, c_void_p(dt_out_ptr) if dt_out_ptr else None))


def dis_step_fixed_dt(ctx, n, dt_ptr):
    return check(load().dis_step_fixed_dt(ctx, n, c_void_p(dt_ptr)))


def dis_check(ctx):
    bp, bc = c_int(-1), c_int(-1)
    rc = load().dis_check(ctx, ctypes.byref(bp), ctypes.byref(bc))
    return rc, bp.value, bc.value


def dis_state_bytes(ctx, kind):
    return load().dis_state_bytes(ctx, kind)


def dis_last_launches(ctx):
    return load().dis_last_launches(ctx)


def dis_step_timed(ctx, n, ms_ptr):
    return check(load().dis_step_timed(ctx, n, c_void_p(ms_ptr)))


def dis_adj_forward(ctx, n_steps, every, material, dt_in_ptr, dt_out_ptr):
    J = c_double(0.0)
    check(load().dis_adj_forward(ctx, n_steps, every, material, c_void_p(dt_in_ptr) if dt_in_ptr else None,
                                 c_void_p(dt_out_ptr) if dt_out_ptr else None, ctypes.byref(J)))
    return J.value


def dis_adjoint(ctx, qbar_ptr, qbar_on_device, jbar, out_kind, grad_ptr, grad_on_device, params_ptr, mask):
    return check(load().dis_adjoint(ctx, c_void_p(qbar_ptr) if qbar_ptr else None, int(qbar_on_device),
                                    float(jbar), out_kind, c_void_p(grad_ptr), int(grad_on_device),
                                    c_void_p(params_ptr) if params_ptr else None, mask))


def dis_last_error():
    return load().dis_last_error().decode()


def dis_destroy(ctx):
    load().dis_destroy(ctx)
