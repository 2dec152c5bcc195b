"""Helpers shared by the GPU parity tests: run the oracle and the CUDA path on
the same seeded workload and compare per-field relative L1.

Metric (per field f):  L1_f = sum |gpu - oracle| / max(sum |oracle|, N s_f)
with a field scale s_f so that fields that are (nearly) zero do not divide by
zero: 1 for the volume fraction and the stretch components, rho_ref c_ref for
momentum, 0 for the strictly positive densities and energy.  For primitives
the pressure scale is the energy density (pressure in a stiff material is
recovered from rho E with an amplification gamma p_inf / p), velocity is
scaled by c_ref, and the phasic densities are left to the conservative check
(they are ill-conditioned where a material is a trace).
"""
import numpy as np

from oracle import closures as OC
from oracle import scheme as OS


def oracle_run(wl, steps, patch_ids=None, dt_list=None):
    """Oracle conservative arrays (per patch) after `steps` steps, and dts."""
    outs, dts = [], []
    ids = range(len(wl.patches)) if patch_ids is None else patch_ids
    for k in ids:
        p = wl.patches[k]
        q, d = OS.run(p.prim, wl.dim, wl.materials, OS.grid_of(p, wl.dim, getattr(wl, "geometry", "planar")),
                      dict(cfl=wl.cfl, thinc=wl.thinc, scheme=getattr(wl, "scheme", "rk3"),
                           limiter=getattr(wl, "limiter", "minmod")), steps,
                      None if dt_list is None else dt_list[k])
        outs.append(q.numpy())
        dts.append(d)
    return outs, dts


def oracle_prim(wl, cons_arrays):
    out = []
    for a in cons_arrays:
        q = OS.cons_from_array(a, wl.dim, wl.reactive)
        out.append(OS.prim_to_array(OC.cons_to_prim(q, wl.materials), wl.dim, wl.reactive).numpy())
    return out


def _names(wl, kind):
    return OS._names(wl.dim, wl.reactive, kind)


def cons_scales(wl, ora):
    o = np.asarray(ora).reshape(ora.shape[0], -1)
    names = _names(wl, "cons")
    ix = {n: k for k, n in enumerate(names)}
    ar_max = max(np.abs(o[ix["ar1"]]).max(), np.abs(o[ix["ar2"]]).max())
    rc = np.sqrt(ar_max * np.abs(o[ix["E"]]).max())  # ~ rho c
    s = []
    for n in names:
        if n == "phi1" or n.startswith("V"):
            s.append(1.0)
        elif n in ("mx", "my"):
            s.append(rc)
        else:
            s.append(0.0)
    return np.array(s)


def rel_l1(gpu, ora, scales=None):
    g = np.asarray(gpu).reshape(gpu.shape[0], -1)
    o = np.asarray(ora).reshape(ora.shape[0], -1)
    n = g.shape[1]
    num = np.abs(g - o).sum(1)
    den = np.abs(o).sum(1)
    if scales is not None:
        den = np.maximum(den, n * scales)
    return np.where(den > 0, num / np.maximum(den, 1e-300), num)


def cons_l1(wl, gpu, ora):
    return rel_l1(gpu, ora, cons_scales(wl, ora))


def max_rel(gpu, ora, scales=None):
    """Element-wise companion of rel_l1: per field max |gpu - ora| / max(max
    |ora|, s_f), so that one bad cell cannot hide in the sum."""
    g = np.asarray(gpu).reshape(gpu.shape[0], -1)
    o = np.asarray(ora).reshape(ora.shape[0], -1)
    den = np.abs(o).max(1)
    if scales is not None:
        den = np.maximum(den, scales)
    return np.abs(g - o).max(1) / np.maximum(den, 1e-300)


def cons_max(wl, gpu, ora):
    return max_rel(gpu, ora, cons_scales(wl, ora))


_RECORD = {}


def record(name, **kw):
    """Keep the measured errors of a parity case (JSON at record_path)."""
    import json
    _RECORD[name] = {k: (np.asarray(v).tolist() if isinstance(v, (np.ndarray, list, tuple)) else v)
                     for k, v in kw.items()}
    with open(record_path("parity.json"), "w") as f:
        json.dump(_RECORD, f, indent=1)


def prim_l1(wl, gpu_prim, ora_prim, ora_cons):
    """Primitive comparison on p, velocities, stretch, lam (see module doc)."""
    names = _names(wl, "prim")
    oc = np.asarray(ora_cons).reshape(ora_cons.shape[0], -1)
    cnames = _names(wl, "cons")
    E = np.abs(oc[cnames.index("E")]).max()
    ar = max(np.abs(oc[cnames.index("ar1")]).max(), np.abs(oc[cnames.index("ar2")]).max())
    c_ref = np.sqrt(E / ar)
    g = np.asarray(gpu_prim).reshape(gpu_prim.shape[0], -1)
    o = np.asarray(ora_prim).reshape(ora_prim.shape[0], -1)
    out = {}
    for k, nme in enumerate(names):
        if nme in ("rho1", "rho2"):
            continue
        s = {"p": E, "u": c_ref, "v": c_ref}.get(nme, 1.0)
        out[nme] = float(np.abs(g[k] - o[k]).sum() / max(np.abs(o[k]).sum(), g.shape[1] * s))
    return out


def record_path(name):
    """Path of a side file (measured errors as JSON) named `name`, in the
    directory given by DIS_RECORD_DIR (default: the system temp directory)."""
    import os
    import tempfile
    d = os.environ.get("DIS_RECORD_DIR") or tempfile.gettempdir()
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, name)
