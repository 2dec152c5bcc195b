"""High-level solver over the C ABI: one context = one batch of patches.

PyTorch provides device memory (the workspace is a torch uint8 tensor lent
to the library) and the stream; all arithmetic runs in libdis.so.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L


_EOS = {"sg": L.DIS_EOS_STIFFENED, "romenskii": L.DIS_EOS_ROMENSKII, "jwl": L.DIS_EOS_JWL}


def _material(m: dict) -> L.DisMaterial:
    return L.DisMaterial(m["gamma"], m["p_inf"], m["e_inf"], m["G"], m["plastic"], m["sigma_y"],
                         m["chi0"], m["reactive"], m["Q"], m["cv"], m["A"], m["T_act"],
                         int(m.get("rate_law", 0)), float(m.get("p_ign", 0.0)), _EOS[m.get("eos", "sg")],
                         float(m.get("rho0", 0.0)), float(m.get("K0", 0.0)), float(m.get("alpha_r", 0.0)),
                         float(m.get("beta_r", 0.0)), float(m.get("jwl_A", 0.0)), float(m.get("jwl_B", 0.0)),
                         float(m.get("jwl_R1", 0.0)), float(m.get("jwl_R2", 0.0)),
                         float(m.get("prod_gamma", 0.0)), float(m.get("prod_p_inf", 0.0)),
                         float(m.get("prod_cv", 0.0)), float(m.get("jc_c2", 0.0)), float(m.get("jc_c3", 0.0)),
                         float(m.get("jc_n", 0.0)), float(m.get("jc_m", 0.0)), float(m.get("jc_Tmelt", 0.0)),
                         float(m.get("jc_T0", 0.0)))


def _patch(p, dim) -> L.DisPatch:
    bc = (ctypes.c_int32 * 4)(*[int(b) for b in p.bc])
    return L.DisPatch(p.nx, p.ny if dim == 2 else 1, p.dx, p.dy if dim == 2 else 1.0, bc,
                      float(getattr(p, "x0", 0.0)))


def alu_peaks(stream=None):
    """Measured float32 and float64 FMA throughput of the current device in
    TFLOP/s, and the two probe launch times in ms (include/dis.h:
    dis_alu_peaks)."""
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    ms = np.zeros(2)
    L.check(L.load().dis_alu_peaks(None if stream is None else ctypes.c_void_p(stream), ctypes.byref(f32),
                                   ctypes.byref(f64), ms.ctypes.data))
    return f32.value, f64.value, ms


def pack(arrays) -> np.ndarray:
    """Concatenate per-patch (nfields, ny, nx) arrays into the packed layout."""
    return np.ascontiguousarray(np.concatenate([np.asarray(a, np.float64).reshape(-1) for a in arrays]))


def unpack(flat, shapes):
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(flat[o:o + n].reshape(s))
        o += n
    return out


class Solver:
    """Diffuse-interface step on a batch of patches (see include/dis.h)."""

    def __init__(self, dim, patches, materials, reactive_material=-1, cfl=0.8, thinc=False,
                 precision="fp64", device=None, scheme="rk3", geometry="planar", limiter="minmod"):
        if not torch.cuda.is_available():
            raise RuntimeError("Solver needs a CUDA device (no CPU fallback)")
        dev = torch.device(device or "cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        torch.cuda.set_device(self.device)
        self.dim = dim
        self.patches = list(patches)
        self.reactive = reactive_material >= 0
        self.nf = (11 if dim == 2 else 8) + (1 if self.reactive else 0)
        prec = {"fp64": L.DIS_FP64, "fp32_bulk": L.DIS_FP32_BULK}[precision]
        sch = {"rk3": L.DIS_RK3, "hancock": L.DIS_HANCOCK}[scheme]
        geo = {"planar": L.DIS_PLANAR, "cyl": L.DIS_CYLINDRICAL}[geometry]
        lim = {"minmod": L.DIS_MINMOD, "vanleer": L.DIS_VANLEER}[limiter]
        opts = L.DisOptions(float(cfl), int(bool(thinc)), prec, sch, geo, lim)
        self.stream = torch.cuda.current_stream(self.device)
        self.ctx = L.dis_create(dim, [_patch(p, dim) for p in self.patches], reactive_material, opts,
                                self.stream.cuda_stream)
        self.materials = [dict(m) for m in materials]
        L.dis_set_materials(self.ctx, [_material(m) for m in self.materials])
        nbytes = L.dis_workspace_bytes(self.ctx)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        L.dis_bind_workspace(self.ctx, aligned, nbytes)
        self.shapes = [(self.nf, p.ny if dim == 2 else 1, p.nx) for p in self.patches]
        self.state_numel = sum(int(np.prod(s)) for s in self.shapes)

    @classmethod
    def from_workload(cls, wl, precision="fp64", **kw):
        kw.setdefault("scheme", getattr(wl, "scheme", "rk3"))
        kw.setdefault("geometry", getattr(wl, "geometry", "planar"))
        kw.setdefault("limiter", getattr(wl, "limiter", "minmod"))
        return cls(wl.dim, wl.patches, wl.materials, wl.reactive_material, wl.cfl, wl.thinc,
                   precision, **kw)

    # -- state ----------------------------------------------------------------
    def set_state(self, x, kind=L.DIS_PRIMITIVE):
        if isinstance(x, torch.Tensor) and x.is_cuda:
            x = x.contiguous().to(torch.float64)
            assert x.numel() == self.state_numel
            L.dis_set_state(self.ctx, kind, x.data_ptr(), True)
            self._keep = x
        else:
            x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1))
            assert x.size == self.state_numel, (x.size, self.state_numel)
            L.dis_set_state(self.ctx, kind, x.ctypes.data, False)

    def set_state_async(self, host, kind=L.DIS_PRIMITIVE):
        """Pipelined host -> device transfer of a pinned CPU tensor (include/dis.h:
        dis_set_state_async); keep it alive and unchanged until sync()."""
        assert isinstance(host, torch.Tensor) and not host.is_cuda and host.dtype == torch.float64
        assert host.numel() == self.state_numel and host.is_contiguous()
        L.dis_set_state_async(self.ctx, kind, host.data_ptr())

    def get_state_async(self, host, kind=L.DIS_CONSERVATIVE):
        """Pipelined device -> host transfer into a pinned CPU tensor (include/dis.h:
        dis_get_state_async); its contents are valid after sync()."""
        assert isinstance(host, torch.Tensor) and not host.is_cuda and host.dtype == torch.float64
        assert host.numel() == self.state_numel and host.is_contiguous()
        L.dis_get_state_async(self.ctx, kind, host.data_ptr())

    def sync(self):
        L.dis_sync(self.ctx)

    def set_patch(self, patch, arr, kind=L.DIS_PRIMITIVE):
        """State of one patch ([nfields, ny, nx] float64, host array or CUDA
        tensor) (include/dis.h: dis_set_patch_state)."""
        lib = L.load()
        if isinstance(arr, torch.Tensor) and arr.is_cuda:
            t = arr.contiguous().to(torch.float64)
            L.check(lib.dis_set_patch_state(self.ctx, patch, kind, ctypes.c_void_p(t.data_ptr()), 1))
            torch.cuda.synchronize()
        else:
            a = np.ascontiguousarray(np.asarray(arr, np.float64))
            L.check(lib.dis_set_patch_state(self.ctx, patch, kind, ctypes.c_void_p(a.ctypes.data), 0))

    def get_patch(self, patch, shape, kind=L.DIS_CONSERVATIVE):
        """State of one patch as a host array of `shape` ([nfields, ny, nx])
        (include/dis.h: dis_get_patch_state)."""
        h = np.empty(shape, np.float64)
        L.check(L.load().dis_get_patch_state(self.ctx, patch, kind, ctypes.c_void_p(h.ctypes.data), 0))
        return h

    def query(self):
        """Device-reduced totals, phi range, dt, step time and bytes
        (include/dis.h: dis_query) as a dict."""
        st = L.DisStats()
        L.check(L.load().dis_query(self.ctx, ctypes.byref(st)))
        return {"mass": list(st.mass), "momentum": list(st.momentum), "energy": st.energy,
                "reactant": st.reactant, "phi_min": st.phi_min, "phi_max": st.phi_max,
                "dt_min": st.dt_min, "dt_max": st.dt_max, "kernel_ms": st.kernel_ms, "bytes": st.bytes,
                "steps": st.steps, "launches": st.launches, "status": st.status,
                "bad_patch": st.bad_patch, "bad_cell": st.bad_cell}

    def set_prim(self, prim_arrays):
        self.set_state(pack(prim_arrays), L.DIS_PRIMITIVE)

    def get_state(self, kind=L.DIS_CONSERVATIVE, out=None):
        """Packed state as a numpy array (host) or into a CUDA tensor `out`."""
        if out is not None:
            assert out.is_cuda and out.dtype == torch.float64 and out.numel() == self.state_numel
            L.dis_get_state(self.ctx, kind, out.data_ptr(), True)
            return out
        h = np.empty(self.state_numel, np.float64)
        L.dis_get_state(self.ctx, kind, h.ctypes.data, False)
        return h

    def get_arrays(self, kind=L.DIS_CONSERVATIVE):
        return unpack(self.get_state(kind), self.shapes)

    # -- stepping ---------------------------------------------------------------
    def step(self, n=1, return_dt=False):
        if return_dt:
            dt = np.empty(len(self.patches), np.float64)
            L.dis_step(self.ctx, n, dt.ctypes.data)
            return dt
        L.dis_step(self.ctx, n, None)
        return None

    def step_fixed_dt(self, n, dt):
        dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (len(self.patches),)))
        L.dis_step_fixed_dt(self.ctx, n, dt.ctypes.data)

    def step_timed(self, n=1):
        """Mean device ms per launch over n steps: float64 [prim, flux x, flux y,
        update]; FP32-bulk [CFL pass or primitive pre-pass, stage kernel, 0, 0]."""
        ms = np.zeros(4, np.float64)
        L.dis_step_timed(self.ctx, n, ms.ctypes.data)
        return ms

    def tile_choice(self):
        """(TX, TY, precomputed primitives, tuned ms per step of each variant)
        of an FP32-bulk context (include/dis.h: dis_tile_choice)."""
        tx, ty, pre = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        ms = np.zeros(L.DIS_NVARIANTS, np.float64)
        L.check(L.load().dis_tile_choice(self.ctx, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(pre),
                                         ms.ctypes.data))
        return tx.value, ty.value, bool(pre.value), ms

    def set_variant(self, v):
        """Fix the FP32-bulk stage variant (-1: tune on the next step)."""
        L.check(L.load().dis_set_variant(self.ctx, int(v)))

    def set_schedule(self, schedule):
        """1D FP32-bulk batches: 0 per-step launches, 1 the persistent batch
        kernel, -1 chosen by the tuner (include/dis.h: dis_set_schedule)."""
        L.check(L.load().dis_set_schedule(self.ctx, int(schedule)))

    def schedule(self):
        """(schedule in use, tuned one-step ms of the persistent kernel per
        variant) (include/dis.h: dis_schedule)."""
        sc = ctypes.c_int(0)
        ms = np.zeros(L.DIS_NVARIANTS, np.float64)
        L.check(L.load().dis_schedule(self.ctx, ctypes.byref(sc), ms.ctypes.data))
        return sc.value, ms

    def check(self):
        return L.dis_check(self.ctx)

    # -- parameters and adjoint ---------------------------------------------------
    PARAM_KEYS = ("G", "sigma_y", "Q")

    def params(self) -> np.ndarray:
        """Differentiable parameters [G_l, sigma_y_l, Q_l for l = 0, 1]."""
        return np.array([m[k] for m in self.materials for k in self.PARAM_KEYS], np.float64)

    def set_params(self, theta):
        theta = np.asarray(theta, np.float64).reshape(L.DIS_NPARAM)
        for l, m in enumerate(self.materials):
            for k, key in enumerate(self.PARAM_KEYS):
                m[key] = float(theta[3 * l + k])
        L.dis_set_materials(self.ctx, [_material(m) for m in self.materials])

    def adj_forward(self, n_steps, every=20, material=-1, dts=None):
        """Recorded forward run for `adjoint` (include/dis.h: dis_adj_forward).
        Returns (J, dts[n_steps, n_patches])."""
        out = np.empty((n_steps, len(self.patches)), np.float64)
        din = None
        if dts is not None:
            din = np.ascontiguousarray(np.broadcast_to(np.asarray(dts, np.float64).reshape(n_steps, -1),
                                                       (n_steps, len(self.patches))))
        J = L.dis_adj_forward(self.ctx, n_steps, every, material, din.ctypes.data if din is not None else None,
                              out.ctypes.data)
        return J, out

    def adj_reference(self, on=True):
        """Diagnostic: reverse the face Riemann problems with dual numbers
        (include/dis.h: dis_adj_reference)."""
        L.check(L.load().dis_adj_reference(self.ctx, int(bool(on))))

    def adjoint(self, qbar=None, jbar=0.0, kind=L.DIS_CONSERVATIVE, param_mask=(1 << L.DIS_NPARAM) - 1,
                out=None):
        """Gradient of <qbar, q_final> + jbar J with respect to the initial state
        (`kind` variables, packed) and the parameters.  qbar / out may be CUDA
        tensors (device path) or host arrays."""
        gp = np.zeros(L.DIS_NPARAM, np.float64)
        keep = []
        if qbar is None:
            qp, qdev = None, False
        elif isinstance(qbar, torch.Tensor) and qbar.is_cuda:
            qbar = qbar.contiguous().to(torch.float64)
            keep.append(qbar)
            qp, qdev = qbar.data_ptr(), True
        else:
            qbar = np.ascontiguousarray(np.asarray(qbar, np.float64).reshape(-1))
            keep.append(qbar)
            qp, qdev = qbar.ctypes.data, False
        if out is not None:
            assert out.is_cuda and out.dtype == torch.float64 and out.numel() == self.state_numel
            L.dis_adjoint(self.ctx, qp, qdev, jbar, kind, out.data_ptr(), True, gp.ctypes.data, param_mask)
            return out, gp
        g = np.empty(self.state_numel, np.float64)
        L.dis_adjoint(self.ctx, qp, qdev, jbar, kind, g.ctypes.data, False, gp.ctypes.data, param_mask)
        return g, gp

    @property
    def launches(self):
        return L.dis_last_launches(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            L.dis_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AmrSolver:
    """The structured AMR hierarchy of include/dis.h (dis_amr_*) over the
    domain of a one-patch workload, float64: the workload's scheme (SSP-RK3,
    or MUSCL-Hancock in planar geometry) and geometry (planar or
    cylindrical)."""

    def __init__(self, wl, max_levels=2, block=8, eps=0.1, buffer=2, u_floor=1.0, regrid_every=4,
                 device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("AmrSolver needs a CUDA device (no CPU fallback)")
        assert len(wl.patches) == 1
        dev = torch.device(device or "cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(dev)
        self.device = dev
        self.wl = wl
        self.dim = wl.dim
        self.reactive = wl.reactive_material >= 0
        self.nf = (11 if wl.dim == 2 else 8) + (1 if self.reactive else 0)
        self.stream = torch.cuda.current_stream(dev)
        geo = {"planar": L.DIS_PLANAR, "cyl": L.DIS_CYLINDRICAL}[getattr(wl, "geometry", "planar")]
        sch = {"rk3": L.DIS_RK3, "hancock": L.DIS_HANCOCK}[getattr(wl, "scheme", "rk3")]
        opts = L.DisOptions(float(wl.cfl), int(bool(wl.thinc)), L.DIS_FP64, sch, geo,
                            {"minmod": L.DIS_MINMOD, "vanleer": L.DIS_VANLEER}[getattr(wl, "limiter", "minmod")])
        aopt = L.DisAmrOptions(int(max_levels), int(block), float(eps), int(buffer), float(u_floor),
                               int(regrid_every))
        self.max_levels = int(max_levels)
        p = wl.patches[0]
        self.base = (p.nx, p.ny if wl.dim == 2 else 1)
        lib = L.load()
        out = ctypes.c_void_p()
        dp = _patch(p, wl.dim)
        L.check(lib.dis_amr_create(wl.dim, ctypes.byref(dp), wl.reactive_material, ctypes.byref(opts),
                                   ctypes.byref(aopt), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(out)))
        self.h = out
        mats = (L.DisMaterial * 2)(*[_material(m) for m in wl.materials])
        L.check(lib.dis_amr_set_materials(self.h, mats, 2))

    def set_prim(self, prim):
        a = np.ascontiguousarray(prim, dtype=np.float64)
        L.check(L.load().dis_amr_set_state(self.h, a.ctypes.data, L.DIS_PRIMITIVE))

    def step(self, n=1):
        dts = np.zeros(n)
        L.check(L.load().dis_amr_step(self.h, n, dts.ctypes.data))
        return dts

    def levels(self):
        n = ctypes.c_int()
        counts = (ctypes.c_int * self.max_levels)()
        L.check(L.load().dis_amr_levels(self.h, ctypes.byref(n), counts))
        return n.value, list(counts)

    def get_level(self, level, kind=L.DIS_CONSERVATIVE):
        nx, ny = self.base[0] << level, (self.base[1] << level) if self.dim == 2 else 1
        out = np.empty((self.nf, ny, nx))
        act = np.zeros((ny, nx), dtype=np.uint8)
        L.check(L.load().dis_amr_get_level(self.h, level, kind, out.ctypes.data, act.ctypes.data))
        return out, act.astype(bool)

    def totals(self):
        out = np.zeros(self.nf)
        L.check(L.load().dis_amr_totals(self.h, out.ctypes.data))
        return out

    def check(self):
        lv, p, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rc = L.load().dis_amr_check(self.h, ctypes.byref(lv), ctypes.byref(p), ctypes.byref(c))
        return rc, lv.value, p.value, c.value

    def close(self):
        if getattr(self, "h", None):
            L.load().dis_amr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
