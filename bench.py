"""Benchmark: cell-updates/s of the diffuse-interface step on one GB300.

Workload: premixed reactive air over an elastoplastic plate on a 2048 x 1024
grid (all rows of the step: ghost map, CFL reduction, primitive recovery,
MUSCL/THINC-BVD, HLLC, RK3, plastic and reactive updates).  A bench "step" is
one time step of the whole grid.  One cell-update = one full step of one cell.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  The reference arm (--impl reference) times the float64
CPU oracle on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s and % HBM peak, FP32-bulk vs plain FP64 on one GB300 at stated L1"

# Arithmetic and DRAM traffic of the dominant kernels, counted by ncu on the
# kernels as built (executed FADD + FMUL + 2 FFMA, resp. DADD + DMUL + 2 DFMA,
# thread level).  FP32-bulk stage kernel, per cell-stage, one launch on the
# full 2048 x 1024 reactive plate (stage 2, which reads two states and writes
# one), per tile shape (TX, TY); None where that shape was not captured (the
# register budget does not change the arithmetic).
STAGE32_FLOP = {(16, 15): None, (32, 15): 1336.1, (32, 7): None}
# float64 x-face flux kernel: FP64 FLOP per face (1024 x 512 capture)
FLUX_FP64_FLOP_PER_FACE = 868.1
STAGE32_DRAM = {(16, 15): None, (32, 15): 145.7, (32, 7): None}
# The FP32-bulk MUSCL-Hancock kernel on the same grid (one launch of the
# 32 x 7 tile): FP32 FLOP and DRAM bytes per cell-update.
HANCOCK32_FLOP = {(32, 7): 2606.7}
HANCOCK32_DRAM = {(32, 7): 85.6}
# DRAM bytes per x-flux launch of the float64 step, per face (73.07 MB for
# 524800 faces on 1024 x 512); traffic grows with the face count.
FLUX_DRAM_BYTES_PER_FACE = 73.07e6 / 524800
UNIT = "cell-updates/s"
NX, NY = 2048, 1024


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def state_bytes(dim, reactive, precision):
    """Bytes of one cell's stored state: float64, nfields x 8; FP32-bulk,
    (nfields + 1) x 4 (float32 fields, the soft energy, phi1 as a
    float-float pair)."""
    nf = (11 if dim == 2 else 8) + (1 if reactive else 0)
    return 8 * nf if precision == "fp64" else 4 * (nf + 1)


def workload(nx=None, ny=None):
    from paper_2009_14555_gb300 import workloads as W
    return W.reactive_plate_2d(nx or NX, ny or NY)


def max_over_ranks(x, device=None):
    """Largest value of x over the ranks of the process group (x itself
    without one): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank, world, ms_per_step):
    """Whole-job cell-updates/s: every rank advances its own replica of the
    workload (replicas only: the step has no collective)."""
    return cells_per_rank * world / (ms_per_step * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.p = None
        # the samples go to a temporary file (DIS_RECORD_DIR keeps them)
        import tempfile
        d = os.environ.get("DIS_RECORD_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return self
        # wait for the first sample so the sampler's start-up is outside the timed region
        t0 = time.time()
        while time.time() - t0 < 5.0:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2009_14555_gb300.solver import Solver, pack

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = workload(args.nx, args.ny)
    cells = wl.cells
    prim = pack([p.prim for p in wl.patches])
    results = {}
    precisions = ["fp64", "fp32_bulk"]
    for prec in precisions:
        s = Solver.from_workload(wl, precision=prec)
        if prec == "fp32_bulk" and args.variant is not None:
            s.set_variant(args.variant)
        s.set_state(prim, kind=1)
        stream = s.stream
        for _ in range(args.warmup):
            s.step(1)
        torch.cuda.synchronize()
        launches = 0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev0.record(stream)
            for k in range(args.steps):
                s.step(1)
                launches += s.launches
            ev1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
        tot_ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
        rc, _, _ = s.check()
        final = s.get_state(kind=0)  # state after warm-up + timed steps, for the L1 comparison
        kernel_ms = s.step_timed(2)  # per-launch device time, outside the timed region
        tile = s.tile_choice() if prec == "fp32_bulk" else (0, 0, False, None)
        results[prec] = dict(ms_total=tot_ms, ms_per_step=tot_ms / args.steps, wall=wall,
                             launches=launches, clocks=clk.summary(), ok=rc == 0, solver=s,
                             kernel_ms=kernel_ms, final=final, tile=tile)
    # end-to-end through the C ABI with host buffers: H2D of the step's input
    # state from pinned memory, the step, D2H of the result, every step.
    s = results["fp32_bulk"]["solver"]
    hin = torch.from_numpy(prim).pin_memory()
    hout = torch.empty(s.state_numel, dtype=torch.float64).pin_memory()
    from paper_2009_14555_gb300 import _lib as L

    def e2e_step():
        # pipelined through the public API: the copy of this step's input,
        # the step and the copy of the previous step's result overlap
        s.set_state_async(hin, kind=1)
        s.step(1)
        s.get_state_async(hout, kind=0)

    e2e_step()  # warm-up
    s.sync()
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    s.sync()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dev)
    nbytes = prim.nbytes

    r = results["fp32_bulk"]
    r64 = results["fp64"]
    value = job_throughput(cells, world, r["ms_per_step"])
    value64 = job_throughput(cells, world, r64["ms_per_step"])
    hbm, kind = peaks()
    from paper_2009_14555_gb300.solver import alu_peaks
    f32_peak, f64_peak, _ = alu_peaks(torch.cuda.current_stream().cuda_stream)
    nxw, nyw = args.nx or NX, args.ny or NY
    faces_x = (nxw + 1) * nyw
    # algorithmic bytes per cell-update: read + write the stored state once
    alg32 = 2 * state_bytes(2, True, "fp32_bulk")
    alg64 = 2 * state_bytes(2, True, "fp64")
    hbm32 = alg32 * cells / (r["ms_per_step"] * 1e-3) / 1e9
    hbm64 = alg64 * cells / (r64["ms_per_step"] * 1e-3) / 1e9
    t64 = r64["kernel_ms"][1] * 1e-3
    flux64_tflops = FLUX_FP64_FLOP_PER_FACE * faces_x / t64 / 1e12
    # dominant kernel: the FP32-bulk stage kernel, one launch per RK stage (a
    # third of a cell-update for every cell), live event time per launch
    t32 = r["kernel_ms"][1] * 1e-3
    tx, ty = r["tile"][0], r["tile"][1]
    launch_bytes = alg32 / 3.0 * cells
    stage_gbs = launch_bytes / t32 / 1e9
    flop = STAGE32_FLOP.get((tx, ty))
    dram = STAGE32_DRAM.get((tx, ty))
    stage_tflops = flop * cells / t32 / 1e12 if flop else None
    # per-field L1 of the FP32-bulk state against the float64 GPU state after the
    # same number of steps (the float64 GPU path matches the oracle to 1e-10)
    a32, a64 = r["final"].reshape(12, -1), r64["final"].reshape(12, -1)
    names = ["phi1", "ar1", "ar2", "mx", "my", "E", "V11", "V12", "V21", "V22", "V33", "arl"]
    floor = {"phi1": 1.0, "V11": 1.0, "V12": 1.0, "V21": 1.0, "V22": 1.0, "V33": 1.0}
    rc_ = float(np.sqrt(np.abs(a64[1:3]).max() * np.abs(a64[5]).max()))
    floor.update(mx=rc_, my=rc_)
    l1 = {n: float(np.abs(a32[k] - a64[k]).sum() / max(np.abs(a64[k]).sum(), a64.shape[1] * floor.get(n, 0.0)))
          for k, n in enumerate(names)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (phi1 as a float-float pair)",
        "data": "synthetic",
        "config": {"workload": f"2d_reactive_plate_{nxw}x{nyw}", "cells": cells,
                   "precision": "fp32_bulk", "scheme": "ssp_rk3",
                   "l2": "working set larger than L2 (3 state buffers of 109 MB)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm",
                     "kernel": f"k_stage32<{tx}x{ty}> (FP32-bulk Runge-Kutta stage)",
                     "achieved": stage_gbs, "peak": hbm, "unit": "GB/s", "frac": stage_gbs / hbm,
                     "traffic": dram * cells if dram else None,
                     "algorithmic_bytes_per_launch": launch_bytes,
                     "note": f"algorithmic bytes = {alg32} B per cell-update (state read + written once) / 3 "
                             f"stage launches x {cells} cells, over the live CUDA-event time of one stage launch; "
                             f"peak = {kind} copy bandwidth; traffic = ncu DRAM bytes of one launch"},
        "alu": {"kernel": f"k_stage32<{tx}x{ty}>", "achieved": stage_tflops, "peak": f32_peak, "unit": "TFLOP/s",
                "frac": stage_tflops / f32_peak if stage_tflops else None,
                "flop_per_cell_stage": flop,
                "note": "executed FP32 FLOP per cell-stage (ncu) x cells / live event time per launch; "
                        "peak = measured FMA-loop throughput of this GPU (dis_alu_peaks)"},
        "measured_peaks": {"fp32_tflops": f32_peak, "fp64_tflops": f64_peak, "hbm_gbs": hbm},
        "l1_vs_fp64": l1,
        "hbm": {"achieved_gbs": hbm32, "peak_gbs": hbm, "frac": hbm32 / hbm,
                "algorithmic_bytes_per_cell_update": alg32, "peak_kind": kind},
        "kernels_ms_per_launch": {"cfl_pass_first_step_only": float(r["kernel_ms"][0]),
                                  "stage": float(r["kernel_ms"][1])},
        "tile": {"tx": tx, "ty": ty, "tuned_ms_per_step": [round(float(x), 4) for x in r["tile"][3]]},
        "fp64": {"value": value64, "ms_per_step": r64["ms_per_step"],
                 "speedup_fp32_bulk": value / value64,
                 "hbm": {"achieved_gbs": hbm64, "frac": hbm64 / hbm, "algorithmic_bytes_per_cell_update": alg64},
                 "roofline": {"bound": "alu", "kernel": "k_flux x (float64)", "achieved": flux64_tflops,
                              "peak": f64_peak, "unit": "TFLOP/s", "frac": flux64_tflops / f64_peak,
                              "traffic": FLUX_DRAM_BYTES_PER_FACE * faces_x,
                              "note": "peak = measured float64 FMA-loop throughput (dis_alu_peaks)"},
                 "kernels_ms_per_launch": dict(zip(["prim", "flux_x", "flux_y", "update"],
                                                   map(float, r64["kernel_ms"]))),
                 "clocks": r64["clocks"]},
        "e2e": {"value": job_throughput(cells, world, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
        "status_ok": bool(r["ok"] and r64["ok"]),
    }
    line["fp64"]["hancock"] = hancock_bench(wl, prim, args.steps, args.warmup)
    line["fp64"]["hancock"]["speedup_vs_rk3"] = line["fp64"]["hancock"]["value"] / value64
    h32 = hancock_bench(wl, prim, args.steps, args.warmup, precision="fp32_bulk")
    h32["speedup_vs_rk3"] = h32["value"] / value
    line["fp32_bulk_hancock"] = h32
    if not args.no_configs:
        line["configs"] = configs_bench(args.warmup)
    if not args.no_batch:
        line["batch_1d"] = batch_bench()
    if not args.no_widened:
        try:
            line["widened_rows"] = widened_bench(args.warmup)
        except Exception as e:  # the headline line above is measured: still print it
            line["widened_rows"] = {"error": repr(e)}
    if not args.no_adjoint:
        line["adjoint"] = adjoint_bench()
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    for v in results.values():
        v["solver"].close()
    if world > 1:
        dist.destroy_process_group()


def adjoint_bench(n=256, steps=200, every=20):
    """The adjoint case (256^2 shock-disc, 200 steps, checkpoint every 20):
    time of the recorded forward run (float64, and FP32-bulk with float64
    checkpoints) and of the checkpointed float64 reverse sweep (gradients with
    respect to the initial primitive state and the six material parameters)."""
    import torch
    from paper_2009_14555_gb300 import workloads as W
    from paper_2009_14555_gb300.solver import Solver, pack
    wl = W.adjoint_case_2d(n, steps=steps)
    prim = pack([p.prim for p in wl.patches])
    cells = wl.cells
    out = {"workload": f"2d_shock_disc_adjoint_{n} ({steps} steps, checkpoint every {every})"}
    for prec in ("fp64", "fp32_bulk"):
        s = Solver.from_workload(wl, precision=prec)
        s.set_state(prim)
        s.adj_forward(2, every=2, material=0)  # warm-up (allocation, tuning, first launches)
        s.adjoint(None, 1.0, kind=1)
        s.set_state(prim)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, _ = s.adj_forward(steps, every=every, material=0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        g, gp = s.adjoint(None, 1.0, kind=1)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ok = s.check()[0] == 0 and bool(np.isfinite(g).all())
        s.close()
        out[prec] = {"forward_s": t1 - t0, "reverse_s": t2 - t1,
                     "reverse_cell_updates_per_s": cells * steps / (t2 - t1),
                     "reverse_over_forward": (t2 - t1) / (t1 - t0), "J": J, "status_ok": ok}
    return out


def _timed_steps(wl, prim, precision, steps, warmup, **kw):
    """cell-updates/s of `steps` steps after `warmup` (device events on the
    solver's stream, inputs resident)."""
    import torch
    from paper_2009_14555_gb300.solver import Solver
    s = Solver.from_workload(wl, precision=precision, **kw)
    s.set_state(prim, kind=1)
    s.step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rc = s.check()[0]
    s.close()
    return {"value": wl.cells / (ms * 1e-3), "ms_per_step": ms, "steps": steps, "status_ok": rc == 0}


def configs_bench(warmup=3):
    """The two smaller configurations at their full length: the 1D solid|gas
    problem (1000 cells, 500 steps; launch-latency bound) and the 512^2
    shock-disc with THINC (2000 steps; its 3 FP32-bulk states fit in L2).
    cell-updates/s over the whole run, both precisions (device events,
    inputs resident), and the algorithmic-byte HBM fraction."""
    from paper_2009_14555_gb300 import workloads as W
    from paper_2009_14555_gb300.solver import pack
    hbm, _ = peaks()
    out = {}
    for key, wl in (("1d_solid_gas_1000_500", W.solid_gas_1d(1000, steps=500)),
                    ("2d_shock_disc_512_2000", W.shock_disc_2d(512, steps=2000))):
        prim = pack([p.prim for p in wl.patches])
        row = {"cells": wl.cells, "steps": wl.steps}
        for prec in ("fp32_bulk", "fp64"):
            r = _timed_steps(wl, prim, prec, wl.steps, warmup)
            b = 2 * state_bytes(wl.dim, wl.reactive, prec)
            r["hbm_frac"] = b * r["value"] / 1e9 / hbm
            r["algorithmic_bytes_per_cell_update"] = b
            row[prec] = r
        row["speedup_fp32_bulk"] = row["fp32_bulk"]["value"] / row["fp64"]["value"]
        out[key] = row
    return out


def widened_bench(warmup=3):
    """The rows beyond the planar Arrhenius step, on full-size inputs.

    Cylindrical geometry: the shock-sphere problem in (r, z), 1024 x 2048
    cells, stepped with the geometric source and, for the cost of s_g, the
    same input in planar geometry.  The k sqrt(lam) reaction law: 1024 copies
    of the 4000-cell detonation-into-copper problem (the resolution of the
    paper's one-dimensional test) in one batch.  Johnson-Cook plasticity, the
    AMR hierarchy (SSP-RK3, MUSCL-Hancock, and SSP-RK3 in (r, z)) and the AMR
    form of the one-dimensional test follow, each measured on its own
    (jc_bench, amr_bench, amr_detonation_bench)."""
    import copy
    from paper_2009_14555_gb300 import workloads as W
    from paper_2009_14555_gb300.solver import pack
    out = {}
    wl = W.sphere_shock_rz(2048, steps=0)
    prim = pack([p.prim for p in wl.patches])
    cyl = {"workload": "2d_sphere_shock_rz_1024x2048 (x = r, y = z)", "cells": wl.cells}
    for prec, steps in (("fp32_bulk", 200), ("fp64", 30)):
        c = _timed_steps(wl, prim, prec, steps, warmup)
        p = _timed_steps(wl, prim, prec, steps, warmup, geometry="planar")
        cyl[prec] = dict(c, planar_ms_per_step=p["ms_per_step"],
                         cyl_over_planar=c["ms_per_step"] / p["ms_per_step"])
    out["cylindrical"] = cyl
    one = W.detonation_copper_1d(4000, steps=0)
    wl = copy.copy(one)
    wl.patches = [one.patches[0]] * 1024
    prim = pack([p.prim for p in wl.patches])
    det = {"workload": "1d_detonation_copper_4000 x 1024 (k sqrt(lam) law, pressure switch)",
           "cells": wl.cells}
    for prec, steps in (("fp32_bulk", 200), ("fp64", 30)):
        det[prec] = _timed_steps(wl, prim, prec, steps, warmup)
    out["sqrt_rate_law"] = det
    for key, fn in (("johnson_cook", jc_bench), ("amr", amr_bench),
                    ("amr_hancock", lambda: amr_bench(kind="hancock")),
                    ("amr_cylindrical", lambda: amr_bench(kind="cylindrical")),
                    ("amr_detonation_1d", amr_detonation_bench)):
        try:
            out[key] = fn()
        except Exception as e:  # the other rows are measured: keep them
            out[key] = {"error": repr(e)}
    return out


def jc_bench(nr=512, steps=30, warmup=3):
    """Johnson-Cook plasticity (float64): the shock-driven hemispherical
    indentation of Section 4.4 in (r, z), nr x 5 nr cells, and the same input
    with the copper's plasticity replaced by perfect plasticity at c1 (the
    cost of the Johnson-Cook relaxation's bisection and temperature)."""
    from paper_2009_14555_gb300 import workloads as W
    from paper_2009_14555_gb300.solver import pack
    wl = W.indentation_rz(nr, steps=0)
    prim = pack([p.prim for p in wl.patches])
    row = {"workload": f"2d_indentation_rz_{nr}x{5 * nr} (Johnson-Cook copper, x = r, y = z)", "cells": wl.cells,
           "precision": "fp64"}
    row["johnson_cook"] = _timed_steps(wl, prim, "fp64", steps, warmup)
    perfect = dict(wl.materials[0], plastic=1)
    wp = W.indentation_rz(nr, steps=0)
    wp.materials = [perfect, wp.materials[1]]
    wp.reactive_material = -1
    prim_p = pack([p.prim[:-1] for p in wp.patches])
    row["perfect_plasticity"] = _timed_steps(wp, prim_p, "fp64", steps, warmup)
    row["jc_over_perfect"] = row["johnson_cook"]["ms_per_step"] / row["perfect_plasticity"]["ms_per_step"]
    return row


def amr_detonation_bench(n=1000, levels=3, steps=40, warmup=2):
    """The one-dimensional test of Section 4.1 in its AMR setting: 1000 base
    cells and two more levels of ratio 2 (effective 4000 cells), the generic
    explosive against Romenskii copper, float64; 40 level-0 steps from the
    booster's ignition (longer runs reach a cell that leaves the hyperbolic
    region where the detonation meets the copper); against the uniform
    4000-cell grid over the same physical time."""
    import torch
    from paper_2009_14555_gb300 import workloads as W
    from paper_2009_14555_gb300.solver import AmrSolver, Solver, pack
    wl = W.detonation_copper_1d(n, steps=0, explosive="generic")
    g = AmrSolver(wl, max_levels=levels, block=8, eps=0.1, regrid_every=2)
    g.set_prim(wl.patches[0].prim)
    g.step(warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step(steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    nl, counts = g.levels()
    rc = g.check()[0]
    g.close()
    fine = n << (levels - 1)
    fw = W.detonation_copper_1d(fine, steps=0, explosive="generic")
    f = Solver.from_workload(fw)
    f.set_state(pack([fw.patches[0].prim]), kind=1)
    f.step(2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(f.stream)
    f.step(2 ** (levels - 1) * 10)
    e1.record(f.stream)
    torch.cuda.synchronize()
    ms_fine = e0.elapsed_time(e1) / 10
    f.close()
    return {"workload": f"1d_detonation_generic_explosive_{n} base, {levels} levels (effective {fine} cells)",
            "precision": "fp64", "ms_per_level0_step": ms, "levels_used": nl, "blocks_per_level": counts,
            "uniform_finest_ms_same_time": ms_fine, "speedup_vs_uniform_finest": ms_fine / ms,
            "status_ok": rc == 0,
            "note": "a single 1D problem: launch- and host-latency bound on either path"}


def _amr_case(kind, n):
    """Base workload of an AMR bench row: the 2D shock-disc on n x n cells
    (SSP-RK3 or MUSCL-Hancock), or its (r, z) form, the shock-sphere on
    n/2 x n cells."""
    from paper_2009_14555_gb300 import workloads as W
    if kind == "cylindrical":
        return W.sphere_shock_rz(n, steps=0, shock_z=0.3)
    wl = W.shock_disc_2d(n, steps=0, shock_x=0.3)
    if kind == "hancock":
        wl.scheme = "hancock"
    return wl


def amr_bench(n=256, levels=3, steps=12, warmup=2, kind="rk3"):
    """The structured AMR hierarchy (float64) on the 2D shock-disc (kind
    "rk3", "hancock") or the (r, z) shock-sphere (kind "cylindrical"): an
    n x n base (n/2 x n in (r, z)) and `levels` levels of ratio 2, block 16,
    flagging threshold 0.3, regrid every 4 level-0 steps; against the
    uniform grid of the finest resolution over the same physical time
    (2^(L-1) of its steps per level-0 step)."""
    import torch
    from paper_2009_14555_gb300.solver import AmrSolver, Solver
    wl = _amr_case(kind, n)
    nx0, ny0 = wl.patches[0].nx, wl.patches[0].ny
    g = AmrSolver(wl, max_levels=levels, block=16, eps=0.3, regrid_every=4)
    g.set_prim(wl.patches[0].prim)
    g.step(warmup)
    nl, counts = g.levels()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dts = g.step(steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    nl2, counts2 = g.levels()
    rc = g.check()[0]
    # cells each level owns (blocks of (2 x 16)^2 cells) and the level steps per level-0 step
    upd = nx0 * ny0 + sum(counts2[l] * (32 * 32) * 2 ** l for l in range(1, nl2))
    g.close()
    fine = n << (levels - 1)
    fw = _amr_case(kind, fine)
    f = Solver.from_workload(fw)
    from paper_2009_14555_gb300.solver import pack
    f.set_state(pack([fw.patches[0].prim]), kind=1)
    f.step(2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(f.stream)
    f.step(2 ** (levels - 1))
    e1.record(f.stream)
    torch.cuda.synchronize()
    ms_fine = e0.elapsed_time(e1)
    f.close()
    shape = (f"2d_shock_disc_{n}x{n}" if kind != "cylindrical" else f"2d_sphere_shock_rz_{n // 2}x{n} (x = r, y = z)")
    fx, fy = nx0 << (levels - 1), ny0 << (levels - 1)
    return {"workload": f"{shape} base, {levels} levels (finest {fx}x{fy}), block 16, eps 0.3",
            "precision": "fp64", "scheme": wl.scheme, "geometry": wl.geometry,
            "ms_per_level0_step": ms, "levels_used": nl2, "blocks_per_level": counts2,
            "cell_updates_per_level0_step": upd, "value": upd / (ms * 1e-3), "unit": UNIT,
            "finest_equivalent_cell_updates_per_s": fx * fy * 2 ** (levels - 1) / (ms * 1e-3),
            "uniform_finest_ms_same_time": ms_fine, "speedup_vs_uniform_finest": ms_fine / ms,
            "status_ok": rc == 0, "note": "wall time per level-0 step (the hierarchy synchronises each step); "
                                          "uniform: 2^(L-1) float64 steps of the finest grid, CUDA events"}


def hancock_bench(wl, prim, steps, warmup, precision="fp64"):
    """The step with the single-stage MUSCL-Hancock update on the same
    workload: cell-updates/s (device events, inputs resident).  FP32-bulk: one
    fused kernel per step, so the step time is the kernel's (plus the rate
    buffer's clear and copy), and the HBM fraction is that of the kernel."""
    import torch
    from paper_2009_14555_gb300.solver import Solver
    s = Solver.from_workload(wl, precision=precision, scheme="hancock")
    s.set_state(prim, kind=1)
    s.step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rc = s.check()[0]
    launches = s.launches
    out = {"value": wl.cells / (ms * 1e-3), "ms_per_step": ms, "steps": steps,
           "launches_per_step": launches // steps, "status_ok": rc == 0}
    if precision == "fp32_bulk":
        b = 2 * state_bytes(wl.dim, wl.reactive, precision)
        t = s.tile_choice()
        hbm = peaks()[0]
        gbs = b * wl.cells / (ms * 1e-3) / 1e9
        dram = HANCOCK32_DRAM.get(tuple(t[:2]))
        out.update(tile=list(t[:2]), tuned_ms_per_step=[round(float(x), 4) for x in t[3][:3]],
                   algorithmic_bytes_per_cell_update=b, hbm_frac=gbs / hbm,
                   roofline={"bound": "hbm", "kernel": f"k_hancock32<{t[0]}x{t[1]}> (one launch per step)",
                             "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                             "traffic": dram * wl.cells if dram else None,
                             "note": "algorithmic bytes of the step over the step time (one kernel per step "
                                     "plus the rate buffer's clear and copy)"})
    s.close()
    return out


def batch_bench(steps=300, warmup=3):
    """4096 independent 1D two-material problems (256-4096 cells, seed 3) in one
    batch, 300 steps in one dis_step call: cell-updates/s for both precisions
    (each problem has its own dt; FP32-bulk: the tuner's schedule, per-step
    launches or the persistent batch kernel), and the FP32-bulk single-stage
    MUSCL-Hancock form (one kernel per step)."""
    import torch
    from paper_2009_14555_gb300 import workloads as W
    from paper_2009_14555_gb300.solver import Solver, pack
    wl = W.batched_riemann_1d()
    prim = pack([p.prim for p in wl.patches])
    out = {"workload": "1d_batch_4096 (256-4096 cells log-uniform, seed 3)", "cells": wl.cells,
           "problems": len(wl.patches)}
    for prec in ("fp32_bulk", "fp64", "fp32_bulk_hancock"):
        scheme = "hancock" if prec.endswith("hancock") else "rk3"
        s = Solver.from_workload(wl, precision=prec.replace("_hancock", ""), scheme=scheme)
        s.set_state(prim, kind=1)
        s.step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        rc, bp, bc = s.check()
        # problems whose state left the finite range (each problem is independent)
        bad_ids = [k for k, a in enumerate(s.get_arrays()) if not np.isfinite(a).all()]
        bad = len(bad_ids)
        b = 2 * state_bytes(1, False, prec.replace("_hancock", ""))
        out[prec] = {"value": wl.cells / (ms * 1e-3), "ms_per_step": ms, "steps": steps,
                     "launches": s.launches, "nonfinite_problems": bad, "nonfinite_ids": bad_ids[:16],
                     "first_flagged": [int(bp), int(bc)] if rc else None,
                     "algorithmic_bytes_per_cell_update": b,
                     "hbm_frac": b * wl.cells / (ms * 1e-3) / 1e9 / peaks()[0]}
        if prec.startswith("fp32_bulk"):
            t = s.tile_choice()
            sc, bms = s.schedule()
            out[prec]["tile"] = list(t[:3])
            out[prec]["schedule"] = "persistent" if sc == 1 else "per-step launches"
            out[prec]["tuned_ms_per_step"] = [round(float(x), 4) for x in t[3]]
            out[prec]["tuned_ms_persistent_one_step"] = [round(float(x), 4) for x in bms]
        s.close()
    return out


def _oracle_rate(budget_s, steps, nx, ny):
    """Cell-updates/s of the float64 CPU oracle stepping the reactive plate on
    an nx x ny grid: `steps` steps, or as many as fit in budget_s (at least
    one); returns (rate, steps, seconds)."""
    from oracle import scheme as OS
    from oracle import closures as OC
    wl = workload(nx, ny)
    p = wl.patches[0]
    grid = OS.grid_of(p, 2)
    q = OC.prim_to_cons(OS.prim_from_array(p.prim, 2, True), wl.materials)
    t0 = time.perf_counter()
    n = 0
    while True:
        q, _ = OS.step(q, grid, wl.materials, dict(cfl=wl.cfl, thinc=wl.thinc))
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el > budget_s):
            break
    return nx * ny * n / el, n, el


def cpu_baseline(budget_s=15.0, steps=None, nx=256, ny=128, single_core_s=5.0):
    """The float64 CPU oracle on a bounded sample of the same workload (the
    reactive plate on an nx x ny grid) with all host threads, and (unless
    single_core_s is None) on one thread on a quarter of that grid."""
    import torch
    rate, n, el = _oracle_rate(budget_s, steps, nx, ny)
    out = {"value": rate, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
           "sample": f"{n} steps of the reactive plate at {nx}x{ny} (same physics, smaller grid)",
           "seconds": el}
    if single_core_s is None:
        return out
    threads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        r1, n1, el1 = _oracle_rate(single_core_s, None if steps is None else 1, nx // 2, ny // 2)
    finally:
        torch.set_num_threads(threads)
    out["single_core"] = {"value": r1, "unit": UNIT, "cores": 1,
                          "sample": f"{n1} steps of the reactive plate at {nx // 2}x{ny // 2}", "seconds": el1}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each step samples a grid sized so that the whole run stays near 90 s
    # (the oracle advances ~6e3 cells per second on 16 cores)
    per_step_s = 90.0 / (max(1, args.steps) + args.warmup)
    ny = int(max(8, min(128, np.sqrt(6.0e3 * per_step_s / 2.0))))
    nx = 2 * ny
    for _ in range(args.warmup):
        cpu_baseline(steps=1, nx=nx, ny=ny, single_core_s=None)
    res = cpu_baseline(steps=max(1, args.steps), nx=nx, ny=ny, single_core_s=None)
    line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["seconds"] / max(1, args.steps) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"2d_reactive_plate_{NX}x{NY}", "sample": res["sample"]},
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "cores": res["cores"],
                             "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 1D measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 1D solid|gas and 512^2 shock-disc measurements")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-case measurement")
    ap.add_argument("--no-widened", action="store_true",
                    help="skip the cylindrical-geometry and k sqrt(lam) measurements")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--nx", type=int, default=None, help="profiling only: smaller grid")
    ap.add_argument("--ny", type=int, default=None, help="profiling only: smaller grid")
    ap.add_argument("--variant", type=int, default=None,
                    help="profiling only: fix the FP32-bulk stage variant instead of tuning")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
