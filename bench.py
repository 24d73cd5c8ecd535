#!/usr/bin/env python
"""Throughput of the PSM-LBM step (arXiv 2502.20049) on GB300: MLUPS and the
fraction of the HBM roofline, with the CPU oracle timed beside it.

One "step" is one pass of the whole hot path on one batch of cells: body poses,
remap of the geometry field onto eps, PSM collision (Eq. 4), streaming, and the
FP64 force/torque reduction -- one fused kernel launch (libpsm, psm_step).

Default workload (the largest single-GPU configuration): D3Q19 BGK, FP16
shifted PDF storage, AA pattern in place, 1024 x 1024 x 960 = 1.0e9 cells,
uniform inflow 0.04, tau 0.55, a synthetic counter-rotating rotor pair (6 and
5 twisted elliptic blades, span 240 cells) at +-3e-4 rad/step, remapped every
step.  Beside it (``variants``, each with its own roofline fraction): the
rotating-ellipsoid 256^3 D3Q19 TRT workload in FP32 / FP16 / BF16 / FP64 and
with the cumulant operator, the D3Q27 rotor workload 512 x 512 x 640 in FP32 /
FP16 / BF16, the 1e9-cell workload in FP32, FP16 / FP32 ratios per workload,
and the adjoint / forward step cost on 128^3.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); every rank runs its own replica of
the workload (weak scaling, no data-path collective); the time is the maximum
over ranks.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PSM-LBM MLUPS on 1×GB300 and % of HBM roofline; adjoint/forward step cost"
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes per cell update of the step kernel, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum over one launch / cells) for
# the workload, streaming, storage and kernel variant named in the key, as the
# kernel is now; the other keys report traffic null.
NCU_BYTES_PER_CELL = {
    # 256x256x240 case of the 1e9-cell rotor workload (one AA odd and one even
    # launch, 15,728,640 cells each): per cell, scaled to the full lattice
    "c5/aa/fp16/tma": (1.140013e9 + 1.137385e9) / 2 / 15728640,
}


FLUID_NAME = {"bgk": "BGK", "trt": "TRT", "cumulant": "cumulant"}

# streaming of each workload as configured (the 256^3 two-grid: measured
# faster than AA there; the D3Q27 and 1e9-cell runs in place)
DEFAULT_STREAMING = {"c2": "twogrid", "c3_fp32": "aa", "c3_fp16": "aa", "c3_bf16": "aa", "c5": "aa"}

# planes of the 1e9-cell workload the CPU oracle steps as its bounded sample:
# the full 1024 x 1024 cross-section through the front rotor's hub and blades
C5_SAMPLE_Z0, C5_SAMPLE_NZ = 358, 4


def with_fluid(case, desc, fluid):
    """The workload with another fluid operator (None: its own)."""
    if not fluid or fluid == case.fluid:
        return case, desc
    return case.with_(fluid=fluid), desc.replace(FLUID_NAME[case.fluid], FLUID_NAME[fluid], 1)


def workload(name: str, streaming: str, fluid: str | None = None, scale: float = 1.0):
    """The named workload; scale < 1 shrinks the lattice and the bodies alike
    (a small case of the same kernels, for profiling)."""
    from paper_2502_20049_gb300 import workloads as W

    def dims(*d):
        return tuple(int(round(v * scale)) for v in d)

    if name == "c2":
        n = dims(256)[0]
        case = W.c2_ellipsoid(scale=scale, n=n)
        body = "40/20/8" if scale == 1.0 else f"40/20/8 x{scale:g}"
        desc = (f"D3Q19 TRT FP32 {n}^3, inflow 0.05, tau 0.55, ellipsoid {body} rotating 2e-4 rad/step about z, "
                f"remap every step")
    elif name == "c5":
        d = dims(1024, 1024, 960)
        case = W.c5_large(dims=d)
        desc = f"D3Q19 BGK FP16-shifted {d[0]}x{d[1]}x{d[2]}, counter-rotating rotor x2, remap every step"
    elif name in ("c3_fp32", "c3_fp16", "c3_bf16"):
        d = dims(512, 512, 640)
        storage = name.split("_")[1]
        case = W.c3_rotor(storage, scale=scale, dims=d)
        desc = (f"D3Q27 BGK {storage.upper()}{'-shifted' if storage != 'fp32' else ''} {d[0]}x{d[1]}x{d[2]}, "
                f"counter-rotating rotor, remap every step")
    else:
        raise SystemExit(f"unknown workload {name}")
    case = case.with_(streaming=streaming or DEFAULT_STREAMING[name])
    return with_fluid(case, desc, fluid)


# the bounded sample the CPU oracle steps: planes [z0, z0 + nz) of the full
# workload (the whole x-y cross-section through the first body), about 4.2e6
# cells, with the bodies that reach those planes
SAMPLE_PLANES = {"c2": (96, 64), "c3_fp32": (232, 16), "c3_fp16": (232, 16), "c3_bf16": (232, 16),
                 "c5": (C5_SAMPLE_Z0, C5_SAMPLE_NZ)}


def oracle_sample(name: str, fluid: str | None = None):
    """(oracle Sim, description, cells) of the sample: the workload's own
    lattice, collision and bodies on a slab of its planes (the oracle's z0
    offset keeps world cell centres), FP64, equilibrium start."""
    import oracle

    case, desc = workload(name, None, fluid)
    z0, nz = SAMPLE_PLANES[name]
    cfg = oracle.Config(nx=case.nx, ny=case.ny, nz=nz, Q=case.Q, bc_z=0, rho0=case.rho0, u_in=tuple(case.u_in),
                        fluid={"bgk": 0, "trt": 1, "cumulant": 2}[case.fluid], tau=case.tau,
                        trt_lambda=case.trt_lambda, solid=case.solid, weighting=case.weighting,
                        cum_rates=tuple(case.cum_rates), z0=z0)
    sim = oracle.Sim(cfg)
    kept = 0
    for b in case.bodies:
        dims, lo = oracle.shape_box(b.kind, b.params)
        if (b.omega[0] == 0.0 and b.omega[1] == 0.0 and b.v[2] == 0.0
                and tuple(b.Q0) == (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)):
            zlo, zhi = b.R0[2] + lo[2] - 2.0, b.R0[2] + lo[2] + dims[2] + 2.0  # turning about z only
        else:
            reach = float(np.linalg.norm(np.maximum(np.abs(lo), np.abs(np.asarray(lo) + dims)))) + 2.0
            zlo, zhi = b.R0[2] - reach, b.R0[2] + reach
        if zhi < z0 or zlo > z0 + nz:
            continue  # never reaches the sampled planes
        sub, blo = oracle.voxelize(b.kind, b.params, b.s)
        sim.add_body(oracle.BodySpec(sub=sub, s=b.s, lo=blo, R0=tuple(b.R0), Q0=np.array(b.Q0),
                                     omega=tuple(b.omega), v=tuple(b.v)))
        kept += 1
    sim.init_eq(case.rho0, case.u_in)
    cells = case.nx * case.ny * nz
    sdesc = (f"FP64 oracle, planes {z0}..{z0 + nz - 1} ({case.nx}x{case.ny}x{nz} cells, {kept} of "
             f"{len(case.bodies)} bodies reach them) of: {desc}")
    return sim, sdesc, cells


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        loaded = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in loaded for k, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(loaded)}


def cpu_baseline(name: str, steps: int = 3, fluid: str | None = None):
    """The oracle as it stands on this host's cores: `steps` steps of the bounded sample."""
    sim, sdesc, cells = oracle_sample(name, fluid)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    mlups = cells * steps / dt / 1e6
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": sim.threads, "kind": "oracle",
            "sample": f"{steps} steps of the {sdesc}; {dt:.1f} s"}


def run_reference(args):
    from paper_2502_20049_gb300 import replicas

    rank, world, _ = replicas.env()
    if rank != 0:
        return
    sim, sdesc, cells = oracle_sample(args.workload, args.fluid)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = cells * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": sdesc, "sample_cells": cells},
            "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": sim.threads, "kind": "oracle",
                             "sample": f"each step one oracle step of the {sdesc}"},
            "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(sol, steps: int, stream) -> float:
    """Device time (s) of `steps` psm_step launches, CUDA events on the solver's stream."""
    import torch

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sol.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    sol.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def e2e_with_output(sol, args, cells, world, dist, nb, ft_out):
    """The end-to-end loop of the headline plus, every `--e2e-output-every`
    steps, the density and velocity of every cell (psm_get_macroscopic, FP64)
    copied into pinned host buffers allocated before the timed region.  None
    when the buffers would take more than a quarter of the host's free memory."""
    import torch

    from paper_2502_20049_gb300 import replicas

    # at least one export in the timed region (the interval shrinks to the step count)
    k = min(args.e2e_output_every, args.steps)
    need = 32 * cells
    free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    if k <= 0:
        return {"skipped": "--e2e-output-every 0"}
    if need > free // 4:
        return {"skipped": f"needs {need / 1e9:.1f} GB of pinned host memory, {free / 1e9:.1f} GB free"}
    rho = torch.empty(cells, dtype=torch.float64, pin_memory=True)
    u = torch.empty(3 * cells, dtype=torch.float64, pin_memory=True)
    sol.synchronize()
    t0 = time.perf_counter()
    exports = 0
    for s in range(args.steps):
        sol.step(1)
        for b in range(nb):
            sol.force_torque(b, sol.step_count - 1, 1, out=ft_out)
        if (s + 1) % k == 0:
            sol.macroscopic(rho, u)
            exports += 1
    t = replicas.max_over_ranks(dist, time.perf_counter() - t0, device="cuda")
    assert bool(torch.isfinite(rho[:: max(1, cells // 4096)]).all())
    return {"value": round(replicas.aggregate_rate(cells * args.steps, world, t) / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": 96 * nb, "d2h_bytes_per_step": round(48 * nb + need * exports / args.steps),
            "note": f"as e2e, and every {k} steps the density and velocity of every cell (psm_get_macroscopic, "
                    f"FP64, {need / 1e9:.2f} GB) copied to pinned host memory; {exports} exports in the timed "
                    f"region"}


def variant_mlups(name, streaming, storage, steps, warmup, stream, peak, fluid=None, geoms=None):
    """MLUPS and HBM roofline fraction of one storage / streaming / fluid-operator
    variant of a workload (same timing rules as the headline)."""
    from paper_2502_20049_gb300 import psm

    case, _ = workload(name, streaming, fluid)
    case = case.with_(storage=storage)
    sol = psm.Solver.from_case(case, stream=int(stream.cuda_stream), geoms=geoms)
    sol.step(warmup)
    t = time_steps(sol, steps, stream)
    v = sol.kernel_variant
    bpc = sol.bytes_per_cell_update()
    sol.close()
    gbs = bpc * case.cells * steps / t / 1e9
    return {"mlups": round(case.cells * steps / t / 1e6, 1), "kernel": v, "streaming": case.streaming,
            "hbm_gbs": round(gbs, 1), "frac": round(gbs / peak, 4), "bytes_per_cell": bpc, "steps": steps}


# variants measured beside the headline: (key, workload, streaming, storage, fluid, steps)
VARIANTS = [
    ("c2/fp32/twogrid", "c2", "twogrid", "fp32", None, 200),
    ("c2/fp16/twogrid", "c2", "twogrid", "fp16", None, 200),
    ("c2/bf16/twogrid", "c2", "twogrid", "bf16", None, 200),
    ("c2/fp64/twogrid", "c2", "twogrid", "fp64", None, 20),
    ("c2/fp32/aa", "c2", "aa", "fp32", None, 200),
    ("c2/fp16/aa", "c2", "aa", "fp16", None, 200),
    ("c2/fp32/twogrid/cumulant", "c2", "twogrid", "fp32", "cumulant", 200),
    ("c2/fp16/twogrid/cumulant", "c2", "twogrid", "fp16", "cumulant", 200),
    ("c3/fp32/aa", "c3_fp32", "aa", "fp32", None, 20),
    ("c3/fp16/aa", "c3_fp16", "aa", "fp16", None, 20),
    ("c3/bf16/aa", "c3_bf16", "aa", "bf16", None, 20),
    ("c5/fp32/aa", "c5", "aa", "fp32", None, 10),
    ("c5/fp16/aa", "c5", "aa", "fp16", None, 10),
]


def adjoint_cost(stream, steps: int = 512, K: int = 64):
    """Adjoint workload: 128^3 D3Q19 TRT FP32, rotating ellipsoid, checkpoint every
    K steps.  Returns forward and backward time per step and their ratio (backward
    includes the recompute of every segment)."""
    import time as _t

    from paper_2502_20049_gb300 import psm
    from paper_2502_20049_gb300 import workloads as W

    case = W.c4_adjoint(steps=steps)
    # warm-up: one short recorded run and its backward pass (loads the kernels)
    warm = psm.Solver.from_case(case, stream=int(stream.cuda_stream))
    warm.record(4, init_from_inflow=True)
    warm.step(8)
    warm.backward()
    warm.close()
    sol = psm.Solver.from_case(case, stream=int(stream.cuda_stream))
    sol.step(4)
    t_fwd = time_steps(sol, steps, stream)
    sol2 = psm.Solver.from_case(case, stream=int(stream.cuda_stream))
    sol2.record(K, init_from_inflow=True)
    t_rec = time_steps(sol2, steps, stream)
    import torch

    # the eps gradient stays in HBM (a device tensor, as the autograd path uses)
    ge = torch.empty((case.nz, case.ny, case.nx), dtype=torch.float64, device="cuda")
    t0 = _t.perf_counter()
    sol2.backward(grad_eps=ge)
    t_bwd = _t.perf_counter() - t0
    sol.close()
    sol2.close()
    return {"workload": f"D3Q19 TRT FP32 128^3, rotating ellipsoid 20/10/4, {steps} steps, checkpoint every {K}",
            "forward_ms_per_step": round(t_fwd / steps * 1e3, 4),
            "recorded_forward_ms_per_step": round(t_rec / steps * 1e3, 4),
            "backward_ms_per_step": round(t_bwd / steps * 1e3, 4),
            "ratio": round(t_bwd / t_fwd, 3),
            "note": "backward: wall time of psm_backward (recompute of every segment with the TMA step kernel, "
                    "on a second stream one segment ahead of the adjoint sweep; adjoint kernel; scalar sums), "
                    "eps gradient written to a device tensor; its buffers are allocated by psm_record; after "
                    "one warm-up backward pass of 8 steps"}


def run_ours(args):
    import torch

    import __graft_entry__ as G
    from paper_2502_20049_gb300 import replicas

    rank, world, local = replicas.env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the product path has no CPU fallback)")
    torch.cuda.set_device(local)
    dist = replicas.init()
    G.build()
    from paper_2502_20049_gb300 import psm

    if args.adjoint_only:
        # the adjoint workload alone (for profiling the backward kernels)
        print(json.dumps({"adjoint": adjoint_cost(torch.cuda.current_stream())}), flush=True)
        return
    case, desc = workload(args.workload, args.streaming, args.fluid, args.scale)
    if args.storage:
        case = case.with_(storage=args.storage)
        desc = desc.replace("FP32", args.storage.upper()).replace("FP16-shifted", args.storage.upper())
    stream = torch.cuda.current_stream()
    geoms = {}
    sol = psm.Solver.from_case(case, stream=int(stream.cuda_stream), geoms=geoms)
    if args.kernel != "auto":
        sol.set_kernel_variant(args.kernel)
    cells = case.cells
    sol.step(args.warmup)
    torch.cuda.synchronize()
    replicas.barrier(dist)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t = time_steps(sol, args.steps, stream)
    replicas.barrier(dist)
    t_max = replicas.max_over_ranks(dist, t, device="cuda")
    value = replicas.aggregate_rate(cells * args.steps, world, t_max) / 1e6
    ms = t_max / args.steps * 1e3

    # roofline of the step kernel (the only kernel in the step): algorithmic
    # bytes per launch = 2 Q b per cell (one read, one write of every PDF)
    bpc = sol.bytes_per_cell_update()
    achieved = bpc * cells / (t / args.steps) / 1e9
    peak, peak_kind = peaks()
    key = f"{args.workload}/{case.streaming}/{case.storage}/{sol.kernel_variant}" + (
        f"/{args.fluid}" if args.fluid else "")
    traffic = NCU_BYTES_PER_CELL.get(key) if args.scale == 1.0 else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": f"hbm_gbs of {peak_kind}",
                "traffic": None if traffic is None else round(traffic * cells),
                "algorithmic_bytes_per_cell": bpc, "kernel": f"k_step ({sol.kernel_variant} loads)"}

    # end to end through the public API: every step one psm_step call (the
    # bodies' poses travel as launch parameters) and a synchronous read of that
    # step's force/torque of every body into pinned host memory; the PDF state
    # is the solver's own and stays in HBM
    nb = len(case.bodies)
    out = torch.empty((1, 6), dtype=torch.float64, pin_memory=True)
    sol.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sol.step(1)
        for b in range(nb):
            sol.force_torque(b, sol.step_count - 1, 1, out=out)
    t_e2e = replicas.max_over_ranks(dist, time.perf_counter() - t0, device="cuda")
    e2e = {"value": round(replicas.aggregate_rate(cells * args.steps, world, t_e2e) / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": 96 * nb, "d2h_bytes_per_step": 48 * nb,
           "note": "per step: psm_step(h, 1), whose input is each body's pose (rotation and position, 12 doubles "
                   "per body, computed on the host and passed as launch parameters), then psm_force_torque of "
                   "every body into pinned host memory (synchronising); no PDF state is copied: it is the "
                   "solver's state and stays in HBM"}
    e2e_out = e2e_with_output(sol, args, cells, world, dist, nb, out)
    kernel = sol.kernel_variant
    sol.close()

    line = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64"}.get(case.storage, "f32"), "data": "synthetic",
            "config": {"workload": desc, "cells": cells, "streaming": case.streaming, "storage": case.storage,
                       "stencil": f"D3Q{case.Q}", "parallelism": f"replicas x{world}",
                       "l2": f"PDF working set {cells * case.Q * psm.STORAGE_BYTES[case.storage] / 1e9:.2f} GB "
                             f"> 129 MB L2, no flush"},
            "roofline": roofline, "e2e": e2e, "e2e_output": e2e_out, "gpu_launches": args.steps}
    ck = clk.summary()
    if ck:
        line["clocks"] = ck
    if not args.no_extras:
        vs = {}
        for vkey, name, streaming, storage, fluid, steps in VARIANTS:
            same = (name == args.workload and streaming == case.streaming and storage == case.storage
                    and fluid == args.fluid and args.scale == 1.0)
            if same:
                vs[vkey] = {"mlups": round(cells * args.steps / t / 1e6, 1), "kernel": kernel,
                            "streaming": case.streaming, "hbm_gbs": round(achieved, 1),
                            "frac": round(achieved / peak, 4), "bytes_per_cell": bpc, "steps": args.steps,
                            "note": "the headline run"}
                continue
            vs[vkey] = variant_mlups(name, streaming, storage, steps, 3, stream, peak, fluid=fluid, geoms=geoms)
        line["variants"] = vs
        # FP16-shifted storage against FP32, same workload and streaming, one GPU each
        ratios = {}
        for wl, st in (("c2", "twogrid"), ("c2", "aa"), ("c3", "aa"), ("c5", "aa")):
            a, b = vs.get(f"{wl}/fp16/{st}"), vs.get(f"{wl}/fp32/{st}")
            if a and b:
                ratios[f"{wl}/{st}"] = round(a["mlups"] / b["mlups"], 3)
        a, b = vs.get("c2/fp16/twogrid/cumulant"), vs.get("c2/fp32/twogrid/cumulant")
        if a and b:
            ratios["c2/twogrid/cumulant"] = round(a["mlups"] / b["mlups"], 3)
        line["fp16_over_fp32"] = ratios
        line["adjoint"] = adjoint_cost(stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, fluid=args.fluid)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c5", choices=["c2", "c5", "c3_fp32", "c3_fp16", "c3_bf16"])
    ap.add_argument("--streaming", default=None, choices=["aa", "twogrid"],
                    help="default: the workload's own (two-grid for c2, AA for c3 and c5)")
    ap.add_argument("--storage", default=None, choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "plain", "tma"])
    ap.add_argument("--fluid", default=None, choices=["bgk", "trt", "cumulant"],
                    help="fluid operator (default: the workload's own)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-output-every", type=int, default=100,
                    help="steps between the macroscopic exports of the second end-to-end loop, at most --steps "
                         "(0: skip it)")
    ap.add_argument("--no-extras", action="store_true", help="skip the variant and adjoint measurements")
    ap.add_argument("--adjoint-only", action="store_true", help="only the adjoint cost measurement")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload's lattice and bodies (a small case for profiling; not a bench line)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
