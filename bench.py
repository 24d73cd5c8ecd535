#!/usr/bin/env python
"""Throughput of the PSM-LBM step (arXiv 2502.20049) on GB300: MLUPS and the
fraction of the HBM roofline, with the CPU oracle timed beside it.

One "step" is one pass of the whole hot path on one batch of cells: body poses,
remap of the geometry field onto eps, PSM collision (Eq. 4), streaming, and the
FP64 force/torque reduction -- one fused kernel launch (libpsm, psm_step).

Default workload: D3Q19 TRT, FP32 PDFs, 256^3 lattice, uniform inflow 0.05,
tau 0.55, an ellipsoid (semi-axes 40/20/8) rotating at 2e-4 rad/step about z
and remapped every step (synthetic data shaped like the paper's 256^3 GPU
block).

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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PSM-LBM MLUPS on 1×GB300 and % of HBM roofline; adjoint/forward step cost"
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes per cell update of the step kernel, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum over one launch / cells; one
# full-size launch of the 256^3 workload) for the workload, streaming, storage
# and kernel variant named in the key, as the kernel is now.
NCU_BYTES_PER_CELL = {
    "c2/twogrid/fp32/tma": 2.503963e9 / 16777216,
    "c2/twogrid/fp16/tma": 1.230960e9 / 16777216,
}


FLUID_NAME = {"bgk": "BGK", "trt": "TRT", "cumulant": "cumulant"}


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
    case = case.with_(streaming=streaming)
    return with_fluid(case, desc, fluid)


def reference_sample(name: str, fluid: str | None = None):
    """The bounded sample the CPU oracle runs per step: the same workload on a
    48^3 lattice with the body scaled by 48/n (about 0.1 MLUP per step)."""
    from paper_2502_20049_gb300 import workloads as W

    if name == "c2":
        case = W.c2_ellipsoid(scale=48 / 256, n=48, steps=1)
    elif name == "c5":
        case = W.c5_large(dims=(48, 48, 48), steps=1)
    else:
        case = W.c3_rotor(name.split("_")[1], scale=48 / 512, dims=(48, 48, 60), steps=1)
    return with_fluid(case, "", fluid)[0]


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
    """The oracle as it stands on this host's cores: `steps` steps of the full workload."""
    from oracle.cases import sim_from_case as oracle_sim

    case, _ = workload(name, "twogrid", fluid)
    case = case.with_(storage="fp64")
    sim = oracle_sim(case)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    mlups = case.cells * steps / dt / 1e6
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": sim.threads, "kind": "oracle",
            "sample": f"{steps} steps of the full {case.nx}x{case.ny}x{case.nz} workload, FP64 two-grid, "
                      f"{dt:.1f} s"}


def run_reference(args):
    from paper_2502_20049_gb300 import replicas

    rank, world, _ = replicas.env()
    if rank != 0:
        return
    from oracle.cases import sim_from_case as oracle_sim

    case = reference_sample(args.workload, args.fluid)
    sim = oracle_sim(case)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = case.cells * args.steps / dt / 1e6
    _, desc = workload(args.workload, args.streaming, args.fluid)
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sample_cells": case.cells},
            "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": sim.threads, "kind": "oracle",
                             "sample": f"each step one oracle step of the workload on a "
                                       f"{case.nx}x{case.ny}x{case.nz} lattice (body scaled to fit)"},
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


def variant_mlups(name, streaming, storage, kernel, steps, warmup, stream, fluid=None):
    """MLUPS of one storage / streaming / fluid-operator variant of the workload (same timing rules)."""
    from paper_2502_20049_gb300 import psm

    case, _ = workload(name, streaming, fluid)
    case = case.with_(storage=storage)
    sol = psm.Solver.from_case(case, stream=int(stream.cuda_stream))
    if kernel != "auto":
        sol.set_kernel_variant(kernel)
    sol.step(warmup)
    t = time_steps(sol, steps, stream)
    v = sol.kernel_variant
    sol.close()
    return {"mlups": round(case.cells * steps / t / 1e6, 1), "kernel": v,
            "hbm_gbs": round(2 * case.Q * psm.STORAGE_BYTES[storage] * case.cells * steps / t / 1e9, 1)}


def adjoint_cost(stream, steps: int = 512, K: int = 64):
    """Adjoint workload: 128^3 D3Q19 TRT FP32, rotating ellipsoid, checkpoint every
    K steps.  Returns forward and backward time per step and their ratio (backward
    includes the recompute of every segment)."""
    import time as _t

    from paper_2502_20049_gb300 import psm
    from paper_2502_20049_gb300 import workloads as W

    case = W.c4_adjoint(steps=steps)
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
                    "adjoint kernel, scalar sums), eps gradient written to a device tensor; its buffers are "
                    "allocated by psm_record"}


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
    sol = psm.Solver.from_case(case, stream=int(stream.cuda_stream))
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
    traffic = NCU_BYTES_PER_CELL.get(key)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": f"hbm_gbs of {peak_kind}",
                "traffic": None if traffic is None else round(traffic * cells),
                "algorithmic_bytes_per_cell": bpc, "kernel": f"k_step ({sol.kernel_variant} loads)"}

    # end to end through the public API: every step one psm_step call (the
    # pose rides in the launch parameters) and a synchronous read of that
    # step's force/torque into pinned host memory
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
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 48 * nb,
           "note": "per step: psm_step(h, 1) with the body poses as launch parameters, then psm_force_torque "
                   "into pinned host memory (synchronising)"}
    sol.close()

    line = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64"}.get(case.storage, "f32"), "data": "synthetic",
            "config": {"workload": desc, "cells": cells, "streaming": case.streaming, "storage": case.storage,
                       "stencil": f"D3Q{case.Q}", "parallelism": f"replicas x{world}",
                       "l2": f"PDF working set {cells * case.Q * psm.STORAGE_BYTES[case.storage] / 1e9:.2f} GB "
                             f"> 129 MB L2, no flush"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": args.steps}
    ck = clk.summary()
    if ck:
        line["clocks"] = ck
    if not args.no_extras:
        vs = {}
        for streaming, storage in (("twogrid", "fp16"), ("twogrid", "bf16"), ("aa", "fp32"), ("aa", "fp16")):
            if streaming == case.streaming and storage == case.storage:
                continue
            vs[f"{storage}/{streaming}"] = variant_mlups(args.workload, streaming, storage, "auto", 300, 5, stream,
                                                         fluid=args.fluid)
        # the cumulant operator (the paper's performance runs use it; D3Q19) on the same workload
        if case.Q == 19 and case.fluid != "cumulant":
            for streaming, storage in (("twogrid", "fp32"), ("twogrid", "fp16"), ("aa", "fp16")):
                vs[f"{storage}/{streaming}/cumulant"] = variant_mlups(args.workload, streaming, storage, "auto", 300,
                                                                       5, stream, fluid="cumulant")
        line["variants"] = vs
        # FP16-shifted storage against this storage, same streaming, one GPU each
        other = "fp16/" + case.streaming
        if case.storage == "fp32" and other in vs:
            line["fp16_over_fp32"] = round(vs[other]["mlups"] / (cells * args.steps / t / 1e6), 3)
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
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2", choices=["c2", "c5", "c3_fp32", "c3_fp16", "c3_bf16"])
    ap.add_argument("--streaming", default="twogrid", choices=["aa", "twogrid"])
    ap.add_argument("--storage", default=None, choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "plain", "tma"])
    ap.add_argument("--fluid", default=None, choices=["bgk", "trt", "cumulant"],
                    help="fluid operator (default: the workload's own)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
