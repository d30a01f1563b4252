#!/usr/bin/env python3
"""Benchmark of the FTLE hot path: FTLE points/s for one pass of the whole path (RK4 flowmap,
least-squares gradient / Cauchy-Green / lambda_max / FTLE, FP64 refinement of float-sensitive
nodes) over a synthetic workload, inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 2] [--impl ours|reference]

Default workload: 256^3 jittered Kuhn tetrahedral mesh (16,777,216 nodes, 14-neighbour lists)
over [0,2pi]^3, ABC flow A=sqrt(3) B=sqrt(2) C=1, RK4 dt=0.01 over T=5 (500 steps),
compensated-float advection with the FP64 path for float-sensitive nodes; the gradient reads the
paper's fixed-width -1-padded neighbour list.  --workload 1 is the 2048 x 1024 jittered
triangle mesh with the double gyre (T = 15), 3 the 64-instance batch, 4 the differentiable one.
Launch shapes come from the autotuner (tuned outside the timed region).

Each step's kernels are bracketed by CUDA events on the launching stream; L2 is flushed by a
320 MiB write between steps, outside the events.  Prints one JSON line (rank 0).
`--impl reference` times the FP64 CPU oracle on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "FTLE points/sec (flowmap+gradient+lambda_max) at stated tol"
UNIT = "points/s"
FLUSH_BYTES = 320 << 20


# Algorithmic FP32 flops of one compensated RK4 step per node as the kernels take it (FMA = 2
# flops; one sincospi or sincos counted as 20 flops: argument reduction plus degree-7/8 minimax
# polynomials; a small-angle rotation of a (sin, cos) pair 15).
#   double gyre: stage one 74 (error-free f 17, two sincospi 40, first-order corrections 10,
#                slope and velocity 7), per-step terms 6, stage two 39 (two rotations without
#                the fourth-order cosine term 26, angles 7, slope 2, increment 1, velocity 3),
#                stage four 43 (two rotations 30, the same 13), stage three 27 (angles and
#                their differences 11, four first-order turns 12, slope and velocity 4), update
#                22 (the step scale in two parts)
#   ABC:         stage one 87 when evaluated afresh (three compensated sincos 78, increments 9)
#                or 24 when carried from the previous step (stage four's three pairs turned to
#                first order by the rest of the step's increment 15, increments 9; fresh once
#                every abc_refresh = 8 steps), stage two 48 (three rotations without the
#                fourth-order cosine term 39, increments 9), stage three 24 (three first-order
#                turns 15, increments 9), stage four 54 (three rotations 45, increments 9) or 48
#                on a carried step (its rotations without that term, as at stage two), update 27
ABC_REFRESH = 8
FLOPS_PER_POINT_STEP = {"dg": 211, "abc": 240 - (63 + 6) * (ABC_REFRESH - 1) / ABC_REFRESH}


def peak_fp32_tflops(sms: int, mhz: float) -> float:
    """FP32 FMA throughput: 128 lanes per SM, 2 flops per FMA."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def load_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "fallback": True}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.out = Path(os.environ.get("TMPDIR", "/tmp")) / f"ftle_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in self.out.read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.bus_id and self.bus_id[-12:] not in parts[1].lower():
                continue
            rows.append(parts)
        self.out.unlink(missing_ok=True)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    from paper_2408_02758_gb300 import dist as D

    r = D.from_env()
    return r.world, r.rank, r.local


# ----------------------------------------------------------------------------- workload description

L2_NOTE = "flushed between steps (320 MiB write, outside the events)"


def layout_of(args) -> str:
    return "stencil" if args.stencil else ("csr" if args.csr else "ell")


def workload_config(w, world: int, layout: str) -> dict:
    """The `config` of a single-problem line; both arms print the same one."""
    import numpy as np

    width = int(np.diff(w.mesh.row_ptr).max()) if w.mesh.n_nodes else 0
    return {"workload": w.name, "nodes": w.mesh.n_nodes, "nnz": w.mesh.nnz, "steps_rk4": w.n_steps, "T": w.T,
            "dt": w.dt, "precision": w.precision, "l2": L2_NOTE,
            "neighbours": {"stencil": "implicit lattice stencil", "csr": "CSR rows",
                           "ell": f"fixed-width list, width {width} (-1 padded)"}[layout],
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def batched_config(wl_all, world: int) -> dict:
    return {"workload": "dg2d_batched_64", "instances": len(wl_all), "nodes": sum(w.mesh.n_nodes for w in wl_all),
            "node_steps": sum(w.mesh.n_nodes * w.n_steps for w in wl_all), "precision": "fp32c",
            "parallelism": f"instances split longest-first over {world} GPUs" if world > 1 else "single GPU",
            "l2": "flushed between steps", "execution": "one CUDA graph (persistent LPT queues)"}


def differentiable_config(w) -> dict:
    return {"workload": w.name, "nodes": w.mesh.n_nodes, "steps_rk4": w.n_steps, "ckpt_every": w.extra["ckpt_every"],
            "precision": "fp32c", "loss": "mean FTLE over nodes with x0 in [0.5, 1.5]", "l2": "flushed between steps"}


# ----------------------------------------------------------------------------- CPU oracle leg


def oracle_window(w, rows_lo: int, rows_hi: int):
    """Oracle FTLE of lattice rows [rows_lo, rows_hi) of a 2D workload (nodes plus a one-row halo)."""
    import numpy as np

    import oracle as O

    nx = w.mesh.shape[0]
    nodes = np.arange(rows_lo * nx, rows_hi * nx)
    t0 = time.perf_counter()
    out = O.ftle_sample(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, nodes, w.T, w.dt)
    return len(nodes), time.perf_counter() - t0, out


def oracle_block(w, n_nodes: int, seed: int = 0):
    """Oracle FTLE of a contiguous block of nodes of any workload (2D or 3D)."""
    import numpy as np

    import oracle as O

    start = (seed * 7919 * 1024) % max(1, w.mesh.n_nodes - n_nodes)
    nodes = np.arange(start, start + n_nodes)
    t0 = time.perf_counter()
    O.ftle_sample(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, nodes, w.T, w.dt)
    return len(nodes), time.perf_counter() - t0


def cpu_sample_size(w, target_s: float) -> int:
    """Nodes of the workload the oracle processes in about target_s seconds on this host."""
    import oracle as O

    probe = 2048 if w.mesh.dim == 2 else 1024
    n, dt = oracle_block(w, probe)
    rate = n / max(dt, 1e-3)
    del O
    return int(max(probe, min(w.mesh.n_nodes // 2, rate * target_s)))


def run_reference(args, w, world, rank):
    """FP64 CPU oracle as the reference arm: each step a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle as O

    O.build()
    n_per_step = cpu_sample_size(w, 4.0)
    for k in range(args.warmup):
        oracle_block(w, n_per_step, seed=k)
    times = []
    for k in range(args.steps):
        n, dt = oracle_block(w, n_per_step, seed=args.warmup + k)
        times.append(dt)
    value = n_per_step * args.steps / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, world, layout_of(args)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{n_per_step} contiguous nodes of {w.name} per step (full path: RK4 + QR "
                                   f"least squares + Jacobi), their neighbours advected too"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- batched workload


def run_batched(args, world, rank, local):
    """64 double-gyre instances of uneven size and horizon, replayed from one captured CUDA graph;
    compared with the same instances run one by one through ftle_compute."""
    import numpy as np

    from paper_2408_02758_gb300 import inputs as I

    from paper_2408_02758_gb300 import dist as D

    wl_all = I.batched_preset(64, scale=args.scale)
    total = sum(w.mesh.n_nodes for w in wl_all)
    ranks = D.Ranks(world, rank, local)
    # one GPU per rank; the ranks split the instances longest-first (no data-path collective)
    mine = D.lpt_assign([w.mesh.n_nodes * w.n_steps for w in wl_all], world)[rank]
    wl = [wl_all[i] for i in mine]
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle as O

        O.build()
        small = sorted(wl, key=lambda w: w.mesh.n_nodes * w.n_steps)[:8]
        t0 = time.perf_counter()
        done = 0
        for w in small:
            O.ftle(w.flow.kind, w.flow.params, w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, w.T, w.dt)
            done += w.mesh.n_nodes
        dt = time.perf_counter() - t0
        v = done / dt
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
                          "steps": 1, "warmup": 0, "ms_per_step": 1000 * dt, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": batched_config(wl_all, world),
                          "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                                           "sample": f"the 8 cheapest of 64 instances ({done} nodes)"},
                          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    import torch

    from paper_2408_02758_gb300 import ftle

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    D.init(ranks, "nccl", dev)
    ftle.lib()
    meshes = [ftle.DeviceMesh.from_mesh(w.mesh, device=dev) for w in wl]
    outs = [torch.empty(w.mesh.n_nodes, dtype=torch.float32, device=dev) for w in wl]
    ws = ftle.workspace_empty(ftle.ftle_batch_workspace_bytes(meshes, "fp32c"), device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    from paper_2408_02758_gb300 import autotune

    # launch shapes from the autotuner, tuned before the timed region (scheduling only: the
    # per-node arithmetic, hence every result, is the same for every candidate)
    with torch.cuda.stream(stream):
        tuned = autotune.params_for_batch(meshes, [w.flow for w in wl], [w.T for w in wl], 0.01, "fp32c")
    plan = ftle.BatchPlan(meshes, [w.flow for w in wl], [w.T for w in wl], 0.01, "fp32c", outs, ws,
                          options=ftle.make_options(**tuned), stream=sh)
    K, W = args.steps, args.warmup
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(W + K)]
    dopt = ftle.make_options(defer_fp64=True)  # FP64 pass of the flagged nodes once, after refinement
    with torch.cuda.stream(stream):
        for k in range(W + K):
            if k == W:
                torch.cuda.synchronize()
                D.barrier(ranks)
                clocks = ClockSampler(None)
                clocks.start()
                time.sleep(0.3)
            flush.fill_(float(k))
            ev[k][0].record(stream)
            plan.launch(stream=sh)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        D.barrier(ranks)
        clk = clocks.stop()
        # the same instances one at a time
        single = []
        for w, dm in zip(wl, meshes):
            ftle.compute(dm, w.flow, w.T, w.dt, "fp32c", stream=sh)
            flush.fill_(0.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ftle.compute(dm, w.flow, w.T, w.dt, "fp32c", stream=sh)
            e1.record(stream)
            torch.cuda.synchronize()
            single.append(e0.elapsed_time(e1))
    plan.destroy()
    ms = D.max_over_ranks(sum(ev[k][0].elapsed_time(ev[k][1]) for k in range(W, W + K)) / K, ranks, device=dev)
    single_sum = D.sum_over_ranks(sum(single), ranks, device=dev)
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    flops = sum(w.mesh.n_nodes * w.n_steps for w in wl_all) * FLOPS_PER_POINT_STEP["dg"] / world
    peak = peak_fp32_tflops(sms, float(peaks.get("sm_max_mhz", 2070.0)))
    ach = flops / (ms / 1000) / 1e12
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": total / (ms / 1000), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": batched_config(wl_all, world), "tuned": tuned,
        "roofline": {"kernel": "whole batched graph (k_batch_advect dominates)", "bound": "alu", "achieved": ach,
                     "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None},
        "single_instance_sum_ms": single_sum, "batched_speedup_vs_single": single_sum / ms / world,
        "clocks": clk, "gpu_launches": 5 * K, "cpu_baseline": None, "e2e": None}), flush=True)


# ----------------------------------------------------------------------------- differentiable workload


def run_differentiable(args, world, rank, local):
    """d(region-mean FTLE)/d(A, eps, omega) on the 1024 x 512 jittered triangle mesh, T = 15,
    checkpoints every 50 steps: forward (advection with checkpoints, FTLE core, refinement) plus
    the reverse-mode adjoint, against the plain forward path on the same GPU."""
    import numpy as np
    import torch

    from paper_2408_02758_gb300 import ftle
    from paper_2408_02758_gb300 import inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ftle.lib()
    w = I.preset(4, scale=args.scale)
    n = w.mesh.n_nodes
    ce = w.extra["ckpt_every"]
    dm = ftle.DeviceMesh.from_mesh(w.mesh, device=dev)
    wt = torch.from_numpy(w.extra["weights"]).float().to(dev)
    phi = ftle.flowmap_empty(2, n, "fp32c", device=dev)
    ck = ftle.checkpoints_empty(2, n, w.n_steps, ce, "fp32c", device=dev)
    out = ftle.ftle_out_empty(n, "fp32c", device=dev)
    ws = ftle.workspace_empty(ftle.ftle_workspace_bytes(n), device=dev)
    bws = ftle.workspace_empty(ftle.ftle_backward_workspace_bytes(n, 2), device=dev)
    grad = torch.empty(3, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    K, W = args.steps, args.warmup
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(W + K)]
    dopt = ftle.make_options(defer_fp64=True)  # FP64 pass of the flagged nodes once, after refinement
    with torch.cuda.stream(stream):
        for k in range(W + K):
            if k == W:
                torch.cuda.synchronize()
                clocks = ClockSampler(None)
                clocks.start()
                time.sleep(0.3)
            flush.fill_(float(k))
            e = ev[k]
            e[0].record(stream)  # plain forward
            ftle.ftle_compute(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi, out, None, ws, stream=sh)
            e[1].record(stream)
            flush.fill_(float(k))
            e[2].record(stream)  # forward with checkpoints + backward
            ftle.ftle_advect(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi, ck, ce, stream=sh)
            ftle.ftle_gradient_eig(dm, phi, "fp32c", w.T, out, None, ws, options=dopt, stream=sh)
            ftle.ftle_refine(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi, out, None, ws, options=dopt, stream=sh)
            ftle.ftle_backward(dm, w.flow, 0.0, w.T, w.dt, "fp32c", phi, ck, ce, wt, grad, bws, stream=sh)
            e[3].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
    fwd = statistics.mean(ev[k][0].elapsed_time(ev[k][1]) for k in range(W, W + K))
    both = statistics.mean(ev[k][2].elapsed_time(ev[k][3]) for k in range(W, W + K))
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC + " and d(region-mean FTLE)/d(A,eps,omega)", "value": n / (both / 1000), "unit": UNIT,
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": both, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": differentiable_config(w),
        "forward_only_ms": fwd, "forward_plus_backward_ms": both, "backward_over_forward": (both - fwd) / fwd,
        "gradient": grad.cpu().tolist(), "clocks": clk, "gpu_launches": 10 * K, "cpu_baseline": None, "e2e": None,
        "roofline": None}), flush=True)


def run_differentiable_reference(args, world, rank, local):
    """The FP64 oracle as the reference arm of the differentiable workload: its forward-mode
    derivative of the weighted FTLE sum, each step on a bounded sample of the region's nodes (a
    contiguous block of rows with their neighbours; the whole path: RK4 with tangents, QR least
    squares, Jacobi eigenvectors)."""
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    from paper_2408_02758_gb300 import inputs as I

    O.build()
    w = I.preset(4, scale=args.scale)
    wts = w.extra["weights"].astype(np.float64)
    region = np.flatnonzero(wts > 0)

    def sample_step(n_rows: int, k: int):
        start = (k * 7919 * 256) % max(1, len(region) - n_rows)
        rows = region[start:start + n_rows]
        sc, srp, sci, m = O.submesh(w.mesh.coords, w.mesh.row_ptr, w.mesh.col_idx, rows)
        sw = np.zeros(sc.shape[1])
        sw[:m] = wts[rows]
        t0 = time.perf_counter()
        O.param_grad(sc.astype(np.float64), srp, sci, w.flow.params[:3], w.T, w.dt, sw)
        return time.perf_counter() - t0

    probe = 1024
    rate = probe / max(sample_step(probe, 0), 1e-3)
    n_rows = int(max(probe, min(len(region) // 2, rate * 4.0)))
    for k in range(args.warmup):
        sample_step(n_rows, k)
    times = [sample_step(n_rows, args.warmup + k) for k in range(args.steps)]
    value = n_rows * args.steps / sum(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC + " and d(region-mean FTLE)/d(A,eps,omega)", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * sum(times) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": differentiable_config(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{n_rows} contiguous region nodes of {w.name} per step (forward-mode "
                                   f"derivative of their weighted FTLE, neighbours advected too)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


# ----------------------------------------------------------------------------- GPU arm


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", type=int, default=2,
                    help="preset index: 0 structured 2D, 1 triangle 2D, 2 tet 3D (default), 3 batched, "
                         "4 differentiable")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--csr", action="store_true",
                    help="gradient over the CSR rows instead of the fixed-width neighbour list")
    ap.add_argument("--stencil", action="store_true",
                    help="gradient over the lattice's implicit neighbours (no neighbour index read)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="lattice axes scaled by this factor (smaller cases for profiler captures)")
    ap.add_argument("--no-tune", action="store_true", help="default launch shapes instead of the autotuner's")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world, rank, local = dist_setup()
    from paper_2408_02758_gb300 import inputs as I

    if args.workload == 3:
        run_batched(args, world, rank, local)
        return
    if args.workload == 4:
        (run_differentiable if args.impl == "ours" else run_differentiable_reference)(args, world, rank, local)
        return
    w = I.preset(args.workload, scale=args.scale)

    if args.impl == "reference":
        run_reference(args, w, world, rank)
        return

    import numpy as np
    import torch

    from paper_2408_02758_gb300 import ftle

    from paper_2408_02758_gb300 import dist as D

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ranks = D.Ranks(world, rank, local)
    D.init(ranks, "nccl", dev)
    ftle.lib()

    # CPU baseline first (before any GPU work, so nothing forked or threaded interferes)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O

        O.build()
        n_cpu = cpu_sample_size(w, 12.0)
        n_done, t_cpu = oracle_block(w, n_cpu, seed=1)
        cpu = {"value": n_done / t_cpu, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
               "sample": f"{n_done} contiguous nodes of {w.name} (full path, FP64 oracle as it stands), "
                         f"{t_cpu:.1f} s"}

    dm = ftle.DeviceMesh.from_mesh(w.mesh, device=dev)
    if not args.csr:
        dm.attach_ell()  # mesh preparation, outside the timed region (like the CSR lists)
    if args.stencil:
        dm.attach_stencil({I.AXIS: ftle.STENCIL_AXIS, I.TRI: ftle.STENCIL_TRI, I.KUHN: ftle.STENCIL_KUHN}[
            w.mesh.meta["stencil"]], w.mesh.shape)
    prec = w.precision
    n = w.mesh.n_nodes
    phi = ftle.flowmap_empty(w.mesh.dim, n, prec, device=dev)
    out = ftle.ftle_out_empty(n, prec, device=dev)
    ws = ftle.workspace_empty(ftle.ftle_workspace_bytes(n), device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    K, W = args.steps, args.warmup
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(W + K)]
    # launch shapes from the autotuner, tuned before the timed region on this problem (scheduling
    # only: every candidate computes the same per-node arithmetic)
    tuned = {}
    if not args.no_tune:
        from paper_2408_02758_gb300 import autotune

        with torch.cuda.stream(stream):
            tuned = autotune.params_for_compute(dm, w.flow, w.T, w.dt, prec)
    # the calls ftle_compute makes, timed one by one: the flagged nodes' FP64 pass runs once, after
    # the re-advection (defer_fp64), as inside ftle_compute
    opt = ftle.make_options(defer_fp64=True, **tuned)

    def step(k):
        flush.fill_(float(k))
        e = ev[k]
        e[0].record(stream)
        ftle.ftle_advect(dm, w.flow, 0.0, w.T, w.dt, prec, phi, stream=sh)
        e[1].record(stream)
        ftle.ftle_gradient_eig(dm, phi, prec, w.T, out, None, ws, options=opt, stream=sh)
        e[2].record(stream)
        ftle.ftle_refine(dm, w.flow, 0.0, w.T, w.dt, prec, phi, out, None, ws, options=opt, stream=sh)
        e[3].record(stream)

    with torch.cuda.stream(stream):
        for k in range(W):
            step(k)
        torch.cuda.synchronize()
        D.barrier(ranks)
        torch.cuda.synchronize()
        bus = None
        try:
            bus = torch.cuda.get_device_properties(dev).pci_bus_id
        except Exception:
            bus = None
        clocks = ClockSampler(bus)
        clocks.start()
        time.sleep(0.3)
        t_wall = time.perf_counter()
        for k in range(W, W + K):
            step(k)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        D.barrier(ranks)
        clk = clocks.stop()
    counters = ftle.ftle_read_counters(ws, stream=sh)

    t_step = [ev[k][0].elapsed_time(ev[k][3]) for k in range(W, W + K)]
    t_adv = [ev[k][0].elapsed_time(ev[k][1]) for k in range(W, W + K)]
    t_grad = [ev[k][1].elapsed_time(ev[k][2]) for k in range(W, W + K)]
    t_ref = [ev[k][2].elapsed_time(ev[k][3]) for k in range(W, W + K)]
    ms = D.max_over_ranks(sum(t_step) / K, ranks, device=dev)  # the slowest rank sets the pace
    value = n * world / (ms / 1000.0)

    # end to end through the host-buffer entry point (pinned buffers, copies inside the timing)
    e2e = None
    if args.e2e_steps > 0:
        ch = torch.from_numpy(np.ascontiguousarray(w.mesh.coords)).pin_memory()
        rp = torch.from_numpy(w.mesh.row_ptr).pin_memory()
        ci = torch.from_numpy(w.mesh.col_idx).pin_memory()
        oh = torch.empty(n, dtype=torch.float64 if prec == "fp64" else torch.float32).pin_memory()
        hws = ftle.workspace_empty(ftle.ftle_host_workspace_bytes(w.mesh.dim, n, w.mesh.nnz, prec), device=dev)
        # the host-buffer call gathers through the CSR rows it copies: its gradient shape is tuned on
        # those rows (the advection's on the device path above)
        htuned = {k: v for k, v in tuned.items() if k.startswith("advect_")}
        if not args.no_tune:
            from paper_2408_02758_gb300 import autotune

            csr = ftle.DeviceMesh(dm.coords, dm.row_ptr, dm.col_idx)
            with torch.cuda.stream(stream):
                htuned.update(autotune.params_for_gradient(csr, phi, prec, w.T))
        hopt = ftle.make_options(**htuned)
        for _ in range(2):
            ftle.ftle_compute_host(ch, rp, ci, w.flow, 0.0, w.T, w.dt, prec, oh, hws, options=hopt, stream=sh)
        te = []
        gc.collect()
        gc.disable()  # wall-clock timing: no collector pass inside a call (as timeit does)
        try:
            for _ in range(args.e2e_steps):
                flush.fill_(0.0)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ftle.ftle_compute_host(ch, rp, ci, w.flow, 0.0, w.T, w.dt, prec, oh, hws, options=hopt, stream=sh)
                te.append(time.perf_counter() - t0)
        finally:
            gc.enable()
        h2d = ch.numel() * ch.element_size() + rp.numel() * 4 + ci.numel() * 4
        e2e = {"value": n / statistics.mean(te), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(oh.numel() * oh.element_size()),
               "ms_per_call": {"mean": 1e3 * statistics.mean(te), "median": 1e3 * statistics.median(te),
                               "min": 1e3 * min(te), "max": 1e3 * max(te),
                               "each": [round(1e3 * t, 3) for t in te]},
               "tuned": htuned or "defaults (--no-tune)"}
        del hws

    if rank != 0:
        return
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    kind = "dg" if w.flow.kind == I.DOUBLE_GYRE else "abc"
    adv_ms = statistics.mean(t_adv)
    flops = n * w.n_steps * FLOPS_PER_POINT_STEP[kind]
    achieved = flops / (adv_ms / 1000.0) / 1e12
    peak = peak_fp32_tflops(sms, float(peaks.get("sm_max_mhz", 2070.0)))
    nnz = w.mesh.nnz
    phi_b = 8 * w.mesh.dim * n if prec in ("fp32c", "fp64") else 4 * w.mesh.dim * n
    coord_b = w.mesh.coords.dtype.itemsize * w.mesh.dim * n
    idx_b = 0 if args.stencil else (4 * (n + 1) + 4 * nnz if args.csr else 4 * dm.desc.ell_width * n)
    grad_bytes = idx_b + coord_b + phi_b + (8 if prec == "fp64" else 4) * n
    grad_ms = statistics.mean(t_grad)
    prof = ROOT / "profiles" / f"traffic_{w.name}.json"
    traffic = json.loads(prof.read_text()) if prof.exists() else {}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(w, world, layout_of(args)), "tuned": tuned or "defaults (--no-tune)",
        "roofline": {"kernel": "k_advect (RK4 flowmap)", "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 flops x {peaks.get('sm_max_mhz', 2070.0)} MHz "
                                    "(max SM clock of measured peaks)",
                     "flops_per_point_step": FLOPS_PER_POINT_STEP[kind], "ms": adv_ms,
                     "traffic": traffic.get("k_advect"), "target_frac": 0.60,
                     "target_met": achieved / peak >= 0.60,
                     "measure": "algorithmic flops of the step as implemented / time (ncu's FP32-pipe busy "
                                "fraction, higher, is in profiles/)"},
        "roofline_gradient": {"kernel": "gradient stage (float gradient kernel + counter memset; the flagged nodes' FP64 pass runs in the refine stage)", "bound": "hbm",
                              "achieved": grad_bytes / (grad_ms / 1000.0) / 1e9, "peak": peaks.get("hbm_gbs"),
                              "unit": "GB/s", "frac": grad_bytes / (grad_ms / 1000.0) / 1e9 / peaks.get("hbm_gbs", 6800.0),
                              "bytes_per_launch": grad_bytes, "ms": grad_ms, "traffic": traffic.get("k_grad_f32"),
                              "target_frac": 0.70,
                              "target_met": grad_bytes / (grad_ms / 1000.0) / 1e9 / peaks.get("hbm_gbs", 6800.0) >= 0.70},
        "stage_ms": {"advect": adv_ms, "gradient": grad_ms, "refine": statistics.mean(t_ref),
                     "wall_per_step_incl_flush": 1000 * t_wall / K},
        "counters": counters,
        "clocks": clk,
        "gpu_launches": (6 if kind == "dg" else 5) * K,  # advect, gradient, mark, (a(t) table,) re-advect, FP64 pass
        "cpu_baseline": cpu,
        "e2e": e2e,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
