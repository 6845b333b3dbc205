"""Throughput of the fused D2Q8 porous MRT-LB step on GB300, in MLUPS and as a fraction of the
HBM roofline.

Default workload: lid-driven porous cavity 4096 x 4096 (eps = 0.4, Da = 1e-3, Re = 100, lid
velocity 0.1, halfway bounce-back walls, FP32 deviation storage, A-B pull streaming).  One
"step" is one time step of the whole lattice (gather, collision, store).  Prints ONE JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--precision fp32|fp16|bf16] [--size L]

Multi-GPU: the method has no cross-domain exchange in this workload set-up, so N ranks run N
independent replicas (weak scaling); value = all cells updated / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline (FP32 vs FP16 store); adjoint/forward time at stated err"
PREC = {"fp32": 0, "fp16": 1, "bf16": 2}
# algorithmic bytes per lattice update: 8 populations read + 8 written
BYTES_PER_LU = {"fp32": 64, "fp16": 32, "bf16": 32}


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values (the slowest rank's time), on every rank."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cavity_params(L):
    lid = 0.1
    return dict(nu=lid * L / 100.0, phi=0.4, K=1e-3 * L * L, lid=lid)


KERNEL_SOURCES = {"k_step": ("lbm_device.cuh", "tiles.cuh", "step.cu"), "k_step_ip": ("lbm_device.cuh", "inplace.cu")}


def source_hash(kernel="k_step"):
    """Hash of the sources that define a step kernel (a recorded ncu traffic figure is only
    reported while these are unchanged)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1311_7239_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel_key):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(kernel_key)
        if e and e.get("source_hash") == source_hash("k_step_ip" if kernel_key.startswith("k_step_ip") else "k_step"):
            return float(e["bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = "clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 3 + k and r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _oracle_job(job):
    """One oracle process: (L, side, warmup, steps, seconds) -> (cell updates, seconds, steps) of the
    FP64 oracle on a side x side sample of the L x L cavity; `steps` steps, or as many as fit in
    `seconds` when steps is 0."""
    import numpy as np

    from oracle import mrt_d2q8 as fl

    L, side, warmup, steps, seconds = job
    prm = cavity_params(L)
    flow = fl.Flow(nx=side, ny=side, phi=np.full((side, side), prm["phi"]), K=np.full((side, side), prm["K"]),
                   nu=prm["nu"], bc_x="wall", bc_y="wall", u_top=(prm["lid"], 0.0))
    f = fl.initial_state(flow)
    for _ in range(max(warmup, 1)):
        f = fl.step(f, flow)
    n = 0
    t0 = time.perf_counter()
    while (n < steps) if steps else (time.perf_counter() - t0 < seconds):
        f = fl.step(f, flow)
        n += 1
    return side * side * n, time.perf_counter() - t0, n


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_pool(jobs):
    """Run oracle jobs in fresh single-threaded processes (spawned, so safe after CUDA is up), one
    process per job, all at once."""
    import multiprocessing as mp

    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            return pool.map(_oracle_job, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu_baseline(L, seconds=6.0):
    """The FP64 oracle, as it stands, on bounded samples of the workload (square cavities with the
    workload's parameters) on this host's cores: one single-threaded process per core on its own
    512^2 sample (the aggregate is the value), and one process alone at 512^2, 1024^2 and 2048^2."""
    cores = host_cores()
    allc = oracle_pool([(L, 512, 1, 0, seconds)] * cores)
    total = sum(c for c, _, _ in allc) / max(t for _, t, _ in allc) / 1e6
    single = {}
    for side in (512, 1024, 2048):
        c, t, n = oracle_pool([(L, side, 1, 0, seconds)])[0]
        single[f"{side}x{side}"] = {"MLUPS": c / t / 1e6, "steps": n}
    return {"value": total, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{cores} single-threaded processes of the numpy FP64 oracle, each on its own 512x512 lid-driven "
                      f"porous cavity with the workload's eps, Da, nu, lid, for about {seconds:g} s; value = cells x steps "
                      f"of all processes / the longest process time",
            "host_nproc": os.cpu_count(), "single_core": single}


def run_reference(args, rank, world):
    """The oracle as it stands on this host's cores: one single-threaded process per core, each
    running W untimed and K timed steps of its own square sample of the workload, the sample side
    chosen so that the K steps take about a minute at most; value = all processes' cell updates /
    the longest process time."""
    if rank != 0:
        return 0
    L = args.size
    cores = host_cores()
    side = int(max(16, min(256, math.sqrt(60.0 / (max(args.steps, 1) * 1e-6)))))
    res = oracle_pool([(L, side, args.warmup, args.steps, 0.0)] * cores)
    dt = max(t for _, t, _ in res)
    mlups = sum(c for c, _, _ in res) / dt / 1e6
    b = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
         "sample": f"{cores} single-threaded processes of the numpy FP64 oracle, each on its own {side}x{side} lid-driven "
                   f"porous cavity with the workload's eps, Da, nu, lid"}
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"lid-driven porous cavity {L}x{L} (each step sampled on {cores} x {side}x{side}), eps=0.4, "
                                   f"Da=1e-3, Re=100, lid=0.1", "nx": L, "ny": L},
            "cpu_baseline": b, "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def make_lattice(lbm, L, prec, stream, streaming=0, walls="halfway"):
    """The benchmark cavity: halfway bounce-back walls, or the paper's wall nodes with
    non-equilibrium extrapolation (walls="nee")."""
    prm = cavity_params(L)
    bc = lbm.NEE if walls == "nee" else lbm.WALL
    cfg = lbm.default_config(nx=L, ny=L, bc_x=bc, bc_y=bc, nu=prm["nu"], phi=prm["phi"], K=prm["K"],
                             u_wall=[(0, 0), (0, 0), (0, 0), (prm["lid"], 0)], precision=PREC[prec], p_rest=prm["phi"],
                             dev_scale_log2=10, streaming=streaming)
    cfg.stream = stream.cuda_stream
    return lbm.Lattice(cfg)


def timed_steps(lbm, L, prec, steps, warmup, local_rank, dist=None, streaming=0, walls="halfway"):
    """(ms for `steps` steps, clock summary, lattice) with CUDA events on the lattice's stream."""
    import torch

    stream = torch.cuda.Stream()
    lat = make_lattice(lbm, L, prec, stream, streaming, walls)
    lat.bench_stream = stream  # the lattice's stream, for events
    lat.step(warmup)
    lat.sync()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        start.record(stream)
        lat.step(steps)
        stop.record(stream)
        stop.synchronize()
    torch.cuda.synchronize()
    lat.sync()
    return start.elapsed_time(stop), clk.summary(), lat


TARGETS = {"fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-3}  # relative L2 error against the FP64 oracle


def accuracy_record():
    """Relative L2 errors vs the FP64 oracle measured by the GPU parity tests (committed record),
    with a per-precision summary: the target, the worst recorded field error and whether it is met
    (BF16 storage misses its 1e-3 target; its runs are recorded, not counted as parity)."""
    try:
        with open(os.path.join(ROOT, "profiles", "accuracy.json")) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    summary = {}
    for c in rec.get("cases", []):
        prec = c.get("precision")
        if prec not in TARGETS:
            continue
        errs = [v for k, v in c.items() if k.startswith("rel_l2") and isinstance(v, float)]
        if not errs:
            continue
        s = summary.setdefault(prec, {"target": TARGETS[prec], "worst_rel_l2": 0.0, "cases": 0})
        s["worst_rel_l2"] = max(s["worst_rel_l2"], max(errs))
        s["cases"] += 1
    for s in summary.values():
        s["meets_target"] = s["worst_rel_l2"] <= s["target"]
    rec["by_precision"] = summary
    return rec


def inplace_form(lbm, L, steps, warmup, local_rank):
    """The benchmark cavity with in-place streaming (one population buffer): same bytes per update
    as the A-B form, half the population memory."""
    import torch

    out = {}
    peak, _ = peaks()
    for prec in ("fp32", "fp16"):
        ms, clk, lat = timed_steps(lbm, L, prec, steps, warmup, local_rank, streaming=1)
        mem = lat.memory_bytes()
        lat.close()
        torch.cuda.empty_cache()
        stream = torch.cuda.Stream()
        ab = make_lattice(lbm, L, prec, stream)
        mem_ab = ab.memory_bytes()
        ab.close()
        bw = BYTES_PER_LU[prec] * L * L * steps / (ms * 1e-3) / 1e9
        out[prec] = {"value": L * L * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "achieved_gbs": bw, "roofline_frac": bw / peak,
                     "algorithmic_bytes_per_lu": BYTES_PER_LU[prec], "steps": steps, "device_bytes": mem,
                     "device_bytes_ab": mem_ab, "clocks": clk}
    return {"workload": f"lid-driven porous cavity {L}x{L}, eps=0.4, Da=1e-3, Re=100, lid=0.1, in-place streaming", **out}


def wall_nodes_form(lbm, L, steps, warmup, local_rank):
    """The benchmark cavity with the paper's wall treatment (wall nodes with non-equilibrium
    extrapolation on all four sides) instead of halfway bounce-back, A-B and in-place streaming;
    in-place steps first compute the boundary nodes' states (one small extra launch per step)."""
    import torch

    out = {}
    peak, _ = peaks()
    for prec in ("fp32", "fp16"):
        for streaming in (0, 1):
            ms, clk, lat = timed_steps(lbm, L, prec, steps, warmup, local_rank, streaming=streaming, walls="nee")
            lat.close()
            torch.cuda.empty_cache()
            bw = BYTES_PER_LU[prec] * L * L * steps / (ms * 1e-3) / 1e9
            out[f"{prec}_{'inplace' if streaming else 'ab'}"] = {
                "value": L * L * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "achieved_gbs": bw, "roofline_frac": bw / peak,
                "algorithmic_bytes_per_lu": BYTES_PER_LU[prec], "steps": steps, "clocks": clk}
    return {"workload": f"lid-driven porous cavity {L}x{L}, eps=0.4, Da=1e-3, Re=100, lid=0.1, extrapolated wall nodes", **out}


def thermal_form(lbm, L, steps, warmup, local_rank):
    """Natural convection (D2Q8 flow + D2Q5 temperature in one pass), FP32: 104 B per update."""
    import torch

    from paper_1311_7239_gb300 import workloads

    out = {}
    peak, _ = peaks()
    for prec, bpl in (("fp32", 104), ("fp16", 52)):
        stream = torch.cuda.Stream()
        cfg = workloads.natural_convection(lbm, L=L, precision=PREC[prec])
        cfg.stream = stream.cuda_stream
        lat = lbm.Lattice(cfg)
        lat.step(warmup)
        lat.sync()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            start.record(stream)
            lat.step(steps)
            stop.record(stream)
            stop.synchronize()
        lat.sync()
        lat.close()
        ms = start.elapsed_time(stop)
        bw = bpl * L * L * steps / (ms * 1e-3) / 1e9
        out[prec] = {"value": L * L * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "achieved_gbs": bw, "roofline_frac": bw / peak,
                     "algorithmic_bytes_per_lu": bpl, "steps": steps, "clocks": clk.summary()}
    return {"workload": f"natural convection {L}x{L}, Ra=1e5, Pr=1, eps=0.6, Da=1e-2 (D2Q8 + D2Q5 fused)", **out}


def heterogeneous_form(lbm, L, steps, warmup, local_rank):
    """The bench cavity with a random medium (eps, K per cell: 72 B per update), in addition a
    per-cell viscosity ratio (J = 4 in the lower half: 76 B per update), and the random medium with
    FP16 storage (40 B per update)."""
    import numpy as np
    import torch

    from paper_1311_7239_gb300 import synth

    peak, _ = peaks()
    prm = cavity_params(L)
    eps, K = synth.heterogeneous_medium(L, L, H=L, seed=7, da_mean=1e-3, corr_len=32.0, eps_mean=0.4, eps_sd=0.05, eps_lo=0.2)
    J = np.where(np.arange(L)[:, None] < L // 2, 4.0, 1.0).astype(np.float32) * np.ones((L, L), np.float32)
    out = {}
    for name, prec, bpl, with_j in (("medium", "fp32", 72, False), ("medium_and_J", "fp32", 76, True),
                                    ("medium_fp16", "fp16", 40, False)):
        stream = torch.cuda.Stream()
        lat = make_lattice(lbm, L, prec, stream)
        lat.set_medium(torch.tensor(eps, dtype=torch.float32, device="cuda"), torch.tensor(K, dtype=torch.float32, device="cuda"))
        if with_j:
            lat.set_viscosity_ratio(torch.tensor(J, device="cuda"))
        lat.init_equilibrium(prm["phi"], 0.0, 0.0, phi_p_uniform=True)
        lat.step(warmup)
        lat.sync()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            start.record(stream)
            lat.step(steps)
            stop.record(stream)
            stop.synchronize()
        lat.sync()
        lat.close()
        ms = start.elapsed_time(stop)
        bw = bpl * L * L * steps / (ms * 1e-3) / 1e9
        out[name] = {"value": L * L * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "achieved_gbs": bw, "roofline_frac": bw / peak,
                     "algorithmic_bytes_per_lu": bpl, "steps": steps, "clocks": clk.summary()}
    return {"workload": f"lid-driven cavity {L}x{L}, random eps/K (and J = 4 in the lower half); FP32, and FP16 storage "
                        f"(medium_fp16)", **out}


def ensemble_form(lbm, steps, local_rank):
    """512 porous cavities/channels (sides 64..1024): batched persistent launch vs one by one."""
    import torch

    from paper_1311_7239_gb300 import workloads

    res = {}
    peak, _ = peaks()
    for key in ("fp32", "fp16", "fp32_inplace"):
        prec = key.split("_")[0]
        cfgs, media = workloads.ensemble(lbm, n=512, seed=42, precision=PREC[prec])
        if key.endswith("inplace"):  # one population pool updated in place
            for c in cfgs:
                c.streaming = lbm.STREAM_INPLACE
        b = workloads.build(lbm, cfgs, media)
        cells = b.info()["cells"]
        device_bytes = b.info()["bytes"]
        nt, k, _ = b.tune(steps=8)
        tiling = "flat" if b.get_tiling() == lbm.TILING_FLAT else "rows"
        ipc = b.get_items_per_cta()
        b.step(32)
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        with ClockSampler(local_rank) as clk:
            e0.record(s)
            b.step(steps)
            e1.record(s)
            e1.synchronize()
        ms_b = e0.elapsed_time(e1)
        each = max(2, min(steps // 16, 640))
        e0.record(s)
        b.step_each(each)
        e1.record(s)
        e1.synchronize()
        ms_e = e0.elapsed_time(e1)
        b.sync()
        b.close()
        bpl = BYTES_PER_LU[prec] + 8  # + per-cell eps and K
        mlups = cells * steps / (ms_b * 1e-3) / 1e6
        res[key] = {"batched_MLUPS": mlups, "one_by_one_MLUPS": cells * each / (ms_e * 1e-3) / 1e6,
                    "batched_roofline_frac": mlups * 1e6 * bpl / 1e9 / peak, "algorithmic_bytes_per_lu": bpl,
                    "launch": {"threads_per_cta": nt, "ctas_per_sm": k, "items_per_cta": ipc, "tiling": tiling},
                    "steps": steps,
                    "one_by_one_steps": each,
                    "device_bytes": device_bytes, "clocks": clk.summary()}
        torch.cuda.empty_cache()
    return {"workload": "512 heterogeneous porous cavities/channels, sides U{64..1024}, Re U[10,400], seed 42",
            "cells": cells, **res}


def adjoint_form(lbm, T):
    """Pressure-driven heterogeneous channel 2048x1024: adjoint (gradient of the outlet flux w.r.t.
    per-cell log K and eps, sqrt(T) checkpointing) time vs forward time."""
    import torch

    from paper_1311_7239_gb300 import workloads

    cfg, eps, logk = workloads.adjoint_channel(lbm)
    stream = torch.cuda.Stream()
    cfg.stream = stream.cuda_stream
    lat = lbm.Lattice(cfg)
    lat.set_medium_log(torch.tensor(eps, device="cuda"), torch.tensor(logk, device="cuda"))
    lat.init_equilibrium(float(cfg.p_rest), 0.0, 0.0, phi_p_uniform=True)
    lat.step(8)
    lat.sync()
    lat.init_equilibrium(float(cfg.p_rest), 0.0, 0.0, phi_p_uniform=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(T)
    e1.record(stream)
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    # first call: allocates the workspace (checkpoints, segment, adjoint state) that later calls reuse
    lat.init_equilibrium(float(cfg.p_rest), 0.0, 0.0, phi_p_uniform=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.adjoint(T, "flux")
    first_ms = (time.perf_counter() - t0) * 1e3
    # timed call, as in an optimisation loop
    lat.init_equilibrium(float(cfg.p_rest), 0.0, 0.0, phi_p_uniform=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L, gk, ge = lat.adjoint(T, "flux")
    adj_ms = (time.perf_counter() - t0) * 1e3
    finite = bool(torch.isfinite(gk).all() and torch.isfinite(ge).all())
    ws_gb = lat.memory_bytes() / 1e9
    lat.close()
    return {"workload": "pressure-driven heterogeneous channel 2048x1024, outlet-flux loss, T steps", "T": T,
            "forward_ms": fwd_ms, "adjoint_ms": adj_ms, "adjoint_over_forward": adj_ms / fwd_ms,
            "first_call_ms": first_ms, "device_GB_with_workspace": ws_gb, "loss": L,
            "gradients_finite": finite, "checkpoint_interval": int(math.ceil(math.sqrt(T))),
            "accuracy": "gradient vs FP64 oracle adjoint and central differences: tests/test_gpu_adjoint.py (1e-4 of max)"}


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_1311_7239_gb300 import lbm

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    L = args.size
    prm = cavity_params(L)
    prec = args.precision
    streaming = 1 if args.streaming == "inplace" else 0
    ms, clocks, lat = timed_steps(lbm, L, prec, args.steps, args.warmup, local_rank, dist, streaming, args.walls)
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
        dist.barrier()
    cells = L * L
    mlups = cells * args.steps * world / (ms * 1e-3) / 1e6

    # end to end through the C-ABI with host buffers: each step takes its wall velocities from
    # pinned host memory and returns the cavity-centre probe (p, u, v, T) to pinned host memory.
    # The loop a serving user runs: step t is enqueued before the host reads step t - 1's probe
    # (lbm_probe_async into one of two pinned buffers, an event per step), so the GPU never waits
    # for the host; every step's result is read on the host inside the timed region.
    stream = lat.bench_stream
    walls = torch.zeros(4, 2, dtype=torch.float32).pin_memory()
    walls[3, 0] = prm["lid"]
    probe = torch.zeros(4, dtype=torch.float32).pin_memory()
    probes = [torch.zeros(4, dtype=torch.float32).pin_memory() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(10, min(args.steps, 2000))
    for _ in range(max(3, args.warmup)):  # untimed: the first host-buffer calls set up their staging
        lat.set_walls(walls)
        lat.step(1)
        lat.probe(L // 2, L // 2, probe)
        lat.probe_async(L // 2, L // 2, probes[0])
    lat.sync()
    read = []

    def pipelined(n, every=0, fields=None):
        for k in range(n):
            lat.set_walls(walls)
            lat.step(1)
            lat.probe_async(L // 2, L // 2, probes[k & 1])
            evs[k & 1].record(stream)
            if every and (k + 1) % every == 0:
                lat.macros(*fields)
            if k:
                evs[(k - 1) & 1].synchronize()
                read.append(float(probes[(k - 1) & 1][1]))  # the host reads step k - 1's u
        evs[(n - 1) & 1].synchronize()
        read.append(float(probes[(n - 1) & 1][1]))

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pipelined(e2e_steps)
    e2e_s = time.perf_counter() - t0
    lat.sync()
    e2e_mlups = cells * e2e_steps * world / e2e_s / 1e6
    # the same with a probe that waits for its step (lbm_probe into pinned host memory)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.set_walls(walls)
        lat.step(1)
        lat.probe(L // 2, L // 2, probe)
    e2e_sync_s = time.perf_counter() - t0
    lat.sync()
    e2e_sync = {"value": cells * e2e_steps * world / e2e_sync_s / 1e6, "unit": "MLUPS", "steps": e2e_steps,
                "call": "lbm_set_walls(host) + lbm_step(1) + lbm_probe(host, waits for the step) per step"}
    # the pipelined loop with the fields a user reads: p, ux, uy of the whole lattice to pinned host
    # memory through lbm_macros every `every` steps
    every = 100
    fields = [torch.empty(L, L, dtype=torch.float32).pin_memory() for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pipelined(e2e_steps, every, fields)
    lat.sync()
    e2e_f_s = time.perf_counter() - t0
    e2e_fields = {"value": cells * e2e_steps * world / e2e_f_s / 1e6, "unit": "MLUPS", "every_steps": every,
                  "d2h_bytes_per_readout": int(sum(t.numel() for t in fields) * 4), "steps": e2e_steps,
                  "call": "as e2e, plus lbm_macros(p, ux, uy to pinned host memory) every 100 steps"}
    assert len(read) == 2 * e2e_steps and all(math.isfinite(v) for v in read)
    del fields
    lat.close()

    peak, peak_kind = peaks()
    forms = {}
    if not args.no_forms:
        for other in PREC:
            if other == prec:
                continue
            ms_o, clk_o, lat_o = timed_steps(lbm, L, other, max(3, args.steps // 2), args.warmup, local_rank, dist)
            lat_o.close()
            bw = BYTES_PER_LU[other] * cells / (ms_o * 1e-3 / max(3, args.steps // 2)) / 1e9
            forms[other] = {"value": cells * max(3, args.steps // 2) / (ms_o * 1e-3) / 1e6, "unit": "MLUPS",
                            "roofline_frac": bw / peak, "achieved_gbs": bw, "algorithmic_bytes_per_lu": BYTES_PER_LU[other],
                            "clocks": clk_o}
    if rank != 0:
        return 0
    bpl = BYTES_PER_LU[prec]
    achieved = bpl * cells / (ms * 1e-3 / args.steps) / 1e9
    kernel_key = (f"k_step_{prec}_uniform_{L}" if not streaming else f"k_step_ip_{prec}_uniform_{L}") + ("_nee" if args.walls == "nee" else "")
    traffic = traffic_for(kernel_key)
    line = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f32 (f16 storage)", "bf16": "f32 (bf16 storage)"}[prec], "data": "synthetic",
        "config": {"workload": f"lid-driven porous cavity {L}x{L}, eps=0.4, Da=1e-3, Re=100, lid=0.1, "
                               f"{prec} deviation storage, {'in-place' if streaming else 'A-B pull'} streaming"
                               + (", extrapolated wall nodes" if args.walls == "nee" else ""),
                   "nx": L, "ny": L, "precision": prec,
                   "l2": f"inputs larger than L2 ({1 if streaming else 2} population buffer(s) of {bpl // 2 * cells / 1e6:.0f} MB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs", "kernel": "k_step_ip" if streaming else "k_step",
                     "algorithmic_bytes_per_lu": bpl},
        "gpu_launches": args.steps,
        "e2e": {"value": e2e_mlups, "unit": "MLUPS", "h2d_bytes_per_step": int(walls.numel() * 4),
                "d2h_bytes_per_step": int(probe.numel() * 4), "steps": e2e_steps,
                "call": "lbm_set_walls(pinned host) + lbm_step(1) + lbm_probe_async(pinned host) per step; the host reads "
                        "each step's probe after enqueueing the next step",
                "synchronous_probe": e2e_sync, "with_field_readout": e2e_fields},
        "clocks": clocks,
    }
    if not args.no_forms:
        line["forms"] = forms
        line["forms"]["thermal"] = thermal_form(lbm, 2048, max(64, args.steps // 4), args.warmup, local_rank)
        line["forms"]["heterogeneous"] = heterogeneous_form(lbm, args.size, max(64, args.steps // 4), args.warmup, local_rank)
        line["forms"]["inplace"] = inplace_form(lbm, args.size, max(64, args.steps // 4), args.warmup, local_rank)
        line["forms"]["wall_nodes"] = wall_nodes_form(lbm, args.size, max(64, args.steps // 4), args.warmup, local_rank)
        line["forms"]["adjoint"] = adjoint_form(lbm, T=args.adjoint_steps)
        if not args.no_ensemble:
            line["forms"]["ensemble"] = ensemble_form(lbm, args.ensemble_steps, local_rank)
    acc = accuracy_record()
    if acc:
        line["accuracy"] = acc
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(L)
    print(json.dumps(line), flush=True)
    return 0


def run_case(args, local_rank):
    """One small run of a kernel family, for profiler captures (no timing output)."""
    import torch

    from paper_1311_7239_gb300 import lbm, workloads

    torch.cuda.set_device(local_rank)
    if args.case == "adjoint":  # heterogeneous pressure channel (default 1024x512), T = 64
        cfg, eps, logk = workloads.adjoint_channel(lbm, nx=args.adjoint_nx, ny=args.adjoint_nx // 2)
        lat = lbm.Lattice(cfg)
        lat.set_medium_log(torch.tensor(eps, device="cuda"), torch.tensor(logk, device="cuda"))
        lat.init_equilibrium(float(cfg.p_rest), 0.0, 0.0, phi_p_uniform=True)
        L, _, _ = lat.adjoint(64, "flux")
        lat.close()
        print(json.dumps({"case": "adjoint", "loss": L}))
    elif args.case == "batch":  # 64 lattices of the ensemble (--precision), one 64-thread CTA per work item
        cfgs, media = workloads.ensemble(lbm, n=64, seed=42, precision=PREC[args.precision])
        b = workloads.build(lbm, cfgs, media)
        b.set_launch(64, 0)
        b.step(8)
        b.sync()
        print(json.dumps({"case": "batch", **b.info()}))
        b.close()
    elif args.case == "nusselt":  # natural convection run to steady state, Nu vs Table 1 (3.451)
        L = args.size
        cfg = workloads.natural_convection(lbm, L=L, precision=PREC[args.precision])
        stream = torch.cuda.Stream()
        cfg.stream = stream.cuda_stream
        lat = lbm.Lattice(cfg)
        chunk, steps, prev, hist = 50000 if L > 512 else 20000, 0, None, []
        t0 = time.perf_counter()
        while steps < args.steps:
            lat.step(chunk)
            steps += chunk
            nl, nr = lat.nusselt(lbm.LEFT), lat.nusselt(lbm.RIGHT)
            hist.append((steps, nl, nr))
            if prev is not None and abs(nl - prev) <= 2e-5 * nl and abs(nl - nr) <= 1e-3 * nl:
                break
            prev = nl
        lat.close()
        print(json.dumps({"case": "nusselt", "L": L, "precision": args.precision, "steps": steps, "Nu_left": nl, "Nu_right": nr,
                          "table1_present": 3.451, "rel_diff": abs(nl - 3.451) / 3.451, "seconds": time.perf_counter() - t0,
                          "history": hist[-5:]}))
    elif args.case in ("fp16", "thermal", "inplace"):  # 2048^2 cavity FP16 storage / natural convection (--precision) /
        stream = torch.cuda.Stream()                     # cavity with in-place streaming (--precision)
        if args.case in ("fp16", "inplace"):
            cfg = make_lattice(lbm, 2048 if args.walls == "halfway" else args.size, "fp16" if args.case == "fp16" else args.precision,
                               stream, 1 if args.case == "inplace" else 0, args.walls).cfg
        else:
            cfg = workloads.natural_convection(lbm, L=2048, precision=PREC[args.precision])
            cfg.stream = stream.cuda_stream
        lat = lbm.Lattice(cfg)
        lat.step(10)
        lat.sync()
        lat.close()
        print(json.dumps({"case": args.case, "steps": 10}))
    return 0


def run_sweep(args, local_rank):
    """Throughput over lattice sizes (one JSON line per size and storage precision)."""
    import torch

    from paper_1311_7239_gb300 import lbm

    torch.cuda.set_device(local_rank)
    peak, peak_kind = peaks()
    for L in [int(v) for v in args.sweep.split(",")]:
        for prec in PREC:
            steps = max(64, int(args.steps * (4096 / L) ** 2))
            steps = min(steps, 64000) // 32 * 32
            ms, clk, lat = timed_steps(lbm, L, prec, steps, args.warmup, local_rank,
                                       streaming=1 if args.streaming == "inplace" else 0, walls=args.walls)
            lat.close()
            cells = L * L
            bw = BYTES_PER_LU[prec] * cells * steps / (ms * 1e-3) / 1e9
            l2 = 2 * BYTES_PER_LU[prec] // 2 * cells / 1e6
            print(json.dumps({"size": L, "precision": prec, "streaming": args.streaming, "steps": steps,
                              "MLUPS": cells * steps / (ms * 1e-3) / 1e6,
                              "achieved_gbs": bw, "roofline_frac": bw / peak, "peak_source": peak_kind,
                              "state_MB": l2, "l2_resident": l2 < 129.0, "clocks": clk}), flush=True)
            torch.cuda.empty_cache()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=list(PREC))
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--streaming", default="ab", choices=["ab", "inplace"],
                    help="population streaming of the main line and the sweep (A-B buffers or in-place)")
    ap.add_argument("--walls", default="halfway", choices=["halfway", "nee"],
                    help="cavity walls: halfway bounce-back, or wall nodes with non-equilibrium extrapolation")
    ap.add_argument("--no-cpu", action="store_true", help="skip the timed CPU oracle baseline")
    ap.add_argument("--no-forms", action="store_true", help="skip the other storage precisions")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 512-lattice ensemble form")
    ap.add_argument("--adjoint-steps", type=int, default=4000, help="T of the adjoint form")
    ap.add_argument("--ensemble-steps", type=int, default=10000, help="steps of the 512-lattice ensemble form")
    ap.add_argument("--adjoint-nx", type=int, default=1024, help="channel length of --case adjoint (height nx / 2)")
    ap.add_argument("--case", default="", choices=["", "adjoint", "batch", "fp16", "thermal", "nusselt", "inplace"],
                    help="run one small case of a kernel family (for profiler captures) and exit")
    ap.add_argument("--sweep", default="", help="comma-separated lattice sizes: print one line per size and precision")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.sweep:
        return run_sweep(args, local_rank)
    if args.case:
        return run_case(args, local_rank)
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
