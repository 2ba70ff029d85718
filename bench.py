"""Benchmark: cell-updates/s (potential + acceleration) of tree build + gravity walk on one GB300.

Workload: isolated AMR mesh of 8^3-cell blocks, leaf levels 3-6 around a Plummer sphere (a = 0.05 L)
with 20 % log-normal noise: 4096 leaf-blocks = 2,097,152 cells.  One step = tree build (FP64 moments)
+ FP32-Kahan gravity walk with the BH MAC (theta = 0.5, eta_SB = 1.2); the APE walk
(a_lim = 1e-2 a_max) and the plain FP64 walk are timed beside it.  Inputs stay resident in HBM for
`value`; `e2e` repeats the step through the C ABI with the density copied from pinned host memory
and the potential/acceleration copied back inside the timed region.  L2 is flushed (a 256 MB write)
before every timed step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own independent problem (weak scaling, no collective on the data
path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/sec (potential+accel) on 1 GB300 at median accel err ≤1e-3 vs FP64 walk"
UNIT = "cell-updates/s"
WORKLOAD = "isolated AMR Plummer (a=0.05L) + 20% log-normal noise, leaf levels 3-6, 4096 blocks of 8^3 = 2,097,152 cells"

# algorithmic FP32 operations per unit of work of the walk
FLOPS_PER_INTERACTION = 20      # 3 sub, |d|^2 (5), r^-1/r^-3/m r^-3 (4), a (6), phi (2); rsqrt not counted
FLOPS_PER_MAC_BH = 15           # d (3), |d|^2 (5), theta^2 d^2 compare (1) + safe box 3 sub + 3 compare
FLOPS_PER_MAC_APE = 18          # APE: G M h^2 and a_lim d^4 (4 more)
SMS, FP32_LANES = 152, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def setup_problem(seed):
    from paper_1708_06142_gb300 import inputs
    return inputs.plummer_amr(seed=seed)


def cpu_baseline(mesh, rho, target_seconds=12.0, theta=0.5):
    """The FP64 oracle (tree build + BH walk) on a bounded random sample of target cells, all host cores."""
    from oracle import oracle
    from paper_1708_06142_gb300 import inputs
    nt = 512
    t0 = time.perf_counter()
    oracle.gravity_walk(mesh, rho, inputs.sample_cells(mesh.ncell, nt, seed=99), theta=theta)
    dt = time.perf_counter() - t0
    nt = int(min(mesh.ncell, max(1024, nt * target_seconds / max(dt, 1e-3))))
    tg = inputs.sample_cells(mesh.ncell, nt, seed=12345)
    t0 = time.perf_counter()
    oracle.gravity_walk(mesh, rho, tg, theta=theta)
    dt = time.perf_counter() - t0
    return {"value": nt / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle tree build + BH theta=0.5 walk for {nt} random target cells of the same "
                      f"2,097,152-cell mesh ({dt:.1f} s)", "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    mesh, rho = setup_problem(1)
    from oracle import oracle
    from paper_1708_06142_gb300 import inputs
    # each step: the oracle on a bounded sample sized so that warmup + steps stay within minutes
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    probe = inputs.sample_cells(mesh.ncell, 256, seed=7)
    t0 = time.perf_counter()
    oracle.gravity_walk(mesh, rho, probe, theta=0.5)
    dt = time.perf_counter() - t0
    nt = int(min(mesh.ncell, max(512, 256 * per_step / max(dt, 1e-3))))
    times = []
    for s in range(args.warmup + args.steps):
        tg = inputs.sample_cells(mesh.ncell, nt, seed=1000 + s)
        t0 = time.perf_counter()
        oracle.gravity_walk(mesh, rho, tg, theta=0.5)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = nt * len(times) / sum(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mac": "BH theta=0.5, eta_SB=1.2", "sample_cells_per_step": nt},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{nt} random target cells of the 2,097,152-cell mesh per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1708_06142_gb300.treesolver import TreeSolver

    mesh, rho = setup_problem(1 + rank)
    ncell = mesh.ncell
    stream = torch.cuda.Stream(device=dev)
    ts = TreeSolver(local, stream=stream)
    d_rho = torch.from_numpy(rho.reshape(-1)).to(dev)
    pot = torch.empty(ncell, dtype=torch.float32, device=dev)
    acc = torch.empty(ncell, 3, dtype=torch.float32, device=dev)
    pot64 = torch.empty(ncell, dtype=torch.float64, device=dev)
    acc64 = torch.empty(ncell, 3, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # setup (untimed): ingest the mesh, a_max for the APE limit, accuracy of FP32 vs the FP64 walk
    with torch.cuda.stream(stream):
        ts.tree_build(mesh, d_rho)
        ts.gravity_walk(pot64, acc64, theta=0.5, precision="fp64")
        ts.gravity_walk(pot, acc, theta=0.5)
    ts.sync()
    a64 = acc64.cpu().numpy()
    amax = float(np.linalg.norm(a64, axis=1).max())
    ea = np.linalg.norm(acc.double().cpu().numpy() - a64, axis=1) / amax
    accuracy = {"median_e_a_vs_fp64_walk": float(np.median(ea)), "p99_e_a_vs_fp64_walk": float(np.quantile(ea, 0.99)),
                "max_e_a_vs_fp64_walk": float(ea.max())}
    bh = ts.gravity_params(mac="bh", theta=0.5)
    ape = ts.gravity_params(mac="ape", a_lim=1e-2 * amax)
    bh64 = ts.gravity_params(mac="bh", theta=0.5, precision="fp64")

    def step(params, out_p, out_a):
        ts.tree_build(None, d_rho)
        ts.gravity_walk(out_p, out_a, params)

    def timed(params, out_p, out_a, K, W):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        walk_ms, step_ms, n_int, n_mac = [], [], 0, 0
        with torch.cuda.stream(stream):
            for _ in range(W):
                step(params, out_p, out_a)
            stream.synchronize()
            for k in range(K):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                ts.tree_build(None, d_rho)
                ev[k][1].record(stream)
                ts.gravity_walk(out_p, out_a, params)
                ev[k][2].record(stream)
            stream.synchronize()
        ts.sync()
        st = ts.stats()
        st.update(ts.walk_counters())
        for a, b, c in ev:
            step_ms.append(a.elapsed_time(c))
            walk_ms.append(b.elapsed_time(c))
        return np.array(step_ms), np.array(walk_ms), st

    # main timed region: BH FP32-Kahan
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    step_ms, walk_ms, st = timed(bh, pot, acc, args.steps, args.warmup)
    torch.cuda.synchronize()
    clocks = clk.stop()
    total_ms = float(step_ms.sum())
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * ncell * args.steps / (total_ms * 1e-3)

    # secondary measurements (same procedure, fewer steps)
    k2 = max(3, min(args.steps, 10))
    ape_ms, ape_walk, ape_st = timed(ape, pot, acc, k2, 2)
    f64_ms, f64_walk, f64_st = timed(bh64, pot64, acc64, k2, 2)

    # end to end through the C ABI from pinned host buffers
    h_rho = torch.from_numpy(rho.reshape(-1).copy()).pin_memory()
    h_pot = torch.empty(ncell, dtype=torch.float32).pin_memory()
    h_acc = torch.empty(ncell, 3, dtype=torch.float32).pin_memory()
    e2e_ms = []
    with torch.cuda.stream(stream):
        for k in range(args.warmup + args.steps):
            flush.fill_(float(k))
            stream.synchronize()
            t0 = time.perf_counter()
            d_rho.copy_(h_rho, non_blocking=True)
            ts.tree_build(None, d_rho)
            ts.gravity_walk(pot, acc, bh)
            h_pot.copy_(pot, non_blocking=True)
            h_acc.copy_(acc, non_blocking=True)
            stream.synchronize()
            if k >= args.warmup:
                e2e_ms.append(1e3 * (time.perf_counter() - t0))
    ts.sync()
    e2e_total = float(np.sum(e2e_ms))
    if world > 1:
        t = torch.tensor([e2e_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())

    walk_s = float(np.mean(walk_ms)) * 1e-3
    flops = FLOPS_PER_INTERACTION * st["interactions"] + FLOPS_PER_MAC_BH * st["mac_tests"]
    peak_fp32 = SMS * FP32_LANES * 2 * 2.07e9 / 1e12
    achieved = flops / walk_s / 1e12
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "walk_traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get("dram_bytes_per_launch")
        except Exception:
            traffic = None

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mac": "BH theta=0.5, eta_SB=1.2", "precision": "FP32 interactions + Kahan",
                       "step": "tree_build (FP64 moments) + gravity_walk", "cells": ncell,
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": f"independent problem per GPU x{world}"},
            "accuracy": accuracy,
            "walk_ms": float(np.mean(walk_ms)), "build_ms": float(np.mean(step_ms - walk_ms)),
            "interactions_per_cell": st["interactions"] / ncell, "mac_tests_per_cell": st["mac_tests"] / ncell,
            "lane_utilisation": st["active_lanes"] / (32.0 * max(1, st["pops"])), "pops_per_warp": st["pops"] / (ncell / 32),
            "ape": {"value": ncell * k2 / (ape_ms.sum() * 1e-3), "unit": UNIT, "a_lim": "1e-2 a_max",
                    "walk_ms": float(np.mean(ape_walk)), "interactions_per_cell": ape_st["interactions"] / ncell},
            "fp64_walk": {"value": ncell * k2 / (f64_ms.sum() * 1e-3), "unit": UNIT,
                          "walk_ms": float(np.mean(f64_walk))},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                         "frac": achieved / peak_fp32, "traffic": traffic,
                         "kernel": "k_gravity_walk<float, isolated, BH>",
                         "peak_note": "FP32 pipe: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (nominal unit counts and max clock)"},
            "e2e": {"value": world * ncell * args.steps / (e2e_total * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": ncell * 8, "d2h_bytes_per_step": ncell * 16},
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(mesh, rho)
        print(json.dumps(out), flush=True)
    ts.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
