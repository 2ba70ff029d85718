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
FLOPS_EWALD_CORR = 93           # trilinear correction: 3 scale, 3 frac, 3 (1-f), 16 weights, 64 FMA, 4 adds
FLOPS_MIMG = 9                  # minimum image, 3 axes x (mul, rint, fma)
FLOPS_EWALD_TAYLOR = 36         # nearest point 6, offsets 6, C 6, A_c 3 x 6, sign-restored sums 3 - 6 shared,
                                # displacement scaled by the FP16 Jacobian's scale 3
FLOPS_MLP = 17408               # 4-64-64-64-4 forward: 2 (4*64 + 64*64 + 64*64 + 64*4) BF16 tensor flops
FLOPS_COL_NODE = 40             # direction, psi, bin indices of one accepted node
FLOPS_COL_WEIGHT = 3            # one (pixel, weight) accumulation
PEAK_FP32 = SMS * FP32_LANES * 2 * 2.07e9 / 1e12   # TFLOP/s, nominal unit counts at the max SM clock
PEAK_FP64 = 1.25                # TFLOP/s, nominal GB300 FP64


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _roof(bound, flops_or_bytes, ms, peak, unit, kernel, note=""):
    achieved = flops_or_bytes / (ms * 1e-3) / 1e12
    r = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak, "kernel": kernel}
    if note:
        r["peak_note"] = note
    return r


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--configs", default="", help="comma list of sphere32,disk2p1i,periodic3p,abu,columns,batched,macsweep,mlp_profile: measure the "
                                                  "other workloads (one JSON line each) instead of the main line")
    ap.add_argument("--out", default="", help="also append the JSON lines to this file")
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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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


def _emit(args, rec):
    line = json.dumps(rec)
    print(line, flush=True)
    if args.out:
        with open(args.out, "a") as f:
            f.write(line + "\n")


def _timed_ms(fn, stream, k=5, w=2):
    """Mean CUDA-event time of fn() on `stream` over k runs after w warm-ups."""
    import torch
    for _ in range(w):
        fn()
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
    stream.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def _oracle_rate(fn, ncell, seconds=8.0):
    """Oracle cells/s on a random target sample sized to take about `seconds`."""
    from oracle import oracle
    from paper_1708_06142_gb300 import inputs
    t0 = time.perf_counter()
    fn(inputs.sample_cells(ncell, 128, seed=5))
    dt = time.perf_counter() - t0
    nt = int(min(ncell, max(256, 128 * seconds / max(dt, 1e-3))))
    t0 = time.perf_counter()
    fn(inputs.sample_cells(ncell, nt, seed=6))
    dt = time.perf_counter() - t0
    return {"value": nt / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle", "sample": f"{nt} targets"}


def run_configs(args):
    """Measurements of the other workloads (each a JSON line): throughput, accuracy against the GPU's
    own FP64 walks (ts_error_metrics on the device), the oracle's own rate on the host cores
    (cpu_baseline).  Parity with the FP64 oracle at these sizes is checked by the GPU tests."""
    import torch
    from oracle import oracle
    from paper_1708_06142_gb300 import inputs
    from paper_1708_06142_gb300.treesolver import Batch, TreeSolver
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    which = [c.strip() for c in args.configs.split(",") if c.strip()]

    def emet(ts, acc, acc_ref):
        """eq. ea on the device (ts_error_metrics) against an FP64 reference computed on the GPU"""
        em = ts.error_metrics(acc=acc, acc_ref=acc_ref)
        return {"median_e_a": em["e_a_median"], "p99_e_a": em["e_a_p99"], "max_e_a": em["e_a_max"]}

    if "sphere32" in which:
        mesh, rho = inputs.sphere_32(seed=0)
        ts = TreeSolver(0, stream=stream)
        d = torch.from_numpy(rho.reshape(-1)).to(dev)
        with torch.cuda.stream(stream):
            ts.tree_build(mesh, d)
        p32, a32 = torch.empty(mesh.ncell, device=dev), torch.empty(mesh.ncell, 3, device=dev)
        p64 = torch.empty(mesh.ncell, dtype=torch.float64, device=dev)
        a64 = torch.empty(mesh.ncell, 3, dtype=torch.float64, device=dev)
        g32, g64 = ts.gravity_params(theta=0.5), ts.gravity_params(theta=0.5, precision="fp64")

        def step32():
            ts.tree_build(None, d)
            ts.gravity_walk(p32, a32, g32)

        def step64():
            ts.tree_build(None, d)
            ts.gravity_walk(p64, a64, g64)

        m32, m64 = _timed_ms(step32, stream, 20, 3), _timed_ms(step64, stream, 5, 2)
        ts.sync()
        # the N^2 direct sum on the GPU: the FP64 walk with theta -> 0 opens every node down to the
        # cells (the parity of both walks with the FP64 oracle is the tests' job)
        pd, ad = torch.empty_like(p64), torch.empty_like(a64)
        with torch.cuda.stream(stream):
            ts.gravity_walk(pd, ad, ts.gravity_params(theta=1e-6, precision="fp64"))
        ts.sync()
        _emit(args, {"config": "sphere32: isolated 32^3 uniform sphere, BH theta=0.5", "cells": mesh.ncell,
                     "fp32_cells_per_s": mesh.ncell / (m32 * 1e-3), "fp64_cells_per_s": mesh.ncell / (m64 * 1e-3),
                     "fp32_vs_fp64_walk_same_mac": emet(ts, a32, a64),
                     "bh_vs_direct_sum": emet(ts, a64, ad),
                     "cpu_baseline": _oracle_rate(lambda t: oracle.gravity_walk(mesh, rho, t, theta=0.5), mesh.ncell)})

    if "disk2p1i" in which:
        mesh, rho = inputs.disk_2p1i(seed=2)
        ts = TreeSolver(0, stream=stream)
        d = torch.from_numpy(rho.reshape(-1)).to(dev)
        with torch.cuda.stream(stream):
            ts.tree_build(mesh, d)
        t0 = time.perf_counter()
        ts.ewald_field(64)
        t_table = time.perf_counter() - t0
        t0 = time.perf_counter()
        loss = ts.surrogate_train()
        t_train = time.perf_counter() - t0
        p32, a32 = torch.empty(mesh.ncell, device=dev), torch.empty(mesh.ncell, 3, device=dev)
        pm, am = torch.empty(mesh.ncell, device=dev), torch.empty(mesh.ncell, 3, device=dev)
        p64 = torch.empty(mesh.ncell, dtype=torch.float64, device=dev)
        a64 = torch.empty(mesh.ncell, 3, dtype=torch.float64, device=dev)
        gt, gm = ts.gravity_params(theta=0.5), ts.gravity_params(theta=0.5, ewald="mlp")
        g64 = ts.gravity_params(theta=0.5, precision="fp64")

        def mk(p, a, g):
            def f():
                ts.tree_build(None, d)
                ts.gravity_walk(p, a, g)
            return f

        mt = _timed_ms(mk(p32, a32, gt), stream, 5, 2)
        st_t = {**ts.stats(), **ts.walk_counters()}
        mm = _timed_ms(mk(pm, am, gm), stream, 3, 1)
        st_m = {**ts.stats(), **ts.walk_counters()}
        pty, aty = torch.empty_like(p32), torch.empty_like(a32)
        gty = ts.gravity_params(theta=0.5, ewald="taylor")
        t0 = time.perf_counter()
        ts.gravity_walk(pty, aty, gty)        # builds the Taylor table (set-up, timed separately)
        ts.sync()
        t_taylor = time.perf_counter() - t0
        mty = _timed_ms(mk(pty, aty, gty), stream, 3, 1)
        st_ty = {**ts.stats(), **ts.walk_counters()}
        m64 = _timed_ms(mk(p64, a64, g64), stream, 2, 1)
        st_64 = {**ts.stats(), **ts.walk_counters()}
        ts.sync()
        fl_t = (FLOPS_PER_INTERACTION + FLOPS_EWALD_CORR + FLOPS_MIMG) * st_t["interactions"] + \
            (FLOPS_PER_MAC_BH + FLOPS_MIMG) * st_t["mac_tests"]
        fl_64 = (FLOPS_PER_INTERACTION + FLOPS_EWALD_CORR + FLOPS_MIMG) * st_64["interactions"] + \
            (FLOPS_PER_MAC_BH + FLOPS_MIMG) * st_64["mac_tests"]
        bf16 = _peaks().get("bf16_tflops_sustained", 1723.4)
        roofs = {"table_fp32": _roof("alu", fl_t, st_t["walk_ms"], PEAK_FP32, "TFLOP/s",
                                     "k_gravity_walk<float, correction table, BH>"),
                 "mlp_tensor": _roof("tensor", FLOPS_MLP * st_m["interactions"], st_m["walk_ms"], bf16, "TFLOP/s",
                                     "k_gravity_walk<float, learned correction, BH> (mma.sync m16n8k16 bf16)",
                                     "measured cuBLAS bf16 sustained"),
                 "table_fp64": _roof("alu", fl_64, st_64["walk_ms"], PEAK_FP64, "TFLOP/s",
                                     "k_gravity_walk<double, correction table, BH>", "nominal GB300 FP64")}
        _emit(args, {"config": "disk2p1i: x,y periodic / z isolated 256^3, box 1x1x4, BH theta=0.5", "cells": mesh.ncell,
                     "table_cells_per_s": mesh.ncell / (mt * 1e-3), "mlp_cells_per_s": mesh.ncell / (mm * 1e-3),
                     "fp64_table_cells_per_s": mesh.ncell / (m64 * 1e-3),
                     "taylor_cells_per_s": mesh.ncell / (mty * 1e-3),
                     "walk_ms": {"table": st_t["walk_ms"], "mlp": st_m["walk_ms"], "fp64_table": st_64["walk_ms"],
                                 "taylor": st_ty["walk_ms"]},
                     "taylor_vs_fp64_table_walk": emet(ts, aty, a64),
                     "interactions_per_cell": st_t["interactions"] / mesh.ncell,
                     "mac_tests_per_cell": st_t["mac_tests"] / mesh.ncell,
                     "lane_utilisation": st_t["active_lanes"] / (32.0 * max(1, st_t["pops"])),
                     "roofline": roofs,
                     "table_vs_fp64_table_walk": emet(ts, a32, a64),
                     "mlp_vs_fp64_table_walk": emet(ts, am, a64),
                     "accuracy_note": "against the FP64 walk with the trilinear table on every cell; the accuracy of "
                                      "each lookup against the exact Ewald series is measured by the GPU tests",
                     "setup_s": {"table_64": t_table, "taylor_table_64_and_first_walk": t_taylor,
                                 "surrogate_train": t_train, "surrogate_loss": loss},
                     "cpu_baseline": _oracle_rate(lambda t: oracle.gravity_walk(mesh, rho, t, ewald="series"),
                                                  mesh.ncell, seconds=6.0)})

    if "periodic3p" in which:
        mesh, rho = inputs.turbulent_periodic(seed=3)
        ts = TreeSolver(0, stream=stream)
        d = torch.from_numpy(rho.reshape(-1)).to(dev)
        with torch.cuda.stream(stream):
            ts.tree_build(mesh, d)
        ts.ewald_field(64)
        p32, a32 = torch.empty(mesh.ncell, device=dev), torch.empty(mesh.ncell, 3, device=dev)
        p64 = torch.empty(mesh.ncell, dtype=torch.float64, device=dev)
        a64 = torch.empty(mesh.ncell, 3, dtype=torch.float64, device=dev)
        g32 = ts.gravity_params(theta=0.5, zero_mean=True)
        g64 = ts.gravity_params(theta=0.5, precision="fp64", zero_mean=True)

        def stp(p, a, g):
            def f():
                ts.tree_build(None, d)
                ts.gravity_walk(p, a, g)
            return f

        m32 = _timed_ms(stp(p32, a32, g32), stream, 5, 2)
        st = {**ts.stats(), **ts.walk_counters()}
        m64 = _timed_ms(stp(p64, a64, g64), stream, 2, 1)
        st64 = {**ts.stats(), **ts.walk_counters()}
        em = ts.error_metrics(pot=p32, acc=a32, pot_ref=p64, acc_ref=a64, mod_const=True)
        pt, at = torch.empty_like(p32), torch.empty_like(a32)
        gty = ts.gravity_params(theta=0.5, zero_mean=True, ewald="taylor")
        ts.gravity_walk(pt, at, gty)          # builds the Taylor table (untimed set-up)
        mty = _timed_ms(stp(pt, at, gty), stream, 5, 2)
        sty = {**ts.stats(), **ts.walk_counters()}
        fl = (FLOPS_PER_INTERACTION + FLOPS_EWALD_CORR + FLOPS_MIMG) * st["interactions"] + \
            (FLOPS_PER_MAC_BH + FLOPS_MIMG) * st["mac_tests"]
        _emit(args, {"config": "periodic3p: fully periodic 128^3 log-normal, gravity BH theta=0.5, 64^3 table",
                     "cells": mesh.ncell, "fp32_cells_per_s": mesh.ncell / (m32 * 1e-3),
                     "fp64_cells_per_s": mesh.ncell / (m64 * 1e-3),
                     "taylor_fp32_cells_per_s": mesh.ncell / (mty * 1e-3),
                     "walk_ms": {"fp32": st["walk_ms"], "fp64": st64["walk_ms"], "taylor_fp32": sty["walk_ms"]},
                     "interactions_per_cell": st["interactions"] / mesh.ncell,
                     "fp32_vs_fp64_walk": {k: em[k] for k in ("e_a_median", "e_a_p99", "e_phi_median", "e_phi_p99")},
                     "taylor_fp32_vs_fp64_table_walk": emet(ts, at, a64),
                     "roofline": {"fp32": _roof("alu", fl, st["walk_ms"], PEAK_FP32, "TFLOP/s",
                                                "k_gravity_walk<float, correction table, BH>"),
                                  "taylor_fp32": _roof("alu", (FLOPS_PER_INTERACTION + FLOPS_EWALD_TAYLOR + FLOPS_MIMG) *
                                                       sty["interactions"] + (FLOPS_PER_MAC_BH + FLOPS_MIMG) *
                                                       sty["mac_tests"], sty["walk_ms"], PEAK_FP32, "TFLOP/s",
                                                       "k_gravity_walk<float, Taylor table, BH>"),
                                  "table_l1": {"bound": "l1", "achieved_table_TB_per_s":
                                               128 * st["interactions"] / (st["walk_ms"] * 1e-3) / 1e12,
                                               "note": "8 corners x 16 B per interaction, served by L1/L2"}},
                     "cpu_baseline": _oracle_rate(lambda t: oracle.gravity_walk(mesh, rho, t, ewald="series"),
                                                  mesh.ncell, seconds=6.0)})

    if "mlp_profile" in which:
        # a small learned-correction case for kernel profiles: 64^3 cells of the 2P1I disk in a
        # 1x1x4 box, a network trained for only 2,000 steps (its accuracy is not the point here)
        mesh, rho = inputs.disk_2p1i(seed=2, n=64)
        ts = TreeSolver(0, stream=stream)
        d = torch.from_numpy(rho.reshape(-1)).to(dev)
        with torch.cuda.stream(stream):
            ts.tree_build(mesh, d)
        loss = ts.surrogate_train(steps=2000)
        pm, am = torch.empty(mesh.ncell, device=dev), torch.empty(mesh.ncell, 3, device=dev)
        gm = ts.gravity_params(theta=0.5, ewald="mlp")

        def stepm():
            ts.tree_build(None, d)
            ts.gravity_walk(pm, am, gm)

        mm = _timed_ms(stepm, stream, 3, 1)
        st = {**ts.stats(), **ts.walk_counters()}
        bf16 = _peaks().get("bf16_tflops_sustained", 1723.4)
        _emit(args, {"config": "mlp_profile: 2P1I disk 64^3 (box 1x1x4), learned correction, BH 0.5, 2,000 training steps",
                     "cells": mesh.ncell, "cells_per_s": mesh.ncell / (mm * 1e-3), "walk_ms": st["walk_ms"],
                     "interactions_per_cell": st["interactions"] / mesh.ncell, "loss": loss,
                     "roofline": {"mlp_tensor": _roof("tensor", FLOPS_MLP * st["interactions"], st["walk_ms"], bf16,
                                                      "TFLOP/s", "k_gravity_walk<float, learned correction, BH>",
                                                      "measured cuBLAS bf16 sustained")}})

    if "abu" in which:
        # Adaptive Block Update on the AMR benchmark mesh after three kinds of density change: the
        # whole core (r < 0.1) +5 % (a global change: nearly every block must be walked), a clump of
        # leaf-blocks within 0.05 of (0.6, 0.5, 0.5) +2 %, and the outer octant (x, y, z > 0.5,
        # r > 0.25) +20 % (little mass: local changes only).  Tolerance 1e-3 a_max.
        mesh, rho = setup_problem(1)
        ts = TreeSolver(0, stream=stream)
        d = torch.from_numpy(rho.reshape(-1)).to(dev)
        with torch.cuda.stream(stream):
            ts.tree_build(mesh, d)
        p0, a0 = torch.empty(mesh.ncell, device=dev), torch.empty(mesh.ncell, 3, device=dev)
        gp = ts.gravity_params(theta=0.5)
        ts.gravity_walk(p0, a0, gp)
        ts.sync()
        amax = float(a0.norm(dim=1).max())
        ctr = mesh.lo[mesh.leaves] + mesh.size[mesh.leaves] / 2
        r = np.linalg.norm(ctr - 0.5, axis=1)
        cases = {"core r < 0.1 +5%": (r < 0.1, 1.05),
                 "clump |x - (0.6, 0.5, 0.5)| < 0.05 +2%": (np.linalg.norm(ctr - [0.6, 0.5, 0.5], axis=1) < 0.05, 1.02),
                 "outer octant +20%": ((ctr > 0.5).all(1) & (r > 0.25), 1.20)}
        pf, af = torch.empty_like(p0), torch.empty_like(a0)
        pa, aa = torch.empty_like(p0), torch.empty_like(a0)
        res = {}
        for name, (sel, f) in cases.items():
            rho2 = rho.copy()
            rho2[sel] *= f
            d2 = torch.from_numpy(rho2.reshape(-1)).to(dev)

            def full():
                ts.tree_build(None, d2)
                ts.gravity_walk(pf, af, gp)

            m_full = _timed_ms(full, stream, 5, 2)
            nupd = []

            def abu():
                pa.copy_(p0)
                aa.copy_(a0)
                ts.tree_build(None, d2)
                nupd.append(ts.gravity_walk_abu(pa, aa, 1e-3 * amax, params=gp))

            m_abu = _timed_ms(abu, stream, 5, 2)
            em = ts.error_metrics(acc=aa, acc_ref=af.double())
            res[name] = {"blocks_changed": int(sel.sum()), "blocks_walked": int(nupd[-1]), "full_step_ms": m_full,
                         "abu_step_ms": m_abu, "speedup": m_full / m_abu,
                         "abu_vs_full_walk": {"e_a_median": em["e_a_median"], "e_a_p99": em["e_a_p99"],
                                              "e_a_max": em["e_a_max"]}}
        _emit(args, {"config": "abu: 2,097,152-cell AMR Plummer, BH 0.5, a_tol = 1e-3 a_max, three density changes",
                     "cells": mesh.ncell, "blocks": int(mesh.nleaf), "cases": res,
                     "abu_step_ms_note": "includes restoring the previous solution (2 device copies) and one host sync"})

    if "columns" in which:
        mesh, rho = inputs.turbulent_periodic(seed=3)
        ts = TreeSolver(0, stream=stream)
        d = torch.from_numpy(rho.reshape(-1)).to(dev)
        with torch.cuda.stream(stream):
            ts.tree_build(mesh, d)
        cols = torch.empty(mesh.ncell, 48, device=dev)
        cp = ts.column_params(n_side=2, theta=0.5)

        def stepc():
            ts.tree_build(None, d)
            ts.column_walk(cols, cp)

        mc = _timed_ms(stepc, stream, 5, 2)
        ts.sync()
        st = ts.stats()
        # mean visual extinction (eq. av) of every cell from its map (k = 1): one pass over the map
        av = torch.empty(mesh.ncell, device=dev)
        m_av = _timed_ms(lambda: ts.column_av(cols, 1.0, av), stream, 10, 3)
        nnz = float((ts.noderay_table() > 0).sum(-1).mean())   # mean (pixel, weight) pairs per table entry
        fl_c = (FLOPS_COL_NODE + FLOPS_COL_WEIGHT * nnz + FLOPS_MIMG) * st["interactions"]
        _emit(args, {"config": "columns: fully periodic 128^3 log-normal, N_PIX=48, theta=0.5", "cells": mesh.ncell,
                     "roofline": {"fp32": _roof("alu", fl_c, st["walk_ms"], PEAK_FP32, "TFLOP/s", "k_column_walk",
                                                f"{nnz:.2f} weights per lookup (table mean)"),
                                  "output_hbm": _roof("hbm", mesh.ncell * 48 * 4, st["walk_ms"],
                                                      _peaks().get("hbm_gbs", 6678.2) / 1e3, "TB/s",
                                                      "k_column_walk output stream")},
                     "cell_column_updates_per_s": mesh.ncell / (mc * 1e-3), "walk_ms": st["walk_ms"],
                     "interactions_per_cell": st["interactions"] / mesh.ncell,
                     "output_GB_per_s": mesh.ncell * 48 * 4 / (st["walk_ms"] * 1e-3) / 1e9,
                     "accuracy_note": "the column densities against the FP64 oracle are checked by the GPU tests",
                     "extinction_av": {"ms": m_av, "roofline": _roof("hbm", mesh.ncell * (48 + 1) * 4, m_av,
                                                                     _peaks().get("hbm_gbs", 6678.2) / 1e3, "TB/s",
                                                                     "k_column_av (map read + A_V write)")},
                     "cpu_baseline": _oracle_rate(lambda t: oracle.column_walk(mesh, rho, t, nside=2, theta=0.5),
                                                  mesh.ncell, seconds=6.0)})

    if "macsweep" in which:
        # the comparison of MACs of Sec. 4 (Fig. perf:acc) on a uniform 128^3 Bonnor-Ebert-like
        # sphere: each MAC's FP32 walk time against its largest acceleration error over the whole
        # domain; the reference is the N^2 sum (the FP32 + Kahan walk with theta -> 0, which opens
        # every node down to the cells)
        mesh, rho = inputs.be_sphere(128)
        ts = TreeSolver(0, stream=stream)
        d = torch.from_numpy(rho.reshape(-1)).to(dev)
        with torch.cuda.stream(stream):
            ts.tree_build(mesh, d)
        pr, ar = torch.empty(mesh.ncell, device=dev), torch.empty(mesh.ncell, 3, device=dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            ts.gravity_walk(pr, ar, ts.gravity_params(theta=1e-6))
        ts.sync()
        t_ref = time.perf_counter() - t0
        aref = ar.double()
        amax = float(aref.norm(dim=1).max())
        p, a = torch.empty_like(pr), torch.empty_like(ar)
        runs = []
        aold = None
        for mac, par, kw in (("bh", 1.0, dict(theta=1.0)), ("bh", 0.5, dict(theta=0.5)), ("bh", 0.2, dict(theta=0.2)),
                             ("ape_abs", 1e-2, dict(mac="ape", a_lim=1e-2 * amax)),
                             ("ape_abs", 1e-3, dict(mac="ape", a_lim=1e-3 * amax)),
                             ("ape_rel", 1e-2, dict(mac="ape", eps_rel=1e-2)),
                             ("mpe_abs", 1e-2, dict(mac="mpe", a_lim=1e-2 * amax)),
                             ("mpe_abs", 1e-3, dict(mac="mpe", a_lim=1e-3 * amax))):
            if mac == "ape_rel":
                kw = dict(kw, a_old=aold)
            g = ts.gravity_params(**kw)

            def walk():
                ts.gravity_walk(p, a, g)

            ms = _timed_ms(walk, stream, 5, 2)
            st = {**ts.stats(), **ts.walk_counters()}
            em = ts.error_metrics(acc=a, acc_ref=aref)
            if mac == "bh" and par == 0.5:
                aold = a.norm(dim=1).contiguous()      # |a| of the previous step for the relative limit
            runs.append({"mac": mac, "param": par, "walk_ms": ms, "interactions_per_cell": st["interactions"] / mesh.ncell,
                         "e_a_median": em["e_a_median"], "e_a_p99": em["e_a_p99"], "e_a_max": em["e_a_max"],
                         "t_x_e_a_max": ms * em["e_a_max"]})
        _emit(args, {"config": "macsweep: isolated uniform 128^3 Bonnor-Ebert-like sphere, FP32 + Kahan walks",
                     "cells": mesh.ncell, "reference": "N^2 sum (FP32 + Kahan walk, theta -> 0)",
                     "reference_s": t_ref, "runs": runs,
                     "note": "param: theta (bh), epsilon with a_lim = epsilon a_max (ape_abs, mpe_abs), epsilon with "
                             "a_lim = epsilon |a_old| per cell from the theta = 0.5 walk (ape_rel)"})

    if "batched" in which:
        grids = inputs.batched_grids(64)
        solvers, dens = [], []
        for mesh, rho in grids:
            ts = TreeSolver(0)
            dd = torch.from_numpy(np.ascontiguousarray(rho).reshape(-1)).to(dev)
            ts.tree_build(mesh, dd)
            if any(mesh.bc):
                ts.ewald_field(32)
            solvers.append(ts)
            dens.append(dd)
        torch.cuda.synchronize()
        b = Batch(solvers)
        gp = solvers[0].gravity_params(theta=0.5)
        cp = solvers[0].column_params(n_side=2, theta=0.5)
        pots = [torch.empty(m.ncell, device=dev) for m, _ in grids]
        accs = [torch.empty(m.ncell, 3, device=dev) for m, _ in grids]
        cols = [torch.empty(m.ncell, 48, device=dev) for m, _ in grids]
        best = None
        tried = []
        # autotune: the persistent per-class kernels (items per dequeue, CTAs per SM) and the per-grid
        # kernels spread over 4, 8 or 16 streams
        for mode, x, y in ((0, 1, 0), (0, 4, 0), (0, 16, 0), (0, 4, 2), (1, 4, 0), (1, 8, 0), (1, 16, 0)):
            if mode == 0:
                b.set_mode(0, 8)
                b.set_tuning(x, y)
            else:
                b.set_mode(1, x)
            b.run(gp, pots, accs, cp, cols, densities=dens, use_graph=True)
            b.sync()
            b.run(gp, pots, accs, cp, cols, densities=dens, use_graph=True)
            ms = b.sync()["ms"]
            tried.append({"mode": mode, "p1": x, "p2": y, "ms": ms})
            if best is None or ms < best[0]:
                best = (ms, mode, x, y)
        if best[1] == 0:
            b.set_mode(0, 8)
            b.set_tuning(best[2], best[3])
        else:
            b.set_mode(1, best[2])

        def batch_ms(g):
            b.run(g, pots, accs, cp, cols, densities=dens, use_graph=True)
            b.sync()
            ts_ = []
            for _ in range(5):
                b.run(g, pots, accs, cp, cols, densities=dens, use_graph=True)
                ts_.append(b.sync()["ms"])
            return float(np.median(ts_))

        def separate_s(g):
            # the same work as 64 x 3 single-grid launches, each grid on its own stream
            res = []
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for ts, dd, p, a, c in zip(solvers, dens, pots, accs, cols):
                    ts.tree_build(None, dd)
                    ts.gravity_walk(p, a, g)
                    ts.column_walk(c, cp)
                for ts in solvers:
                    ts.sync()
                res.append(time.perf_counter() - t0)
            return float(np.median(res[1:]))

        gty = solvers[0].gravity_params(theta=0.5, ewald="taylor")
        m_taylor, sep_taylor = batch_ms(gty), separate_s(gty)
        m_table = batch_ms(gp)
        times = [m_table]
        st = b.sync()
        t_sep = separate_s(gp)
        ncell = sum(m.ncell for m, _ in grids)
        # the last batched run (trilinear lookup) against each sampled grid's own FP64 walk
        errs = []
        for k in (0, 1, 2, 5, 7):
            ts = solvers[k]
            p64 = torch.empty(ts.ncell, dtype=torch.float64, device=dev)
            a64 = torch.empty(ts.ncell, 3, dtype=torch.float64, device=dev)
            ts.gravity_walk(p64, a64, ts.gravity_params(theta=0.5, precision="fp64"))
            ts.sync()
            errs.append(emet(ts, accs[k], a64)["median_e_a"])
        _emit(args, {"config": "batched: 64 grids 32^3-128^3, isolated/3P/2P1I, gravity BH 0.5 + columns N_PIX=48",
                     "cells": ncell, "ms_per_run": float(np.median(times)),
                     "cell_updates_per_s": ncell / (np.median(times) * 1e-3),
                     "separate_launches_s": t_sep,
                     "taylor_lookup": {"ms_per_run": m_taylor, "cell_updates_per_s": ncell / (m_taylor * 1e-3),
                                       "separate_launches_s": sep_taylor},
                     "tuning": {"chosen": {"mode": best[1], "p1": best[2], "p2": best[3]},
                                "note": "mode 0: persistent per-class kernels (p1 items per dequeue, p2 CTAs/SM, 0 = max); "
                                        "mode 1: per-grid kernels on p1 streams", "tried": tried},
                     "interactions": st["interactions"], "column_interactions": st["column_interactions"],
                     "median_e_a_vs_fp64_walk_sampled_grids": errs})


def other_workloads(dev, stream):
    """Short measurements of the other walks on their own workloads, reported in the main line (the
    column walk of the 128^3 log-normal box with N_PIX = 48, and the fully periodic gravity walk of
    the same box with the first-order Taylor lookup); each with its roofline fraction."""
    import torch
    from paper_1708_06142_gb300 import inputs
    from paper_1708_06142_gb300.treesolver import TreeSolver
    out = {}
    mesh, rho = inputs.turbulent_periodic(seed=3)
    ts = TreeSolver(dev.index, stream=stream)
    d = torch.from_numpy(rho.reshape(-1)).to(dev)
    with torch.cuda.stream(stream):
        ts.tree_build(mesh, d)
    cols = torch.empty(mesh.ncell, 48, device=dev)
    cp = ts.column_params(n_side=2, theta=0.5)
    _timed_ms(lambda: ts.column_walk(cols, cp), stream, 3, 1)
    ts.sync()
    st = ts.stats()
    nnz = float((ts.noderay_table() > 0).sum(-1).mean())
    fl = (FLOPS_COL_NODE + FLOPS_COL_WEIGHT * nnz + FLOPS_MIMG) * st["interactions"]
    out["columns_128_npix48"] = {"walk_ms": st["walk_ms"], "cell_column_updates_per_s": mesh.ncell / (st["walk_ms"] * 1e-3),
                                 "interactions_per_cell": st["interactions"] / mesh.ncell,
                                 "roofline": _roof("alu", fl, st["walk_ms"], PEAK_FP32, "TFLOP/s", "k_column_walk")}
    ts.ewald_field(64)
    pot = torch.empty(mesh.ncell, device=dev)
    acc = torch.empty(mesh.ncell, 3, device=dev)
    g = ts.gravity_params(theta=0.5, ewald="taylor", zero_mean=True)
    _timed_ms(lambda: ts.gravity_walk(pot, acc, g), stream, 3, 1)
    ts.sync()
    st = {**ts.stats(), **ts.walk_counters()}
    fl = (FLOPS_PER_INTERACTION + FLOPS_EWALD_TAYLOR + FLOPS_MIMG) * st["interactions"] + \
         (FLOPS_PER_MAC_BH + FLOPS_MIMG) * st["mac_tests"]
    out["periodic3p_128_taylor"] = {"walk_ms": st["walk_ms"], "cell_updates_per_s": mesh.ncell / (st["walk_ms"] * 1e-3),
                                    "interactions_per_cell": st["interactions"] / mesh.ncell,
                                    "roofline": _roof("alu", fl, st["walk_ms"], PEAK_FP32, "TFLOP/s",
                                                      "k_gravity_walk<float, table, Taylor>")}
    ts.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.configs:
        return run_configs(args)
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1708_06142_gb300.treesolver import TreeSolver
    from paper_1708_06142_gb300.shard import max_over_ranks, weak_throughput

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
    # accuracy of the FP32 walk against the FP64 walk on every cell (eq. ea, device metric kernels)
    em = ts.error_metrics(pot=pot, acc=acc, pot_ref=pot64, acc_ref=acc64)
    amax = em["a_ref_max"]
    accuracy = {"median_e_a_vs_fp64_walk": em["e_a_median"], "p99_e_a_vs_fp64_walk": em["e_a_p99"],
                "max_e_a_vs_fp64_walk": em["e_a_max"], "median_e_phi_vs_fp64_walk": em["e_phi_median"],
                "p99_e_phi_vs_fp64_walk": em["e_phi_p99"], "cells_compared": em["n"]}
    bh = ts.gravity_params(mac="bh", theta=0.5)
    ape = ts.gravity_params(mac="ape", a_lim=1e-2 * amax)
    mpe = ts.gravity_params(mac="mpe", a_lim=1e-2 * amax)
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

    # main timed region: BH FP32-Kahan (the FP32 walk reads only the FP32 records: the builds skip
    # the FP64 shadow records, switched back on for the FP64 walk below)
    ts.fp64_records(False)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    step_ms, walk_ms, st = timed(bh, pot, acc, args.steps, args.warmup)
    torch.cuda.synchronize()
    clocks = clk.stop()
    total_ms = max_over_ranks(float(step_ms.sum()), dev)
    value = weak_throughput([ncell * args.steps] * world, total_ms * 1e-3)

    # secondary measurements (same procedure, fewer steps)
    k2 = max(3, min(args.steps, 10))
    ape_ms, ape_walk, ape_st = timed(ape, pot, acc, k2, 2)
    mpe_ms, mpe_walk, mpe_st = timed(mpe, pot, acc, k2, 2)   # includes the on-demand B2/B3 moments
    ts.fp64_records(True)
    f64_ms, f64_walk, f64_st = timed(bh64, pot64, acc64, k2, 2)
    ts.fp64_records(False)
    # the paper's other forms of the walk on the same mesh: the potential alone with the acceleration
    # by numerical differentiation (Sec. 2.2.2) and the SumSquare MAC (Sec. 2.2.1), each against the
    # FP64 direct-summation BH walk (acc64 holds the last FP64 walk of the timing above)
    nd = ts.gravity_params(mac="bh", theta=0.5, accel="numdiff")
    nd_ms, nd_walk, _ = timed(nd, pot, acc, k2, 2)
    em_nd = ts.error_metrics(acc=acc, acc_ref=acc64)
    sq = ts.gravity_params(mac="sumsq", a_lim=1e-2 * amax)
    sq_ms, sq_walk, sq_st = timed(sq, pot, acc, 2, 1)
    em_sq = ts.error_metrics(acc=acc, acc_ref=acc64)
    others = other_workloads(dev, stream) if rank == 0 else {}

    # end to end through the C ABI from pinned host buffers: every step copies its density in and its
    # potential and acceleration out, on a copy stream with two device buffers of each: the density
    # of step k + 1 arrives while step k computes, the results of step k leave while step k + 1
    # computes; the 256 MB L2 flush of every step is inside the timed region
    h_rho = torch.from_numpy(rho.reshape(-1).copy()).pin_memory()
    h_pot = [torch.empty(ncell, dtype=torch.float32).pin_memory() for _ in range(2)]
    h_acc = [torch.empty(ncell, 3, dtype=torch.float32).pin_memory() for _ in range(2)]
    d_rhos = [d_rho, torch.empty_like(d_rho)]
    d_pot = [pot, torch.empty_like(pot)]
    d_acc = [acc, torch.empty_like(acc)]
    copy_stream = torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]       # the density of the buffer is copied in
    ev_walk = [torch.cuda.Event() for _ in range(2)]     # the step that used the buffers is done
    ev_copied = [torch.cuda.Event() for _ in range(2)]

    def copy_in(b):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(ev_walk[b])    # (an event never recorded counts as complete)
            d_rhos[b].copy_(h_rho, non_blocking=True)
            ev_in[b].record(copy_stream)

    def e2e_run(nsteps):
        copy_in(0)
        for k in range(nsteps):
            b2 = k % 2
            if k + 1 < nsteps:
                copy_in(1 - b2)                           # once step k - 1 has finished with it
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                if k >= 2:
                    stream.wait_event(ev_copied[b2])      # the step k - 2 copies of this buffer are done
                stream.wait_event(ev_in[b2])
                ts.tree_build(None, d_rhos[b2])
                ts.gravity_walk(d_pot[b2], d_acc[b2], bh)
                ev_walk[b2].record(stream)
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(ev_walk[b2])
                h_pot[b2].copy_(d_pot[b2], non_blocking=True)
                h_acc[b2].copy_(d_acc[b2], non_blocking=True)
                ev_copied[b2].record(copy_stream)

    e2e_run(args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_run(args.steps)
    torch.cuda.synchronize()
    e2e_ms = [1e3 * (time.perf_counter() - t0)]
    ts.sync()
    e2e_total = max_over_ranks(float(np.sum(e2e_ms)), dev)

    walk_s = float(np.mean(walk_ms)) * 1e-3
    from paper_1708_06142_gb300.treesolver import peak_probe
    fma_meas = {k: peak_probe(local, k) for k in ("fp32", "fp32x2", "fp64")}   # after the timed region
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
                       "step": "tree_build (FP64 sums, FP32 records) + gravity_walk", "cells": ncell,
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": f"independent problem per GPU x{world}"},
            "accuracy": accuracy,
            "walk_ms": float(np.mean(walk_ms)), "build_ms": float(np.mean(step_ms - walk_ms)),
            "interactions_per_cell": st["interactions"] / ncell, "mac_tests_per_cell": st["mac_tests"] / ncell,
            "lane_utilisation": st["active_lanes"] / (32.0 * max(1, st["pops"])), "pops_per_warp": st["pops"] / (ncell / 32),
            "ape": {"value": ncell * k2 / (ape_ms.sum() * 1e-3), "unit": UNIT, "a_lim": "1e-2 a_max",
                    "walk_ms": float(np.mean(ape_walk)), "interactions_per_cell": ape_st["interactions"] / ncell},
            "mpe": {"value": ncell * k2 / (mpe_ms.sum() * 1e-3), "unit": UNIT, "a_lim": "1e-2 a_max",
                    "walk_ms": float(np.mean(mpe_walk)), "interactions_per_cell": mpe_st["interactions"] / ncell},
            "fp64_walk": {"value": ncell * k2 / (f64_ms.sum() * 1e-3), "unit": UNIT,
                          "walk_ms": float(np.mean(f64_walk))},
            "numdiff": {"value": ncell * k2 / (nd_ms.sum() * 1e-3), "unit": UNIT, "walk_ms": float(np.mean(nd_walk)),
                        "form": "potential-only BH walk + numerical differentiation (Sec. 2.2.2)",
                        "median_e_a_vs_fp64_direct": em_nd["e_a_median"], "p99_e_a_vs_fp64_direct": em_nd["e_a_p99"],
                        "max_e_a_vs_fp64_direct": em_nd["e_a_max"]},
            "sumsq": {"value": ncell * 2 / (sq_ms.sum() * 1e-3), "unit": UNIT, "walk_ms": float(np.mean(sq_walk)),
                      "form": "SumSquare MAC, a_lim = 1e-2 a_max (one thread per target, priority queue)",
                      "interactions_per_cell": sq_st["interactions"] / ncell,
                      "median_e_a_vs_fp64_bh": em_sq["e_a_median"], "max_e_a_vs_fp64_bh": em_sq["e_a_max"]},
            "other_workloads": others,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                         "frac": achieved / peak_fp32, "traffic": traffic,
                         "kernel": "k_gravity_walk<float, isolated, BH>",
                         "peak_note": "FP32 pipe: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (nominal unit counts and max clock)",
                         "peak_measured_fma_tflops": fma_meas},
            "e2e": {"value": weak_throughput([ncell * args.steps] * world, e2e_total * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": ncell * 8, "d2h_bytes_per_step": ncell * 16,
                    "note": "wall time of K steps from pinned host buffers; the density of step k + 1 is copied in "
                            "and the results of step k - 1 are copied out while step k computes (double-buffered "
                            "inputs and outputs); the per-step L2 flush is inside the timed region"},
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
