#!/usr/bin/env python
"""Benchmark of the coupled LB-FD time step (arXiv 2311.15242) on GB300.

Workload: the 2D buoyant bubble rise in a walled channel, D2Q9 256 x 1024,
bubble diameter 64, density ratio 10, viscosity ratio 10, Eo = 10, Mo = 0.1,
Bi = 1, bulk C0 = 0.5, psi = 0 initially (seeded synthetic initial state).
A step is one full coupled update (LB step + surfactant FD step with its SOR
solve and rescale) of the whole grid.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbs|reference]

Timing: W untimed warm-up steps, then K steps, each timed with CUDA events on
the solver's stream; L2 (126 MB) is flushed by a 256 MiB write before every
timed step, outside the events.  With N > 1 (torchrun) every rank runs an
independent replica (weak scaling); the slowest rank's time is reported.
The reference arm (--impl reference) times the FP64 CPU oracle on the same
workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "coupled-step MLUPS and % of HBM roofline (1 GB300), mixed/batched vs plain FP32"
UNIT = "MLUPS"

# Algorithmic bytes per cell of the 2D kernel groups: each input and output
# field of the group read or written once.  rb: bytes of a field value, pb:
# of a stored moving population.
#   collide (the fused step, k_lbfd2): 16 moving and 2 rest populations and
#     the flag read and written; read g (2), psi, rho^R, rho^B, j (2), a,
#     chi, C, S, B, psi^(t-1), C^(t-1) (14 fields); write the next moments
#     rho^R, rho^B, rho^N, j (2), the right-hand sides (2), S, B, the SOR
#     guess (2) and psi^(t-1), C^(t-1) (13 fields)
#   grad (k_grad2n): read rho^R, rho^B, rho^N of t+1 (3), write g (2), a,
#     chi (4); the moments alternate between two sets, nothing is copied
#   surf (k_surf2 + k_scale2): read a, chi, psi, C; read psi, C, write psi, C
#   sor: 32 B a sweep and cell in FP32 (psi, C, two right-hand sides, a, chi
#     read; psi, C written: the count of a plain unblocked sweep), whatever
#     the sweeps the blocked kernel runs in shared memory; the one-launch form
#     (k_sorfuse2) also carries the grad group's fields and, of the surf
#     group's, a and chi for the total (psi, C are the last sweep's) and the
#     rescale's read and write of psi, C (7 + 2 + 4 fields)
def alg_bytes_2d(group, storage, sweeps=0, fused_sor=False):
    rb = 8 if storage == "f64" else 4
    pb = POP_BYTES[storage]
    if group == "collide":
        return 2 * (16 * pb + 2 * rb + 1) + (14 + 13) * rb
    if group == "grad":
        return 7 * rb
    if group == "surf":
        return 8 * rb
    if group == "sor":
        return 8 * rb * sweeps + (13 * rb if fused_sor else 0)
    raise KeyError(group)

# D3Q19: fixed bytes per cell of each group (FP32 fields, flags) and the
# number of populations it reads plus writes (stored in the storage type)
ALG3_FIXED = {"force": 60, "fd": 52, "collide": 46, "stream": 34, "grad": 32, "surf": 32}
ALG3_POPS = {"collide": 76, "stream": 76}
# one red or black half-sweep: psi, C, a, chi of every cell read, the two
# right-hand sides read and psi, C written for half of the cells
SOR3_BYTES_PER_HALF_SWEEP = 24
POP_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}

# DRAM bytes (read + write) a cell of one launch of each fused 2D kernel
# (dram__bytes_read.sum + dram__bytes_write.sum over cells), from ncu
# captures, per SOR tile variant: "bytes_per_cell" on the bench workload
# itself (256 x 1024; ncu empties the caches before the launch),
# "bytes_per_cell_hbm" on the 2048 x 2048 bubble array (4.2 M cells, about
# six times the L2), which the 4096 x 4096 array's roofline scales by its
# cells (the kernels' traffic grows with the cells).  Reported only while the
# files that hold their device code (FUSED2_FILES) hash as below.
TRAFFIC = {"kernel_sha": "76d859fe8b6be644",
           "bytes_per_cell": {"4": {"collide": 130.0, "sor": 30.3},
                              "6": {"collide": 129.9, "sor": 28.3}},
           "bytes_per_cell_hbm": {"4": {"collide": 243.8, "sor": 200.1},
                                  "6": {"collide": 243.8, "sor": 200.3}}}

def src_hash(files=None):
    """Hash of the CUDA sources (every .cu/.cuh file, or the named ones)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2311_15242_gb300", "csrc")
    for n in sorted(os.listdir(d)):
        if n.endswith((".cu", ".cuh")) and (files is None or n in files):
            h.update(open(os.path.join(d, n), "rb").read())
    return h.hexdigest()[:16]


# the files that hold the device code of the fused 2D kernels
FUSED2_FILES = ("lbs_dev.cuh", "lbs_k2d.cuh", "lbs_fused2.cuh")


def traffic_valid(sor_launches, sor_variant, table="bytes_per_cell"):
    """The captured DRAM traffic applies: same kernel source, the fused
    two-launch step, a captured SOR tile variant."""
    return (TRAFFIC["kernel_sha"] == src_hash(FUSED2_FILES) and sor_launches == 1
            and str(sor_variant) in TRAFFIC[table])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """SM clock and clock-event reasons sampled during the timed region.

    Read-only NVML queries from a background thread every 5 ms (the timed
    region can be shorter than nvidia-smi's sampling period); nvidia-smi is
    the fallback when NVML cannot be loaded."""
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index, pci_bus_id=None):
        import ctypes
        import threading
        self.idx, self.rows, self.stop_ev = gpu_index, [], threading.Event()
        self.nv = self.h = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            h = ctypes.c_void_p()
            ok = False
            if pci_bus_id:
                ok = nv.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), ctypes.byref(h)) == 0
            if not ok and nv.nvmlDeviceGetHandleByIndex_v2(gpu_index, ctypes.byref(h)) != 0:
                raise OSError("nvml handle")
            self.nv, self.h = nv, h
        except OSError:
            self.nv = None
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _sample(self):
        import ctypes
        nv, h = self.nv, self.h
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk))  # NVML_CLOCK_SM
        nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
        fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(h, ctypes.byref(rs))
        self.rows.append((clk.value, mx.value, rs.value))

    def _run(self):
        while not self.stop_ev.is_set():
            self._sample()
            self.stop_ev.wait(0.005)

    def start(self):
        if self.nv is not None:
            self.thread.start()
            return
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", "--query-gpu=clocks.sm,clocks.max.sm,"
                 "clocks_event_reasons.active", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.nv is not None:
            self.stop_ev.set()
            self.thread.join(timeout=2)
            self._sample()
        elif getattr(self, "p", None) is not None:
            self.p.terminate()
            self.p.wait(timeout=5)
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                try:
                    self.rows.append((float(parts[0]), float(parts[1]), int(parts[2], 16)))
                except (ValueError, IndexError):
                    pass
        if not self.rows:
            return None
        reasons = sorted({name for _, _, r in self.rows for bit, name in self.BITS.items() if r & bit})
        return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                "sm_max_mhz": max(r[1] for r in self.rows), "reasons": reasons,
                "samples": len(self.rows), "source": "nvml" if self.nv is not None else "nvidia-smi"}


def profile_case(args):
    """Small workloads stepped with individual launches, for kernel
    profilers (ncu cannot trace the kernel nodes of a graph that holds a
    conditional node): 2d = the bubble array on 2048 x 2048 (8 x 8 bubbles,
    4.2 M cells, about 0.76 GB of FP32 state, 6x the L2) with the fused step,
    3d = the sheared droplet at 256 x 128 x 64, half the bench's cells (state
    about 3.5x the L2), batch = the first 8 instances of the 64-instance
    sweep with the bench's tiles (32 x 4, SOR variant 5)."""
    import torch
    from paper_2311_15242_gb300 import Batch, Solver
    torch.cuda.set_device(0)
    if args.profile_case == "2d":
        cfg = W.bubble_array_2d(n=2048, k=8)
        f = W.initial_fields(cfg)
        s = Solver(cfg, storage=args.storage)
        s.set_sor_tile(4 if args.sor_tile is None else args.sor_tile)
        s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
        s.set_graph(False)
        s.step(args.steps)
        s.sync()
        print(json.dumps({"profile_case": "2d", "cells": cfg["nx"] * cfg["ny"],
                          "steps": args.steps, "sor_sweeps": s.diagnostics()["sor_iters_psi"]}))
        return 0
    if args.profile_case == "3d":
        cfg = W.shear_droplet_3d(nx=256, ny=128, nz=64, R=24.0)
        f = W.initial_fields(cfg)
        s = Solver(cfg, storage=args.storage3d)
        if args.sor_tile_3d is not None:
            s.set_sor_tile(args.sor_tile_3d)
        s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
        s.set_graph(False)
        s.step(args.steps)
        s.sync()
        print(json.dumps({"profile_case": "3d", "cells": cfg["nx"] * cfg["ny"] * cfg["nz"],
                          "steps": args.steps, "sor_sweeps": s.diagnostics()["sor_iters_psi"]}))
        return 0
    cfgs = W.bubble_sweep_2d(64, seed=0)[:8]
    b = Batch(cfgs, storage="f32")
    for k, c in enumerate(cfgs):
        f = W.initial_fields(c, seed=k)
        b.init_fields(k, f["phi"], f["psi"], f["C"], f["u"])
    b.set_tiles(32, 4, 5)
    b.set_graph(False)
    b.step(args.steps)
    b.sync()
    print(json.dumps({"profile_case": "batch", "instances": len(cfgs),
                      "cells": sum(c["nx"] * c["ny"] for c in cfgs), "steps": args.steps}))
    return 0


def workload3d():
    """The 3D sheared droplet: D3Q19 256 x 128 x 128, walls at z moving
    along +-x, droplet radius 24, viscosity ratio 1, Ca = 0.2, C0 = 0.5, psi
    at its Langmuir equilibrium; bfloat16 populations with FP32 collision is
    the form this configuration names (FP32 and FP16 timed beside it)."""
    cfg = W.shear_droplet_3d()
    return cfg, "shear_droplet_3d_256x128x128_Ca0.2"


# compulsory state of a coupled step, bytes per cell-update: the two
# population sets read and written once, and psi, C, S, B (FP32) read and
# written once; the whole step's HBM roofline is peak / B_STEP MLUPS
B_STEP = {("d2q9", "f32"): 2 * 18 * 4 + 2 * 4 * 4, ("d2q9", "f16"): 2 * 18 * 2 + 32,
          ("d2q9", "bf16"): 2 * 18 * 2 + 32, ("d3q19", "f32"): 2 * 38 * 4 + 32,
          ("d3q19", "f16"): 2 * 38 * 2 + 32, ("d3q19", "bf16"): 2 * 38 * 2 + 32}


def step_roofline(mlups, lattice, storage, hbm, where):
    """MLUPS x B_STEP against the measured HBM bandwidth ("where" says
    whether the state lives in HBM or fits in the L2)."""
    b = B_STEP[(lattice, storage)]
    gbs = mlups * 1e6 * b / 1e9
    return {"b_alg_per_cell": b, "achieved_gbs": gbs, "frac": gbs / hbm, "state": where}


def roofline2(kmean, cells, storage, sweeps, hbm, src, traffic=None, sor_launches=1):
    """Roofline of the dominant kernel group of a 2D step (bytes of
    alg_bytes_2d).  The SOR group runs in `sor_launches` launches: one for
    every round and the gradient, total and rescale (the one-launch form),
    or one a round."""
    groups = [g for g in kmean if kmean[g] > 0 and g in ("collide", "grad", "surf", "sor")]
    dom = max(groups, key=lambda g: kmean[g])
    fused = sor_launches == 1
    per_cell = alg_bytes_2d(dom, storage, sweeps, fused)
    n = sor_launches if dom == "sor" else 1
    alg = per_cell * cells / n
    launch_ms = kmean[dom] / n
    achieved = alg / (launch_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
            "launch_timing": "in-graph CUDA events on the solver's stream over the "
                             "profiled pass of the same steps after the timed region",
            "peak_source": src, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
            "alg_bytes_per_cell": per_cell, "alg_bytes_per_launch": alg,
            "avg_launch_ms": launch_ms, "sor_sweeps": sweeps}


def roofline3(kmean, cells, storage, rounds, hbm, src):
    """Roofline of the dominant kernel group of the 3D step (bytes as above;
    the SOR group's launch is one half-sweep, two per round)."""
    sc = 2 if storage == "f64" else 1
    pb = POP_BYTES[storage]
    dom = max(kmean, key=lambda g: kmean[g])
    if dom == "sor":
        alg = SOR3_BYTES_PER_HALF_SWEEP * sc * cells
        launch_ms = kmean[dom] / (2 * rounds)
    else:
        alg = (ALG3_FIXED[dom] * sc + ALG3_POPS.get(dom, 0) * pb) * cells
        launch_ms = kmean[dom]
    achieved = alg / (launch_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
            "peak_source": src, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
            "alg_bytes_per_launch": alg, "avg_launch_ms": launch_ms}


def time_steps(s, stream, flush, warmup, steps, torch, profiled=True):
    """Device time of `steps` steps of solver s (after `warmup`), each timed
    with CUDA events on the solver's stream after an L2 flush outside them,
    with the step's graph free of profiling events.  With `profiled`, a
    second pass of `steps` steps (after one warm-up) with the in-graph
    events of lbs_profile gives the per-group times; the events themselves
    cost time (about 0.02 ms of a 2D step), so they stay out of the timed
    steps."""
    def run(n_warm, n, prof):
        s.profile(prof)
        tt, kts = 0.0, []
        for k in range(n_warm + n):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.step(1)
                b.record(stream)
            b.synchronize()
            if k >= n_warm:
                tt += a.elapsed_time(b)
                if prof:
                    kts.append(s.kernel_times())
        s.sync()
        return tt, kts
    tt, _ = run(warmup, steps, False)
    kmean = {}
    if profiled:
        _, kts = run(1, steps, True)
        kmean = {g: float(np.mean([k[g] for k in kts])) for g in kts[0]}
    return tt, kmean


def bench_batch(args, stream, flush, torch):
    """MLUPS of the 64-instance bubble-rise sweep (widths 64-256, heights
    512-1024, D = 32, Eo, Bi, E0, C0 drawn from the seeded generator) as one
    batch with autotuned tiles, and of the same instances stepped one
    single-instance context after another (same steps, same timing: CUDA
    events around each chunk of 8 steps, an L2 flush before each chunk)."""
    from paper_2311_15242_gb300 import Batch, Solver, autotune
    cfgs = W.bubble_sweep_2d(64, seed=0)
    cells = sum(c["nx"] * c["ny"] for c in cfgs)
    fs = [W.initial_fields(c, seed=k) for k, c in enumerate(cfgs)]
    out = {"workload": "bubble_sweep_2d_64", "instances": len(cfgs), "cells": cells,
           "steps": args.batch_steps, "l2": "flushed before every timed graph launch"}
    chunk = 8
    nchunks = max(1, args.batch_steps // chunk)
    for st in ("f32", "f16"):
        b = Batch(cfgs, storage=st, stream=stream)
        for k, f in enumerate(fs):
            b.init_fields(k, f["phi"], f["psi"], f["C"], f["u"])
        tune = autotune.tune(b, [c["nx"] for c in cfgs], use_cache=False)
        b.step(chunk)  # warm-up (builds the graph)
        b.sync()
        tt = 0.0
        for _ in range(nchunks):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                b.step(chunk)
                e1.record(stream)
            e1.synchronize()
            tt += e0.elapsed_time(e1)
        b.sync()
        d = b.diagnostics()
        out[f"mlups_{st}"] = cells * chunk * nchunks / (tt / 1e3) / 1e6
        out[f"tiles_{st}"] = {k: tune[k] for k in ("tx", "ty", "sor")}
        out[f"sor_rounds_max_{st}"] = max(x["sor_rounds"] for x in d)
        out[f"gpu_launches_per_step_{st}"] = b.kernel_count()
        b.close()
    # plain: each instance in its own context, one after another
    tt = 0.0
    for k, c in enumerate(cfgs):
        s = Solver(c, storage="f32", stream=stream)
        s.init_fields(fs[k]["phi"], fs[k]["psi"], fs[k]["C"], fs[k]["u"])
        s.step(2)
        s.sync()
        for _ in range(nchunks):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.step(chunk)
                e1.record(stream)
            e1.synchronize()
            tt += e0.elapsed_time(e1)
        s.sync()
        s.close()
    out["plain_mlups_f32"] = cells * chunk * nchunks / (tt / 1e3) / 1e6
    out["speedup_f32"] = out["mlups_f32"] / out["plain_mlups_f32"]
    return out


def workload():
    cfg = W.bubble_rise_2d()
    name = ("bubble_rise_2d D2Q9 256x1024 walls-x periodic-y, D=64, rho 0.1/1, "
            "mu ratio 10, Eo=10, Mo=0.1, Bi=1, Pe=10, C0=0.5")
    return cfg, name


def max_over_ranks(x, dist, device):
    """The largest x over the ranks of the job (its time is its slowest
    rank's)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank, steps, world, ms):
    """Cells updated by all ranks per second (weak scaling: every rank runs
    its own replica of the workload), in millions."""
    return world * cells_per_rank * steps / (ms / 1e3) / 1e6


def reference_arm(args, rank):
    """FP64 CPU oracle on the host cores (OpenMP over its independent cell
    loops; the lexicographic SOR and the sums stay sequential), same workload
    and metric."""
    if rank != 0:
        return 0
    from oracle.ora import Oracle, threads
    cores = threads(os.cpu_count() or 1)
    cfg, name = workload()
    f = W.initial_fields(cfg, seed=0)
    o = Oracle(cfg)
    o.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    cells = cfg["nx"] * cfg["ny"]
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = cells * args.steps / dt / 1e6
    sample = f"{name}: steps {args.warmup + 1}..{args.warmup + args.steps} of the seeded run"
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": name, "cells": cells},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "host_cpus": os.cpu_count(), "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def _oracle_rate(cfg, budget_s):
    """MLUPS of the oracle over a bounded run (after its first step)."""
    from oracle.ora import Oracle
    f = W.initial_fields(cfg, seed=0)
    o = Oracle(cfg)
    o.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    cells = cfg["nx"] * cfg["ny"] * cfg.get("nz", 1)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    n = int(max(2, min(60, budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return cells * n / dt / 1e6, n


def cpu_baseline(cfg, name, budget_s=10.0):
    """The oracle as it stands on a bounded sample of the workload, on all of
    the host's cores (OpenMP over its independent cell loops) and on one."""
    from oracle.ora import threads
    allc = threads(os.cpu_count() or 1)
    v_all, n_all = _oracle_rate(cfg, budget_s)
    threads(1)
    v_one, n_one = _oracle_rate(cfg, budget_s)
    threads(allc)
    return {"value": v_all, "unit": UNIT, "cores": allc, "kind": "oracle",
            "host_cpus": os.cpu_count(), "value_1_core": v_one,
            "sample": f"{name}: steps 2..{n_all + 1} ({allc} threads) and 2..{n_one + 1} "
                      "(1 thread) of the seeded run on the full grid; the SOR and the sums "
                      "of the oracle are sequential"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lbs", choices=["lbs", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "f16", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip timing the other population storage forms")
    ap.add_argument("--no-bubble3d", action="store_true",
                    help="skip the 3D bubble rise measurement")
    ap.add_argument("--no-migration", action="store_true",
                    help="skip the 3D droplet migration measurement")
    ap.add_argument("--no-octant", action="store_true",
                    help="skip the 3D adsorption octant measurement")
    ap.add_argument("--no-big2d", action="store_true",
                    help="skip the 4096 x 4096 bubble-array measurement")
    ap.add_argument("--no-3d", action="store_true",
                    help="skip the D3Q19 (3D sheared droplet) measurement")
    ap.add_argument("--sor-tile", type=int, default=None,
                    help="blocked SOR variant of the 2D step (0..8) instead of tuning it")
    ap.add_argument("--sor-tile-3d", type=int, default=None,
                    help="SOR variant of the 3D step (0..2) instead of tuning it")
    ap.add_argument("--profile-case", choices=["2d", "3d", "batch"], default=None,
                    help="run a small workload with individual launches for kernel "
                         "profilers and exit (see profile_case)")
    ap.add_argument("--storage3d", default="bf16", choices=["f32", "f64", "f16", "bf16"])
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched sweep measurement")
    ap.add_argument("--batch-steps", type=int, default=16,
                    help="timed steps of the batched sweep (a multiple of 8)")
    ap.add_argument("--steps3", type=int, default=20,
                    help="timed steps of each 3D storage form")
    ap.add_argument("--eager", action="store_true",
                    help="individual kernel launches instead of one graph per step "
                         "(for kernel profilers)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_case:
        return profile_case(args)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2311_15242_gb300 import Solver

    cfg, name = workload()
    cells = cfg["nx"] * cfg["ny"]
    f = W.initial_fields(cfg, seed=0)
    s = Solver(cfg, storage=args.storage)
    s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    # blocked SOR variant: given, or chosen by timing on this context (steps of
    # warm-up; the eager mode for kernel profilers takes it as given)
    from paper_2311_15242_gb300 import autotune
    if args.sor_tile is not None or args.eager:
        tuned = {"sor": 4 if args.sor_tile is None else args.sor_tile}
        s.set_sor_tile(tuned["sor"])
    else:
        tuned = autotune.tune_single(s, cfg["nx"], use_cache=False)
        s.init_fields(f["phi"], f["psi"], f["C"], f["u"])
    # the timed steps run without the in-graph profiling events (they cost
    # about 0.02 ms a step); a profiled pass after them gives the group times
    s.profile(False)
    if args.eager:
        s.set_graph(False)
    stream = s.stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def one_step(profiled):
        with torch.cuda.stream(stream):
            flush.fill_(1)  # evict L2 (outside the events)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(1)
            b.record(stream)
        b.synchronize()
        kt = s.kernel_times() if profiled else None
        return a.elapsed_time(b), kt

    for _ in range(args.warmup):
        one_step(False)
    s.sync()

    props = torch.cuda.get_device_properties(local)
    bus = getattr(props, "pci_bus_id", None)
    dom = getattr(props, "pci_domain_id", 0)
    pci = f"{dom:08x}:{bus:02x}:00.0" if isinstance(bus, int) else None
    clocks = Clocks(local, pci)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(args.steps):
        t, _ = one_step(False)
        times.append(t)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    s.sync()
    # per-group times: the same steps again with the in-graph events
    s.profile(True)
    one_step(False)
    ktimes = [one_step(True)[1] for _ in range(args.steps)]
    s.profile(False)
    s.sync()
    total_ms = float(sum(times))
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, "cuda")
    value = whole_job_mlups(cells, args.steps, world, total_ms)

    # per-group device time (mean over the profiled steps)
    groups = list(ktimes[0].keys())
    kmean = {g: float(np.mean([k[g] for k in ktimes])) for g in groups}
    dg = s.diagnostics()
    sweeps, rounds = dg["sor_iters_psi"], max(dg["sor_rounds"], 1)
    hbm, src = peaks()
    sha = src_hash()
    # the fused step: two launches (k_lbfd2, k_sorfuse2); else the fused
    # step, the gradient, one launch a round, the total and the rescale
    nk = s.kernel_count()
    sor_launches = 1 if nk == 2 else nk - 4
    roof = roofline2(kmean, cells, args.storage, sweeps, hbm, src, sor_launches=sor_launches)
    roof["sor_launches_per_step"] = sor_launches
    if traffic_valid(sor_launches, tuned["sor"]):
        roof["traffic"] = TRAFFIC["bytes_per_cell"][str(tuned["sor"])][roof["kernel"]] * cells
    steproof = {"2d_" + args.storage: step_roofline(value / world, "d2q9", args.storage, hbm,
                                                   "L2 (46 MB of state)")}

    # end to end through the C ABI with host buffers
    pin = {k: torch.from_numpy(np.ascontiguousarray(f[k])).pin_memory().numpy()
           for k in ("phi", "psi", "C")}
    # page-locked host arrays for the final fields (allocated outside the timing)
    shp = tuple(s.shape)
    pout = {k: torch.empty(((3,) if k == "u" else ()) + shp, dtype=torch.float64).pin_memory().numpy()
            for k in ("rho", "u", "phi", "psi", "C")}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.init_fields(pin["phi"], pin["psi"], pin["C"], None)
    d2h = 0
    for _ in range(args.steps):
        s.step(1)
        s.step_result()  # the step's result: steps, conserved total, rescale factor
        d2h += 24 + 4  # those three numbers and the status word
    s.fields(out=pout)
    e2e_dt = time.perf_counter() - t0
    N = cells
    e2e = {"value": cells * args.steps / e2e_dt / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": 3 * N * 8 / args.steps,
           "d2h_bytes_per_step": (d2h + 7 * N * 8) / args.steps}

    # the other storage forms of the same step on the same workload and timing
    forms = {args.storage: value}
    if rank == 0 and not args.no_forms:
        for st in ("f32", "f16", "bf16"):
            if st in forms:
                continue
            s2 = Solver(cfg, storage=st, stream=stream)
            s2.set_sor_tile(tuned["sor"])
            s2.init_fields(f["phi"], f["psi"], f["C"], f["u"])
            tt, _ = time_steps(s2, stream, flush, args.warmup, args.steps, torch, profiled=False)
            forms[st] = cells * args.steps / (tt / 1e3) / 1e6
            steproof["2d_" + st] = step_roofline(forms[st], "d2q9", st, hbm, "L2 (46 MB of state)")
            s2.close()

    # the batched sweep (64 2D instances) against the same instances run one
    # context at a time
    batched = None
    if rank == 0 and not args.no_batch:
        batched = bench_batch(args, stream, flush, torch)
        for st in ("f32", "f16"):
            if batched.get("mlups_" + st):
                steproof["batched_" + st] = step_roofline(batched["mlups_" + st], "d2q9", st,
                                                          hbm, "HBM (8.0 M cells)")

    # the D3Q19 configuration (3D sheared droplet), each storage form
    d3 = None
    if rank == 0 and not args.no_3d:
        cfg3, name3 = workload3d()
        cells3 = cfg3["nx"] * cfg3["ny"] * cfg3["nz"]
        f3 = W.initial_fields(cfg3)
        d3 = {"workload": name3, "cells": cells3, "storage": "bf16", "mlups": {},
              "ms_per_step": {}, "steps": args.steps3, "warmup": args.warmup}
        for st in ("bf16", "f32", "f16"):
            s3 = Solver(cfg3, storage=st, stream=stream)
            s3.init_fields(f3["phi"], f3["psi"], f3["C"], f3["u"])
            if args.sor_tile_3d is not None:
                s3.set_sor_tile(args.sor_tile_3d)
                t3 = {"sor": args.sor_tile_3d}
            else:
                t3 = autotune.tune_single(s3, cfg3["nx"], lattice="d3q19", use_cache=False)
                d3.setdefault("sor_tune_ms", {})[st] = t3.get("timings")
            d3.setdefault("sor_variant", {})[st] = t3["sor"]
            s3.init_fields(f3["phi"], f3["psi"], f3["C"], f3["u"])
            tt, km = time_steps(s3, stream, flush, args.warmup, args.steps3, torch)
            d3["mlups"][st] = cells3 * args.steps3 / (tt / 1e3) / 1e6
            d3["ms_per_step"][st] = tt / args.steps3
            if st == "bf16":
                dg3 = s3.diagnostics()
                r3 = max(dg3["sor_rounds"], 1)
                d3["kernel_ms"] = km
                d3["sor_sweeps"] = dg3["sor_iters_psi"]
                d3["roofline"] = roofline3(km, cells3, st, r3, hbm, src)
                d3["gpu_launches_per_step"] = s3.kernel_count()
            steproof["3d_" + st] = step_roofline(d3["mlups"][st], "d3q19", st, hbm,
                                                 "HBM (1.1 GB of state)")
            s3.close()

    # Sec. 3.1's adsorption test in 3D: one octant of a droplet between mirror
    # planes (R = 30, 150^3 cells), FP32 and bfloat16
    octant = None
    if rank == 0 and not args.no_octant:
        cfgo = W.adsorption_octant_3d(R=30)
        cellso = cfgo["nx"] * cfgo["ny"] * cfgo["nz"]
        fo = W.initial_fields(cfgo)
        octant = {"workload": "adsorption_octant_3d D3Q19 150^3, mirror planes on every axis, "
                              "R=30, C0=5e-4, r_a=0.2 (Sec. 3.1)", "cells": cellso, "mlups": {},
                  "ms_per_step": {}, "steps": args.steps3, "warmup": args.warmup}
        for st in ("f32", "bf16"):
            so = Solver(cfgo, storage=st, stream=stream)
            so.init_fields(fo["phi"], fo["psi"], fo["C"], fo["u"])
            to = autotune.tune_single(so, cfgo["nx"], lattice="d3q19", use_cache=False)
            octant.setdefault("sor_variant", {})[st] = to["sor"]
            so.init_fields(fo["phi"], fo["psi"], fo["C"], fo["u"])
            tt, km = time_steps(so, stream, flush, args.warmup, args.steps3, torch)
            octant["mlups"][st] = cellso * args.steps3 / (tt / 1e3) / 1e6
            octant["ms_per_step"][st] = tt / args.steps3
            if st == "f32":
                octant["kernel_ms"] = km
            steproof["octant3d_" + st] = step_roofline(octant["mlups"][st], "d3q19", st, hbm,
                                                       "HBM (3.4 M cells)")
            so.close()

    # Sec. 3.4's bubble rise in 3D with soluble surfactant (Eo = 1, Mo = 0.1,
    # 2R/L_x = 0.4), R = 30 in the 5R x 5R x 10R channel
    bubble3 = None
    if rank == 0 and not args.no_bubble3d:
        cfgr = W.bubble_rise_3d(R=30)
        cellsr = cfgr["nx"] * cfgr["ny"] * cfgr["nz"]
        fr = W.initial_fields(cfgr)
        bubble3 = {"workload": "bubble_rise_3d D3Q19 150x150x300, walls x/y, periodic z, R=30, "
                               "Eo=1, Mo=0.1, rho/mu ratio 10, Bi=10, Pe=10 (Sec. 3.4)",
                   "cells": cellsr, "mlups": {}, "ms_per_step": {}, "steps": args.steps3,
                   "warmup": args.warmup}
        for st in ("f32", "bf16"):
            sr = Solver(cfgr, storage=st, stream=stream)
            sr.init_fields(fr["phi"], fr["psi"], fr["C"], fr["u"])
            tr = autotune.tune_single(sr, cfgr["nx"], lattice="d3q19", use_cache=False)
            bubble3.setdefault("sor_variant", {})[st] = tr["sor"]
            sr.init_fields(fr["phi"], fr["psi"], fr["C"], fr["u"])
            tt, km = time_steps(sr, stream, flush, args.warmup, args.steps3, torch)
            bubble3["mlups"][st] = cellsr * args.steps3 / (tt / 1e3) / 1e6
            bubble3["ms_per_step"][st] = tt / args.steps3
            if st == "f32":
                bubble3["kernel_ms"] = km
            steproof["bubble3d_" + st] = step_roofline(bubble3["mlups"][st], "d3q19", st, hbm,
                                                       "HBM (6.75 M cells)")
            sr.close()
        del fr

    # Sec. 3.2's migration test in 3D: a droplet driven by a fixed surfactant
    # gradient (linear EOS, no transport), R = 30 in the 5R x 5R x 10R box
    migration = None
    if rank == 0 and not args.no_migration:
        cfgm = W.migration_3d(R=30)
        cellsm = cfgm["nx"] * cfgm["ny"] * cfgm["nz"]
        fm = W.initial_fields(cfgm)
        migration = {"workload": "migration_3d D3Q19 150x150x300, walls x/y, periodic z, R=30, "
                                 "linear EOS, psi fixed at psi_inf z/L_z (Sec. 3.2)",
                     "cells": cellsm, "mlups": {}, "ms_per_step": {}, "steps": args.steps3,
                     "warmup": args.warmup}
        for st in ("f32", "bf16"):
            sm = Solver(cfgm, storage=st, stream=stream)
            sm.init_fields(fm["phi"], fm["psi"], fm["C"], fm["u"])
            tt, km = time_steps(sm, stream, flush, args.warmup, args.steps3, torch)
            migration["mlups"][st] = cellsm * args.steps3 / (tt / 1e3) / 1e6
            migration["ms_per_step"][st] = tt / args.steps3
            if st == "f32":
                migration["kernel_ms"] = km
            sm.close()
        del fm

    # one 2D instance far beyond the L2: the bubble rise's physics on a
    # 4096 x 4096 grid with a 16 x 16 array of bubbles (16.8 M cells)
    big = None
    if rank == 0 and not args.no_big2d:
        cfgb = W.bubble_array_2d()
        cellsb = cfgb["nx"] * cfgb["ny"]
        fb = W.initial_fields(cfgb)
        big = {"workload": "bubble_array_2d D2Q9 4096x4096 walls-x periodic-y, 16x16 bubbles "
                           "D=64 (the bubble rise's physics)", "cells": cellsb, "mlups": {},
               "ms_per_step": {}, "steps": args.steps3, "warmup": args.warmup}
        for st in ("f32", "f16"):
            sb = Solver(cfgb, storage=st, stream=stream)
            sb.init_fields(fb["phi"], fb["psi"], fb["C"], fb["u"])
            tb = autotune.tune_single(sb, cfgb["nx"], use_cache=False)
            big.setdefault("sor_variant", {})[st] = tb["sor"]
            sb.init_fields(fb["phi"], fb["psi"], fb["C"], fb["u"])
            tt, km = time_steps(sb, stream, flush, args.warmup, args.steps3, torch)
            big["mlups"][st] = cellsb * args.steps3 / (tt / 1e3) / 1e6
            big["ms_per_step"][st] = tt / args.steps3
            if st == "f32":
                dgb = sb.diagnostics()
                big["kernel_ms"] = km
                big["sor_sweeps"] = dgb["sor_iters_psi"]
                nkb = sb.kernel_count()
                sl = 1 if nkb == 2 else nkb - 4
                big["roofline"] = roofline2(km, cellsb, st, dgb["sor_iters_psi"], hbm, src,
                                            sor_launches=sl)
                if traffic_valid(sl, tb["sor"], "bytes_per_cell_hbm"):
                    big["roofline"]["traffic"] = (
                        TRAFFIC["bytes_per_cell_hbm"][str(tb["sor"])][big["roofline"]["kernel"]]
                        * cellsb)
                    big["roofline"]["traffic_source"] = (
                        "ncu on the 2048 x 2048 bubble array, scaled by cells")
            steproof["big2d_" + st] = step_roofline(big["mlups"][st], "d2q9", st, hbm,
                                                    "HBM (3 GB of state)")
            sb.close()
        del fb

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
           "data": "synthetic",
           "config": {"workload": name, "cells": cells, "storage": args.storage,
                      "sor_tile": tuned["sor"],
                      "l2": "flushed before every timed step (256 MiB write)",
                      "parallelism": f"replicas x{world}" if world > 1 else "single"},
           "roofline": roof, "kernel_ms": kmean, "sor_sweeps": sweeps, "sor_rounds": rounds,
           "sor_tune_ms": tuned.get("timings"),
           "gpu_launches": args.steps * s.kernel_count(),
           "forms_mlups": forms, "d3q19": d3, "batched": batched, "big2d": big,
           "adsorption_octant_3d": octant, "migration_3d": migration,
           "bubble_rise_3d": bubble3,
           "step_roofline": steproof,
           "clocks": clk, "e2e": e2e, "impl": "lbs", "src_sha": sha}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, name)
    s.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
