"""Benchmark: FP64 grid-point RK4 updates per second of the BSSN sweep.

Workload (default, N = 1): vacuum BSSN gauge wave on a 256^3 periodic grid
(24 evolved fields, 3.2 GB of state per time level), 1+log slicing and
Gamma-driver shift, amplitude 0.01, wavelength = box, dt = h/4.
One step = one full RK4 step (4 fused stage launches) over the whole grid.
The state (3.2 GB) is larger than L2 (129 MB), so every step streams from HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Prints one JSON line (rank 0).  With N > 1 (torchrun, one rank per GPU) every
rank evolves its own 256^3 instance (independent replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 256
METRIC = "FP64 grid-point RK4 updates/sec at 256^3"
UNIT = "grid-point updates/s"
WORKLOAD = "gauge_wave_256^3_vacuum_bssn_1+log_gamma_driver"
STATE_FIELDS = 24
# Algorithmic bytes per point per stage (each field read/written once from HBM):
# stage 1: U_n read, U_1 and acc written (3 x 24); stages 2-3: U_s, U_n, acc read,
# U_next, acc written (5 x 24); stage 4: U_s, U_n, acc read, U_n written (4 x 24).
BYTES_PER_POINT_STAGE = [8 * 3 * 24, 8 * 5 * 24, 8 * 5 * 24, 8 * 4 * 24]
# RK4 combine flops per field per stage (stage 1: 2; 2-3: 4; 4: 3)
COMBINE_FLOPS = [2, 4, 4, 3]
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one stage-1 launch
# of the vacuum stage kernel, from the committed ncu capture of the 96^3 case
# (3.027 + 7.288 GB), and the hash of the kernel sources it was taken on.  Reported scaled to the bench
# grid by points; null when the kernel sources differ from the profiled ones.
NCU_TRAFFIC = {"sources_sha256_16": "c1e137dd9707b898", "grid": 96, "bytes_per_launch": 10.314704e9}
KERNEL_SOURCES = ["common.cuh", "stage_kernel.cuh", "stage_vac.cu", "generated/bssn_algebra.cuh"]


def kernel_sources_hash():
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2606_02053_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=N_GRID, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reference_arm(args):
    """The oracle (plain FP64 CPU code) timed on the host cores, same metric."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    res = cpu_baseline_sample(args.grid, planes=16, repeats=max(1, args.steps))
    line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "grid": args.grid, "fields": STATE_FIELDS},
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"]},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(n, planes, repeats=1, state=None):
    """Oracle right-hand side on `planes` z-planes of the n^3 gauge wave; an RK4
    step costs four such evaluations per point (the combine is negligible)."""
    import numpy as np

    import oracle as O

    O.set_threads(os.cpu_count() or 1)
    h = 1.0 / n
    op = O.params_array(slicing=0, shift=1, eta=2.0, ko_sigma=0.1)
    og = O.OGrid((n, n, n), h)
    if state is None:
        state = O.init(og, op, O.id_array(0, A=0.01))
    O.rhs_planes(og, op, state, 0, 1)  # warm-up (thread pool)
    t0 = time.perf_counter()
    for _ in range(repeats):
        O.rhs_planes(og, op, state, 0, planes)
    dt = (time.perf_counter() - t0) / repeats
    pts = planes * n * n
    per_step = 4.0 * dt
    counts = O.flop_count(og, op, state)
    return {"value": pts / per_step, "seconds_per_step": per_step, "cores": O.max_threads(),
            "sample": f"oracle RHS on {planes} of {n} z-planes ({pts} points) x4 stages per RK4 step, "
                      f"{repeats} repeat(s); host threads {O.max_threads()}",
            "flops": counts}


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch

    from paper_2606_02053_gb300 import build
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.evolve import Evolution

    ws_, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws_ > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    n = args.grid
    h = 1.0 / n
    dt = 0.25 * h
    p = C.make_params(slicing=0, shift=1, eta=2.0, ko_sigma=0.1)
    g = C.make_grid(n, h)
    ev = Evolution(g, p, device=f"cuda:{local}")
    ev.init(C.make_id(0, A=0.01))
    U1 = torch.empty_like(ev.state)
    U2 = torch.empty_like(ev.state)
    acc = torch.empty_like(ev.state)
    stream = torch.cuda.current_stream()

    def stage_calls(t, events=None):
        seq = [(ev.state, U1), (U1, U2), (U2, U1), (U1, None)]
        for s, (src, dst) in enumerate(seq, start=1):
            if events is not None:
                events[s - 1][0].record(stream)
            C.check(C.cosmos_rk4_stage(g, p, s, src, ev.state, dst, acc, t, dt, ev.ws_rhs, stream))
            if events is not None:
                events[s - 1][1].record(stream)

    for w in range(args.warmup):
        stage_calls(w * dt)
    torch.cuda.synchronize()
    ev_pairs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(4)]
                for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        stage_calls((args.warmup + k) * dt, ev_pairs[k])
    stop.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed = start.elapsed_time(stop) * 1e-3
    stage_ms = [[ev_pairs[k][s][0].elapsed_time(ev_pairs[k][s][1]) for k in range(args.steps)] for s in range(4)]
    if dist:
        tt = torch.tensor([elapsed], device=f"cuda:{local}")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    nranks = ws_
    pts = float(n) ** 3
    value = nranks * pts * args.steps / elapsed
    gpu_launches = 4 * args.steps

    # ---- end to end through the C ABI with host buffers (pinned) ----
    nbytes = ev.state.numel() * 8
    host_in = torch.empty(ev.state.numel(), dtype=torch.float64, pin_memory=True)
    host_in.copy_(ev.state)
    host_out = torch.empty_like(host_in, pin_memory=True)
    dev = torch.empty_like(ev.state)
    e2e_steps = max(1, min(args.steps, 10))
    C.check(C.cosmos_evolve_host(g, p, host_in, host_out, dev, 1, 0.0, dt, ev.ws_rk4, stream))  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        C.check(C.cosmos_evolve_host(g, p, host_in, host_out, dev, 1, k * dt, dt, ev.ws_rk4, stream))
    e2e_t = time.perf_counter() - t0
    e2e = {"value": nranks * pts * e2e_steps / e2e_t if not dist else None, "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    if dist:
        tt = torch.tensor([e2e_t], device=f"cuda:{local}")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e["value"] = nranks * pts * e2e_steps / float(tt.item())

    # ---- FP64 peak of this GPU (in-run DFMA probe) ----
    scratch = torch.empty(152 * 8 * 256, dtype=torch.float64, device=f"cuda:{local}")
    fp64_peak = max(C.cosmos_probe_fp64(scratch, stream) for _ in range(3))

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # ---- CPU baseline (oracle) + algorithmic flop count ----
    cpu = None
    if not args.no_cpu_baseline:
        host_state = ev.get()
        cpu = cpu_baseline_sample(n, planes=16, repeats=1, state=host_state)
    avg_stage = [statistics.mean(v) * 1e-3 for v in stage_ms]
    dom = max(range(4), key=lambda s: avg_stage[s])
    roof = None
    if cpu is not None:
        c = cpu["flops"]
        rhs_flops = c["add"] + c["mul"] + c["div"] + c["sqrt"]
        flops_launch = pts * (rhs_flops + COMBINE_FLOPS[dom] * STATE_FIELDS)
        achieved = flops_launch / avg_stage[dom] / 1e12
        peak = fp64_peak / 1e12
        traffic = None
        if kernel_sources_hash() == NCU_TRAFFIC["sources_sha256_16"]:
            traffic = NCU_TRAFFIC["bytes_per_launch"] * (n / NCU_TRAFFIC["grid"]) ** 3
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_note": "bytes per launch, ncu at 96^3 scaled by points",
                "kernel": f"stage_kernel<T_vac, stage {dom + 1}>",
                "peak_source": "FP64 DFMA throughput measured in this run (cosmos_probe_fp64); nominal 1.25",
                "algorithmic_flops_per_point_rhs": rhs_flops,
                "hbm_GBps_algorithmic": pts * BYTES_PER_POINT_STAGE[dom] / avg_stage[dom] / 1e9}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": n, "fields": STATE_FIELDS, "dt_over_h": 0.25,
                       "parallelism": f"replicas{nranks}" if nranks > 1 else "single",
                       "l2": "inputs larger than L2 (3.2 GB state per level)"},
            "stage_ms": [1e3 * s for s in avg_stage], "roofline": roof, "gpu_launches": gpu_launches,
            "e2e": e2e, "clocks": clk,
            "cpu_baseline": None if cpu is None else {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"],
                                                      "kind": "oracle", "sample": cpu["sample"]}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
