"""Benchmark: FP64 grid-point RK4 updates per second of the BSSN sweep.

Workload (default, N = 1): vacuum BSSN gauge wave on a 256^3 periodic grid
(24 evolved fields, 3.2 GB of state per time level), 1+log slicing and
Gamma-driver shift, amplitude 0.01, wavelength = box, dt = h/4.
One step = one full RK4 step (4 fused stage launches) over the whole grid.
The state (3.2 GB) is larger than L2 (129 MB), so every step streams from HBM.

The same line carries the rest of the metric, measured on one GPU: the same
sweep on a generic state (sweep_generic), the 64-instance batched scan against
the per-instance loop (batched) and the 96^3 adjoint against finite
differences (adjoint).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--decompose]
Prints one JSON line (rank 0).  With N > 1 (torchrun, one rank per GPU) every
rank evolves its own 256^3 instance (independent replicas, weak scaling); with
--decompose the ranks hold z-slabs of one 256^3 grid (strong scaling).
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
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each pass of the vacuum stage, from the committed ncu capture of the 96^3
# case (the derivative pass: exponent scan + limb conversion + integer pass;
# the algebra pass: the mean over a step's stages 1, 2, 3, 4), and the hash of
# the kernel sources it was taken on.  Reported scaled to the bench grid by
# points; null when the kernel sources differ from the profiled ones.
NCU_TRAFFIC = {"sources_sha256_16": "6129913db8cd4ae6", "grid": 96,
               "bytes_per_launch": {
                   # exponent scan (stage 1 only) + limb copy + integer pass, mean over the 4 stages of a step
                   "derivative": ((169877760 + 3258880) + (169882880 + 122540544) + (237195264 + 1092143360)
                                  + (169875712 + 122436608) + (237027584 + 1092392960)
                                  + (169882112 + 121968384) + (237173760 + 1092693760)
                                  + (169882880 + 122204928) + (237097728 + 1092242688)) / 4,
                   # algebra pass, modes 1, 2, 2, 3 of one step
                   "algebra": ((1396294400 + 521755648)
                               + (1671427584 + 385866240)
                               + (1672915200 + 386181120)
                               + (1646590720 + 483951104)) / 4}}
# derivative-pass buffer: first + second derivatives and KO terms per point (vacuum)
DERIV_DOUBLES = 162
KERNEL_SOURCES = ["common.cuh", "stage_kernel.cuh", "stage_int.cuh", "limbs.cu", "stage_vac.cu",
                  "generated/bssn_algebra.cuh"]


def generated_algebra_ops(variant="vac"):
    """Operation count of the generated pointwise algebra of a matter variant
    (the expression DAG after common-subexpression elimination: every named
    intermediate and every symmetric tensor component formed once), read from
    the comment the code generator writes into the generated header."""
    import ast
    import re

    path = os.path.join(ROOT, "paper_2606_02053_gb300", "csrc", "generated", "bssn_algebra.cuh")
    with open(path) as fh:
        for line in fh:
            m = re.match(r"// variant (\w+): .* ops (\{.*\})", line)
            if m and m.group(1) == variant:
                return sum(ast.literal_eval(m.group(2)).values())
    raise RuntimeError("no operation count for variant " + variant)


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_sources_hash():
    """Hash of the code of the files that make the stage kernels: comments
    removed and every run of whitespace (line breaks included) made one space,
    so that only changes to the code itself change it."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2606_02053_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        text = re.sub(r"\s+", " ", text).strip()
        h.update(text.encode())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20 for the sweep and the reference arm, 150 for the scan)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=N_GRID, help=argparse.SUPPRESS)
    ap.add_argument("--no-cpu-baseline", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-extras", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--state", default="gauge", choices=["gauge", "generic"], help=argparse.SUPPRESS)
    ap.add_argument("--decompose", action="store_true",
                    help="hold the 256^3 grid as one z-slab per rank (ghost-plane exchange every RK4 stage; "
                         "strong scaling) instead of one whole grid per rank")
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "scan", "adjoint", "flrw", "fmr", "isocurvature", "mode"],
                    help="sweep: single 256^3 grid (headline); scan: 64-instance batched threshold scan; "
                         "adjoint: gradients of collapse diagnostics at 96^3; flrw: 128^3 FLRW + zeta, "
                         "200 steps, constraint norms; fmr: 128^3 FLRW + zeta with two nested 96^3 "
                         "refinement levels; isocurvature: 128^3 fluid + scalar isocurvature data; mode: "
                         "128^3 single-mode FLRW perturbation")
    ap.add_argument("--adjoint-steps", type=int, default=256, help=argparse.SUPPRESS)
    ap.add_argument("--adjoint-grid", type=int, default=96, help=argparse.SUPPRESS)
    ap.add_argument("--instances", type=int, default=64, help=argparse.SUPPRESS)
    a = ap.parse_args()
    if a.steps is None:
        a.steps = 150 if a.workload == "scan" and a.impl != "reference" else 20
        if a.workload == "fmr":
            a.steps = 16
    return a


def flrw_workload(args):
    """128^3 radiation FLRW + Gaussian zeta (mu = 0.5, sigma = L/8, H0 L = 40, w = 1/3),
    200 RK4 steps with dt = h/4: fluid-sweep throughput (CUDA events around the
    steps, constraint evaluations excluded) and the Hamiltonian / momentum
    constraint norms every 20 steps."""
    import torch

    from paper_2606_02053_gb300 import build
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.evolve import Evolution

    build.build()
    n, steps, every = 128, 200, 20
    h = 1.0 / n
    p = C.make_params(slicing=0, shift=1, fluid=1, w=1.0 / 3.0, H0=40.0)
    ev = Evolution(C.make_grid(n, h, x0=(-(n // 2) * h,) * 3), p)
    ident = C.make_id(1, mu=0.5, sigma=0.125)
    dt = 0.25 * h
    ev.init(ident)
    ev.step(0.0, dt, steps=max(args.warmup, 1))  # warm-up, then restart from the initial data
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev.init(ident)
    torch.cuda.synchronize()
    init_ms = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    norms = [(0, ev.constraints()[1].tolist())]  # synchronous: the norms come back to the host
    constraints_ms = 1e3 * (time.perf_counter() - t0)
    total_ms = 0.0
    for s0 in range(0, steps, every):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ev.step(s0 * dt, dt, steps=every)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        norms.append((s0 + every, ev.constraints()[1].tolist()))
    value = n ** 3 * steps / (total_ms * 1e-3)
    line = {"metric": "FP64 grid-point RK4 updates/sec, 128^3 FLRW + zeta (fluid)", "value": value, "unit": UNIT,
            "n_gpus": 1, "steps": steps, "warmup": max(args.warmup, 1), "ms_per_step": total_ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "flrw_zeta_128^3_radiation_fluid", "grid": n, "mu": 0.5, "sigma": 0.125,
                       "H0L": 40.0, "dt_over_h": 0.25},
            "constraint_norms": {"columns": ["step", "L2_H", "L2_Mx", "L2_My", "L2_Mz", "Linf_H", "Linf_Mx",
                                             "Linf_My", "Linf_Mz"],
                                 "rows": [[s] + v for s, v in norms]},
            "initial_data_ms": init_ms, "constraints_ms_per_evaluation": constraints_ms,
            "gpu_launches": steps * 4 * 6}  # per stage: primitives, fluxes, exponents, limbs, derivative, algebra
    print(json.dumps(line), flush=True)


def isocurvature_workload(args):
    """128^3 FLRW + zeta with a massless-scalar isocurvature profile (initial-data
    kind 2: phi = A exp(-r^2/(2 sigma^2)), A = 0.02, the fluid energy from the
    discrete Hamiltonian constraint with both sources), fluid + scalar, 100 RK4
    steps of dt = h/4: throughput and the constraint norms at the start and the end."""
    import torch

    from paper_2606_02053_gb300 import build
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.evolve import Evolution

    build.build()
    n, steps = 128, 100
    h = 1.0 / n
    p = C.make_params(slicing=0, shift=1, fluid=1, scalar=1, w=1.0 / 3.0, H0=40.0)
    ev = Evolution(C.make_grid(n, h, x0=(-(n // 2) * h,) * 3), p)
    ident = C.make_id(2, A=0.02, mu=0.3, sigma=0.125, q=(1.0, 0.9, 1.1))
    dt = 0.25 * h
    ev.init(ident)
    ev.step(0.0, dt, steps=max(args.warmup, 1))
    ev.init(ident)
    norms0 = ev.constraints()[1].tolist()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ev.step(0.0, dt, steps=steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    norms1 = ev.constraints()[1].tolist()
    line = {"metric": "FP64 grid-point RK4 updates/sec, 128^3 isocurvature data (fluid + scalar)",
            "value": n ** 3 * steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": max(args.warmup, 1), "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "isocurvature_128^3_fluid_scalar", "grid": n, "A": 0.02, "mu": 0.3,
                       "sigma": 0.125, "q": [1.0, 0.9, 1.1], "H0L": 40.0, "dt_over_h": 0.25},
            "constraint_norms": {"columns": ["L2_H", "L2_Mx", "L2_My", "L2_Mz", "Linf_H", "Linf_Mx", "Linf_My",
                                             "Linf_Mz"], "start": norms0, "end": norms1},
            "gpu_launches": steps * 4 * 6}
    print(json.dumps(line), flush=True)


def mode_workload(args):
    """The paper's first example on a 128^3 grid: radiation FLRW (w = 1/3, H0 = 2)
    with the lapse perturbed by one Fourier mode along x, alpha = 1 + 1e-7 cos(2 pi x),
    harmonic slicing with the background trace and a frozen shift, no
    Kreiss-Oliger term, evolved to t = 0.5 (256 steps of dt = h/4): throughput
    and the complex amplitude of the mode in K at the end (the linear-theory
    comparison is the test suite's)."""
    import numpy as np
    import torch

    from paper_2606_02053_gb300 import build
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.evolve import Evolution

    build.build()
    n, H0, eps, w = 128, 2.0, 1e-7, 1.0 / 3.0
    h = 1.0 / n
    steps = int(round(0.5 / (0.25 * h)))
    p = C.make_params(slicing=1, shift=0, ko_sigma=0.0, fluid=1, w=w, H0=H0)
    ev = Evolution(C.make_grid(n, h), p)
    x = h * np.arange(n)
    s = np.zeros((28, n, n, n))
    s[0] = s[1] = s[4] = s[6] = 1.0
    s[7] = -3.0 * H0
    s[17] = (1.0 + eps * np.cos(2.0 * np.pi * x))[None, None, :]
    s[24] = 3.0 * H0 * H0 / (8.0 * np.pi)
    dt = 0.25 * h
    ev.set_state(s)
    ev.step(0.0, dt, steps=max(args.warmup, 1))
    ev.set_state(s)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ev.step(0.0, dt, steps=steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    K = ev.view()[7, :, :, :n].mean(dim=(0, 1)).cpu().numpy()
    amp = complex(K @ (np.exp(-2j * np.pi * x) * (2.0 / n)))
    line = {"metric": "FP64 grid-point RK4 updates/sec, 128^3 single-mode FLRW perturbation",
            "value": n ** 3 * steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": max(args.warmup, 1), "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "single_mode_128^3_radiation_fluid", "grid": n, "eps": eps, "H0": H0,
                       "t_end": steps * dt, "dt_over_h": 0.25, "slicing": "harmonic", "shift": "frozen"},
            "K_mode_amplitude_end": [amp.real, amp.imag],
            "gpu_launches": steps * 4 * 6}
    print(json.dumps(line), flush=True)


def fmr_workload(args):
    """Fixed mesh refinement: 128^3 radiation FLRW + Gaussian zeta (mu = 0.5,
    sigma = L/8, H0 L = 40, w = 1/3) on level 0 and two nested 96^3 levels
    (89^3 interior points each, spacings h/2 and h/4) centred on the
    perturbation; one step = one level-0 step of dt = h/4 with 2 and 4
    substeps of levels 1 and 2.  Reports interior grid-point RK4 updates per
    second over all levels, the same level arrays stepped as plain periodic
    grids (no ghost filling or injection) for the overhead, and the interior
    constraint norms of every level at the start and the end."""
    import numpy as np
    import torch

    from paper_2606_02053_gb300 import build, inputs
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.evolve import Evolution
    from paper_2606_02053_gb300.fmr import Hierarchy

    build.build()
    n0, nc, nlev = 128, 96, 3
    h0 = 1.0 / n0
    lv = inputs.nested_boxes(n0, h0, (-(n0 // 2) * h0,) * 3, nlev, [nc] * (nlev - 1))
    p = C.make_params(slicing=0, shift=1, fluid=1, w=1.0 / 3.0, H0=40.0)
    H = Hierarchy(lv, p, pitch_align=32)
    ident = C.make_id(1, mu=0.5, sigma=0.125)
    dt0 = 0.25 * h0
    stream = torch.cuda.current_stream()

    def interior_norms():
        out = []
        for l in range(nlev):
            ev = Evolution(H.grid(l), p)
            ev.state.copy_(H.states[l])
            hm, _ = ev.constraints(want_fields=True)
            lo, hi = lv[l]["lo"], lv[l]["hi"]
            v = hm[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].reshape(4, -1)
            out.append([float(np.sqrt((v[m] ** 2).mean())) for m in range(4)])
            del ev
        return out

    H.init(ident)
    H.step(0.0, dt0, max(args.warmup, 1))
    H.init(ident)
    norms0 = interior_norms()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    H.step(0.0, dt0, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    norms1 = interior_norms()
    interior = sum(H.interior_points(l) * 2 ** l for l in range(nlev))
    arrays = sum(lv[l]["n"][0] * lv[l]["n"][1] * lv[l]["n"][2] * 2 ** l for l in range(nlev))
    # the same level arrays stepped as plain periodic grids, as many steps each
    evs = [Evolution(H.grid(l), p) for l in range(nlev)]
    for l, ev in enumerate(evs):
        ev.state.copy_(H.states[l])
        ev.step(0.0, dt0 / 2 ** l, 1)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(args.steps):
        for l, ev in enumerate(evs):
            ev.step(0.0, dt0 / 2 ** l, 2 ** l)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    del evs
    value = interior * args.steps / (ms * 1e-3)
    launches_per_level_step = 24  # 4 stages x (primitives, fluxes, exponents, limbs, derivative, algebra)
    launches_per_fill = 4         # time interpolation, x, y and z passes
    launches = sum(2 ** l * (launches_per_level_step + (4 * launches_per_fill if l else 0)) for l in range(nlev))
    launches += sum(2 ** (l - 1) for l in range(1, nlev))  # injections
    launches += launches_per_fill * (nlev - 1)              # final ghost fills
    line = {"metric": "FP64 interior grid-point RK4 updates/sec, 128^3 FLRW + zeta with 2 nested 96^3 levels",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 1),
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fmr_flrw_zeta_128^3_plus_2x96^3_levels", "levels": nlev, "grid": n0,
                       "level_arrays": [list(v["n"]) for v in lv], "interior": [H.interior_points(l)
                                                                               for l in range(nlev)],
                       "mu": 0.5, "sigma": 0.125, "H0L": 40.0, "dt_over_h": 0.25,
                       "interior_updates_per_step": interior, "array_updates_per_step": arrays},
            "plain_level_steps": {"ms_per_step": ms_plain / args.steps,
                                  "fmr_overhead": ms / ms_plain - 1.0},
            "interior_constraint_norms_L2": {"columns": ["level", "H", "Mx", "My", "Mz"],
                                             "start": [[l] + v for l, v in enumerate(norms0)],
                                             "end": [[l] + v for l, v in enumerate(norms1)]},
            "gpu_launches": launches * args.steps}
    print(json.dumps(line), flush=True)


def measure_scan(n_instances, K, W, rank=0, world=1, autotune=True):
    """Batched threshold scan against the plain per-instance loop: `n_instances` FLRW +
    zeta instances on uneven 64^3..96^3 grids (radiation fluid w = 1/3, H0 L = 40, mu,
    sigma, axis ratios from SplitMix64 seed 2606), dt = h/4 per instance.  The batch
    runs W warm-up and K timed steps as one CUDA graph; the loop (cosmos_rk4_step per
    grid) runs the same steps from the same states; both end in the same states."""
    import torch

    from paper_2606_02053_gb300 import inputs
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.batch import BatchScan
    from paper_2606_02053_gb300.dist import max_over_ranks, shard_instances, sum_over_ranks

    inst_all = inputs.scan_instances(n_instances, seed=2606)
    mine = shard_instances([d["n"] ** 3 for d in inst_all], world)[rank]
    inst = [inst_all[i] for i in mine]
    p = C.make_params(slicing=0, shift=1, fluid=1, w=1.0 / 3.0, H0=40.0)
    grids, dts, ids = [], [], []
    for d in inst:
        n = d["n"]
        h = 1.0 / n
        grids.append(C.make_grid(n, h, x0=(-(n // 2) * h,) * 3))
        dts.append(0.25 * h)
        ids.append(C.make_id(1, mu=d["mu"], sigma=d["sigma"], q=d["q"]))
    total_pts = float(sum(g.nx * g.ny * g.nz for g in grids))
    b = BatchScan(grids, p, dts, max_steps=W + K)
    b.init(ids)
    init_states = [s.clone() for s in b.states]
    tune = b.autotune(reps=2) if autotune else None
    stream = torch.cuda.Stream()
    b.run(0, W, use_graph=True, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.run(W, K, use_graph=True, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    t_batch = max_over_ranks(e0.elapsed_time(e1) * 1e-3)
    # plain per-instance loop, same steps, one shared workspace
    nbmax = max(C.cosmos_workspace_bytes(g, p, C.COSMOS_OP_RK4) for g in grids)
    ws = torch.empty((nbmax + 7) // 8, dtype=torch.float64, device="cuda")
    loop_states = [s.clone() for s in init_states]
    for g, st, dt in zip(grids, loop_states, dts):
        for k in range(W):
            C.check(C.cosmos_rk4_step(g, p, st, k * dt, dt, ws))
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for g, st, dt in zip(grids, loop_states, dts):
        for k in range(W, W + K):
            C.check(C.cosmos_rk4_step(g, p, st, k * dt, dt, ws))
    f1.record()
    torch.cuda.synchronize()
    t_loop = max_over_ranks(f0.elapsed_time(f1) * 1e-3)
    max_diff = max_over_ranks(max(float((a - c).abs().max()) for a, c in zip(b.states, loop_states)))
    scale = max(float(a.abs().max()) for a in loop_states)
    total_pts = sum_over_ranks(total_pts)
    del b, init_states, loop_states, ws
    torch.cuda.empty_cache()
    return {"instances": len(inst_all), "grid_sizes": [d["n"] for d in inst_all], "points_total": int(total_pts),
            "steps_timed": K, "warmup": W, "value": total_pts * K / t_batch,
            "per_instance_loop_value": total_pts * K / t_loop, "speedup": t_loop / t_batch,
            "ms_per_step": 1e3 * t_batch / K, "loop_ms_per_step": 1e3 * t_loop / K,
            "max_abs_diff_vs_loop": max_diff, "max_rel_diff_vs_loop": max_diff / scale, "autotune": tune,
            "gpu_launches": K * 4 * 6}  # per stage: primitives, fluxes, exponents, limbs, derivative, algebra


def scan_workload(args):
    """The batched threshold scan as its own line (150 steps by default)."""
    import torch

    from paper_2606_02053_gb300 import build

    ws_, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws_ > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
    if rank == 0:
        build.build()
    if ws_ > 1:
        tdist.barrier()
    r = measure_scan(args.instances, args.steps, args.warmup, rank, ws_)
    if rank != 0:
        return
    line = {"metric": f"batched threshold-scan FP64 grid-point RK4 updates/sec ({r['instances']} instances, "
                      f"{min(r['grid_sizes'])}^3-{max(r['grid_sizes'])}^3)",
            "value": r["value"], "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "n_gpus": ws_,
            "config": {"workload": f"flrw_zeta_scan_{r['instances']}_instances_fluid_w1/3",
                       "instances": r["instances"], "points_total": r["points_total"],
                       "grid_sizes": r["grid_sizes"]},
            "per_instance_loop_value": r["per_instance_loop_value"], "batched_speedup": r["speedup"],
            "batched_vs_loop_max_abs_diff": r["max_abs_diff_vs_loop"], "autotune": r["autotune"],
            "gpu_launches": r["gpu_launches"]}
    print(json.dumps(line), flush=True)


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
    """The oracle (plain FP64 CPU code) timed on the host cores, same metric.  One step
    evaluates the four right-hand sides of an RK4 step on a slab of `planes` z-planes of
    the 256^3 gauge-wave state (the oracle cannot step the whole grid in a bench run):
    the timed region really takes ms_per_step x steps, and value = points updated / s."""
    import oracle as O

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n, planes = args.grid, 8
    O.set_threads(os.cpu_count() or 1)
    h = 1.0 / n
    op = O.params_array(slicing=0, shift=1, eta=2.0, ko_sigma=0.1)
    og = O.OGrid((n, n, n), h)
    state = O.init(og, op, O.id_array(0, A=0.01))

    def step():
        for _ in range(4):
            O.rhs_planes(og, op, state, 0, planes)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    elapsed = time.perf_counter() - t0
    value = planes * n * n * args.steps / elapsed
    sample = (f"oracle: the 4 right-hand sides of an RK4 step on {planes} of {n} z-planes ({planes * n * n} points) "
              f"per step, {args.steps} steps after {args.warmup} warm-up; host threads {O.max_threads()}")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "grid": n, "fields": STATE_FIELDS,
                       "sampled": f"each step updates {planes} of the {n} z-planes; the rate is per point"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(n, planes, repeats=1, state=None, warmups=0):
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
    for _ in range(warmups):  # untimed repeats of the timed sample
        O.rhs_planes(og, op, state, 0, planes)
    t0 = time.perf_counter()
    for _ in range(repeats):
        O.rhs_planes(og, op, state, 0, planes)
    dt = (time.perf_counter() - t0) / repeats
    pts = planes * n * n
    per_step = 4.0 * dt
    cores = O.max_threads()
    # the same oracle on one core, on a 2-plane slab
    O.set_threads(1)
    t1 = time.perf_counter()
    O.rhs_planes(og, op, state, 0, 2)
    one_core = 2 * n * n / (4.0 * (time.perf_counter() - t1))
    O.set_threads(os.cpu_count() or 1)
    counts = O.flop_count(og, op, state)
    parts = O.flop_count_parts(og, op, state)
    return {"value": pts / per_step, "seconds_per_step": per_step, "cores": cores, "value_1_core": one_core,
            "sample": f"oracle RHS on {planes} of {n} z-planes ({pts} points) x4 stages per RK4 step, "
                      f"{repeats} repeat(s); host threads {cores}; value_1_core: 2 planes on one thread",
            "flops": counts, "flops_parts": parts}


def measure_adjoint(n, steps, every=16, point_checks=True):
    """FLRW + Gaussian zeta on n^3 (mu = 0.6, sigma = L/8, radiation fluid, H0 L = 40),
    `steps` RK4 steps (dt = h/4), checkpoints every `every` steps.  Gradients of the
    minimum central lapse and of the peak compaction with respect to mu and to zeta at
    every point, by the adjoint; checked with central differences (h = 1e-6) along mu
    and, with point_checks, on 8 random points and 2 random directions of zeta.  The
    adjoint's cost is set against the plain finite-difference loop (2 forward runs per
    scalar), whose forward run is timed here."""
    import numpy as np
    import torch

    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.adjoint import CollapseRun, CosmosAdjoint

    h = 1.0 / n
    p = C.make_params(slicing=0, shift=1, fluid=1, w=1.0 / 3.0, H0=40.0)
    run = CollapseRun(n, p, dt=0.25 * h, steps=steps, checkpoint_every=every)
    x = (-(n // 2) + torch.arange(n, dtype=torch.float64, device="cuda")) * h
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    shape = torch.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * (1.0 / 8.0) ** 2)).reshape(-1).contiguous()
    mu0 = 0.6

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    run.forward(mu0 * shape)  # warm-up
    mu = torch.tensor(mu0, dtype=torch.float64, device="cuda", requires_grad=True)
    zeta = (mu * shape).contiguous()
    out, t_fwd = timed(lambda: CosmosAdjoint.apply(zeta, run))
    (g_mu_min,), _ = timed(lambda: torch.autograd.grad(out[0], mu, retain_graph=True))
    # per-point gradients of both diagnostics in one reverse sweep (each checkpoint segment
    # replayed once for both); one sweep per diagnostic timed beside it
    amin, cpeak, rec = run.forward((mu0 * shape).contiguous())
    (zb_min, zb_comp), t_both = timed(lambda: run.backward_many(rec, [(1.0, 0.0), (0.0, 1.0)]))
    zb_min1, t_bmin = timed(lambda: run.backward(rec, 1.0, 0.0))
    assert torch.equal(zb_min1, zb_min)  # the same reverse arithmetic either way
    del zb_min1
    g_mu_comp = float(torch.dot(zb_comp, shape))
    hfd = 1e-6
    checks = []

    def fd(direction, label):
        zp = (mu0 * shape + hfd * direction).contiguous()
        zm = (mu0 * shape - hfd * direction).contiguous()
        (a1, c1, _), t1 = timed(lambda: run.forward(zp))
        a2, c2, _ = run.forward(zm)
        fmin, fcomp = (a1 - a2) / (2 * hfd), (c1 - c2) / (2 * hfd)
        amn = float(torch.dot(zb_min, direction))
        acp = float(torch.dot(zb_comp, direction))
        checks.append({"what": label, "fd_min_lapse": fmin, "adj_min_lapse": amn, "fd_compaction": fcomp,
                       "adj_compaction": acp})
        return t1

    t_fwd_plain = fd(shape, "mu")
    if point_checks:
        rng = np.random.default_rng(2606)
        centre = n // 2
        for _ in range(8):
            i, j, k = (int(v) for v in rng.integers(centre - n // 8, centre + n // 8, size=3))
            e = torch.zeros_like(shape)
            e[(k * n + j) * n + i] = 1.0
            fd(e, f"zeta[{i},{j},{k}]")
        for r in range(2):
            d = torch.from_numpy(rng.standard_normal(n ** 3)).cuda() * shape
            fd(d, f"random direction {r}")

    def rel(a, b):
        return abs(a - b) / max(abs(a), abs(b), 1e-300)

    mu_check = checks[0]
    t_adj = t_fwd + t_both
    nscal = n ** 3
    res = {"grid": n, "steps": steps, "checkpoint_every": every, "mu": mu0, "sigma": 0.125, "H0L": 40.0,
           "forward_s": t_fwd, "forward_plain_s": t_fwd_plain, "backward_both_s": t_both,
           "backward_one_diagnostic_s": t_bmin, "adjoint_total_s": t_adj,
           "speedup_all_zeta_points": (2 * nscal * t_fwd_plain) / t_adj,
           "speedup_11_scalars": (2 * 11 * t_fwd_plain) / t_adj,
           "speedup_note": "finite-difference loop time (2 plain forward runs per scalar, the forward run timed "
                           "here) / adjoint time (forward with checkpoints + one reverse sweep giving both "
                           "diagnostics' gradients)",
           "min_central_lapse": float(out[0]), "min_lapse_step": rec["nstar"], "peak_compaction": float(out[1]),
           "peak_shell": rec["kstar"], "dmin_dmu": float(g_mu_min), "dcomp_dmu": g_mu_comp,
           "mu_fd_rel_diff_min_lapse": rel(mu_check["fd_min_lapse"], float(g_mu_min)),
           "mu_fd_rel_diff_compaction": rel(mu_check["fd_compaction"], g_mu_comp),
           "gpu_launches_per_forward_step": 16 + 8 + 1}  # 4 stages x 6 kernels + the central-lapse read
    if point_checks:
        res["fd_checks"] = checks
        res["worst_rel_diff_min_lapse"] = max(rel(c["fd_min_lapse"], c["adj_min_lapse"]) for c in checks)
        res["worst_rel_diff_compaction"] = max(rel(c["fd_compaction"], c["adj_compaction"]) for c in checks)
    del run
    torch.cuda.empty_cache()
    return res


def adjoint_workload(args):
    """Gradients of collapse diagnostics at 96^3 x 256 steps as their own line, with the
    per-point finite-difference checks."""
    from paper_2606_02053_gb300 import build

    build.build()
    r = measure_adjoint(args.adjoint_grid, args.adjoint_steps)
    n, steps = r["grid"], r["steps"]
    line = {"metric": f"adjoint gradient of collapse diagnostics ({n}^3, {steps} steps): speedup over finite differences",
            "value": r["speedup_all_zeta_points"], "unit": "x (FD loop time / adjoint time, all zeta points)",
            "n_gpus": 1, "steps": steps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "flrw_zeta_adjoint", "grid": n, "mu": r["mu"], "sigma": r["sigma"],
                       "H0L": r["H0L"], "checkpoint_every": r["checkpoint_every"]}, **r}
    print(json.dumps(line), flush=True)


def decomposed_workload(args):
    """The headline gauge wave held as z-slabs, one per rank (strong scaling): before
    every RK4 stage the ranks exchange 3 ghost planes with their two neighbours
    (periodic) and take the largest per-field exponent (NCCL); each rank advances its
    own planes with cosmos_rk4_stage_slab.  With one rank the slab's ghost planes come
    from its own planes.  Bitwise the whole-grid results (tests/test_gpu_slab.py)."""
    import torch

    from paper_2606_02053_gb300 import build
    from paper_2606_02053_gb300 import cosmos as C
    from paper_2606_02053_gb300.dist import max_over_ranks
    from paper_2606_02053_gb300.slab import DistExchange, LocalExchange, Slab, SlabEvolution, slab_bounds

    ws_, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws_ > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
    if rank == 0:
        build.build()
    if ws_ > 1:
        tdist.barrier()
    n = args.grid
    h = 1.0 / n
    dt = 0.25 * h
    p = C.make_params(slicing=0, shift=1, eta=2.0, ko_sigma=0.1)
    k0, k1 = slab_bounds(n, ws_)[rank]
    slab = Slab((n, n, n), (h, h, h), (0.0, 0.0, 0.0), p, k0, k1, device=f"cuda:{local}")
    # the gauge wave depends on x alone: every plane of the slab, ghosts included, is the whole grid's
    C.check(C.cosmos_init_grid(slab.g, p, C.make_id(0, A=0.01), slab.state, None))
    evo = SlabEvolution([slab], DistExchange() if ws_ > 1 else LocalExchange())
    evo.step(0.0, dt, steps=args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    if ws_ > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    evo.step(args.warmup * dt, dt, steps=args.steps)
    e1.record()
    torch.cuda.synchronize()
    if ws_ > 1:
        tdist.barrier()
    clk = clocks.stop()
    elapsed = max_over_ranks(e0.elapsed_time(e1) * 1e-3)
    if rank == 0:
        line = {"metric": METRIC, "value": float(n) ** 3 * args.steps / elapsed, "unit": UNIT, "n_gpus": ws_,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": n, "fields": STATE_FIELDS, "dt_over_h": 0.25,
                           "parallelism": f"z-slabs x{ws_} (3 ghost planes a side, exchange every stage)",
                           "l2": "inputs larger than L2 (3.2 GB state per level)"},
                "gpu_launches": 16 * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    if ws_ > 1:
        tdist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.decompose:
        return decomposed_workload(args)
    if args.workload == "scan":
        return scan_workload(args)
    if args.workload == "adjoint":
        return adjoint_workload(args)
    if args.workload == "flrw":
        return flrw_workload(args)
    if args.workload == "fmr":
        return fmr_workload(args)
    if args.workload == "isocurvature":
        return isocurvature_workload(args)
    if args.workload == "mode":
        return mode_workload(args)

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
    host_gauge_wave = ev.get() if rank == 0 and not args.no_cpu_baseline else None
    if args.state == "generic":  # profiling only: the same sweep on the generic state of sweep_generic
        from paper_2606_02053_gb300 import inputs

        ev.set_state(inputs.smooth_state(n, seed=2562, kmax=6, scale=0.5))
    U1 = torch.empty_like(ev.state)
    U2 = torch.empty_like(ev.state)
    acc = torch.empty_like(ev.state)
    stream = torch.cuda.current_stream()

    # pass options as cosmos_rk4_step uses them: the algebra pass of stages 1-3 records the exponents
    # of the state it writes (+32, stage 1 clearing the record first: +64), the derivative pass of
    # stages 2-4 takes them instead of scanning (+16)
    pass_opts = {(1, 1): 0, (1, 2): 32 + 64, (2, 1): 16, (2, 2): 32, (3, 1): 16, (3, 2): 32, (4, 1): 16, (4, 2): 0}

    def stage_calls(t, events=None):
        """One RK4 step as 4 stages x (derivative pass, algebra pass), the sequence of
        cosmos_rk4_step; events bracket each pass on the launching stream."""
        seq = [(ev.state, U1), (U1, U2), (U2, U1), (U1, None)]
        for s, (src, dst) in enumerate(seq, start=1):
            for pss in (1, 2):
                if events is not None:
                    events[s - 1][pss - 1][0].record(stream)
                C.check(C.cosmos_stage_pass(g, p, pss + pass_opts[(s, pss)], s, src, ev.state, dst, acc, t, dt,
                                            ev.ws_rhs, stream))
                if events is not None:
                    events[s - 1][pss - 1][1].record(stream)

    for w in range(args.warmup):
        stage_calls(w * dt)
    torch.cuda.synchronize()
    ev_pairs = [[[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
                 for _ in range(4)] for _ in range(args.steps)]
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
    # pass_ms[pass][stage] = list over steps
    pass_ms = [[[ev_pairs[k][s][q][0].elapsed_time(ev_pairs[k][s][q][1]) for k in range(args.steps)] for s in range(4)]
               for q in range(2)]
    from paper_2606_02053_gb300.dist import max_over_ranks

    elapsed = max_over_ranks(elapsed)
    nranks = ws_
    pts = float(n) ** 3
    value = nranks * pts * args.steps / elapsed
    # per step: exponent scan (stage 1), 4 x (limb copy, integer derivative pass, algebra pass),
    # exponent record compaction (stages 1-3)
    gpu_launches = 16 * args.steps

    # ---- end to end through the C ABI with host buffers (pinned) ----
    # Every step copies its inputs from pinned host memory and reads its result
    # back.  The line's figure: a sequence of independent 256^3 states, one RK4
    # step each, through cosmos_evolve_host_many (the copies of other states
    # overlap each state's step); beside it the single state of
    # cosmos_evolve_host, whose copies overlap only the first and last passes.
    nbytes = ev.state.numel() * 8
    host_in = torch.empty(ev.state.numel(), dtype=torch.float64, pin_memory=True)
    host_in.copy_(ev.state)
    host_out = torch.empty_like(host_in, pin_memory=True)
    host_out2 = torch.empty_like(host_in, pin_memory=True)
    dev = torch.empty_like(ev.state)
    E2E_STATES, E2E_BUFS = 8, 3
    devs = [dev] + [torch.empty_like(ev.state) for _ in range(E2E_BUFS - 1)]
    ins = [host_in] * E2E_STATES
    outs = [host_out if k % 2 == 0 else host_out2 for k in range(E2E_STATES)]
    C.check(C.cosmos_evolve_host_many(g, p, ins[:2], outs[:2], devs, 1, 0.0, dt, ev.ws_rk4, stream))  # warm
    torch.cuda.synchronize()
    # the host link is shared with other tenants of the machine: three rounds,
    # the median reported (all three kept in the line)
    rounds = []
    for r in range(3):
        t0 = time.perf_counter()
        C.check(C.cosmos_evolve_host_many(g, p, ins, outs, devs, 1, 0.0, dt, ev.ws_rk4, stream))
        rounds.append(nranks * pts * E2E_STATES / max_over_ranks(time.perf_counter() - t0))
    e2e_steps = max(1, min(args.steps, 5))
    C.check(C.cosmos_evolve_host(g, p, host_in, host_out, dev, 1, 0.0, dt, ev.ws_rk4, stream))  # warm
    torch.cuda.synchronize()
    serial = []
    for r in range(3):
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            C.check(C.cosmos_evolve_host(g, p, host_in, host_out, dev, 1, k * dt, dt, ev.ws_rk4, stream))
        serial.append(nranks * pts * e2e_steps / max_over_ranks(time.perf_counter() - t0))
    del devs
    # plain copy rates of the host link in this run (context for the rounds)
    link = {}
    for name, (dst, src) in (("h2d_GBps", (dev, host_in)), ("d2h_GBps", (host_out, dev))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        link[name] = nbytes / (time.perf_counter() - t0) / 1e9
    e2e = {"value": statistics.median(rounds), "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "rounds": rounds,
           "steps_per_round": E2E_STATES,
           "mode": (f"cosmos_evolve_host_many: {E2E_STATES} independent 256^3 states per round, one RK4 step each, "
                    f"copied in from and back to pinned host memory ({E2E_BUFS} device buffers; the copies of other "
                    "states overlap each state's step)"),
           "serial": {"value": statistics.median(serial), "rounds": serial, "steps_per_round": e2e_steps,
                      "mode": "cosmos_evolve_host: one state, copied in and out around every step"},
           "link": link}

    # ---- FP64 peak of this GPU (in-run DFMA probe) ----
    scratch = torch.empty(152 * 8 * 256, dtype=torch.float64, device=f"cuda:{local}")
    fp64_peak = max(C.cosmos_probe_fp64(scratch, stream) for _ in range(3))

    # ---- the rest of the metric, on one GPU only (at N > 1 every rank would hold its GPU) ----
    generic = batched = adjoint = None
    if ws_ == 1 and not args.no_extras:
        # the same sweep on a generic state: all 24 fields vary in x, y and z (the gauge wave
        # depends on x alone, so most of its derivatives are exactly zero)
        from paper_2606_02053_gb300 import inputs

        ev.set_state(inputs.smooth_state(n, seed=2562, kmax=6, scale=0.5))
        for w in range(3):
            stage_calls(w * dt)
        gk = 5
        gev = [[[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
                for _ in range(4)] for _ in range(gk)]
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for k in range(gk):
            stage_calls((3 + k) * dt, gev[k])
        g1.record(stream)
        torch.cuda.synchronize()
        tg = g0.elapsed_time(g1) * 1e-3
        gpass = [statistics.mean([gev[k][st][q][0].elapsed_time(gev[k][st][q][1]) for k in range(gk) for st in range(4)])
                 for q in range(2)]
        generic = {"value": pts * gk / tg, "unit": UNIT, "ms_per_step": 1e3 * tg / gk, "steps": gk, "warmup": 3,
                   "derivative_pass_ms": gpass[0], "algebra_pass_ms": gpass[1],
                   "state": "inputs.smooth_state(256, seed=2562, kmax=6, scale=0.5): every field a base value plus "
                            "3 seeded Fourier modes with wave numbers up to 6 per axis"}
        del ev, U1, U2, acc, dev, host_in, host_out
        torch.cuda.empty_cache()
        # batched threshold scan (64 instances, 64^3..96^3, fluid) against the per-instance loop;
        # 10 of the workload's 150 steps are timed, so that the whole line stays within minutes
        batched = measure_scan(64, 10, 3)
        batched["steps_note"] = "10 timed steps of the 150-step workload (plus 3 warm-up); same per-step work"
        # adjoint gradients of the collapse diagnostics, 96^3 x 256 steps, checkpoints every 16
        adjoint = measure_adjoint(96, 256, 16, point_checks=False)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # ---- CPU baseline (oracle) + algorithmic flop count ----
    cpu = None
    if not args.no_cpu_baseline:
        host_state = host_gauge_wave
        cpu = cpu_baseline_sample(n, planes=n // 2, repeats=1, state=host_state)
    # average launch duration per kernel (over the 4 stages and all steps)
    avg = {name: statistics.mean([x for st in pass_ms[q] for x in st]) * 1e-3
           for q, name in enumerate(["derivative", "algebra"])}
    stage_avg = [statistics.mean(pass_ms[0][s]) + statistics.mean(pass_ms[1][s]) for s in range(4)]
    roof, roof2, sweep = None, None, None
    if cpu is not None:
        parts = cpu["flops_parts"]
        fl = lambda d: d["add"] + d["mul"] + d["div"] + d["sqrt"]  # noqa: E731
        combine = statistics.mean(COMBINE_FLOPS) * STATE_FIELDS
        # algebra pass: the generated algebra's operations + the KO multiply-add (2 per field) + the RK4
        # combine; the oracle's count (its plain loops form every symmetric component twice) beside it
        alg_flops = generated_algebra_ops("vac") + 2 * STATE_FIELDS + combine
        oracle_flops = {"derivative": fl(parts["derivatives"]) + fl(parts["ko"]),
                        "algebra": fl(parts["algebra"]) + combine}
        bytes_point = {"derivative": 8 * (STATE_FIELDS + DERIV_DOUBLES),
                       "algebra": 8 * (DERIV_DOUBLES + statistics.mean([b / 8 for b in BYTES_PER_POINT_STAGE]))}
        peak = fp64_peak / 1e12
        hbm_peak, hbm_src = hbm_peak_gbs()
        traffic_ok = kernel_sources_hash() == NCU_TRAFFIC["sources_sha256_16"]

        def traffic(name):
            return NCU_TRAFFIC["bytes_per_launch"][name] * (n / NCU_TRAFFIC["grid"]) ** 3 if traffic_ok else None

        def roof_algebra():
            achieved = pts * alg_flops / avg["algebra"] / 1e12
            return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": traffic("algebra"),
                    "traffic_note": "bytes per launch, ncu small-case capture scaled by points",
                    "kernel": "algebra pass (stage_kernel<T_vac>)", "avg_launch_ms": 1e3 * avg["algebra"],
                    "algorithmic_flops_per_point": alg_flops,
                    "flops_note": "generated algebra after CSE + KO multiply-add + RK4 combine",
                    "oracle_flops_per_point": oracle_flops["algebra"],
                    "algorithmic_bytes_per_point": bytes_point["algebra"],
                    "hbm_GBps_algorithmic": pts * bytes_point["algebra"] / avg["algebra"] / 1e9,
                    "peak_source": "FP64 DFMA throughput measured in this run (cosmos_probe_fp64); nominal 1.25"}

        def roof_derivative():
            achieved = pts * bytes_point["derivative"] / avg["derivative"] / 1e9
            return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": traffic("derivative"),
                    "traffic_note": "bytes per launch (exponent scan + limb conversion + integer pass), ncu small-case "
                                    "capture scaled by points",
                    "kernel": "derivative pass (limb pre-pass + ideriv_kernel<T_vac>)",
                    "avg_launch_ms": 1e3 * avg["derivative"],
                    "algorithmic_bytes_per_point": bytes_point["derivative"],
                    "stencil_flops_per_point_fp64_equivalent": oracle_flops["derivative"],
                    "stencil_TFLOPs_fp64_equivalent": pts * oracle_flops["derivative"] / avg["derivative"] / 1e12,
                    "arithmetic": "exact integer (fixed-point digits), not the FP64 pipe",
                    "peak_source": "HBM copy bandwidth " + hbm_src}

        rf = {"derivative": roof_derivative, "algebra": roof_algebra}
        dom = max(avg, key=avg.get)
        other = "algebra" if dom == "derivative" else "derivative"
        roof, roof2 = rf[dom](), rf[other]()
        # the whole step against the sum of its passes' own roofline times: the algebra pass's
        # generated FP64 operations at the FP64 peak, the derivative pass's bytes at the HBM peak
        # (its stencils run in integer units, so no FP64 bound applies to it)
        t_alg = 4 * pts * alg_flops / (peak * 1e12)
        t_der = 4 * pts * bytes_point["derivative"] / (hbm_peak * 1e9)
        t_fp64_equiv = 4 * pts * (alg_flops + oracle_flops["derivative"]) / (peak * 1e12)
        sweep = {"roofline_ms_per_step": 1e3 * (t_alg + t_der), "algebra_fp64_ms_per_step": 1e3 * t_alg,
                 "derivative_hbm_ms_per_step": 1e3 * t_der, "ms_per_step": 1e3 * elapsed / args.steps,
                 "frac": (t_alg + t_der) / (elapsed / args.steps),
                 "note": "sum of the two passes' roofline times / measured RK4 step (4 stages)",
                 "context_fp64_equivalent_ms_per_step": 1e3 * t_fp64_equiv,
                 "context_note": "FP64 time of the algebra plus the stencils counted as the FP64 flops they stand "
                                 "for (integer units do them): not a bound on the executed work"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": n, "fields": STATE_FIELDS, "dt_over_h": 0.25,
                       "parallelism": f"replicas{nranks}" if nranks > 1 else "single",
                       "l2": "inputs larger than L2 (3.2 GB state per level)"},
            "stage_ms": stage_avg, "roofline": roof, "roofline_other_kernel": roof2, "roofline_sweep": sweep,
            "gpu_launches": gpu_launches,
            "sweep_generic": generic, "batched": batched, "adjoint": adjoint,
            "e2e": e2e, "clocks": clk,
            "cpu_baseline": None if cpu is None else {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"],
                                                      "kind": "oracle", "sample": cpu["sample"],
                                                      "value_1_core": cpu["value_1_core"]}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
