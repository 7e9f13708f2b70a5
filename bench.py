"""Benchmark: grid-point stage updates per second (PSU/s) of the multilevel
stencil step (ghost reconstruction + advection RHS + RK3-TVD stage) and the
HBM-roofline fraction of its dominant kernel, on one GB300.

Default workload ("large single grid"): one periodic tree, 24^3 blocks at
levels 3-8 refined in nested balls around a seeded Gaussian blob (~40k
leaves, ~0.55 G points), 6.2 lifted wavelet, FP32 storage and arithmetic,
WENO-Z5 flux, RK3, constant velocity (1, 0.5, 0.25), fixed tree.  Inputs are
larger than L2 (no flush needed).  One step = 3 stages over every point.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32|f64]
                  [--scheme wenoz5|cons5|cons3] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the plain reference
implementation of the same path) on the host cores, on a bounded sample of
the same workload, and prints the same metric.
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

from paper_2112_07537_gb300 import inputs as I  # noqa: E402

METRIC = "point-stage updates/s (ghost fill + RHS + RK3 stage)"
UNIT = "PSU/s"
# nested refinement balls around the blob centre, level 3 -> 3 + len(radii)
WORKLOADS = {"large": (0.35, 0.25, 0.17, 0.11, 0.06),   # 42 400 leaves, 586 M points
             "medium": (0.35, 0.25, 0.17),              # 11 768 leaves, 163 M points
             "small": (0.3, 0.2)}
U = (1.0, 0.5, 0.25)


def workload_tree(name="large"):
    return I.tree_sphere((1, 1, 1), 1.0, 3, WORKLOADS[name], centre=(0.5, 0.5, 0.5))


def clocks_sampler(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]]
    while not stop.is_set():
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=5)
            if r.returncode == 0 and r.stdout.strip():
                out.append([t.strip() for t in r.stdout.strip().splitlines()[0].split(",")])
        except Exception:
            pass
        stop.wait(0.2)


def summarize_clocks(samples):
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    sm = [float(s[0]) for s in samples if s[0].replace(".", "").isdigit()]
    mx = [float(s[1]) for s in samples if s[1].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for s in samples for i in range(4) if "Active" in s[3 + i]
                      and not s[3 + i].startswith("Not")})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(samples)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(budget_s=15.0):
    """The FP64 oracle (single-threaded C) on a bounded sample of the workload:
    the 2x2x2-tree two-level grid (15 leaves of 16^3) with the workload's
    scheme, as many RK3 steps as fit the time budget."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    nt, tl, nb = (2, 2, 2), 0.5, 16
    lev, anc = I.tree_config1()
    og = O.Grid(nt, tl, nb, 6, 2, 0, 1, lev, anc)
    phi = I.gaussian(I.point_coords(nt, tl, nb, lev, anc), (0.5, 0.5, 0.5), 0.1)
    dt = O.dt_cfl(og, 0.5, U)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s or steps == 0:
        phi = O.rk3_step(og, phi, dt, O.WENOZ5, U)
        steps += 1
    el = time.perf_counter() - t0
    pts = og.nleaf * nb ** 3
    return {"value": pts * 3 * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} RK3 steps (WENO-Z5, 6.2 ghosts) of the 15-leaf 16^3 two-level "
                      f"grid, {pts} points, {el:.1f} s, single thread"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    base = cpu_baseline(budget_s=max(2.0, 60.0 / max(1, args.steps + args.warmup)))
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "FP64 CPU oracle on a bounded sample (see cpu_baseline)"},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--scheme", default="wenoz5", choices=["wenoz5", "cons5", "cons3"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2112_07537_gb300 import build, mrgb
    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    W = max(3, args.warmup)
    prec = mrgb.F32 if args.precision == "f32" else mrgb.F64
    scheme = {"wenoz5": mrgb.WENOZ5, "cons5": mrgb.CONS5, "cons3": mrgb.CONS3}[args.scheme]
    lev, anc = workload_tree(args.workload)
    radii = WORKLOADS[args.workload]
    nb = 24
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = mrgb.Grid((1, 1, 1), 1.0, nb, 3, int(lev.max()), 6, 2, lev, anc, precision=prec,
                      nfields=1, stream=stream, fixed_tree=True)
        g.field_set(0, mrgb.INIT_GAUSSIAN, [0.5, 0.5, 0.5, 0.08, 1.0])
    n = g.nleaf
    pts = n * nb ** 3
    hmin = 1.0 / (nb * 2 ** int(lev.max()))
    dt = 0.5 * hmin / sum(abs(u) for u in U)

    for _ in range(W):
        g.step(0, dt, U, scheme)
    stream.synchronize()

    samples, stop = [], threading.Event()
    th = threading.Thread(target=clocks_sampler, args=(stop, samples), daemon=True)
    th.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = g.launch_count()
    g.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.step(0, dt, U, scheme)
    e1.record(stream)
    e1.synchronize()
    g.profile(False)
    ms = e0.elapsed_time(e1)
    launches = g.launch_count() - l0
    torch.cuda.synchronize()
    stop.set()
    th.join(timeout=2)
    prof = g.profile_read()
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the public API with host buffers
    es = 4 if prec == mrgb.F32 else 8
    host = torch.empty((n, nb, nb, nb), dtype=g.dtype, pin_memory=True)
    g.field_copy_out(0, host.numpy())
    ke = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        g.field_copy_in(0, host.numpy())
        g.step(0, dt, U, scheme)
        g.field_copy_out(0, host.numpy())
    e2e_s = time.perf_counter() - t0

    psu = world * pts * 3 * args.steps / (ms / 1e3)
    hbm, src = peaks()
    # dominant kernel of the step
    name, (tot, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    bpp = {"f32": 4, "f64": 8}[args.precision]
    alg_bytes = {"rhs_stage": pts * bpp * 32.0 / 3 / 4,  # 8 B stage 1, 12 B stages 2-3 (FP32)
                 "ghost_part1": pts * bpp * 2.0, "ghost_part2": 0.0, "ghost_merge": 0.0}
    per_launch = alg_bytes.get(name, pts * bpp * 2.0)
    achieved = per_launch / (tot / cnt / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": psu, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": W, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"{args.workload} single grid, fixed tree: 1 tree, 24^3 blocks, "
                               f"levels 3-{int(lev.max())} (nested balls r={radii}), {n} leaves, "
                               f"{pts} points; 6.2 lifted "
                               f"wavelet ghosts; {args.scheme} + RK3; u={U}; CFL 0.5",
                   "leaves": n, "points": pts, "l2": "inputs larger than L2 (no flush)",
                   "scheme": args.scheme, "precision": args.precision},
        "roofline": {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "peak_source": src,
                     "traffic": None,
                     "alg_bytes_per_launch": per_launch},
        "kernels": {k: {"ms_total": v[0], "launches": v[1], "share": v[0] / sum(x[0] for x in prof.values())}
                    for k, v in prof.items()},
        "gpu_launches": launches,
        "e2e": {"value": pts * 3 * ke / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": pts * es, "d2h_bytes_per_step": pts * es},
        "clocks": summarize_clocks(samples),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
