"""Benchmark: grid-point stage updates per second (PSU/s) of the multilevel
stencil step (ghost reconstruction + advection RHS + RK3-TVD stage, with grid
adaptation) and the HBM-roofline fraction of its dominant kernel, on one GB300,
for the FP32 form and, on the same workload and GPU, the plain FP64 form.

Default workload ("large single grid"): one periodic tree of 24^3 blocks,
levels 3-8; FP32 scalar (sum of seeded sharp Gaussians) advected by three
FP32 velocity fields (seeded divergence-free Taylor-Green-like field);
6.2 lifted wavelet, eps_refine = 1e-5, eps_coarsen = 1e-7; WENO-Z5 + RK3,
CFL 0.5; adaptation every 2 steps inside the timed region.  The initial grid
is built by alternating analytic sampling and refinement from a uniform
level-3 grid, then one full adaptation (all untimed).  Fields are far larger
than L2 (no flush needed).  The same workload then runs in FP64 (per-block
padded ghosts, FP64 stencil) for the FP32-over-FP64 speed-up.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32|f64]
                  [--scheme wenoz5|cons5|cons3] [--workload large|fixed-*]
                  [--impl ours|reference] [--no-fp64] [--no-cpu-baseline]

fixed-large / fixed-medium / fixed-small: the stencil step alone (no
adaptation, constant velocity) on fixed nested-ball trees, used for kernel
profiling.  --impl reference times the FP64 CPU oracle (the plain restatement
of the same path) on the host cores on a bounded sample and prints the same
metric.
"""
from __future__ import annotations

import argparse
import json
import math
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
WORKLOADS = {"fixed-large": (0.35, 0.25, 0.17, 0.11, 0.06),   # 42 400 leaves, 586 M points
             "fixed-medium": (0.35, 0.25, 0.17),              # 11 768 leaves, 163 M points
             "fixed-small": (0.3, 0.2)}                       # 3 424 leaves, 47 M points
# large single grid scalar: ~535 leaves per Gaussian, so 75 give the ~40 000
# leaves (~550 M points) of the large configuration
GAUSS = dict(seed=5, n=75, smin=0.0015, smax=0.006)
# the same adaptive path on a small grid (for profiler captures of a few GB)
GAUSS_SMALL = dict(seed=5, n=3, smin=0.0015, smax=0.006)
EPS_R, EPS_C, CFL, ADAPT_EVERY = 1e-5, 1e-7, 0.5, 2
U = (1.0, 0.5, 0.25)


def workload_tree(name="fixed-large"):
    return I.tree_sphere((1, 1, 1), 1.0, 3, WORKLOADS[name], centre=(0.5, 0.5, 0.5))


def gauss_params(seed, n, smin, smax):
    """n seeded Gaussians: centres U[0.15, 0.85]^3, sigma U[smin, smax], amp 1,
    as MR_INIT_GAUSSIAN_SUM parameter lists of at most 51 Gaussians each."""
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        c = rng.uniform(0.15, 0.85, 3)
        rows.append([*c, rng.uniform(smin, smax), 1.0])
    return [[len(ch)] + [x for r in ch for x in r] for ch in (rows[i:i + 51] for i in range(0, n, 51))]


def set_gaussians(mrgb, g, fid, chunks):
    """The field = the sum of the Gaussians of every chunk."""
    for k, p in enumerate(chunks):
        g.field_set(fid, mrgb.INIT_GAUSSIAN_SUM if k == 0 else mrgb.INIT_GAUSSIAN_SUM_ADD, p)


TG = (1.0, 0.3)  # Taylor-Green scale and phase (seeded constants of the velocity field)


def init_large(mrgb, stream, prec, cap, gauss=GAUSS):
    """Initial adapted grid (untimed): uniform level 3, then alternate analytic
    sampling and refinement until no block refines, sample again, and run
    one full adaptation."""
    lev, anc = I.uniform_leaves((1, 1, 1), 3)
    g = mrgb.Grid((1, 1, 1), 1.0, 24, 3, 8, 6, 2, lev, anc, precision=prec, nfields=4,
                  capacity=cap, stream=stream, velocity=True)
    p = gauss_params(**gauss)
    for _ in range(12):
        set_gaussians(mrgb, g, 0, p)
        if g.adapt_iter(0, EPS_R, EPS_C, flags=mrgb.ADAPT_REFINE) == 0:
            break
    set_gaussians(mrgb, g, 0, p)
    for d in range(3):
        g.field_set(1 + d, mrgb.INIT_TAYLOR_GREEN, [d, TG[0], TG[1]])
    g.adapt(0, EPS_R, EPS_C)
    return g


# deformation of a compact Gaussian blob (Sec. 5.3): sigma 0.1, beta 2 sigma at
# (0.35, 0.35, 0.35); eps_r 1e-2, eps_r/eps_c 100; CFL 0.5 on the finest
# spacing present; adaptation every 12 steps; velocity times cos(pi t / 3)
DEFORM = dict(eps_r=1e-2, ratio=100.0, cfl=0.5, adapt_every=12, umax=4.0)
COMPACT = [0.35, 0.35, 0.35, 0.1, 0.2, 1.0]


def init_deformation(mrgb, stream, prec, cap, wav):
    """Initial grid of the deformation test: uniform level 2, then alternate
    analytic sampling and refinement until no block refines, sample again,
    set the velocity fields and run one full adaptation."""
    lev, anc = I.uniform_leaves((1, 1, 1), 2)
    g = mrgb.Grid((1, 1, 1), 1.0, 24, 2, 8, wav[0], wav[1], lev, anc, precision=prec, nfields=4,
                  capacity=cap, stream=stream, velocity=True)
    er = DEFORM["eps_r"]
    for _ in range(12):
        g.field_set(0, mrgb.INIT_COMPACT_GAUSSIAN, COMPACT)
        if g.adapt_iter(0, er, er / DEFORM["ratio"], flags=mrgb.ADAPT_REFINE) == 0:
            break
    g.field_set(0, mrgb.INIT_COMPACT_GAUSSIAN, COMPACT)
    for d in range(3):
        g.field_set(1 + d, mrgb.INIT_DEFORMATION, [d, 1.0])
    g.adapt(0, er, er / DEFORM["ratio"])
    return g


# batched uneven instances: 64 independent periodic grids (trees of a 4x4x4
# forest in independent-tree mode), blocks of 16^3, levels 1-5, 1-3 seeded
# Gaussians each (sigma U[0.05, 0.2], centres U[0, 1]^3), a constant velocity
# of unit norm per grid (held in the three velocity fields), 4.2 lifted
# wavelet, FP32, one eps for all grids (their block counts differ through
# their fields)
BATCH = dict(ngrid=64, nt=(4, 4, 4), nb=16, lmin=1, lmax=5, seed=11, eps_r=1e-3, eps_c=1e-5)


def batch_specs():
    rng = np.random.default_rng(BATCH["seed"])
    specs = []
    for _ in range(BATCH["ngrid"]):
        nblob = int(rng.integers(1, 4))
        blobs = [(rng.uniform(0, 1, 3), rng.uniform(0.05, 0.2)) for _ in range(nblob)]
        u = rng.normal(size=3)
        specs.append((blobs, u / np.linalg.norm(u)))
    return specs


def batch_fields(g, specs):
    """Host-evaluated fields of every tree in its own coordinates (scalar:
    sum of the tree's Gaussians, nearest periodic image; velocity: the
    tree's constant)."""
    lev, anc, _ = g.leaves()
    nt, nb = BATCH["nt"], BATCH["nb"]
    tree = (anc[:, 0] >> lev) + nt[0] * ((anc[:, 1] >> lev) + nt[1] * (anc[:, 2] >> lev))
    loc = anc - np.stack([tree % nt[0], (tree // nt[0]) % nt[1], tree // (nt[0] * nt[1])], 1) * \
        (1 << lev)[:, None]
    xyz = I.point_coords((1, 1, 1), 1.0, nb, lev, loc)
    phi = np.zeros((len(lev), nb, nb, nb), np.float32)
    vel = [np.zeros_like(phi) for _ in range(3)]
    for k, (blobs, u) in enumerate(specs):
        sel = np.nonzero(tree == k)[0]
        if not len(sel):
            continue
        sub = [a[sel] for a in xyz]
        acc = np.zeros((len(sel), nb, nb, nb))
        for c, sg in blobs:
            acc += I.gaussian(sub, tuple(c), sg)
        phi[sel] = acc
        for d in range(3):
            vel[d][sel] = u[d]
    return phi, vel


def init_batched(mrgb, stream, prec, cap):
    """Initial grids of the batch (untimed): uniform at lmin, alternate
    sampling and refinement until no block refines, sample, one full
    adaptation."""
    nt = BATCH["nt"]
    lev, anc = I.uniform_leaves(nt, BATCH["lmin"])
    g = mrgb.Grid(nt, 1.0, BATCH["nb"], BATCH["lmin"], BATCH["lmax"], 4, 2, lev, anc, precision=prec,
                  nfields=4, capacity=cap, stream=stream, velocity=True, independent_trees=True)
    specs = batch_specs()
    for _ in range(12):
        phi, _ = batch_fields(g, specs)
        g.field_copy_in(0, phi)
        if g.adapt_iter(0, BATCH["eps_r"], BATCH["eps_c"], flags=mrgb.ADAPT_REFINE) == 0:
            break
    phi, vel = batch_fields(g, specs)
    g.field_copy_in(0, phi)
    for d in range(3):
        g.field_copy_in(1 + d, vel[d])
    g.adapt(0, BATCH["eps_r"], BATCH["eps_c"])
    return g


def split_batch(mrgb, stream, g):
    """The grids of a batch as separate one-tree grids (same leaves, same
    field values), for the sequential comparison."""
    lev, anc, _ = g.leaves()
    nt, nb = BATCH["nt"], BATCH["nb"]
    tree = (anc[:, 0] >> lev) + nt[0] * ((anc[:, 1] >> lev) + nt[1] * (anc[:, 2] >> lev))
    loc = anc - np.stack([tree % nt[0], (tree // nt[0]) % nt[1], tree // (nt[0] * nt[1])], 1) * \
        (1 << lev)[:, None]
    vals = [g.field_copy_out(f) for f in range(4)]
    out = []
    for k in range(BATCH["ngrid"]):
        sel = np.nonzero(tree == k)[0]
        s = mrgb.Grid((1, 1, 1), 1.0, nb, BATCH["lmin"], BATCH["lmax"], 4, 2, lev[sel], loc[sel],
                      precision=g.precision, nfields=4, capacity=max(64, 4 * len(sel)), stream=stream,
                      velocity=True)
        sl, sa, _ = s.leaves()
        pos = {(int(l), tuple(int(x) for x in a)): i for i, (l, a) in enumerate(zip(lev[sel], loc[sel]))}
        order = np.array([sel[pos[(int(l), tuple(int(x) for x in a))]] for l, a in zip(sl, sa)])
        for f in range(4):
            s.field_copy_in(f, np.ascontiguousarray(vals[f][order]))
        out.append(s)
    return out


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


def _oracle_sample(steps=2):
    """One bounded sample of the large workload on the FP64 oracle: a periodic
    tree of 22 blocks of 24^3 on levels 1-2, the scalar (two Gaussians) and
    the three Taylor-Green-like velocity components, 6.2 lifted wavelet;
    `steps` RK3 steps of WENO-Z5 with the per-tree velocity ghosts (as the
    device path), then one adaptation iteration of all four fields.  Returns
    (point-stage updates, seconds)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    nt, tl, nb = (1, 1, 1), 1.0, 24
    lev, anc = I.uniform_leaves(nt, 1)
    lev, anc = I.refine_leaves(lev, anc, np.isin(np.arange(len(lev)), [0, 1]))
    og = O.Grid(nt, tl, nb, 6, 2, 0, 4, lev, anc)
    xyz = I.point_coords(nt, tl, nb, og.lev, og.anc)
    phi = I.gaussian(xyz, (0.75, 0.25, 0.25), 0.06) + I.gaussian(xyz, (0.75, 0.75, 0.75), 0.025)
    w = 2 * np.pi
    vel = [TG[0] * np.sin(w * xyz[0] + TG[1]) * np.cos(w * xyz[1]) * np.cos(w * xyz[2]),
           -TG[0] * np.cos(w * xyz[0] + TG[1]) * np.sin(w * xyz[1]) * np.cos(w * xyz[2]),
           np.zeros_like(xyz[0])]
    dt = CFL * (tl / (nb * 4)) / (2 * TG[0])
    t0 = time.perf_counter()
    vpads = [O.ghost_fill(og, O.ghost_fill(og, v, 3)[1], 3)[0] for v in vel]
    for _ in range(steps):
        phi = O.rk3_step_velpad(og, phi, vpads, dt, O.WENOZ5)
    O.adapt_iter_fields(og, [phi] + vel, 1e-3, 1e-5)
    return 3 * steps * og.nleaf * nb ** 3, time.perf_counter() - t0


def _oracle_worker(_):
    return _oracle_sample()


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(all_cores=True):
    """The FP64 oracle as it stands (plain C, one thread per process) on a
    bounded sample of the workload (_oracle_sample), once on one core and,
    with all_cores, as one spawned process per host core running the same
    sample concurrently (value = all processes' updates / wall time)."""
    psu, sec = _oracle_sample()
    ncpu = os.cpu_count() or 1
    out = {"value": psu / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
           "cpu": _cpu_model(), "nproc": ncpu, "single_thread": psu / sec,
           "sample": f"2 RK3 steps (WENO-Z5, 6.2 ghosts, 3 velocity fields with per-tree ghosts) + one "
                     f"4-field adaptation iteration of a 22-leaf 24^3 tree ({psu // 6} points), "
                     f"{sec:.1f} s on one core"}
    if all_cores and ncpu > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(ncpu) as pool:
            res = pool.map(_oracle_worker, range(ncpu))
        wall = time.perf_counter() - t0
        out.update(value=sum(r[0] for r in res) / wall, cores=ncpu, all_core_wall_s=wall,
                   sample=out["sample"] + f"; all cores: {ncpu} spawned processes each running the sample, "
                                          f"{wall:.1f} s wall")
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    base = cpu_baseline(all_cores=True)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "FP64 CPU oracle on a bounded sample of the large single-grid "
                                   "workload (see cpu_baseline.sample)"},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def make_grid(args, mrgb, stream, prec, cap):
    """The workload's grid (untimed set-up): returns (grid, lmax, umax)."""
    nb = 24
    with __import__("torch").cuda.stream(stream):
        if args.workload == "deformation":
            wav = tuple(int(c) for c in args.wavelet.split("."))
            return init_deformation(mrgb, stream, prec, min(cap, 30000), wav), 8, DEFORM["umax"]
        if args.workload in ("large", "adaptive-small"):
            g = init_large(mrgb, stream, prec, cap, GAUSS if args.workload == "large" else GAUSS_SMALL)
            return g, 8, 2.0 * TG[0]  # |u| + |v| <= 2 s for the Taylor-Green-like field
        if args.workload == "batched":
            # one dt for the batch: sum_d |u_d| <= sqrt(3) for unit velocities
            return init_batched(mrgb, stream, prec, min(cap, 60000)), BATCH["lmax"], 3 ** 0.5
        lev, anc = workload_tree(args.workload)
        lmax = int(lev.max())
        g = mrgb.Grid((1, 1, 1), 1.0, nb, 3, lmax, 6, 2, lev, anc, precision=prec,
                      nfields=1, stream=stream, fixed_tree=True)
        g.field_set(0, mrgb.INIT_GAUSSIAN, [0.5, 0.5, 0.5, 0.08, 1.0])
        return g, lmax, sum(abs(u) for u in U)


class Stepper:
    """One benchmark step of the workload (RK3 step, adaptation every
    ADAPT_EVERY steps on the adaptive workloads)."""

    def __init__(self, args, mrgb, g, lmax, umax):
        self.args, self.mrgb, self.g = args, mrgb, g
        self.scheme = {"wenoz5": mrgb.WENOZ5, "cons5": mrgb.CONS5, "cons3": mrgb.CONS3}[args.scheme]
        self.adaptive = args.workload in ("large", "adaptive-small", "batched")
        self.eps = (BATCH["eps_r"], BATCH["eps_c"]) if args.workload == "batched" else (EPS_R, EPS_C)
        self.deform = args.workload == "deformation"
        self.nb = BATCH["nb"] if args.workload == "batched" else 24
        self.umax = umax
        self.dt = CFL * (1.0 / (self.nb * 2 ** lmax)) / umax
        if args.diffusion:
            g.set_diffusion(args.nu, args.diffusion)
            hmin = 1.0 / (self.nb * 2 ** lmax)
            self.dt = min(self.dt, 0.1 * hmin * hmin / args.nu)  # explicit diffusion limit
        self.state = {"t": 0.0, "n": 0, "lm": g.query().max_level, "i": 0}

    def __call__(self):
        """One step; returns the point-stage updates it performed."""
        g, mrgb, st = self.g, self.mrgb, self.state
        pts = g.nleaf * self.nb ** 3
        i = st["i"]
        st["i"] += 1
        if self.deform:
            # dt from the finest spacing present (reading of Sec. 5.3)
            t = st["t"]
            dtd = DEFORM["cfl"] * (1.0 / (self.nb * 2 ** st["lm"])) / self.umax
            sc = [math.cos(math.pi * tt / 3) for tt in (t, t + dtd, t + dtd / 2)]
            g.step_vel_scaled(0, dtd, (1, 2, 3), self.scheme, sc)
            st["t"] = t + dtd
            st["n"] += 1
            if st["n"] % DEFORM["adapt_every"] == 0:
                g.adapt(0, DEFORM["eps_r"], DEFORM["eps_r"] / DEFORM["ratio"])
                st["lm"] = g.query().max_level
        elif self.adaptive:
            g.step_vel(0, self.dt, (1, 2, 3), self.scheme)
            if (i + 1) % ADAPT_EVERY == 0:
                g.adapt(0, *self.eps)
        else:
            g.step(0, self.dt, U, self.scheme)
        return 3 * pts


def max_over_ranks(ms, dist, device="cuda"):
    """The job's time: the largest of the ranks' timed regions (every rank
    receives it).  Without a process group, the rank's own time."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms):
    """Whole-job throughput: every rank processes units_per_rank units (weak
    scaling, independent replicas), the job takes ms."""
    return world * units_per_rank / (ms / 1e3)


def timed(args, g, step, stream, W, dist):
    """W warm-up steps, then args.steps timed steps between CUDA events on the
    grid's stream, with clocks sampled during the timed region."""
    import torch
    for _ in range(W):
        step()
    stream.synchronize()
    samples, stop = [], threading.Event()
    th = threading.Thread(target=clocks_sampler, args=(stop, samples), daemon=True)
    th.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stats0 = g.query()
    l0 = g.launch_count()
    cudart = torch.cuda.cudart()
    cudart.cudaProfilerStart()  # an attached profiler captures the timed steps only
    g.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    psu = 0
    e0.record(stream)
    for _ in range(args.steps):
        psu += step()
    e1.record(stream)
    e1.synchronize()
    g.profile(False)
    cudart.cudaProfilerStop()
    ms = e0.elapsed_time(e1)
    launches = g.launch_count() - l0
    torch.cuda.synchronize()
    stop.set()
    th.join(timeout=2)
    prof = g.profile_read()
    # algorithmic bytes of the ghost reconstruction: the pre-pass (id 0) and
    # the plain gather (id 1) share one fill, so they are timed together
    ghost_bytes = g.profile_bytes(0) + g.profile_bytes(1)
    ms = max_over_ranks(ms, dist)
    return dict(ms=ms, psu=psu, launches=launches, prof=prof, ghost_bytes=ghost_bytes, stats0=stats0,
                stats1=g.query(), clocks=summarize_clocks(samples))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--scheme", default="wenoz5", choices=["wenoz5", "cons5", "cons3"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain form of the workload")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (no autotuner)")
    ap.add_argument("--stage-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="FP32 stage kernel: 0 tuned, 1 k_fused, 2 k_march")
    ap.add_argument("--workload", default="large",
                    choices=["large", "adaptive-small", "deformation", "batched"] + sorted(WORKLOADS))
    ap.add_argument("--wavelet", default="4.2", choices=["2.2", "4.2", "6.2", "4.0", "6.0"],
                    help="wavelet of the deformation workload")
    ap.add_argument("--capacity", type=int, default=60000)
    ap.add_argument("--diffusion", type=int, default=0, choices=[0, 2, 4],
                    help="add nu * DIFF-2/DIFF-4 Laplacian to the stencil step")
    ap.add_argument("--nu", type=float, default=1e-4)
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
    batched = args.workload == "batched"
    nb = BATCH["nb"] if batched else 24
    adaptive = args.workload in ("large", "adaptive-small", "batched")
    deform = args.workload == "deformation"
    stream = torch.cuda.Stream()
    g, lmax, umax = make_grid(args, mrgb, stream, prec, args.capacity)
    if not args.no_autotune:
        g.autotune(True)  # launch shapes tuned on this grid during the warm-up steps
    if args.stage_kernel:
        g.set_stage_kernel(args.stage_kernel)  # FP32 stage kernel forced (profiling)
    step = Stepper(args, mrgb, g, lmax, umax)
    r = timed(args, g, step, stream, W, dist)
    ms, psu_count, prof, stats0, stats1 = r["ms"], r["psu"], r["prof"], r["stats0"], r["stats1"]

    # end to end through the public API with host buffers: each step copies
    # the scalar in from pinned host memory and reads it back
    es = 4 if prec == mrgb.F32 else 8
    e2e = None
    if not args.no_e2e:
        cap = min(args.capacity, 30000) if deform else args.capacity if adaptive else g.nleaf
        host = torch.empty(cap * nb ** 3, dtype=g.dtype, pin_memory=True)
        ke = max(2, min(args.steps, 4))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_psu, h2d, d2h = 0, 0, 0
        for i in range(ke):
            n = g.nleaf * nb ** 3
            g.field_copy_out(0, host[:n].numpy())  # establishes the host copy
            g.field_copy_in(0, host[:n].numpy())
            h2d += n * es
            e2e_psu += step()
            n = g.nleaf * nb ** 3
            g.field_copy_out(0, host[:n].numpy())
            d2h += n * es
        e2e_s = time.perf_counter() - t0
        e2e = {"value": e2e_psu / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d // ke,
               "d2h_bytes_per_step": d2h // ke}
        del host

    # RK steps alone (no adaptation), stream-ordered and replayed as one CUDA
    # graph per step, on the same grid and velocity
    graph_cmp = None
    if adaptive or deform:
        import torch as _t
        ev = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
        res = {}
        for mode in (0, 1):
            g.use_graphs(bool(mode))
            g.step_vel(0, step.dt, (1, 2, 3), step.scheme)  # capture (graph mode) / warm
            ev[0].record(stream)
            for _ in range(4):
                g.step_vel(0, step.dt, (1, 2, 3), step.scheme)
            ev[1].record(stream)
            ev[1].synchronize()
            res[mode] = ev[0].elapsed_time(ev[1]) / 4
        graph_cmp = {"ms_per_rk_step_stream": res[0], "ms_per_rk_step_graph": res[1],
                     "graph_replays": g.graph_replays(), "leaves": g.nleaf}
        g.use_graphs(False)

    psu = whole_job_rate(world, psu_count, ms)
    hbm, src = peaks()
    try:
        cpk = mrgb.device_peaks()
    except Exception as ex:  # reported, not fatal
        cpk = {"error": str(ex)}
    rprof = dict(prof)
    if "ghost_part1" in rprof:
        t0_, n0_ = rprof.pop("ghost_part1")
        t1_, _ = rprof.pop("ghost_plain", (0.0, 0))
        rprof["ghost_fill"] = (t0_ + t1_, n0_)  # per pre-pass launch
    name, (tot, cnt) = max(rprof.items(), key=lambda kv: kv[1][0])
    bpp = 4 if prec == mrgb.F32 else 8
    mean_pts = psu_count / (3 * args.steps)
    vel_fields = adaptive or deform
    # algorithmic bytes per point-stage of the fused stage: phi read, RK
    # output written, u^n read in stages 1-2 (2/3 on average), plus the three
    # velocity components when the velocity is a field
    per_pt = bpp * (1 + 1 + 2.0 / 3 + (3 if vel_fields else 0))
    alg = {"rhs_stage": mean_pts * per_pt}
    if "ghost_fill" in rprof and r["ghost_bytes"] > 0:
        # requested-shell points written + source values read, per
        # reconstructed leaf, summed by the library over the launches (mean
        # per pre-pass launch)
        alg["ghost_fill"] = r["ghost_bytes"] / rprof["ghost_fill"][1]
    per_launch = alg.get(name, None)
    achieved = per_launch / (tot / cnt / 1e3) / 1e9 if per_launch else None
    gs = GAUSS if args.workload == "large" else GAUSS_SMALL
    if deform:
        workload = (f"deformation of a compact Gaussian blob (sigma 0.1, beta 0.2 at 0.35^3) by the "
                    f"incompressible deformation field times cos(pi t/3): 1 tree, 24^3 blocks, levels 2-8, "
                    f"{args.wavelet} wavelet, eps_r {DEFORM['eps_r']}, eps_c {DEFORM['eps_r'] / DEFORM['ratio']}, "
                    f"{args.scheme} + RK3, CFL {DEFORM['cfl']} on the finest spacing present, adapt every "
                    f"{DEFORM['adapt_every']} steps; {stats0.nleaf}->{stats1.nleaf} leaves, t = {step.state['t']:.4f}")
    elif batched:
        workload = (f"batched uneven instances: {BATCH['ngrid']} independent periodic grids (trees of a "
                    f"{BATCH['nt']} forest, each its own domain) advanced with one launch per phase, 16^3 blocks, "
                    f"levels {BATCH['lmin']}-{BATCH['lmax']}, {stats0.nleaf}->{stats1.nleaf} leaves in all, "
                    f"{mean_pts / 1e6:.1f} M points; per grid 1-3 seeded Gaussians (sigma U[0.05,0.2]) and a "
                    f"constant unit velocity (seed {BATCH['seed']}); 4.2 lifted wavelet, eps_r {BATCH['eps_r']}, "
                    f"eps_c {BATCH['eps_c']}; {args.scheme} + RK3, CFL {CFL}, one dt for the batch; adapt every "
                    f"{ADAPT_EVERY} steps")
    elif adaptive:
        workload = (f"{args.workload} single grid, adaptive: 1 tree, 24^3 blocks, levels "
                    f"{stats0.min_level}-{stats0.max_level} (lmin 3, lmax 8), {stats0.nleaf}->{stats1.nleaf} "
                    f"leaves, {mean_pts / 1e6:.0f} M points; scalar ({gs['n']} seeded Gaussians, seed "
                    f"{gs['seed']}, sigma {gs['smin']}-{gs['smax']}) + 3 velocity fields (Taylor-Green-like, "
                    f"scale {TG[0]}, phase {TG[1]}); 6.2 lifted wavelet, eps_r {EPS_R}, eps_c {EPS_C}; "
                    f"{args.scheme} + RK3, CFL {CFL}; adapt every {ADAPT_EVERY} steps")
    else:
        workload = (f"{args.workload} single grid, fixed tree, stencil step only: 1 tree, 24^3 blocks, "
                    f"levels 3-{lmax} (nested balls r={WORKLOADS[args.workload]}), {g.nleaf} leaves; "
                    f"6.2 lifted wavelet ghosts; {args.scheme} + RK3; u={U}; CFL {CFL}")
    shares = {k: v[0] / sum(x[0] for x in prof.values()) for k, v in prof.items()}
    # whole-step roofline: algorithmic bytes per point-stage of the stencil
    # step (survey measurement definition) times the achieved rate
    step_gbs = psu * per_pt / 1e9
    line = {
        "metric": METRIC, "value": psu, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": W, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": workload, "leaves": [stats0.nleaf, stats1.nleaf],
                   "mean_points": mean_pts, "l2": "fields larger than L2 (no flush)",
                   "scheme": args.scheme, "precision": args.precision,
                   "diffusion": f"DIFF-{args.diffusion}, nu={args.nu}" if args.diffusion else None},
        "roofline": {"bound": "hbm",
                     "kernel": "ghost_fill (k_prep + k_fill_plain)" if name == "ghost_fill" else name,
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm if achieved else None, "peak_source": src,
                     "traffic": None, "alg_bytes_per_launch": per_launch,
                     "alg_bytes_per_point_stage": per_pt if name == "rhs_stage" else None},
        "roofline_step": {"bound": "hbm", "alg_bytes_per_point_stage": per_pt, "achieved": step_gbs,
                          "peak": hbm, "unit": "GB/s", "frac": step_gbs / hbm},
        "kernels": {k: {"ms_total": v[0], "launches": v[1], "share": shares[k]} for k, v in prof.items()},
        "gpu_launches": r["launches"],
        "e2e": e2e,
        "clocks": r["clocks"],
        "compute_peaks": cpk,
        "rk_step_graph": graph_cmp,
        "autotune": mrgb.autotune_table(),
    }
    if "rhs_stage" in prof:
        t_rhs, n_rhs = prof["rhs_stage"]
        sec = t_rhs / n_rhs / 1e3
        a_rhs = mean_pts * per_pt / sec / 1e9
        line["roofline_stage_kernel"] = {"kernel": "rhs_stage", "achieved": a_rhs, "peak": hbm,
                                         "unit": "GB/s", "frac": a_rhs / hbm}
        # WENO-Z5: about 235 flops per point-stage (3 directions x ~75 + the
        # stage combination), CONS-5 about 45 (survey measurement table)
        fl = {"wenoz5": 235.0, "cons5": 45.0, "cons3": 30.0}[args.scheme]
        key = "fp32_fma_tflops" if prec == mrgb.F32 else "fp64_fma_tflops"
        if key in cpk:
            tf = mean_pts * fl / sec / 1e12
            line["roofline_stage_kernel"]["compute"] = {"flops_per_point_stage": fl, "achieved_tflops": tf,
                                                        "peak_tflops": cpk[key], "frac": tf / cpk[key]}
    if batched:
        # the same grids as separate one-tree grids, stepped one after another
        # (same steps, same adaptations): what batching saves
        per_grid = g.query().count_per_level
        singles = split_batch(mrgb, stream, g)
        del g
        steppers = [Stepper(args, mrgb, s_, BATCH["lmax"], 3 ** 0.5) for s_ in singles]
        for st_ in steppers:
            st_.dt = step.dt
        torch.cuda.synchronize()
        l_seq0 = sum(s_.launch_count() for s_ in singles)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        psu_seq = 0
        e0.record(stream)
        for _ in range(args.steps):
            for st_ in steppers:
                psu_seq += st_()
        e1.record(stream)
        e1.synchronize()
        ms_seq = e0.elapsed_time(e1)
        counts = sorted(s_.nleaf for s_ in singles)
        line["sequential"] = {"value": psu_seq / (ms_seq / 1e3), "unit": UNIT, "ms_per_step": ms_seq / args.steps,
                              "grids": len(singles), "leaves_per_grid": {"min": counts[0], "max": counts[-1],
                                                                         "median": counts[len(counts) // 2]},
                              "gpu_launches": sum(s_.launch_count() for s_ in singles) - l_seq0}
        line["batched_over_sequential"] = psu / line["sequential"]["value"]
        del per_grid
    if adaptive and not batched and prec == mrgb.F32 and not args.no_fp64:
        # the plain FP64 form on the same workload and GPU: free the FP32 grid
        del step, g
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        g64, lmax64, umax64 = make_grid(args, mrgb, stream, mrgb.F64, args.capacity)
        step64 = Stepper(args, mrgb, g64, lmax64, umax64)
        # the FP64 form is ~4x slower: at most 8 timed steps (an even count
        # keeps the one-adaptation-per-two-steps mix of the FP32 run)
        import copy
        a64 = copy.copy(args)
        a64.steps = max(2, min(args.steps, 8) // 2 * 2)
        r64 = timed(a64, g64, step64, stream, 3, None)
        v64 = whole_job_rate(world, r64["psu"], r64["ms"])
        line["fp64_plain"] = {"value": v64, "unit": UNIT, "ms_per_step": r64["ms"] / a64.steps,
                              "leaves": [r64["stats0"].nleaf, r64["stats1"].nleaf], "steps": a64.steps,
                              "warmup": 3,
                              "gpu_launches": r64["launches"], "clocks": r64["clocks"],
                              "tolerance": "FP64 path: 1e-12 of the field maximum vs the oracle",
                              "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in r64["prof"].items()}}
        line["fp32_over_fp64"] = psu / v64
        line["fp32_tolerance"] = ("FP32 path: 1e-5 of the field maximum vs the FP64 oracle after 100 steps; "
                                  "refine/coarsen decisions exact (criterion field adapted in FP64, "
                                  "block norms in float pairs); velocity fields adapted in FP32 arithmetic")
        del step64, g64
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
