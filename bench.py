#!/usr/bin/env python
"""Benchmark of the SPH hot path: neighbour interactions per second
(density + force) on one GB300, and the fraction of the FP32 roofline.

One step = one full kick-drift-kick step of the largest workload, 64M
particles Poisson-sampled from a lognormal density field (sigma_lnrho = 1.5,
P(k) ~ k^-2 on 256^3, periodic unit box): drift, cell grid (A1: a regrid,
or on a grid still valid for the drifted particles a refresh of positions
and boxes), octree split (A2), density with the smoothing-length iteration
(A4, A5), force (A6) and the kicks (A7). The metric counts density
interactions of the converged pass (ordered pairs j != i, r_ij < h_i) plus
force interactions (r_ij < max(h_i, h_j)) and divides by the device time of
the whole step. `--workload` selects another configuration; by default the
line also carries a summary of the other four (both interaction forms).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded
sample of the same workload). With torchrun (N > 1) every rank runs an
independent replica (the workload does not shard across GPUs; "replicas
only") and rank 0 prints the aggregate.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH neighbour interactions/sec (density+force) on 1 GB300; % FP32 roofline"
UNIT = "interactions/s"
FLOPS_DENSITY = 29   # per density interaction (FFMA = 2)
FLOPS_FORCE = 44     # per force interaction
SORT_BYTES_PER_PARTICLE = 16 + 13 * (4 + 4)  # pair-axis sorts: pm read, 13 keys + indices
SOD_DT = 7e-4        # 0.1 * min(h / c) of the initial state, rounded down


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["plain", "batched", "symmetric"], default="batched")
    ap.add_argument("--no-pair-sort", action="store_true",
                    help="per-pass form without the pair-axis sorts (whole source leaves)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the library's autotuner (tile, n_split, cell_factor) before timing")
    ap.add_argument("--tune", default=None,
                    help="fixed 'tile,n_split,cell_factor' instead of the autotuner (profiling runs)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the other interaction form for comparison")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload's particle count (same recipe) for profiling")
    ap.add_argument("--workload", default="lognormal", choices=["sod", "uniform", "clustered",
                                                                "batched", "lognormal"])
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the summary of the other configurations (both forms)")
    ap.add_argument("--config-steps", type=int, default=8,
                    help="timed steps per form in the summary of the other configurations")
    return ap.parse_args()


def workload(name, scale=1.0):
    """(particles, dt, name); dt None: chosen after the first density by cfl_dt."""
    from paper_1606_02738_gb300 import inputs
    k = {"uniform": 1, "sod": 2, "clustered": 3, "batched": 4, "lognormal": 5}[name]
    p = inputs.config(k, scale)
    tag = {1: "uniform_32k", 2: "sod3d_972k", 3: "plummer_clustered_4M", 4: "batched_256_boxes",
           5: "lognormal_64M"}[k]
    if scale != 1.0:
        tag = f"{tag}_scaled_{p.n}"
    return p, (SOD_DT if k == 2 else None), tag


ORACLE_MAX_N = 2_000_000  # larger workloads: the oracle legs run the same recipe shrunk


def oracle_workload(name, scale, p):
    """The particle set the oracle legs time: the workload itself, or for sets
    above ORACLE_MAX_N particles a part of about 1M particles (the oracle's
    untimed set-up density of every particle would otherwise take minutes):
    the first boxes of a multi-box set, else the same recipe and seed shrunk.
    Returns (particles, note)."""
    if p.n <= ORACLE_MAX_N:
        return p, ""
    target = ORACLE_MAX_N // 2
    if p.n_boxes > 1:
        import numpy as np
        k = int(np.searchsorted(p.box_offsets, target, side="left"))
        k = max(1, min(k, p.n_boxes))
        q = p.subset_boxes(0, k)
        return q, f" (the first {k} of its {p.n_boxes} boxes, {q.n} of {p.n} particles)"
    q, _, _ = workload(name, scale * target / p.n)
    return q, f" (the {name} recipe shrunk from {p.n} to {q.n} particles)"


def cfl_dt(ctx, gamma=5.0 / 3.0):
    """0.1 min_i h_i / (c_i + |v_i|), c = sqrt(gamma (gamma - 1) u), from the
    state after the first density (a global step small enough for every
    particle; the paper's test problems use the same global-step form)."""
    import torch
    h = ctx.get("h")
    u = ctx.get("u").double()
    v = ctx.get("v").double()
    c = torch.sqrt(gamma * (gamma - 1.0) * u.clamp_min(0.0))
    return float(0.1 * (h / (c + v.norm(dim=1))).min())


# ----------------------------------------------------------- distributed

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def reduce(self, value: float, op: str) -> float:
        if not self.pg:
            return value
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=getattr(self.pg.ReduceOp, op))
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def whole_job_rate(d: Dist, units: float, ms: float) -> tuple[float, float]:
    """Units all ranks processed / the slowest rank's time (units/s), and that
    time in ms (0 units or 0 ms -> rate 0)."""
    ms_max = d.reduce(float(ms), "MAX")
    total = d.reduce(float(units), "SUM")
    return (total / (ms_max / 1000.0) if ms_max > 0 else 0.0), ms_max


# ---------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi sampling (200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(gpu_index), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------- roofline

def fp32_peak_tflops(sm_count: int) -> tuple[float, str]:
    mhz = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        mhz = float(mp.get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    peak = sm_count * 128 * 2 * mhz * 1e6 / 1e12
    return peak, (f"derived: {sm_count} SMs x 128 FP32 lanes x 2 flop/FFMA x {mhz:.0f} MHz "
                  f"(MEASURED_PEAKS.json sm_max_mhz)")


def hbm_peak_gbs() -> tuple[float, str]:
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(mp["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


def kernel_traffic(kernel: str, mode: str, workload_name: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from a committed ncu capture of this kernel in this form on this workload,
    only while the source files it was taken on are unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(f"{kernel}_{mode}")
    except (OSError, ValueError):
        return None
    if not rec or rec.get("workload") != workload_name:
        return None
    if rec.get("source_sha") != source_sha(rec.get("sources", [])):
        return None
    return rec.get("bytes_per_launch")


def source_sha(files) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1606_02738_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def time_per_box(p, dt, args, dev, stream, flush, tuned, sph, torch):
    """The batched-boxes workload with one context per box: each box's step is
    its own launch sequence (and graph), the boxes one after another, timed
    with the same protocol as the single context holding all boxes."""
    kw = {}
    if tuned:
        kw = {k: tuned[k] for k in ("tile", "n_split", "cell_factor")}
    ctxs = []
    for b in range(p.n_boxes):
        c = sph.Context(mode=sph.SPH_MODE_BATCHED, device=dev, **kw).load(p.subset_box(b))
        c.density()
        c.force()
        ctxs.append(c)
    for _ in range(args.warmup):
        for c in ctxs:
            c.step(dt, 1)
    torch.cuda.synchronize(dev)
    s0 = [c.stats() for c in ctxs]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        for c in ctxs:
            c.step(dt, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    s1 = [c.stats() for c in ctxs]
    ms = sum(a.elapsed_time(b) for a, b in ev)
    inter = sum(b["total_density_interactions"] - a["total_density_interactions"] +
                b["total_force_interactions"] - a["total_force_interactions"]
                for a, b in zip(s0, s1))
    launches = sum(b["kernel_launches"] - a["kernel_launches"] for a, b in zip(s0, s1))
    for c in ctxs:
        c.close()
    return {"contexts": p.n_boxes, "value": inter / (ms / 1000.0), "ms_per_step": ms / args.steps,
            "interactions_per_step": inter / args.steps,
            "kernel_launches_per_step": launches / args.steps}


def kernel_roofline(s0, s1, inter_d, inter_f, ms, peak):
    """Achieved FP32 rate of the density and force kernels from the library's
    CUDA events (algorithmic flops of the counted interactions / kernel time)."""
    kern = {}
    for name, flops, t_key, n_key, ikey in (
            ("density", FLOPS_DENSITY, "t_density_ms", "density_launches", inter_d),
            ("force", FLOPS_FORCE, "t_force_ms", "force_launches", inter_f)):
        t = s1[t_key] - s0[t_key]
        n = max(1, s1[n_key] - s0[n_key])
        achieved = flops * ikey / (t / 1000.0) / 1e12 if t > 0 else 0.0
        kern[name] = {"achieved": achieved, "frac": achieved / peak, "launches": n,
                      "ms_per_launch": t / n, "share_of_step": t / ms if ms > 0 else 0.0,
                      "flops_per_launch": flops * ikey / n}
    return kern


def step_kinds(s0, s1):
    """Steps of the timed region by kind: on the reused grid (of those, redone on
    a new grid, and launched as one CUDA graph), and with a regrid."""
    return {k: int(s1[k] - s0[k]) for k in ("reused_steps", "redone_steps", "graph_steps")}


def time_form(p, dt, mode, steps, warmup, dev, stream, flush, sph, torch, peak,
              pair_sort=True):
    """One interaction form on one workload with the bench's protocol: load,
    density + force, the library's autotuner (untimed), `warmup` steps, then
    `steps` KDK steps timed one by one with CUDA events, L2 flushed between.
    Returns the rate, ms per step, kernel rooflines and step kinds."""
    c = sph.Context(mode=mode, profile=True, pair_sort=pair_sort, device=dev)
    c.load(p)
    c.density()
    c.force()
    tuned = c.autotune()
    if dt is None:
        dt = cfl_dt(c, p.gamma)
    for _ in range(warmup):
        c.step(dt, 1)
    torch.cuda.synchronize(dev)
    s0 = c.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        c.step(dt, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    s1 = c.stats()
    c.close()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    inter_d = s1["total_density_interactions"] - s0["total_density_interactions"]
    inter_f = s1["total_force_interactions"] - s0["total_force_interactions"]
    kern = kernel_roofline(s0, s1, inter_d, inter_f, ms, peak)
    mname = {sph.SPH_MODE_PLAIN: "plain", sph.SPH_MODE_BATCHED: "batched",
             sph.SPH_MODE_SYMMETRIC: "symmetric"}[mode]
    return {"mode": mname, "autotune": tuned,
            "dt": dt, "value": (inter_d + inter_f) / (ms / 1000.0), "ms_per_step": ms / steps,
            "interactions_per_step": (inter_d + inter_f) / steps,
            "density_frac": kern["density"]["frac"], "force_frac": kern["force"]["frac"],
            "kernels": kern, "steps": step_kinds(s0, s1)}


def config_summary(headline, args, dev, stream, flush, sph, torch, peak):
    """The other configurations, both gather forms, with the bench's protocol
    (fewer steps): rate, ms per step, batched / per-pass ratio and the FP32
    fractions of the interaction kernels; for sets of at most 1M particles
    also the symmetric pair-task form (its force serialises each top cell's
    tasks, so larger sets would take minutes)."""
    out = {}
    for name in ("uniform", "sod", "clustered", "batched", "lognormal"):
        if name == headline:
            continue
        p, dt, wname = workload(name, args.scale)
        rec = {"n_particles": p.n}
        modes = [sph.SPH_MODE_BATCHED, sph.SPH_MODE_PLAIN]
        if p.n <= 1_000_000:
            modes.append(sph.SPH_MODE_SYMMETRIC)
        for mode in modes:
            r = time_form(p, dt, mode, args.config_steps, 3, dev, stream, flush, sph, torch,
                          peak)
            rec[r["mode"]] = {k: r[k] for k in ("value", "ms_per_step", "density_frac",
                                                "force_frac", "autotune", "steps")}
        rec["batched_over_plain"] = rec["batched"]["value"] / rec["plain"]["value"]
        if "symmetric" in rec:
            rec["batched_over_symmetric"] = rec["batched"]["value"] / rec["symmetric"]["value"]
        out[wname] = rec
        del p
    return out


# ------------------------------------------------------------ CPU oracle

def step_label(kinds, steps):
    """What the timed steps were, from the library's step counters."""
    reg = steps - kinds["reused_steps"]
    return (f"kick-drift-kick steps: {reg} with a regrid, {kinds['reused_steps']} on the "
            f"previous grid (positions and boxes refreshed; {kinds['graph_steps']} of them "
            f"one CUDA graph launch, {kinds['redone_steps']} redone on a new grid); each: "
            f"density with the h iteration, force, kicks")


def cpu_baseline(p, min_s: float = 10.0, max_reps: int = 20, note: str = "") -> dict:
    """The FP64 oracle, as it stands, on h-iterated density + force
    evaluations of the workload (all particles, from the generator's h),
    repeated until at least `min_s` seconds of CPU work, on this host's
    cores."""
    import oracle
    oracle.build()
    inter, dt, reps = 0, 0.0, 0
    while reps < max_reps and (dt < min_s or reps == 0):
        s = oracle.State.from_particles(p)
        t0 = time.perf_counter()
        oracle.compute_density(s)
        oracle.compute_force(s)
        dt += time.perf_counter() - t0
        inter += int(s.n_dens.sum() + s.n_force.sum())
        reps += 1
    return {"value": inter / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{reps} h-iterated density + force evaluations of all {p.n} particles "
                      f"of the initial state ({inter} interactions, {dt:.2f} s){note}",
            "seconds": dt, "single_core": cpu_single_core(p)}


_ONE_CORE = r"""
import sys, time, json
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_1606_02738_gb300 import inputs
p = inputs.config(int(sys.argv[2]), float(sys.argv[3]))
s = oracle.State.from_particles(p)
oracle.compute_density(s)
rng = np.random.default_rng(11)
sub = np.sort(rng.choice(p.n, size=min(int(sys.argv[4]), p.n), replace=False))
t0 = time.perf_counter()
d = oracle.density(s.x, s.m, s.box[0], s.h, s.n_ngb, subset=sub)
f = oracle.force(s.x, s.v, s.m, s.u, s.h, s.rho, s.omega, s.box[0], s.gamma, subset=sub)
dt = time.perf_counter() - t0
print(json.dumps({"inter": int(d["count"][sub].sum() + f["count"][sub].sum()), "seconds": dt,
                  "threads": oracle.num_threads(), "n_sub": int(sub.size)}))
"""


def cpu_single_core(p, n_sub: int = 10000, scale: float = 0.1):
    """The oracle on one host core (OMP_NUM_THREADS=1, a fresh process): h-iterated
    density + force of a seeded subset of a Sod tube shrunk by `scale` (same recipe,
    same per-particle work), with the full neighbour context (the set-up density
    of all its particles is untimed)."""
    if p.name != "cfg2_sod":
        return None
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", _ONE_CORE, ROOT, "2", str(scale), str(n_sub)],
                             env=env, capture_output=True, text=True, timeout=600, check=True)
        r = json.loads(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None
    return {"value": r["inter"] / r["seconds"], "unit": UNIT, "cores": r["threads"],
            "sample": f"h-iterated density + force of {r['n_sub']} particles of the Sod tube "
                      f"shrunk to {scale:g} of its particles ({r['inter']} interactions, "
                      f"{r['seconds']:.2f} s)"}


def run_reference(args, d: Dist):
    """--impl reference: the oracle on the host cores, each step a bounded
    sample (density + force of a seeded particle subset, full neighbour
    context) of the same workload."""
    if d.rank != 0:
        return
    import numpy as np
    import oracle
    oracle.build()
    p0, dt, wname = workload(args.workload, args.scale)
    p, note = oracle_workload(args.workload, args.scale, p0)
    s = oracle.State.from_particles(p)
    oracle.compute_density(s)          # untimed set-up: every h, rho, Omega
    total = args.steps + args.warmup
    frac = min(1.0, 8.0 / max(1, total))
    n_sub = max(1000, min(int(p.n * frac), 200_000))
    rng = np.random.default_rng(7)
    inter = 0
    t_timed = 0.0
    for k in range(total):
        sub = np.sort(rng.choice(p.n, size=min(n_sub, p.n), replace=False))
        t0 = time.perf_counter()
        dd = oracle.density(s.x, s.m, s.box[0], s.h, s.n_ngb, subset=sub)
        ff = oracle.force(s.x, s.v, s.m, s.u, s.h, s.rho, s.omega, s.box[0], s.gamma, subset=sub)
        el = time.perf_counter() - t0
        if k >= args.warmup:
            t_timed += el
            inter += int(dd["count"][sub].sum() + ff["count"][sub].sum())
    value = inter / t_timed
    sample = (f"each step: h-iterated density + force of a seeded subset of {n_sub} of the "
              f"{p.n} particles (k-d tree over all), {args.steps} timed steps{note}")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * t_timed / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wname, "n_particles": p0.n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- ours

def run_ours(args, d: Dist):
    import torch
    from paper_1606_02738_gb300 import sph

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the CUDA path has no CPU fallback)")
    torch.cuda.set_device(d.local)
    dev = torch.device("cuda", d.local)
    p, dt, wname = workload(args.workload, args.scale)
    mode = {"batched": sph.SPH_MODE_BATCHED, "plain": sph.SPH_MODE_PLAIN,
            "symmetric": sph.SPH_MODE_SYMMETRIC}[args.mode]
    stream = torch.cuda.current_stream(dev)
    fixed = {}
    if args.tune:
        t, ns, cf = args.tune.split(",")
        fixed = {"tile": int(t), "n_split": int(ns), "cell_factor": float(cf)}
    ctx = sph.Context(mode=mode, profile=True, pair_sort=not args.no_pair_sort, device=dev,
                      **fixed)
    ctx.load(p)
    ctx.density()
    ctx.force()
    tuned = None if (args.no_autotune or fixed) else ctx.autotune()  # untimed set-up
    if fixed:
        tuned = dict(fixed, fixed=True)
    if dt is None:
        dt = cfl_dt(ctx, p.gamma)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    for _ in range(args.warmup):
        ctx.step(dt, 1)
    torch.cuda.synchronize(dev)
    s0 = ctx.stats()
    d.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(d.local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))             # evict L2 between timed steps (not timed)
        ev[k][0].record(stream)
        ctx.step(dt, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    d.barrier()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    s1 = ctx.stats()
    # density passes each particle needed in the last timed step (histogram)
    niter = torch.bincount(ctx.get("niter").long().clamp(0, 31)).cpu().tolist()
    passes_hist = {str(k): v / p.n for k, v in enumerate(niter) if v}
    ms = sum(a.elapsed_time(b) for a, b in ev)
    inter_d = s1["total_density_interactions"] - s0["total_density_interactions"]
    inter_f = s1["total_force_interactions"] - s0["total_force_interactions"]
    inter = inter_d + inter_f
    value, ms_max = whole_job_rate(d, inter, ms)

    # roofline of the interaction kernels (CUDA events around each launch,
    # recorded by the library on this stream)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_src = fp32_peak_tflops(sm_count)
    kern = kernel_roofline(s0, s1, inter_d, inter_f, ms, peak)
    kinds = step_kinds(s0, s1)
    dom = max(kern, key=lambda k: kern[k]["share_of_step"])
    roof = {"bound": "alu", "achieved": kern[dom]["achieved"], "peak": peak, "unit": "TFLOP/s",
            "frac": kern[dom]["achieved"] / peak, "traffic": kernel_traffic(dom, args.mode, wname),
            "kernel": dom, "peak_source": peak_src,
            "flops_per_interaction": {"density": FLOPS_DENSITY, "force": FLOPS_FORCE},
            "kernels": kern}
    # the second denominator: the FFMA rate this GPU sustains, measured now
    # (after the timed region, so it does not heat the timed steps)
    ffma = sph.sph_fp32_peak(dev.index if dev.index is not None else 0)
    roof["peak_ffma_measured"] = {"value": ffma["tflops"], "unit": "TFLOP/s",
                                  "frac": kern[dom]["achieved"] / ffma["tflops"],
                                  "how": "sph_fp32_peak: independent FFMA chains, full "
                                         "occupancy, best of 5 launches"}
    # the pair-axis sort kernel: HBM-bound, algorithmic bytes per particle =
    # one float4 read + 13 (key, index) pairs written
    t_sort = s1["t_sort_ms"] - s0["t_sort_ms"]
    n_sort = s1["sort_launches"] - s0["sort_launches"]
    if t_sort > 0 and n_sort > 0:
        gbs = SORT_BYTES_PER_PARTICLE * p.n * n_sort / (t_sort / 1000.0) / 1e9
        hbm = hbm_peak_gbs()
        roof["axis_sort"] = {"bound": "hbm", "achieved": gbs, "peak": hbm[0], "unit": "GB/s",
                             "frac": gbs / hbm[0], "peak_source": hbm[1],
                             "bytes_per_particle": SORT_BYTES_PER_PARTICLE,
                             "ms_per_launch": t_sort / n_sort, "launches": n_sort}
    stages = {k: (s1[k] - s0[k]) / args.steps for k in
              ("t_grid_ms", "t_sort_ms", "t_lists_ms", "t_density_ms", "t_ghost_ms",
               "t_force_ms", "t_integrate_ms")}

    # end to end through the C ABI with host buffers, as a host-driven run
    # does it: H2D of the particle state from pinned memory, init + density +
    # force + one KDK step, D2H of x, v, u, h, which are the next step's input
    host = {k: torch.as_tensor(getattr(p, k)).pin_memory() for k in ("x", "v", "m", "u", "h")}
    dbuf = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    outs = {"x": torch.empty((p.n, 3), dtype=torch.float64).pin_memory(),
            "v": torch.empty((p.n, 3), dtype=torch.float32).pin_memory(),
            "u": torch.empty(p.n, dtype=torch.float32).pin_memory(),
            "h": torch.empty(p.n, dtype=torch.float64).pin_memory()}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = sum(t.numel() * t.element_size() for t in outs.values())
    e2e_ms, e2e_inter = 0.0, 0
    for k in range(args.e2e_steps + 1):
        flush.fill_(float(k))
        torch.cuda.synchronize(dev)
        sa = ctx.stats()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for key in host:
            dbuf[key].copy_(host[key], non_blocking=True)
        sph.sph_init(ctx.ctx, p.box_offsets, p.box, **dbuf)
        ctx.density()
        ctx.force()
        ctx.step(dt, 1)
        for key, out in outs.items():
            out.copy_(ctx.get(key), non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
        sb = ctx.stats()
        for key in outs:  # the step's result is the next step's input (swap the buffers)
            host[key], outs[key] = outs[key], host[key]
        if k == 0:
            continue  # first pass warms the allocations
        e2e_ms += a.elapsed_time(b)
        e2e_inter += (sb["total_density_interactions"] - sa["total_density_interactions"] +
                      sb["total_force_interactions"] - sa["total_force_interactions"])
    e2e_val, e2e_ms_max = whole_job_rate(d, e2e_inter, e2e_ms)
    e2e_val = e2e_val if e2e_ms_max > 0 else None

    # the other interaction form, same workload, same protocol (comparison)
    other = None
    if not args.no_compare:
        omode = sph.SPH_MODE_PLAIN if mode == sph.SPH_MODE_BATCHED else sph.SPH_MODE_BATCHED
        other = time_form(p, dt, omode, args.steps, args.warmup, dev, stream, flush, sph, torch,
                          peak, pair_sort=not args.no_pair_sort)
        other.pop("kernels", None)

    # config 4: the same boxes as one context each (one launch sequence per box)
    per_box = None
    if p.n_boxes > 1 and not args.no_compare:
        per_box = time_per_box(p, dt, args, dev, stream, flush, tuned, sph, torch)

    configs = None
    if not args.no_configs and not args.no_compare:
        configs = config_summary(args.workload, args, dev, stream, flush, sph, torch, peak)

    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        q, note = oracle_workload(args.workload, args.scale, p)
        cpu = cpu_baseline(q, note=note)

    if d.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wname, "n_particles": p.n, "dt": dt,
                       "step": step_label(kinds, args.steps),
                       "reused_steps": kinds["reused_steps"],
                       "redone_steps": kinds["redone_steps"],
                       "graph_steps": kinds["graph_steps"],
                       "mode": args.mode, "l2": "flushed between timed steps (512 MiB write)",
                       "parallelism": "replicas" if d.world > 1 else "single GPU",
                       "interactions_per_step": inter / args.steps,
                       "particle_updates_per_s": p.n * d.world / (ms_max / args.steps / 1000.0),
                       "pairs_tested_last_step": s1["density_pair_candidates"] +
                       s1["force_pair_candidates"],
                       "density_passes_last_step": s1["density_passes"],
                       "batched_fallbacks_last_step": s1["batched_fallbacks"],
                       "fallback_causes_last_step": s1["fallback_causes"],
                       "tier2_groups_last_step": s1["tier2_groups"],
                       "tier3_entries_last_step": s1["tier3_entries"],
                       "stage_max": [s1["stage_max_density"], s1["stage_max_force"]],
                       "direct_warps_last_step": [s1["direct_list_warps"],
                                                  s1["direct_stage_warps"]],
                       "density_passes_hist_last_step": passes_hist,
                       "neighbour_cache_last_step": {
                           "groups": s1["n_groups"],
                           "density_on_cache": s1["cache_density_groups"],
                           "force_on_cache": s1["cache_force_groups"],
                           "built": s1["cache_built_groups"]},
                       "pair_sort": not args.no_pair_sort,
                       "autotune": tuned,
                       "leaves": s1["n_leaves"]},
            "roofline": roof,
            "stage_ms_per_step": stages,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "step": "H2D x v m u h (the previous step's result), sph_init, "
                            "sph_density, sph_force, sph_step(dt, 1), D2H x v u h"},
            "gpu_launches": int(s1["kernel_launches"] - s0["kernel_launches"]),
            "other_form": other,
            "per_box_launches": per_box,
            "configs": configs,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    d = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, d)
        else:
            run_ours(args, d)
    finally:
        d.close()


if __name__ == "__main__":
    main()
