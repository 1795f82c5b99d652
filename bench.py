#!/usr/bin/env python3
"""Benchmark: particle-steps/s of the n-run unsteady DSMC ensemble on GB300.

One bench step = one whole ensemble (`dsmc_run_ensemble`): the 512 runs of
the 64x32 duct (cell = 1 mean free path, dt = 0.2 mean collision time, hard
spheres, impulsively started inflow) for 400 time steps with 8 sample times
-- every time step is Generation, Motion, Enumeration/Indexing, Interaction
and (at sample steps) Sampling of all runs.  The particle pool (~1 GB at
full fill) is larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload.  Under torchrun
(N > 1) every rank runs its own share of runs (run indices offset by rank)
and the ensemble's group sums are summed over ranks once per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s over n-run ensemble on 1 GB300, batched vs plain at equal error"
UNIT = "particle-steps/s"
FALLBACK_HBM = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--runs", type=int, default=None, help="override runs per GPU")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the plain-mode, profile and CPU-baseline legs")
    p.add_argument("--workload", default="duct64x32_n512",
                   choices=["duct64x32_n8", "duct64x32_n512", "jet256x128_n64",
                            "plate128x64x64_n16", "mixed_n1024"],
                   help="workload (default: the 512-run duct the metric is quoted on; the others "
                        "are the parity workloads, measured the same way)")
    p.add_argument("--partner", default="uniform", choices=["uniform", "subcell", "nearest"],
                   help="choice of the second collision partner (gas model variant)")
    p.add_argument("--n-sub", type=int, default=2, help="subcells per axis (--partner subcell)")
    p.add_argument("--window", type=int, default=1,
                   help="time-averaged samples: each sample sums the last WINDOW steps up to its "
                        "sample time (1: instantaneous samples)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOAD_TEXT = {
    "duct64x32_n8": "2-D duct 64x32, HS, 8 runs x 200 steps, 4 sample times",
    "duct64x32_n512": "2-D duct 64x32, HS, 512 runs x 400 steps, 8 sample times",
    "jet256x128_n64": "2-D pulsed VHS jet 256x128, 64 runs x 1000 steps, 20 sample times",
    "plate128x64x64_n16": "3-D plate box 128x64x64, HS, 16 runs x 600 steps, 12 sample times",
    "mixed_n1024": "1024 duct runs on 31 grids 32x16..512x256 (log-uniform cells), filled, "
                   "300 steps, 4 sample times, one launch per kernel kind per step",
}


def workload(runs=None, name="duct64x32_n512", partner="uniform", n_sub=2):
    from paper_cs_9902024_gb300 import workloads as W
    w = W.by_name(name)
    if runs:
        w = W.scaled(w, runs=runs)
    if partner != "uniform":
        w = W.with_partner(w, partner, n_sub)
    return w


# oracle sample: whole runs for the duct workloads; the first steps of up to
# 16 runs for the large ones (a whole run of those takes minutes on a core)
ORACLE_PROBE_STEPS = {"duct64x32_n8": None, "duct64x32_n512": None, "jet256x128_n64": 20,
                      "plate128x64x64_n16": 4}


def oracle_rate(w, threads, probe_steps, target_s):
    """Particle-steps/s of the FP64 oracle (threads over run groups) on a
    bounded sample of workload w sized to about target_s seconds: a probe of
    up to 16 runs sizes the sample (more whole runs, or more steps)."""
    from oracle import run_ensemble
    runs, steps = w["runs"], w["steps"]
    r0 = min(runs, 16)
    s0 = steps if probe_steps is None else min(steps, probe_steps)
    t0 = time.perf_counter()
    run_ensemble(w, runs=r0, steps=s0, sample_steps=[], threads=threads)
    tp = max(time.perf_counter() - t0, 1e-3)
    if s0 == steps:
        rs, ss = int(min(runs, max(r0, r0 * round(target_s / tp)))), steps
    else:
        # later steps can hold more particles than the probe's: at most 5x
        rs, ss = r0, int(min(steps, 5 * s0, max(s0, s0 * target_s / tp)))
    t0 = time.perf_counter()
    _, st = run_ensemble(w, runs=rs, steps=ss, sample_steps=[], threads=threads)
    dt = time.perf_counter() - t0
    text = "%d of the %d runs x %d of the %d steps, FP64, %d thread(s) over run groups, %.1f s" % (
        rs, runs, ss, steps, threads, dt)
    return st["particle_steps"] / dt, text, dt


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def kernel_hash():
    # the device code: the kernel source up to its host launchers, and the
    # shared header, without comments and blank space
    h = hashlib.sha256()
    for p in ("paper_cs_9902024_gb300/csrc/dsmc_kernels.cu",
              "paper_cs_9902024_gb300/csrc/dsmc_internal.cuh"):
        with open(os.path.join(ROOT, p)) as f:
            text = f.read()
        cut = text.find("\n// Host launchers\n")
        text = text if cut < 0 else text[:cut]
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


# Algorithmic bytes per particle-step of the method's steps (FP32 SoA
# state; 2-D, 3-D): Motion reads x and the two (three) in-plane velocity
# components and writes x and the cell index; Indexing reads the cell index
# twice (histogram and scatter), writes the LCR and permutes the state
# (x, v, id read once and written once); Interaction reads the cell's
# velocities and writes the collided ones (with the cell data, ~16 B), and,
# when partners are chosen by position, reads every particle's position
# once more (D x 4 B).
def _method_bytes(D, positional=False):
    t = 4
    return {"motion": (2 * D + D) * t + 4 if D == 2 else 40,
            "scatter": 12,
            "permute": 2 * (D * t + 3 * t + 4),
            "interaction": 16 + (D * t if positional else 0)}


METHOD_ROWS = {"motion": ("move",), "indexing": ("scan", "scatter", "cell", "cell_big"),
               "interaction": ("collide", "collide_big")}


def algorithmic_bytes(w, st, steps, runs, cells=None):
    """Bytes each kernel group moves over one ensemble (FP32 state).

    "method": the algorithmic bytes of the method's step that the kernel
    carries out (28 B per moved particle for Motion in 2-D, 40 in 3-D; 12
    for the LCR scatter and 48 [56] for the permute of Indexing, 60 [68] in
    all; 16 for Interaction), times the particles it processes.
    "layout": the bytes of this data layout (one read of every
    input, one write of every output, no re-reads): the cell-relative
    offsets and stored cell keys, the 4-byte LCR entries (slots), the staged
    velocities."""
    D = w["dim"]
    t = 4
    if cells is None:
        cells = runs * w["ncell"][0] * w["ncell"][1] * (w["ncell"][2] if D == 3 else 1)
    moved_old = st["particle_steps"] - st["generated"]
    pool = st["pool_steps"]
    big = st.get("big_pool_steps", 0)
    positional = w["gas"].get("partner", 0) != 0
    mb = _method_bytes(D, positional)
    pos = D * t if positional else 0
    # read the LCR entry (4), gather offsets and v; write offsets, cell key,
    # v (ids are carried in debug mode only)
    gather = 4 + (D * t + 3 * t) + (D * t + 3 * t + 4)
    method = {
        "move": moved_old * mb["motion"],
        "scatter": pool * mb["scatter"],
        "cell": (pool - big) * mb["permute"],
        "cell_big": big * mb["permute"],
        "collide": (pool - big) * mb["interaction"],
        "collide_big": big * mb["interaction"],
        "scan": 0,
    }
    layout = {
        # read the in-cell offsets (D), v (D; the third component only at
        # wall hits) and the cell key, write the offsets (D) and the new key;
        # the count atomics stay in L2
        "move": moved_old * (2 * D * t + D * t + 8),
        # read the cell key, write the LCR entry (the slot)
        "scatter": pool * 8,
        # the tile kernel: particles of cells up to 128 (+ the start table);
        # cells above 128 particles: one CTA per cell, the same bytes
        "cell": (pool - big) * gather + cells * steps * 4,
        "cell_big": big * gather,
        # per cell: start, NTC remainder (read + write), (sigma c_r)_max;
        # the velocity of every particle in cells up to 128 read once (the
        # larger cells are the big-cell kernel's), both velocities of every
        # collision written; a positional partner choice also reads every
        # particle's position once
        "collide": (cells * steps * 24 + (pool - big) * (3 * t + pos)
                    + st["collisions"] * 2 * 3 * t),
        "collide_big": big * (3 * t + pos),
        # read counts, write starts
        "scan": cells * steps * 8,
        # write the entrants (x, v, key)
        "generate": st["generated"] * (D * t + 3 * t + 4),
    }
    return method, layout


def traffic_per_launch(workload, kernel, prs, path=None, khash=None, partner="uniform"):
    """DRAM bytes per launch of `kernel` from the ncu counters kept in
    profiles/traffic.json for the workload's family (grid and gas, any run
    count; a collision-partner variant is a family of its own): bytes per
    particle of the captured launch times the particles the kernel processed
    per launch in this profile pass (cells up to 128 particles for the tile
    kernels, the larger ones for the big-cell kernels).  None when there is
    no entry or the device code has changed since the capture (its hash
    differs)."""
    path = path or os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tj = json.load(f)
        family = workload.rsplit("_n", 1)[0] + ("" if partner == "uniform" else "_" + partner)
        ent = tj.get(family, {}).get(kernel)
        if not ent or ent.get("kernel_hash") != (khash or kernel_hash()):
            return None
        per_particle = ent["dram_bytes"] / ent["particles"]
        units = prs["pool_steps"]
        if kernel in ("cell", "collide"):
            units -= prs["big_pool_steps"]
        elif kernel in ("cell_big", "collide_big"):
            units = prs["big_pool_steps"]
        return per_particle * units / prs["launches_kernel"][kernel]
    except (OSError, ValueError, KeyError, ZeroDivisionError):
        return None


def method_rows(method, kern_ms, peak):
    """Achieved bandwidth of each of the method's steps on its algorithmic
    bytes: the bytes of the step's kernels over their summed time."""
    rows = {}
    for row, ks in METHOD_ROWS.items():
        ms = sum(kern_ms.get(k, 0.0) for k in ks)
        by = sum(method.get(k, 0) for k in ks)
        if ms > 0 and by > 0:
            gbs = by / (ms / 1e3) / 1e9
            rows[row] = {"kernels": list(ks), "ms": ms, "bytes": by, "achieved_gbs": gbs,
                         "frac": gbs / peak}
    return rows


# ---------------------------------------------------------------------------
def workload_config(w, args, runs=None):
    """The workload part of the bench line's config, the same in both arms."""
    if args.workload == "mixed_n1024":
        return {"workload": w["name"] + " (" + WORKLOAD_TEXT["mixed_n1024"] + ")",
                "runs": w["runs"], "grids": len(w["groups"]), "steps_per_run": w["steps"],
                "sample_times": len(w["groups"][0]["sample_steps"])}
    cells = 1
    for a in range(w["dim"]):
        cells *= w["ncell"][a]
    return {"workload": w["name"] + " (" + WORKLOAD_TEXT[args.workload] + ")",
            "runs_per_gpu": runs if runs is not None else w["runs"],
            "steps_per_run": w["steps"], "cells_per_run": cells,
            "sample_times": len(w["sample_steps"]),
            "partner": args.partner + (" (%d subcells per axis)" % args.n_sub
                                       if args.partner == "subcell" else "")}


def sample_windows(w, L):
    """Windows of L steps ending at the workload's sample times (None for
    instantaneous samples); they must be disjoint."""
    if L <= 1:
        return None
    ss = w["sample_steps"]
    win = [(max(1, t - L + 1), t) for t in ss]
    for (a, _), (_, b) in zip(win[1:], win[:-1]):
        if a <= b:
            raise SystemExit("windows of %d steps overlap at the sample times %s" % (L, ss))
    return win


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import run_ensemble
    cores = min(cpu_cores(), 16)
    if args.workload == "mixed_n1024":
        # the mixed workload: the first steps of up to 16 runs of its median
        # grid (as the measured arm's CPU leg)
        from paper_cs_9902024_gb300 import workloads as W
        m = W.by_name(args.workload)
        cfg = workload_config(m, args)
        w = m["groups"][len(m["groups"]) // 2]
        sample_runs, sample_steps = min(16, w["runs"]), min(20, w["steps"])
    else:
        w = workload(args.runs, args.workload, args.partner, args.n_sub)
        cfg = workload_config(w, args)
        sample_runs = min(64, w["runs"])
        probe = ORACLE_PROBE_STEPS[args.workload]
        sample_steps = w["steps"] if probe is None else min(w["steps"], 5 * probe)
    cfg.update(mode="FP64 oracle on the host cores, threads over run groups", state="fp64")
    wr = dict(w)

    def one():
        t0 = time.perf_counter()
        _, st = run_ensemble(wr, runs=sample_runs, steps=sample_steps, sample_steps=[],
                             threads=cores)
        return time.perf_counter() - t0, st["particle_steps"]

    for _ in range(args.warmup):
        one()
    tot_t, tot_ps = 0.0, 0
    for _ in range(args.steps):
        dt, ps = one()
        tot_t += dt
        tot_ps += ps
    value = tot_ps / tot_t
    sample = "%d of the %d runs x %d of the %d steps of %s per step, FP64 oracle, %d threads over runs" % (
        sample_runs, w["runs"], sample_steps, w["steps"], w["name"], cores)
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def roofline_of(w, prs, steps, runs, cells=None):
    """Per-kernel-kind times of a profile-mode run -> the kernels' table, the
    dominant kernel's roofline entry and the method steps' rows."""
    algo, layout = algorithmic_bytes(w, prs, steps, runs, cells)
    peak, src = measured_peaks()
    kern = {}
    total_ms = sum(prs["ms_kernel"].values())
    for k, msk in prs["ms_kernel"].items():
        if msk <= 0:
            continue
        e = {"ms": msk, "share": msk / total_ms, "launches": prs["launches_kernel"][k]}
        if algo.get(k):
            e["achieved_gbs"] = algo[k] / (msk / 1e3) / 1e9
            e["frac_of_%s_hbm" % src] = e["achieved_gbs"] / peak
        if layout.get(k):
            e["layout_gbs"] = layout[k] / (msk / 1e3) / 1e9
            e["layout_frac_of_%s_hbm" % src] = e["layout_gbs"] / peak
        kern[k] = e
    dom = max((k for k in kern if algo.get(k)), key=lambda k: kern[k]["ms"])
    achieved = kern[dom]["achieved_gbs"]
    roof = {"kernel": "k_" + dom, "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": None,
            "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
            "bytes_per_launch": algo[dom] / prs["launches_kernel"][dom],
            "bytes": "the method's algorithmic bytes of the kernel's step",
            "layout_achieved": kern[dom].get("layout_gbs"),
            "layout_frac": (kern[dom].get("layout_gbs") or 0.0) / peak}
    return kern, roof, method_rows(algo, prs["ms_kernel"], peak), dom


def bench_mixed(args):
    """The mixed-size ensemble: every step one launch per kernel kind over
    the 1024 runs of 31 grids (work queues), device-timed; end to end with
    every part's group sums copied to the host; the same ensemble as 31
    concurrent per-grid contexts for comparison; per-kernel roofline from a
    profile-mode run; the FP64 oracle on a bounded sample."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import workloads as W
    from paper_cs_9902024_gb300.dsmc import MixedEnsemble
    m = W.mixed_n1024()
    steps = m["steps"]
    T = len(m["groups"][0]["sample_steps"])
    me = MixedEnsemble(m)
    for _ in range(max(args.warmup, 3)):
        me.run()
    ps = me.stats()["particle_steps"]
    stream = me.parts[0].stream
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            me.run()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    value = ps * args.steps / (ms / 1e3)
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        me.run()
        raws = [np.stack([me.raw(gi, t) for t in range(T)]) for gi in range(len(m["groups"]))]
        for st in me.stats()["groups"]:
            h2d += st["h2d_bytes"]
            d2h += st["d2h_bytes"]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    del raws
    stats = me.stats()
    n_launch = len(me.parts)
    me.close()
    # -- the same ensemble as concurrent per-grid contexts ----------------
    mc = MixedEnsemble(m, mode="concurrent")
    mc.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mc.run()
    torch.cuda.synchronize()
    conc_s = time.perf_counter() - t0
    mc.close()
    # -- per-kernel-kind device times (profile mode) ---------------------
    mp = MixedEnsemble(m, profile=True)
    mp.run()
    prs = dict(mp.mixed_stats())
    mp.close()
    cells = sum(w["runs"] * w["ncell"][0] * w["ncell"][1] for w in m["groups"])
    kern, roof, rows, dom = roofline_of(m["groups"][0], prs, steps, m["runs"], cells)
    # -- the FP64 oracle on a bounded sample: the first steps of 16 runs of
    #    the median grid, threads over run groups ------------------------
    from oracle import run_ensemble
    wm = m["groups"][len(m["groups"]) // 2]
    cores = min(cpu_cores(), 16)
    t0 = time.perf_counter()
    _, sto = run_ensemble(wm, runs=min(16, wm["runs"]), steps=20, sample_steps=[], threads=cores)
    dto = time.perf_counter() - t0
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(m, args),
                       mode="one launch per kernel kind per step, work queues, CUDA graph per step",
                       state="fp32", sampling="fp64 group sums",
                       l2="inputs larger than L2 (pool ~30 GB)"),
        "clocks": clk.summary(),
        "e2e": {"value": ps * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        # every step: generate, move, move_slow, scan (two passes), scatter,
        # cell, cell_big, collide_big, collide, step_end (+ reduce at sample
        # steps); each part's fill: 6
        "gpu_launches": args.steps * (steps * 11 + 6 * n_launch + T),
        "particle_steps_per_step": ps,
        "particles_at_end": stats["particles_now"],
        "concurrent_contexts": {"value": ps / conc_s, "unit": UNIT, "contexts": n_launch,
                                "note": "one batched context per grid, each on its own stream "
                                        "and host thread; wall clock of one ensemble"},
        "roofline": roof, "method_steps": rows, "kernels": kern,
        "cpu_baseline": {"value": sto["particle_steps"] / dto, "unit": UNIT, "cores": cores,
                         "kind": "oracle",
                         "sample": "16 runs of the %dx%d grid x 20 of the 300 steps, FP64, %d "
                                   "thread(s) over run groups, %.1f s"
                                   % (wm["ncell"][0], wm["ncell"][1], cores, dto)},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.workload == "mixed_n1024" and args.partner != "uniform":
        raise SystemExit("the mixed workload is measured with the uniform partner choice")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mixed_n1024":
        return bench_mixed(args)
    ws, rank, local = dist_env()
    import numpy as np
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = local
    torch.cuda.set_device(device)
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300.dsmc import Ensemble
    from paper_cs_9902024_gb300 import shard
    w = workload(args.runs, args.workload, args.partner, args.n_sub)
    runs = w["runs"]
    shard.groups(runs, ws)          # every rank must hold >= 16 runs when sharded
    steps = w["steps"]
    n_samples = len(w["sample_steps"])
    stream = torch.cuda.Stream(device=device)
    win = sample_windows(w, args.window)
    ens = Ensemble(w, device=device, stream=stream, run_offset=shard.run_offset(rank, runs),
                   autotune=True)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(max(args.warmup, 3)):
        ens.run(windows=win)
    st = ens.stats()
    ps_per_step = st["particle_steps"]
    # fill: 6 launches (cells, counts, scan (two passes), particles, ids);
    # every time step: generate, move, move_slow, scan1, scan2, scatter,
    # cell, cell_big, collide_big, collide, step_end, and reduce at the
    # sample steps only
    launches_per_step = 6 + steps * 11 + n_samples
    # -- device-timed region: inputs resident, results stay on the device --
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(device) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            ens.run(windows=win)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    ps_total = ps_per_step * args.steps
    if ws > 1:
        ms = shard.allreduce_max(ms)
        ps_total = shard.allreduce_sum(ps_total)
    value = ps_total / (ms / 1e3)
    # -- end to end through the C ABI with host buffers --------------------
    barrier()
    torch.cuda.synchronize()
    h2d = d2h = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ens.run(windows=win)
        raws = np.stack([ens.raw(t) for t in range(n_samples)])
        if ws > 1:
            raws = shard.allreduce_group_sums(raws)
        s2 = ens.stats()
        h2d += s2["h2d_bytes"]
        d2h += s2["d2h_bytes"]
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        e2e_s = shard.allreduce_max(e2e_s)
    e2e = {"value": ps_total / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(w, args, runs),
                       mode="batched, CUDA graph per step", state="fp32",
                       sampling="fp64 group sums" + (
                           ", each sample time-averaged over %d steps" % args.window
                           if win else ""),
                       l2="inputs larger than L2 (pool ~1 GB)",
                       parallelism="runs sharded over %d GPU(s)" % ws),
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "launch_shape": dict(st["shape"], autotuned=bool(st["tuned"])),
        "particle_steps_per_step": ps_per_step,
    }
    if rank == 0 and ws == 1 and not args.no_extras:
        # -- plain per-run loop on the same workload (a sample of the runs:
        #    the per-run loop's cost is the same for every run) ------------
        plain_runs = max(2, min(64, runs // 8))
        pe = Ensemble(w, mode="plain", device=device, stream=stream)
        pe.run(runs=min(8, plain_runs), windows=win)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pe.run(runs=plain_runs, windows=win)
        e1.record(stream)
        torch.cuda.synchronize()
        pst = pe.stats()
        pms = e0.elapsed_time(e1)
        # same-seed batched run of the same 64 runs: identical sums
        be = Ensemble(w, device=device, stream=stream).run(runs=plain_runs, windows=win)
        same = all(np.array_equal(pe.raw(t), be.raw(t)) for t in range(n_samples))
        out["plain"] = {"value": pst["particle_steps"] / (pms / 1e3), "unit": UNIT,
                        "runs_timed": plain_runs, "ms": pms,
                        "batched_over_plain": value / (pst["particle_steps"] / (pms / 1e3)),
                        "sample_error": "equal: plain and batched group sums bit-identical"
                        if same else "DIFFERENT"}
        pe.close()
        be.close()
        # -- per-kernel device times (profile mode: CUDA events around every
        #    launch on the library's stream) and the roofline ------------
        #    The profile ensemble takes the timed ensemble's (tuned) launch
        #    shape and runs the workload twice; the per-kernel times are the
        #    means over both runs.
        pr = Ensemble(w, profile=True, device=device, stream=stream, shape=st["shape"])
        passes = []
        for _ in range(2):
            pr.run(windows=win)
            passes.append(pr.stats())
        pr.close()
        prs = dict(passes[-1])
        for key in ("ms_kernel", "launches_kernel"):
            prs[key] = {k: sum(p[key][k] for p in passes) / len(passes) for k in passes[-1][key]}
        prs["ms_steps"] = sum(p["ms_steps"] for p in passes) / len(passes)
        kern, roof, rows, dom = roofline_of(w, prs, steps, runs)
        roof["traffic"] = traffic_per_launch(args.workload, dom, prs, partner=args.partner)
        out["roofline"] = roof
        out["method_steps"] = rows
        out["kernels"] = kern
        out["profile_run_ms"] = prs["ms_steps"]
        out["profile_shape"] = passes[-1]["shape"]
        # -- the FP64 oracle on the host cores, bounded samples (threads over
        #    run groups: at most G = 16), and on one core ------------------
        cores = min(cpu_cores(), 16)
        probe = ORACLE_PROBE_STEPS[args.workload]
        rate, text, _ = oracle_rate(w, cores, probe, 15.0)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": text}
        rate1, text1, _ = oracle_rate(w, 1, probe if probe is not None else 40, 8.0)
        out["cpu_baseline_1core"] = {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                     "sample": text1}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ens.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
