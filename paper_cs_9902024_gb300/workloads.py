"""Synthetic workloads shaped like the paper's unsteady DSMC problems.

This module only *describes* inputs: geometry, gas, boundaries, run counts,
time step and sample times. It holds none of the DSMC method's arithmetic
(no motion, indexing, collision or sampling code) and imports nothing from the
CUDA path or from the oracle, so both sides can be driven from the same
description.

The paper (Sec. 2 and Sec. 3) runs two unsteady problems -- a 3-D water vapour
flow in a comet's inner atmosphere and an impulsively started flow past a body
-- whose geometry and gas model it does not give.  The five workloads below
stand in for them; the scales they state in words ("cell size 1 mean free
path", "dt = 0.2 mean collision time", "~20 particles per cell") are turned
into numbers with the kinetic-theory definitions

    lambda = 1 / (sqrt(2) * pi * d^2 * n)           (hard-sphere mean free path)
    cbar   = sqrt(8 k T / (pi m))                   (mean thermal speed)
    tau    = lambda / cbar                          (mean collision time)

A workload is a plain dict:

    dim, ncell[3], L[3] (L[2] is the depth in 2-D), gas{mass,d_ref,T_ref,
    omega,F_N[,partner,n_sub]}, fill{kind,n,T,U}, bcs[list of dict], runs,
    steps, dt, sample_steps, seed, name
"""
from __future__ import annotations

import math

KB = 1.380649e-23

# boundary kinds
OUTFLOW, INFLOW, SPECULAR, DIFFUSE = 0, 1, 2, 3
# faces: 2*axis + side; 6 = internal plate
XMIN, XMAX, YMIN, YMAX, ZMIN, ZMAX, PLATE = 0, 1, 2, 3, 4, 5, 6

M_AR = 6.63e-26          # kg, molecular mass used by every workload
D_HS = 3.66e-10          # m, hard-sphere diameter


def mean_free_path(d, n):
    return 1.0 / (math.sqrt(2.0) * math.pi * d * d * n)


def mean_speed(T, m=M_AR):
    return math.sqrt(8.0 * KB * T / (math.pi * m))


def sound_speed(T, m=M_AR, gamma=5.0 / 3.0):
    return math.sqrt(gamma * KB * T / m)


def bc(kind, face, lo=(0, 0), hi=(1 << 30, 1 << 30), step_from=1, step_to=0,
       n=0.0, T=0.0, U=(0.0, 0.0, 0.0), plate_axis=0, plate_index=0):
    """One boundary segment. `lo`/`hi` are tangential cell ranges [lo, hi)
    along the face's two tangential axes (in increasing axis order); the
    default covers the whole face.  `step_from..step_to` (1-based, inclusive,
    0 = forever) is when the segment is active; later segments override
    earlier ones where both apply."""
    return dict(kind=kind, face=face, lo=list(lo), hi=list(hi),
                step_from=step_from, step_to=step_to, n=n, T=T, U=list(U),
                plate_axis=plate_axis, plate_index=plate_index)


def _clip_ranges(w):
    """Clamp open-ended tangential ranges to the face's cell counts."""
    nc = w["ncell"]
    for b in w["bcs"]:
        if b["face"] == PLATE:
            ax = b["plate_axis"]
        else:
            ax = b["face"] // 2
        tang = [a for a in range(3) if a != ax]
        for k in range(2):
            t = tang[k]
            lim = nc[t] if (t < w["dim"]) else 1
            b["lo"][k] = max(0, min(b["lo"][k], lim))
            b["hi"][k] = max(b["lo"][k], min(b["hi"][k], lim))
    return w


def duct(nx=64, ny=32, runs=8, steps=200, n_samples=4, seed=1, ppc=20.0,
         name="duct", filled=False):
    """2-D rectangular duct, impulsively started inflow on the left face
    (n=1e20 m^-3, T=300 K, drift 400 m/s), diffuse walls at 300 K top and
    bottom, outflow on the right; cell = 1 mean free path, dt = 0.2 mean
    collision time, ~`ppc` particles per cell at full fill.  The duct starts
    empty, or (`filled`) filled with the inflow state (the same n, T and
    drift), so that it holds ~`ppc` particles per cell from the first step."""
    n_in, T_in, U_in = 1.0e20, 300.0, 400.0
    lam = mean_free_path(D_HS, n_in)
    depth = 1.0
    Vc = lam * lam * depth
    F_N = n_in * Vc / ppc
    dt = 0.2 * lam / mean_speed(T_in)
    w = dict(
        name=name, dim=2, ncell=[nx, ny, 1], L=[nx * lam, ny * lam, depth],
        gas=dict(mass=M_AR, d_ref=D_HS, T_ref=T_in, omega=0.5, F_N=F_N),
        fill=(dict(kind=1, n=n_in, T=T_in, U=[U_in, 0.0, 0.0]) if filled
              else dict(kind=0, n=0.0, T=T_in, U=[0.0, 0.0, 0.0])),
        bcs=[
            bc(INFLOW, XMIN, n=n_in, T=T_in, U=(U_in, 0.0, 0.0)),
            bc(OUTFLOW, XMAX),
            bc(DIFFUSE, YMIN, T=300.0),
            bc(DIFFUSE, YMAX, T=300.0),
        ],
        runs=runs, steps=steps, dt=dt,
        sample_steps=[steps * (k + 1) // n_samples for k in range(n_samples)],
        seed=seed,
    )
    return _clip_ranges(w)


def duct64x32_n8(**kw):
    """Plain method, tiny: 64x32 duct, 200 steps, n = 8 runs, samples at
    steps 50/100/150/200, Philox seed 1."""
    args = dict(nx=64, ny=32, runs=8, steps=200, n_samples=4, seed=1,
                name="duct64x32_n8_s200")
    args.update(kw)
    return duct(**args)


def duct64x32_n512(**kw):
    """Batched ensemble of the 64x32 duct: n = 512 runs, 400 steps, 8 sample
    times."""
    args = dict(nx=64, ny=32, runs=512, steps=400, n_samples=8, seed=1,
                name="duct64x32_n512_s400")
    args.update(kw)
    return duct(**args)


def pulsed_jet(nx=256, ny=128, runs=64, steps=1000, n_samples=20, seed=1,
               pulse=100, orifice=16, F_N=4.49e10, name="jet256x128"):
    """2-D planar chamber, VHS argon (omega=0.81, d_ref=4.17e-10 m at 273 K),
    sonic inflow through a centred `orifice`-cell opening in the left wall at
    n=5e21 m^-3, T=300 K for `pulse` steps, then closed (diffuse 300 K wall);
    the rest of the left wall is diffuse at 300 K, the other faces are
    outflow to vacuum.  Cell = lambda(d_ref) at the orifice state, dt = 0.2
    tau there.  F_N = 4.49e10 is the reading of the workload's "peak ~2M
    particles per run": at that weight a drifting-Maxwellian flux through the
    16-cell orifice injects about 2.0e6 particles over the 100-step pulse."""
    n_o, T_o = 5.0e21, 300.0
    d_ref = 4.17e-10
    m = M_AR
    lam = mean_free_path(d_ref, n_o)
    depth = 1.0
    dt = 0.2 * lam / mean_speed(T_o)
    U_o = sound_speed(T_o)
    y0 = (ny - orifice) // 2
    w = dict(
        name=name, dim=2, ncell=[nx, ny, 1], L=[nx * lam, ny * lam, depth],
        gas=dict(mass=m, d_ref=d_ref, T_ref=273.0, omega=0.81, F_N=F_N),
        fill=dict(kind=0, n=0.0, T=T_o, U=[0.0, 0.0, 0.0]),
        bcs=[
            bc(DIFFUSE, XMIN, T=300.0),
            bc(INFLOW, XMIN, lo=(y0, 0), hi=(y0 + orifice, 1), step_from=1,
               step_to=pulse, n=n_o, T=T_o, U=(U_o, 0.0, 0.0)),
            bc(OUTFLOW, XMAX), bc(OUTFLOW, YMIN), bc(OUTFLOW, YMAX),
        ],
        runs=runs, steps=steps, dt=dt,
        sample_steps=[steps * (k + 1) // n_samples for k in range(n_samples)],
        seed=seed,
    )
    return _clip_ranges(w)


def jet256x128_n64(**kw):
    args = dict(name="jet256x128_n64_s1000")
    args.update(kw)
    return pulsed_jet(**args)


def plate3d(nx=128, ny=64, nz=64, runs=16, steps=600, n_samples=12, seed=1,
            plate=16, plate_x=32, ppc=15.0, name="plate128x64x64"):
    """3-D impulsively started Mach-5 flow past a zero-thickness normal flat
    plate (plate x plate cells, diffuse at 300 K) at x = plate_x cells,
    centred in y and z.  Hard-sphere gas, freestream n=1e20 m^-3, T=200 K;
    the box starts filled with freestream; x- and the four lateral faces are
    freestream inflow (which also removes leavers), x+ is outflow.  Cell =
    1 mean free path, dt = 0.2 tau, ~`ppc` particles per cell."""
    n_f, T_f = 1.0e20, 200.0
    lam = mean_free_path(D_HS, n_f)
    U = 5.0 * sound_speed(T_f)
    Vc = lam ** 3
    F_N = n_f * Vc / ppc
    dt = 0.2 * lam / mean_speed(T_f)
    fs = dict(n=n_f, T=T_f, U=(U, 0.0, 0.0))
    y0 = (ny - plate) // 2
    z0 = (nz - plate) // 2
    w = dict(
        name=name, dim=3, ncell=[nx, ny, nz], L=[nx * lam, ny * lam, nz * lam],
        gas=dict(mass=M_AR, d_ref=D_HS, T_ref=T_f, omega=0.5, F_N=F_N),
        fill=dict(kind=1, n=n_f, T=T_f, U=[U, 0.0, 0.0]),
        bcs=[
            bc(INFLOW, XMIN, **fs), bc(OUTFLOW, XMAX),
            bc(INFLOW, YMIN, **fs), bc(INFLOW, YMAX, **fs),
            bc(INFLOW, ZMIN, **fs), bc(INFLOW, ZMAX, **fs),
            bc(DIFFUSE, PLATE, lo=(y0, z0), hi=(y0 + plate, z0 + plate),
               T=300.0, plate_axis=0, plate_index=plate_x),
        ],
        runs=runs, steps=steps, dt=dt,
        sample_steps=[steps * (k + 1) // n_samples for k in range(n_samples)],
        seed=seed,
    )
    return _clip_ranges(w)


def plate128x64x64_n16(**kw):
    args = dict(name="plate128x64x64_n16_s600")
    args.update(kw)
    return plate3d(**args)


def mixed(n_runs=1024, cells_lo=32 * 16, cells_hi=512 * 256, steps=300, n_samples=4, seed=1,
          draw_seed=12345, name="duct_mixed", grids=None, filled=True):
    """Mixed-size ensemble: n_runs runs of the duct, each on its own grid,
    the cell count drawn log-uniformly in [cells_lo, cells_hi] with aspect
    2:1 and nx a multiple of 16.  The runs start filled with the inflow
    state (`filled`), so that a run holds ~20 particles per cell from the
    first step: log-uniform from ~10k to ~2.6M particles per run over the
    default range.  `grids`, a list of (nx, runs), replaces the draw with
    those grids (ny = nx / 2).  Runs that share a grid form one group; run
    r keeps global index r, so its draws do not depend on the grouping.
    Returns dict(name, runs, steps, groups): each group is a duct workload
    with `runs` its run count and `run0` the global index of its first run
    (global indices are handed out grid by grid, so each group's runs are
    one consecutive range)."""
    import numpy as np
    if grids is None:
        rng = np.random.default_rng(draw_seed)
        cells = np.exp(rng.uniform(np.log(cells_lo), np.log(cells_hi), size=n_runs))
        nx = np.clip(np.round(np.sqrt(2.0 * cells) / 16.0) * 16, 32, 512).astype(int)
        grids = [(g, int((nx == g).sum())) for g in sorted(set(nx.tolist()))]
    else:
        n_runs = sum(r for _, r in grids)
    groups = []
    # global run indices are assigned in grid order, so that every group is
    # one consecutive range of runs (one run_offset per group)
    start = 0
    for g, cnt in grids:
        w = duct(nx=g, ny=g // 2, runs=cnt, steps=steps, n_samples=n_samples, seed=seed,
                 name="%s_%dx%d" % (name, g, g // 2), filled=filled)
        w["run0"] = start
        groups.append(w)
        start += cnt
    assert start == n_runs
    return dict(name=name, runs=n_runs, steps=steps, groups=groups)


def mixed_n1024(**kw):
    return mixed(**kw)


# choice of the second particle of an NTC candidate pair (gas["partner"]):
# uniform over the cell, within the first particle's subcell (gas["n_sub"]
# subcells per axis), or the nearest other particle of the cell
PARTNER_UNIFORM, PARTNER_SUBCELL, PARTNER_NEAREST = 0, 1, 2
PARTNER_NAMES = {"uniform": PARTNER_UNIFORM, "subcell": PARTNER_SUBCELL,
                 "nearest": PARTNER_NEAREST}


def with_partner(w, scheme, n_sub=2):
    """The same workload with another collision-partner choice (`scheme` a
    PARTNER_NAMES key); its name gains the scheme (and subcell count)."""
    p = PARTNER_NAMES[scheme]
    w = dict(w)
    w["gas"] = dict(w["gas"], partner=p, n_sub=n_sub if p == PARTNER_SUBCELL else 1)
    if p != PARTNER_UNIFORM:
        w["name"] = w["name"] + ("_sub%d" % n_sub if p == PARTNER_SUBCELL else "_nn")
    return w


def by_name(name, **kw):
    table = {"duct64x32_n8": duct64x32_n8, "duct64x32_n512": duct64x32_n512,
             "jet256x128_n64": jet256x128_n64, "plate128x64x64_n16": plate128x64x64_n16,
             "mixed_n1024": mixed_n1024}
    return table[name](**kw)


def scaled(w, runs=None, steps=None, n_samples=None):
    """Same workload with fewer runs / steps (for tests and CPU samples)."""
    w = dict(w)
    w["bcs"] = [dict(b) for b in w["bcs"]]
    if runs is not None:
        w["runs"] = runs
    if steps is not None:
        w["steps"] = steps
        ns = n_samples if n_samples is not None else len(w["sample_steps"])
        w["sample_steps"] = sorted(set(
            max(1, steps * (k + 1) // ns) for k in range(ns)))
    return w
