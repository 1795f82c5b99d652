"""Comparison of the device path with the oracle, step by step.

Per-particle errors (every particle that sits in the same cell on both
sides, matched by id):

* position: |x_gpu - x_orc| / max(|x_orc|, h), the relative error of the
  particle's own position vector (over the simulated axes), floored at one
  cell size h for particles within a cell of the origin; also reported in
  cell sizes, max over the axes of |x_gpu - x_orc|_a / dx_a, the stricter
  measure the FP64 lockstep is held to;
* velocity: |v_gpu - v_orc| / max(|v_orc|, v_floor), the error of the
  particle's own velocity vector relative to its own speed, with a floor
  v_floor = 0.1 c_mp(T_ref), c_mp = sqrt(2 k T_ref / m): binary32 collision
  arithmetic rounds relative to the pair's relative speed (thermal scale),
  so a nearly resting particle's error is bounded by that scale, not by its
  own speed (fewer than 1e-3 of a Maxwellian gas's particles are slower
  than 0.1 c_mp).
"""
import math

import numpy as np

KB = 1.380649e-23


def cells_of_order(count):
    """Cell of each particle of a state in LCR order, from the
    per-cell counts of the same step."""
    return np.repeat(np.arange(len(count)), count)


def velocity_floor(w):
    g = w["gas"]
    return 0.1 * math.sqrt(2.0 * KB * g["T_ref"] / g["mass"])


def particle_errors(w, x, v, xo, vo, v_floor=None):
    """Per-particle errors of matched particles: position relative to its
    own position vector (floor: one cell), position in cell sizes, velocity
    relative to its own speed (floor v_floor)."""
    dim = w["dim"]
    d = np.array([w["L"][a] / w["ncell"][a] for a in range(dim)])
    if not len(x):
        z = np.zeros(0)
        return z, z, z
    dx = x[:, :dim] - xo[:, :dim]
    ex = np.linalg.norm(dx, axis=1) / np.maximum(np.linalg.norm(xo[:, :dim], axis=1), d.max())
    ec = np.max(np.abs(dx) / d, axis=1)
    fl = velocity_floor(w) if v_floor is None else v_floor
    sp = np.maximum(np.linalg.norm(vo, axis=1), fl)
    ev = np.linalg.norm(v - vo, axis=1) / sp
    return ex, ec, ev


def compare_run(ens, orc, run, w, rtol_x=None, rtol_v=None):
    """Compare one run's state after the same step on both sides.

    Returns a dict with the number of particles whose cell differs (or that
    live on one side only), the largest per-particle errors over the
    particles whose cell agrees (err_x relative to the particle's position,
    err_x_cell in cell sizes, err_v relative to the particle's own speed;
    p999_* the 99.9th percentiles), and whether the integer outputs of the step (counts, LCR,
    NTC candidate and accepted counts) agree everywhere."""
    x, v, ids = ens.get_state(run)
    xo, vo, io = orc.get_state(run)
    cnt, cand, acc, lcr = ens.get_cells(run)
    co, cando, acco, lcro = orc.get_cells(run)
    cg = cells_of_order(cnt)
    cr = cells_of_order(co)
    gmap = dict(zip(ids.tolist(), range(len(ids))))
    omap = dict(zip(io.tolist(), range(len(io))))
    common = sorted(set(gmap) & set(omap))
    only = len(gmap) + len(omap) - 2 * len(common)
    gi = np.array([gmap[i] for i in common], dtype=np.int64)
    oi = np.array([omap[i] for i in common], dtype=np.int64)
    same_cell = cg[gi] == cr[oi] if len(common) else np.zeros(0, bool)
    mism = only + int((~same_cell).sum())
    ex = ec = ev = px = pv = 0.0
    n_cmp = 0
    if same_cell.any():
        g, o = gi[same_cell], oi[same_cell]
        exs, ecs, evs = particle_errors(w, x[g], v[g], xo[o], vo[o])
        ex, ec, ev = float(exs.max()), float(ecs.max()), float(evs.max())
        px, pv = float(np.quantile(exs, 0.999)), float(np.quantile(evs, 0.999))
        n_cmp = len(g)
    exact = (np.array_equal(ids, io) and np.array_equal(cnt, co) and np.array_equal(cand, cando)
             and np.array_equal(acc, acco) and np.array_equal(lcr, lcro))
    return dict(mismatch=mism, err_x=ex, err_x_cell=ec, err_v=ev, p999_x=px, p999_v=pv,
                n_compared=n_cmp,
                exact=exact, n=len(ids),
                count_equal=np.array_equal(cnt, co), cand_equal=np.array_equal(cand, cando),
                acc_equal=np.array_equal(acc, acco), lcr_equal=np.array_equal(lcr, lcro),
                ids_equal=np.array_equal(ids, io), cnt=cnt, co=co, cand=cand, cando=cando,
                acc=acc, acco=acco)


def copy_oracle_state_to_device(orc, ens, runs, fp32):
    """Give both sides the same starting state: the oracle's particles (and
    its NTC remainders and (sigma c_r)_max), rounded to binary32 on both
    sides when the device holds FP32 state."""
    for r in runs:
        x, v, ids = orc.get_state(r)
        rem, smax = orc.get_cell_state(r)
        nid = orc.next_id(r)
        if fp32:
            x = x.astype(np.float32).astype(np.float64)
            v = v.astype(np.float32).astype(np.float64)
            smax = smax.astype(np.float32).astype(np.float64)
            orc.set_state(r, x, v, ids, nid)
            orc.set_cell_state(r, rem, smax)
        ens.set_state(r, x, v, ids, nid)
        ens.set_cell_state(r, rem, smax)


def zscores(mg, mo, mask):
    """z = (gpu - oracle) / combined SE of density, temperature and the three
    velocity components over the masked (sample, cell) entries.

    Entries whose combined SE is zero are not dropped: equal means there
    count as z = 0 and unequal means as |z| = inf (a failure).  Only NaN
    entries (a quantity undefined on a side, 0/0) are left out; their count
    is returned."""
    zs, excluded = [], 0
    pairs = [(mg["density"], mo["density"], mg["se_density"], mo["se_density"]),
             (mg["temperature"], mo["temperature"], mg["se_temperature"], mo["se_temperature"])]
    for a in range(3):
        pairs.append((mg["velocity"][..., a], mo["velocity"][..., a],
                      mg["se_velocity"][..., a], mo["se_velocity"][..., a]))
    for qg, qo, sg, so in pairs:
        d = (qg - qo)[mask]
        s = np.sqrt(sg ** 2 + so ** 2)[mask]
        with np.errstate(divide="ignore", invalid="ignore"):
            z = np.where(s > 0, d / np.where(s > 0, s, 1.0), np.where(d == 0, 0.0, np.inf))
        bad = np.isnan(d) | np.isnan(s)
        excluded += int(bad.sum())
        zs.append(z[~bad])
    return np.concatenate(zs), excluded
