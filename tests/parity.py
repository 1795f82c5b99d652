"""Comparison of the device path with the oracle, step by step."""
import numpy as np


def cells_of_order(count):
    """Cell of each particle of a state in (cell, id) order, from the
    per-cell counts of the same step."""
    return np.repeat(np.arange(len(count)), count)


def compare_run(ens, orc, run, w, rtol_x, rtol_v):
    """Compare one run's state after the same step on both sides.

    Returns a dict with the number of particles whose cell differs (or that
    live on one side only), the largest per-particle relative errors over
    the particles whose cell agrees (positions relative to the domain
    extent, velocities relative to the largest speed in the run), and
    whether the integer outputs of the step (counts, LCR, NTC candidate
    and accepted counts) agree everywhere."""
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
    L = np.array(w["L"][:w["dim"]])
    ex = ev = 0.0
    if same_cell.any():
        g, o = gi[same_cell], oi[same_cell]
        ex = float(np.max(np.abs(x[g, :w["dim"]] - xo[o, :w["dim"]]) / L))
        vref = max(float(np.abs(vo).max()), 1.0)
        ev = float(np.max(np.abs(v[g] - vo[o])) / vref)
    exact = (np.array_equal(ids, io) and np.array_equal(cnt, co) and np.array_equal(cand, cando)
             and np.array_equal(acc, acco) and np.array_equal(lcr, lcro))
    return dict(mismatch=mism, err_x=ex, err_v=ev, exact=exact, n=len(ids),
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
