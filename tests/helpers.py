"""Small workload builders shared by the tests (inputs only)."""
import copy

from paper_cs_9902024_gb300 import workloads as W


def box(dim=2, ncell=(8, 8, 1), L=None, kinds=None, Tw=300.0, fill_n=1e20,
        fill_T=300.0, fill_U=(0.0, 0.0, 0.0), ppc=50.0, d_ref=W.D_HS, omega=0.5,
        T_ref=300.0, dt=1e-6, runs=1, steps=1, fill=1, extra_bcs=()):
    """Closed box with one boundary kind per face (default specular),
    optionally filled with an equilibrium gas."""
    ncell = list(ncell)
    if dim == 2:
        ncell[2] = 1
    if L is None:
        L = [0.01 * ncell[0], 0.01 * ncell[1], 0.01 * ncell[2] if dim == 3 else 1.0]
    Vc = (L[0] / ncell[0]) * (L[1] / ncell[1]) * (L[2] / ncell[2])
    F_N = fill_n * Vc / ppc
    kinds = kinds or {}
    bcs = []
    for f in range(2 * dim):
        k = kinds.get(f, W.SPECULAR)
        bcs.append(W.bc(k, f, T=Tw))
    bcs.extend(copy.deepcopy(list(extra_bcs)))
    w = dict(name="box", dim=dim, ncell=ncell, L=list(L),
             gas=dict(mass=W.M_AR, d_ref=d_ref, T_ref=T_ref, omega=omega, F_N=F_N),
             fill=dict(kind=fill, n=fill_n, T=fill_T, U=list(fill_U)),
             bcs=bcs, runs=runs, steps=steps, dt=dt, sample_steps=[steps], seed=7)
    return W._clip_ranges(w)


def cell_index(w, x):
    """Cell of each position, from the definition floor(x / dx) clamped."""
    import numpy as np
    n = w["ncell"]
    d = [w["L"][a] / n[a] for a in range(3)]
    idx = []
    for a in range(3):
        if a < w["dim"]:
            i = np.floor(x[:, a] / d[a]).astype(np.int64)
            idx.append(np.clip(i, 0, n[a] - 1))
        else:
            idx.append(np.zeros(len(x), dtype=np.int64))
    return idx[0] + n[0] * (idx[1] + n[1] * idx[2])
