"""Parity at the full sizes of the paper-shaped workloads (GPU).

* The 512-run 64x32 duct, 400 steps, 8 samples -- the ensemble bench.py
  times, in the same launch configuration (batched, CUDA graphs, FP32
  state) -- against the FP64 oracle's 512-run ensemble: density, velocity
  and temperature within 3 combined standard errors.
* The 128x64x64 plate box and the 256x128 pulsed jet on their full grids:
  FP64 device state in lockstep with the oracle for one run (readdressing
  array, cell counts and NTC counts exact; positions and velocities to
  rounding), which exercises the grouped Generation (tens of thousands of
  inflow elements) and cells of thousands of particles.
* Both at full size in FP32 with all their runs: no device error, particle
  conservation (fill + generated - removed = particles left)."""
import os

import numpy as np
import pytest

from oracle import Oracle, macro_from_acc, run_ensemble
from paper_cs_9902024_gb300 import workloads as W
from tests.parity import particle_errors, zscores

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc
    return dsmc


def _zfrac(mg, mo, mask):
    z, excluded = zscores(mg, mo, mask)
    return z, float(np.mean(np.abs(z) > 3)), excluded


def test_bench_ensemble_full_size_within_3_combined_se(D):
    w = W.duct64x32_n512()
    ens = D.Ensemble(w, autotune=True).run()     # as bench.py launches it
    T = len(w["sample_steps"])
    ms = [ens.macro(t) for t in range(T)]
    mg = {k: np.stack([m[k] for m in ms]) for k in ms[0]}
    raw = np.stack([ens.raw(t) for t in range(T)])
    st = ens.stats()
    assert st["error_word"] == 0
    acc_o, st_o = run_ensemble(w, threads=min(os.cpu_count() or 1, 16))
    mo = macro_from_acc(acc_o, w, w["runs"])
    mask = np.minimum(raw[..., 0].sum(1), acc_o[..., 0].sum(1)) >= 400
    z, frac, excluded = _zfrac(mg, mo, mask)
    rel = np.nanmedian(np.abs(mg["density"][mask] / mo["density"][mask] - 1))
    print("512-run duct: %d comparisons (%d NaN entries left out), |z|>3 fraction %.4f, "
          "max |z| %.2f, median rel. density error %.2e"
          % (z.size, excluded, frac, np.abs(z).max(), rel))
    assert z.size > 50000
    assert excluded <= 0.01 * z.size
    assert frac < 0.01
    for k in ("generated", "particle_steps", "collisions"):
        assert st[k] == pytest.approx(st_o[k], rel=0.01), k


def _exact_one_run(ens, orc, w, tol_x=1e-10, tol_v=1e-9):
    """Integer outputs bit-exact; every particle's own position error (in
    cell sizes) and velocity error (relative to its own speed, 0.1 c_mp
    floor) within tol_x / tol_v."""
    x, v, ids = ens.get_state(0)
    xo, vo, io = orc.get_state(0)
    assert np.array_equal(ids, io)
    cnt, cand, acc, lcr = ens.get_cells(0)
    co, cando, acco, lcro = orc.get_cells(0)
    assert np.array_equal(cnt, co)
    assert np.array_equal(lcr, lcro)
    assert np.array_equal(cand, cando)
    assert np.array_equal(acc, acco)
    _, ec, ev = particle_errors(w, x, v, xo, vo)
    assert float(ec.max()) <= tol_x
    assert float(ev.max()) <= tol_v
    return cnt


def _lockstep_one_run(D, w, steps):
    ens = D.Ensemble(w, precision="fp64", debug=True)
    ens.debug_begin(runs=1)
    orc = Oracle(w, runs=1)
    orc.init_run(0)
    ens.debug_step(steps)
    for s in range(1, steps + 1):
        orc.step(0, s)
    return ens, orc


def test_plate_box_full_grid_fp64_exact(D):
    w = W.plate128x64x64_n16(runs=1)
    ens, orc = _lockstep_one_run(D, w, 2)
    cnt = _exact_one_run(ens, orc, w)
    assert cnt.sum() > 7_000_000
    st = ens.stats()
    so = orc.stats(0)
    for k in ("generated", "removed", "wall_hits", "candidates", "collisions"):
        assert st[k] == so[k], k


def test_pulsed_jet_full_grid_fp64_exact(D):
    w = W.jet256x128_n64(runs=1)
    ens, orc = _lockstep_one_run(D, w, 12)
    cnt = _exact_one_run(ens, orc, w)
    assert cnt.max() > 1024         # cells of the radix-sorted one-CTA-per-cell path
    st = ens.stats()
    so = orc.stats(0)
    for k in ("generated", "removed", "wall_hits", "candidates", "collisions"):
        assert st[k] == so[k], k


@pytest.mark.parametrize("name", ["jet256x128_n64", "plate128x64x64_n16"])
def test_full_ensembles_conserve_particles(D, name):
    w = getattr(W, name)()
    ens = D.Ensemble(w).run()
    st = ens.stats()
    assert st["error_word"] == 0
    fill = 0
    if w["fill"]["kind"]:
        e0 = D.Ensemble(w).run(steps=0, sample_steps=[])
        fill = e0.stats()["particles_now"]
        e0.close()
    assert st["particles_now"] == fill + st["generated"] - st["removed"]
    assert st["collisions"] > 0
    # the last sample's particle count is the pool left after the run
    raw = ens.raw(len(w["sample_steps"]) - 1)
    assert int(raw[..., 0].sum()) == st["particles_now"]
