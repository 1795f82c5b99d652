"""Step-level parity of the CUDA path with the FP64 oracle (GPU).

FP64 device state: both sides take every discrete decision (cell, leaver,
collision acceptance, inflow count, entrant speed) in double precision, so
the readdressing array, the cell counts and the NTC candidate / accepted
counts must agree exactly for every step, and positions and velocities to
rounding.  FP32 device state: the same comparison from identical inputs over
one step and from t = 0 up to the first float-driven change of a cell
assignment (the "short horizon"), with mismatches counted."""
import numpy as np
import pytest

from oracle import Oracle
from paper_cs_9902024_gb300 import workloads as W
from tests.parity import compare_run, copy_oracle_state_to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc
    return dsmc


def _lockstep(D, w, runs, steps, precision="fp64", every=1):
    ens = D.Ensemble(w, precision=precision, debug=True)
    ens.debug_begin(runs=runs)
    orc = Oracle(w, runs=runs)
    for r in range(runs):
        orc.init_run(r)
    results = []
    # step 0 state (filled workloads) must already agree
    if w["fill"]["kind"]:
        for r in range(runs):
            x, v, ids = ens.get_state(r)
            xo, vo, io = orc.get_state(r)
            assert np.array_equal(ids, io)
            assert np.allclose(x, xo, rtol=0, atol=1e-13 * max(w["L"]))
            assert np.allclose(v, vo, rtol=1e-13, atol=1e-10)
    for s in range(1, steps + 1):
        ens.debug_step(1)
        for r in range(runs):
            orc.step(r, s)
        if s % every == 0 or s == steps:
            results.append([compare_run(ens, orc, r, w, 0, 0) for r in range(runs)])
    return ens, orc, results


def _assert_exact(results, tol_x=1e-10, tol_v=1e-10):
    """Bit-exact integer outputs; per-particle errors (positions in cell
    sizes, velocities relative to the particle's own speed, see
    tests/parity.py) within tol_x / tol_v."""
    for per_step in results:
        for res in per_step:
            assert res["mismatch"] == 0
            assert res["ids_equal"] and res["count_equal"] and res["lcr_equal"]
            assert res["cand_equal"] and res["acc_equal"]
            assert res["err_x_cell"] <= tol_x and res["err_v"] <= tol_v


def test_fp64_duct_every_step(D):
    """Empty duct filling from the inflow face: generation, diffuse walls,
    outflow, warp-path cells; 4 runs, 40 steps, every step compared."""
    w = W.duct64x32_n8(runs=4)
    ens, orc, res = _lockstep(D, w, runs=4, steps=40)
    _assert_exact(res)
    assert res[-1][0]["n"] > 4000
    st = ens.stats()
    so = [orc.stats(r) for r in range(4)]
    for k in ("generated", "removed", "wall_hits", "candidates", "collisions", "particle_steps"):
        assert st[k] == sum(s[k] for s in so), k


def test_fp64_plate3d_filled(D):
    """3-D box filled with a Mach-5 freestream, inflow on five faces, outflow
    on one, a diffuse plate inside: fill, lateral effusion inflow, plate
    hits, 3-D cell keys."""
    w = W.plate3d(nx=24, ny=12, nz=12, plate=6, plate_x=8, ppc=6, runs=2, steps=12,
                  n_samples=2)
    ens, orc, res = _lockstep(D, w, runs=2, steps=12)
    _assert_exact(res)
    assert ens.stats()["wall_hits"] > 0


def test_fp64_plate3d_grouped_generation(D):
    """Five inflow faces with 5184 elements: Generation runs as three CTAs
    per run after a counting pass, and each run's entrants must still be
    numbered in (element, k) order."""
    w = W.plate3d(nx=48, ny=24, nz=24, plate=8, plate_x=16, ppc=2, runs=2, steps=6,
                  n_samples=2)
    ens, orc, res = _lockstep(D, w, runs=2, steps=6)
    _assert_exact(res)
    assert ens.stats()["generated"] > 10000


def test_fp64_jet_big_cells_and_pulse(D):
    """VHS jet through an orifice that closes after 5 steps, with a particle
    weight low enough that cells near the orifice hold hundreds of particles
    (the one-CTA-per-cell path)."""
    w = W.pulsed_jet(nx=24, ny=16, runs=2, steps=10, n_samples=2, orifice=4, pulse=5,
                     F_N=4.49e10 * 4)
    ens, orc, res = _lockstep(D, w, runs=2, steps=10)
    _assert_exact(res, tol_x=1e-10, tol_v=1e-9)
    cnt = res[4][0]["cnt"]
    assert cnt.max() > 128, cnt.max()          # big-cell path taken
    assert ens.stats()["collisions"] > 0


def test_fp64_big_cells_wide_slot_spans(D):
    """Cells of 129 to 8000 particles (the radix-sorted paths: a quarter CTA
    per cell up to 1024 particles, a whole CTA above) whose particles' pool
    slots span one, two and three radix digits: some cells sit in one block
    of the pool, the others are spread over a pool of ~70k particles.  After
    one step every cell's particles are in pre-step slot order (LCR), and
    counts, NTC counts and the state agree exactly with the oracle.  (A
    fourth digit needs a pool above 2^24 particles; the pass loop is the
    same.)"""
    from tests.helpers import box
    w = box(dim=2, ncell=(6, 4, 1), ppc=50, dt=1e-7, runs=1, steps=1, fill=0)
    rng = np.random.default_rng(11)
    # (cell x, cell y, particles, in one block of the pool?)
    cells = [(5, 0, 600, True), (1, 1, 1500, False), (3, 1, 3000, False), (1, 2, 5000, True),
             (4, 2, 8000, False), (2, 3, 129, True), (5, 3, 1024, False), (0, 0, 1025, True),
             (0, 1, 8000, False), (2, 0, 8000, False), (3, 0, 8000, False), (4, 0, 8000, False),
             (0, 2, 8000, False), (2, 2, 8000, False)]
    dx = [w["L"][a] / w["ncell"][a] for a in range(2)]
    blocks, spread = [], []
    for cx, cy, n, block in cells:
        x = np.zeros((n, 3))
        x[:, 0] = (cx + rng.uniform(0.05, 0.95, n)) * dx[0]
        x[:, 1] = (cy + rng.uniform(0.05, 0.95, n)) * dx[1]
        (blocks if block else spread).append(x)
    sp = np.concatenate(spread)
    sp = sp[rng.permutation(len(sp))]
    cuts = np.sort(rng.choice(len(sp), len(blocks), replace=False))
    parts, prev = [], 0
    for c, blk in zip(cuts, blocks):
        parts += [sp[prev:c], blk]
        prev = c
    parts.append(sp[prev:])
    x = np.concatenate(parts)
    n = len(x)
    assert n > 65536
    ids = rng.permutation(n).astype(np.uint32)
    v = rng.normal(0.0, 250.0, (n, 3))
    ens = D.Ensemble(w, precision="fp64", debug=True, capacity_per_run=131072)
    ens.debug_begin(runs=1)
    orc = Oracle(w, runs=1)
    orc.init_run(0)
    orc.set_state(0, x, v, ids, n)
    ens.set_state(0, x, v, ids, n)
    ens.debug_step(1)
    orc.step(0, 1)
    res = compare_run(ens, orc, 0, w, 0, 0)
    _assert_exact([[res]])
    cnt, _, _, lcr = ens.get_cells(0)
    assert sorted(cnt[cnt > 128].tolist()) == sorted(c[2] for c in cells)
    st = ens.stats()
    assert st["collisions"] > 0 and st["error_word"] == 0
    # within each cell the pre-step slots ascend; the big cells' slot spans
    # need one, two and three 8-bit digits
    starts = np.concatenate([[0], np.cumsum(cnt)])
    digits = set()
    for c in np.nonzero(cnt > 128)[0]:
        seg = lcr[starts[c]:starts[c + 1]]
        assert np.all(np.diff(seg) > 0)
        digits.add((int(seg.max() - seg.min()).bit_length() + 7) // 8)
    assert digits == {1, 2, 3}, digits


def test_fp64_tiles_above_the_budget(D):
    """A 256-particle tile budget: nearly every tile of 256 cells holds more
    particles and is ordered in consecutive cell ranges that fit; LCR,
    counts, NTC counts and states still equal the oracle's every step."""
    w = W.duct64x32_n8(runs=2)
    ens = D.Ensemble(w, precision="fp64", debug=True, shape={"tile_budget": 256})
    ens.debug_begin(runs=2)
    orc = Oracle(w, runs=2)
    for r in range(2):
        orc.init_run(r)
    for s in range(1, 41):
        ens.debug_step(1)
        for r in range(2):
            orc.step(r, s)
        if s % 10 == 0:
            _assert_exact([[compare_run(ens, orc, r, w, 0, 0) for r in range(2)]])
    assert ens.stats()["shape"]["tile_budget"] == 256
    assert compare_run(ens, orc, 0, w, 0, 0)["n"] > 2000


@pytest.mark.parametrize("kinds", [(0, 3), (3, 0)])
def test_fp64_exact_corner_tie(D, kinds):
    """A flight reaching an x face and a y face at exactly the same time
    meets the x face first on the device as in the oracle (outflow x with
    diffuse y: removed, no wall hit; diffuse x with outflow y: re-emitted)."""
    from tests.helpers import box
    w = box(dim=2, ncell=(4, 4, 1), kinds={W.XMIN: kinds[0], W.YMIN: kinds[1]}, fill=0, dt=1e-5)
    d = w["L"][0] / 4
    x = np.array([[0.5 * d, 0.5 * d, 0.0]])
    v = np.array([[-1000.0, -1000.0, 0.0]])
    ids = np.array([0], dtype=np.uint32)
    ens = D.Ensemble(w, precision="fp64", debug=True, capacity_per_run=1024)
    ens.debug_begin(runs=1)
    orc = Oracle(w, runs=1)
    orc.init_run(0)
    orc.set_state(0, x, v, ids, 1)
    ens.set_state(0, x, v, ids, 1)
    ens.debug_step(1)
    orc.step(0, 1)
    st, so = ens.stats(), orc.stats(0)
    for k in ("removed", "wall_hits"):
        assert st[k] == so[k], k
    if kinds[0] == W.OUTFLOW:
        assert st["removed"] == 1 and st["wall_hits"] == 0
    else:
        assert st["wall_hits"] >= 1
    _assert_exact([[compare_run(ens, orc, 0, w, 0, 0)]])


def test_fp64_specular_and_tiny_cells(D):
    """Closed specular box, one particle per few cells, ragged grid."""
    from tests.helpers import box
    w = box(dim=2, ncell=(13, 7, 1), ppc=3, dt=5e-6, runs=3, steps=15)
    ens, orc, res = _lockstep(D, w, runs=3, steps=15)
    _assert_exact(res)


def test_fp32_one_step_from_identical_state(D):
    """FP32 device state, one step from the oracle's state (rounded to
    binary32 on both sides): cell assignments differ only where a particle
    sits within float rounding of a cell face, every particle's own error
    <= 1e-5 (position in cell sizes -- the stricter measure -- and velocity
    relative to its own speed with the 0.1 c_mp floor), and the integer
    outputs agree in every cell the mismatches do
    not touch -- except where the oracle's NTC value x = M + rem lies within
    binary32 rounding of an integer (the device forms the product in FP32
    and only carries the remainder in FP64)."""
    w = W.duct64x32_n8(runs=2)
    orc = Oracle(w, runs=2)
    for r in range(2):
        orc.init_run(r)
    k0 = 80
    for s in range(1, k0 + 1):
        for r in range(2):
            orc.step(r, s)
    ens = D.Ensemble(w, precision="fp32", debug=True)
    ens.debug_begin(runs=2)
    ens.debug_step(k0)                       # align the device step counter
    copy_oracle_state_to_device(orc, ens, range(2), fp32=True)
    total_mis = 0
    total_n = 0
    for s in range(k0 + 1, k0 + 4):
        ens.debug_step(1)
        for r in range(2):
            orc.step(r, s)
        for r in range(2):
            res = compare_run(ens, orc, r, w, 0, 0)
            total_mis += res["mismatch"]
            total_n += res["n"]
            assert res["err_x_cell"] <= 1e-5 and res["err_v"] <= 1e-5, (
                res["err_x_cell"], res["err_v"])
            diff = res["cnt"] != res["co"]
            assert diff.sum() <= 2 * res["mismatch"]
            rem_o, _ = orc.get_cell_state(r)
            x_o = res["cando"] + rem_o
            near = (res["co"] >= 2) & (np.minimum(rem_o, 1.0 - rem_o) <= 1e-6 * np.maximum(x_o, 1.0))
            same = ~diff & ~near
            assert np.array_equal(res["cand"][same], res["cando"][same])
        copy_oracle_state_to_device(orc, ens, range(2), fp32=True)
    assert total_mis <= max(4, 1e-3 * total_n), (total_mis, total_n)


def test_fp32_short_horizon(D):
    """FP32 device state from t = 0, 8 runs: each run's short horizon is its
    first step at which binary32 arithmetic shows -- a particle in another
    cell, an NTC candidate / accepted count that differs (binary32
    (sigma c_r)_max and acceptance ratios), or a particle whose own relative
    error exceeds 1e-5: its position relative to its position vector
    (floored at one cell) or its velocity relative to its own speed
    (floored at 0.1 c_mp).  Every step before a run's horizon matches the
    oracle exactly in its integer outputs (ids, cell counts, LCR, NTC
    counts) with every particle within 1e-5.  The position error in cell
    sizes, which grows with the steps as the velocity's rounding is
    integrated, is reported beside it.  The horizon is reported per run and
    must reach at least 10 steps in every run."""
    runs = 8
    w = W.duct64x32_n8(runs=runs)
    ens = D.Ensemble(w, precision="fp32", debug=True)
    ens.debug_begin(runs=runs)
    orc = Oracle(w, runs=runs)
    for r in range(runs):
        orc.init_run(r)
    horizon = [None] * runs
    kind = [None] * runs
    worst_x = [0.0] * runs
    worst_c = [0.0] * runs
    worst_v = [0.0] * runs
    checked = [0] * runs
    max_steps = 80
    for s in range(1, max_steps + 1):
        ens.debug_step(1)
        live = [r for r in range(runs) if horizon[r] is None]
        for r in range(runs):
            orc.step(r, s)
        for r in live:
            x = compare_run(ens, orc, r, w)
            if x["mismatch"]:
                horizon[r], kind[r] = s, "cell assignment"
                continue
            if not (x["cand_equal"] and x["acc_equal"]):
                horizon[r], kind[r] = s, "collision count"
                continue
            assert x["ids_equal"] and x["count_equal"] and x["lcr_equal"], (r, s)
            if x["err_x"] > 1e-5 or x["err_v"] > 1e-5:
                horizon[r], kind[r] = s, "error %.2e / %.2e" % (x["err_x"], x["err_v"])
                continue
            worst_x[r] = max(worst_x[r], x["err_x"])
            worst_c[r] = max(worst_c[r], x["err_x_cell"])
            worst_v[r] = max(worst_v[r], x["err_v"])
            checked[r] += x["n_compared"]
        if all(h is not None for h in horizon):
            break
    for r in range(runs):
        print("fp32 run %d: horizon %s (%s); up to it max per-particle relative error: "
              "x %.2e (%.2e cells), v %.2e; %d particle-steps compared" % (
                  r, horizon[r] if horizon[r] else ">%d" % max_steps, kind[r] or "none",
                  worst_x[r], worst_c[r], worst_v[r], checked[r]))
    reached = [h if h is not None else max_steps + 1 for h in horizon]
    assert min(reached) >= 10, reached
    # every run compared many particles before its horizon
    assert min(checked) >= 10000, checked
