"""Ensemble-level parity of the CUDA path with the oracle, mode equivalence
and edge cases (GPU)."""
import numpy as np
import pytest

from oracle import Oracle, macro_from_acc, run_ensemble
from paper_cs_9902024_gb300 import workloads as W
from tests.parity import zscores

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc
    return dsmc


def _zscores(mg, mo, nmin_mask):
    z, excluded = zscores(mg, mo, nmin_mask)
    assert excluded <= 0.01 * max(z.size, 1), excluded
    return z


def _gpu_macro(ens, T):
    ms = [ens.macro(t) for t in range(T)]
    return {k: np.stack([m[k] for m in ms]) for k in ms[0]}


def test_duct_ensemble_fp32_within_3_combined_se(D):
    """The configuration of the paper-sized small case (64x32 duct, 8 runs,
    200 steps, samples at 50/100/150/200): FP32 batched device ensemble vs
    the FP64 oracle; density, velocity and temperature per (sample, cell)
    within 3 combined standard errors."""
    w = W.duct64x32_n8()
    acc_o, st_o = run_ensemble(w, threads=8)
    mo = macro_from_acc(acc_o, w, w["runs"])
    ens = D.Ensemble(w)
    ens.run()
    T = len(w["sample_steps"])
    mg = _gpu_macro(ens, T)
    raw = np.stack([ens.raw(t) for t in range(T)])
    npool = np.minimum(raw[..., 0].sum(1), acc_o[..., 0].sum(1))
    mask = npool >= 40
    z = _zscores(mg, mo, mask)
    frac = np.mean(np.abs(z) > 3)
    rel_n = np.nanmedian(np.abs(mg["density"][mask] / mo["density"][mask] - 1))
    print("duct64x32_n8 fp32: %d comparisons, |z|>3 fraction %.4f, max |z| %.2f, median rel err "
          "density %.3g" % (z.size, frac, np.abs(z).max(), rel_n))
    assert z.size > 10000
    assert frac < 0.01
    st = ens.stats()
    # counters agree statistically with the oracle's
    for k in ("generated", "particle_steps", "collisions"):
        assert st[k] == pytest.approx(st_o[k], rel=0.02), k


def test_duct_ensemble_fp64_matches_oracle_sums(D):
    """FP64 device state: the group sums of every sample equal the oracle's
    to rounding (the sampling and the fixed-order reduction over runs)."""
    w = W.duct64x32_n8()
    acc_o, st_o = run_ensemble(w, threads=8)
    ens = D.Ensemble(w, precision="fp64")
    ens.run()
    raw = np.stack([ens.raw(t) for t in range(len(w["sample_steps"]))])
    assert np.array_equal(raw[..., 0], acc_o[..., 0])
    assert np.allclose(raw, acc_o, rtol=1e-9, atol=1e-6)
    st = ens.stats()
    for k in ("generated", "removed", "wall_hits", "candidates", "collisions", "particle_steps"):
        assert st[k] == st_o[k], k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_plain_equals_batched_bitwise(D, precision):
    """The plain per-run loop and the batched graph-captured form give
    bit-identical sums (same draws, same per-cell order, same run order in
    the reduction): equal sample error by construction."""
    w = W.duct64x32_n8(runs=19, steps=60, n_samples=3)      # ragged groups (G = 16)
    a = D.Ensemble(w, precision=precision, mode="batched").run()
    b = D.Ensemble(w, precision=precision, mode="plain").run()
    c = D.Ensemble(w, precision=precision, mode="batched", use_graph=False).run()
    for t in range(3):
        ra, rb, rc = a.raw(t), b.raw(t), c.raw(t)
        assert np.array_equal(ra, rb) and np.array_equal(ra, rc)
    sa, sb = a.stats(), b.stats()
    for k in ("generated", "removed", "candidates", "collisions", "particle_steps"):
        assert sa[k] == sb[k]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_particle_ids_are_bookkeeping_only(D, precision):
    """Particle ids are kept only in debug mode (the test hooks report them);
    no step reads them -- wall draws are keyed by a particle's place in its
    run's order -- so an ensemble with ids and one without give
    bit-identical sums and counters (duct with diffuse walls and inflow,
    19 runs)."""
    w = W.duct64x32_n8(runs=19, steps=60, n_samples=3)
    a = D.Ensemble(w, precision=precision, debug=True).run()
    b = D.Ensemble(w, precision=precision).run()
    for t in range(3):
        assert np.array_equal(a.raw(t), b.raw(t)), t
    sa, sb = a.stats(), b.stats()
    for k in ("generated", "removed", "wall_hits", "candidates", "collisions", "particle_steps"):
        assert sa[k] == sb[k], k
    assert sa["wall_hits"] > 0


def test_edge_cases(D):
    # one run, sample at step 1 and at the last step
    w = W.duct64x32_n8(runs=1, steps=5)
    ens = D.Ensemble(w).run(sample_steps=[1, 5])
    assert ens.raw(0)[..., 0].sum() > 0
    # zero steps, no samples: nothing moves, no error
    ens.run(steps=0, sample_steps=[])
    assert ens.stats()["particle_steps"] == 0
    # an empty closed box: no particles at any time
    from tests.helpers import box
    e = D.Ensemble(box(fill=0, runs=3, steps=4)).run()
    assert e.stats()["particles_now"] == 0
    assert np.all(e.raw(0) == 0)
    # invalid sample lists are rejected, the context stays usable
    with pytest.raises(D.DsmcError) as ex:
        ens.run(steps=5, sample_steps=[3, 2])
    assert ex.value.status == D.E_INVALID
    with pytest.raises(D.DsmcError):
        ens.run(steps=5, sample_steps=[6])
    ens.run(steps=5, sample_steps=[5])
    with pytest.raises(D.DsmcError):
        ens.raw(1)


def test_capacity_overflow_is_reported_not_faulted(D):
    """A pool far too small overflows on the device; the kernels keep every
    access in bounds, the run returns DSMC_E_CAPACITY, and the context
    works again with a proper capacity."""
    w = W.duct64x32_n8(runs=4, steps=40)
    ens = D.Ensemble(w, capacity_per_run=300)
    with pytest.raises(D.DsmcError) as ex:
        ens.run()
    assert ex.value.status == D.E_CAPACITY
    ens.close()
    ok = D.Ensemble(w).run()
    assert ok.stats()["error_word"] == 0


def test_macro_quantities_match_oracle_formulae(D):
    """The device's macroscopic quantities equal the oracle's formulae
    applied to the device's own group sums."""
    w = W.duct64x32_n8(runs=20, steps=50, n_samples=2)
    ens = D.Ensemble(w).run()
    for t in range(2):
        raw = ens.raw(t)
        m = ens.macro(t)
        ref = macro_from_acc(raw[None], w, 20)
        for k in ("density", "temperature", "se_density", "se_temperature"):
            a, b = m[k], ref[k][0]
            fin = np.isfinite(b)
            assert np.array_equal(np.isfinite(a), fin), k
            assert np.allclose(a[fin], b[fin], rtol=1e-10, atol=1e-12), k
        assert np.allclose(m["velocity"], ref["velocity"][0], rtol=1e-10, atol=1e-9, equal_nan=True)


def test_autotune_keeps_results(D):
    """options.autotune searches launch shapes on a trial ensemble; the real
    run's group sums are bit-identical to the fixed-shape run."""
    w = W.duct64x32_n8(runs=32, steps=120, n_samples=3)
    a = D.Ensemble(w, autotune=True).run()
    b = D.Ensemble(w).run()
    for t in range(3):
        assert np.array_equal(a.raw(t), b.raw(t))
    sa, sb = a.stats(), b.stats()
    assert sa["tuned"] == 1 and sb["tuned"] == 0
    assert sa["shape"]["tile_budget"] in (2048, 3072, 4608)
    for k in ("generated", "removed", "candidates", "collisions", "particle_steps"):
        assert sa[k] == sb[k], k
    print("autotuned shape:", sa["shape"], "default:", sb["shape"])
    # the tuned shape given explicitly to a new context: same shape, same sums
    c = D.Ensemble(w, shape=sa["shape"]).run()
    assert c.stats()["shape"] == sa["shape"] and c.stats()["tuned"] == 0
    for t in range(3):
        assert np.array_equal(a.raw(t), c.raw(t))


def test_explicit_launch_shape(D):
    """options.shape replaces the default launch shape entry by entry; the
    group sums do not change, including a small tile budget (most tiles on
    the per-cell path) created after a context with a large budget (the tile
    kernel's shared-memory limit must not drop under the larger context).
    Out-of-range entries are refused."""
    w = W.duct64x32_n8(runs=16, steps=40, n_samples=2)
    big = D.Ensemble(w, shape={"tile_budget": 16384, "move_blocks": 152})
    ref = D.Ensemble(w).run()
    small = D.Ensemble(w, shape={"tile_budget": 256, "scatter_blocks": 7,
                                 "collide_blocks": 3}).run()
    big.run()
    assert big.stats()["shape"]["tile_budget"] == 16384
    assert big.stats()["shape"]["move_blocks"] == 152
    s = small.stats()["shape"]
    assert (s["tile_budget"], s["scatter_blocks"], s["collide_blocks"]) == (256, 7, 3)
    for t in range(2):
        assert np.array_equal(ref.raw(t), small.raw(t))
        assert np.array_equal(ref.raw(t), big.raw(t))
    for bad in ({"tile_budget": 100}, {"tile_budget": 20000}, {"move_blocks": -1},
                {"collide_blocks": 1 << 21}):
        with pytest.raises(D.DsmcError):
            D.Ensemble(w, shape=bad)


def test_sample_windows_match_oracle_and_modes(D):
    """Time-averaged samples: FP64 device sums equal the oracle's (counts
    exactly), plain == batched bit for bit, and the device density divides
    by runs x window length."""
    w = W.duct64x32_n8(runs=5, steps=60, n_samples=2)
    win = [(10, 19), (40, 60)]
    acc_o, _ = run_ensemble(w, windows=win)
    e64 = D.Ensemble(w, precision="fp64").run(windows=win)
    for t in range(2):
        raw = e64.raw(t)
        assert np.array_equal(raw[..., 0], acc_o[t][..., 0])
        assert np.allclose(raw, acc_o[t], rtol=1e-9, atol=1e-6)
    a = D.Ensemble(w).run(windows=win)
    b = D.Ensemble(w, mode="plain").run(windows=win)
    for t in range(2):
        assert np.array_equal(a.raw(t), b.raw(t))
    raw = a.raw(1)
    m = a.macro(1)
    d = [w["L"][k] / w["ncell"][k] for k in range(3)]
    Vc = d[0] * d[1] * w["L"][2]
    n_expect = raw[..., 0].sum(axis=0) * w["gas"]["F_N"] / (5 * 21 * Vc)
    assert np.allclose(m["density"], n_expect, rtol=1e-12)


def test_checks_pass_on_normal_runs(D):
    """options.checks: the device pass over the final pool (cell keys inside
    the table and inside their cell's range, ids increasing within a cell,
    offsets inside the cell, finite velocities) passes after ordinary
    runs -- batched FP32, FP64, plain, and a filled 3-D box -- and leaves
    the results as they are without it."""
    w = W.duct64x32_n8(runs=6, steps=60, n_samples=2)
    for kw in (dict(), dict(precision="fp64"), dict(mode="plain")):
        a = D.Ensemble(w, checks=True, **kw).run()
        b = D.Ensemble(w, **kw).run()
        for t in range(2):
            assert np.array_equal(a.raw(t), b.raw(t)), kw
        a.close()
        b.close()
    w3 = W.plate3d(nx=24, ny=12, nz=12, plate=6, plate_x=8, ppc=6, runs=2, steps=8, n_samples=1)
    D.Ensemble(w3, checks=True).run().close()


def test_checks_catch_a_corrupted_pool(D):
    """A state holding ids at or above the run's next id (impossible in a
    run, where ids are handed out in order; set here through the test hook)
    fails the pool check after a step: it reports DSMC_E_STATE with the
    failing positions, and nothing faults."""
    from tests.helpers import box
    w = box(dim=2, ncell=(4, 4, 1), ppc=20, dt=1e-7, runs=1, steps=1, fill=0)
    rng = np.random.default_rng(3)
    n = 60
    d = w["L"][0] / 4
    x = np.zeros((n, 3))
    x[:, 0] = (1 + rng.uniform(0.1, 0.9, n)) * d
    x[:, 1] = (2 + rng.uniform(0.1, 0.9, n)) * d
    v = rng.normal(0.0, 1.0, (n, 3))
    ids = np.arange(n, dtype=np.uint32)
    ids[10:20] = n + 100                 # ten ids beyond the next id
    ens = D.Ensemble(w, precision="fp64", debug=True, checks=True, capacity_per_run=1024)
    ens.debug_begin(runs=1)
    ens.set_state(0, x, v, ids, n)
    with pytest.raises(D.DsmcError) as e:
        ens.debug_step(1)
    assert e.value.status == D.E_STATE and "consistency check failed" in str(e.value)
    ens.close()


def test_tune_cache_stores_then_loads_the_shape(D, tmp_path):
    """autotune="load": the first ensemble searches the launch shape and
    appends it to the cache file; a second context reads it back (no
    search) and gives bit-identical sums."""
    path = str(tmp_path / "shapes.txt")
    w = W.duct64x32_n8(runs=32, steps=120, n_samples=2)
    a = D.Ensemble(w, autotune="load", tune_cache=path).run()
    sa = a.stats()
    assert sa["tuned"] == 1
    lines = open(path).read().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 1
    b = D.Ensemble(w, autotune="load", tune_cache=path).run()
    sb = b.stats()
    assert sb["tuned"] == 2 and sb["shape"] == sa["shape"]
    for t in range(2):
        assert np.array_equal(a.raw(t), b.raw(t))
    assert len([ln for ln in open(path).read().split("\n") if ln.strip()]) == 1
    a.close()
    b.close()
