"""The mixed-size ensemble (runs on grids of different sizes, one part per
grid) against the oracle and against each part run alone (GPU).

The single-launch form (dsmc_mixed_run: one launch per kernel kind per step
over every part, CTAs claiming (part, tile) items from device counters) must
give every part exactly what dsmc_run_ensemble gives it alone; in FP64 state
every part's group sums must equal the oracle's; in FP32 state the
ensemble-averaged density, velocity and temperature must lie within 3
combined standard errors of the FP64 oracle's, with the relative error of
each precision reported (the precision sweep of the mixed-size workload)."""
import os

import numpy as np
import pytest

from oracle import macro_from_acc, run_ensemble
from paper_cs_9902024_gb300 import workloads as W
from tests.parity import zscores

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc
    return dsmc


def _threads():
    return min(os.cpu_count() or 1, 16)


def test_single_launch_equals_each_part_alone(D):
    """Single-launch mixed ensemble (graphs, FP32) vs each part's own
    batched dsmc_run_ensemble: group sums and counters bit-identical; the
    same with direct launches and with profiling."""
    m = W.mixed(grids=[(32, 3), (48, 2), (64, 5), (96, 2)], steps=40, n_samples=2)
    me = D.MixedEnsemble(m).run()
    T = len(m["groups"][0]["sample_steps"])
    for gi, w in enumerate(m["groups"]):
        alone = D.Ensemble(w, run_offset=w["run0"]).run()
        for t in range(T):
            assert np.array_equal(me.raw(gi, t), alone.raw(t)), (gi, t)
        sa, sm = alone.stats(), me.parts[gi].stats()
        for k in ("particle_steps", "generated", "removed", "wall_hits", "candidates",
                  "collisions", "particles_now", "pool_steps"):
            assert sa[k] == sm[k], (gi, k)
        alone.close()
    st = me.mixed_stats()
    assert st["error_word"] == 0 and st["particle_steps"] == me.stats()["particle_steps"]
    ref = [[me.raw(gi, t) for t in range(T)] for gi in range(len(m["groups"]))]
    me.close()
    for kw in (dict(use_graph=False), dict(profile=True)):
        me2 = D.MixedEnsemble(m, **kw).run()
        for gi in range(len(m["groups"])):
            for t in range(T):
                assert np.array_equal(me2.raw(gi, t), ref[gi][t]), (kw, gi, t)
        if kw.get("profile"):
            ms = me2.mixed_stats()["ms_kernel"]
            assert ms["move"] > 0 and ms["cell"] > 0 and ms["collide"] > 0
        me2.close()


def _sweep_mix():
    # one grid of 256 x 128 cells (~655k particles per run), filled
    return W.mixed(grids=[(32, 16), (64, 16), (128, 16), (256, 16)], steps=60, n_samples=2)


def test_mixed_precision_sweep_against_the_oracle(D):
    """FP64 and FP32 device state on a filled mini-mix with a 256 x 128 grid,
    each against the FP64 oracle of the same global runs: FP64 group sums
    exact (counts) and to 1e-9 (moments); FP32 within 3 combined standard
    errors for >= 99% of (sample, cell, quantity) comparisons in cells with
    >= 40 sampled particles.  The median relative error of the density of
    each precision is printed."""
    m = _sweep_mix()
    assert max(w["ncell"][0] for w in m["groups"]) >= 256
    me64 = D.MixedEnsemble(m, precision="fp64").run()
    me32 = D.MixedEnsemble(m, precision="fp32").run()
    zall, excl = [], 0
    for gi, w in enumerate(m["groups"]):
        G = min(w["runs"], 16)
        acc, st = run_ensemble(w, runs=w["runs"], run0=w["run0"], groups=G, threads=_threads())
        T = len(w["sample_steps"])
        r64 = np.stack([me64.raw(gi, t) for t in range(T)])
        assert np.array_equal(r64[..., 0], acc[..., 0]), gi
        assert np.allclose(r64, acc, rtol=1e-9, atol=1e-6), gi
        assert me64.parts[gi].stats()["collisions"] == st["collisions"]
        mo = macro_from_acc(acc, w, w["runs"])
        mg = {k: np.stack([me32.macro(gi, t)[k] for t in range(T)]) for k in mo}
        m64 = {k: np.stack([me64.macro(gi, t)[k] for t in range(T)]) for k in mo}
        r32 = np.stack([me32.raw(gi, t) for t in range(T)])
        mask = np.minimum(r32[..., 0].sum(1), acc[..., 0].sum(1)) >= 40
        z, e = zscores(mg, mo, mask)
        zall.append(z)
        excl += e
        rel32 = np.nanmedian(np.abs(mg["density"][mask] / mo["density"][mask] - 1))
        rel64 = np.nanmax(np.abs(m64["density"][mask] / mo["density"][mask] - 1))
        print("mixed %dx%d, %d runs: fp64 max rel. density error %.1e; fp32 median rel. density "
              "error %.2e, |z|>3 fraction %.4f of %d" % (w["ncell"][0], w["ncell"][1], w["runs"],
                                                          rel64, rel32, np.mean(np.abs(z) > 3),
                                                          z.size))
    z = np.concatenate(zall)
    assert z.size > 20000
    assert excl <= 0.01 * z.size
    assert np.mean(np.abs(z) > 3) < 0.01
    me64.close()
    me32.close()


def test_mixed_full_size_fp32(D):
    """The 1024-run mixed ensemble (grids 32x16 .. 512x256 drawn
    log-uniformly, filled, 300 steps, one launch per kernel kind per step)
    in FP32: no device error, and in every part the particles left equal
    the fill plus the entrants minus the leavers."""
    m = W.mixed_n1024()
    me = D.MixedEnsemble(m)
    me.run(steps=0, sample_steps=[])
    fill = [s["particles_now"] for s in me.stats()["groups"]]
    me.run()
    st = me.stats()
    assert st["error_word"] == 0
    for f, s in zip(fill, st["groups"]):
        assert s["particles_now"] == f + s["generated"] - s["removed"]
    per_run = [f / w["runs"] for f, w in zip(fill, m["groups"])]
    ms = me.mixed_stats()["ms_steps"]
    print("mixed 1024-run ensemble: %d parts, %.3e particle-steps in %.1f ms (%.3e /s); "
          "%.3g to %.3g particles per run at the start"
          % (len(m["groups"]), st["particle_steps"], ms, st["particle_steps"] / (ms / 1e3),
             min(per_run), max(per_run)))
    assert min(per_run) < 15000 and max(per_run) > 2_000_000
    me.close()
