"""The mixed-size ensemble (runs on different grids, grouped by grid into
concurrent batched contexts) against the oracle (GPU)."""
import os

import numpy as np
import pytest

from oracle import run_ensemble
from paper_cs_9902024_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc
    return dsmc


def _small():
    return W.mixed(n_runs=40, cells_hi=96 * 48, steps=80, n_samples=2)


def test_mixed_fp64_group_sums_equal_oracle(D):
    """FP64 device state: every grid's group sums equal the oracle's for
    the same global runs (counts exactly, moments to 1e-9)."""
    m = _small()
    assert len(m["groups"]) >= 3
    me = D.MixedEnsemble(m, precision="fp64").run()
    for gi, w in enumerate(m["groups"]):
        G = min(w["runs"], 16)
        acc, st = run_ensemble(w, runs=w["runs"], run0=w["run0"], groups=G,
                               threads=min(os.cpu_count() or 1, 16))
        for t in range(len(w["sample_steps"])):
            raw = me.raw(gi, t)
            assert np.array_equal(raw[..., 0], acc[t][..., 0]), (gi, t)
            assert np.allclose(raw, acc[t], rtol=1e-9, atol=1e-6), (gi, t)
        assert me.parts[gi].stats()["collisions"] == st["collisions"]
    me.close()


def test_mixed_full_size_fp32_conserves_particles(D):
    """The 1024-run mixed ensemble (grids 32x16 .. 512x256, 300 steps) in
    FP32: no device error, and in every group the particles left equal the
    entrants minus the leavers (the duct starts empty)."""
    m = W.mixed_n1024()
    me = D.MixedEnsemble(m).run()
    st = me.stats()
    assert st["error_word"] == 0
    for s in st["groups"]:
        assert s["particles_now"] == s["generated"] - s["removed"]
    print("mixed 1024-run ensemble: %d groups, %.3e particle-steps, %d particles at the end"
          % (len(m["groups"]), st["particle_steps"], st["particles_now"]))
    me.close()
