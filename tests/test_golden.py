"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle only): the oracle must keep reproducing them exactly, and the FP64
device path must reproduce them (counts exactly, moment sums to 1e-9)."""
import os

import numpy as np
import pytest

from oracle import run_ensemble
from tests.golden.make_golden import golden_workload

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load():
    tot, counts, scal = {}, None, {}
    with open(os.path.join(HERE, "duct16x8_r3_s30.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            if p[0] == "totals":
                tot[(int(p[1]), int(p[2]))] = np.array([float(x) for x in p[3:]])
            elif p[0] == "counts":
                counts = np.array([int(x) for x in p[3:]])
            else:
                scal[p[0]] = int(p[1])
    return tot, counts, scal


def _check(acc, tol):
    tot, counts, _ = _load()
    for (t, g), v in tot.items():
        got = acc[t, g].sum(axis=0)
        assert got[0] == v[0]
        assert np.allclose(got, v, rtol=tol, atol=0), (t, g)
    assert np.array_equal(acc[1, 0, :, 0].astype(np.int64), counts)


def test_oracle_reproduces_golden():
    w = golden_workload()
    acc, st = run_ensemble(w, threads=1)
    _check(acc, 0.0)
    _, _, scal = _load()
    assert st["particle_steps"] == scal["particle_steps"]
    assert st["collisions"] == scal["collisions"]


@pytest.mark.gpu
def test_fp64_device_reproduces_golden():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc
    w = golden_workload()
    ens = dsmc.Ensemble(w, precision="fp64").run()
    acc = np.stack([ens.raw(t) for t in range(len(w["sample_steps"]))])
    _check(acc, 1e-9)
    _, _, scal = _load()
    st = ens.stats()
    assert st["particle_steps"] == scal["particle_steps"]
    assert st["collisions"] == scal["collisions"]
