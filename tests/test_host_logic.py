"""Host-side logic without a GPU: the mixed-size ensemble's grouping and the
bench's algorithmic-byte accounting."""
import os
import sys

import numpy as np

from paper_cs_9902024_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_mixed_ensemble_groups_cover_every_run_once():
    m = W.mixed_n1024()
    assert m["runs"] == 1024
    start = 0
    sizes = []
    for g in m["groups"]:
        nx, ny = g["ncell"][0], g["ncell"][1]
        assert nx % 16 == 0 and 32 <= nx <= 512 and ny == nx // 2
        assert g["run0"] == start            # one consecutive range of global runs per grid
        start += g["runs"]
        sizes += [nx * ny] * g["runs"]
    assert start == 1024
    # grids in increasing size, each grid once
    nxs = [g["ncell"][0] for g in m["groups"]]
    assert nxs == sorted(set(nxs))
    # cell counts spread log-uniformly over about two and a half decades
    ls = np.log10(sizes)
    assert ls.min() < np.log10(32 * 16 * 4) and ls.max() > np.log10(512 * 256 / 4)
    q = np.quantile(ls, [0.25, 0.5, 0.75])
    mid = 0.5 * (np.log10(32 * 16) + np.log10(512 * 256))
    assert abs(q[1] - mid) < 0.25
    # the same draw every time
    m2 = W.mixed_n1024()
    assert [g["runs"] for g in m2["groups"]] == [g["runs"] for g in m["groups"]]


def test_algorithmic_bytes_split_between_tile_and_big_cell_kernels():
    sys.path.insert(0, ROOT)
    import bench
    w = W.duct64x32_n8()
    st = {"particle_steps": 1000, "generated": 100, "pool_steps": 1200, "big_pool_steps": 300,
          "collisions": 50}
    a = bench.algorithmic_bytes(w, st, steps=10, runs=8)
    gather = 8 + 2 * (2 * 4 + 3 * 4) + 8
    cells = 8 * 64 * 32
    assert a["cell"] == (1200 - 300) * gather + cells * 10 * 4
    assert a["cell_big"] == 300 * gather
    assert a["move"] == 900 * (3 * 2 * 4 + 12)
    assert a["scatter"] == 1200 * 20
    st0 = dict(st, big_pool_steps=0)
    a0 = bench.algorithmic_bytes(w, st0, steps=10, runs=8)
    assert a0["cell"] + a0["cell_big"] == a["cell"] + a["cell_big"]
