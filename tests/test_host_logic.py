"""Host-side logic without a GPU: the mixed-size ensemble's grouping and the
bench's algorithmic-byte accounting."""
import os
import json
import sys

import numpy as np
import pytest

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
    method, layout = bench.algorithmic_bytes(w, st, steps=10, runs=8)
    # the method's bytes per particle-step (2-D): Motion 28, Indexing 60 (12
    # scatter + 48 permute), Interaction 16
    assert method["move"] == 900 * 28
    assert method["scatter"] == 1200 * 12
    assert method["cell"] == 900 * 48 and method["cell_big"] == 300 * 48
    assert method["scatter"] + method["cell"] + method["cell_big"] == 1200 * 60
    assert method["collide"] + method["collide_big"] == 1200 * 16
    # the implementation's layout bytes
    # LCR slot 4; gather offsets 8, v 12; write offsets 8, key 4, v 12
    gather = 4 + (2 * 4 + 3 * 4) + (2 * 4 + 3 * 4 + 4)
    cells = 8 * 64 * 32
    assert layout["cell"] == (1200 - 300) * gather + cells * 10 * 4
    assert layout["cell_big"] == 300 * gather
    assert layout["move"] == 900 * (3 * 2 * 4 + 8)
    assert layout["scatter"] == 1200 * 8      # read the key, write the slot
    st0 = dict(st, big_pool_steps=0)
    m0, l0 = bench.algorithmic_bytes(w, st0, steps=10, runs=8)
    assert l0["cell"] + l0["cell_big"] == layout["cell"] + layout["cell_big"]
    assert m0["cell"] + m0["cell_big"] == method["cell"] + method["cell_big"]
    # 3-D: Motion 40, permute 56
    w3 = W.plate3d(nx=8, ny=4, nz=4, runs=1)
    m3, _ = bench.algorithmic_bytes(w3, st0, steps=10, runs=1)
    assert m3["move"] == 900 * 40 and m3["cell"] == 1200 * 56


def test_partner_variant_bytes_and_traffic_family(tmp_path):
    """A positional partner choice adds one read of every particle's
    position to Interaction (8 B in 2-D, 12 in 3-D); its traffic entry is a
    family of its own, so the uniform choice's DRAM counters never stand in
    for it."""
    sys.path.insert(0, ROOT)
    import bench
    st = {"particle_steps": 1000, "generated": 100, "pool_steps": 1200, "big_pool_steps": 300,
          "collisions": 50}
    w = W.duct64x32_n8()
    mu, lu = bench.algorithmic_bytes(w, st, steps=10, runs=8)
    for scheme in ("subcell", "nearest"):
        wp = W.with_partner(w, scheme, 2)
        mp, lp = bench.algorithmic_bytes(wp, st, steps=10, runs=8)
        assert mp["collide"] + mp["collide_big"] == 1200 * (16 + 8)
        assert lp["collide"] - lu["collide"] == 900 * 8
        assert lp["collide_big"] - lu["collide_big"] == 300 * 8
        assert mp["cell"] == mu["cell"] and lp["move"] == lu["move"]
    w3 = W.with_partner(W.plate3d(nx=8, ny=4, nz=4, runs=1), "nearest")
    m3, _ = bench.algorithmic_bytes(w3, dict(st, big_pool_steps=0), steps=10, runs=1)
    assert m3["collide"] == 1200 * (16 + 12)
    # the traffic of the uniform family is not used for a variant
    tj = tmp_path / "traffic.json"
    tj.write_text(json.dumps({"duct64x32": {"cell": {"kernel_hash": "h", "dram_bytes": 4.0e6,
                                                     "particles": 1.0e5}}}))
    prs = {"pool_steps": 2000, "big_pool_steps": 0, "launches_kernel": {"cell": 10}}
    assert bench.traffic_per_launch("duct64x32_n512", "cell", prs, path=str(tj),
                                    khash="h") == pytest.approx(40.0 * 2000 / 10)
    assert bench.traffic_per_launch("duct64x32_n512", "cell", prs, path=str(tj), khash="h",
                                    partner="nearest") is None


def test_sample_windows_end_at_the_sample_times():
    sys.path.insert(0, ROOT)
    import bench
    w = W.duct64x32_n512()
    assert bench.sample_windows(w, 1) is None
    win = bench.sample_windows(w, 25)
    assert [b for _, b in win] == w["sample_steps"]
    assert all(b - a + 1 == 25 for a, b in win)
    assert len(bench.sample_windows(w, 50)) == 8       # 50-step gaps: just disjoint
    with pytest.raises(SystemExit):
        bench.sample_windows(w, 51)


def test_with_partner_keeps_the_workload():
    w = W.duct64x32_n512()
    for scheme, code in (("uniform", 0), ("subcell", 1), ("nearest", 2)):
        wp = W.with_partner(w, scheme, n_sub=3)
        assert wp["gas"]["partner"] == code
        assert wp["gas"]["n_sub"] == (3 if scheme == "subcell" else 1)
        for k in ("dim", "ncell", "L", "bcs", "runs", "steps", "dt", "sample_steps", "seed"):
            assert wp[k] == w[k], k
        for k in ("mass", "d_ref", "T_ref", "omega", "F_N"):
            assert wp["gas"][k] == w["gas"][k]
        assert (wp["name"] == w["name"]) == (scheme == "uniform")
    assert "partner" not in w["gas"]


def test_method_rows_are_bytes_over_summed_kernel_time():
    sys.path.insert(0, ROOT)
    import bench
    method = {"move": 28e9, "scatter": 12e9, "cell": 48e9, "cell_big": 0, "scan": 0,
              "collide": 16e9, "collide_big": 0}
    ms = {"move": 10.0, "scan": 1.0, "scatter": 4.0, "cell": 15.0, "collide": 8.0}
    rows = bench.method_rows(method, ms, peak=4000.0)
    assert abs(rows["motion"]["achieved_gbs"] - 2800.0) < 1e-6
    assert abs(rows["indexing"]["achieved_gbs"] - 60e9 / 0.020 / 1e9) < 1e-6
    assert abs(rows["interaction"]["frac"] - 2000.0 / 4000.0) < 1e-12


def test_traffic_scales_the_captured_bytes_per_particle(tmp_path):
    """The bench's DRAM traffic per launch: the captured bytes per particle
    of the same workload family times the particles the kernel processed per
    launch (tile kernels: cells up to 128 particles; big-cell kernels: the
    rest); nothing when the family, the kernel or the device-code hash does
    not match."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    path = tmp_path / "traffic.json"
    json.dump({"duct64x32": {"cell": {"kernel_hash": "abc", "dram_bytes": 4.0e8, "particles": 1.0e7},
                             "cell_big": {"kernel_hash": "abc", "dram_bytes": 6.0e8, "particles": 1.0e7}}},
              open(path, "w"))
    prs = {"pool_steps": 1000, "big_pool_steps": 200, "launches_kernel": {"cell": 10, "cell_big": 5}}
    t = bench.traffic_per_launch("duct64x32_n512", "cell", prs, path=str(path), khash="abc")
    assert t == 40.0 * 800 / 10
    t = bench.traffic_per_launch("duct64x32_n8", "cell_big", prs, path=str(path), khash="abc")
    assert t == 60.0 * 200 / 5
    assert bench.traffic_per_launch("duct64x32_n512", "cell", prs, path=str(path), khash="xyz") is None
    assert bench.traffic_per_launch("jet256x128_n64", "cell", prs, path=str(path), khash="abc") is None
    assert bench.traffic_per_launch("duct64x32_n512", "move", prs, path=str(path), khash="abc") is None
