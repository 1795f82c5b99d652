"""Run sharding across processes (CPU, gloo, world size 2): two ranks that
each run half of an ensemble with their global run offsets, then sum their
group sums, reproduce the one-process ensemble exactly."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from oracle import run_ensemble
from paper_cs_9902024_gb300 import shard
from paper_cs_9902024_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_equal_one_process(tmp_path):
    out = str(tmp_path / "acc.npy")
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-m", "tests.shard_worker", "--rank", str(r),
                               "--world", "2", "--port", str(port), "--per", "16", "--out", out],
                              cwd=ROOT) for r in range(2)]
    for p in procs:
        assert p.wait(timeout=300) == 0
    got = np.load(out)
    w = W.duct64x32_n8(steps=40, n_samples=2)
    ref, st = run_ensemble(w, runs=32, threads=4)
    # group g holds global runs g and g + 16 on both sides: the same two
    # addends, so the sums agree bit for bit
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)
    with open(out + ".ps") as f:
        assert int(f.read()) == st["particle_steps"]


def test_shard_arithmetic():
    assert shard.run_offset(3, 512) == 1536
    assert shard.groups(512, 8) == 16
    assert shard.groups(5, 1) == 5
    with pytest.raises(ValueError):
        shard.groups(8, 2)
