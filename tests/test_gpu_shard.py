"""Run sharding on the device (GPU): two processes, each with its own device
context holding 16 runs at global run offsets 0 and 16, summed over the two
ranks with the host reduction bench.py uses (gloo), equal one 32-run device
context bit for bit, in FP32 and in FP64 state.  Group g holds global runs
g and g + 16 on both sides, added in the same order, and every run's draws
depend only on its global index (the independent-runs level of the paper,
Sec. 1.3: one exchange after all runs)."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_cs_9902024_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_two_device_shards_equal_one_context(tmp_path, precision):
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300.dsmc import Ensemble
    out = str(tmp_path / "acc.npy")
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-m", "tests.shard_worker", "--rank", str(r),
                               "--world", "2", "--port", str(port), "--per", "16", "--out", out,
                               "--gpu", precision], cwd=ROOT) for r in range(2)]
    for p in procs:
        assert p.wait(timeout=600) == 0
    got = np.load(out)
    w = W.duct64x32_n8(steps=40, n_samples=2)
    ens = Ensemble(w, precision=precision).run(runs=32)
    ref = np.stack([ens.raw(t) for t in range(len(w["sample_steps"]))])
    st = ens.stats()
    ens.close()
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)
    with open(out + ".ps") as f:
        assert int(f.read()) == st["particle_steps"]
