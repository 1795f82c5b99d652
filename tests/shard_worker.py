"""One rank of the two-process sharding tests (run as a module under the
gloo backend).  Each rank runs its share of the ensemble with its global
run offset -- through the oracle on the CPU, or (--gpu fp32|fp64) through
the library on the device -- and the group sums are reduced over the ranks
on the host with the same helper bench.py uses across GPUs."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch.distributed as dist  # noqa: E402

from oracle import run_ensemble  # noqa: E402
from paper_cs_9902024_gb300 import shard  # noqa: E402
from paper_cs_9902024_gb300 import workloads as W  # noqa: E402


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--rank", type=int, required=True)
    p.add_argument("--world", type=int, required=True)
    p.add_argument("--port", type=int, required=True)
    p.add_argument("--per", type=int, default=16)
    p.add_argument("--out", required=True)
    p.add_argument("--gpu", default=None, choices=[None, "fp32", "fp64"])
    a = p.parse_args()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(a.port)
    dist.init_process_group("gloo", rank=a.rank, world_size=a.world)
    w = W.duct64x32_n8(steps=40, n_samples=2)
    G = shard.groups(a.per, a.world)
    if a.gpu:
        # the device ensemble of this rank's runs (both ranks share the one
        # GPU of a test box: independent ensembles, nothing waits across them)
        import __graft_entry__ as g
        g.build()
        from paper_cs_9902024_gb300.dsmc import Ensemble
        ens = Ensemble(w, precision=a.gpu, run_offset=shard.run_offset(a.rank, a.per))
        ens.run(runs=a.per)
        acc = np.stack([ens.raw(t) for t in range(len(w["sample_steps"]))])
        st = ens.stats()
        ens.close()
    else:
        acc, st = run_ensemble(w, runs=a.per, run0=shard.run_offset(a.rank, a.per), groups=G)
    tot = shard.allreduce_group_sums(acc)
    ps = shard.allreduce_sum(st["particle_steps"])
    if a.rank == 0:
        np.save(a.out, tot)
        with open(a.out + ".ps", "w") as f:
            f.write("%d\n" % int(ps))
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
