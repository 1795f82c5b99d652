"""One rank of the two-process sharding test (run as a module under the
gloo backend; CPU only).  Each rank runs its share of the ensemble through
the oracle with its global run offset, and the group sums are reduced with
the same helper bench.py uses across GPUs."""
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
    a = p.parse_args()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(a.port)
    dist.init_process_group("gloo", rank=a.rank, world_size=a.world)
    w = W.duct64x32_n8(steps=40, n_samples=2)
    G = shard.groups(a.per, a.world)
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
