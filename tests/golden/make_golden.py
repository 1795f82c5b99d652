"""Writes the stored expected values under tests/golden/ by calling only the
oracle (oracle/), never the CUDA path.

    python tests/golden/make_golden.py

duct16x8_r3_s30.txt: a 16x8 cell version of the duct workload (impulsively
started drifting-Maxwellian inflow, diffuse walls, outflow; the unsteady
problem class of Sec. 1.1), 3 runs, 30 steps, samples after steps 15 and
30, Philox seed 1.  Stored: per sample and group the cell totals of the 7
moments (N, sum v_a, sum v_a^2), and the per-cell particle counts of sample
1, group 0.  A later change to the oracle's arithmetic that moves these
values must name, in its commit message, the passage of the paper (or the
reading of it) that justifies it.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import run_ensemble  # noqa: E402
from paper_cs_9902024_gb300 import workloads as W  # noqa: E402


def golden_workload():
    return W.duct(nx=16, ny=8, runs=3, steps=30, n_samples=2, seed=1, name="duct16x8_r3_s30")


def main():
    w = golden_workload()
    acc, st = run_ensemble(w, threads=1)
    lines = ["# duct16x8_r3_s30: oracle group sums (see make_golden.py)",
             "# totals: sample group m0..m6 (cell sums of N, sum v_a, sum v_a^2)"]
    T, G = acc.shape[0], acc.shape[1]
    for t in range(T):
        for g in range(G):
            tot = acc[t, g].sum(axis=0)
            lines.append("totals %d %d %s" % (t, g, " ".join(repr(float(x)) for x in tot)))
    lines.append("counts 1 0 " + " ".join(str(int(x)) for x in acc[1, 0, :, 0]))
    lines.append("particle_steps %d" % st["particle_steps"])
    lines.append("collisions %d" % st["collisions"])
    with open(os.path.join(HERE, "duct16x8_r3_s30.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
