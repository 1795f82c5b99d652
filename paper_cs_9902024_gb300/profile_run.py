"""Run one workload's ensemble with direct launches (no CUDA graphs, default
launch shapes), for a profiler to capture chosen launches of it.

    python -m paper_cs_9902024_gb300.profile_run duct 256 301
    python -m paper_cs_9902024_gb300.profile_run duct 256 301 760,2432,3072,1216
    python -m paper_cs_9902024_gb300.profile_run jet 8 60
    python -m paper_cs_9902024_gb300.profile_run duct 256 101 0,0,0,0 nearest

Arguments: workload (duct: the 64x32 channel, HS, its 8 sample times; jet:
the 256x128 pulsed jet, VHS; plate: the 128x64x64 box with a plate; mixed:
runs on grids of 32x16 to 256x128 cells; the last three with 2 sample
times), runs, steps, and optionally a launch shape (move CTAs, scatter
CTAs, sort/gather tile budget, collision CTAs; 0 keeps a default) and the
choice of collision partner (uniform, subcell: 2 per axis, nearest; not for
mixed).  Each step launches the step's kernels once, in
a fixed order, so the n-th launch of a kernel is its n-th step.  Prints the
particle-steps done and the device error word (non-zero exit if set)."""
import sys

from . import workloads as W
from .dsmc import Ensemble, MixedEnsemble


def main(argv):
    name = argv[0] if argv else "duct"
    runs = int(argv[1]) if len(argv) > 1 else 256
    steps = int(argv[2]) if len(argv) > 2 else 301
    shape = None
    if len(argv) > 3:
        from .dsmc import SHAPE_KEYS
        shape = dict(zip(SHAPE_KEYS, (int(v) for v in argv[3].split(","))))
        if not any(shape.values()):
            shape = None
    partner = argv[4] if len(argv) > 4 else "uniform"
    if name == "mixed":
        m = W.mixed(grids=[(32, runs), (64, runs), (128, runs), (256, runs)], steps=steps,
                    n_samples=2)
        e = MixedEnsemble(m, use_graph=False, shape=shape).run()
        st, err = e.stats(), e.mixed_stats()["error_word"]
    else:
        if name == "duct":
            w = W.duct64x32_n512(runs=runs, steps=steps)
        else:
            make = {"jet": W.jet256x128_n64, "plate": W.plate128x64x64_n16}[name]
            w = make(runs=runs, steps=steps, n_samples=2)
        w = W.with_partner(w, partner, 2)
        e = Ensemble(w, use_graph=False, shape=shape).run()
        st = e.stats()
        err = st["error_word"]
    print("%s: %d runs x %d steps, particle_steps %d, pool_steps %d (in cells above 128: %d), "
          "particles now %d, error word %d, shape %s" % (
              name, runs, steps, st["particle_steps"], st["pool_steps"],
              st.get("big_pool_steps", 0), st["particles_now"], err,
              st.get("shape", e.parts[0].stats()["shape"] if name == "mixed" else None)))
    e.close()
    return 1 if err else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
