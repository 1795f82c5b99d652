"""FP64 CPU oracle for the ensemble DSMC step (test infrastructure only).

Only tests/, the smoke check and bench.py's CPU-baseline leg import this
package.  It is independent of the CUDA path: it shares no code with it and
never calls it.
"""
from .oracle import (Oracle, build_oracle, oracle_lib, run_ensemble, philox,
                     draw, inflow_flux, sample_xi, sigma_cr, scatter,
                     partner, macro_from_acc, NMOM)

__all__ = ["Oracle", "build_oracle", "oracle_lib", "run_ensemble", "philox",
           "draw", "inflow_flux", "sample_xi", "sigma_cr", "scatter",
           "partner", "macro_from_acc", "NMOM"]
