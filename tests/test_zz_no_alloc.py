"""The no-allocation entry point (dsmc_run_ensemble_noalloc) against the
allocating one (dsmc_run_ensemble + dsmc_get_samples), through the C ABI.

Some callers cannot allocate device memory when they want a result: their
device memory was handed to another allocator or a fixed budget up front, or
they run a real-time loop where cudaMalloc/cudaFree (which can synchronise
the device) are forbidden.  The no-allocation path runs the same kernels inside a
fixed scratch array in the library's device image.  Its group sums must equal
the allocating path's exactly (same kernels, same draws, same order), on two
calls in a row (the scratch keeps the previous call's contents, so the second
call checks that everything that must start from zero is reset)."""
import numpy as np
import pytest

from paper_cs_9902024_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc
    return dsmc


def test_noalloc_matches_allocating_run_twice(D):
    w = W.duct64x32_n8(runs=6, steps=80, n_samples=4)
    ref_ens = D.Ensemble(w).run()
    ref = np.stack([ref_ens.raw(t) for t in range(len(w["sample_steps"]))])
    ref_stats = ref_ens.stats()
    ref_ens.close()
    ens = D.Ensemble(w, torch_memory=False)
    for _ in range(2):
        out = ens.run_noalloc()
        assert out.shape == ref.shape
        # tolerance of the allocating path's own mode tests: bit-identical
        assert np.array_equal(out, ref)
        st = ens.stats()
        for k in ("particle_steps", "generated", "removed", "candidates", "collisions"):
            assert st[k] == ref_stats[k], k
    ens.close()


def test_noalloc_rejects_oversized_problem_and_used_context(D):
    big = W.duct64x32_n512()
    ens = D.Ensemble(big, torch_memory=False)
    with pytest.raises(D.DsmcError) as ex:
        ens.run_noalloc()
    assert ex.value.status == D.E_INVALID
    assert "bytes of device scratch" in str(ex.value)
    ens.close()
    w = W.duct64x32_n8(runs=2, steps=10, n_samples=1)
    used = D.Ensemble(w, torch_memory=False).run()
    with pytest.raises(D.DsmcError) as ex:
        used.run_noalloc()
    assert ex.value.status == D.E_STATE
    used.close()
