"""Failure paths made on the host or by a bounded wait (GPU): an allocator
that refuses memory, particles that hit the per-step surface-event limit, a
bulk-copy wait that runs out.  None of them faults or hangs the device; each
is reported through a status or a counter and the context stays usable."""
import ctypes as C

import numpy as np
import pytest

from oracle import Oracle
from paper_cs_9902024_gb300 import workloads as W
from tests.helpers import box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc
    return dsmc


def test_allocator_refusal_reports_oom(D):
    """An allocation callback that returns NULL: dsmc_run_ensemble returns
    DSMC_E_OOM, frees what it got, and the same context then runs with an
    allocator that works."""
    import torch
    lib = D.load_library()
    w = W.duct64x32_n8(runs=2, steps=10, n_samples=1)
    dom, cells, gas, arr, nb = D._structs(w)
    held = {}
    state = {"refuse": True}

    def _alloc(nbytes, user, strm):
        if state["refuse"]:
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        held[t.data_ptr()] = t
        return t.data_ptr()

    def _free(p, nbytes, user, strm):
        held.pop(p, None)

    acb, fcb = D.ALLOC_FN(_alloc), D.FREE_FN(_free)
    opt = D.Options(struct_size=C.sizeof(D.Options))
    opt.alloc, opt.free = acb, fcb
    opt.use_graph = 1
    h = C.c_void_p()
    assert lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(gas), arr, nb, C.byref(opt),
                           C.byref(h)) == D.OK
    ss = np.array(w["sample_steps"], dtype=np.int32)
    args = (h, w["runs"], w["dt"], w["steps"], ss.ctypes.data_as(C.POINTER(C.c_int32)), len(ss),
            w["seed"])
    assert lib.dsmc_run_ensemble(*args) == D.E_OOM
    assert not held
    state["refuse"] = False
    assert lib.dsmc_run_ensemble(*args) == D.OK
    lib.dsmc_destroy(h)
    assert not held


def test_surface_event_limit_counted_like_the_oracle(D):
    """A specular box crossed many times per step: flights stop at the 16th
    surface event of a step (counted), on the device exactly as in the
    oracle (FP64 state), and the run completes."""
    w = box(dim=2, ncell=(4, 4, 1), ppc=2, dt=3e-3, runs=2, steps=3)
    ens = D.Ensemble(w, precision="fp64", debug=True)
    ens.debug_begin(runs=2)
    orc = Oracle(w, runs=2)
    for r in range(2):
        orc.init_run(r)
    ens.debug_step(3)
    for s in range(1, 4):
        for r in range(2):
            orc.step(r, s)
    st = ens.stats()
    so = [orc.stats(r) for r in range(2)]
    assert st["bounce_limit"] > 0
    assert st["bounce_limit"] == sum(s["bounce_limit"] for s in so)
    for r in range(2):
        x, v, ids = ens.get_state(r)
        xo, vo, io = orc.get_state(r)
        assert np.array_equal(ids, io)
        assert np.allclose(x, xo, rtol=0, atol=1e-12 * max(w["L"]))


def test_bounded_wait_timeout_reported(D):
    """A bulk-copy barrier that nothing completes: the wait gives up after
    its poll limit, DSMC_E_TIMEOUT comes back, and the context still runs."""
    w = W.duct64x32_n8(runs=2, steps=5, n_samples=1)
    ens = D.Ensemble(w, debug=True)
    ens.debug_begin(runs=2)
    assert ens.debug_timeout_probe(256) == D.E_TIMEOUT
    assert "bounded wait" in D.load_library().dsmc_last_error(ens.h).decode()
    ens.debug_step(2)
    ens.close()
    ok = D.Ensemble(w).run()
    assert ok.stats()["error_word"] == 0


def test_cell_over_the_limit_reported_not_faulted(D):
    """Cells of ~9000 particles (above the 8192 per-cell limit) in FP32 and
    FP64: the run returns DSMC_E_CAPACITY (BIGCELL), every particle is still
    carried into the next pool, and nothing faults."""
    for prec in ("fp32", "fp64"):
        w = box(dim=2, ncell=(2, 2, 1), ppc=9000, dt=1e-6, runs=1, steps=2)
        ens = D.Ensemble(w, precision=prec)
        with pytest.raises(D.DsmcError) as ex:
            ens.run()
        assert ex.value.status == D.E_CAPACITY
        assert ens.stats()["error_word"] & 0x4
        assert ens.stats()["particles_now"] > 30000
        ens.close()
