"""Pins of the oracle's random-number layer (CPU).

Philox4x32-10 is a published generator; here it is checked for the
properties its construction fixes (a counter bijection with full avalanche)
and for the statistics the DSMC draws rely on.  Its bit-for-bit definition is
cross-checked on the GPU against cuRAND's Philox4_32_10 (test_gpu_rng.py)."""
import numpy as np
import pytest
from scipy import stats

from oracle import philox, draw


def _bits(x):
    return np.unpackbits(np.asarray(x, dtype=">u4").view(np.uint8)).sum()


def test_u01_open_interval_and_binary32_exact():
    us = np.array([draw(1, r, s, e, 6, k) for r in range(3) for s in range(5)
                   for e in range(20) for k in range(4)]).ravel()
    assert np.all(us > 0.0) and np.all(us < 1.0)
    # every uniform is (m + 1/2) / 2^23 with integer m: exact in binary32
    assert np.all(us.astype(np.float32).astype(np.float64) == us)
    m = us * 2.0 ** 23 - 0.5
    assert np.all(m == np.floor(m))


def test_philox_avalanche():
    """Flipping any one bit of the counter or key changes about half of the
    128 output bits (a dropped xor or a round missing would not)."""
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(40):
        ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        base = philox(ctr, key)
        for word in range(6):
            for bit in (0, 13, 31):
                c2, k2 = ctr.copy(), key.copy()
                if word < 4:
                    c2[word] ^= np.uint32(1 << bit)
                else:
                    k2[word - 4] ^= np.uint32(1 << bit)
                out = philox(c2, k2)
                flips.append(_bits(np.bitwise_xor(base, out)))
    flips = np.array(flips)
    assert 60 < flips.mean() < 68
    assert flips.min() > 30


def test_philox_uniform_and_uncorrelated():
    u = np.array([draw(3, 0, 1, e, 5, 0) for e in range(20000)])
    flat = u.ravel()
    assert abs(flat.mean() - 0.5) < 4 * np.sqrt(1 / 12 / flat.size)
    assert abs(flat.var() - 1 / 12) < 0.003
    hist, _ = np.histogram(flat, bins=64, range=(0, 1))
    chi2 = stats.chisquare(hist)
    assert chi2.pvalue > 1e-4
    # the four lanes of one draw and consecutive entities are uncorrelated
    c = np.corrcoef(u.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.03
    assert abs(np.corrcoef(flat[:-1], flat[1:])[0, 1]) < 0.02


def test_runs_steps_purposes_give_distinct_streams():
    """The run index shifts the stream (the paper's per-run RNG shift,
    Sec. 1.1): different run / step / purpose / sub never repeat a block."""
    seen = set()
    for run in range(4):
        for step in range(4):
            for purpose in range(1, 7):
                for sub in range(3):
                    for e in range(3):
                        seen.add(tuple(draw(11, run, step, e, purpose, sub)))
    assert len(seen) == 4 * 4 * 6 * 3 * 3


def test_box_muller_gaussian_via_fill():
    """Velocities of a filled box are N(U, kT/m) per component."""
    from oracle import Oracle
    from tests.helpers import box
    w = box(dim=3, ncell=(6, 6, 6), ppc=200, fill_U=(100.0, -50.0, 0.0), fill_T=250.0)
    o = Oracle(w, runs=1)
    o.init_run(0)
    _, v, _ = o.get_state(0)
    sd = np.sqrt(1.380649e-23 * 250.0 / w["gas"]["mass"])
    for a, U in enumerate((100.0, -50.0, 0.0)):
        z = (v[:, a] - U) / sd
        assert abs(z.mean()) < 4 / np.sqrt(len(z))
        assert abs(z.var() - 1) < 0.03
        assert abs(stats.kurtosis(z)) < 0.1
        assert stats.kstest(z, "norm").pvalue > 1e-4
