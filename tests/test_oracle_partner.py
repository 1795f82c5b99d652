"""Pins of the oracle's choice of the second collision partner (CPU).

The NTC candidate's first particle is uniform over the cell; the gas model's
variants choose the second uniformly over the cell, within the first one's
subcell, or as its nearest neighbour.  The pins: the nearest neighbour
against a k-d tree search (scipy), the subcell rule against particles placed
in known subcells of a rectangular cell, one subcell per cell against the
uniform rule, and the mean distance between partners against the closed form
for two random points of a square or a cube.  Whole steps: one subcell per
cell reproduces the uniform scheme bit for bit, and every scheme conserves
energy in a closed specular box."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import Oracle, partner
from paper_cs_9902024_gb300 import workloads as W
from tests.helpers import box

# mean distance between two independent uniform points of the unit square
# and of the unit cube (closed forms)
MEAN_DIST_SQUARE = (2.0 + math.sqrt(2.0) + 5.0 * math.asinh(1.0)) / 15.0
MEAN_DIST_CUBE = (4.0 + 17.0 * math.sqrt(2.0) - 6.0 * math.sqrt(3.0)
                  + 21.0 * math.asinh(1.0) + 42.0 * math.log(2.0 + math.sqrt(3.0))
                  - 7.0 * math.pi) / 105.0


def _grid(dim, scheme, n_sub=2, L=None):
    w = box(dim=dim, ncell=(4, 3, 2), L=L)
    return W.with_partner(w, scheme, n_sub)


def _cell_geometry(w, c):
    n = w["ncell"]
    d = np.array([w["L"][a] / (n[a] if a < w["dim"] else 1) for a in range(3)])
    ci = np.array([c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1])], dtype=float)
    return ci * d, d


def test_invalid_partner_arguments():
    w = _grid(2, "subcell", n_sub=2)
    lo, d = _cell_geometry(w, 0)
    x = lo + np.array([[0.1, 0.1, 0.5], [0.9, 0.9, 0.5]]) * d
    assert partner(w, 0, x, 0, 0.5) == 1
    assert partner(w, 0, x[:1], 0, 0.5) == -1          # one particle: no pair
    assert partner(w, 0, x, 2, 0.5) == -1              # i out of range
    bad = W.with_partner(w, "subcell", n_sub=0)
    assert partner(bad, 0, x, 0, 0.5) == -1
    bad = dict(w, gas=dict(w["gas"], partner=3))
    assert partner(bad, 0, x, 0, 0.5) == -1


def test_closed_forms():
    assert MEAN_DIST_SQUARE == pytest.approx(0.5214054331, abs=1e-9)
    assert MEAN_DIST_CUBE == pytest.approx(0.6617071822, abs=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_nearest_is_the_kdtree_nearest_neighbour(dim):
    """The nearest scheme returns the k-d tree's nearest other particle, over
    the grid's axes only (in 2-D the third coordinate is random and must not
    matter), for any u1."""
    w = _grid(dim, "nearest", L=[0.04, 0.06, 0.04 if dim == 3 else 1.0])
    rng = np.random.default_rng(11)
    ncells = 12 * (2 if dim == 3 else 1)
    for _ in range(150):
        N = int(rng.integers(2, 40))
        c = int(rng.integers(0, ncells))
        lo, d = _cell_geometry(w, c)
        x = lo + rng.uniform(0.0, 1.0, (N, 3)) * d
        tree = cKDTree(x[:, :dim])
        for i in range(N):
            _, idx = tree.query(x[i, :dim], k=2)
            ref = int(idx[1] if idx[0] == i else idx[0])
            assert partner(w, c, x, i, float(rng.uniform())) == ref


def test_nearest_ties_go_to_the_first_in_lcr_order():
    # unit cells: the positions and their differences are exact
    w = _grid(2, "nearest", L=[4.0, 3.0, 1.0])
    lo, d = _cell_geometry(w, 5)
    mid = lo + 0.5 * d
    e = np.array([0.25 * d[0], 0.0, 0.0])
    for x in (np.array([mid, mid + e, mid - e]), np.array([mid, mid - e, mid + e])):
        assert partner(w, 5, x, 0, 0.9) == 1
    # a particle equidistant from 0 and 2 picks 0
    x = np.array([mid - e, mid, mid + e])
    assert partner(w, 5, x, 1, 0.1) == 0


def test_uniform_rule_and_one_subcell():
    """Sweeping u1 over the midpoints of N-1 equal bins visits every other
    particle once, in LCR order; with one subcell per cell the subcell scheme
    returns the same particle for every (positions, i, u1)."""
    wu = _grid(2, "uniform")
    ws = _grid(2, "subcell", n_sub=1)
    rng = np.random.default_rng(3)
    for _ in range(60):
        N = int(rng.integers(2, 30))
        c = int(rng.integers(0, 12))
        lo, d = _cell_geometry(wu, c)
        x = lo + rng.uniform(0.0, 1.0, (N, 3)) * d
        for i in range(N):
            seen = [partner(wu, c, x, i, (r + 0.5) / (N - 1)) for r in range(N - 1)]
            assert seen == [m for m in range(N) if m != i]
            for u1 in rng.uniform(0.0, 1.0, 4):
                assert partner(ws, c, x, i, u1) == partner(wu, c, x, i, u1)


@pytest.mark.parametrize("dim,n_sub", [(2, 3), (3, 2)])
def test_subcell_picks_within_placed_subcells(dim, n_sub):
    """Particles are placed inside chosen subcells of a rectangular cell (a
    different size per axis, so that exchanging axes moves particles to other
    subcells).  For a particle with K others in its subcell, the midpoints of
    K equal bins of u1 give exactly those others in LCR order; a particle
    alone in its subcell takes the uniform rule over the whole cell."""
    L = [0.03 * 4, 0.05 * 3, 0.07 * 2 if dim == 3 else 1.0]
    w = _grid(dim, "subcell", n_sub=n_sub, L=L)
    rng = np.random.default_rng(17)
    ncells = 12 * (2 if dim == 3 else 1)
    for _ in range(40):
        c = int(rng.integers(0, ncells))
        lo, d = _cell_geometry(w, c)
        N = int(rng.integers(2, 25))
        sub = rng.integers(0, n_sub, (N, 3))
        if dim == 2:
            sub[:, 2] = 0
        frac = (sub + rng.uniform(0.05, 0.95, (N, 3))) / n_sub
        x = lo + frac * d
        if dim == 2:
            x[:, 2] = rng.uniform(0.0, L[2], N)
        key = [tuple(s[:dim]) for s in sub]
        for i in range(N):
            mates = [m for m in range(N) if m != i and key[m] == key[i]]
            if mates:
                K = len(mates)
                got = [partner(w, c, x, i, (r + 0.5) / K) for r in range(K)]
                assert got == mates
            else:
                got = [partner(w, c, x, i, (r + 0.5) / (N - 1)) for r in range(N - 1)]
                assert got == [m for m in range(N) if m != i]


@pytest.mark.parametrize("dim", [2, 3])
def test_mean_partner_distance_closed_form(dim):
    """Uniform positions in a cube-shaped (or square) cell: uniform partners
    lie at the mean distance of two random points of the cell, subcell
    partners (2 per axis, every subcell occupied) at half of it."""
    side = 0.02
    L = [side * 4, side * 3, side * 2 if dim == 3 else 1.0]
    ref = MEAN_DIST_CUBE if dim == 3 else MEAN_DIST_SQUARE
    rng = np.random.default_rng(23 + dim)
    for scheme, scale in (("uniform", 1.0), ("subcell", 0.5)):
        w = _grid(dim, scheme, n_sub=2, L=L)
        c = 7
        lo, d = _cell_geometry(w, c)
        dist = []
        for _ in range(1500):
            N = 80
            x = lo + rng.uniform(0.0, 1.0, (N, 3)) * d
            for i in rng.integers(0, N, 6):
                j = partner(w, c, x, int(i), float(rng.uniform()))
                dist.append(np.linalg.norm((x[j] - x[i])[:dim]) / side)
        dist = np.array(dist)
        se = dist.std() / math.sqrt(len(dist))
        assert abs(dist.mean() - scale * ref) < 4.0 * se, (scheme, dist.mean(), scale * ref)


def _run(w, runs, steps):
    o = Oracle(w, runs=runs)
    out = []
    for r in range(runs):
        o.init_run(r)
        for s in range(1, steps + 1):
            o.step(r, s)
        x, v, _ = o.get_state(r)
        out.append((x, v, o.get_cells(r), o.stats(r)))
    o.close()
    return out


def test_one_subcell_step_equals_uniform():
    w = W.duct64x32_n8(runs=2, steps=30)
    a = _run(w, 2, 30)
    b = _run(W.with_partner(w, "subcell", n_sub=1), 2, 30)
    for (xa, va, ca, sa), (xb, vb, cb, sb) in zip(a, b):
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        for p, q in zip(ca, cb):
            assert np.array_equal(p, q)
        assert sa == sb
        assert sa["collisions"] > 0


@pytest.mark.parametrize("scheme", ["uniform", "subcell", "nearest"])
def test_closed_specular_box_conserves_energy(scheme):
    """Specular walls and elastic collisions: the kinetic energy of a closed
    box is constant whichever partner the scheme picks, and the positional
    schemes change the trajectory (they pick other pairs)."""
    base = box(dim=2, ncell=(6, 6, 1), ppc=30.0, dt=5e-6, steps=15)
    w = W.with_partner(base, scheme, n_sub=2)
    o = Oracle(w, runs=1)
    o.init_run(0)
    _, v0, _ = o.get_state(0)
    e0 = (v0 ** 2).sum()
    for s in range(1, 16):
        o.step(0, s)
    _, v1, _ = o.get_state(0)
    st = o.stats(0)
    o.close()
    assert st["collisions"] > 100
    assert abs((v1 ** 2).sum() - e0) <= 1e-12 * e0
    if scheme != "uniform":
        ou = Oracle(base, runs=1)
        ou.init_run(0)
        for s in range(1, 16):
            ou.step(0, s)
        _, vu, _ = ou.get_state(0)
        ou.close()
        assert not np.array_equal(vu, v1)
