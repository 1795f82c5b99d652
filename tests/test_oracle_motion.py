"""Pins of Motion (free flight and surface interaction) in the oracle (CPU)."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_cs_9902024_gb300 import workloads as W
from tests.helpers import box

KB = 1.380649e-23
M = W.M_AR


def fold(y, L):
    """Position and velocity sign in a specularly reflecting slab [0, L]
    after unreflected travel to y: the triangle wave of period 2L."""
    r = np.mod(y, 2 * L)
    pos = np.where(r > L, 2 * L - r, r)
    sign = np.where(np.mod(np.floor(y / L), 2) == 0, 1.0, -1.0)
    return pos, sign


@pytest.mark.parametrize("dim", [2, 3])
def test_specular_box_is_unfolded_free_flight(dim):
    """All faces specular, no collisions: each coordinate follows the
    triangle wave of free flight (several reflections per step, corners)."""
    w = box(dim=dim, ncell=(5, 4, 3), d_ref=0.0, fill=0, dt=1e-5)
    L = w["L"]
    rng = np.random.default_rng(1)
    n = 3000
    x = np.zeros((n, 3)); v = np.zeros((n, 3))
    for a in range(dim):
        x[:, a] = rng.uniform(0, L[a], n)
        v[:, a] = rng.uniform(-3.2, 3.2, n) * L[a] / w["dt"] / 3.0 * (1.0 if dim == 2 else 0.9)
    v[:, 2] = rng.normal(0, 300, n) if dim == 2 else v[:, 2]
    ids = np.arange(n, dtype=np.uint32)
    o = Oracle(w, runs=1)
    o.init_run(0)
    o.set_state(0, x, v, ids, n)
    o.step(0, 1)
    x1, v1, id1 = o.get_state(0)
    assert len(id1) == n
    order = np.argsort(id1)
    x1, v1 = x1[order], v1[order]
    for a in range(dim):
        pos, sign = fold(x[:, a] + v[:, a] * w["dt"], L[a])
        assert np.allclose(x1[:, a], pos, rtol=0, atol=1e-12 * L[a])
        assert np.array_equal(v1[:, a], sign * v[:, a])
    if dim == 2:
        assert np.array_equal(v1[:, 2], v[:, 2])


def test_outflow_removes_and_open_faces():
    """A particle crossing an outflow face is removed; one that does not
    reach it stays, with x = x0 + v dt exactly."""
    w = box(dim=2, ncell=(4, 4, 1), kinds={W.XMAX: W.OUTFLOW}, d_ref=0.0, fill=0, dt=1e-5)
    L = w["L"][0]
    x = np.array([[0.9 * L, 0.02, 0], [0.5 * L, 0.02, 0], [0.2 * L, 0.01, 0]])
    v = np.array([[0.2 * L / 1e-5, 0, 0], [0.2 * L / 1e-5, 0, 0], [-0.1 * L / 1e-5, 0, 7.0]])
    o = Oracle(w, runs=1)
    o.init_run(0)
    o.set_state(0, x, v, np.arange(3, dtype=np.uint32), 3)
    o.step(0, 1)
    x1, v1, ids = o.get_state(0)
    assert sorted(ids.tolist()) == [1, 2]
    k = list(ids).index(1)
    assert x1[k, 0] == x[1, 0] + v[1, 0] * 1e-5
    assert o.stats(0)["removed"] == 1


def test_diffuse_box_accommodates_to_wall_temperature():
    """No collisions, diffuse walls at Tw: a gas started at 150 K ends as an
    isotropic Maxwellian at Tw with zero mean velocity (the flux-weighted
    re-emission law; a half-range Maxwellian re-emission would not)."""
    Tw = 300.0
    w = box(dim=2, ncell=(4, 4, 1), kinds={f: W.DIFFUSE for f in range(4)}, Tw=Tw,
            fill_T=150.0, fill_U=(200.0, 0.0, 0.0), d_ref=0.0, ppc=400, dt=2e-6)
    o = Oracle(w, runs=1)
    o.init_run(0)
    for s in range(1, 401):
        o.step(0, s)
    _, v, _ = o.get_state(0)
    sd = math.sqrt(KB * Tw / M)
    n = len(v)
    # in-plane components hit the walls; w is redrawn at every wall hit
    for a in range(3):
        assert abs(v[:, a].mean()) < 5 * sd / math.sqrt(n)
        assert v[:, a].var() / sd ** 2 == pytest.approx(1.0, abs=0.05)
    T = M * (v ** 2).sum(1).mean() / (3 * KB)
    assert T == pytest.approx(Tw, rel=0.02)


def test_diffuse_wall_hit_rate_is_effusion_flux():
    """Equilibrium gas in a diffuse box at the wall temperature: wall hits
    per step = n cbar/4 * (wall area) * dt / F_N."""
    T = 300.0
    w = box(dim=2, ncell=(6, 6, 1), kinds={f: W.DIFFUSE for f in range(4)}, Tw=T,
            fill_T=T, d_ref=0.0, ppc=200, dt=2e-7)
    o = Oracle(w, runs=1)
    o.init_run(0)
    steps = 40
    for s in range(1, steps + 1):
        o.step(0, s)
    hits = o.stats(0)["wall_hits"]
    n = 1e20
    cbar = math.sqrt(8 * KB * T / (math.pi * M))
    perim = 2 * (w["L"][0] + w["L"][1]) * w["L"][2]
    expect = n * cbar / 4 * perim * w["dt"] * steps / w["gas"]["F_N"]
    assert abs(hits - expect) < 5 * math.sqrt(expect) + 0.01 * expect


def test_effusion_through_orifice():
    """Specular box with a 4-cell outflow orifice: leavers per step =
    n cbar / 4 * A_orifice * dt / F_N while the density is still n."""
    T = 300.0
    orifice = W.bc(W.OUTFLOW, W.XMAX, lo=(6, 0), hi=(10, 1))
    w = box(dim=2, ncell=(16, 16, 1), fill_T=T, d_ref=0.0, ppc=100, dt=5e-7,
            extra_bcs=[orifice])
    o = Oracle(w, runs=1)
    o.init_run(0)
    N0 = o.count(0)
    steps = 30
    for s in range(1, steps + 1):
        o.step(0, s)
    removed = o.stats(0)["removed"]
    assert removed < 0.05 * N0
    n = 1e20
    cbar = math.sqrt(8 * KB * T / (math.pi * M))
    A = 4 * (w["L"][1] / 16) * w["L"][2]
    expect = n * cbar / 4 * A * w["dt"] * steps / w["gas"]["F_N"]
    assert abs(removed - expect) < 5 * math.sqrt(expect)


@pytest.mark.parametrize("kind", [W.SPECULAR, W.DIFFUSE])
def test_plate_reflects_inside_and_passes_outside(kind):
    """A zero-thickness plate normal to x reflects particles that cross it
    inside its rectangle and lets the others through."""
    w = box(dim=3, ncell=(8, 8, 8), d_ref=0.0, fill=0, dt=1e-5,
            extra_bcs=[W.bc(kind, W.PLATE, lo=(2, 2), hi=(6, 6), T=300.0,
                            plate_axis=0, plate_index=4)])
    L = w["L"][0]
    d = L / 8
    xp = 4 * d
    rng = np.random.default_rng(3)
    n = 400
    x = np.zeros((n, 3)); v = np.zeros((n, 3))
    x[:, 0] = xp - rng.uniform(0.05, 0.5, n) * d
    x[:, 1] = rng.uniform(0.5, 7.5, n) * d
    x[:, 2] = rng.uniform(0.5, 7.5, n) * d
    v[:, 0] = 0.9 * d / w["dt"]
    o = Oracle(w, runs=1)
    o.init_run(0)
    o.set_state(0, x, v, np.arange(n, dtype=np.uint32), n)
    o.step(0, 1)
    x1, v1, ids = o.get_state(0)
    x1 = x1[np.argsort(ids)]; v1 = v1[np.argsort(ids)]
    inside = (x[:, 1] >= 2 * d) & (x[:, 1] < 6 * d) & (x[:, 2] >= 2 * d) & (x[:, 2] < 6 * d)
    free = x[:, 0] + v[:, 0] * w["dt"]
    assert np.allclose(x1[~inside, 0], free[~inside], atol=1e-12 * L)
    assert np.all(x1[inside, 0] <= xp)            # stayed on the upstream side
    assert np.all(v1[inside, 0] < 0)
    if kind == W.SPECULAR:
        assert np.allclose(x1[inside, 0], 2 * xp - free[inside], atol=1e-12 * L)
        assert np.array_equal(v1[inside, 0], -v[inside, 0])
    assert o.stats(0)["wall_hits"] == inside.sum()


@pytest.mark.parametrize("order", ["x_outflow_y_diffuse", "x_diffuse_y_outflow"])
def test_simultaneous_corner_hit_takes_x_face_first(order):
    """A flight that reaches two faces at exactly the same time (a corner)
    meets the x face first.  Outflow on x: the particle leaves without a
    wall hit.  Diffuse on x, outflow on y: it is re-emitted by the x wall
    (one wall hit) from the corner, where the y face still removes it
    unless its new velocity points into the domain."""
    if order == "x_outflow_y_diffuse":
        kinds = {W.XMIN: W.OUTFLOW, W.YMIN: W.DIFFUSE}
    else:
        kinds = {W.XMIN: W.DIFFUSE, W.YMIN: W.OUTFLOW}
    w = box(dim=2, ncell=(4, 4, 1), kinds=kinds, fill=0, dt=1e-5)
    d = w["L"][0] / 4
    assert d == w["L"][1] / 4
    x = np.array([[0.5 * d, 0.5 * d, 0.0]])          # equal distances to both faces
    v = np.array([[-1000.0, -1000.0, 0.0]])          # equal speeds: exactly equal times
    o = Oracle(w, runs=1)
    o.init_run(0)
    o.set_state(0, x, v, np.array([0], dtype=np.uint32), 1)
    o.step(0, 1)
    st = o.stats(0)
    if order == "x_outflow_y_diffuse":
        assert st["removed"] == 1 and st["wall_hits"] == 0
    else:
        assert st["wall_hits"] >= 1
        n_left = o.count(0)
        assert st["removed"] + n_left == 1
        if n_left:
            xs, vs, _ = o.get_state(0)
            assert xs[0, 0] >= 0.0 and xs[0, 1] >= 0.0
