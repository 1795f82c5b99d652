"""Pins of Enumeration/Indexing, Interaction and Sampling in the oracle (CPU)."""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

from oracle import Oracle, run_ensemble, scatter, sigma_cr
from paper_cs_9902024_gb300 import workloads as W
from tests.helpers import box, cell_index

KB = 1.380649e-23
M = W.M_AR


def test_lcr_is_stable_sort_by_cell():
    """After a step P is ordered by cell, and inside each cell by pre-step
    slot (the order one serial pass over P fills the readdressing array in):
    the readdressing array equals a stable sort of the survivors' slots by
    cell, counts equal a bincount, and LCR is a permutation of the surviving
    pre-step slots (old particles in their pre-step order, then the entrants
    in generation order)."""
    w = W.duct64x32_n8(runs=1, steps=40)
    o = Oracle(w, runs=1)
    o.init_run(0)
    for s in range(1, 41):
        n_old = o.count(0)
        _, _, ids_before = o.get_state(0)
        o.step(0, s)
    x, v, ids = o.get_state(0)
    cells = cell_index(w, x)
    count, cand, acc, lcr = o.get_cells(0)
    assert np.array_equal(count, np.bincount(cells, minlength=len(count)))
    assert len(np.unique(lcr)) == len(lcr)
    # a stable sort of the surviving slots by their cell reproduces LCR
    order = np.lexsort((lcr, cells))
    assert np.array_equal(order, np.arange(len(ids)))
    assert np.all(np.diff(cells) >= 0)
    same = np.diff(cells) == 0
    assert np.all(np.diff(lcr)[same] > 0)
    # old particles keep their slot (their position in the pre-step order);
    # new ones have slots >= n_old in generation (= id) order
    old = lcr < n_old
    assert np.array_equal(ids[old], ids_before[lcr[old]])
    assert np.all(ids[~old] >= ids_before.max(initial=0))
    # a new particle's slot minus n_old is its generation index: id - slot
    # is the same for all of them
    if (~old).any():
        assert len(np.unique(ids[~old].astype(np.int64) - (lcr[~old] - n_old))) == 1


def test_scatter_conserves_momentum_and_energy():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        v1 = rng.normal(0, 400, 3) + rng.normal(0, 1000, 3)
        v2 = rng.normal(0, 400, 3)
        u3, u4 = rng.uniform(0, 1, 2)
        a, b = scatter(v1, v2, u3, u4)
        p0, p1 = v1 + v2, a + b
        e0, e1 = (v1 ** 2).sum() + (v2 ** 2).sum(), (a ** 2).sum() + (b ** 2).sum()
        assert np.allclose(p1, p0, rtol=0, atol=1e-12 * np.abs(v1).max())
        assert abs(e1 - e0) <= 1e-14 * e0 * 8
        g0, g1 = v1 - v2, a - b
        assert math.isclose(np.linalg.norm(g1), np.linalg.norm(g0), rel_tol=1e-14)
        # post-collision direction: cos(chi) = 2 u3 - 1 about the x axis
        assert math.isclose(g1[0] / np.linalg.norm(g1), 2 * u3 - 1, abs_tol=1e-12)
        assert math.isclose(math.atan2(g1[2], g1[1]) % (2 * math.pi), 2 * math.pi * u4,
                            abs_tol=1e-9) or abs(1 - abs(2 * u3 - 1)) < 1e-6


def test_hard_sphere_cross_section():
    w = W.duct64x32_n8()
    for g in (1.0, 400.0, 2500.0):
        assert sigma_cr(w, g) == pytest.approx(math.pi * W.D_HS ** 2 * g, rel=1e-15)


@pytest.mark.parametrize("omega", [0.5, 0.75, 0.81, 1.0])
def test_vhs_reference_diameter_property(omega):
    """The VHS d_ref is the hard-sphere diameter whose equilibrium
    <sigma c_r> matches at T_ref: integrate the oracle's sigma*c_r over the
    equilibrium relative-speed law at T_ref (reduced mass m/2) and compare
    with pi d_ref^2 <c_r>, <c_r> = 4 sqrt(kT/(pi m))."""
    T = 273.0
    w = W.jet256x128_n64()
    over = dict(omega=omega, T_ref=T)
    mr = M / 2
    a = mr / (2 * KB * T)
    f = lambda g: 4 * math.pi * (a / math.pi) ** 1.5 * g * g * math.exp(-a * g * g)
    mean_sc, _ = integrate.quad(lambda g: f(g) * sigma_cr(w, g, over), 0, 20 / math.sqrt(a), limit=200)
    cr = 4 * math.sqrt(KB * T / (math.pi * M))
    assert mean_sc == pytest.approx(math.pi * 4.17e-10 ** 2 * cr, rel=1e-8)
    # power law in the relative speed: sigma_T c_r ~ c_r^(2 - 2 omega)
    r = sigma_cr(w, 800.0, over) / sigma_cr(w, 400.0, over)
    assert r == pytest.approx(2.0 ** (2 - 2 * omega), rel=1e-12)


def _equilibrium_rate(omega, T, T_ref, d, n):
    """Collisions per unit volume and time in equilibrium: n^2 <sigma c_r>/2
    with <sigma c_r> = pi d^2 <c_r>(T_ref) (T/T_ref)^(1-omega) and
    <c_r>(T) = 4 sqrt(kT/(pi m)) (hard sphere: omega = 1/2, T_ref = T)."""
    cr = 4 * math.sqrt(KB * T_ref / (math.pi * M))
    return 0.5 * n * n * math.pi * d * d * cr * (T / T_ref) ** (1 - omega)


@pytest.mark.parametrize("omega,T_ref", [(0.5, 300.0), (0.81, 273.0), (0.81, 600.0)])
def test_ntc_equilibrium_collision_rate(omega, T_ref):
    """Equilibrium box: accepted collisions per step match the closed form
    n^2 <sigma c_r> V dt / (2 F_N) (NTC with N(N-1) is unbiased)."""
    T, n = 300.0, 1e20
    w = box(dim=2, ncell=(8, 8, 1), fill_T=T, ppc=200, dt=4e-6, omega=omega, T_ref=T_ref,
            d_ref=W.D_HS)
    o = Oracle(w, runs=1)
    o.init_run(0)
    steps = 25
    for s in range(1, steps + 1):
        o.step(0, s)
    st = o.stats(0)
    V = w["L"][0] * w["L"][1] * w["L"][2]
    expect = _equilibrium_rate(omega, T, T_ref, W.D_HS, n) * V * w["dt"] * steps / w["gas"]["F_N"]
    assert st["collisions"] == pytest.approx(expect, rel=0.04)
    assert st["candidates"] > st["collisions"]


def test_maxwell_molecule_relaxation():
    """VHS omega = 1 (Maxwell molecules): sigma c_r is constant, every
    candidate is accepted, and in a homogeneous box an anisotropic
    temperature relaxes as T_x - T ~ exp(-nu t / 2), nu = n sigma c_r.  In a
    cell of N particles each collision multiplies E[T_x - T] by
    (1 - 1/(N-1)) exactly; the test checks that discrete law."""
    n = 1e20
    w = box(dim=2, ncell=(1, 1, 1), L=[0.05, 0.05, 1.0], fill=0, ppc=1500, omega=1.0,
            T_ref=300.0, dt=4e-6, fill_n=n)
    rng = np.random.default_rng(2)
    N = 1500
    sd = math.sqrt(KB * 300.0 / M)
    ratios = []
    colls = []
    for rep in range(6):
        x = np.zeros((N, 3)); v = np.zeros((N, 3))
        x[:, 0] = rng.uniform(0, 0.05, N); x[:, 1] = rng.uniform(0, 0.05, N)
        v[:, 0] = rng.normal(0, sd * math.sqrt(2.2), N)
        v[:, 1] = rng.normal(0, sd * math.sqrt(0.4), N)
        v[:, 2] = rng.normal(0, sd * math.sqrt(0.4), N)
        o = Oracle(w, runs=1, seed=40 + rep)
        o.init_run(0)
        o.set_state(0, x, v, np.arange(N, dtype=np.uint32), N)
        def aniso(vv):
            T = (vv ** 2).sum(1).mean()
            return (vv[:, 0] ** 2).mean() - T / 3
        a0 = aniso(v)
        traj = []
        for s in range(1, 9):
            o.step(0, s)
            traj.append(aniso(o.get_state(0)[1]) / a0)
            colls.append(o.stats(0)["collisions"])
        st = o.stats(0)
        assert st["collisions"] == st["candidates"]          # accept prob = 1
        ratios.append(traj)
    ratios = np.array(ratios).mean(0)
    C_per_step = np.array(colls).reshape(6, 8)
    C_mean = C_per_step.mean(0)
    predicted = (1 - 1 / (N - 1)) ** C_mean
    assert np.allclose(ratios, predicted, atol=0.03)
    # and the continuum law exp(-nu t / 2)
    nu = n * math.pi * W.D_HS ** 2 * math.sqrt(2 * KB * 300.0 / (M / 2)) / special.gamma(1.5)
    t = w["dt"] * np.arange(1, 9)
    assert np.allclose(ratios, np.exp(-nu * t / 2), atol=0.04)


def test_sampling_is_brute_force_sum():
    w = W.duct64x32_n8(runs=1)
    o = Oracle(w, runs=1)
    o.init_run(0)
    for s in range(1, 31):
        o.step(0, s)
    mom = o.sample(0)
    x, v, _ = o.get_state(0)
    c = cell_index(w, x)
    nc = mom.shape[0]
    assert np.array_equal(mom[:, 0], np.bincount(c, minlength=nc).astype(float))
    for a in range(3):
        assert np.allclose(mom[:, 1 + a], np.bincount(c, v[:, a], minlength=nc), rtol=1e-12, atol=1e-9)
        assert np.allclose(mom[:, 4 + a], np.bincount(c, v[:, a] ** 2, minlength=nc), rtol=1e-12)


def test_ensemble_groups_are_sums_of_runs():
    """run_ensemble's group accumulators equal the per-run samples of the
    step-level API summed per group (g = run mod G) -- independently of the
    number of worker threads."""
    w = W.duct64x32_n8(runs=5, steps=12, n_samples=2)
    acc1, st1 = run_ensemble(w, threads=1)
    acc3, st3 = run_ensemble(w, threads=3)
    assert np.array_equal(acc1, acc3) and st1 == st3
    o = Oracle(w, runs=5)
    G = 5
    ref = np.zeros_like(acc1)
    for r in range(5):
        o.init_run(r)
        t = 0
        for s in range(1, 13):
            o.step(r, s)
            if s in w["sample_steps"]:
                ref[t, r % G] += o.sample(r)
                t += 1
    assert np.array_equal(ref, acc1)


def test_sample_windows_sum_single_step_samples():
    """Time-averaged samples (Sec. 1.1's averaging interval): a window's
    group sums are the sums of the one-step samples of its steps, and a
    one-step window is the plain sample."""
    from oracle import run_ensemble
    from paper_cs_9902024_gb300 import workloads as W
    w = W.duct64x32_n8(runs=3, steps=40, n_samples=2)
    single, _ = run_ensemble(w, sample_steps=list(range(21, 31)))
    win, _ = run_ensemble(w, windows=[(21, 30)])
    assert np.array_equal(win[0][..., 0], single[..., 0].sum(axis=0))
    assert np.allclose(win[0], single.sum(axis=0), rtol=1e-12, atol=1e-9)
    one, _ = run_ensemble(w, windows=[(20, 20), (40, 40)])
    plain, _ = run_ensemble(w, sample_steps=[20, 40])
    assert np.array_equal(one, plain)


def test_hard_sphere_relaxation_to_maxwellian():
    """Homogeneous hard-sphere gas started on a speed shell (every particle
    at the same speed, isotropic directions: each velocity component has
    kurtosis 9/5) relaxes to the Maxwellian at the same energy: after ~19
    collisions per particle every component has kurtosis 3 and passes a
    Kolmogorov-Smirnov test against N(0, kT/m); energy and the momentum
    along the wall-free axis are conserved to rounding throughout."""
    n = 1e20
    N = 2000
    w = box(dim=2, ncell=(1, 1, 1), L=[0.05, 0.05, 1.0], fill=0, ppc=N, omega=0.5,
            T_ref=300.0, dt=2e-5, fill_n=n)
    rng = np.random.default_rng(5)
    c0 = math.sqrt(3 * KB * 300.0 / M)
    kurt0, kurt1, pks = [], [], []
    for rep in range(3):
        x = np.zeros((N, 3))
        x[:, 0] = rng.uniform(0, 0.05, N)
        x[:, 1] = rng.uniform(0, 0.05, N)
        dirs = rng.normal(size=(N, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        v = c0 * dirs
        v -= v.mean(0)                       # zero net momentum
        E0 = (v ** 2).sum()
        kurt0.append(((v ** 4).mean(0) / (v ** 2).mean(0) ** 2).mean())
        o = Oracle(w, runs=1, seed=70 + rep)
        o.init_run(0)
        o.set_state(0, x, v, np.arange(N, dtype=np.uint32), N)
        for s in range(1, 41):
            o.step(0, s)
        vv = o.get_state(0)[1]
        assert abs((vv ** 2).sum() / E0 - 1) < 1e-12
        # specular walls reverse x and y; the z momentum only collisions change
        assert abs(vv[:, 2].sum()) < 1e-9 * c0 * N
        assert o.stats(0)["collisions"] > 8 * N       # > 16 collisions per particle
        kurt1.append(((vv ** 4).mean(0) / (vv ** 2).mean(0) ** 2).mean())
        T = M * (vv ** 2).sum() / (3 * N * KB)
        sd = math.sqrt(KB * T / M)
        for a in range(3):
            pks.append(stats.kstest(vv[:, a] / sd, "norm").pvalue)
    assert abs(np.mean(kurt0) - 1.8) < 0.05
    assert abs(np.mean(kurt1) - 3.0) < 0.2
    assert min(pks) > 1e-4
