"""Pins of Generation (inflow) in the oracle against kinetic-theory closed
forms and direct numerical integration (CPU)."""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

from oracle import Oracle, inflow_flux, sample_xi
from paper_cs_9902024_gb300 import workloads as W
from tests.helpers import box

KB = 1.380649e-23
M = W.M_AR


def flux_by_quadrature(n, T, Un):
    """Number flux through a plane: integral over u > 0 of u n phi(u), phi
    the 1-D Maxwellian of mean Un and variance kT/m."""
    sd = math.sqrt(KB * T / M)
    f = lambda u: u * n * math.exp(-0.5 * ((u - Un) / sd) ** 2) / (sd * math.sqrt(2 * math.pi))
    val, _ = integrate.quad(f, 0.0, Un + 40 * sd if Un > 0 else 40 * sd, limit=200)
    return val


@pytest.mark.parametrize("T", [200.0, 300.0])
def test_effusion_flux_closed_form(T):
    """U = 0: flux = n cbar / 4, cbar = sqrt(8kT/(pi m)) (textbook effusion)."""
    n = 1e20
    cbar = math.sqrt(8 * KB * T / (math.pi * M))
    assert inflow_flux(n, T, 0.0, M) == pytest.approx(n * cbar / 4, rel=1e-13)


@pytest.mark.parametrize("Un", [-300.0, -50.0, 120.0, 400.0, 1317.4])
def test_drifting_flux_matches_quadrature(Un):
    n, T = 1e20, 300.0
    assert inflow_flux(n, T, Un, M) == pytest.approx(flux_by_quadrature(n, T, Un), rel=1e-8)


def test_hypersonic_flux_limit():
    """s >> 1: every molecule moves inward, flux -> n U."""
    n, T = 1e20, 200.0
    U = 20 * math.sqrt(2 * KB * T / M)
    assert inflow_flux(n, T, U, M) == pytest.approx(n * U, rel=1e-12)


def _xi_pdf_cdf(s):
    Z = 0.5 * (math.exp(-s * s) + math.sqrt(math.pi) * s * (1 + math.erf(s)))
    f = lambda x: x * math.exp(-(x - s) ** 2) / Z
    cdf = lambda x: integrate.quad(f, 0.0, x)[0] if x > 0 else 0.0
    mean = ((s / 2) * math.exp(-s * s) + math.sqrt(math.pi) / 4 * (1 + 2 * s * s) * (1 + math.erf(s))) / Z
    return f, np.vectorize(cdf), mean


@pytest.mark.parametrize("s", [-0.7, 0.0, 0.9129, 1.1316, 4.564])
def test_entrant_normal_speed_distribution(s):
    """Inward normal speed ratio of entering molecules has density
    xi exp(-(xi-s)^2) / Z on xi > 0: KS test and the closed-form mean."""
    xs = np.array([sample_xi(s, 5, 0, 1, e, k)[0] for e in range(40) for k in range(150)])
    assert np.all(xs > 0)
    _, cdf, mean = _xi_pdf_cdf(s)
    assert stats.kstest(xs, cdf).pvalue > 1e-3
    assert abs(xs.mean() - mean) < 5 * xs.std() / math.sqrt(len(xs))


def test_generation_count_and_velocities():
    """Duct inflow: entrants per element per step average to
    flux * A * dt / F_N; their normal velocity has the closed-form mean and
    their tangential components are N(U_t, kT/m)."""
    w = W.duct64x32_n8(runs=1)
    w["gas"]["d_ref"] = 0.0          # no collisions: velocities stay as drawn
    for b in w["bcs"]:               # specular side walls only flip v_y, whose
        if b["face"] in (W.YMIN, W.YMAX):   # law is symmetric about 0
            b["kind"] = W.SPECULAR
    o = Oracle(w, runs=1)
    o.init_run(0)
    n_in, T, U = 1e20, 300.0, 400.0
    lam = w["L"][0] / w["ncell"][0]
    dt = w["dt"]
    per_elem = flux_by_quadrature(n_in, T, U) * lam * 1.0 * dt / w["gas"]["F_N"]
    steps = 30
    for s in range(1, steps + 1):
        o.step(0, s)
    gen = o.stats(0)["generated"]
    expect = per_elem * w["ncell"][1] * steps
    # stochastic rounding: variance <= 1/4 per element and step
    assert abs(gen - expect) < 6 * math.sqrt(0.25 * w["ncell"][1] * steps)
    # the particles still near the inlet are a fair sample of entrants only
    # after one step; use a fresh run for the velocity statistics
    o2 = Oracle(w, runs=1)
    o2.init_run(0)
    o2.step(0, 1)
    x, v, _ = o2.get_state(0)
    cmp_ = math.sqrt(2 * KB * T / M)
    _, _, mean_xi = _xi_pdf_cdf(U / cmp_)
    sd = math.sqrt(KB * T / M)
    many = []
    for rep in range(2, 40):
        o3 = Oracle(w, runs=1, seed=100 + rep)
        o3.init_run(0)
        o3.step(0, 1)
        many.append(o3.get_state(0)[1])
    v = np.concatenate([v] + many)
    assert abs(v[:, 0].mean() - cmp_ * mean_xi) < 5 * v[:, 0].std() / math.sqrt(len(v))
    for a in (1, 2):
        z = v[:, a] / sd
        assert abs(z.mean()) < 5 / math.sqrt(len(z))
        assert abs(z.var() - 1) < 0.06
        assert stats.kstest(z, "norm").pvalue > 1e-4


def test_segment_override_and_pulse():
    """A later segment overrides an earlier one where both apply, and an
    inflow segment generates only during its active steps (pulsed jet)."""
    w = W.pulsed_jet(nx=32, ny=16, runs=1, steps=20, n_samples=1, orifice=4, pulse=3,
                     F_N=4.49e10 * 400)
    w["gas"]["d_ref"] = 0.0
    o = Oracle(w, runs=1)
    o.init_run(0)
    counts = []
    for s in range(1, 7):
        before = o.stats(0)["generated"]
        o.step(0, s)
        counts.append(o.stats(0)["generated"] - before)
    assert all(c > 0 for c in counts[:3])
    assert all(c == 0 for c in counts[3:])
    # entrants enter only through the 4 orifice cells of the left face
    o = Oracle(w, runs=1)
    o.init_run(0)
    o.step(0, 1)
    x, v, _ = o.get_state(0)
    lam = w["L"][1] / w["ncell"][1]
    y0 = (16 - 4) // 2
    # back-trace each particle to x = 0 along its (collision-free) path
    inside = x[:, 0] < lam  # moved less than one cell in one step
    t_back = x[inside, 0] / v[inside, 0]
    y_entry = x[inside, 1] - v[inside, 1] * t_back
    assert np.all(y_entry > y0 * lam - 1e-12) and np.all(y_entry < (y0 + 4) * lam + 1e-12)
