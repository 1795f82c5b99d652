"""ctypes wrapper around the C oracle (dsmc_oracle.c).

Test infrastructure only: used by tests/, the smoke check and the CPU
baseline; the product path never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "dsmc_oracle.c")]
NMOM = 7
MAX_BC = 32
KB = 1.380649e-23

_lock = threading.Lock()
_lib = None


def build_oracle(force=False):
    """Compile the oracle with gcc (IEEE double, no fused multiply-add)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in SOURCES + [os.path.join(HERE, "dsmc_oracle.h")])
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp] + SOURCES + ["-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Bc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("face", C.c_int32),
                ("lo", C.c_int32 * 2), ("hi", C.c_int32 * 2),
                ("step_from", C.c_int32), ("step_to", C.c_int32),
                ("plate_axis", C.c_int32), ("plate_index", C.c_int32),
                ("n", C.c_double), ("T", C.c_double), ("U", C.c_double * 3)]


class Config(C.Structure):
    _fields_ = [("dim", C.c_int32), ("ncell", C.c_int32 * 3), ("L", C.c_double * 3),
                ("mass", C.c_double), ("d_ref", C.c_double), ("T_ref", C.c_double),
                ("omega", C.c_double), ("F_N", C.c_double),
                ("fill", C.c_int32), ("fill_n", C.c_double), ("fill_T", C.c_double),
                ("fill_U", C.c_double * 3),
                ("n_bc", C.c_int32), ("bc", Bc * MAX_BC),
                ("partner", C.c_int32), ("n_sub", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in (
        "particle_steps", "generated", "removed", "wall_hits", "candidates",
        "collisions", "clamps", "bounce_limit", "reject_limit")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def oracle_lib():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = C.CDLL(LIB_PATH)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int32)
            u32p = C.POINTER(C.c_uint32)
            i64p = C.POINTER(C.c_int64)
            lib.orc_philox.argtypes = [u32p, u32p, u32p]
            lib.orc_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                     C.c_uint32, C.c_uint32, dp]
            lib.orc_inflow_flux.restype = C.c_double
            lib.orc_inflow_flux.argtypes = [C.c_double] * 4
            lib.orc_sample_xi.argtypes = [C.c_double, C.c_uint64, C.c_uint32, C.c_uint32,
                                          C.c_uint32, C.c_uint32, dp]
            lib.orc_sigma_cr.restype = C.c_double
            lib.orc_sigma_cr.argtypes = [C.POINTER(Config), C.c_double]
            lib.orc_scatter.argtypes = [dp, dp, C.c_double, C.c_double]
            lib.orc_partner.restype = C.c_int64
            lib.orc_partner.argtypes = [C.POINTER(Config), C.c_int, dp, C.c_int64, C.c_int64,
                                        C.c_double]
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [C.POINTER(Config), C.c_int, C.c_double, C.c_uint64]
            lib.orc_destroy.argtypes = [P]
            lib.orc_init_run.argtypes = [P, C.c_int]
            lib.orc_step.argtypes = [P, C.c_int, C.c_int]
            lib.orc_count.restype = C.c_int64
            lib.orc_count.argtypes = [P, C.c_int]
            lib.orc_next_id.restype = C.c_uint32
            lib.orc_next_id.argtypes = [P, C.c_int]
            lib.orc_get_state.argtypes = [P, C.c_int, dp, dp, u32p]
            lib.orc_set_state.argtypes = [P, C.c_int, C.c_int64, dp, dp, u32p, C.c_uint32]
            lib.orc_get_cells.argtypes = [P, C.c_int, ip, ip, ip, i64p]
            lib.orc_get_cell_state.argtypes = [P, C.c_int, dp, dp]
            lib.orc_set_cell_state.argtypes = [P, C.c_int, dp, dp]
            lib.orc_sample.argtypes = [P, C.c_int, dp]
            lib.orc_get_stats.argtypes = [P, C.c_int, C.POINTER(Stats)]
            lib.orc_run_ensemble.argtypes = [C.POINTER(Config), C.c_int, C.c_double, C.c_int,
                                             ip, C.c_int, C.c_uint64, C.c_int, dp,
                                             C.POINTER(Stats)]
            lib.orc_run_ensemble_part.argtypes = [C.POINTER(Config), C.c_uint32, C.c_int, C.c_int,
                                                  C.c_double, C.c_int, ip, C.c_int, C.c_uint64,
                                                  C.c_int, dp, C.POINTER(Stats)]
            lib.orc_run_ensemble_windows.argtypes = [C.POINTER(Config), C.c_uint32, C.c_int,
                                                     C.c_int, C.c_double, C.c_int, ip, ip,
                                                     C.c_int, C.c_uint64, C.c_int, dp,
                                                     C.POINTER(Stats)]
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def make_config(w, gas_override=None):
    """Marshal a workload dict (paper_cs_9902024_gb300.workloads) into the
    oracle's own config struct."""
    cfg = Config()
    cfg.dim = w["dim"]
    for a in range(3):
        cfg.ncell[a] = w["ncell"][a]
        cfg.L[a] = w["L"][a]
    g = dict(w["gas"])
    if gas_override:
        g.update(gas_override)
    cfg.mass, cfg.d_ref, cfg.T_ref = g["mass"], g["d_ref"], g["T_ref"]
    cfg.omega, cfg.F_N = g["omega"], g["F_N"]
    cfg.partner, cfg.n_sub = g.get("partner", 0), g.get("n_sub", 1)
    f = w["fill"]
    cfg.fill = f["kind"]
    cfg.fill_n, cfg.fill_T = f["n"], f["T"]
    for a in range(3):
        cfg.fill_U[a] = f["U"][a]
    if len(w["bcs"]) > MAX_BC:
        raise ValueError("too many boundary segments")
    cfg.n_bc = len(w["bcs"])
    for q, b in enumerate(w["bcs"]):
        s = cfg.bc[q]
        s.kind, s.face = b["kind"], b["face"]
        for k in range(2):
            s.lo[k], s.hi[k] = b["lo"][k], b["hi"][k]
        s.step_from, s.step_to = b["step_from"], b["step_to"]
        s.plate_axis, s.plate_index = b["plate_axis"], b["plate_index"]
        s.n, s.T = b["n"], b["T"]
        for a in range(3):
            s.U[a] = b["U"][a]
    return cfg


def ncells_of(w):
    n = w["ncell"]
    return n[0] * n[1] * (n[2] if w["dim"] == 3 else 1)


def philox(ctr, key):
    lib = oracle_lib()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def draw(seed, run, step, entity, purpose, sub):
    u = np.zeros(4)
    oracle_lib().orc_draw(seed, run, step, entity, purpose, sub, _ptr(u, C.c_double))
    return u


def inflow_flux(n, T, Un, m):
    return oracle_lib().orc_inflow_flux(n, T, Un, m)


def sample_xi(s, seed, run, step, e, k):
    xi = C.c_double()
    used = oracle_lib().orc_sample_xi(s, seed, run, step, e, k, C.byref(xi))
    return xi.value, used


def sigma_cr(w, g, gas_override=None):
    cfg = make_config(w, gas_override)
    return oracle_lib().orc_sigma_cr(C.byref(cfg), g)


def partner(w, cell, x, i, u1):
    """The second particle of an NTC candidate whose first is i, for the
    particles of `cell` at absolute positions x (N x 3, LCR order)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    cfg = make_config(w)
    return int(oracle_lib().orc_partner(C.byref(cfg), int(cell), _ptr(x, C.c_double),
                                        len(x), int(i), float(u1)))


def scatter(v1, v2, u3, u4):
    a = np.array(v1, dtype=np.float64)
    b = np.array(v2, dtype=np.float64)
    oracle_lib().orc_scatter(_ptr(a, C.c_double), _ptr(b, C.c_double), u3, u4)
    return a, b


class Oracle:
    """Step-level access to the oracle: one context holds n runs."""

    def __init__(self, w, runs=None, dt=None, seed=None, gas_override=None):
        self.lib = oracle_lib()
        self.w = w
        self.cfg = make_config(w, gas_override)
        self.runs = runs if runs is not None else w["runs"]
        self.dt = dt if dt is not None else w["dt"]
        self.seed = seed if seed is not None else w["seed"]
        self.ncells = ncells_of(w)
        self.h = self.lib.orc_create(C.byref(self.cfg), self.runs, self.dt, self.seed)
        if not self.h:
            raise ValueError("orc_create rejected the configuration")

    def close(self):
        if self.h:
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            raise RuntimeError("%s failed (%d)" % (what, rc))

    def init_run(self, run):
        self._check(self.lib.orc_init_run(self.h, run), "orc_init_run")

    def step(self, run, step):
        self._check(self.lib.orc_step(self.h, run, step), "orc_step")

    def count(self, run):
        return int(self.lib.orc_count(self.h, run))

    def next_id(self, run):
        return int(self.lib.orc_next_id(self.h, run))

    def get_state(self, run):
        n = self.count(run)
        x = np.zeros((max(n, 1), 3))
        v = np.zeros((max(n, 1), 3))
        ids = np.zeros(max(n, 1), dtype=np.uint32)
        self._check(self.lib.orc_get_state(self.h, run, _ptr(x, C.c_double),
                                           _ptr(v, C.c_double), _ptr(ids, C.c_uint32)),
                    "orc_get_state")
        return x[:n], v[:n], ids[:n]

    def set_state(self, run, x, v, ids, next_id):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        n = len(ids)
        if n == 0:
            x = np.zeros((1, 3)); v = np.zeros((1, 3)); ids = np.zeros(1, dtype=np.uint32)
        self._check(self.lib.orc_set_state(self.h, run, n, _ptr(x, C.c_double),
                                           _ptr(v, C.c_double), _ptr(ids, C.c_uint32),
                                           next_id), "orc_set_state")

    def get_cells(self, run):
        nc = self.ncells
        count = np.zeros(nc, dtype=np.int32)
        cand = np.zeros(nc, dtype=np.int32)
        acc = np.zeros(nc, dtype=np.int32)
        lcr = np.zeros(max(self.count(run), 1), dtype=np.int64)
        self._check(self.lib.orc_get_cells(self.h, run, _ptr(count, C.c_int32),
                                           _ptr(cand, C.c_int32), _ptr(acc, C.c_int32),
                                           _ptr(lcr, C.c_int64)), "orc_get_cells")
        return count, cand, acc, lcr[:self.count(run)]

    def get_cell_state(self, run):
        rem = np.zeros(self.ncells)
        smax = np.zeros(self.ncells)
        self._check(self.lib.orc_get_cell_state(self.h, run, _ptr(rem, C.c_double),
                                                _ptr(smax, C.c_double)), "orc_get_cell_state")
        return rem, smax

    def set_cell_state(self, run, rem, smax):
        rem = np.ascontiguousarray(rem, dtype=np.float64)
        smax = np.ascontiguousarray(smax, dtype=np.float64)
        self._check(self.lib.orc_set_cell_state(self.h, run, _ptr(rem, C.c_double),
                                                _ptr(smax, C.c_double)), "orc_set_cell_state")

    def sample(self, run):
        mom = np.zeros((self.ncells, NMOM))
        self._check(self.lib.orc_sample(self.h, run, _ptr(mom, C.c_double)), "orc_sample")
        return mom

    def stats(self, run):
        s = Stats()
        self._check(self.lib.orc_get_stats(self.h, run, C.byref(s)), "orc_get_stats")
        return s.as_dict()


def run_ensemble(w, runs=None, steps=None, sample_steps=None, seed=None,
                 threads=1, dt=None, gas_override=None, run0=0, groups=None, windows=None):
    """Whole ensemble through the oracle.  Returns (acc, stats) with
    acc[t, g, cell, k] the group sums (g = run mod G, G = min(runs, 16)).
    With run0 / groups: the runs with global indices run0 .. run0 + runs - 1
    of a larger ensemble whose group count is `groups`.  With windows =
    [(first, last), ...]: time-averaged samples over those step ranges."""
    lib = oracle_lib()
    cfg = make_config(w, gas_override)
    runs = runs if runs is not None else w["runs"]
    steps = steps if steps is not None else w["steps"]
    ss = np.asarray(sample_steps if sample_steps is not None else w["sample_steps"],
                    dtype=np.int32)
    seed = seed if seed is not None else w["seed"]
    dt = dt if dt is not None else w["dt"]
    G = min(runs, 16) if groups is None else groups
    if windows is not None:
        fi = np.ascontiguousarray([a for a, _ in windows], dtype=np.int32)
        la = np.ascontiguousarray([b for _, b in windows], dtype=np.int32)
    else:
        fi = la = ss
    nc = ncells_of(w)
    acc = np.zeros((len(fi), G, nc, NMOM))
    st = Stats()
    rc = lib.orc_run_ensemble_windows(C.byref(cfg), run0, runs, G, dt, steps,
                                      _ptr(fi, C.c_int32), _ptr(la, C.c_int32), len(fi), seed,
                                      threads, _ptr(acc, C.c_double), C.byref(st))
    if rc != 0:
        raise RuntimeError("orc_run_ensemble failed (%d)" % rc)
    return acc, st.as_dict()


def macro_from_acc(acc, w, runs):
    """Density, velocity and temperature per (sample, cell) from the pooled
    group sums, with batch-means standard errors over the G groups:
        n = sum N * F_N / (runs * Vc),  u = sum v / sum N,
        T = m / (3k) * (sum |v|^2 / sum N - |u|^2).
    Cells with no particles give NaN."""
    gas = w["gas"]
    d = [w["L"][a] / w["ncell"][a] for a in range(3)]
    Vc = d[0] * d[1] * d[2]
    T_, G = acc.shape[0], acc.shape[1]
    grp_runs = np.array([len(range(g, runs, G)) for g in range(G)], dtype=np.float64)

    def est(s, nr):
        N = s[..., 0]
        with np.errstate(invalid="ignore", divide="ignore"):
            dens = N * gas["F_N"] / (nr * Vc)
            vel = s[..., 1:4] / N[..., None]
            c2 = (s[..., 4] + s[..., 5] + s[..., 6]) / N
            temp = gas["mass"] / (3.0 * KB) * (c2 - (vel ** 2).sum(-1))
        return dens, vel, temp

    pooled = acc.sum(axis=1)
    dens, vel, temp = est(pooled, float(runs))
    gd, gv, gt = est(acc, grp_runs[None, :, None])
    sq = np.sqrt(G)
    with np.errstate(invalid="ignore"):
        se_d = np.nanstd(gd, axis=1, ddof=1) / sq if G > 1 else np.full_like(dens, np.nan)
        se_v = np.nanstd(gv, axis=1, ddof=1) / sq if G > 1 else np.full_like(vel, np.nan)
        se_t = np.nanstd(gt, axis=1, ddof=1) / sq if G > 1 else np.full_like(temp, np.nan)
    return dict(density=dens, velocity=vel, temperature=temp,
                se_density=se_d, se_velocity=se_v, se_temperature=se_t)
