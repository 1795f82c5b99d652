"""Python binding of libdsmc.so (ctypes): argument marshalling only.

Every step of the DSMC path runs in the library's CUDA kernels; this module
converts a workload description into the C structs of include/dsmc.h, hands
PyTorch's caching allocator to the library as its device-memory callbacks,
and copies results into numpy arrays.  There is no CPU fallback: without the
compiled library or a CUDA device every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdsmc.so")

OK, E_INVALID, E_OOM, E_CUDA, E_CAPACITY, E_TIMEOUT, E_STATE = range(7)
MODE_BATCHED, MODE_PLAIN = 0, 1
FP32, FP64 = 0, 1
Q_RAW, Q_DENSITY, Q_VELOCITY, Q_TEMPERATURE, Q_SE_DENSITY, Q_SE_VELOCITY, Q_SE_TEMPERATURE = range(7)
NMOM = 7
MAX_BC = 32
KERNEL_KINDS = ["generate", "move", "scan", "scatter", "cell", "cell_big", "reduce", "other",
                "collide", "collide_big"]

EXPORTS = [
    "dsmc_create", "dsmc_run_ensemble", "dsmc_get_samples", "dsmc_get_stats", "dsmc_destroy",
    "dsmc_last_error", "dsmc_debug_begin", "dsmc_debug_step", "dsmc_debug_get_state",
    "dsmc_debug_set_state", "dsmc_debug_get_cells", "dsmc_debug_get_cell_state",
    "dsmc_debug_set_cell_state", "dsmc_debug_sample", "dsmc_debug_philox",
    "dsmc_run_ensemble_noalloc", "dsmc_debug_timeout_probe", "dsmc_run_ensemble_windows",
    "dsmc_mixed_create", "dsmc_mixed_run", "dsmc_mixed_get_stats", "dsmc_mixed_last_error",
    "dsmc_mixed_destroy",
]
MIXED_PROFILE, MIXED_NO_GRAPH = 1, 2


class DsmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dsmc status %d: %s" % (status, msg))
        self.status = status


class Domain(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("dim", C.c_int32), ("extent", C.c_double * 3),
                ("fill", C.c_int32), ("fill_n", C.c_double), ("fill_T", C.c_double),
                ("fill_U", C.c_double * 3)]


class Cells(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("n", C.c_int32 * 3)]


class Gas(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("mass", C.c_double), ("d_ref", C.c_double),
                ("T_ref", C.c_double), ("omega", C.c_double), ("F_N", C.c_double),
                ("partner", C.c_int32), ("n_sub", C.c_int32)]


class Boundary(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("kind", C.c_int32), ("face", C.c_int32),
                ("lo", C.c_int32 * 2), ("hi", C.c_int32 * 2), ("step_from", C.c_int32),
                ("step_to", C.c_int32), ("plate_axis", C.c_int32), ("plate_index", C.c_int32),
                ("n", C.c_double), ("T", C.c_double), ("U", C.c_double * 3)]


# entries of dsmc_options.shape / dsmc_stats.shape
SHAPE_KEYS = ("move_blocks", "scatter_blocks", "tile_budget", "collide_blocks")

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("mode", C.c_int32), ("precision", C.c_int32),
                ("capacity_factor", C.c_double), ("capacity_per_run", C.c_int64),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("stream", C.c_void_p), ("use_graph", C.c_int32), ("debug", C.c_int32),
                ("device", C.c_int32), ("profile", C.c_int32), ("run_offset", C.c_int64),
                ("autotune", C.c_int32), ("shape", C.c_int32 * 4), ("checks", C.c_int32),
                ("reserved_", C.c_int32), ("tune_cache", C.c_char_p)]
TUNE_OFF, TUNE_SEARCH, TUNE_LOAD = 0, 1, 2


class Stats(C.Structure):
    _fields_ = [("struct_size", C.c_uint32)] + [(k, C.c_uint64) for k in (
        "particle_steps", "generated", "removed", "wall_hits", "candidates", "collisions",
        "clamps", "bounce_limit", "reject_limit", "pool_steps")] + [
        ("error_word", C.c_uint32), ("steps_done", C.c_int32), ("particles_now", C.c_int64),
        ("capacity", C.c_int64), ("ms_steps", C.c_double), ("ms_kernel", C.c_double * 12),
        ("launches_kernel", C.c_int64 * 12), ("h2d_bytes", C.c_uint64), ("d2h_bytes", C.c_uint64),
        ("shape", C.c_int32 * 4), ("tuned", C.c_int32), ("big_pool_steps", C.c_uint64)]


_lib = None
_lock = threading.Lock()


def load_library(path=LIB_PATH):
    """Load libdsmc.so (built by paper_cs_9902024_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise DsmcError(E_STATE, "libdsmc.so not built (run paper_cs_9902024_gb300.build)")
        lib = C.CDLL(path)
        P, dp, ip, u32p, i64p = (C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_uint32), C.POINTER(C.c_int64))
        lib.dsmc_create.argtypes = [C.POINTER(Domain), C.POINTER(Cells), C.POINTER(Gas),
                                    C.POINTER(Boundary), C.c_int, C.POINTER(Options), C.POINTER(P)]
        lib.dsmc_run_ensemble.argtypes = [P, C.c_int, C.c_double, C.c_int, ip, C.c_int, C.c_uint64]
        lib.dsmc_get_samples.argtypes = [P, C.c_int, C.c_int, dp, C.c_size_t]
        lib.dsmc_get_stats.argtypes = [P, C.POINTER(Stats)]
        lib.dsmc_destroy.argtypes = [P]
        lib.dsmc_destroy.restype = None
        lib.dsmc_last_error.argtypes = [P]
        lib.dsmc_last_error.restype = C.c_char_p
        lib.dsmc_debug_begin.argtypes = [P, C.c_int, C.c_double, C.c_uint64]
        lib.dsmc_debug_step.argtypes = [P, C.c_int]
        lib.dsmc_debug_get_state.argtypes = [P, C.c_int, dp, dp, u32p, C.c_int64, i64p]
        lib.dsmc_debug_set_state.argtypes = [P, C.c_int, C.c_int64, dp, dp, u32p, C.c_uint32]
        lib.dsmc_debug_get_cells.argtypes = [P, C.c_int, ip, ip, ip, i64p, C.c_int64]
        lib.dsmc_debug_get_cell_state.argtypes = [P, C.c_int, dp, dp]
        lib.dsmc_debug_set_cell_state.argtypes = [P, C.c_int, dp, dp]
        lib.dsmc_debug_sample.argtypes = [P, C.c_int, dp]
        lib.dsmc_debug_philox.argtypes = [C.c_int64, u32p, u32p, u32p]
        lib.dsmc_debug_timeout_probe.argtypes = [P, C.c_uint32]
        lib.dsmc_run_ensemble_windows.argtypes = [P, C.c_int, C.c_double, C.c_int, ip, ip, C.c_int,
                                                  C.c_uint64]
        lib.dsmc_run_ensemble_noalloc.argtypes = [P, C.c_int, C.c_double, C.c_int, ip, C.c_int,
                                                  C.c_uint64, dp, C.c_size_t]
        lib.dsmc_mixed_create.argtypes = [C.POINTER(P), C.c_int, C.c_int, C.POINTER(P)]
        lib.dsmc_mixed_run.argtypes = [P, ip, C.c_double, C.c_int, ip, C.c_int, C.c_uint64]
        lib.dsmc_mixed_get_stats.argtypes = [P, C.POINTER(Stats)]
        lib.dsmc_mixed_last_error.argtypes = [P]
        lib.dsmc_mixed_last_error.restype = C.c_char_p
        lib.dsmc_mixed_destroy.argtypes = [P]
        lib.dsmc_mixed_destroy.restype = None
        for name in EXPORTS:
            getattr(lib, name).restype = getattr(lib, name).restype if name in (
                "dsmc_destroy", "dsmc_last_error", "dsmc_mixed_last_error",
                "dsmc_mixed_destroy") else C.c_int
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _structs(w):
    dom = Domain(struct_size=C.sizeof(Domain), dim=w["dim"])
    for a in range(3):
        dom.extent[a] = w["L"][a]
    f = w["fill"]
    dom.fill, dom.fill_n, dom.fill_T = f["kind"], f["n"], f["T"]
    for a in range(3):
        dom.fill_U[a] = f["U"][a]
    cells = Cells(struct_size=C.sizeof(Cells))
    for a in range(3):
        cells.n[a] = w["ncell"][a] if a < w["dim"] else 1
    g = w["gas"]
    gas = Gas(struct_size=C.sizeof(Gas), mass=g["mass"], d_ref=g["d_ref"], T_ref=g["T_ref"],
              omega=g["omega"], F_N=g["F_N"], partner=g.get("partner", 0),
              n_sub=g.get("n_sub", 1))
    nb = len(w["bcs"])
    if nb > MAX_BC:
        raise DsmcError(E_INVALID, "too many boundary segments")
    arr = (Boundary * max(nb, 1))()
    for q, b in enumerate(w["bcs"]):
        s = arr[q]
        s.struct_size = C.sizeof(Boundary)
        s.kind, s.face = b["kind"], b["face"]
        for k in range(2):
            s.lo[k], s.hi[k] = b["lo"][k], b["hi"][k]
        s.step_from, s.step_to = b["step_from"], b["step_to"]
        s.plate_axis, s.plate_index = b["plate_axis"], b["plate_index"]
        s.n, s.T = b["n"], b["T"]
        for a in range(3):
            s.U[a] = b["U"][a]
    return dom, cells, gas, arr, nb


class Ensemble:
    """One problem (geometry, gas, boundaries) on one GPU.

    `mode`: "batched" (all runs per launch, CUDA graphs) or "plain" (one run
    after another); `precision`: "fp32" or "fp64" particle state;
    `autotune`: True (or "search") searches the launch shape on the first
    run of a size, "load" takes it from the file `tune_cache` (searching
    and storing it there when absent); `shape`: a dict with any of
    SHAPE_KEYS replacing the default launch shape (e.g. stats()["shape"] of
    a tuned ensemble); `checks`: verify the pool after every run."""

    def __init__(self, w, mode="batched", precision="fp32", capacity_factor=0.0,
                 capacity_per_run=0, debug=False, profile=False, use_graph=True, device=0,
                 torch_memory=True, stream=None, run_offset=0, autotune=False,
                 shape=None, checks=False, tune_cache=None):
        import torch  # device memory and streams only
        if not torch.cuda.is_available():
            raise DsmcError(E_CUDA, "no CUDA device: the DSMC path has no CPU fallback")
        self.lib = load_library()
        self.w = w
        self.device = device
        self.ncells = int(np.prod([w["ncell"][a] if a < w["dim"] else 1 for a in range(3)]))
        self._tensors = {}
        self._torch = torch
        opt = Options(struct_size=C.sizeof(Options))
        opt.mode = MODE_PLAIN if mode == "plain" else MODE_BATCHED
        opt.precision = FP64 if precision == "fp64" else FP32
        opt.capacity_factor = capacity_factor
        opt.capacity_per_run = capacity_per_run
        opt.use_graph = 1 if use_graph else 0
        opt.debug = 1 if debug else 0
        opt.profile = 1 if profile else 0
        opt.device = device
        opt.run_offset = run_offset
        opt.autotune = (TUNE_LOAD if autotune == "load" else
                        TUNE_SEARCH if autotune else TUNE_OFF)
        opt.checks = 1 if checks else 0
        self._tune_cache = tune_cache.encode() if tune_cache else None
        opt.tune_cache = self._tune_cache
        if shape:
            for i, k in enumerate(SHAPE_KEYS):
                opt.shape[i] = int(shape.get(k, 0))
        if torch_memory:
            dev = torch.device("cuda", device)

            def _alloc(nbytes, user, strm):
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
                p = t.data_ptr()
                self._tensors[p] = t
                return p

            def _free(p, nbytes, user, strm):
                self._tensors.pop(p, None)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            opt.alloc = self._alloc_cb
            opt.free = self._free_cb
        if stream is None:
            self.stream = torch.cuda.Stream(device=device)
        else:
            self.stream = stream
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        self._opt = opt
        dom, cells, gas, arr, nb = _structs(w)
        h = C.c_void_p()
        st = self.lib.dsmc_create(C.byref(dom), C.byref(cells), C.byref(gas), arr, nb,
                                  C.byref(opt), C.byref(h))
        if st != OK:
            raise DsmcError(st, "dsmc_create failed")
        self.h = h
        self.runs = None
        self.n_samples = 0

    # -- helpers ---------------------------------------------------------
    def _check(self, st, what):
        if st != OK:
            msg = self.lib.dsmc_last_error(self.h)
            raise DsmcError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dsmc_destroy(self.h)
            self.h = None
            self._tensors.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- main entry points -------------------------------------------------
    def run(self, runs=None, steps=None, sample_steps=None, seed=None, dt=None, windows=None):
        """dsmc_run_ensemble, or with windows=[(first, last), ...]
        dsmc_run_ensemble_windows (time-averaged samples)."""
        w = self.w
        runs = w["runs"] if runs is None else runs
        steps = w["steps"] if steps is None else steps
        seed = w["seed"] if seed is None else seed
        dt = w["dt"] if dt is None else dt
        if windows is not None:
            fi = np.ascontiguousarray([a for a, _ in windows], dtype=np.int32)
            la = np.ascontiguousarray([b for _, b in windows], dtype=np.int32)
            n = len(fi)
            st = self.lib.dsmc_run_ensemble_windows(
                self.h, runs, dt, steps, _ptr(fi, C.c_int32) if n else None,
                _ptr(la, C.c_int32) if n else None, n, seed)
            self._check(st, "dsmc_run_ensemble_windows")
        else:
            ss = np.ascontiguousarray(w["sample_steps"] if sample_steps is None else sample_steps,
                                      dtype=np.int32)
            n = len(ss)
            st = self.lib.dsmc_run_ensemble(self.h, runs, dt, steps,
                                            _ptr(ss, C.c_int32) if n else None, n, seed)
            self._check(st, "dsmc_run_ensemble")
        self.runs = runs
        self.n_samples = n
        return self

    def run_noalloc(self, runs=None, steps=None, sample_steps=None, seed=None, dt=None):
        """dsmc_run_ensemble_noalloc: the run inside the library's fixed device
        scratch (no device allocation); returns the group sums of every
        sample, shape (samples, G, ncells, 7)."""
        w = self.w
        runs = w["runs"] if runs is None else runs
        steps = w["steps"] if steps is None else steps
        ss = np.ascontiguousarray(w["sample_steps"] if sample_steps is None else sample_steps,
                                  dtype=np.int32)
        seed = w["seed"] if seed is None else seed
        dt = w["dt"] if dt is None else dt
        G = min(runs, 16)
        out = np.zeros((max(len(ss), 1), G, self.ncells, NMOM))
        st = self.lib.dsmc_run_ensemble_noalloc(self.h, runs, dt, steps,
                                                _ptr(ss, C.c_int32) if len(ss) else None, len(ss),
                                                seed, _ptr(out, C.c_double), out.size)
        self._check(st, "dsmc_run_ensemble_noalloc")
        return out[:len(ss)]

    def raw(self, t):
        G = min(self.runs, 16)
        out = np.empty((G, self.ncells, NMOM))
        self._check(self.lib.dsmc_get_samples(self.h, t, Q_RAW, _ptr(out, C.c_double), out.size),
                    "dsmc_get_samples")
        return out

    def quantity(self, t, q):
        width = 3 if q in (Q_VELOCITY, Q_SE_VELOCITY) else 1
        out = np.empty((self.ncells, width))
        self._check(self.lib.dsmc_get_samples(self.h, t, q, _ptr(out, C.c_double), out.size),
                    "dsmc_get_samples")
        return out[:, 0] if width == 1 else out

    def macro(self, t):
        return dict(density=self.quantity(t, Q_DENSITY), velocity=self.quantity(t, Q_VELOCITY),
                    temperature=self.quantity(t, Q_TEMPERATURE),
                    se_density=self.quantity(t, Q_SE_DENSITY),
                    se_velocity=self.quantity(t, Q_SE_VELOCITY),
                    se_temperature=self.quantity(t, Q_SE_TEMPERATURE))

    def stats(self):
        s = Stats(struct_size=C.sizeof(Stats))
        self._check(self.lib.dsmc_get_stats(self.h, C.byref(s)), "dsmc_get_stats")
        return _stats_dict(s)

    # -- test hooks ------------------------------------------------------
    def debug_begin(self, runs=None, dt=None, seed=None):
        w = self.w
        runs = w["runs"] if runs is None else runs
        self._check(self.lib.dsmc_debug_begin(self.h, runs, w["dt"] if dt is None else dt,
                                              w["seed"] if seed is None else seed),
                    "dsmc_debug_begin")
        self.runs = runs

    def debug_timeout_probe(self, polls=64):
        """dsmc_debug_timeout_probe: returns the status (E_TIMEOUT expected)."""
        return self.lib.dsmc_debug_timeout_probe(self.h, polls)

    def debug_step(self, n=1):
        self._check(self.lib.dsmc_debug_step(self.h, n), "dsmc_debug_step")

    def get_state(self, run):
        n = C.c_int64()
        self._check(self.lib.dsmc_debug_get_state(self.h, run, None, None, None, 0, C.byref(n)),
                    "dsmc_debug_get_state")
        m = max(n.value, 1)
        x = np.zeros((m, 3)); v = np.zeros((m, 3)); ids = np.zeros(m, dtype=np.uint32)
        self._check(self.lib.dsmc_debug_get_state(self.h, run, _ptr(x, C.c_double),
                                                  _ptr(v, C.c_double), _ptr(ids, C.c_uint32),
                                                  m, C.byref(n)), "dsmc_debug_get_state")
        k = n.value
        return x[:k], v[:k], ids[:k]

    def set_state(self, run, x, v, ids, next_id):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        self._check(self.lib.dsmc_debug_set_state(self.h, run, len(ids), _ptr(x, C.c_double),
                                                  _ptr(v, C.c_double), _ptr(ids, C.c_uint32),
                                                  next_id), "dsmc_debug_set_state")

    def get_cells(self, run):
        nc = self.ncells
        count = np.zeros(nc, dtype=np.int32)
        cand = np.zeros(nc, dtype=np.int32)
        acc = np.zeros(nc, dtype=np.int32)
        self._check(self.lib.dsmc_debug_get_cells(self.h, run, _ptr(count, C.c_int32), None, None,
                                                  None, 0), "dsmc_debug_get_cells")
        n = int(count.sum())
        lcr = np.zeros(max(n, 1), dtype=np.int64)
        self._check(self.lib.dsmc_debug_get_cells(self.h, run, _ptr(count, C.c_int32),
                                                  _ptr(cand, C.c_int32), _ptr(acc, C.c_int32),
                                                  _ptr(lcr, C.c_int64), n), "dsmc_debug_get_cells")
        return count, cand, acc, lcr[:n]

    def get_cell_state(self, run):
        rem = np.zeros(self.ncells); smax = np.zeros(self.ncells)
        self._check(self.lib.dsmc_debug_get_cell_state(self.h, run, _ptr(rem, C.c_double),
                                                       _ptr(smax, C.c_double)),
                    "dsmc_debug_get_cell_state")
        return rem, smax

    def set_cell_state(self, run, rem, smax):
        rem = np.ascontiguousarray(rem, dtype=np.float64)
        smax = np.ascontiguousarray(smax, dtype=np.float64)
        self._check(self.lib.dsmc_debug_set_cell_state(self.h, run, _ptr(rem, C.c_double),
                                                       _ptr(smax, C.c_double)),
                    "dsmc_debug_set_cell_state")

    def sample_now(self, run):
        mom = np.zeros((self.ncells, NMOM))
        self._check(self.lib.dsmc_debug_sample(self.h, run, _ptr(mom, C.c_double)),
                    "dsmc_debug_sample")
        return mom


def philox_gpu(ctr, key):
    """The library's device Philox4x32-10 on (n, 4) counters and (n, 2) keys."""
    lib = load_library()
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(c)
    st = lib.dsmc_debug_philox(len(c), _ptr(c, C.c_uint32), _ptr(k, C.c_uint32),
                               _ptr(out, C.c_uint32))
    if st != OK:
        raise DsmcError(st, "dsmc_debug_philox failed")
    return out


def _stats_dict(s):
    d = {k: getattr(s, k) for k, _ in Stats._fields_
         if k not in ("ms_kernel", "launches_kernel", "shape")}
    d["shape"] = {k: s.shape[i] for i, k in enumerate(SHAPE_KEYS)}
    d["ms_kernel"] = {KERNEL_KINDS[i]: s.ms_kernel[i] for i in range(len(KERNEL_KINDS))}
    d["launches_kernel"] = {KERNEL_KINDS[i]: int(s.launches_kernel[i])
                            for i in range(len(KERNEL_KINDS))}
    return d


class MixedEnsemble:
    """A mixed-size ensemble (workloads.mixed): the runs that share a grid
    form one part (a context; its runs' global indices through
    run_offset).  mode "single" (default): every time step is one launch
    per kernel kind over all parts (dsmc_mixed_run), the CTAs claiming
    (part, tile) work items from device counters.  mode "concurrent": one
    batched context per part, all advanced at once from one host thread
    and one CUDA stream each (the GPU's block scheduler sharing the SMs).
    Both give every part the samples dsmc_run_ensemble gives it alone."""

    def __init__(self, m, precision="fp32", device=0, mode="single", profile=False,
                 use_graph=True, **kw):
        import torch
        self.m = m
        self.mode = mode
        self.parts = []
        self.lib = load_library()
        self.h = None
        for w in m["groups"]:
            stream = torch.cuda.Stream(device=device) if mode == "concurrent" else None
            if mode != "concurrent" and self.parts:
                stream = self.parts[0].stream
            self.parts.append(Ensemble(w, precision=precision, device=device, stream=stream,
                                       run_offset=w["run0"], **kw))
        if mode == "single":
            arr = (C.c_void_p * len(self.parts))(*[e.h.value for e in self.parts])
            h = C.c_void_p()
            flags = (MIXED_PROFILE if profile else 0) | (0 if use_graph else MIXED_NO_GRAPH)
            st = self.lib.dsmc_mixed_create(arr, len(self.parts), flags, C.byref(h))
            if st != OK:
                raise DsmcError(st, "dsmc_mixed_create failed")
            self.h = h

    def run(self, steps=None, sample_steps=None, seed=None):
        w0 = self.m["groups"][0]
        if self.mode == "concurrent":
            from concurrent.futures import ThreadPoolExecutor
            with ThreadPoolExecutor(max_workers=len(self.parts)) as ex:
                for f in [ex.submit(e.run, steps=steps, sample_steps=sample_steps, seed=seed)
                          for e in self.parts]:
                    f.result()
            return self
        steps = w0["steps"] if steps is None else steps
        ss = np.ascontiguousarray(w0["sample_steps"] if sample_steps is None else sample_steps,
                                  dtype=np.int32)
        seed = w0["seed"] if seed is None else seed
        runs = np.ascontiguousarray([w["runs"] for w in self.m["groups"]], dtype=np.int32)
        st = self.lib.dsmc_mixed_run(self.h, _ptr(runs, C.c_int32), w0["dt"], steps,
                                     _ptr(ss, C.c_int32) if len(ss) else None, len(ss), seed)
        if st != OK:
            msg = self.lib.dsmc_mixed_last_error(self.h)
            raise DsmcError(st, "dsmc_mixed_run: %s" % (msg.decode() if msg else ""))
        for e, w in zip(self.parts, self.m["groups"]):
            e.runs = w["runs"]
            e.n_samples = len(ss)
        return self

    def raw(self, group, t):
        return self.parts[group].raw(t)

    def macro(self, group, t):
        return self.parts[group].macro(t)

    def mixed_stats(self):
        """Totals of the last single-launch run (device time of its step
        loop; per-kernel times in profile mode)."""
        s = Stats(struct_size=C.sizeof(Stats))
        st = self.lib.dsmc_mixed_get_stats(self.h, C.byref(s))
        if st != OK:
            raise DsmcError(st, "dsmc_mixed_get_stats failed")
        return _stats_dict(s)

    def stats(self):
        per = [e.stats() for e in self.parts]
        keys = ("particle_steps", "generated", "removed", "wall_hits", "candidates", "collisions",
                "particles_now", "pool_steps", "big_pool_steps")
        out = {k: sum(int(s[k]) for s in per) for k in keys}
        out["error_word"] = 0
        for s in per:
            out["error_word"] |= int(s["error_word"])
        out["groups"] = per
        return out

    def close(self):
        if self.h is not None:
            self.lib.dsmc_mixed_destroy(self.h)
            self.h = None
        for e in self.parts:
            e.close()
        self.parts = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
