/*
 * dsmc.h -- C ABI of the GB300 ensemble DSMC library (libdsmc.so).
 *
 * One call advances n statistically independent runs of an unsteady DSMC
 * simulation from t = 0 (the outer loop of the sequential algorithm, Sec. 1.1
 * of Bogdanov et al., "Algorithms of Two-Level Parallelization for DSMC of
 * Unsteady Flows in Molecular Gasdynamics"), every time step made of the
 * inner loop's subroutines (Sec. 1.1, Fig. 1):
 *   Generation   particles enter through inflow boundaries;
 *   Motion       free flight, specular / diffuse surface interaction, leavers
 *                removed from P;
 *   Enumeration, Indexing
 *                particles counted per cell and the readdressing array LCR
 *                built (one entry per particle, ordered by cell);
 *   Interaction  collisions in every cell independently (no-time-counter
 *                candidate count, hard-sphere / VHS cross section);
 *   Sampling     cell macroparameters at the given moments, averaged over
 *                the runs ("ensemble averaging", Sec. 1.1).
 * All runs advance together on one GPU (the paper's independent-runs level,
 * Sec. 1.3, mapped to a batch dimension; its data-parallel level, Sec. 1.4,
 * mapped to GPU threads).
 *
 * Conventions for every entry point:
 *  - Every struct starts with `struct_size` = sizeof(the struct) as the
 *    caller compiled it; a smaller or zero value is rejected with
 *    DSMC_E_INVALID.  The library copies every input struct and array; the
 *    caller keeps ownership of what it passes in.
 *  - Host pointers are plain host memory unless stated otherwise.
 *  - No call throws; errors are returned as dsmc_status and described by
 *    dsmc_last_error(ctx).  A context is used by one host thread at a time.
 *  - Units are SI.  Geometry is a uniform Cartesian grid of n[0] x n[1]
 *    (x n[2]) cells on [0, L_x) x [0, L_y) (x [0, L_z)); cell index
 *    c = i + n[0] * (j + n[1] * k).  In 2-D, n[2] = 1 and extent[2] is the
 *    depth (the third velocity component is carried, not the coordinate).
 */
#ifndef DSMC_H
#define DSMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DSMC_OK = 0,
    DSMC_E_INVALID = 1,    /* bad argument; nothing was changed */
    DSMC_E_OOM = 2,        /* device allocation failed */
    DSMC_E_CUDA = 3,       /* a CUDA call failed (message in last_error) */
    DSMC_E_CAPACITY = 4,   /* particle pool or a per-cell limit overflowed on
                              the device; the run's results are incomplete */
    DSMC_E_TIMEOUT = 5,    /* a bounded device wait expired (DSMC_ERR_TIMEOUT) */
    DSMC_E_STATE = 6       /* call out of order (e.g. samples before a run) */
} dsmc_status;

enum { DSMC_BC_OUTFLOW = 0, DSMC_BC_INFLOW = 1, DSMC_BC_SPECULAR = 2, DSMC_BC_DIFFUSE = 3 };
enum { DSMC_FACE_XMIN = 0, DSMC_FACE_XMAX = 1, DSMC_FACE_YMIN = 2, DSMC_FACE_YMAX = 3,
       DSMC_FACE_ZMIN = 4, DSMC_FACE_ZMAX = 5, DSMC_FACE_PLATE = 6 };
enum { DSMC_MODE_BATCHED = 0, DSMC_MODE_PLAIN = 1 };
enum { DSMC_FP32 = 0, DSMC_FP64 = 1 };
enum { DSMC_TUNE_OFF = 0, DSMC_TUNE_SEARCH = 1, DSMC_TUNE_LOAD = 2 };

typedef enum {
    DSMC_Q_RAW_MOMENTS = 0,        /* [G][ncells][7] group sums, see below */
    DSMC_Q_DENSITY = 1,            /* [ncells]   n (m^-3) */
    DSMC_Q_VELOCITY = 2,           /* [ncells][3] mean velocity (m/s) */
    DSMC_Q_TEMPERATURE = 3,        /* [ncells]   T (K) */
    DSMC_Q_STDERR_DENSITY = 4,     /* [ncells]   batch-means standard errors */
    DSMC_Q_STDERR_VELOCITY = 5,    /* [ncells][3] */
    DSMC_Q_STDERR_TEMPERATURE = 6  /* [ncells] */
} dsmc_quantity;

#define DSMC_NMOM 7     /* N, sum u, sum v, sum w, sum u^2, sum v^2, sum w^2 */
#define DSMC_MAX_BC 32
#define DSMC_MAX_GROUPS 16

/* Computational domain (the array C of Sec. 1.1 is built from it). */
typedef struct {
    uint32_t struct_size;
    int32_t dim;            /* 2 or 3 */
    double extent[3];       /* L_x, L_y, L_z (m); 2-D: extent[2] = depth */
    int32_t fill;           /* 0: start empty; 1: start filled with a uniform
                               freestream (fill_n, fill_T, fill_U) */
    double fill_n, fill_T, fill_U[3];
} dsmc_domain;

typedef struct {
    uint32_t struct_size;
    int32_t n[3];           /* cells per axis; n[2] = 1 in 2-D */
} dsmc_cells;

/* Monatomic gas, variable-hard-sphere model:
 *   sigma_T(c_r) = pi d_ref^2 (2 k T_ref / (m_r c_r^2))^(omega - 1/2)
 *                  / Gamma(5/2 - omega),  m_r = mass / 2;
 * omega = 0.5 is the hard sphere pi d_ref^2.  F_N = real molecules per
 * simulated particle.
 * `partner` chooses the second particle of an NTC candidate pair (the first
 * is uniform over the cell; the paper's Interaction, Sec. 1.1, leaves the
 * pair selection to the gas model):
 *   DSMC_PARTNER_UNIFORM  uniform over the cell's other particles;
 *   DSMC_PARTNER_SUBCELL  uniform over the other particles of the first
 *                         one's subcell -- the cell split into n_sub (1..64)
 *                         equal parts per axis, a particle's subcell per axis
 *                         floor(n_sub * offset / cell size) -- or, if it is
 *                         alone there, uniform over the cell's others;
 *   DSMC_PARTNER_NEAREST  the other particle of the cell nearest to it
 *                         (Euclidean distance over the grid's axes; of equal
 *                         distances the first in LCR order).
 * A caller whose struct_size ends before `partner` gets the uniform choice. */
#define DSMC_PARTNER_UNIFORM 0
#define DSMC_PARTNER_SUBCELL 1
#define DSMC_PARTNER_NEAREST 2
typedef struct {
    uint32_t struct_size;
    double mass, d_ref, T_ref, omega, F_N;
    int32_t partner;        /* DSMC_PARTNER_* */
    int32_t n_sub;          /* subcells per axis (DSMC_PARTNER_SUBCELL) */
} dsmc_gas;

/* One boundary segment.  Faces: 2 * axis + side (side 0 at coordinate 0,
 * side 1 at L).  [lo, hi) are cell ranges along the face's two tangential
 * axes in increasing axis order (2-D: the second range is [0, 1)).  Where
 * several segments cover a face cell at a step, the last listed active one
 * applies; an uncovered face cell is open (outflow).  INFLOW injects a
 * drifting Maxwellian (n, T, U) and removes particles leaving through it;
 * OUTFLOW removes leavers; SPECULAR reflects; DIFFUSE re-emits at T.
 * face = DSMC_FACE_PLATE describes a zero-thickness internal plate normal to
 * `plate_axis` at coordinate plate_index * cell size, covering [lo, hi) of
 * the tangential cells, SPECULAR or DIFFUSE on both sides.  A segment is
 * active for steps step_from..step_to (1-based, inclusive; 0 = forever). */
typedef struct {
    uint32_t struct_size;
    int32_t kind, face;
    int32_t lo[2], hi[2];
    int32_t step_from, step_to;
    int32_t plate_axis, plate_index;
    double n, T, U[3];
} dsmc_boundary;

/* Device memory callbacks (e.g. a framework's caching allocator).  `stream`
 * is the cudaStream_t the memory will be used on.  alloc returns a device
 * pointer aligned to at least 256 bytes, or NULL. */
typedef void* (*dsmc_alloc_fn)(size_t bytes, void* user, void* stream);
typedef void (*dsmc_free_fn)(void* ptr, size_t bytes, void* user, void* stream);

typedef struct {
    uint32_t struct_size;
    int32_t mode;             /* DSMC_MODE_BATCHED: all runs in one launch per
                                 kernel per step (CUDA-graph captured);
                                 DSMC_MODE_PLAIN: one run after another */
    int32_t precision;        /* particle state / collision arithmetic:
                                 DSMC_FP32 or DSMC_FP64 (sampling sums and the
                                 NTC remainder are FP64 in both) */
    double capacity_factor;   /* pool size = factor x estimate (0 -> 1.25) */
    int64_t capacity_per_run; /* > 0 overrides the estimate */
    dsmc_alloc_fn alloc;      /* NULL: cudaMalloc / cudaFree */
    dsmc_free_fn free;
    void* alloc_user;
    void* stream;             /* cudaStream_t; NULL: the library's own stream */
    int32_t use_graph;        /* batched mode: capture one step per graph */
    int32_t debug;            /* keep per-cell candidate / accepted counts,
                                 the LCR of the last step and particle ids
                                 (test hooks; no step reads them, so the
                                 results are the same either way) */
    int32_t device;           /* CUDA device ordinal */
    int32_t profile;          /* time every kernel with CUDA events (direct
                                 launches, no graph); see dsmc_stats */
    int64_t run_offset;       /* global index of run 0 of this context: the
                                 runs draw as runs run_offset.. (sharding an
                                 ensemble over processes or GPUs) */
    int32_t autotune;         /* batched mode, runs of >= 100 steps:
                                 DSMC_TUNE_SEARCH = on the first run of a
                                 problem size, advance a trial ensemble to
                                 mid-run and time candidate launch shapes
                                 (sort/gather tile budget, grid sizes of the
                                 Motion, scatter and collision kernels) over
                                 short windows, keeping the fastest per kernel
                                 time per particle; the real run then starts
                                 from t = 0.  DSMC_TUNE_LOAD = take the shape
                                 stored in the file `tune_cache` for this GPU
                                 and problem (device name, SM count,
                                 precision, grid, runs, steps and a hash of
                                 the domain, gas and boundaries); if there is
                                 none, search as above and append the result
                                 to the file.  Results do not depend on the
                                 shapes.  DSMC_TUNE_OFF = fixed shapes
                                 (default) */
    int32_t shape[4];         /* batched mode: entries > 0 replace the default
                                 launch shape (as dsmc_stats.shape: Motion
                                 CTAs, scatter CTAs, sort/gather tile budget
                                 in particles, collision CTAs), e.g. a shape
                                 an earlier autotune found; 0 keeps the
                                 default.  CTA counts lie in [1, 2^20], the
                                 tile budget in [256, 16384] (rounded up to a
                                 multiple of 8); else DSMC_E_INVALID.  With
                                 autotune the tuned shape replaces it.
                                 Results do not depend on the shape. */
    int32_t checks;           /* 1: after every run a device pass verifies the
                                 final pool -- each particle's cell key inside
                                 the table and its position inside that
                                 cell's range, ids increasing within a cell,
                                 offsets inside the cell, finite velocities;
                                 a failure makes the run return DSMC_E_STATE
                                 with the count and the first failing
                                 position.  0: no check (default) */
    int32_t reserved_;
    const char* tune_cache;   /* DSMC_TUNE_LOAD: path of the launch-shape
                                 cache (a text file of "key shape" lines; the
                                 library reads it and appends to it) */
} dsmc_options;
/* Callers built against an older dsmc_options (without checks and
 * tune_cache: struct_size = offsetof(dsmc_options, checks)) are accepted;
 * the fields they do not have are zero. */

typedef struct {
    uint32_t struct_size;
    uint64_t particle_steps;  /* sum over runs and steps of particles moved */
    uint64_t generated, removed, wall_hits;
    uint64_t candidates, collisions, clamps;   /* NTC counters; clamps: pairs
                                                  with sigma c_r > max */
    uint64_t bounce_limit, reject_limit;       /* numerical guards hit */
    uint64_t pool_steps;      /* sum over steps of the pool size after the
                                 step (particles written by Indexing) */
    uint32_t error_word;      /* device error bits (DSMC_ERR_*) */
    int32_t steps_done;
    int64_t particles_now;    /* particles in all runs after the last step */
    int64_t capacity;         /* particle pool capacity (all runs) */
    double ms_steps;          /* device time of the last run's step loop */
    double ms_kernel[12];     /* profile mode: device time per kernel kind */
    int64_t launches_kernel[12];
    uint64_t h2d_bytes;       /* host -> device bytes of the last run */
    uint64_t d2h_bytes;       /* device -> host bytes since the last run began
                                 (counters at its end plus dsmc_get_samples) */
    int32_t shape[4];         /* launch shape in use: Motion CTAs, scatter
                                 CTAs, sort/gather tile budget (particles),
                                 collision CTAs */
    int32_t tuned;            /* 1: the shape came from an autotune search; 2:
                                 from the tune cache file */
    uint64_t big_pool_steps;  /* the part of pool_steps in cells above 128
                                 particles (ordered and gathered one cell per
                                 CTA) */
} dsmc_stats;

/* device error bits */
#define DSMC_ERR_POOL      0x1u   /* particle pool overflow */
#define DSMC_ERR_GEN       0x2u   /* per-run generation buffer overflow */
#define DSMC_ERR_BIGCELL   0x4u   /* a cell exceeded the per-cell limit */
#define DSMC_ERR_BIGLIST   0x8u   /* too many large cells in one step */
#define DSMC_ERR_TIMEOUT   0x10u  /* a bounded device wait (bulk-copy completion) expired */

/* kernel kinds of dsmc_stats.ms_kernel */
enum { DSMC_K_GENERATE = 0, DSMC_K_MOVE = 1, DSMC_K_SCAN = 2, DSMC_K_SCATTER = 3,
       DSMC_K_CELL = 4, DSMC_K_CELL_BIG = 5, DSMC_K_REDUCE = 6, DSMC_K_OTHER = 7,
       DSMC_K_COLLIDE = 8, DSMC_K_COLLIDE_BIG = 9 };

typedef struct dsmc_ctx dsmc_ctx;

/* Create a context for one problem: domain and grid, gas model, `n_b`
 * boundary segments (n_b <= DSMC_MAX_BC) and options (NULL: defaults) --
 * the data of one unsteady run of the paper's Sec. 1.1 (the computational
 * grid and the arrays P, LCR and C are sized from them at the first run;
 * the boundary conditions drive Generation and Motion).  No device memory
 * is allocated until the first run.  *out receives the context; release it
 * with dsmc_destroy.  Errors: DSMC_E_INVALID (bad geometry, gas or boundary
 * description), DSMC_E_CUDA (device selection). */
dsmc_status dsmc_create(const dsmc_domain* domain, const dsmc_cells* cells,
                        const dsmc_gas* gas, const dsmc_boundary* b, int n_b,
                        const dsmc_options* opt, dsmc_ctx** out);

/* Run n_runs independent runs for `steps` steps of length dt (s) from t = 0.
 * Sample k is taken after step sample_steps[k] (1-based, strictly
 * increasing, <= steps; at most 4096 samples), once Interaction of that step
 * is done.  Run r draws every random number from Philox4x32-10 keyed by
 * `seed` with (r, step, entity, purpose, draw) as the counter, so results do
 * not depend on mode, launch shape or stream.  Blocks until the device is
 * done.  Device memory is owned by the library (through the callbacks) and
 * reused by later calls.  Errors: DSMC_E_INVALID, DSMC_E_OOM, DSMC_E_CUDA,
 * DSMC_E_CAPACITY (results incomplete; rerun with a larger capacity). */
dsmc_status dsmc_run_ensemble(dsmc_ctx* ctx, int n_runs, double dt, int steps,
                              const int32_t* sample_steps, int n_samples,
                              uint64_t seed);

/* dsmc_run_ensemble with time-averaged samples: sample k sums the moments
 * after Interaction of every step first[k] .. last[k] (inclusive) of every
 * run -- the averaging interval dt_av of the unsteady-flow method (Sec. 1.1:
 * macroparameters averaged over an interval short against the flow's time
 * scale and over the n runs); first = last gives dsmc_run_ensemble.  Windows
 * lie in [1, steps], increasing and disjoint (at most 4096).  Each run's
 * sums over a window are formed in step order, then added to the group
 * sums in increasing run order (the same in batched and plain modes).
 * Errors as dsmc_run_ensemble. */
dsmc_status dsmc_run_ensemble_windows(dsmc_ctx* ctx, int n_runs, double dt, int steps,
                                      const int32_t* first, const int32_t* last, int n_windows,
                                      uint64_t seed);

/* Copy sample `sample_idx` of the last run into out[0 .. out_len).  The
 * runs are split into G = min(n_runs, 16) groups (run r in group r mod G);
 * RAW_MOMENTS gives the group sums [G][ncells][7] of N, sum v_a and
 * sum v_a^2; the macroscopic quantities pool all groups:
 *   n = sum N F_N / (n_runs L V_c),  u = sum v / sum N  (L: the sample's
 *   window length in steps, 1 for dsmc_run_ensemble),
 *   T = m / (3 k) (sum |v|^2 / sum N - |u|^2)  (NaN where sum N = 0);
 * STDERR_* are the standard deviations over the G group estimates divided
 * by sqrt(G).  Errors: DSMC_E_INVALID (index or out_len too small),
 * DSMC_E_STATE (no completed run). */
dsmc_status dsmc_get_samples(dsmc_ctx* ctx, int sample_idx, dsmc_quantity q,
                             double* out, size_t out_len);

dsmc_status dsmc_get_stats(dsmc_ctx* ctx, dsmc_stats* out);
void dsmc_destroy(dsmc_ctx* ctx);
/* Message of the last failed call on ctx (static string if ctx is NULL). */
const char* dsmc_last_error(const dsmc_ctx* ctx);

/* Same result as dsmc_run_ensemble followed by dsmc_get_samples(RAW_MOMENTS)
 * for every sample, for callers that may not allocate device memory:
 * a process whose device memory was all handed to another allocator or a
 * fixed budget at start-up (a cudaMalloc there fails or steals from it),
 * or a real-time loop that forbids allocator calls (cudaMalloc/cudaFree
 * can synchronise the device and stall for milliseconds).  No counterpart
 * in the paper: it is a deployment variant of the batched ensemble run.
 *  - The whole run lives in one scratch array that is part of the library's
 *    device image: 48 MiB on every GPU that loads the library, held until
 *    the process exits.  A problem that needs more is rejected with
 *    DSMC_E_INVALID and a message giving the bytes it needs (config-0-sized
 *    ensembles fit; batched-512-run ensembles do not).
 *  - The call makes no cudaMalloc, cudaFree, event or graph call.  Its first
 *    call on a device looks up the scratch array's device address; make
 *    that first call before any stream capture.  (The CUDA driver may also
 *    reserve local-memory backing for a kernel on its first launch.)
 *  - raw_out (host memory, raw_len doubles) receives sample k's group sums
 *    at raw_out[k][G][ncells][7], G = min(n_runs, 16), laid out as
 *    dsmc_get_samples(RAW_MOMENTS) gives them.  The call blocks until done.
 *  - Every call on a device shares the one scratch array: calls whose GPU
 *    work overlaps (several contexts or threads on the same device, or
 *    streams that run concurrently) race and corrupt each other's results.
 *    Each call resets what must start from zero; nothing else carries over.
 *  - ctx must not own device buffers yet (a context that ran
 *    dsmc_run_ensemble or a debug hook: DSMC_E_STATE); options.debug and
 *    options.profile are rejected.  Afterwards dsmc_get_samples has no run
 *    to read (DSMC_E_STATE); dsmc_get_stats reports the call's counters. */
dsmc_status dsmc_run_ensemble_noalloc(dsmc_ctx* ctx, int n_runs, double dt, int steps,
                                      const int32_t* sample_steps, int n_samples,
                                      uint64_t seed, double* raw_out, size_t raw_len);

/* ---- mixed-size ensembles ------------------------------------------- */

/* Several problems advanced together: a mixed-size ensemble whose runs sit
 * on grids of different sizes (one context per grid, its runs one batch).
 * Every time step is one launch per kernel kind over the runs of all
 * parts.  The CTAs of the tile-shaped kernels -- Motion, LCR scatter,
 * sort/gather, collisions -- claim their work items, (part, tile) or
 * (part, chunk of particles), from device counters as they finish earlier
 * ones, so that processors that are done with their share move to runs
 * with work left: the dynamic reallocation of processors between runs of
 * the two-level scheme with dynamic load balancing (Sec. 3, the "heap" of
 * processors handed to parallel sections by their load), with CTAs as the
 * processors.
 *
 * dsmc_mixed_create takes n_parts (1 .. 64) contexts of one device,
 * precision and dimension.  Each keeps its own grid, boundaries, options
 * (capacity, allocator) and run_offset; the mixed ensemble launches on
 * parts[0]'s stream, from its own graphs.  The contexts stay owned by the
 * caller and must outlive the mixed ensemble; they must not be used
 * elsewhere while it runs.  flags: DSMC_MIXED_PROFILE times every kernel
 * kind with CUDA events (direct launches, no graph; dsmc_mixed_get_stats);
 * DSMC_MIXED_NO_GRAPH launches directly.  The launch shape is the default
 * one (no autotune).  Errors: DSMC_E_INVALID (count, NULL part, parts on
 * different devices or with different precision or dimension),
 * DSMC_E_OOM, DSMC_E_CUDA. */
typedef struct dsmc_mixed dsmc_mixed;
#define DSMC_MIXED_PROFILE 1
#define DSMC_MIXED_NO_GRAPH 2
dsmc_status dsmc_mixed_create(dsmc_ctx* const* parts, int n_parts, int flags, dsmc_mixed** out);

/* Run n_runs[i] runs of part i (host array of n_parts entries), every part
 * for the same `steps` steps of length dt with the same sample steps and
 * seed -- what dsmc_run_ensemble(parts[i], n_runs[i], ...) computes for each
 * part alone, bit for bit (a run's draws depend only on its global index
 * run_offset + r and the seed; every sum is formed in the same order).
 * Afterwards dsmc_get_samples and dsmc_get_stats on each part read its
 * samples and counters.  Blocks until the device is done.  Errors: as
 * dsmc_run_ensemble (the failing part's message is copied to
 * dsmc_mixed_last_error). */
dsmc_status dsmc_mixed_run(dsmc_mixed* m, const int32_t* n_runs, double dt, int steps,
                           const int32_t* sample_steps, int n_samples, uint64_t seed);

/* Totals over the parts of the last dsmc_mixed_run: counters summed,
 * ms_steps the device time of its step loop, per-kernel-kind times with
 * DSMC_MIXED_PROFILE, shape the launch shape of the queue-driven kernels. */
dsmc_status dsmc_mixed_get_stats(dsmc_mixed* m, dsmc_stats* out);
const char* dsmc_mixed_last_error(const dsmc_mixed* m);
void dsmc_mixed_destroy(dsmc_mixed* m);

/* ---- test hooks (step-level access for parity tests) ---------------- */

/* Allocate for n_runs and set up the step-0 state (filled or empty) without
 * running a step; the sample list is empty. */
dsmc_status dsmc_debug_begin(dsmc_ctx* ctx, int n_runs, double dt, uint64_t seed);
/* Advance every run by n_steps steps. */
dsmc_status dsmc_debug_step(dsmc_ctx* ctx, int n_steps);
/* Particles of `run` in the current P order (by cell, each cell in LCR
 * order): x[n][3], v[n][3], id[n]; at most cap particles are written,
 * *n_out gets the count. */
dsmc_status dsmc_debug_get_state(dsmc_ctx* ctx, int run, double* x, double* v,
                                 uint32_t* id, int64_t cap, int64_t* n_out);
/* Replace the particles of `run` (any order; this order numbers the slots
 * of the next step's LCR) and its next particle id. */
dsmc_status dsmc_debug_set_state(dsmc_ctx* ctx, int run, int64_t n, const double* x,
                                 const double* v, const uint32_t* id, uint32_t next_id);
/* Last step's per-cell counts, NTC candidates and accepted collisions
 * ([ncells] each; needs options.debug for cand/accepted/lcr) and its LCR:
 * lcr[k] = pre-step slot (old particles 0..n_old-1 in their previous order,
 * then the step's entrants in generation order) of the k-th particle. */
dsmc_status dsmc_debug_get_cells(dsmc_ctx* ctx, int run, int32_t* count, int32_t* cand,
                                 int32_t* accepted, int64_t* lcr, int64_t cap);
dsmc_status dsmc_debug_get_cell_state(dsmc_ctx* ctx, int run, double* rem, double* smax);
dsmc_status dsmc_debug_set_cell_state(dsmc_ctx* ctx, int run, const double* rem,
                                      const double* smax);
/* Moments [ncells][7] of `run`'s current particles (FP64). */
dsmc_status dsmc_debug_sample(dsmc_ctx* ctx, int run, double* mom);
/* The device Philox4x32-10 on n host (ctr[4], key[2]) pairs -> out[4n]. */
dsmc_status dsmc_debug_philox(int64_t n, const uint32_t* ctr, const uint32_t* key,
                              uint32_t* out);

/* Test hook for the bounded device waits (no counterpart in the paper):
 * runs one kernel whose bulk-copy barrier is never completed, so its wait
 * gives up after `polls` polls (1 .. 2^20) and sets DSMC_ERR_TIMEOUT, as the
 * step kernels' waits would; nothing stays in flight on the device.  Needs
 * dsmc_debug_begin.  Returns DSMC_E_TIMEOUT; the run's state and counters
 * are untouched and the context stays usable. */
dsmc_status dsmc_debug_timeout_probe(dsmc_ctx* ctx, uint32_t polls);

#ifdef __cplusplus
}
#endif
#endif
