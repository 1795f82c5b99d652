/*
 * dsmc_oracle.h -- plain, slow FP64 CPU oracle for the ensemble DSMC step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path includes, links or
 * calls this code; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it follows: the sequential unsteady-DSMC algorithm of Sec. 1.1 (the
 * flowchart of Fig. 1): per time step Generation -> Motion -> Enumeration /
 * Indexing (the readdressing array LCR) -> Interaction -> Sampling at given
 * moments, repeated over n statistically independent runs whose random number
 * generator is shifted per run.  The per-step physics (inflow flux of a
 * drifting Maxwellian, diffuse and specular walls, the no-time-counter
 * collision count, hard-sphere / variable-hard-sphere cross sections and
 * isotropic scattering) is deferred by the paper to Bird (1994) and is
 * restated here from kinetic theory; every point where that restatement is a
 * reading and not a quotation is listed with the design notes.
 *
 * Parity status per function (see the pins in tests/test_oracle_*.py):
 *   orc_philox            pinned (statistics; GPU cross-check vs cuRAND)
 *   orc_inflow_flux       pinned (effusion closed form n*cbar/4 at U=0)
 *   orc_sample_xi         pinned (KS test vs the closed-form density)
 *   generation            pinned (mean counts vs flux; effusion)
 *   motion                pinned (free flight, reflection brute force,
 *                          diffuse wall equilibrium, effusion orifice)
 *   enumeration/indexing  pinned (vs a stable sort of the slots by cell)
 *   interaction           pinned (per-collision conservation, equilibrium
 *                          HS and VHS rates, Maxwell-molecule relaxation)
 *   orc_partner           pinned (nearest: k-d tree search; subcell: one
 *                          subcell reduces to the uniform rule, placed
 *                          subcells, mean partner separation closed form)
 *   sampling              pinned (brute-force sums)
 */
#ifndef DSMC_ORACLE_H
#define DSMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_BC 32
#define ORC_NMOM 7   /* N, sum u, sum v, sum w, sum u^2, sum v^2, sum w^2 */

enum { ORC_OUTFLOW = 0, ORC_INFLOW = 1, ORC_SPECULAR = 2, ORC_DIFFUSE = 3 };
enum { ORC_FACE_PLATE = 6 };
/* choice of the second particle of an NTC candidate pair (the first is
 * uniform over the cell): uniform over the cell's other particles; uniform
 * over the other particles of the first one's subcell (n_sub per axis), the
 * cell-wide rule when it has none; the nearest other particle of the cell */
enum { ORC_PARTNER_UNIFORM = 0, ORC_PARTNER_SUBCELL = 1, ORC_PARTNER_NEAREST = 2 };

typedef struct {
    int32_t kind;          /* ORC_OUTFLOW .. ORC_DIFFUSE */
    int32_t face;          /* 2*axis + side (0..5), or ORC_FACE_PLATE */
    int32_t lo[2], hi[2];  /* tangential cell range [lo, hi), axes ascending */
    int32_t step_from;     /* first active step (1-based) */
    int32_t step_to;       /* last active step, 0 = forever */
    int32_t plate_axis;    /* plates: normal axis */
    int32_t plate_index;   /* plates: plane at plate_index * cell size */
    double n, T, U[3];     /* inflow state; T = wall temperature */
} orc_bc;

typedef struct {
    int32_t dim;           /* 2 or 3 */
    int32_t ncell[3];      /* ncell[2] = 1 in 2-D */
    double L[3];           /* extents (m); L[2] = depth in 2-D */
    double mass, d_ref, T_ref, omega, F_N;
    int32_t fill;          /* 0 empty, 1 uniform freestream */
    double fill_n, fill_T, fill_U[3];
    int32_t n_bc;
    orc_bc bc[ORC_MAX_BC];
    int32_t partner;       /* ORC_PARTNER_* */
    int32_t n_sub;         /* subcells per axis (ORC_PARTNER_SUBCELL) */
} orc_config;

/* counters of one run, accumulated over all steps */
typedef struct {
    uint64_t particle_steps, generated, removed, wall_hits;
    uint64_t candidates, collisions, clamps, bounce_limit, reject_limit;
} orc_stats;

typedef struct orc_ctx orc_ctx;

/* Philox4x32-10 (Salmon et al., SC'11): out = bijection(ctr) under key. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* the four uniforms in (0,1) that one draw gives (see orc_u01 in the .c) */
void orc_draw(uint64_t seed, uint32_t run, uint32_t step, uint32_t entity,
              uint32_t purpose, uint32_t sub, double u[4]);

/* number flux (m^-2 s^-1) through a wall of a drifting Maxwellian with
 * inward normal drift Un */
double orc_inflow_flux(double n, double T, double Un, double m);
/* inward normal speed ratio xi of an entering molecule (density
 * proportional to xi*exp(-(xi-s)^2), xi > 0); uses draw blocks 2..63 of
 * particle k of element e.  Returns the number of blocks used (or -1). */
int orc_sample_xi(double s, uint64_t seed, uint32_t run, uint32_t step,
                  uint32_t e, uint32_t k, double* xi);
/* sigma_T(g)*g of the VHS model of cfg (HS for omega = 1/2) */
double orc_sigma_cr(const orc_config* cfg, double g);
/* post-collision velocities of an accepted pair: u3 gives cos(chi), u4 eps */
void orc_scatter(double v1[3], double v2[3], double u3, double u4);
/* the second particle of an NTC candidate whose first particle is i, among
 * the N particles of cell c (absolute positions x[3*m .. 3*m+2], in LCR
 * order), under cfg->partner; u1 is the candidate's second uniform */
int64_t orc_partner(const orc_config* cfg, int c, const double* x, int64_t N, int64_t i,
                    double u1);

orc_ctx* orc_create(const orc_config* cfg, int n_runs, double dt, uint64_t seed);
void orc_destroy(orc_ctx* c);
int orc_init_run(orc_ctx* c, int run);                /* step-0 state */
int orc_step(orc_ctx* c, int run, int step);          /* one DSMC step */
int64_t orc_count(const orc_ctx* c, int run);
uint32_t orc_next_id(const orc_ctx* c, int run);   /* ids handed out so far */
int orc_get_state(const orc_ctx* c, int run, double* x, double* v, uint32_t* id);
int orc_set_state(orc_ctx* c, int run, int64_t n, const double* x,
                  const double* v, const uint32_t* id, uint32_t next_id);
/* last step's Enumeration/Indexing and Interaction outputs, per cell:
 * count, candidate pairs M, accepted collisions; lcr[k] = pre-sort slot of
 * the k-th particle in (cell, slot) order, slots numbered old-then-new */
int orc_get_cells(const orc_ctx* c, int run, int32_t* count, int32_t* cand,
                  int32_t* accepted, int64_t* lcr);
int orc_get_cell_state(const orc_ctx* c, int run, double* rem, double* smax);
int orc_set_cell_state(orc_ctx* c, int run, const double* rem, const double* smax);
int orc_sample(const orc_ctx* c, int run, double* mom /* ncells*ORC_NMOM */);
int orc_get_stats(const orc_ctx* c, int run, orc_stats* s);

/* whole ensemble: acc[t][g][cell][ORC_NMOM], g = run mod G, G = min(n,16),
 * runs of a group summed in increasing run order; `threads` workers take
 * whole groups (the paper's first level, Sec. 1.3). stats: summed over runs */
int orc_run_ensemble(const orc_config* cfg, int n_runs, double dt, int steps,
                     const int32_t* sample_steps, int n_samples, uint64_t seed,
                     int threads, double* acc, orc_stats* stats);

/* the part of an ensemble with global run indices run0 .. run0 + n_runs - 1
 * (one rank's share of runs sharded over processes): run r draws with the
 * global index run0 + r, and its moments go to group (run0 + r) mod G, G
 * being the whole ensemble's group count */
int orc_run_ensemble_part(const orc_config* cfg, uint32_t run0, int n_runs, int G, double dt,
                          int steps, const int32_t* sample_steps, int n_samples, uint64_t seed,
                          int threads, double* acc, orc_stats* stats);

/* the same with time-averaged samples: sample t sums the moments after
 * Interaction of steps first[t] .. last[t] (inclusive) of every run (the
 * averaging interval of Sec. 1.1); each run's window sums are formed in step
 * order and added to its group at the window's last step.  Windows lie in
 * [1, steps], increasing and disjoint. */
int orc_run_ensemble_windows(const orc_config* cfg, uint32_t run0, int n_runs, int G, double dt,
                             int steps, const int32_t* first, const int32_t* last, int n_samples,
                             uint64_t seed, int threads, double* acc, orc_stats* stats);

#ifdef __cplusplus
}
#endif
#endif
