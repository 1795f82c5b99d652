/*
 * dsmc_oracle.c -- plain, slow FP64 CPU oracle for the ensemble DSMC step.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline leg of bench.py; never by the product path.  It shares no code
 * with the CUDA path: both sides were written separately from the same
 * reading of the method and consume the same counter-based random numbers.
 *
 * The structure follows the sequential unsteady-DSMC algorithm of Sec. 1.1
 * (flowchart of Fig. 1):
 *   outer loop (Sec. 1.1, "second loop"): n independent runs, each with its
 *       own shifted random stream (here: the run index is a Philox counter
 *       word);
 *   inner loop: per time step dt
 *       Generation   -- particles enter through the inflow boundaries;
 *       Motion       -- free flight, surface interaction, leavers removed;
 *       Enumeration  -- particles counted per cell;
 *       Indexing     -- readdressing array LCR (particle <-> cell);
 *       Interaction  -- collisions, every cell independently;
 *       Sampling     -- cell macroparameters at the given moments.
 * The arrays are those of Sec. 1.1: P (particles), LCR (readdressing, one
 * entry per particle) and C (per cell: NTC remainder and (sigma*c_r)_max).
 *
 * All arithmetic is IEEE double, evaluated left to right as written (the
 * build uses -ffp-contract=off so that no multiply-add is fused).
 */
#include "dsmc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define KB 1.380649e-23
#define MAX_BOUNCE 16      /* surface events per particle per step */
#define GEN_BLOCKS 64      /* draw blocks reserved per generated particle */
#define NGROUP_MAX 16

/* Philox purposes: the fourth counter word's top 4 bits */
enum { P_FILL_COUNT = 1, P_FILL_PART = 2, P_GEN_COUNT = 3, P_GEN_PART = 4,
       P_WALL = 5, P_COLL = 6 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its definition (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
 *   (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1,
 *                     lo(M0*c0))
 * with the key bumped by the Weyl constants after every round.             */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0,1): the top 23 bits m of a word give (m + 1/2) / 2^23, a
 * value that is exact in binary32 and binary64 alike */
static double orc_u01(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* One draw: counter = (entity, purpose<<28 | sub, step, run), key = seed. */
void orc_draw(uint64_t seed, uint32_t run, uint32_t step, uint32_t entity,
              uint32_t purpose, uint32_t sub, double u[4])
{
    uint32_t ctr[4] = { entity, (purpose << 28) | (sub & 0x0FFFFFFFu), step, run };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox(ctr, key, out);
    for (int i = 0; i < 4; ++i) u[i] = orc_u01(out[i]);
}

/* Box-Muller: two independent standard normals from two uniforms */
static void orc_gauss2(double u1, double u2, double* z0, double* z1)
{
    double r = sqrt(-2.0 * log(u1));
    double a = 2.0 * M_PI * u2;
    *z0 = r * cos(a);
    *z1 = r * sin(a);
}

/* ------------------------------------------------------------------------ */
/* Kinetic theory used by Generation, Motion and Interaction                 */

/* Flux of a drifting Maxwellian (number density n, temperature T, inward
 * normal drift Un) through a plane: with c_mp = sqrt(2kT/m), s = Un/c_mp,
 *   N'/A = n c_mp / (2 sqrt(pi)) [exp(-s^2) + sqrt(pi) s (1 + erf s)];
 * at s = 0 it is the effusion flux n cbar / 4. */
double orc_inflow_flux(double n, double T, double Un, double m)
{
    double cmp = sqrt(2.0 * KB * T / m);
    double s = Un / cmp;
    return n * cmp / (2.0 * sqrt(M_PI)) *
           (exp(-s * s) + sqrt(M_PI) * s * (1.0 + erf(s)));
}

/* Entering molecules have inward normal speed ratio xi = u_n / c_mp with
 * density f(xi) ~ xi exp(-(xi - s)^2) on xi > 0.  Acceptance-rejection with
 * a normal proposal centred on the mode xi_m = (s + sqrt(s^2 + 2)) / 2 and
 * variance 1/2: the ratio f/proposal is proportional to xi exp(-xi/xi_m)
 * (because 2 (xi_m - s) = 1 / xi_m), whose maximum is at xi_m, so a
 * proposal is kept with probability (xi/xi_m) exp(1 - xi/xi_m).  Each draw
 * block gives two proposals (Box-Muller on u0,u1) and their two acceptance
 * uniforms (u2, u3). */
int orc_sample_xi(double s, uint64_t seed, uint32_t run, uint32_t step,
                  uint32_t e, uint32_t k, double* xi)
{
    double xm = (s + sqrt(s * s + 2.0)) / 2.0;
    for (int blk = 2; blk < GEN_BLOCKS; ++blk) {
        double u[4], z[2];
        orc_draw(seed, run, step, e, P_GEN_PART, k * GEN_BLOCKS + blk, u);
        orc_gauss2(u[0], u[1], &z[0], &z[1]);
        for (int att = 0; att < 2; ++att) {
            double x = xm + z[att] * sqrt(0.5);
            if (x > 0.0 && u[2 + att] < (x / xm) * exp(1.0 - x / xm)) {
                *xi = x;
                return blk - 1;
            }
        }
    }
    *xi = xm;
    return -1;
}

/* VHS cross-section times relative speed:
 *   sigma_T = pi d_ref^2 (2 k T_ref / (m_r g^2))^(omega - 1/2) / Gamma(5/2 - omega)
 * with reduced mass m_r = m/2; omega = 1/2 gives the hard sphere pi d^2. */
double orc_sigma_cr(const orc_config* cfg, double g)
{
    if (g == 0.0) return 0.0;
    double mr = cfg->mass / 2.0;
    double sig = M_PI * (cfg->d_ref * cfg->d_ref) *
                 pow(2.0 * KB * cfg->T_ref / (mr * g * g), cfg->omega - 0.5) /
                 tgamma(2.5 - cfg->omega);
    return sig * g;
}

/* Isotropic scattering of an equal-mass pair: centre-of-mass velocity kept,
 * relative velocity turned to a uniformly random direction,
 * cos(chi) = 2 u3 - 1, eps = 2 pi u4. */
void orc_scatter(double v1[3], double v2[3], double u3, double u4)
{
    double gx = v1[0] - v2[0], gy = v1[1] - v2[1], gz = v1[2] - v2[2];
    double g = sqrt(gx * gx + gy * gy + gz * gz);
    double cosx = 2.0 * u3 - 1.0;
    double sinx = sqrt(1.0 - cosx * cosx);
    double eps = 2.0 * M_PI * u4;
    double gr[3] = { g * cosx, g * sinx * cos(eps), g * sinx * sin(eps) };
    for (int a = 0; a < 3; ++a) {
        double cm = 0.5 * (v1[a] + v2[a]);
        v1[a] = cm + 0.5 * gr[a];
        v2[a] = cm - 0.5 * gr[a];
    }
}

/* ------------------------------------------------------------------------ */
typedef struct {
    double x[3], v[3];
    uint32_t id;
    double f;        /* fraction of dt to fly this step (1 for old particles) */
} orc_particle;

typedef struct {
    orc_particle* p;  int64_t n, cap;      /* P */
    double* rem;  double* smax;             /* C */
    int32_t* count; int32_t* cand; int32_t* accd;
    int64_t* lcr;  int64_t lcr_cap;         /* LCR of the last step */
    uint32_t next_id;
    int live;
    orc_stats st;
} orc_run;

struct orc_ctx {
    orc_config cfg;
    int n_runs;
    uint32_t run0;        /* global index of run 0 (Philox counter word 3) */
    double dt;
    uint64_t seed;
    double d[3];          /* cell sizes */
    double Vc;            /* cell volume */
    double coef;          /* F_N dt / Vc */
    double smax0;         /* initial (sigma c_r)_max */
    int ncells;
    int tang[3][2];       /* tangential axes of a face normal to axis a */
    int64_t elem_base[ORC_MAX_BC];
    orc_run* runs;
};

static int clampi(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

static int cell_index_1d(const orc_ctx* C, int a, double x)
{
    if (a >= C->cfg.dim) return 0;
    return clampi((int)floor(x / C->d[a]), 0, C->cfg.ncell[a] - 1);
}

static int cell_of(const orc_ctx* C, const double x[3])
{
    int i0 = cell_index_1d(C, 0, x[0]);
    int i1 = cell_index_1d(C, 1, x[1]);
    int i2 = cell_index_1d(C, 2, x[2]);
    return i0 + C->cfg.ncell[0] * (i1 + C->cfg.ncell[1] * i2);
}

static int bc_active(const orc_bc* b, int step)
{
    return step >= b->step_from && (b->step_to == 0 || step <= b->step_to);
}

/* Winning boundary segment at face cell (a, b) of `face` at `step`: the last
 * listed active segment that covers it; -1 means open (outflow). */
static int bc_lookup(const orc_ctx* C, int face, int a, int b, int step)
{
    int win = -1;
    for (int q = 0; q < C->cfg.n_bc; ++q) {
        const orc_bc* s = &C->cfg.bc[q];
        if (s->face != face) continue;
        if (a < s->lo[0] || a >= s->hi[0] || b < s->lo[1] || b >= s->hi[1]) continue;
        if (!bc_active(s, step)) continue;
        win = q;
    }
    return win;
}

static void run_free(orc_run* R)
{
    free(R->p); free(R->rem); free(R->smax); free(R->count); free(R->cand);
    free(R->accd); free(R->lcr);
    memset(R, 0, sizeof(*R));
}

static int run_alloc(orc_ctx* C, orc_run* R)
{
    run_free(R);
    int nc = C->ncells;
    R->rem = calloc(nc, sizeof(double));
    R->smax = malloc(nc * sizeof(double));
    R->count = calloc(nc, sizeof(int32_t));
    R->cand = calloc(nc, sizeof(int32_t));
    R->accd = calloc(nc, sizeof(int32_t));
    if (!R->rem || !R->smax || !R->count || !R->cand || !R->accd) return -1;
    for (int c = 0; c < nc; ++c) R->smax[c] = C->smax0;
    R->live = 1;
    return 0;
}

static int push(orc_run* R, const orc_particle* q)
{
    if (R->n == R->cap) {
        int64_t nc = R->cap ? 2 * R->cap : 1024;
        orc_particle* np = realloc(R->p, nc * sizeof(orc_particle));
        if (!np) return -1;
        R->p = np; R->cap = nc;
    }
    R->p[R->n++] = *q;
    return 0;
}

orc_ctx* orc_create(const orc_config* cfg, int n_runs, double dt, uint64_t seed)
{
    if (!cfg || (cfg->dim != 2 && cfg->dim != 3) || n_runs < 1 || !(dt > 0.0) ||
        cfg->n_bc < 0 || cfg->n_bc > ORC_MAX_BC ||
        cfg->partner < ORC_PARTNER_UNIFORM || cfg->partner > ORC_PARTNER_NEAREST ||
        (cfg->partner == ORC_PARTNER_SUBCELL && cfg->n_sub < 1))
        return NULL;
    orc_ctx* C = calloc(1, sizeof(orc_ctx));
    if (!C) return NULL;
    C->cfg = *cfg;
    if (C->cfg.dim == 2) C->cfg.ncell[2] = 1;
    C->n_runs = n_runs;
    C->dt = dt;
    C->seed = seed;
    for (int a = 0; a < 3; ++a) C->d[a] = C->cfg.L[a] / C->cfg.ncell[a];
    C->Vc = C->d[0] * C->d[1] * C->d[2];
    C->coef = (C->cfg.F_N * dt) / C->Vc;
    C->ncells = C->cfg.ncell[0] * C->cfg.ncell[1] * C->cfg.ncell[2];
    for (int a = 0; a < 3; ++a) {
        int k = 0;
        for (int t = 0; t < 3; ++t)
            if (t != a) C->tang[a][k++] = t;
    }
    /* reference temperature of the initial (sigma c_r)_max: the hottest
     * state the run is started or driven with */
    double T0 = 0.0;
    if (C->cfg.fill) T0 = C->cfg.fill_T;
    int64_t eb = 0;
    for (int q = 0; q < C->cfg.n_bc; ++q) {
        const orc_bc* b = &C->cfg.bc[q];
        if ((b->kind == ORC_INFLOW || b->kind == ORC_DIFFUSE) && b->T > T0) T0 = b->T;
        C->elem_base[q] = eb;
        if (b->kind == ORC_INFLOW && b->face < 6)
            eb += (int64_t)(b->hi[0] - b->lo[0]) * (b->hi[1] - b->lo[1]);
    }
    if (T0 <= 0.0) T0 = C->cfg.T_ref;
    double c0 = 3.0 * sqrt(2.0 * KB * T0 / C->cfg.mass);
    C->smax0 = orc_sigma_cr(&C->cfg, c0);
    C->runs = calloc(n_runs, sizeof(orc_run));
    if (!C->runs) { free(C); return NULL; }
    return C;
}

void orc_destroy(orc_ctx* C)
{
    if (!C) return;
    for (int r = 0; r < C->n_runs; ++r) run_free(&C->runs[r]);
    free(C->runs);
    free(C);
}

/* Step-0 state: empty, or every cell filled with a Poisson-rounded
 * freestream population (uniform in the cell, Maxwellian velocities). */
int orc_init_run(orc_ctx* C, int run)
{
    if (!C || run < 0 || run >= C->n_runs) return -1;
    orc_run* R = &C->runs[run];
    if (run_alloc(C, R)) return -2;
    R->next_id = 0;
    if (!C->cfg.fill) return 0;
    const orc_config* g = &C->cfg;
    double lam = g->fill_n * C->Vc / g->F_N;
    double sd = sqrt(KB * g->fill_T / g->mass);
    for (int c = 0; c < C->ncells; ++c) {
        int i[3] = { c % g->ncell[0], (c / g->ncell[0]) % g->ncell[1],
                     c / (g->ncell[0] * g->ncell[1]) };
        double u[4];
        orc_draw(C->seed, C->run0 + run, 0, c, P_FILL_COUNT, 0, u);
        int64_t N = (int64_t)floor(lam + u[0]);
        for (int64_t k = 0; k < N; ++k) {
            double b0[4], b1[4], z[4];
            orc_draw(C->seed, C->run0 + run, 0, c, P_FILL_PART, (uint32_t)(2 * k), b0);
            orc_draw(C->seed, C->run0 + run, 0, c, P_FILL_PART, (uint32_t)(2 * k + 1), b1);
            orc_gauss2(b0[0], b0[1], &z[0], &z[1]);
            orc_gauss2(b0[2], b0[3], &z[2], &z[3]);
            orc_particle q;
            memset(&q, 0, sizeof(q));
            for (int a = 0; a < 3; ++a) q.v[a] = g->fill_U[a] + sd * z[a];
            for (int a = 0; a < g->dim; ++a) q.x[a] = ((double)i[a] + b1[a]) * C->d[a];
            q.id = R->next_id++;
            q.f = 1.0;
            if (push(R, &q)) return -2;
        }
    }
    return 0;
}

/* Generation: particles entering through every active inflow segment. */
static int generation(orc_ctx* C, orc_run* R, int run, int step)
{
    const orc_config* g = &C->cfg;
    for (int q = 0; q < g->n_bc; ++q) {
        const orc_bc* b = &g->bc[q];
        if (b->kind != ORC_INFLOW || b->face >= 6 || !bc_active(b, step)) continue;
        int axis = b->face / 2, side = b->face % 2;
        int t0 = C->tang[axis][0], t1 = C->tang[axis][1];
        double dir = side ? -1.0 : 1.0;
        double cmp = sqrt(2.0 * KB * b->T / g->mass);
        double sd = sqrt(KB * b->T / g->mass);
        double Un = dir * b->U[axis];
        double s = Un / cmp;
        double area = C->d[t0] * C->d[t1];
        double lam = orc_inflow_flux(b->n, b->T, Un, g->mass) * area * C->dt / g->F_N;
        int w = b->hi[0] - b->lo[0];
        for (int bb = b->lo[1]; bb < b->hi[1]; ++bb)
            for (int aa = b->lo[0]; aa < b->hi[0]; ++aa) {
                if (bc_lookup(C, b->face, aa, bb, step) != q) continue;
                uint32_t e = (uint32_t)(C->elem_base[q] + (aa - b->lo[0]) +
                                        (int64_t)w * (bb - b->lo[1]));
                double u[4];
                orc_draw(C->seed, C->run0 + run, step, e, P_GEN_COUNT, 0, u);
                int64_t G = (int64_t)floor(lam + u[0]);
                if (G >= (1 << 22)) return -3;
                for (int64_t k = 0; k < G; ++k) {
                    double b0[4], b1[4], z0, z1, xi;
                    orc_draw(C->seed, C->run0 + run, step, e, P_GEN_PART, (uint32_t)(k * GEN_BLOCKS), b0);
                    orc_draw(C->seed, C->run0 + run, step, e, P_GEN_PART, (uint32_t)(k * GEN_BLOCKS + 1), b1);
                    orc_gauss2(b1[0], b1[1], &z0, &z1);
                    if (orc_sample_xi(s, C->seed, C->run0 + run, step, e, (uint32_t)k, &xi) < 0)
                        R->st.reject_limit++;
                    orc_particle p;
                    memset(&p, 0, sizeof(p));
                    p.x[axis] = side ? g->L[axis] : 0.0;
                    p.x[t0] = ((double)aa + b0[0]) * C->d[t0];
                    if (t1 < g->dim) p.x[t1] = ((double)bb + b0[1]) * C->d[t1];
                    p.v[axis] = dir * cmp * xi;
                    p.v[t0] = b->U[t0] + sd * z0;
                    p.v[t1] = b->U[t1] + sd * z1;
                    p.f = b0[2];
                    p.id = R->next_id++;
                    if (push(R, &p)) return -2;
                    R->st.generated++;
                }
            }
    }
    return 0;
}

/* Motion: free flight for f*dt with the surface events taken in time order
 * (ties: x, then y, then z faces, then plates in list order).  Returns 1 if
 * the particle stays in the domain, 0 if it left through an open face.
 * `slot` is the particle's place in P this step (old particles in P order,
 * then the entrants in generation order): it keys the particle's wall
 * draws. */
static int motion(orc_ctx* C, orc_run* R, int run, int step, orc_particle* p, int64_t slot)
{
    const orc_config* g = &C->cfg;
    const int dim = g->dim;
    double tau = p->f * C->dt;
    for (int bounce = 0;; ++bounce) {
        int hit = -1;
        double th = 0.0;
        for (int a = 0; a < dim; ++a) {
            double t;
            if (p->v[a] > 0.0) t = (g->L[a] - p->x[a]) / p->v[a];
            else if (p->v[a] < 0.0) t = (0.0 - p->x[a]) / p->v[a];
            else continue;
            if (t < 0.0) t = 0.0;
            if (t <= tau && (hit < 0 || t < th)) { hit = 2 * a + (p->v[a] > 0.0 ? 1 : 0); th = t; }
        }
        for (int q = 0; q < g->n_bc; ++q) {
            const orc_bc* b = &g->bc[q];
            if (b->face != ORC_FACE_PLATE || !bc_active(b, step)) continue;
            int a = b->plate_axis;
            double xp = (double)b->plate_index * C->d[a];
            if (!((p->x[a] < xp && p->v[a] > 0.0) || (p->x[a] > xp && p->v[a] < 0.0))) continue;
            double t = (xp - p->x[a]) / p->v[a];
            if (!(t <= tau && (hit < 0 || t < th))) continue;
            int inside = 1;
            for (int k = 0; k < 2; ++k) {
                int ta = C->tang[a][k];
                if (ta >= dim) continue;
                double y = p->x[ta] + p->v[ta] * t;
                if (!(y >= (double)b->lo[k] * C->d[ta] && y < (double)b->hi[k] * C->d[ta])) inside = 0;
            }
            if (inside) { hit = 100 + q; th = t; }
        }
        if (hit < 0) {
            for (int a = 0; a < dim; ++a) p->x[a] = p->x[a] + p->v[a] * tau;
            return 1;
        }
        if (bounce == MAX_BOUNCE) { R->st.bounce_limit++; return 1; }
        int axis, kind;
        double Tw = 0.0, dir;
        if (hit < 100) {
            axis = hit / 2;
            int side = hit % 2;
            for (int a = 0; a < dim; ++a)
                p->x[a] = (a == axis) ? (side ? g->L[a] : 0.0) : p->x[a] + p->v[a] * th;
            int ia = cell_index_1d(C, C->tang[axis][0], p->x[C->tang[axis][0]]);
            int ib = cell_index_1d(C, C->tang[axis][1], p->x[C->tang[axis][1]]);
            int q = bc_lookup(C, hit, ia, ib, step);
            kind = q < 0 ? ORC_OUTFLOW : g->bc[q].kind;
            if (q >= 0) Tw = g->bc[q].T;
            dir = side ? -1.0 : 1.0;
        } else {
            const orc_bc* b = &g->bc[hit - 100];
            axis = b->plate_axis;
            double xp = (double)b->plate_index * C->d[axis];
            dir = p->v[axis] > 0.0 ? -1.0 : 1.0;
            for (int a = 0; a < dim; ++a)
                p->x[a] = (a == axis) ? xp : p->x[a] + p->v[a] * th;
            kind = b->kind;
            Tw = b->T;
        }
        tau = tau - th;
        if (kind == ORC_OUTFLOW || kind == ORC_INFLOW) { R->st.removed++; return 0; }
        R->st.wall_hits++;
        if (kind == ORC_SPECULAR) {
            p->v[axis] = -p->v[axis];
        } else {
            double u[4], z0, z1;
            orc_draw(C->seed, C->run0 + run, step, (uint32_t)slot, P_WALL, (uint32_t)bounce, u);
            double sw = sqrt(KB * Tw / g->mass);
            orc_gauss2(u[1], u[2], &z0, &z1);
            p->v[axis] = dir * (sw * sqrt(-2.0 * log(u[0])));
            p->v[C->tang[axis][0]] = sw * z0;
            p->v[C->tang[axis][1]] = sw * z1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Choice of the collision partner.  The NTC scheme draws a candidate pair of
 * a cell; the paper's Interaction leaves the choice of the pair to the gas
 * model of Bird (1994), whose refinements select the second particle close
 * to the first so that collision partners are nearer than the cell size.
 * The variants restated here: the first particle i is uniform over the
 * cell's N particles; the second is
 *   uniform  -- uniform over the other N-1 (the r-th other in LCR order,
 *               r = floor(u1 (N-1)));
 *   subcell  -- the cell is split into n_sub subcells per axis; uniform over
 *               the other particles of i's subcell (the r-th of those K in
 *               LCR order, r = floor(u1 K)); if i is alone there, the
 *               uniform rule;
 *   nearest  -- the other particle at the smallest Euclidean distance from
 *               i (over the grid's axes); of equal distances, the first in
 *               LCR order.
 * Positions are read through `stride` bytes per particle.                  */

/* subcell of a particle of cell c: per axis floor(n_sub f / d) of its
 * offset f = x - (cell's lower corner) (clamped to the cell's subcells),
 * linear with axis 0 fastest */
static int subcell_of(const orc_config* cfg, const double d[3], const int ci[3],
                      const double* x)
{
    int s = 0;
    for (int a = cfg->dim - 1; a >= 0; --a) {
        double f = (x[a] - (double)ci[a] * d[a]) / d[a];
        int k = (int)floor(f * (double)cfg->n_sub);
        k = k < 0 ? 0 : (k > cfg->n_sub - 1 ? cfg->n_sub - 1 : k);
        s = s * cfg->n_sub + k;
    }
    return s;
}

static int64_t choose_partner(const orc_config* cfg, const double d[3], int c, const char* xb,
                              size_t stride, int64_t N, int64_t i, double u1)
{
#define POS_OF(m) ((const double*)(xb + (size_t)(m) * stride))
    if (cfg->partner == ORC_PARTNER_NEAREST) {
        const double* xi = POS_OF(i);
        double best = INFINITY;
        int64_t j = -1;
        for (int64_t m = 0; m < N; ++m) {
            if (m == i) continue;
            const double* xm = POS_OF(m);
            double dd = 0.0;
            for (int a = 0; a < cfg->dim; ++a) {
                double e = xm[a] - xi[a];
                dd = dd + e * e;
            }
            if (dd < best) { best = dd; j = m; }
        }
        return j;
    }
    if (cfg->partner == ORC_PARTNER_SUBCELL) {
        int n0 = cfg->ncell[0], n1 = cfg->ncell[1];
        int ci[3] = { c % n0, (c / n0) % n1, c / (n0 * n1) };
        int si = subcell_of(cfg, d, ci, POS_OF(i));
        int64_t K = 0;
        for (int64_t m = 0; m < N; ++m)
            if (m != i && subcell_of(cfg, d, ci, POS_OF(m)) == si) ++K;
        if (K > 0) {
            int64_t r = (int64_t)floor(u1 * (double)K);
            for (int64_t m = 0; m < N; ++m) {
                if (m == i || subcell_of(cfg, d, ci, POS_OF(m)) != si) continue;
                if (r == 0) return m;
                --r;
            }
        }
    }
#undef POS_OF
    int64_t j = (int64_t)floor(u1 * (double)(N - 1));
    if (j >= i) j += 1;
    return j;
}

int64_t orc_partner(const orc_config* cfg, int c, const double* x, int64_t N, int64_t i,
                    double u1)
{
    if (!cfg || !x || N < 2 || i < 0 || i >= N ||
        cfg->partner < ORC_PARTNER_UNIFORM || cfg->partner > ORC_PARTNER_NEAREST ||
        (cfg->partner == ORC_PARTNER_SUBCELL && cfg->n_sub < 1))
        return -1;
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = cfg->L[a] / (a < cfg->dim ? cfg->ncell[a] : 1);
    return choose_partner(cfg, d, c, (const char*)x, 3 * sizeof(double), N, i, u1);
}

/* NTC collisions in one cell: its N particles are q[0..N) in LCR order. */
static void interaction_cell(orc_ctx* C, orc_run* R, int run, int step, int c,
                             orc_particle* q, int64_t N)
{
    int64_t M = 0;
    if (N >= 2) {
        double nn = (double)N * (double)(N - 1);
        double x = 0.5 * nn * C->coef * R->smax[c] + R->rem[c];
        M = (int64_t)floor(x);
        R->rem[c] = x - (double)M;
    }
    double seen = 0.0;
    int64_t acc = 0;
    for (int64_t k = 0; k < M; ++k) {
        double u[4];
        orc_draw(C->seed, C->run0 + run, step, c, P_COLL, (uint32_t)(2 * k), u);
        int64_t i = (int64_t)floor(u[0] * (double)N);
        int64_t j = choose_partner(&C->cfg, C->d, c, (const char*)q[0].x,
                                   sizeof(orc_particle), N, i, u[1]);
        double* v1 = q[i].v;
        double* v2 = q[j].v;
        double gx = v1[0] - v2[0], gy = v1[1] - v2[1], gz = v1[2] - v2[2];
        double gg = sqrt(gx * gx + gy * gy + gz * gz);
        double sc = orc_sigma_cr(&C->cfg, gg);
        if (sc > seen) seen = sc;
        if (sc > R->smax[c]) R->st.clamps++;
        if (u[2] < sc / R->smax[c]) {
            double u2[4];
            orc_draw(C->seed, C->run0 + run, step, c, P_COLL, (uint32_t)(2 * k + 1), u2);
            orc_scatter(v1, v2, u[3], u2[0]);
            ++acc;
        }
    }
    if (seen > R->smax[c]) R->smax[c] = seen;
    R->cand[c] = (int32_t)M;
    R->accd[c] = (int32_t)acc;
    R->st.candidates += (uint64_t)M;
    R->st.collisions += (uint64_t)acc;
}

int orc_step(orc_ctx* C, int run, int step)
{
    if (!C || run < 0 || run >= C->n_runs || step < 1) return -1;
    orc_run* R = &C->runs[run];
    if (!R->live) return -1;
    const int nc = C->ncells;
    int64_t n_old = R->n;
    for (int64_t s = 0; s < n_old; ++s) R->p[s].f = 1.0;
    /* Generation */
    int rc = generation(C, R, run, step);
    if (rc) return rc;
    int64_t n_all = R->n;
    R->st.particle_steps += (uint64_t)n_all;
    /* Motion: slots 0..n_old-1 old particles, n_old.. new ones */
    int32_t* cell = malloc((n_all ? n_all : 1) * sizeof(int32_t));
    if (!cell) return -2;
    for (int64_t s = 0; s < n_all; ++s)
        cell[s] = motion(C, R, run, step, &R->p[s], s) ? cell_of(C, R->p[s].x) : -1;
    /* Enumeration: particles per cell */
    memset(R->count, 0, nc * sizeof(int32_t));
    for (int64_t s = 0; s < n_all; ++s)
        if (cell[s] >= 0) R->count[cell[s]]++;
    /* Indexing: LCR = slots grouped by cell, each cell's slots in array
     * order (one serial pass over P, as the readdressing of Sec. 1.1 fills
     * it): exclusive prefix of the counts, then every surviving slot, in
     * increasing slot order, appended to its cell's range.  Slots number the
     * old particles in their P order, then the entrants in generation order. */
    int64_t* start = malloc((nc + 1) * sizeof(int64_t));
    if (!start) { free(cell); return -2; }
    start[0] = 0;
    for (int c = 0; c < nc; ++c) start[c + 1] = start[c] + R->count[c];
    int64_t n_new = start[nc];
    if (n_new > R->lcr_cap) {
        free(R->lcr);
        R->lcr = malloc((n_new ? n_new : 1) * sizeof(int64_t));
        if (!R->lcr) { free(cell); free(start); return -2; }
        R->lcr_cap = n_new;
    }
    int64_t* fillp = malloc((nc + 1) * sizeof(int64_t));
    if (!fillp) { free(cell); free(start); return -2; }
    memcpy(fillp, start, (nc + 1) * sizeof(int64_t));
    for (int64_t s = 0; s < n_all; ++s)
        if (cell[s] >= 0) R->lcr[fillp[cell[s]]++] = s;
    /* P rewritten in LCR order (leavers dropped) */
    orc_particle* np = malloc((n_new ? n_new : 1) * sizeof(orc_particle));
    if (!np) { free(cell); free(start); free(fillp); return -2; }
    for (int64_t k = 0; k < n_new; ++k) np[k] = R->p[R->lcr[k]];
    free(R->p);
    R->p = np;
    R->n = n_new;
    R->cap = n_new ? n_new : 1;
    /* Interaction: every cell independently */
    for (int c = 0; c < nc; ++c)
        interaction_cell(C, R, run, step, c, R->p + start[c], R->count[c]);
    free(cell); free(start); free(fillp);
    return 0;
}

int64_t orc_count(const orc_ctx* C, int run)
{
    if (!C || run < 0 || run >= C->n_runs) return -1;
    return C->runs[run].n;
}

uint32_t orc_next_id(const orc_ctx* C, int run)
{
    if (!C || run < 0 || run >= C->n_runs) return 0;
    return C->runs[run].next_id;
}

int orc_get_state(const orc_ctx* C, int run, double* x, double* v, uint32_t* id)
{
    if (!C || run < 0 || run >= C->n_runs) return -1;
    const orc_run* R = &C->runs[run];
    for (int64_t k = 0; k < R->n; ++k) {
        for (int a = 0; a < 3; ++a) {
            if (x) x[3 * k + a] = R->p[k].x[a];
            if (v) v[3 * k + a] = R->p[k].v[a];
        }
        if (id) id[k] = R->p[k].id;
    }
    return 0;
}

int orc_set_state(orc_ctx* C, int run, int64_t n, const double* x,
                  const double* v, const uint32_t* id, uint32_t next_id)
{
    if (!C || run < 0 || run >= C->n_runs || n < 0) return -1;
    orc_run* R = &C->runs[run];
    if (!R->live && run_alloc(C, R)) return -2;
    R->n = 0;
    for (int64_t k = 0; k < n; ++k) {
        orc_particle q;
        memset(&q, 0, sizeof(q));
        for (int a = 0; a < 3; ++a) { q.x[a] = x[3 * k + a]; q.v[a] = v[3 * k + a]; }
        q.id = id[k];
        q.f = 1.0;
        if (push(R, &q)) return -2;
    }
    R->next_id = next_id;
    return 0;
}

int orc_get_cells(const orc_ctx* C, int run, int32_t* count, int32_t* cand,
                  int32_t* accepted, int64_t* lcr)
{
    if (!C || run < 0 || run >= C->n_runs) return -1;
    const orc_run* R = &C->runs[run];
    if (!R->live) return -1;
    if (count) memcpy(count, R->count, C->ncells * sizeof(int32_t));
    if (cand) memcpy(cand, R->cand, C->ncells * sizeof(int32_t));
    if (accepted) memcpy(accepted, R->accd, C->ncells * sizeof(int32_t));
    if (lcr && R->lcr) memcpy(lcr, R->lcr, R->n * sizeof(int64_t));
    return 0;
}

int orc_get_cell_state(const orc_ctx* C, int run, double* rem, double* smax)
{
    if (!C || run < 0 || run >= C->n_runs || !C->runs[run].live) return -1;
    if (rem) memcpy(rem, C->runs[run].rem, C->ncells * sizeof(double));
    if (smax) memcpy(smax, C->runs[run].smax, C->ncells * sizeof(double));
    return 0;
}

int orc_set_cell_state(orc_ctx* C, int run, const double* rem, const double* smax)
{
    if (!C || run < 0 || run >= C->n_runs) return -1;
    orc_run* R = &C->runs[run];
    if (!R->live && run_alloc(C, R)) return -2;
    if (rem) memcpy(R->rem, rem, C->ncells * sizeof(double));
    if (smax) memcpy(R->smax, smax, C->ncells * sizeof(double));
    return 0;
}

/* Sampling: per cell N, sum of each velocity component and of its square,
 * summed over the cell's particles in LCR order. */
int orc_sample(const orc_ctx* C, int run, double* mom)
{
    if (!C || run < 0 || run >= C->n_runs) return -1;
    const orc_run* R = &C->runs[run];
    memset(mom, 0, (size_t)C->ncells * ORC_NMOM * sizeof(double));
    for (int64_t k = 0; k < R->n; ++k) {
        const orc_particle* p = &R->p[k];
        double* m = mom + (size_t)cell_of(C, p->x) * ORC_NMOM;
        m[0] += 1.0;
        for (int a = 0; a < 3; ++a) {
            m[1 + a] += p->v[a];
            m[4 + a] += p->v[a] * p->v[a];
        }
    }
    return 0;
}

int orc_get_stats(const orc_ctx* C, int run, orc_stats* s)
{
    if (!C || run < 0 || run >= C->n_runs || !s) return -1;
    *s = C->runs[run].st;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Ensemble of independent runs (the outer loop of Sec. 1.1), optionally
 * spread over threads by whole run groups (the independent-runs level of
 * Sec. 1.3: no exchange until all runs are done). */
typedef struct {
    orc_ctx* C;
    int worker, n_workers, G, steps, n_samples;
    const int32_t* first;   /* sample k averages steps first[k] .. last[k] */
    const int32_t* last;
    double* acc;
    int rc;
} orc_job;

static void* orc_worker(void* arg)
{
    orc_job* J = (orc_job*)arg;
    orc_ctx* C = J->C;
    size_t per = (size_t)C->ncells * ORC_NMOM;
    double* mom = malloc(per * sizeof(double));
    double* win = malloc(per * sizeof(double));   /* the run's sums over the current window */
    if (!mom || !win) { J->rc = -2; free(mom); free(win); return NULL; }
    for (int g = J->worker; g < J->G; g += J->n_workers) {
        /* local runs r whose global index run0 + r falls in group g */
        const int r0 = (int)(((uint32_t)g + (uint32_t)J->G - C->run0 % (uint32_t)J->G) % (uint32_t)J->G);
        for (int r = r0; r < C->n_runs; r += J->G) {
            orc_stats keep;
            int rc = orc_init_run(C, r);
            int t = 0;
            for (int s = 1; rc == 0 && s <= J->steps; ++s) {
                rc = orc_step(C, r, s);
                if (rc == 0 && t < J->n_samples && J->first[t] <= s && s <= J->last[t]) {
                    orc_sample(C, r, mom);
                    /* the window's sums in step order, then added to the group
                     * at the window's last step */
                    if (s == J->first[t])
                        for (size_t i = 0; i < per; ++i) win[i] = mom[i];
                    else
                        for (size_t i = 0; i < per; ++i) win[i] += mom[i];
                    if (s == J->last[t]) {
                        double* dst = J->acc + ((size_t)t * J->G + g) * per;
                        for (size_t i = 0; i < per; ++i) dst[i] += win[i];
                        ++t;
                    }
                }
            }
            if (rc) { J->rc = rc; free(mom); free(win); return NULL; }
            keep = C->runs[r].st;
            run_free(&C->runs[r]);
            C->runs[r].st = keep;
        }
    }
    free(mom);
    free(win);
    return NULL;
}

int orc_run_ensemble(const orc_config* cfg, int n_runs, double dt, int steps,
                     const int32_t* sample_steps, int n_samples, uint64_t seed,
                     int threads, double* acc, orc_stats* stats)
{
    return orc_run_ensemble_part(cfg, 0, n_runs, n_runs < NGROUP_MAX ? n_runs : NGROUP_MAX, dt,
                                 steps, sample_steps, n_samples, seed, threads, acc, stats);
}

int orc_run_ensemble_part(const orc_config* cfg, uint32_t run0, int n_runs, int G, double dt,
                          int steps, const int32_t* sample_steps, int n_samples, uint64_t seed,
                          int threads, double* acc, orc_stats* stats)
{
    return orc_run_ensemble_windows(cfg, run0, n_runs, G, dt, steps, sample_steps, sample_steps,
                                    n_samples, seed, threads, acc, stats);
}

int orc_run_ensemble_windows(const orc_config* cfg, uint32_t run0, int n_runs, int G, double dt,
                             int steps, const int32_t* first, const int32_t* last, int n_samples,
                             uint64_t seed, int threads, double* acc, orc_stats* stats)
{
    for (int t = 0; t < n_samples; ++t)
        if (first[t] < 1 || last[t] > steps || first[t] > last[t] ||
            (t > 0 && first[t] <= last[t - 1]))
            return -1;
    if (G < 1 || G > NGROUP_MAX) return -1;
    orc_ctx* C = orc_create(cfg, n_runs, dt, seed);
    if (!C) return -1;
    C->run0 = run0;
    memset(acc, 0, (size_t)n_samples * G * C->ncells * ORC_NMOM * sizeof(double));
    if (threads < 1) threads = 1;
    if (threads > G) threads = G;
    orc_job* jobs = calloc(threads, sizeof(orc_job));
    pthread_t* th = calloc(threads, sizeof(pthread_t));
    int rc = 0;
    if (!jobs || !th) rc = -2;
    for (int w = 0; rc == 0 && w < threads; ++w) {
        jobs[w] = (orc_job){ C, w, threads, G, steps, n_samples, first, last, acc, 0 };
        if (threads == 1) orc_worker(&jobs[w]);
        else if (pthread_create(&th[w], NULL, orc_worker, &jobs[w])) rc = -2;
    }
    if (threads > 1)
        for (int w = 0; w < threads; ++w) pthread_join(th[w], NULL);
    for (int w = 0; rc == 0 && w < threads; ++w)
        if (jobs[w].rc) rc = jobs[w].rc;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        for (int r = 0; r < n_runs; ++r) {
            const orc_stats* s = &C->runs[r].st;
            stats->particle_steps += s->particle_steps;
            stats->generated += s->generated;
            stats->removed += s->removed;
            stats->wall_hits += s->wall_hits;
            stats->candidates += s->candidates;
            stats->collisions += s->collisions;
            stats->clamps += s->clamps;
            stats->bounce_limit += s->bounce_limit;
            stats->reject_limit += s->reject_limit;
        }
    }
    free(jobs); free(th);
    orc_destroy(C);
    return rc;
}
