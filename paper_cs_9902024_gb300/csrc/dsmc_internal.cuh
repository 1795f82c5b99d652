// dsmc_internal.cuh -- types shared by the host engine and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dsmc.h"

namespace dsmc {

constexpr uint32_t kDead = 0xFFFFFFFFu;   // cell key of a particle that left
constexpr int kMaxBounce = 16;            // surface events per particle and step
constexpr int kGenBlocks = 64;            // Philox blocks per generated particle
constexpr int kWarpMax = 128;             // larger cells go to the big-cell kernels
constexpr int kTileCells = 256;           // cells (= threads) per CTA of the sort/gather kernel
constexpr int kMaxTileBudget = 16384;     // largest particle budget of a sort/gather tile
constexpr int kGenElems = 2048;           // inflow elements per Generation CTA
constexpr int kCollideCells = 128;        // cells per tile (CTA) of the collision kernel
constexpr int kCollidePerThread = 1;      // cells each of its threads collides
constexpr int kCollideThreads = kCollideCells / kCollidePerThread;
constexpr int kScanTile = 4096;           // cells per CTA of the scan
constexpr int kScanThreads = 1024;
constexpr int kMaxSamples = 4096;
// sample_slot[step]: -1, or the sample index k of the window the step belongs
// to, with a flag on the window's first step (the per-run sums restart) and
// on its last step (the runs' sums are added into the group sums)
constexpr int32_t kSlotIndex = 0x000FFFFF, kSlotFirst = 0x00100000, kSlotLast = 0x00200000;

// Philox counter word 1 carries the purpose of a draw in its top 4 bits.
enum Purpose : uint32_t {
    kFillCount = 1, kFillPart = 2, kGenCount = 3, kGenPart = 4, kWall = 5, kColl = 6
};

// One boundary segment with the constants the kernels derive from it (all
// computed once on the host in double precision).
struct BcDev {
    int32_t kind, face, lo[2], hi[2], step_from, step_to, plate_axis, plate_index;
    int32_t axis, side, t0, t1;      // normal axis, side, tangential axes
    int32_t elem_w;                  // inflow: elements along the first tangent
    int32_t pad_;
    int64_t elem_base;               // inflow: first element number
    int64_t n_elem;                  // inflow: element count
    double T, U[3];
    double lam;    // inflow: expected entrants per element and step
    double cmp;    // inflow: most probable speed sqrt(2kT/m)
    double sd;     // sqrt(kT/m): tangential spread (inflow), wall (diffuse)
    double s;      // inflow: inward normal speed ratio U_n / c_mp
    double xm;     // inflow: mode of the entrant speed-ratio density
    double dir;    // +1 on a side-0 face, -1 on a side-1 face
    double xp;     // plate: plane coordinate
    double tlo[2], thi[2];   // plate: tangential rectangle
};

struct Cfg {
    int32_t dim, n[3], ncells, n_bc, n_plate, hs, fill, pad_;
    int32_t partner, n_sub;   // collision-partner choice (DSMC_PARTNER_*), subcells per axis
    int32_t plate_idx[DSMC_MAX_BC];
    double L[3], d[3], inv_d[3], Vc, dt, mass;
    double coef;         // F_N dt / Vc
    float coef_f;        // the same, rounded to binary32
    double F_N;
    double A_hs;         // hard sphere: pi d^2 (sigma_T c_r = A_hs c_r)
    double K_vhs;        // VHS: sigma_T c_r = K_vhs (c_r^2)^(1 - omega)
    double one_m_omega;
    double smax0;        // initial (sigma_T c_r)_max
    double fill_lam, fill_sd, fill_U[3];
    int64_t n_elem;      // inflow elements over all segments
    uint64_t seed;
    uint64_t ncells_magic;   // key / ncells = umul64hi(key, magic); 0 if ncells == 1
    BcDev bc[DSMC_MAX_BC];
};

struct Counters {
    unsigned long long particle_steps, generated, removed, wall_hits;
    unsigned long long candidates, collisions, clamps, bounce_limit, reject_limit;
    unsigned long long pool_steps;
    unsigned long long big_pool_steps;   // particles ordered by the big-cell kernel
    uint32_t error, step, n_big, n_slow;
    uint32_t probe;        // error bits of the timeout test hook only
    uint32_t scan_ticket;  // CTAs of the scan's first pass done (reset by the last)
    uint32_t check_fail;   // options.checks: pool positions that failed the check
    uint32_t check_first;  // the first of them (0xFFFFFFFF: none)
};

// The configuration constants that the streaming kernels use for every
// particle or NTC candidate, carried by value in the launch parameters
// (constant bank) rather than read through the configuration pointer.  The
// field names match Cfg's, so the device helpers accept either; every value
// is the one the Cfg-based code converts to (the results do not depend on
// which is used).
template <typename T>
struct Hot {
    T d[3];                  // cell sizes
    float inv_d[3];          // binary32 reciprocals of d
    T dt;
    int32_t n[3];            // cells per axis
    int32_t ncells;          // cells per run
    uint32_t plate_axes;     // bit a set: a plate is normal to axis a
    int32_t n_plate;         // plates listed below (-1: more than kHotPlates;
                             // then any cell change along plate_axes counts)
    int32_t plate_ax[4], plate_ix[4];   // plate axis and face index (plane
                                        // between cells plate_ix - 1 and plate_ix)
    int32_t hs;
    int32_t dim;
    int32_t partner, n_sub;  // collision-partner choice (DSMC_PARTNER_*), subcells per axis
    uint64_t ncells_magic;
    uint64_t seed;
    T A_hs, K_vhs, one_m_omega;
    double coef;
    float coef_f;
    uint32_t rk[20];         // Philox4x32-10 round keys of the seed (rounds 0..9)
};

// Device pointers of one step (particle pool double-buffered: in -> out).
template <typename T>
struct StepArgs {
    const Cfg* cfg;
    Hot<T> hot;
    Counters* ctr;
    // pool: in/out buffers of positions (dim used), velocities (3), ids
    // (ids only in debug mode, else null: no step reads them); positions are
    // offsets inside the particle's cell; ci_* hold the run-major cell key
    // (run * ncells + cell) of each particle of the pool
    T* xi[3]; T* vi[3]; uint32_t* idi; uint32_t* ci_i;
    T* xo[3]; T* vo[3]; uint32_t* ido; uint32_t* ci_o;
    uint32_t* gc;          // per slot: run-major cell key, or kDead
    uint32_t* lcr;         // per pool position: the particle's slot in the step's
                           // pools (old, then entrants), cell-grouped
    uint32_t* lcr_dbg;     // optional: slot of each sorted particle
    uint32_t* count;       // per cell: particles (Motion counts up, the LCR
                           // scatter counts back down to zero)
    uint32_t* start;       // per cell (+2): exclusive prefix of count; entry
                           // total_cells + 1 keeps the pre-step pool size
    uint32_t* block_sums;  // per scan CTA (+1): block sums, then their prefix
    uint32_t* run_base;    // per run (+1): first pool position of the run
    uint32_t* next_id;     // per run
    double* rem;           // per cell: NTC remainder
    T* smax;               // per cell: (sigma_T c_r)_max
    double* mom;           // per cell x 7: moments at sample steps
    uint32_t* cand;        // optional per cell
    uint32_t* accd;        // optional per cell
    uint32_t* big_list;
    uint32_t* slow_list;   // slots whose flight meets a surface this step
    uint32_t* gen_tot;     // per run x gen_groups: entrants of each element group
    uint32_t* gen_done;    // per run: Generation CTAs finished this step
    int32_t gen_groups;    // Generation CTAs per run (ceil(n_elem / kGenElems))
    const int32_t* sample_slot;   // per step: sample index or -1
    int32_t n_slot;               // entries of sample_slot
    double* acc;           // [samples][G][ncells][7]
    int64_t cap_old, cap_new, gcap, max_big;
    int32_t n_runs;        // runs in this launch
    int32_t run0;          // global index of the first run of the launch
    int32_t G;             // sample groups
    int32_t total_cells;
    int32_t scan_blocks;
    int32_t tile_budget;   // particles a tile CTA stages in shared memory
    int32_t collide_stage; // particles a collision CTA stages in shared memory
};

// Several problems advanced by one launch per kernel kind (the parts of a
// mixed-size ensemble: each part one grid with its own runs, buffers and
// counters).  The tile-shaped kernels take their items -- (part, tile) or
// (part, chunk of slots) -- from device work-queue counters; items are
// numbered part by part in the order of `parts`.
constexpr int kMaxParts = 64;
enum QueueKind : int { kQMove = 0, kQScatter = 1, kQCell = 2, kQCollide = 3, kQueueKinds = 4 };
constexpr uint32_t kMoveChunk = 8192;      // slots per Motion item (a multiple of 1024)
constexpr uint32_t kScatterChunk = 8192;   // slots per scatter item (a multiple of 1024)

template <typename T>
struct MultiArgs {
    const StepArgs<T>* parts;     // device array, n_parts entries
    uint32_t* queue;              // kQueueKinds claim counters, zeroed at each step's end
    int32_t n_parts;
    int32_t collide_stage;        // the collision CTAs' stage (every part's the same)
    int32_t positional;           // some part chooses collision partners by position
    int32_t tile_base[kMaxParts + 1];     // sort/gather tiles before each part
    int32_t ctile_base[kMaxParts + 1];    // collision tiles before each part
    int32_t scan_base[kMaxParts + 1];     // scan CTAs before each part
    int32_t gen_base[kMaxParts + 1];      // Generation CTAs before each part
    int32_t gcount_base[kMaxParts + 1];   // Generation counting CTAs before each part
};

// Launch shape of the step kernels.
struct LaunchShape {
    int dim;
    int sms;
    int move_blocks, move_threads;
    int scatter_blocks, cell_blocks, big_blocks, collide_blocks;
    int tile_budget;
    int collide_stage;   // particles a collision CTA stages (follows collide_blocks)
    int collide_ppc;     // staged particles a cell the default collision shape aims at
    int pdl;   // direct launches overlap with the previous kernel (programmatic
               // dependent launch); 0 while a step is captured into a graph
};

// The kernels are compiled twice (dsmc_kernels.cu): once for FP32 particle
// state with fused multiply-add contraction allowed (namespace f32), once
// for FP64 state without contraction, so that it rounds every operation as
// the FP64 oracle does (namespace f64).  The functions below pick the
// instantiation by `prec`.
#define DSMC_PREC_LAUNCHERS                                                                    \
    void launch_init_cells(const void* args, const LaunchShape& ls, cudaStream_t s);          \
    void launch_fill(const void* args, const LaunchShape& ls, cudaStream_t s);                \
    void launch_generate(const void* args, const LaunchShape& ls, cudaStream_t s);            \
    void launch_move(const void* args, const LaunchShape& ls, cudaStream_t s);                \
    void launch_scan(const void* args, const LaunchShape& ls, cudaStream_t s);                \
    void launch_scatter(const void* args, const LaunchShape& ls, cudaStream_t s);             \
    void launch_cell(const void* args, const LaunchShape& ls, cudaStream_t s);                \
    void launch_cell_big(const void* args, const LaunchShape& ls, cudaStream_t s);            \
    void launch_collide_big(const void* args, const LaunchShape& ls, cudaStream_t s);         \
    void launch_collide(const void* args, const LaunchShape& ls, cudaStream_t s);             \
    void launch_reduce(const void* args, const LaunchShape& ls, cudaStream_t s);              \
    void launch_step_end(const void* args, const LaunchShape& ls, cudaStream_t s);            \
    void launch_macro(const void* args, int sample, int n_runs, int window, double* out,      \
                      cudaStream_t s);                                                         \
    void launch_sample_now(const void* args, cudaStream_t s);                                 \
    void launch_check(const void* args, const LaunchShape& ls, cudaStream_t s);               \
    cudaError_t prepare_kernels(int dim, int tile_budget, int collide_stage);                 \
    int collide_stage_for(int per_sm, int multi);                                             \
    void launch_m_generate(const void* margs, const LaunchShape& ls, cudaStream_t s);         \
    void launch_m_move(const void* margs, const LaunchShape& ls, cudaStream_t s);             \
    void launch_m_scan(const void* margs, const LaunchShape& ls, cudaStream_t s);             \
    void launch_m_scatter(const void* margs, const LaunchShape& ls, cudaStream_t s);          \
    void launch_m_cell(const void* margs, const LaunchShape& ls, cudaStream_t s);             \
    void launch_m_cell_big(const void* margs, const LaunchShape& ls, cudaStream_t s);         \
    void launch_m_collide_big(const void* margs, const LaunchShape& ls, cudaStream_t s);      \
    void launch_m_collide(const void* margs, const LaunchShape& ls, cudaStream_t s);          \
    void launch_m_reduce(const void* margs, const LaunchShape& ls, cudaStream_t s);           \
    void launch_m_step_end(const void* margs, const LaunchShape& ls, cudaStream_t s);         \
    cudaError_t prepare_multi_kernels(int dim, int tile_budget, int collide_stage);           \
    void compute_multi_shape(int dim, int sms, LaunchShape* ls);                              \
    void compute_launch_shape(int dim, int sms, LaunchShape* ls);                             \
    int big_cell_limit();

namespace f32 { DSMC_PREC_LAUNCHERS }
namespace f64 { DSMC_PREC_LAUNCHERS }

#define DSMC_PICK(prec, call) ((prec) == DSMC_FP64 ? f64::call : f32::call)

// `args` points to a StepArgs<float> or StepArgs<double> (`margs` to a
// MultiArgs<float> or MultiArgs<double>) as `prec` says; the multi-part
// launchers' `ls` holds the grid sizes of the queue-driven kernels
// (move_blocks, scatter_blocks, cell_blocks, collide_blocks).
inline void launch_init_cells(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_init_cells(a, ls, s)); }
inline void launch_fill(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_fill(a, ls, s)); }
inline void launch_generate(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_generate(a, ls, s)); }
inline void launch_move(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_move(a, ls, s)); }
inline void launch_scan(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_scan(a, ls, s)); }
inline void launch_scatter(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_scatter(a, ls, s)); }
inline void launch_cell(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_cell(a, ls, s)); }
inline void launch_cell_big(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_cell_big(a, ls, s)); }
inline void launch_collide_big(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_collide_big(a, ls, s)); }
inline void launch_collide(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_collide(a, ls, s)); }
inline void launch_reduce(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_reduce(a, ls, s)); }
inline void launch_step_end(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_step_end(a, ls, s)); }
inline void launch_macro(int p, const void* a, int sample, int n_runs, int window, double* out,
                         cudaStream_t s) { DSMC_PICK(p, launch_macro(a, sample, n_runs, window, out, s)); }
inline void launch_sample_now(int p, const void* a, cudaStream_t s) { DSMC_PICK(p, launch_sample_now(a, s)); }
inline void launch_check(int p, const void* a, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_check(a, ls, s)); }
inline cudaError_t prepare_kernels(int p, int dim, int tile_budget, int collide_stage) { return DSMC_PICK(p, prepare_kernels(dim, tile_budget, collide_stage)); }
inline int collide_stage_for(int p, int per_sm, int multi) { return DSMC_PICK(p, collide_stage_for(per_sm, multi)); }
inline void launch_m_generate(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_generate(m, ls, s)); }
inline void launch_m_move(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_move(m, ls, s)); }
inline void launch_m_scan(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_scan(m, ls, s)); }
inline void launch_m_scatter(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_scatter(m, ls, s)); }
inline void launch_m_cell(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_cell(m, ls, s)); }
inline void launch_m_cell_big(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_cell_big(m, ls, s)); }
inline void launch_m_collide_big(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_collide_big(m, ls, s)); }
inline void launch_m_collide(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_collide(m, ls, s)); }
inline void launch_m_reduce(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_reduce(m, ls, s)); }
inline void launch_m_step_end(int p, const void* m, const LaunchShape& ls, cudaStream_t s) { DSMC_PICK(p, launch_m_step_end(m, ls, s)); }
inline cudaError_t prepare_multi_kernels(int p, int dim, int tile_budget, int collide_stage) { return DSMC_PICK(p, prepare_multi_kernels(dim, tile_budget, collide_stage)); }
inline void compute_multi_shape(int p, int dim, int sms, LaunchShape* ls) { DSMC_PICK(p, compute_multi_shape(dim, sms, ls)); }
inline void compute_launch_shape(int p, int dim, int sms, LaunchShape* ls) { DSMC_PICK(p, compute_launch_shape(dim, sms, ls)); }
inline int big_cell_limit(int p) { return DSMC_PICK(p, big_cell_limit()); }

// precision-independent (defined in the FP32 compilation)
cudaError_t timeout_probe(Counters* ctr, uint32_t polls, cudaStream_t s);
cudaError_t philox_device(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t s);

}  // namespace dsmc
