// dsmc_engine.cu -- host engine and C ABI of libdsmc.so.
//
// The engine owns the device buffers of one problem, sizes them from the
// workload, and drives the step kernels either for all runs at once
// (batched: one launch per kernel per step, replayed from one of four CUDA
// graphs -- buffer parity x whether the step closes a sample window --
// with Generation forked beside Motion) or one run after another (plain,
// direct launches with programmatic dependent launch).  It also holds the
// launch-shape autotuner, the test hooks and the no-allocation entry point.
// Everything a step computes happens in the kernels of dsmc_kernels.cu; the
// host only derives constants, allocates, launches and copies results out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <nvtx3/nvToolsExt.h>
#include <new>
#include <string>
#include <vector>

#include "dsmc_internal.cuh"

using namespace dsmc;

namespace {

constexpr double kB = 1.380649e-23;

struct DevBuf {
    void* p;
    size_t bytes;
};

struct AnyArgs {
    StepArgs<float> f;
    StepArgs<double> d;
};

}  // namespace

struct dsmc_ctx {
    dsmc_domain dom;
    dsmc_cells cells;
    dsmc_gas gas;
    std::vector<dsmc_boundary> bcs;
    dsmc_options opt;
    std::string err;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int prec = DSMC_FP32, dim = 2, ncells = 0, sms = 0;
    Cfg hcfg;
    LaunchShape ls;
    // allocation state
    std::vector<DevBuf> bufs;
    int n_launch = 0;
    int64_t cap_old = 0, cap_new = 0, gcap = 0, max_big = 0;
    int64_t total_cells = 0;
    int n_samples_alloc = 0, steps_alloc = 0, G_alloc = 0;
    bool debug_alloc = false;
    uint64_t generation = 0;      // bumps on every reallocation
    // device pointers
    Cfg* d_cfg = nullptr;
    Counters* d_ctr = nullptr;
    void* X[2][3] = {};
    void* V[2][3] = {};
    uint32_t* ID[2] = {};
    uint32_t* CI[2] = {};            // run-local cell index of each pool particle
    uint32_t *gc = nullptr, *lcr_dbg = nullptr;
    uint32_t* lcr = nullptr;
    uint32_t *count = nullptr, *start = nullptr, *block_sums = nullptr;
    uint32_t *run_base = nullptr, *next_id = nullptr, *cand = nullptr, *accd = nullptr;
    uint32_t* big_list = nullptr;
    uint32_t* slow_list = nullptr;
    uint32_t *gen_tot = nullptr, *gen_done = nullptr;
    double *rem = nullptr, *mom = nullptr, *acc = nullptr, *macro = nullptr;
    void* smax = nullptr;
    int32_t* sample_slot = nullptr;
    int cur = 0;
    int G = 1;
    // graphs (batched): one per buffer parity and kind of step (without /
    // with sampling), valid for graph_key; inside a graph Generation runs
    // on a side stream beside Motion
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    uint64_t graph_key = ~0ull;
    uint64_t tuned_key = 0;          // (runs << 1) | 1 once options.autotune ran
    int tuned_how = 0;               // 1: searched, 2: read from the tune cache
    std::string tune_cache;          // options.tune_cache
    // last run
    bool have_run = false;
    int last_runs = 0, last_steps = 0, last_samples = 0;
    std::vector<int> win_len;        // steps of each sample window of the last run
    // debug stepping
    bool dbg = false;
    std::vector<uint32_t> prev_run_base;
    dsmc_stats stats;
    std::vector<cudaEvent_t> events;
};

static const char* g_static_err = "invalid context";

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return DSMC_E_CUDA;                                                           \
        }                                                                                 \
    } while (0)

static dsmc_status fail(dsmc_ctx* ctx, dsmc_status s, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    return s;
}

// ---------------------------------------------------------------------------
// configuration

static dsmc_status build_cfg(dsmc_ctx* ctx, double dt, uint64_t seed)
{
    Cfg& c = ctx->hcfg;
    std::memset(&c, 0, sizeof(c));
    const dsmc_domain& D = ctx->dom;
    c.dim = D.dim;
    for (int a = 0; a < 3; ++a) c.n[a] = (a < D.dim) ? ctx->cells.n[a] : 1;
    c.ncells = c.n[0] * c.n[1] * c.n[2];
    for (int a = 0; a < 3; ++a) {
        c.L[a] = D.extent[a];
        c.d[a] = c.L[a] / c.n[a];
        c.inv_d[a] = 1.0 / c.d[a];
    }
    c.Vc = c.d[0] * c.d[1] * c.d[2];
    // multiply-high division by ncells: exact for every 32-bit key
    c.ncells_magic = c.ncells > 1 ? (~0ull) / (uint64_t)c.ncells + 1ull : 0ull;
    c.dt = dt;
    c.mass = ctx->gas.mass;
    c.F_N = ctx->gas.F_N;
    c.coef = (ctx->gas.F_N * dt) / c.Vc;
    c.coef_f = (float)c.coef;
    const double omega = ctx->gas.omega;
    const double dref = ctx->gas.d_ref;
    c.hs = (omega == 0.5) ? 1 : 0;
    c.partner = ctx->gas.partner;
    c.n_sub = ctx->gas.partner == DSMC_PARTNER_SUBCELL ? ctx->gas.n_sub : 1;
    c.A_hs = M_PI * (dref * dref);
    const double mr = ctx->gas.mass / 2.0;
    c.K_vhs = M_PI * (dref * dref) * std::pow(2.0 * kB * ctx->gas.T_ref / mr, omega - 0.5) /
              std::tgamma(2.5 - omega);
    c.one_m_omega = 1.0 - omega;
    c.seed = seed;
    c.fill = D.fill;
    c.fill_lam = D.fill_n * c.Vc / ctx->gas.F_N;
    c.fill_sd = std::sqrt(kB * D.fill_T / ctx->gas.mass);
    for (int a = 0; a < 3; ++a) c.fill_U[a] = D.fill_U[a];
    double T0 = D.fill ? D.fill_T : 0.0;
    c.n_bc = (int)ctx->bcs.size();
    int64_t eb = 0;
    for (int q = 0; q < c.n_bc; ++q) {
        const dsmc_boundary& b = ctx->bcs[q];
        BcDev& o = c.bc[q];
        o.kind = b.kind;
        o.face = b.face;
        for (int k = 0; k < 2; ++k) { o.lo[k] = b.lo[k]; o.hi[k] = b.hi[k]; }
        o.step_from = b.step_from;
        o.step_to = b.step_to;
        o.plate_axis = b.plate_axis;
        o.plate_index = b.plate_index;
        o.T = b.T;
        for (int a = 0; a < 3; ++a) o.U[a] = b.U[a];
        const int axis = b.face < 6 ? b.face / 2 : b.plate_axis;
        o.axis = axis;
        o.side = b.face < 6 ? b.face % 2 : 0;
        o.t0 = axis == 0 ? 1 : 0;
        o.t1 = axis == 2 ? 1 : 2;
        o.sd = std::sqrt(kB * b.T / ctx->gas.mass);
        o.dir = o.side ? -1.0 : 1.0;
        if ((b.kind == DSMC_BC_INFLOW || b.kind == DSMC_BC_DIFFUSE) && b.T > T0) T0 = b.T;
        if (b.face == DSMC_FACE_PLATE) {
            c.plate_idx[c.n_plate++] = q;
            o.xp = (double)b.plate_index * c.d[axis];
        }
        o.elem_base = eb;
        if (b.kind == DSMC_BC_INFLOW && b.face < 6) {
            o.elem_w = b.hi[0] - b.lo[0];
            o.n_elem = (int64_t)(b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]);
            eb += o.n_elem;
            o.cmp = std::sqrt(2.0 * kB * b.T / ctx->gas.mass);
            const double Un = o.dir * b.U[axis];
            o.s = Un / o.cmp;
            // drifting-Maxwellian number flux through the face
            const double flux = b.n * o.cmp / (2.0 * std::sqrt(M_PI)) *
                                (std::exp(-o.s * o.s) + std::sqrt(M_PI) * o.s * (1.0 + std::erf(o.s)));
            const double area = c.d[o.t0] * c.d[o.t1];
            o.lam = flux * area * dt / ctx->gas.F_N;
            o.xm = (o.s + std::sqrt(o.s * o.s + 2.0)) / 2.0;
        }
    }
    c.n_elem = eb;
    if (T0 <= 0.0) T0 = ctx->gas.T_ref;
    // sigma_T(c0) c0 at three most probable speeds of the hottest state
    const double c0 = 3.0 * std::sqrt(2.0 * kB * T0 / ctx->gas.mass);
    const double sig0 = M_PI * (dref * dref) *
                        std::pow(2.0 * kB * ctx->gas.T_ref / (mr * c0 * c0), omega - 0.5) /
                        std::tgamma(2.5 - omega);
    c.smax0 = sig0 * c0;
    return DSMC_OK;
}

// particles one run may hold, estimated from the fill, the inflow over the
// whole run and the densest state the run is driven with
static int64_t estimate_per_run(const dsmc_ctx* ctx, int steps)
{
    if (ctx->opt.capacity_per_run > 0) return ctx->opt.capacity_per_run;
    const Cfg& c = ctx->hcfg;
    double fill = c.fill ? (c.fill_lam + 1.0) * c.ncells : 0.0;
    double gen = 0.0, nmax = c.fill ? ctx->dom.fill_n : 0.0;
    for (int q = 0; q < c.n_bc; ++q) {
        const BcDev& b = c.bc[q];
        if (!(b.kind == DSMC_BC_INFLOW && b.face < 6)) continue;
        const int from = std::max(1, b.step_from);
        const int to = b.step_to == 0 ? steps : std::min(steps, b.step_to);
        const int act = std::max(0, to - from + 1);
        gen += std::ceil(b.lam) * (double)b.n_elem * act;
        nmax = std::max(nmax, ctx->bcs[q].n);
    }
    const double dens = 1.5 * nmax * c.Vc * c.ncells / ctx->gas.F_N;
    double est = fill + gen;
    if (dens > fill && est > dens) est = dens;
    const double factor = ctx->opt.capacity_factor > 0 ? ctx->opt.capacity_factor : 1.25;
    return (int64_t)(est * factor) + 1024;
}

static int64_t gen_capacity(const dsmc_ctx* ctx)
{
    const Cfg& c = ctx->hcfg;
    double g = 0.0;
    for (int q = 0; q < c.n_bc; ++q) {
        const BcDev& b = c.bc[q];
        if (b.kind == DSMC_BC_INFLOW && b.face < 6) g += std::ceil(b.lam) * (double)b.n_elem;
    }
    return ((int64_t)g + 32 + 31) / 32 * 32;
}

// ---------------------------------------------------------------------------
// memory

static void* dev_alloc(dsmc_ctx* ctx, size_t bytes)
{
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (ctx->opt.alloc) {
        p = ctx->opt.alloc(bytes, ctx->opt.alloc_user, (void*)ctx->stream);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) ctx->bufs.push_back({p, bytes});
    return p;
}

// NVTX range for the profilers' timelines (header-only NVTX3; a no-op
// when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static void destroy_graphs(dsmc_ctx* ctx)
{
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < 2; ++k)
            if (ctx->gexec[p][k]) {
                cudaGraphExecDestroy(ctx->gexec[p][k]);
                ctx->gexec[p][k] = nullptr;
            }
    ctx->graph_key = ~0ull;
}

static void free_all(dsmc_ctx* ctx)
{
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    destroy_graphs(ctx);
    for (const DevBuf& b : ctx->bufs) {
        if (ctx->opt.free) ctx->opt.free(b.p, b.bytes, ctx->opt.alloc_user, (void*)ctx->stream);
        else cudaFree(b.p);
    }
    ctx->bufs.clear();
    ctx->n_launch = 0;
    ctx->cap_old = 0;
}

// Generation CTAs per run: one per kGenElems inflow elements
static int gen_groups_of(const dsmc_ctx* ctx)
{
    const int64_t g = (ctx->hcfg.n_elem + kGenElems - 1) / kGenElems;
    return g < 1 ? 1 : (int)g;
}

static dsmc_status ensure_alloc(dsmc_ctx* ctx, int n_launch, int64_t cap_run, int steps,
                                int n_samples, int G)
{
    const int64_t cap_old = (cap_run * n_launch + 255) / 256 * 256;
    const int64_t gcap = gen_capacity(ctx);
    const int64_t cap_new = gcap * n_launch;
    const int64_t total_cells = (int64_t)ctx->ncells * n_launch;
    const bool dbg = ctx->opt.debug != 0;
    if (cap_old + cap_new >= 0xFFFFFFF0ll || total_cells >= 0x7FFFFFF0ll)
        return fail(ctx, DSMC_E_INVALID, "problem too large for 32-bit particle slots");
    if (ctx->n_launch == n_launch && ctx->cap_old >= cap_old && ctx->gcap == gcap &&
        ctx->steps_alloc >= steps + 2 && ctx->n_samples_alloc >= n_samples && ctx->G_alloc == G &&
        ctx->debug_alloc == dbg)
        return DSMC_OK;
    free_all(ctx);
    const size_t ts = ctx->prec == DSMC_FP64 ? 8 : 4;
    const int64_t slots = cap_old + cap_new;
    bool ok = true;
    auto A = [&](size_t bytes) -> void* {
        void* p = dev_alloc(ctx, bytes);
        if (!p) ok = false;
        return p;
    };
    ctx->d_cfg = (Cfg*)A(sizeof(Cfg));
    ctx->d_ctr = (Counters*)A(sizeof(Counters));
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 3; ++a) {
            ctx->X[b][a] = a < ctx->dim ? A(ts * slots) : nullptr;
            ctx->V[b][a] = A(ts * slots);
        }
        ctx->ID[b] = dbg ? (uint32_t*)A(4 * slots) : nullptr;   // ids: debug bookkeeping only
        ctx->CI[b] = (uint32_t*)A(4 * cap_old);
    }
    ctx->gc = (uint32_t*)A(4 * slots);
    ctx->lcr = (uint32_t*)A(4 * cap_old);
    ctx->lcr_dbg = dbg ? (uint32_t*)A(4 * cap_old) : nullptr;
    ctx->count = (uint32_t*)A(4 * total_cells);
    ctx->start = (uint32_t*)A(4 * (total_cells + 2));
    const int scan_blocks = (int)((total_cells + kScanTile - 1) / kScanTile);
    ctx->block_sums = (uint32_t*)A(4 * (scan_blocks + 1));
    ctx->run_base = (uint32_t*)A(4 * (n_launch + 1));
    ctx->next_id = (uint32_t*)A(4 * n_launch);
    ctx->rem = (double*)A(8 * total_cells);
    ctx->smax = A(ts * total_cells);
    ctx->mom = (double*)A(8 * DSMC_NMOM * total_cells);
    ctx->cand = dbg ? (uint32_t*)A(4 * total_cells) : nullptr;
    ctx->accd = dbg ? (uint32_t*)A(4 * total_cells) : nullptr;
    const int64_t max_big = cap_old / (kWarpMax + 1) + 1;
    ctx->big_list = (uint32_t*)A(4 * max_big);
    ctx->slow_list = (uint32_t*)A(4 * cap_old);
    ctx->gen_tot = (uint32_t*)A(4 * (size_t)n_launch * gen_groups_of(ctx));
    ctx->gen_done = (uint32_t*)A(4 * (size_t)n_launch);
    ctx->sample_slot = (int32_t*)A(4 * (size_t)(steps + 2));
    ctx->acc = (double*)A(8 * (size_t)std::max(n_samples, 1) * G * ctx->ncells * DSMC_NMOM);
    ctx->macro = (double*)A(8 * 10 * (size_t)ctx->ncells);
    if (!ok) {
        free_all(ctx);
        return fail(ctx, DSMC_E_OOM, "device allocation failed");
    }
    ctx->n_launch = n_launch;
    ctx->cap_old = cap_old;
    ctx->cap_new = cap_new;
    ctx->gcap = gcap;
    ctx->max_big = max_big;
    ctx->total_cells = total_cells;
    ctx->steps_alloc = steps + 2;
    ctx->n_samples_alloc = n_samples;
    ctx->G_alloc = G;
    ctx->debug_alloc = dbg;
    ctx->generation++;
    // the new-region cell keys start dead; every scatter re-kills them
    CK(cudaMemsetAsync(ctx->gc, 0xFF, 4 * slots, ctx->stream));
    return DSMC_OK;
}

template <typename T>
static StepArgs<T> args_for(const dsmc_ctx* ctx, int cur, int run0, int n)
{
    StepArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.cfg = ctx->d_cfg;
    const Cfg& c = ctx->hcfg;
    for (int ax = 0; ax < 3; ++ax) {
        a.hot.d[ax] = (T)c.d[ax];
        a.hot.inv_d[ax] = (float)c.inv_d[ax];
        a.hot.n[ax] = c.n[ax];
    }
    a.hot.dt = (T)c.dt;
    a.hot.ncells = c.ncells;
    a.hot.plate_axes = 0u;
    for (int pi = 0; pi < c.n_plate; ++pi) a.hot.plate_axes |= 1u << c.bc[c.plate_idx[pi]].plate_axis;
    a.hot.n_plate = c.n_plate <= 4 ? c.n_plate : -1;
    for (int pi = 0; pi < 4; ++pi) {
        a.hot.plate_ax[pi] = pi < c.n_plate ? c.bc[c.plate_idx[pi]].plate_axis : 0;
        a.hot.plate_ix[pi] = pi < c.n_plate ? c.bc[c.plate_idx[pi]].plate_index : 0;
    }
    a.hot.hs = c.hs;
    a.hot.dim = c.dim;
    a.hot.partner = c.partner;
    a.hot.n_sub = c.n_sub;
    a.hot.ncells_magic = c.ncells_magic;
    a.hot.seed = c.seed;
    a.hot.A_hs = (T)c.A_hs;
    a.hot.K_vhs = (T)c.K_vhs;
    a.hot.one_m_omega = (T)c.one_m_omega;
    a.hot.coef = c.coef;
    a.hot.coef_f = c.coef_f;
    for (int r = 0; r < 10; ++r) {
        a.hot.rk[2 * r] = (uint32_t)c.seed + (uint32_t)r * 0x9E3779B9u;
        a.hot.rk[2 * r + 1] = (uint32_t)(c.seed >> 32) + (uint32_t)r * 0xBB67AE85u;
    }
    a.ctr = ctx->d_ctr;
    for (int ax = 0; ax < 3; ++ax) {
        a.xi[ax] = (T*)ctx->X[cur][ax];
        a.vi[ax] = (T*)ctx->V[cur][ax];
        a.xo[ax] = (T*)ctx->X[1 - cur][ax];
        a.vo[ax] = (T*)ctx->V[1 - cur][ax];
    }
    a.idi = ctx->ID[cur];
    a.ci_i = ctx->CI[cur];
    a.ci_o = ctx->CI[1 - cur];
    a.ido = ctx->ID[1 - cur];
    a.gc = ctx->gc;
    a.lcr = ctx->lcr;
    a.lcr_dbg = ctx->lcr_dbg;
    a.count = ctx->count;
    a.start = ctx->start;
    a.block_sums = ctx->block_sums;
    a.run_base = ctx->run_base;
    a.next_id = ctx->next_id;
    a.rem = ctx->rem;
    a.smax = (T*)ctx->smax;
    a.mom = ctx->mom;
    a.cand = ctx->cand;
    a.accd = ctx->accd;
    a.big_list = ctx->big_list;
    a.slow_list = ctx->slow_list;
    a.gen_tot = ctx->gen_tot;
    a.gen_done = ctx->gen_done;
    a.gen_groups = gen_groups_of(ctx);
    a.sample_slot = ctx->sample_slot;
    a.n_slot = ctx->steps_alloc;
    a.acc = ctx->acc;
    a.cap_old = ctx->cap_old;
    a.cap_new = ctx->cap_new;
    a.gcap = ctx->gcap;
    a.max_big = ctx->max_big;
    a.n_runs = n;
    a.run0 = run0;
    a.G = ctx->G;
    a.total_cells = (int32_t)((int64_t)ctx->ncells * n);
    a.scan_blocks = (int)((a.total_cells + kScanTile - 1) / kScanTile);
    a.tile_budget = ctx->ls.tile_budget;
    a.collide_stage = ctx->ls.collide_stage;
    return a;
}

static const void* build_args(const dsmc_ctx* ctx, AnyArgs& u, int cur, int run0, int n)
{
    if (ctx->prec == DSMC_FP64) {
        u.d = args_for<double>(ctx, cur, run0, n);
        return &u.d;
    }
    u.f = args_for<float>(ctx, cur, run0, n);
    return &u.f;
}

// ---------------------------------------------------------------------------
// step sequencing

static cudaEvent_t event_at(dsmc_ctx* ctx, size_t i)
{
    while (ctx->events.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->events.push_back(e);
    }
    return ctx->events[i];
}

// One time step.  `ev` (profile mode) records an event after each kernel
// group.  `fork` (graph capture only) runs Generation on the side stream
// beside Motion: they touch disjoint slots and only add to the cell counts.
// `reduce` = false leaves out the reduction over runs, for graphs of steps
// that take no sample (the kernel would find no sample slot and return).
static void enqueue_step(dsmc_ctx* ctx, const void* args, size_t* ev, bool fork = false,
                         bool reduce = true)
{
    const int p = ctx->prec;
    LaunchShape ls = ctx->ls;
    ls.pdl = fork ? 0 : 1;
    cudaStream_t s = ctx->stream;
    auto mark = [&]() {
        if (ev) cudaEventRecord(event_at(ctx, (*ev)++), s);
    };
    if (fork) {
        cudaEventRecord(ctx->ev_fork, s);
        cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
        launch_generate(p, args, ls, ctx->side);
        cudaEventRecord(ctx->ev_join, ctx->side);
        launch_move(p, args, ls, s);
        cudaStreamWaitEvent(s, ctx->ev_join, 0);
    } else {
        launch_generate(p, args, ls, s); mark();
        launch_move(p, args, ls, s); mark();
    }
    launch_scan(p, args, ls, s); mark();
    launch_scatter(p, args, ls, s); mark();
    launch_cell(p, args, ls, s); mark();
    launch_cell_big(p, args, ls, s); mark();
    launch_collide_big(p, args, ls, s); mark();
    launch_collide(p, args, ls, s); mark();
    if (reduce) launch_reduce(p, args, ls, s);
    mark();
    launch_step_end(p, args, ls, s); mark();
}
static const int kStepKernels = 10;
static const int kKindOf[kStepKernels] = {DSMC_K_GENERATE,  DSMC_K_MOVE,        DSMC_K_SCAN,
                                          DSMC_K_SCATTER,   DSMC_K_CELL,        DSMC_K_CELL_BIG,
                                          DSMC_K_COLLIDE_BIG, DSMC_K_COLLIDE,   DSMC_K_REDUCE,
                                          DSMC_K_OTHER};
// position of each tuned kernel group in enqueue_step's order
static const int kGroupMove = 1, kGroupScatter = 3, kGroupCell = 4, kGroupCollide = 7;

static void enqueue_init(dsmc_ctx* ctx, const void* args)
{
    launch_init_cells(ctx->prec, args, ctx->ls, ctx->stream);
    launch_fill(ctx->prec, args, ctx->ls, ctx->stream);
}

static dsmc_status upload_cfg(dsmc_ctx* ctx)
{
    CK(cudaMemcpyAsync(ctx->d_cfg, &ctx->hcfg, sizeof(Cfg), cudaMemcpyHostToDevice, ctx->stream));
    ctx->stats.h2d_bytes += sizeof(Cfg);
    return DSMC_OK;
}

static dsmc_status reset_counters(dsmc_ctx* ctx)
{
    CK(cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), ctx->stream));
    return DSMC_OK;
}

static dsmc_status read_counters(dsmc_ctx* ctx, Counters* h)
{
    CK(cudaMemcpyAsync(h, ctx->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->stats.d2h_bytes += sizeof(Counters);
    CK(cudaStreamSynchronize(ctx->stream));
    return DSMC_OK;
}

static void fill_stats(dsmc_ctx* ctx, const Counters& h)
{
    dsmc_stats& s = ctx->stats;
    s.particle_steps = h.particle_steps;
    s.generated = h.generated;
    s.removed = h.removed;
    s.wall_hits = h.wall_hits;
    s.candidates = h.candidates;
    s.collisions = h.collisions;
    s.clamps = h.clamps;
    s.bounce_limit = h.bounce_limit;
    s.reject_limit = h.reject_limit;
    s.pool_steps = h.pool_steps;
    s.big_pool_steps = h.big_pool_steps;
    s.error_word = h.error;
    s.capacity = ctx->cap_old;
    s.shape[0] = ctx->ls.move_blocks;
    s.shape[1] = ctx->ls.scatter_blocks;
    s.shape[2] = ctx->ls.tile_budget;
    s.shape[3] = ctx->ls.collide_blocks;
    s.tuned = ctx->tuned_key != 0 ? ctx->tuned_how : 0;
}

static dsmc_status check_error_word(dsmc_ctx* ctx, uint32_t e)
{
    if (!e) return DSMC_OK;
    char buf[256];
    if (e & DSMC_ERR_TIMEOUT) {
        std::snprintf(buf, sizeof buf,
                      "device error word 0x%x: a bounded wait for a bulk copy expired", e);
        ctx->err = buf;
        return DSMC_E_TIMEOUT;
    }
    std::snprintf(buf, sizeof buf,
                  "device error word 0x%x (pool=%d gen=%d bigcell=%d biglist=%d); "
                  "raise capacity_factor / capacity_per_run",
                  e, !!(e & DSMC_ERR_POOL), !!(e & DSMC_ERR_GEN), !!(e & DSMC_ERR_BIGCELL),
                  !!(e & DSMC_ERR_BIGLIST));
    ctx->err = buf;
    return DSMC_E_CAPACITY;
}

// sample windows: [first[k], last[k]] inside [1, steps], increasing and
// disjoint (a plain sample list is first = last)
static dsmc_status validate_run(dsmc_ctx* ctx, int n_runs, double dt, int steps,
                                const int32_t* first, const int32_t* last, int n_samples)
{
    if (n_runs < 1 || n_runs > (1 << 20) || ctx->opt.run_offset + n_runs > (1ll << 31))
        return fail(ctx, DSMC_E_INVALID, "n_runs out of range");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, DSMC_E_INVALID, "dt must be > 0");
    if (steps < 0 || steps > (1 << 26)) return fail(ctx, DSMC_E_INVALID, "steps out of range");
    if (n_samples < 0 || n_samples > kMaxSamples || (n_samples > 0 && (!first || !last)))
        return fail(ctx, DSMC_E_INVALID, "bad sample list");
    for (int k = 0; k < n_samples; ++k)
        if (first[k] < 1 || last[k] > steps || first[k] > last[k] ||
            (k > 0 && first[k] <= last[k - 1]))
            return fail(ctx, DSMC_E_INVALID,
                        "sample steps (windows) must be increasing and disjoint in [1, steps]");
    return DSMC_OK;
}

// set up everything a run needs up to (not including) the step-0 state
static dsmc_status prepare(dsmc_ctx* ctx, int n_runs, double dt, int steps, const int32_t* first,
                           const int32_t* last, int n_samples, uint64_t seed, int n_launch)
{
    dsmc_status st = build_cfg(ctx, dt, seed);
    if (st) return st;
    ctx->G = std::min(n_runs, DSMC_MAX_GROUPS);
    const int64_t cap_run = estimate_per_run(ctx, steps);
    st = ensure_alloc(ctx, n_launch, cap_run, steps, n_samples, ctx->G);
    if (st) return st;
    st = upload_cfg(ctx);
    if (st) return st;
    std::vector<int32_t> slot(steps + 2, -1);
    for (int k = 0; k < n_samples; ++k)
        for (int s = first[k]; s <= last[k]; ++s)
            slot[s] = k | (s == first[k] ? kSlotFirst : 0) | (s == last[k] ? kSlotLast : 0);
    ctx->stats.h2d_bytes += 4 * slot.size();
    CK(cudaMemcpyAsync(ctx->sample_slot, slot.data(), 4 * slot.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    // the upload source is a host vector: finish before it goes away
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemsetAsync(ctx->acc, 0,
                       8 * (size_t)std::max(n_samples, 1) * ctx->G * ctx->ncells * DSMC_NMOM,
                       ctx->stream));
    if (ctx->cand) {
        CK(cudaMemsetAsync(ctx->cand, 0, 4 * ctx->total_cells, ctx->stream));
        CK(cudaMemsetAsync(ctx->accd, 0, 4 * ctx->total_cells, ctx->stream));
    }
    st = reset_counters(ctx);
    if (st) return st;
    CK(prepare_kernels(ctx->prec, ctx->dim, ctx->ls.tile_budget, ctx->ls.collide_stage));
    return DSMC_OK;
}

static dsmc_status build_graphs(dsmc_ctx* ctx, int n_runs)
{
    NvtxRange range("dsmc graph capture");
    const uint64_t key = (ctx->generation << 24) ^ (uint64_t)n_runs;
    if (ctx->graph_key == key && ctx->gexec[0][0] && ctx->gexec[0][1] && ctx->gexec[1][0] &&
        ctx->gexec[1][1])
        return DSMC_OK;
    destroy_graphs(ctx);
    if (!ctx->side) CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    if (!ctx->ev_fork) CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    if (!ctx->ev_join) CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    for (int p = 0; p < 2; ++p)
        for (int smp = 0; smp < 2; ++smp) {
            AnyArgs u;
            const void* args = build_args(ctx, u, p, (int)ctx->opt.run_offset, n_runs);
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            enqueue_step(ctx, args, nullptr, true, smp != 0);
            CK(cudaStreamEndCapture(ctx->stream, &g));
            cudaError_t e = cudaGraphInstantiate(&ctx->gexec[p][smp], g, 0);
            cudaGraphDestroy(g);
            CK(e);
        }
    ctx->graph_key = key;
    return DSMC_OK;
}

// ---------------------------------------------------------------------------
// C ABI (C linkage comes from the declarations in dsmc.h)

// Staged particles a cell that the default collision shape aims at: 1.1 x
// the particles a cell holds at the densest state the run is driven with
// (the fill or an inflow), within 18 .. 22 (a denser inflow, as a jet's
// orifice, feeds cells that the big-cell kernels take).
static int collide_ppc_target(const dsmc_ctx* ctx)
{
    double vc = 1.0;
    for (int a = 0; a < 3; ++a) vc *= ctx->dom.extent[a] / (double)ctx->cells.n[a];
    double n = ctx->dom.fill ? ctx->dom.fill_n : 0.0;
    for (const dsmc_boundary& b : ctx->bcs)
        if (b.kind == DSMC_BC_INFLOW && b.face != DSMC_FACE_PLATE) n = std::max(n, b.n);
    const double ppc = std::ceil(1.1 * n * vc / ctx->gas.F_N);
    return (int)std::min(22.0, std::max(18.0, ppc));
}

// the collision stage follows the collision CTAs per SM
static void follow_collide_blocks(int prec, int sms, LaunchShape* ls)
{
    ls->collide_stage = collide_stage_for(prec, std::max(1, ls->collide_blocks / sms), 0);
}

dsmc_status dsmc_create(const dsmc_domain* domain, const dsmc_cells* cells, const dsmc_gas* gas,
                        const dsmc_boundary* b, int n_b, const dsmc_options* opt, dsmc_ctx** out)
{
    if (!out) return DSMC_E_INVALID;
    *out = nullptr;
    if (!domain || !cells || !gas || (n_b > 0 && !b) || n_b < 0 || n_b > DSMC_MAX_BC)
        return DSMC_E_INVALID;
    if (domain->struct_size < sizeof(dsmc_domain) || cells->struct_size < sizeof(dsmc_cells) ||
        gas->struct_size < offsetof(dsmc_gas, partner) ||
        (opt && opt->struct_size < offsetof(dsmc_options, checks)))
        return DSMC_E_INVALID;
    if (domain->dim != 2 && domain->dim != 3) return DSMC_E_INVALID;
    for (int a = 0; a < domain->dim; ++a)
        if (cells->n[a] < 1 || !(domain->extent[a] > 0.0)) return DSMC_E_INVALID;
    if (domain->dim == 2 && !(domain->extent[2] > 0.0)) return DSMC_E_INVALID;
    const int64_t nc = (int64_t)cells->n[0] * cells->n[1] * (domain->dim == 3 ? cells->n[2] : 1);
    if (nc > (1 << 24)) return DSMC_E_INVALID;
    if (!(gas->mass > 0.0) || !(gas->d_ref >= 0.0) || !(gas->F_N > 0.0) || !(gas->T_ref > 0.0) ||
        !(gas->omega >= 0.5 && gas->omega <= 1.0))
        return DSMC_E_INVALID;
    // an older caller's gas ends before the partner choice: uniform
    dsmc_gas g_in;
    std::memset(&g_in, 0, sizeof(g_in));
    std::memcpy(&g_in, gas, std::min<size_t>(gas->struct_size, sizeof(dsmc_gas)));
    g_in.struct_size = sizeof(dsmc_gas);
    if (gas->struct_size < sizeof(dsmc_gas)) {
        g_in.partner = DSMC_PARTNER_UNIFORM;
        g_in.n_sub = 1;
    }
    if (g_in.partner < DSMC_PARTNER_UNIFORM || g_in.partner > DSMC_PARTNER_NEAREST ||
        (g_in.partner == DSMC_PARTNER_SUBCELL && (g_in.n_sub < 1 || g_in.n_sub > 64)))
        return DSMC_E_INVALID;
    if (domain->fill && !(domain->fill_n >= 0.0 && domain->fill_T > 0.0)) return DSMC_E_INVALID;
    for (int q = 0; q < n_b; ++q) {
        const dsmc_boundary& s = b[q];
        if (s.struct_size < sizeof(dsmc_boundary)) return DSMC_E_INVALID;
        if (s.kind < 0 || s.kind > 3) return DSMC_E_INVALID;
        if (s.face == DSMC_FACE_PLATE) {
            if (s.kind != DSMC_BC_SPECULAR && s.kind != DSMC_BC_DIFFUSE) return DSMC_E_INVALID;
            if (s.plate_axis < 0 || s.plate_axis >= domain->dim) return DSMC_E_INVALID;
            if (s.plate_index < 1 || s.plate_index > cells->n[s.plate_axis] - 1) return DSMC_E_INVALID;
        } else if (s.face < 0 || s.face >= 2 * domain->dim) {
            return DSMC_E_INVALID;
        }
        if ((s.kind == DSMC_BC_DIFFUSE || s.kind == DSMC_BC_INFLOW) && !(s.T > 0.0))
            return DSMC_E_INVALID;
        if (s.kind == DSMC_BC_INFLOW && !(s.n >= 0.0)) return DSMC_E_INVALID;
        if (s.lo[0] < 0 || s.hi[0] < s.lo[0] || s.lo[1] < 0 || s.hi[1] < s.lo[1]) return DSMC_E_INVALID;
        const int ax = s.face == DSMC_FACE_PLATE ? s.plate_axis : s.face / 2;
        const int t0 = ax == 0 ? 1 : 0, t1 = ax == 2 ? 1 : 2;
        const int n0 = cells->n[t0], n1 = t1 < domain->dim ? cells->n[t1] : 1;
        if (s.hi[0] > n0 || s.hi[1] > n1) return DSMC_E_INVALID;
        if (s.step_from < 0 || s.step_to < 0) return DSMC_E_INVALID;
    }
    if (opt && opt->struct_size >= sizeof(dsmc_options) &&
        (opt->autotune < DSMC_TUNE_OFF || opt->autotune > DSMC_TUNE_LOAD ||
         (opt->autotune == DSMC_TUNE_LOAD && !opt->tune_cache)))
        return DSMC_E_INVALID;
    if (opt) {
        for (int i = 0; i < 4; ++i) {
            const int32_t v = opt->shape[i];
            const bool ok = v == 0 || (i == 2 ? v >= 256 && v <= kMaxTileBudget
                                              : v >= 1 && v <= (1 << 20));
            if (!ok) return DSMC_E_INVALID;
        }
    }
    dsmc_ctx* ctx = new (std::nothrow) dsmc_ctx();
    if (!ctx) return DSMC_E_OOM;
    ctx->dom = *domain;
    ctx->cells = *cells;
    if (domain->dim == 2) ctx->cells.n[2] = 1;
    ctx->gas = g_in;
    ctx->bcs.assign(b, b + n_b);
    std::memset(&ctx->opt, 0, sizeof(ctx->opt));
    ctx->opt.struct_size = sizeof(dsmc_options);
    ctx->opt.use_graph = 1;
    // an older caller's struct is shorter: the fields it lacks stay zero
    if (opt) std::memcpy(&ctx->opt, opt, std::min<size_t>(opt->struct_size, sizeof(dsmc_options)));
    ctx->opt.struct_size = sizeof(dsmc_options);
    if (ctx->opt.tune_cache) {
        ctx->tune_cache = ctx->opt.tune_cache;   // the library keeps its own copy
        ctx->opt.tune_cache = nullptr;
    }
    ctx->prec = ctx->opt.precision == DSMC_FP64 ? DSMC_FP64 : DSMC_FP32;
    ctx->dim = domain->dim;
    ctx->ncells = (int)nc;
    ctx->device = ctx->opt.device;
    std::memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.struct_size = sizeof(dsmc_stats);
    if (ctx->opt.run_offset < 0 || ctx->opt.run_offset > (1ll << 30) ||
        (ctx->opt.alloc == nullptr) != (ctx->opt.free == nullptr)) {
        delete ctx;
        return DSMC_E_INVALID;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return DSMC_E_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return DSMC_E_CUDA;
    }
    ctx->sms = prop.multiProcessorCount;
    if (ctx->opt.stream) {
        ctx->stream = (cudaStream_t)ctx->opt.stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return DSMC_E_CUDA;
        }
        ctx->own_stream = true;
    }
    // default shape (the occupancy of the tile kernel follows the budget),
    // then the caller's entries
    ctx->ls.tile_budget = ctx->opt.shape[2];
    ctx->ls.collide_ppc = collide_ppc_target(ctx);
    compute_launch_shape(ctx->prec, ctx->dim, ctx->sms, &ctx->ls);
    if (ctx->opt.shape[0] > 0) ctx->ls.move_blocks = ctx->opt.shape[0];
    if (ctx->opt.shape[1] > 0) ctx->ls.scatter_blocks = ctx->opt.shape[1];
    if (ctx->opt.shape[3] > 0) {
        ctx->ls.collide_blocks = ctx->opt.shape[3];
        follow_collide_blocks(ctx->prec, ctx->sms, &ctx->ls);
    }
    *out = ctx;
    return DSMC_OK;
}

void dsmc_destroy(dsmc_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    free_all(ctx);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* dsmc_last_error(const dsmc_ctx* ctx)
{
    if (!ctx) return g_static_err;
    return ctx->err.c_str();
}

// ---------------------------------------------------------------------------
// Launch-shape search (options.autotune).  A trial ensemble of the same size
// is advanced with the current shapes to mid-run (the pool near its typical
// size), then each tunable is set to each candidate in turn for a window of
// kTuneWindow steps timed with events around every kernel group; the cost
// of a candidate is its kernel group's time per particle-step of the window
// (the pool still grows slowly between windows).  Tunables are searched
// one after another, each keeping its best value.  The caller re-prepares
// the buffers afterwards: the trial leaves the pool, counters and sample
// sums dirty.
static const int kTuneWindow = 6;

static dsmc_status autotune(dsmc_ctx* ctx, int n_runs, int steps)
{
    NvtxRange range("dsmc autotune");
    const int r0 = (int)ctx->opt.run_offset;
    AnyArgs u;
    enqueue_init(ctx, build_args(ctx, u, 0, r0, n_runs));
    ctx->cur = 0;
    // 10 windows follow the warm-up; the whole trial stays within `steps`
    const int warm = std::max(1, std::min(std::min(steps / 2, 200), steps - 10 * kTuneWindow));
    for (int s = 0; s < warm; ++s) {
        AnyArgs v;
        enqueue_step(ctx, build_args(ctx, v, ctx->cur, r0, n_runs), nullptr);
        ctx->cur ^= 1;
    }
    // kernel-group cost of the current shapes over one window
    auto window = [&](int group, double* cost) -> dsmc_status {
        Counters h0, h1;
        dsmc_status st = read_counters(ctx, &h0);
        if (st) return st;
        cudaEvent_t e0 = event_at(ctx, 0);
        if (!e0) return fail(ctx, DSMC_E_CUDA, "cudaEventCreate failed");
        CK(cudaEventRecord(e0, ctx->stream));
        size_t evn = 1;
        for (int s = 0; s < kTuneWindow; ++s) {
            AnyArgs v;
            enqueue_step(ctx, build_args(ctx, v, ctx->cur, r0, n_runs), &evn);
            ctx->cur ^= 1;
        }
        st = read_counters(ctx, &h1);
        if (st) return st;
        double ms = 0.0;
        for (int s = 0; s < kTuneWindow; ++s) {
            float m = 0.f;
            const size_t i = 1 + (size_t)s * kStepKernels + (size_t)group;
            CK(cudaEventElapsedTime(&m, ctx->events[i - 1], ctx->events[i]));
            ms += m;
        }
        const double units = (double)(h1.pool_steps - h0.pool_steps);
        *cost = ms / (units > 0.0 ? units : 1.0);
        return DSMC_OK;
    };
    LaunchShape& ls = ctx->ls;
    const int sms = ctx->sms;
    dsmc_status st = DSMC_OK;
    // sort/gather tile budget (sets the tile kernel's grid from occupancy;
    // the other grids go back to their defaults and are searched next)
    {
        const int cand[3] = {2048, 3072, 4608};
        int best = ls.tile_budget;
        double best_cost = 1e300;
        for (int k = 0; k < 3; ++k) {
            ls.tile_budget = cand[k];
            compute_launch_shape(ctx->prec, ctx->dim, sms, &ls);
            CK(prepare_kernels(ctx->prec, ctx->dim, ls.tile_budget, ls.collide_stage));
            double cst = 0.0;
            if ((st = window(kGroupCell, &cst))) return st;
            if (cst < best_cost) { best_cost = cst; best = cand[k]; }
        }
        ls.tile_budget = best;
        compute_launch_shape(ctx->prec, ctx->dim, sms, &ls);
        CK(prepare_kernels(ctx->prec, ctx->dim, ls.tile_budget, ls.collide_stage));
    }
    // collision CTAs: the default count per SM and one or two more (each
    // with the largest stage that lets them share an SM)
    struct Knob { int* v; int group; int cand[3]; };
    const int mb = ls.move_blocks, cpm = std::max(1, ls.collide_blocks / sms);
    Knob knobs[3] = {{&ls.move_blocks, kGroupMove, {mb, 2 * mb, 0}},
                     {&ls.scatter_blocks, kGroupScatter, {4 * sms, 8 * sms, 16 * sms}},
                     {&ls.collide_blocks, kGroupCollide,
                      {cpm * sms, cpm < 8 ? (cpm + 1) * sms : 0, cpm < 7 ? (cpm + 2) * sms : 0}}};
    for (Knob& kn : knobs) {
        int best = *kn.v;
        double best_cost = 1e300;
        for (int k = 0; k < 3 && kn.cand[k] > 0; ++k) {
            *kn.v = kn.cand[k];
            if (kn.v == &ls.collide_blocks) {
                follow_collide_blocks(ctx->prec, sms, &ls);
                CK(prepare_kernels(ctx->prec, ctx->dim, ls.tile_budget, ls.collide_stage));
            }
            double cst = 0.0;
            if ((st = window(kn.group, &cst))) return st;
            if (cst < best_cost) { best_cost = cst; best = kn.cand[k]; }
        }
        *kn.v = best;
        if (kn.v == &ls.collide_blocks) {
            follow_collide_blocks(ctx->prec, sms, &ls);
            CK(prepare_kernels(ctx->prec, ctx->dim, ls.tile_budget, ls.collide_stage));
        }
    }
    ctx->tuned_key = ((uint64_t)n_runs << 1) | 1u;
    return DSMC_OK;
}

// ---- launch-shape cache (options.autotune = DSMC_TUNE_LOAD) ------------
// One line per entry: "<key> <move CTAs> <scatter CTAs> <tile budget>
// <collision CTAs>"; the last line with a key wins.  The key names the GPU
// (name, SM count), the precision, the run count and steps, and hashes the
// problem description (FNV-1a over domain, grid, gas and boundaries).
static uint64_t fnv1a(uint64_t h, const void* p, size_t n)
{
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

static std::string tune_key(const dsmc_ctx* ctx, int n_runs, int steps)
{
    uint64_t h = 14695981039346656037ull;
    const dsmc_domain& d = ctx->dom;
    h = fnv1a(h, &d.dim, sizeof d.dim);
    h = fnv1a(h, d.extent, sizeof d.extent);
    h = fnv1a(h, &d.fill, sizeof d.fill);
    h = fnv1a(h, &d.fill_n, sizeof d.fill_n);
    h = fnv1a(h, &d.fill_T, sizeof d.fill_T);
    h = fnv1a(h, d.fill_U, sizeof d.fill_U);
    h = fnv1a(h, ctx->cells.n, sizeof ctx->cells.n);
    const double g[5] = {ctx->gas.mass, ctx->gas.d_ref, ctx->gas.T_ref, ctx->gas.omega, ctx->gas.F_N};
    h = fnv1a(h, g, sizeof g);
    if (ctx->gas.partner != DSMC_PARTNER_UNIFORM) {
        const int32_t pv[2] = {ctx->gas.partner,
                               ctx->gas.partner == DSMC_PARTNER_SUBCELL ? ctx->gas.n_sub : 1};
        h = fnv1a(h, pv, sizeof pv);
    }
    for (const dsmc_boundary& b : ctx->bcs) {
        const int32_t iv[8] = {b.kind, b.face, b.lo[0], b.lo[1], b.hi[0], b.hi[1], b.step_from, b.step_to};
        const double dv[5] = {b.n, b.T, b.U[0], b.U[1], b.U[2]};
        h = fnv1a(h, iv, sizeof iv);
        h = fnv1a(h, dv, sizeof dv);
        h = fnv1a(h, &b.plate_axis, sizeof b.plate_axis);
        h = fnv1a(h, &b.plate_index, sizeof b.plate_index);
    }
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess) name = prop.name;
    else cudaGetLastError();
    for (char& c : name)
        if (c == ' ' || c == '\t') c = '_';
    char buf[160];
    std::snprintf(buf, sizeof buf, "%s/sm%d/%s/runs%d/steps%d/%016llx", name.c_str(), ctx->sms,
                  ctx->prec == DSMC_FP64 ? "fp64" : "fp32", n_runs, steps, (unsigned long long)h);
    return buf;
}

static bool tune_load(const std::string& path, const std::string& key, int shape[4])
{
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    char k[256];
    int v[4];
    bool found = false;
    while (std::fscanf(f, "%255s %d %d %d %d", k, &v[0], &v[1], &v[2], &v[3]) == 5) {
        if (key == k && v[0] >= 1 && v[1] >= 1 && v[2] >= 256 && v[2] <= kMaxTileBudget && v[3] >= 1) {
            for (int i = 0; i < 4; ++i) shape[i] = v[i];
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

static void tune_store(const std::string& path, const std::string& key, const LaunchShape& ls)
{
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d\n", key.c_str(), ls.move_blocks, ls.scatter_blocks,
                 ls.tile_budget, ls.collide_blocks);
    std::fclose(f);
}

// options.checks: the consistency pass over the pool the last step wrote
// (buffer `cur`), read back; a failure is DSMC_E_STATE.
static dsmc_status run_checks(dsmc_ctx* ctx, int cur, int run0, int n_launch)
{
    CK(cudaMemsetAsync(&ctx->d_ctr->check_fail, 0, sizeof(uint32_t), ctx->stream));
    CK(cudaMemsetAsync(&ctx->d_ctr->check_first, 0xFF, sizeof(uint32_t), ctx->stream));
    AnyArgs u;
    launch_check(ctx->prec, build_args(ctx, u, cur, run0, n_launch), ctx->ls, ctx->stream);
    CK(cudaGetLastError());
    Counters h;
    dsmc_status st = read_counters(ctx, &h);
    if (st) return st;
    if (h.check_fail) {
        char buf[160];
        std::snprintf(buf, sizeof buf,
                      "consistency check failed at %u pool positions (first: %u)", h.check_fail,
                      h.check_first);
        return fail(ctx, DSMC_E_STATE, buf);
    }
    return DSMC_OK;
}

static dsmc_status run_windows(dsmc_ctx* ctx, int n_runs, double dt, int steps,
                               const int32_t* first, const int32_t* last, int n_samples,
                               uint64_t seed)
{
    NvtxRange range("dsmc_run_ensemble");
    if (!ctx) return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    dsmc_status st = validate_run(ctx, n_runs, dt, steps, first, last, n_samples);
    if (st) return st;
    ctx->have_run = false;
    ctx->dbg = false;
    ctx->stats.h2d_bytes = 0;
    ctx->stats.d2h_bytes = 0;
    const bool plain = ctx->opt.mode == DSMC_MODE_PLAIN;
    const int n_launch = plain ? 1 : n_runs;
    st = prepare(ctx, n_runs, dt, steps, first, last, n_samples, seed, n_launch);
    if (st) return st;
    // (runs shorter than 100 steps keep the default shapes: the trial needs
    // room to reach mid-run)
    if (ctx->opt.autotune && !plain && steps >= 100 &&
        ctx->tuned_key != (((uint64_t)n_runs << 1) | 1u)) {
        const bool use_cache = ctx->opt.autotune == DSMC_TUNE_LOAD && !ctx->tune_cache.empty();
        const std::string key = use_cache ? tune_key(ctx, n_runs, steps) : std::string();
        int shape[4];
        if (use_cache && tune_load(ctx->tune_cache, key, shape)) {
            ctx->ls.tile_budget = shape[2];
            compute_launch_shape(ctx->prec, ctx->dim, ctx->sms, &ctx->ls);
            ctx->ls.move_blocks = shape[0];
            ctx->ls.scatter_blocks = shape[1];
            ctx->ls.collide_blocks = shape[3];
            follow_collide_blocks(ctx->prec, ctx->sms, &ctx->ls);
            CK(prepare_kernels(ctx->prec, ctx->dim, ctx->ls.tile_budget, ctx->ls.collide_stage));
            ctx->tuned_key = ((uint64_t)n_runs << 1) | 1u;
            ctx->tuned_how = 2;
        } else {
            st = autotune(ctx, n_runs, steps);
            if (st) return st;
            ctx->tuned_how = 1;
            if (use_cache) tune_store(ctx->tune_cache, key, ctx->ls);
            destroy_graphs(ctx);
            st = prepare(ctx, n_runs, dt, steps, first, last, n_samples, seed, n_launch);
            if (st) return st;
        }
    }
    const bool profile = ctx->opt.profile != 0;
    const bool graph = !plain && !profile && ctx->opt.use_graph;
    if (graph) {
        st = build_graphs(ctx, n_runs);
        if (st) return st;
    }
    for (int k = 0; k < 12; ++k) {
        ctx->stats.ms_kernel[k] = 0.0;
        ctx->stats.launches_kernel[k] = 0;
    }
    // graphs with the reduction over runs at the windows' last steps
    std::vector<char> is_sample(steps + 1, 0);
    for (int k = 0; k < n_samples; ++k) is_sample[last[k]] = 1;
    cudaEvent_t e0 = event_at(ctx, 0), e1 = event_at(ctx, 1);
    if (!e0 || !e1) return fail(ctx, DSMC_E_CUDA, "cudaEventCreate failed");
    size_t evn = 2;
    float ms_init = 0.f;
    CK(cudaEventRecord(e0, ctx->stream));
    for (int r = 0; r < (plain ? n_runs : 1); ++r) {
        AnyArgs u;
        const int r0 = (int)ctx->opt.run_offset + (plain ? r : 0);
        const void* a0 = build_args(ctx, u, 0, r0, n_launch);
        enqueue_init(ctx, a0);
        ctx->cur = 0;
        if (r == 0) {
            // the timed step loop starts after the step-0 state of run 0
            CK(cudaEventRecord(e1, ctx->stream));
        }
        for (int s = 1; s <= steps; ++s) {
            if (graph) {
                CK(cudaGraphLaunch(ctx->gexec[ctx->cur][is_sample[s]], ctx->stream));
            } else {
                AnyArgs v;
                const void* a = build_args(ctx, v, ctx->cur, r0, n_launch);
                enqueue_step(ctx, a, profile ? &evn : nullptr);
            }
            ctx->cur ^= 1;
        }
        if (ctx->opt.checks && plain && r + 1 < n_runs) {
            // each run of the plain loop is checked before the next one
            // reuses the buffers (the last one after the timed loop)
            st = run_checks(ctx, ctx->cur, r0, n_launch);
            if (st) return st;
        }
    }
    cudaEvent_t e2 = event_at(ctx, evn);
    if (!e2) return fail(ctx, DSMC_E_CUDA, "cudaEventCreate failed");
    CK(cudaEventRecord(e2, ctx->stream));
    CK(cudaGetLastError());
    Counters h;
    st = read_counters(ctx, &h);
    if (st) return st;
    CK(cudaEventElapsedTime(&ms_init, e0, e1));
    float ms_all = 0.f;
    CK(cudaEventElapsedTime(&ms_all, e1, e2));
    ctx->stats.ms_steps = ms_all;
    if (profile) {
        // events 2.. are recorded after each kernel, in enqueue order
        size_t i = 2;
        cudaEvent_t prev = e1;
        for (int r = 0; r < (plain ? n_runs : 1); ++r) {
            for (int s = 1; s <= steps; ++s)
                for (int k = 0; k < kStepKernels; ++k, ++i) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, prev, ctx->events[i]);
                    ctx->stats.ms_kernel[kKindOf[k]] += ms;
                    ctx->stats.launches_kernel[kKindOf[k]] += 1;
                    prev = ctx->events[i];
                }
        }
    }
    fill_stats(ctx, h);
    ctx->stats.steps_done = steps;
    uint32_t total = 0;
    CK(cudaMemcpy(&total, ctx->run_base + n_launch, 4, cudaMemcpyDeviceToHost));
    ctx->stats.d2h_bytes += 4;
    ctx->stats.particles_now = total;
    st = check_error_word(ctx, h.error);
    if (st) return st;
    if (ctx->opt.checks) {
        st = run_checks(ctx, ctx->cur, (int)ctx->opt.run_offset + (plain ? n_runs - 1 : 0), n_launch);
        if (st) return st;
    }
    ctx->have_run = true;
    ctx->last_runs = n_runs;
    ctx->last_steps = steps;
    ctx->last_samples = n_samples;
    ctx->win_len.assign(n_samples, 1);
    for (int k = 0; k < n_samples; ++k) ctx->win_len[k] = last[k] - first[k] + 1;
    return DSMC_OK;
}

dsmc_status dsmc_run_ensemble(dsmc_ctx* ctx, int n_runs, double dt, int steps,
                              const int32_t* sample_steps, int n_samples, uint64_t seed)
{
    return run_windows(ctx, n_runs, dt, steps, sample_steps, sample_steps, n_samples, seed);
}

dsmc_status dsmc_run_ensemble_windows(dsmc_ctx* ctx, int n_runs, double dt, int steps,
                                      const int32_t* first, const int32_t* last, int n_windows,
                                      uint64_t seed)
{
    return run_windows(ctx, n_runs, dt, steps, first, last, n_windows, seed);
}

dsmc_status dsmc_get_samples(dsmc_ctx* ctx, int sample_idx, dsmc_quantity q, double* out,
                             size_t out_len)
{
    if (!ctx) return DSMC_E_INVALID;
    if (!ctx->have_run) return fail(ctx, DSMC_E_STATE, "no completed run");
    if (sample_idx < 0 || sample_idx >= ctx->last_samples || !out)
        return fail(ctx, DSMC_E_INVALID, "bad sample index or output");
    CK(cudaSetDevice(ctx->device));
    const size_t nc = (size_t)ctx->ncells;
    if (q == DSMC_Q_RAW_MOMENTS) {
        const size_t n = (size_t)ctx->G * nc * DSMC_NMOM;
        if (out_len < n) return fail(ctx, DSMC_E_INVALID, "out_len too small");
        ctx->stats.d2h_bytes += 8 * n;
        CK(cudaMemcpyAsync(out, ctx->acc + (size_t)sample_idx * n, 8 * n, cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return DSMC_OK;
    }
    int off, width;
    switch (q) {
    case DSMC_Q_DENSITY: off = 0; width = 1; break;
    case DSMC_Q_VELOCITY: off = 1; width = 3; break;
    case DSMC_Q_TEMPERATURE: off = 4; width = 1; break;
    case DSMC_Q_STDERR_DENSITY: off = 5; width = 1; break;
    case DSMC_Q_STDERR_VELOCITY: off = 6; width = 3; break;
    case DSMC_Q_STDERR_TEMPERATURE: off = 9; width = 1; break;
    default: return fail(ctx, DSMC_E_INVALID, "unknown quantity");
    }
    if (out_len < nc * width) return fail(ctx, DSMC_E_INVALID, "out_len too small");
    AnyArgs u;
    const void* a = build_args(ctx, u, ctx->cur, 0, ctx->n_launch);
    launch_macro(ctx->prec, a, sample_idx, ctx->last_runs,
                 sample_idx < (int)ctx->win_len.size() ? ctx->win_len[sample_idx] : 1, ctx->macro,
                 ctx->stream);
    CK(cudaGetLastError());
    ctx->stats.d2h_bytes += 8 * width * nc;
    CK(cudaMemcpy2DAsync(out, 8 * width, ctx->macro + off, 8 * 10, 8 * width, nc,
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DSMC_OK;
}

dsmc_status dsmc_get_stats(dsmc_ctx* ctx, dsmc_stats* out)
{
    if (!ctx || !out || out->struct_size < sizeof(dsmc_stats)) return DSMC_E_INVALID;
    *out = ctx->stats;
    out->struct_size = sizeof(dsmc_stats);
    return DSMC_OK;
}

// ---- test hooks -------------------------------------------------------------

dsmc_status dsmc_debug_begin(dsmc_ctx* ctx, int n_runs, double dt, uint64_t seed)
{
    if (!ctx) return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    dsmc_status st = validate_run(ctx, n_runs, dt, 0, nullptr, nullptr, 0);
    if (st) return st;
    const int steps = 4096;
    st = prepare(ctx, n_runs, dt, steps, nullptr, nullptr, 0, seed, n_runs);
    if (st) return st;
    AnyArgs u;
    enqueue_init(ctx, build_args(ctx, u, 0, 0, n_runs));
    ctx->cur = 0;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->dbg = true;
    ctx->have_run = false;
    ctx->last_runs = n_runs;
    ctx->prev_run_base.assign(n_runs + 1, 0);
    return DSMC_OK;
}

dsmc_status dsmc_debug_step(dsmc_ctx* ctx, int n_steps)
{
    if (!ctx || n_steps < 0) return DSMC_E_INVALID;
    if (!ctx->dbg) return fail(ctx, DSMC_E_STATE, "dsmc_debug_begin first");
    CK(cudaSetDevice(ctx->device));
    const int n = ctx->n_launch;
    for (int s = 0; s < n_steps; ++s) {
        // ordered after the previous step's kernels on the context's stream
        CK(cudaMemcpyAsync(ctx->prev_run_base.data(), ctx->run_base, 4 * (n + 1),
                           cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        AnyArgs u;
        enqueue_step(ctx, build_args(ctx, u, ctx->cur, 0, n), nullptr);
        ctx->cur ^= 1;
    }
    CK(cudaGetLastError());
    Counters h;
    dsmc_status st = read_counters(ctx, &h);
    if (st) return st;
    fill_stats(ctx, h);
    st = check_error_word(ctx, h.error);
    if (!st && ctx->opt.checks) st = run_checks(ctx, ctx->cur, 0, n);
    return st;
}

// run-local cell index <-> per-axis indices
static void decode_host(const dsmc_ctx* ctx, uint32_t lin, int* ci)
{
    const int n0 = ctx->hcfg.n[0], n1 = ctx->hcfg.n[1];
    ci[0] = (int)(lin % n0);
    ci[1] = (int)((lin / n0) % n1);
    ci[2] = (int)(lin / ((uint32_t)n0 * n1));
}

// the pool holds offsets inside each particle's cell; the test hooks speak
// absolute positions: x = i * d + f
template <typename T>
static dsmc_status get_run_state(dsmc_ctx* ctx, int run, std::vector<double>& x,
                                 std::vector<double>& v, std::vector<uint32_t>& id)
{
    uint32_t rb[2];
    CK(cudaMemcpy(rb, ctx->run_base + run, 8, cudaMemcpyDeviceToHost));
    if (rb[1] < rb[0] || (int64_t)rb[1] > ctx->cap_old)
        return fail(ctx, DSMC_E_CAPACITY, "pool overflowed: state not available");
    const size_t n = rb[1] - rb[0];
    x.assign(3 * n, 0.0);
    v.assign(3 * n, 0.0);
    id.assign(n, 0);
    std::vector<T> tmp(n);
    std::vector<uint32_t> cells(n);
    if (n) CK(cudaMemcpy(cells.data(), ctx->CI[ctx->cur] + rb[0], 4 * n, cudaMemcpyDeviceToHost));
    for (int a = 0; a < 3; ++a) {
        if (ctx->X[ctx->cur][a] && n) {
            CK(cudaMemcpy(tmp.data(), (T*)ctx->X[ctx->cur][a] + rb[0], sizeof(T) * n,
                          cudaMemcpyDeviceToHost));
            for (size_t k = 0; k < n; ++k) {
                int ci[3];
                decode_host(ctx, cells[k] - (uint32_t)run * (uint32_t)ctx->ncells, ci);
                x[3 * k + a] = (double)ci[a] * ctx->hcfg.d[a] + (double)tmp[k];
            }
        }
        if (n) CK(cudaMemcpy(tmp.data(), (T*)ctx->V[ctx->cur][a] + rb[0], sizeof(T) * n,
                             cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < n; ++k) v[3 * k + a] = (double)tmp[k];
    }
    if (n) CK(cudaMemcpy(id.data(), ctx->ID[ctx->cur] + rb[0], 4 * n, cudaMemcpyDeviceToHost));
    return DSMC_OK;
}

dsmc_status dsmc_debug_get_state(dsmc_ctx* ctx, int run, double* x, double* v, uint32_t* id,
                                 int64_t cap, int64_t* n_out)
{
    if (!ctx || !ctx->n_launch || run < 0 || run >= ctx->n_launch || !n_out) return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<double> hx, hv;
    std::vector<uint32_t> hid;
    dsmc_status st = ctx->prec == DSMC_FP64 ? get_run_state<double>(ctx, run, hx, hv, hid)
                                            : get_run_state<float>(ctx, run, hx, hv, hid);
    if (st) return st;
    const int64_t n = (int64_t)hid.size();
    *n_out = n;
    const int64_t m = std::min(n, cap);
    if (x) std::memcpy(x, hx.data(), 8 * 3 * m);
    if (v) std::memcpy(v, hv.data(), 8 * 3 * m);
    if (id) std::memcpy(id, hid.data(), 4 * m);
    return DSMC_OK;
}

template <typename T>
static dsmc_status set_run_state(dsmc_ctx* ctx, int run, int64_t n, const double* x, const double* v,
                                 const uint32_t* id, uint32_t next_id)
{
    const int nl = ctx->n_launch;
    std::vector<uint32_t> rb(nl + 1), nid(nl);
    CK(cudaMemcpy(rb.data(), ctx->run_base, 4 * (nl + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(nid.data(), ctx->next_id, 4 * nl, cudaMemcpyDeviceToHost));
    if ((int64_t)rb[nl] > ctx->cap_old) return fail(ctx, DSMC_E_CAPACITY, "pool overflowed");
    const size_t old_total = rb[nl];
    std::vector<std::vector<T>> X(3), V(3);
    std::vector<uint32_t> I(old_total), CIh(old_total);
    if (old_total)
        CK(cudaMemcpy(CIh.data(), ctx->CI[ctx->cur], 4 * old_total, cudaMemcpyDeviceToHost));
    for (int a = 0; a < 3; ++a) {
        X[a].resize(old_total);
        V[a].resize(old_total);
        if (ctx->X[ctx->cur][a])
            CK(cudaMemcpy(X[a].data(), ctx->X[ctx->cur][a], sizeof(T) * old_total, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(V[a].data(), ctx->V[ctx->cur][a], sizeof(T) * old_total, cudaMemcpyDeviceToHost));
    }
    CK(cudaMemcpy(I.data(), ctx->ID[ctx->cur], 4 * old_total, cudaMemcpyDeviceToHost));
    std::vector<std::vector<T>> NX(3), NV(3);
    std::vector<uint32_t> NI, NC;
    std::vector<uint32_t> nrb(nl + 1, 0);
    for (int r = 0; r < nl; ++r) {
        nrb[r] = (uint32_t)NI.size();
        if (r == run) {
            for (int64_t k = 0; k < n; ++k) {
                int ci[3] = {0, 0, 0};
                for (int a = 0; a < 3; ++a) {
                    double f = 0.0;
                    if (a < ctx->dim) {
                        const double xa = x[3 * k + a], d = ctx->hcfg.d[a];
                        int i = (int)std::floor(xa / d);
                        i = std::max(0, std::min(ctx->hcfg.n[a] - 1, i));
                        ci[a] = i;
                        f = xa - (double)i * d;
                    }
                    NX[a].push_back((T)f);
                    NV[a].push_back((T)v[3 * k + a]);
                }
                NI.push_back(id[k]);
                NC.push_back((uint32_t)r * (uint32_t)ctx->ncells +
                             (uint32_t)(ci[0] + ctx->hcfg.n[0] * (ci[1] + ctx->hcfg.n[1] * ci[2])));
            }
        } else {
            for (size_t k = rb[r]; k < rb[r + 1]; ++k) {
                for (int a = 0; a < 3; ++a) {
                    NX[a].push_back(X[a][k]);
                    NV[a].push_back(V[a][k]);
                }
                NI.push_back(I[k]);
                NC.push_back(CIh[k]);
            }
        }
    }
    nrb[nl] = (uint32_t)NI.size();
    if ((int64_t)NI.size() > ctx->cap_old) return fail(ctx, DSMC_E_CAPACITY, "state exceeds pool capacity");
    const size_t tot = NI.size();
    for (int a = 0; a < 3; ++a) {
        if (ctx->X[ctx->cur][a] && tot)
            CK(cudaMemcpy(ctx->X[ctx->cur][a], NX[a].data(), sizeof(T) * tot, cudaMemcpyHostToDevice));
        if (tot) CK(cudaMemcpy(ctx->V[ctx->cur][a], NV[a].data(), sizeof(T) * tot, cudaMemcpyHostToDevice));
    }
    if (tot) CK(cudaMemcpy(ctx->ID[ctx->cur], NI.data(), 4 * tot, cudaMemcpyHostToDevice));
    if (tot) CK(cudaMemcpy(ctx->CI[ctx->cur], NC.data(), 4 * tot, cudaMemcpyHostToDevice));
    nid[run] = next_id;
    CK(cudaMemcpy(ctx->run_base, nrb.data(), 4 * (nl + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->next_id, nid.data(), 4 * nl, cudaMemcpyHostToDevice));
    // the next scatter walks the pre-step pool: its size lives at start[total + 1]
    CK(cudaMemcpy(ctx->start + ctx->total_cells + 1, &nrb[nl], 4, cudaMemcpyHostToDevice));
    return DSMC_OK;
}

dsmc_status dsmc_debug_set_state(dsmc_ctx* ctx, int run, int64_t n, const double* x, const double* v,
                                 const uint32_t* id, uint32_t next_id)
{
    if (!ctx || !ctx->dbg || run < 0 || run >= ctx->n_launch || n < 0 || (n > 0 && (!x || !v || !id)))
        return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    return ctx->prec == DSMC_FP64 ? set_run_state<double>(ctx, run, n, x, v, id, next_id)
                                  : set_run_state<float>(ctx, run, n, x, v, id, next_id);
}

dsmc_status dsmc_debug_timeout_probe(dsmc_ctx* ctx, uint32_t polls)
{
    if (!ctx || polls < 1 || polls > (1u << 20)) return DSMC_E_INVALID;
    if (!ctx->dbg) return fail(ctx, DSMC_E_STATE, "dsmc_debug_begin first");
    CK(cudaSetDevice(ctx->device));
    CK(timeout_probe(ctx->d_ctr, polls, ctx->stream));
    Counters h;
    dsmc_status st = read_counters(ctx, &h);
    if (st) return st;
    CK(cudaMemsetAsync(&ctx->d_ctr->probe, 0, sizeof(uint32_t), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h.probe & DSMC_ERR_TIMEOUT)
        return fail(ctx, DSMC_E_TIMEOUT, "probe: a bounded wait for a bulk copy expired");
    return DSMC_OK;
}

dsmc_status dsmc_debug_get_cells(dsmc_ctx* ctx, int run, int32_t* count, int32_t* cand,
                                 int32_t* accepted, int64_t* lcr, int64_t cap)
{
    if (!ctx || !ctx->dbg || run < 0 || run >= ctx->n_launch) return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    const int nc = ctx->ncells;
    std::vector<uint32_t> st(nc + 1);
    CK(cudaMemcpy(st.data(), ctx->start + (size_t)run * nc, 4 * (nc + 1), cudaMemcpyDeviceToHost));
    if ((int64_t)st[nc] > ctx->cap_old) return fail(ctx, DSMC_E_CAPACITY, "pool overflowed");
    if (count)
        for (int c = 0; c < nc; ++c) count[c] = (int32_t)(st[c + 1] - st[c]);
    if (cand || accepted || lcr) {
        if (!ctx->cand) return fail(ctx, DSMC_E_STATE, "options.debug was not set");
        std::vector<uint32_t> tmp(nc);
        if (cand) {
            CK(cudaMemcpy(tmp.data(), ctx->cand + (size_t)run * nc, 4 * nc, cudaMemcpyDeviceToHost));
            for (int c = 0; c < nc; ++c) cand[c] = (int32_t)tmp[c];
        }
        if (accepted) {
            CK(cudaMemcpy(tmp.data(), ctx->accd + (size_t)run * nc, 4 * nc, cudaMemcpyDeviceToHost));
            for (int c = 0; c < nc; ++c) accepted[c] = (int32_t)tmp[c];
        }
        if (lcr) {
            const size_t n = st[nc] - st[0];
            std::vector<uint32_t> sl(n);
            if (n)
                CK(cudaMemcpy(sl.data(), ctx->lcr_dbg + st[0], 4 * n, cudaMemcpyDeviceToHost));
            const uint32_t b0 = ctx->prev_run_base[run];
            const uint32_t n_old = ctx->prev_run_base[run + 1] - b0;
            const uint64_t gen0 = (uint64_t)ctx->cap_old + (uint64_t)run * ctx->gcap;
            for (size_t k = 0; k < n && (int64_t)k < cap; ++k) {
                const uint64_t s = sl[k];
                lcr[k] = s < (uint64_t)ctx->cap_old ? (int64_t)(s - b0) : (int64_t)(n_old + (s - gen0));
            }
        }
    }
    return DSMC_OK;
}

template <typename T>
static dsmc_status cell_state_io(dsmc_ctx* ctx, int run, double* rem, double* smax, bool get)
{
    const size_t nc = ctx->ncells, off = (size_t)run * nc;
    std::vector<T> tmp(nc);
    if (get) {
        if (rem) CK(cudaMemcpy(rem, ctx->rem + off, 8 * nc, cudaMemcpyDeviceToHost));
        if (smax) {
            CK(cudaMemcpy(tmp.data(), (T*)ctx->smax + off, sizeof(T) * nc, cudaMemcpyDeviceToHost));
            for (size_t c = 0; c < nc; ++c) smax[c] = (double)tmp[c];
        }
    } else {
        if (rem) CK(cudaMemcpy(ctx->rem + off, rem, 8 * nc, cudaMemcpyHostToDevice));
        if (smax) {
            for (size_t c = 0; c < nc; ++c) tmp[c] = (T)smax[c];
            CK(cudaMemcpy((T*)ctx->smax + off, tmp.data(), sizeof(T) * nc, cudaMemcpyHostToDevice));
        }
    }
    return DSMC_OK;
}

dsmc_status dsmc_debug_get_cell_state(dsmc_ctx* ctx, int run, double* rem, double* smax)
{
    if (!ctx || !ctx->n_launch || run < 0 || run >= ctx->n_launch) return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    return ctx->prec == DSMC_FP64 ? cell_state_io<double>(ctx, run, rem, smax, true)
                                  : cell_state_io<float>(ctx, run, rem, smax, true);
}

dsmc_status dsmc_debug_set_cell_state(dsmc_ctx* ctx, int run, const double* rem, const double* smax)
{
    if (!ctx || !ctx->dbg || run < 0 || run >= ctx->n_launch) return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    return ctx->prec == DSMC_FP64
               ? cell_state_io<double>(ctx, run, const_cast<double*>(rem), const_cast<double*>(smax), false)
               : cell_state_io<float>(ctx, run, const_cast<double*>(rem), const_cast<double*>(smax), false);
}

dsmc_status dsmc_debug_sample(dsmc_ctx* ctx, int run, double* mom)
{
    if (!ctx || !ctx->dbg || run < 0 || run >= ctx->n_launch || !mom) return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    AnyArgs u;
    launch_sample_now(ctx->prec, build_args(ctx, u, ctx->cur, 0, ctx->n_launch), ctx->stream);
    CK(cudaGetLastError());
    const size_t per = (size_t)ctx->ncells * DSMC_NMOM;
    CK(cudaMemcpyAsync(mom, ctx->mom + (size_t)run * per, 8 * per, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DSMC_OK;
}

dsmc_status dsmc_debug_philox(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return DSMC_E_INVALID;
    if (n == 0) return DSMC_OK;
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    if (cudaMalloc(&dc, 16 * n) != cudaSuccess || cudaMalloc(&dk, 8 * n) != cudaSuccess ||
        cudaMalloc(&dout, 16 * n) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dc); cudaFree(dk); cudaFree(dout);
        return DSMC_E_OOM;
    }
    dsmc_status st = DSMC_OK;
    if (cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dk, key, 8 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        philox_device(n, dc, dk, dout, 0) != cudaSuccess ||
        cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        st = DSMC_E_CUDA;
    }
    cudaFree(dc); cudaFree(dk); cudaFree(dout);
    return st;
}


// ---------------------------------------------------------------------------
// Mixed-size ensembles: several contexts ("parts", one grid each) advanced
// by one launch per kernel kind per step.  Each part keeps its own buffers,
// counters and samples; the launches see the parts as an array of StepArgs
// in device memory (one array per buffer parity) and the queue-driven
// kernels claim (part, tile) items from shared counters.

struct dsmc_mixed {
    std::vector<dsmc_ctx*> parts;    // caller's order
    std::vector<int> order;          // launch order: parts by decreasing cells per run
    int device = 0, prec = DSMC_FP32, dim = 2, sms = 0, flags = 0;
    cudaStream_t stream = nullptr;   // parts[0]'s stream
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
    LaunchShape ls;
    void* d_args[2] = {nullptr, nullptr};   // StepArgs<T>[n_parts] per buffer parity
    size_t args_cap = 0;
    uint32_t* d_queue = nullptr;
    std::vector<unsigned char> margs[2];    // MultiArgs<T> per buffer parity
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    std::vector<uint64_t> graph_gen;        // parts' allocation generations of the graphs
    std::vector<int> graph_runs;
    int cur = 0;
    std::vector<cudaEvent_t> events;
    dsmc_stats stats;
};

static dsmc_status mfail(dsmc_mixed* m, dsmc_status s, const std::string& msg)
{
    m->err = msg;
    return s;
}

#define CKM(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            m->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return DSMC_E_CUDA;                                                           \
        }                                                                                 \
    } while (0)

static void mixed_destroy_graphs(dsmc_mixed* m)
{
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < 2; ++k)
            if (m->gexec[p][k]) {
                cudaGraphExecDestroy(m->gexec[p][k]);
                m->gexec[p][k] = nullptr;
            }
    m->graph_gen.clear();
    m->graph_runs.clear();
}

static cudaEvent_t mixed_event(dsmc_mixed* m, size_t i)
{
    while (m->events.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        m->events.push_back(e);
    }
    return m->events[i];
}

dsmc_status dsmc_mixed_create(dsmc_ctx* const* parts, int n_parts, int flags, dsmc_mixed** out)
{
    if (!out) return DSMC_E_INVALID;
    *out = nullptr;
    if (!parts || n_parts < 1 || n_parts > kMaxParts) return DSMC_E_INVALID;
    for (int i = 0; i < n_parts; ++i) {
        if (!parts[i]) return DSMC_E_INVALID;
        if (parts[i]->device != parts[0]->device || parts[i]->prec != parts[0]->prec ||
            parts[i]->dim != parts[0]->dim)
            return DSMC_E_INVALID;
        for (int j = 0; j < i; ++j)
            if (parts[j] == parts[i]) return DSMC_E_INVALID;
    }
    dsmc_mixed* m = new (std::nothrow) dsmc_mixed();
    if (!m) return DSMC_E_OOM;
    m->parts.assign(parts, parts + n_parts);
    m->device = parts[0]->device;
    m->prec = parts[0]->prec;
    m->dim = parts[0]->dim;
    m->sms = parts[0]->sms;
    m->flags = flags;
    m->stream = parts[0]->stream;
    std::memset(&m->stats, 0, sizeof(m->stats));
    m->stats.struct_size = sizeof(dsmc_stats);
    // heaviest parts first in the item order: their tiles are claimed
    // first, the small parts' tiles fill in at the end
    m->order.resize(n_parts);
    for (int i = 0; i < n_parts; ++i) m->order[i] = i;
    std::stable_sort(m->order.begin(), m->order.end(),
                     [&](int a, int b) { return parts[a]->ncells > parts[b]->ncells; });
    bool ok = cudaSetDevice(m->device) == cudaSuccess;
    ok = ok && cudaMalloc(&m->d_queue, 4 * kQueueKinds) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        dsmc_mixed_destroy(m);
        return DSMC_E_CUDA;
    }
    m->ls.tile_budget = 0;
    m->ls.collide_ppc = 0;
    for (dsmc_ctx* c : m->parts) m->ls.collide_ppc = std::max(m->ls.collide_ppc, collide_ppc_target(c));
    compute_multi_shape(m->prec, m->dim, m->sms, &m->ls);
    *out = m;
    return DSMC_OK;
}

void dsmc_mixed_destroy(dsmc_mixed* m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    mixed_destroy_graphs(m);
    for (int p = 0; p < 2; ++p)
        if (m->d_args[p]) cudaFree(m->d_args[p]);
    if (m->d_queue) cudaFree(m->d_queue);
    for (cudaEvent_t e : m->events) cudaEventDestroy(e);
    if (m->ev_fork) cudaEventDestroy(m->ev_fork);
    if (m->ev_join) cudaEventDestroy(m->ev_join);
    if (m->side) cudaStreamDestroy(m->side);
    delete m;
}

const char* dsmc_mixed_last_error(const dsmc_mixed* m)
{
    if (!m) return g_static_err;
    return m->err.c_str();
}

// the parts' StepArgs (both buffer parities) in device memory, and the
// MultiArgs of each parity with the item prefix tables in launch order
template <typename T>
static dsmc_status mixed_upload_args(dsmc_mixed* m, const int32_t* n_runs)
{
    const int n = (int)m->parts.size();
    const size_t bytes = sizeof(StepArgs<T>) * n;
    if (m->args_cap < bytes) {
        for (int p = 0; p < 2; ++p) {
            if (m->d_args[p]) cudaFree(m->d_args[p]);
            m->d_args[p] = nullptr;
        }
        m->args_cap = 0;
        for (int p = 0; p < 2; ++p)
            if (cudaMalloc(&m->d_args[p], bytes) != cudaSuccess) {
                cudaGetLastError();
                return mfail(m, DSMC_E_OOM, "device allocation of the parts' arguments failed");
            }
        m->args_cap = bytes;
    }
    for (int p = 0; p < 2; ++p) {
        std::vector<StepArgs<T>> h(n);
        MultiArgs<T> ma;
        std::memset(&ma, 0, sizeof(ma));
        ma.parts = static_cast<const StepArgs<T>*>(m->d_args[p]);
        ma.queue = m->d_queue;
        ma.n_parts = n;
        ma.collide_stage = m->ls.collide_stage;
        for (int k = 0; k < n; ++k) {
            const int i = m->order[k];
            dsmc_ctx* c = m->parts[i];
            h[k] = args_for<T>(c, p, (int)c->opt.run_offset, n_runs[i]);
            if (h[k].hot.partner != DSMC_PARTNER_UNIFORM) ma.positional = 1;
            const int64_t cells = (int64_t)c->ncells * n_runs[i];
            ma.tile_base[k + 1] = ma.tile_base[k] + (int32_t)((cells + kTileCells - 1) / kTileCells);
            ma.ctile_base[k + 1] = ma.ctile_base[k] + (int32_t)((cells + kCollideCells - 1) / kCollideCells);
            ma.scan_base[k + 1] = ma.scan_base[k] + h[k].scan_blocks;
            ma.gen_base[k + 1] = ma.gen_base[k] + n_runs[i] * h[k].gen_groups;
            ma.gcount_base[k + 1] = ma.gcount_base[k] + (h[k].gen_groups > 1 ? n_runs[i] * h[k].gen_groups : 0);
        }
        CKM(cudaMemcpy(m->d_args[p], h.data(), bytes, cudaMemcpyHostToDevice));
        m->margs[p].resize(sizeof(ma));
        std::memcpy(m->margs[p].data(), &ma, sizeof(ma));
    }
    return DSMC_OK;
}

// One time step of every part (as enqueue_step for one context).
static void enqueue_mixed_step(dsmc_mixed* m, int cur, size_t* ev, bool fork, bool reduce)
{
    const void* ma = m->margs[cur].data();
    const int p = m->prec;
    const LaunchShape& ls = m->ls;
    cudaStream_t s = m->stream;
    auto mark = [&]() {
        if (ev) cudaEventRecord(mixed_event(m, (*ev)++), s);
    };
    if (fork) {
        cudaEventRecord(m->ev_fork, s);
        cudaStreamWaitEvent(m->side, m->ev_fork, 0);
        launch_m_generate(p, ma, ls, m->side);
        cudaEventRecord(m->ev_join, m->side);
        launch_m_move(p, ma, ls, s);
        cudaStreamWaitEvent(s, m->ev_join, 0);
    } else {
        launch_m_generate(p, ma, ls, s); mark();
        launch_m_move(p, ma, ls, s); mark();
    }
    launch_m_scan(p, ma, ls, s); mark();
    launch_m_scatter(p, ma, ls, s); mark();
    launch_m_cell(p, ma, ls, s); mark();
    launch_m_cell_big(p, ma, ls, s); mark();
    launch_m_collide_big(p, ma, ls, s); mark();
    launch_m_collide(p, ma, ls, s); mark();
    if (reduce) launch_m_reduce(p, ma, ls, s);
    mark();
    launch_m_step_end(p, ma, ls, s); mark();
}

static dsmc_status mixed_build_graphs(dsmc_mixed* m, const int32_t* n_runs)
{
    const int n = (int)m->parts.size();
    bool same = m->gexec[0][0] && (int)m->graph_gen.size() == n;
    for (int i = 0; same && i < n; ++i)
        same = m->graph_gen[i] == m->parts[i]->generation && m->graph_runs[i] == n_runs[i];
    if (same) return DSMC_OK;
    mixed_destroy_graphs(m);
    for (int p = 0; p < 2; ++p)
        for (int smp = 0; smp < 2; ++smp) {
            cudaGraph_t g = nullptr;
            CKM(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
            enqueue_mixed_step(m, p, nullptr, true, smp != 0);
            CKM(cudaStreamEndCapture(m->stream, &g));
            cudaError_t e = cudaGraphInstantiate(&m->gexec[p][smp], g, 0);
            cudaGraphDestroy(g);
            CKM(e);
        }
    for (int i = 0; i < n; ++i) {
        m->graph_gen.push_back(m->parts[i]->generation);
        m->graph_runs.push_back(n_runs[i]);
    }
    return DSMC_OK;
}

dsmc_status dsmc_mixed_run(dsmc_mixed* m, const int32_t* n_runs, double dt, int steps,
                           const int32_t* sample_steps, int n_samples, uint64_t seed)
{
    NvtxRange range("dsmc_mixed_run");
    if (!m || !n_runs) return DSMC_E_INVALID;
    CKM(cudaSetDevice(m->device));
    const int n = (int)m->parts.size();
    // every part set up as dsmc_run_ensemble would set it up (buffers,
    // configuration, sample table, zeroed sums and counters), with the
    // mixed ensemble's common tile budget
    for (int k = 0; k < n; ++k) {
        const int i = m->order[k];
        dsmc_ctx* c = m->parts[i];
        dsmc_status st = validate_run(c, n_runs[i], dt, steps, sample_steps, sample_steps, n_samples);
        if (!st) {
            c->have_run = false;
            c->dbg = false;
            c->stats.h2d_bytes = 0;
            c->stats.d2h_bytes = 0;
            c->ls.tile_budget = m->ls.tile_budget;
            c->ls.collide_stage = m->ls.collide_stage;
            st = prepare(c, n_runs[i], dt, steps, sample_steps, sample_steps, n_samples, seed,
                         n_runs[i]);
        }
        if (!st && cudaStreamSynchronize(c->stream) != cudaSuccess) {
            cudaGetLastError();
            st = fail(c, DSMC_E_CUDA, "stream synchronisation failed");
        }
        if (st) {
            char buf[64];
            std::snprintf(buf, sizeof buf, "part %d: ", i);
            return mfail(m, st, buf + c->err);
        }
    }
    CKM(prepare_multi_kernels(m->prec, m->dim, m->ls.tile_budget, m->ls.collide_stage));
    dsmc_status st = m->prec == DSMC_FP64 ? mixed_upload_args<double>(m, n_runs)
                                          : mixed_upload_args<float>(m, n_runs);
    if (st) return st;
    CKM(cudaMemsetAsync(m->d_queue, 0, 4 * kQueueKinds, m->stream));
    const bool profile = (m->flags & DSMC_MIXED_PROFILE) != 0;
    const bool graph = !profile && !(m->flags & DSMC_MIXED_NO_GRAPH);
    if (graph) {
        st = mixed_build_graphs(m, n_runs);
        if (st) return st;
    }
    std::vector<char> is_sample(steps + 1, 0);
    for (int k = 0; k < n_samples; ++k) is_sample[sample_steps[k]] = 1;
    cudaEvent_t e0 = mixed_event(m, 0), e1 = mixed_event(m, 1);
    if (!e0 || !e1) return mfail(m, DSMC_E_CUDA, "cudaEventCreate failed");
    // step-0 state of every part
    for (int k = 0; k < n; ++k) {
        const int i = m->order[k];
        dsmc_ctx* c = m->parts[i];
        AnyArgs u;
        const void* a0 = build_args(c, u, 0, (int)c->opt.run_offset, n_runs[i]);
        launch_init_cells(c->prec, a0, c->ls, m->stream);
        launch_fill(c->prec, a0, c->ls, m->stream);
    }
    m->cur = 0;
    CKM(cudaEventRecord(e0, m->stream));
    size_t evn = 2;
    for (int s = 1; s <= steps; ++s) {
        if (graph) CKM(cudaGraphLaunch(m->gexec[m->cur][is_sample[s]], m->stream));
        else enqueue_mixed_step(m, m->cur, profile ? &evn : nullptr, false, true);
        m->cur ^= 1;
    }
    CKM(cudaEventRecord(e1, m->stream));
    CKM(cudaGetLastError());
    CKM(cudaStreamSynchronize(m->stream));
    float ms_all = 0.f;
    CKM(cudaEventElapsedTime(&ms_all, e0, e1));
    dsmc_stats& ms = m->stats;
    std::memset(&ms, 0, sizeof(ms));
    ms.struct_size = sizeof(dsmc_stats);
    ms.ms_steps = ms_all;
    if (profile) {
        size_t i = 2;
        cudaEvent_t prev = e0;
        for (int s = 1; s <= steps; ++s)
            for (int k = 0; k < kStepKernels; ++k, ++i) {
                float t = 0.f;
                cudaEventElapsedTime(&t, prev, m->events[i]);
                ms.ms_kernel[kKindOf[k]] += t;
                ms.launches_kernel[kKindOf[k]] += 1;
                prev = m->events[i];
            }
    }
    ms.shape[0] = m->ls.move_blocks;
    ms.shape[1] = m->ls.scatter_blocks;
    ms.shape[2] = m->ls.tile_budget;
    ms.shape[3] = m->ls.collide_blocks;
    ms.steps_done = steps;
    dsmc_status worst = DSMC_OK;
    for (int i = 0; i < n; ++i) {
        dsmc_ctx* c = m->parts[i];
        Counters h;
        st = read_counters(c, &h);
        if (st) return mfail(m, st, c->err);
        fill_stats(c, h);
        c->stats.steps_done = steps;
        c->stats.ms_steps = ms_all;
        uint32_t total = 0;
        CKM(cudaMemcpy(&total, c->run_base + n_runs[i], 4, cudaMemcpyDeviceToHost));
        c->stats.particles_now = total;
        c->cur = m->cur;
        ms.particle_steps += h.particle_steps;
        ms.generated += h.generated;
        ms.removed += h.removed;
        ms.wall_hits += h.wall_hits;
        ms.candidates += h.candidates;
        ms.collisions += h.collisions;
        ms.clamps += h.clamps;
        ms.bounce_limit += h.bounce_limit;
        ms.reject_limit += h.reject_limit;
        ms.pool_steps += h.pool_steps;
        ms.big_pool_steps += h.big_pool_steps;
        ms.error_word |= h.error;
        ms.particles_now += total;
        ms.capacity += c->cap_old;
        st = check_error_word(c, h.error);
        if (!st && c->opt.checks) st = run_checks(c, m->cur, (int)c->opt.run_offset, n_runs[i]);
        if (st) {
            if (!worst) {
                char buf[64];
                std::snprintf(buf, sizeof buf, "part %d: ", i);
                m->err = buf + c->err;
            }
            worst = worst ? worst : st;
            continue;
        }
        c->have_run = true;
        c->last_runs = n_runs[i];
        c->last_steps = steps;
        c->last_samples = n_samples;
        c->win_len.assign(n_samples, 1);
    }
    return worst;
}

dsmc_status dsmc_mixed_get_stats(dsmc_mixed* m, dsmc_stats* out)
{
    if (!m || !out || out->struct_size < sizeof(dsmc_stats)) return DSMC_E_INVALID;
    *out = m->stats;
    out->struct_size = sizeof(dsmc_stats);
    return DSMC_OK;
}

// ---------------------------------------------------------------------------
// Ensemble run without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want a
// result: processes whose device memory is fully handed to another
// allocator or a fixed budget up front (a cudaMalloc would fail or take from
// that budget), or real-time loops that forbid allocator calls on their
// critical path (cudaMalloc/cudaFree may synchronise the device).  For them, dsmc_run_ensemble_noalloc runs the whole batched step
// loop inside one fixed scratch array that is part of the library's device
// image (kNoallocBytes on every GPU that loads the library, held until the
// process exits).  It calls no cudaMalloc, cudaFree, event or graph creation.

namespace {
constexpr size_t kNoallocBytes = (size_t)48 << 20;
constexpr int kNoallocMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Builds the per-step sample table in the scratch: -1 everywhere, sample k
// (a one-step window) at step sample_steps[k] (the steps were copied to
// `ss` first).
__global__ void k_noalloc_sample_table(int32_t* slot, int n_slot, const int32_t* ss, int n_samples)
{
    for (int i = threadIdx.x; i < n_slot; i += blockDim.x) slot[i] = -1;
    __syncthreads();
    for (int k = threadIdx.x; k < n_samples; k += blockDim.x) slot[ss[k]] = k | kSlotFirst | kSlotLast;
}

// Device address of the scratch array on the context's device.  The lookup
// runs on the first call per device, with that device current.
static dsmc_status noalloc_base(dsmc_ctx* ctx, unsigned char** out)
{
    static unsigned char* base[kNoallocMaxDevices] = {};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (ctx->device < 0 || ctx->device >= kNoallocMaxDevices)
        return fail(ctx, DSMC_E_INVALID, "device ordinal out of range for the no-allocation path");
    if (!base[ctx->device]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        base[ctx->device] = static_cast<unsigned char*>(p);
    }
    *out = base[ctx->device];
    return DSMC_OK;
}

struct ScratchCarver {
    unsigned char* base;
    size_t used;
    void* take(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        if (bytes == 0) bytes = 256;
        void* p = base + used;
        used += bytes;
        return used <= kNoallocBytes ? p : nullptr;
    }
};

// Lays the run's buffers out in the scratch array (the same buffers
// ensure_alloc would allocate, without the debug ones) and returns the
// bytes needed; the pointers are valid only if that is <= kNoallocBytes.
static size_t noalloc_layout(dsmc_ctx* ctx, unsigned char* base, int n_runs, int64_t cap_run,
                             int steps, int n_samples, int32_t** ss_stage)
{
    ScratchCarver sc{base, 0};
    const int64_t cap_old = (cap_run * n_runs + 255) / 256 * 256;
    const int64_t gcap = gen_capacity(ctx);
    const int64_t cap_new = gcap * n_runs;
    const int64_t total_cells = (int64_t)ctx->ncells * n_runs;
    const size_t ts = ctx->prec == DSMC_FP64 ? 8 : 4;
    const int64_t slots = cap_old + cap_new;
    ctx->d_cfg = (Cfg*)sc.take(sizeof(Cfg));
    ctx->d_ctr = (Counters*)sc.take(sizeof(Counters));
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 3; ++a) {
            ctx->X[b][a] = a < ctx->dim ? sc.take(ts * slots) : nullptr;
            ctx->V[b][a] = sc.take(ts * slots);
        }
        ctx->ID[b] = nullptr;
        ctx->CI[b] = (uint32_t*)sc.take(4 * cap_old);
    }
    ctx->gc = (uint32_t*)sc.take(4 * slots);
    ctx->lcr = (uint32_t*)sc.take(4 * cap_old);
    ctx->lcr_dbg = nullptr;
    ctx->count = (uint32_t*)sc.take(4 * total_cells);
    ctx->start = (uint32_t*)sc.take(4 * (total_cells + 2));
    const int scan_blocks = (int)((total_cells + kScanTile - 1) / kScanTile);
    ctx->block_sums = (uint32_t*)sc.take(4 * (scan_blocks + 1));
    ctx->run_base = (uint32_t*)sc.take(4 * (n_runs + 1));
    ctx->next_id = (uint32_t*)sc.take(4 * n_runs);
    ctx->rem = (double*)sc.take(8 * total_cells);
    ctx->smax = sc.take(ts * total_cells);
    ctx->mom = (double*)sc.take(8 * DSMC_NMOM * total_cells);
    ctx->cand = ctx->accd = nullptr;
    const int64_t max_big = cap_old / (kWarpMax + 1) + 1;
    ctx->big_list = (uint32_t*)sc.take(4 * max_big);
    ctx->slow_list = (uint32_t*)sc.take(4 * cap_old);
    ctx->gen_tot = (uint32_t*)sc.take(4 * (size_t)n_runs * gen_groups_of(ctx));
    ctx->gen_done = (uint32_t*)sc.take(4 * (size_t)n_runs);
    ctx->sample_slot = (int32_t*)sc.take(4 * (size_t)(steps + 2));
    ctx->acc = (double*)sc.take(8 * (size_t)std::max(n_samples, 1) * ctx->G * ctx->ncells * DSMC_NMOM);
    ctx->macro = nullptr;
    *ss_stage = (int32_t*)sc.take(4 * (size_t)std::max(n_samples, 1));
    ctx->n_launch = n_runs;
    ctx->cap_old = cap_old;
    ctx->cap_new = cap_new;
    ctx->gcap = gcap;
    ctx->max_big = max_big;
    ctx->total_cells = total_cells;
    ctx->steps_alloc = steps + 2;
    return sc.used;
}

// forget the scratch layout, so that a later dsmc_run_ensemble allocates its
// own buffers: the sizes that ensure_alloc compares are cleared and every
// pointer into the shared scratch array is dropped
static void noalloc_forget(dsmc_ctx* ctx)
{
    ctx->n_launch = 0;
    ctx->cap_old = ctx->cap_new = ctx->gcap = ctx->max_big = 0;
    ctx->total_cells = 0;
    ctx->steps_alloc = 0;
    ctx->n_samples_alloc = 0;
    ctx->G_alloc = 0;
    ctx->generation++;
    ctx->have_run = false;
    ctx->d_cfg = nullptr;
    ctx->d_ctr = nullptr;
    for (int b = 0; b < 2; ++b) {
        for (int a = 0; a < 3; ++a) ctx->X[b][a] = ctx->V[b][a] = nullptr;
        ctx->ID[b] = ctx->CI[b] = nullptr;
    }
    ctx->gc = ctx->lcr_dbg = nullptr;
    ctx->lcr = nullptr;
    ctx->count = ctx->start = ctx->block_sums = ctx->run_base = ctx->next_id = nullptr;
    ctx->cand = ctx->accd = ctx->big_list = ctx->slow_list = ctx->gen_tot = ctx->gen_done = nullptr;
    ctx->rem = ctx->mom = ctx->acc = ctx->macro = nullptr;
    ctx->smax = nullptr;
    ctx->sample_slot = nullptr;
}

// The run proper of dsmc_run_ensemble_noalloc, on the buffers noalloc_layout
// placed in the scratch: clears what must start from zero, builds the
// sample table, advances the steps and copies the counters (and the group
// sums) out.
static dsmc_status noalloc_steps(dsmc_ctx* ctx, int n_runs, int steps, const int32_t* sample_steps,
                                 int n_samples, int32_t* ss_dev, double* raw_out, size_t need,
                                 Counters* h)
{
    const int G = ctx->G;
    // every buffer that must start from zero (or from the dead key) is set
    // here: the scratch keeps the previous call's contents
    CK(cudaMemcpyAsync(ctx->d_cfg, &ctx->hcfg, sizeof(Cfg), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), ctx->stream));
    CK(cudaMemsetAsync(ctx->gc, 0xFF, 4 * (size_t)(ctx->cap_old + ctx->cap_new), ctx->stream));
    CK(cudaMemsetAsync(ctx->acc, 0, 8 * (size_t)std::max(n_samples, 1) * G * ctx->ncells * DSMC_NMOM,
                       ctx->stream));
    if (n_samples > 0)
        CK(cudaMemcpyAsync(ss_dev, sample_steps, 4 * (size_t)n_samples, cudaMemcpyHostToDevice,
                           ctx->stream));
    k_noalloc_sample_table<<<1, 256, 0, ctx->stream>>>(ctx->sample_slot, steps + 2, ss_dev, n_samples);
    CK(cudaGetLastError());
    CK(prepare_kernels(ctx->prec, ctx->dim, ctx->ls.tile_budget, ctx->ls.collide_stage));
    AnyArgs u;
    enqueue_init(ctx, build_args(ctx, u, 0, (int)ctx->opt.run_offset, n_runs));
    ctx->cur = 0;
    for (int s = 1; s <= steps; ++s) {
        AnyArgs v;
        enqueue_step(ctx, build_args(ctx, v, ctx->cur, (int)ctx->opt.run_offset, n_runs), nullptr);
        ctx->cur ^= 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, ctx->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && n_samples > 0)
        e = cudaMemcpyAsync(raw_out, ctx->acc, 8 * need, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess)
        return fail(ctx, DSMC_E_CUDA, std::string("no-allocation run: ") + cudaGetErrorString(e));
    return DSMC_OK;
}

dsmc_status dsmc_run_ensemble_noalloc(dsmc_ctx* ctx, int n_runs, double dt, int steps,
                                      const int32_t* sample_steps, int n_samples, uint64_t seed,
                                      double* raw_out, size_t raw_len)
{
    if (!ctx) return DSMC_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    dsmc_status st = validate_run(ctx, n_runs, dt, steps, sample_steps, sample_steps, n_samples);
    if (st) return st;
    if (!ctx->bufs.empty())
        return fail(ctx, DSMC_E_STATE,
                    "context already owns device buffers: use a fresh context for the "
                    "no-allocation path");
    if (ctx->opt.debug || ctx->opt.profile)
        return fail(ctx, DSMC_E_INVALID, "debug and profile options need allocated buffers");
    const int G = std::min(n_runs, DSMC_MAX_GROUPS);
    const size_t need = (size_t)n_samples * G * ctx->ncells * DSMC_NMOM;
    if (n_samples > 0 && (!raw_out || raw_len < need))
        return fail(ctx, DSMC_E_INVALID, "raw_out missing or smaller than n_samples x G x ncells x 7");
    unsigned char* base = nullptr;
    st = noalloc_base(ctx, &base);
    if (st) return st;
    st = build_cfg(ctx, dt, seed);
    if (st) return st;
    ctx->G = G;
    const int64_t cap_run = estimate_per_run(ctx, steps);
    int32_t* ss_dev = nullptr;
    const size_t bytes = noalloc_layout(ctx, base, n_runs, cap_run, steps, n_samples, &ss_dev);
    if (bytes > kNoallocBytes || ctx->cap_old + ctx->cap_new >= 0xFFFFFFF0ll) {
        noalloc_forget(ctx);
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "problem needs %zu bytes of device scratch; the no-allocation path holds %zu",
                      bytes, kNoallocBytes);
        return fail(ctx, DSMC_E_INVALID, msg);
    }
    // every failure from here on goes through noalloc_forget, so that the
    // context never keeps pointers into the shared scratch
    Counters h;
    const dsmc_status rs = noalloc_steps(ctx, n_runs, steps, sample_steps, n_samples, ss_dev,
                                         raw_out, need, &h);
    noalloc_forget(ctx);
    if (rs) return rs;
    fill_stats(ctx, h);
    ctx->stats.steps_done = steps;
    return check_error_word(ctx, h.error);
}
