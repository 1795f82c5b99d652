// dsmc_kernels.cu -- sm_103a kernels of the ensemble DSMC step.
//
// One time step of all runs of the ensemble (Sec. 1.1, Fig. 1: Generation,
// Motion, Enumeration/Indexing, Interaction, Sampling) as a fixed sequence
// of launches over the whole batch of runs:
//
//   k_generate   one CTA per run: inflow counts, entrants created and moved
//                for their first fractional step (Generation + Motion)
//   k_move       grid-stride over the particle pool: free flight (surface
//                interaction in k_move_slow), new cell key, the cell's
//                count (Motion + Enumeration)
//   k_scan1/2    exclusive prefix over the run-major cell counts: each
//                cell's first pool position, each run's first position
//                (Indexing)
//   k_scatter    LCR[start[cell] + r] = slot, r counted down from the
//                cell's count (Indexing)
//   k_cell       one CTA per 256 cells: each cell's particles put in slot
//                order (the order of one serial pass over the pool) and
//                gathered into the next pool (Indexing)
//   k_cell_big   cells above 128 particles (a CTA, or a quarter CTA, per
//                cell): the cell put in slot order (LSD radix sort of
//                compact slot keys) and gathered into the next pool
//   k_collide_big one warp per such cell: NTC collisions (disjoint pairs
//                side by side) and moments
//   k_collide    one thread per cell, a tile's velocities staged in shared
//                memory: NTC collisions, and the cell moments at sample
//                steps (Interaction + Sampling)
//   k_reduce     fixed-order sum of the runs' cell moments into group
//                accumulators at sample steps (Sampling)
//
// Every random number comes from Philox4x32-10 keyed by the seed with
// (entity, purpose<<28 | draw, step, run) as the counter, so a particle's
// history does not depend on the launch shape or on the other runs.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <utility>

#include "dsmc_internal.cuh"

// This file is compiled twice: with DSMC_KERNELS_FP64 for FP64 particle
// state (no fused multiply-add contraction: every operation rounded as the
// FP64 oracle rounds it), and without it for FP32 state (contraction
// allowed).  Each compilation instantiates the kernels for its precision
// only and defines its launchers in namespace dsmc::f64 or dsmc::f32.
#if defined(DSMC_KERNELS_FP64)
#define DSMC_KT double
#define DSMC_KNS f64
#define DSMC_KPREC DSMC_FP64
#else
#define DSMC_KT float
#define DSMC_KNS f32
#define DSMC_KPREC DSMC_FP32
#endif

namespace dsmc {
namespace DSMC_KNS {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 draw_bits(uint64_t seed, uint32_t run, uint32_t step,
                                           uint32_t entity, uint32_t purpose, uint32_t sub)
{
    return philox(make_uint4(entity, (purpose << 28) | (sub & 0x0FFFFFFFu), step, run),
                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// the same rounds with the key schedule precomputed (rk[2r], rk[2r + 1] =
// the round-r key words), read from the launch parameters
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint32_t* rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

// (m + 1/2) / 2^23 from the top 23 bits: exact in float and double
template <typename T>
__device__ __forceinline__ T u01(uint32_t x)
{
    return ((T)(x >> 9) + (T)0.5) * (T)(1.0 / 8388608.0);
}

__device__ __forceinline__ float dlog(float x) { return logf(x); }
__device__ __forceinline__ double dlog(double x) { return log(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float dpow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double dpow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float dfloor(float x) { return floorf(x); }
__device__ __forceinline__ double dfloor(double x) { return floor(x); }
__device__ __forceinline__ void dsincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void dsincospi(double x, double* s, double* c) { sincospi(x, s, c); }

// Box-Muller pair from two uniforms: sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2)
template <typename T>
__device__ __forceinline__ void gauss2(T u1, T u2, T& z0, T& z1)
{
    const T r = dsqrt((T)-2.0 * dlog(u1));
    T s, c;
    dsincospi((T)2.0 * u2, &s, &c);
    z0 = r * c;
    z1 = r * s;
}

// ---------------------------------------------------------------------------
// Geometry.  A particle's position is held as its run-local cell index (one
// integer per axis while it moves, one linear index in memory) and its
// offset f in [0, d_a] from that cell's lower corner along each axis.  The
// distances Motion needs -- to a wall, a plate or a cell face -- are then
// differences of numbers no larger than a few cells, so binary32 state
// resolves positions to ~1e-7 of a cell rather than of the domain.

// offset in cell units: f / d in double precision; in single precision f
// times the binary32 reciprocal of d (one multiply)
__device__ __forceinline__ double in_cells(const Cfg& c, int a, double f) { return f / c.d[a]; }
__device__ __forceinline__ float in_cells(const Cfg& c, int a, float f) { return f * (float)c.inv_d[a]; }
__device__ __forceinline__ double in_cells(const Hot<double>& c, int a, double f) { return f / c.d[a]; }
__device__ __forceinline__ float in_cells(const Hot<float>& c, int a, float f) { return f * c.inv_d[a]; }

// a straight flight from cell i to cell j along axis a passes the plane of
// a plate normal to a (face index p): min(i, j) < p <= max(i, j).  Every
// flight that meets a plate passes its plane, so a flight for which this is
// false for every plate meets none (the plate's extent and activity are not
// looked at: the test may only send extra flights to the exact path).
__device__ __forceinline__ bool crosses_plate(const Cfg& c, int a, int i, int j)
{
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    for (int pi = 0; pi < c.n_plate; ++pi) {
        const BcDev& b = c.bc[c.plate_idx[pi]];
        if (b.plate_axis == a && lo < b.plate_index && b.plate_index <= hi) return true;
    }
    return false;
}
template <typename T>
__device__ __forceinline__ bool crosses_plate(const Hot<T>& c, int a, int i, int j)
{
    if (c.n_plate < 0) return ((c.plate_axes >> a) & 1u) != 0u;
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    for (int pi = 0; pi < c.n_plate; ++pi)
        if (c.plate_ax[pi] == a && lo < c.plate_ix[pi] && c.plate_ix[pi] <= hi) return true;
    return false;
}

// move whole cells so that 0 <= f <= d along axis a (clamped to the grid)
template <typename T>
__device__ __forceinline__ void renorm(const Cfg& c, int a, int& i, T& f)
{
    const int k = (int)dfloor(in_cells(c, a, f));
    if (k != 0) {
        int ni = i + k;
        ni = ni < 0 ? 0 : (ni > c.n[a] - 1 ? c.n[a] - 1 : ni);
        f = f - (T)(ni - i) * (T)c.d[a];
        i = ni;
    }
}

// x / n for x < 2^24 (float quotient, corrected by one)
__device__ __forceinline__ uint32_t div_small(uint32_t x, uint32_t n)
{
    uint32_t q = (uint32_t)((float)x * __frcp_rn((float)n));
    if (q * n > x) --q;
    else if ((q + 1u) * n <= x) ++q;
    return q;
}

template <int DIM, class C>
__device__ __forceinline__ void decode_cell(const C& c, uint32_t lin, int* ci)
{
    const uint32_t q = div_small(lin, (uint32_t)c.n[0]);
    ci[0] = (int)(lin - q * (uint32_t)c.n[0]);
    if (DIM == 3) {
        const uint32_t q2 = div_small(q, (uint32_t)c.n[1]);
        ci[1] = (int)(q - q2 * (uint32_t)c.n[1]);
        ci[2] = (int)q2;
    } else {
        ci[1] = (int)q;
        ci[2] = 0;
    }
}

template <int DIM, class C>
__device__ __forceinline__ uint32_t encode_cell(const C& c, const int* ci)
{
    return (uint32_t)(ci[0] + c.n[0] * (ci[1] + (DIM == 3 ? c.n[1] * ci[2] : 0)));
}

__device__ __forceinline__ bool bc_active(const BcDev& b, int step)
{
    return step >= b.step_from && (b.step_to == 0 || step <= b.step_to);
}

// last listed active segment covering face cell (a, b); -1 = open
__device__ int bc_lookup(const Cfg& c, int face, int a, int b, int step)
{
    int win = -1;
    for (int q = 0; q < c.n_bc; ++q) {
        const BcDev& s = c.bc[q];
        if (s.face != face) continue;
        if (a < s.lo[0] || a >= s.hi[0] || b < s.lo[1] || b >= s.hi[1]) continue;
        if (!bc_active(s, step)) continue;
        win = q;
    }
    return win;
}

struct LocalCounters {
    uint32_t removed = 0, wall_hits = 0, bounce = 0;
};

// Straight flight for tau that ends strictly inside the box (by a margin far
// above rounding) and passes no plate's plane: no surface event can occur,
// and the result equals move_particle's.  Returns false (state untouched)
// otherwise.
template <typename T, int DIM, class C>
__device__ __forceinline__ bool try_free_flight(const C& c, int* ci, T* f, const T* v, T tau)
{
    const T margin = sizeof(T) == 4 ? (T)1e-5 : (T)1e-12;
    int ni[3];
    T nf[3];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const T d = (T)c.d[a];
        nf[a] = f[a] + v[a] * tau;
        const int k = (int)dfloor(in_cells(c, a, nf[a]));
        ni[a] = ci[a] + k;
        if (ni[a] < 0 || ni[a] > c.n[a] - 1) return false;
        if (k != 0) nf[a] = nf[a] - (T)k * d;
        if (ni[a] == 0 && !(nf[a] > margin * d)) return false;
        if (ni[a] == c.n[a] - 1 && !(nf[a] < d - margin * d)) return false;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
        if (ni[a] != ci[a] && crosses_plate(c, a, ci[a], ni[a])) return false;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { ci[a] = ni[a]; f[a] = nf[a]; }
    return true;
}

template <typename T, int DIM>
__device__ bool move_particle(const Cfg& c, int* ci, T* f, T* v, uint32_t place, uint32_t run,
                              uint32_t step, T tau, LocalCounters& lc, uint32_t& vmask);

// Motion of one particle for time tau: free flight with the surface events
// taken in time order (ties: x, y, z faces, then plates in list order).
// Returns false if the particle left through an open face.  vmask collects
// the velocity components that changed.  `place` -- the particle's place in
// its run's particle order this step (old particles in pool order, then the
// entrants in generation order) -- keys its wall draws.
template <typename T, int DIM>
__device__ bool move_particle(const Cfg& c, int* ci, T* f, T* v, uint32_t place, uint32_t run,
                              uint32_t step, T tau, LocalCounters& lc, uint32_t& vmask)
{
    for (int bounce = 0;; ++bounce) {
        int hit = -1;
        T th = (T)0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const T d = (T)c.d[a];
            T t;
            if (v[a] > (T)0) t = ((T)(c.n[a] - 1 - ci[a]) * d + (d - f[a])) / v[a];
            else if (v[a] < (T)0) t = ((T)ci[a] * d + f[a]) / (-v[a]);
            else continue;
            if (t < (T)0) t = (T)0;
            if (t <= tau && (hit < 0 || t < th)) { hit = 2 * a + (v[a] > (T)0 ? 1 : 0); th = t; }
        }
        for (int pi = 0; pi < c.n_plate; ++pi) {
            const int q = c.plate_idx[pi];
            const BcDev& b = c.bc[q];
            if (!bc_active(b, step)) continue;
            const int a = b.plate_axis;
            const T dist = (T)(b.plate_index - ci[a]) * (T)c.d[a] - f[a];   // x_plate - x
            if (!((dist > (T)0 && v[a] > (T)0) || (dist < (T)0 && v[a] < (T)0))) continue;
            const T t = dist / v[a];
            if (!(t <= tau && (hit < 0 || t < th))) continue;
            bool inside = true;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int tb = k == 0 ? b.t0 : b.t1;
                if (tb >= DIM) continue;
                int ib = ci[tb];
                T fb = f[tb] + v[tb] * t;
                renorm<T>(c, tb, ib, fb);
                if (!(ib >= b.lo[k] && ib < b.hi[k])) inside = false;
            }
            if (inside) { hit = 100 + q; th = t; }
        }
        if (hit < 0) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                f[a] = f[a] + v[a] * tau;
                renorm<T>(c, a, ci[a], f[a]);
            }
            return true;
        }
        if (bounce == kMaxBounce) { lc.bounce++; return true; }
        int axis, kind, t0, t1;
        T dir;
        double Tsd = 0.0;
        if (hit < 100) {
            axis = hit >> 1;
            const int side = hit & 1;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                if (a == axis) {
                    ci[a] = side ? c.n[a] - 1 : 0;
                    f[a] = side ? (T)c.d[a] : (T)0;
                } else {
                    f[a] = f[a] + v[a] * th;
                    renorm<T>(c, a, ci[a], f[a]);
                }
            }
            t0 = axis == 0 ? 1 : 0;
            t1 = axis == 2 ? 1 : 2;
            const int q = bc_lookup(c, hit, ci[t0], t1 < DIM ? ci[t1] : 0, (int)step);
            kind = q < 0 ? DSMC_BC_OUTFLOW : c.bc[q].kind;
            if (q >= 0) Tsd = c.bc[q].sd;
            dir = side ? (T)-1 : (T)1;
        } else {
            const BcDev& b = c.bc[hit - 100];
            axis = b.plate_axis;
            t0 = b.t0;
            t1 = b.t1;
            dir = v[axis] > (T)0 ? (T)-1 : (T)1;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                if (a == axis) {
                    ci[a] = b.plate_index;
                    f[a] = (T)0;
                } else {
                    f[a] = f[a] + v[a] * th;
                    renorm<T>(c, a, ci[a], f[a]);
                }
            }
            kind = b.kind;
            Tsd = b.sd;
        }
        tau = tau - th;
        if (kind == DSMC_BC_OUTFLOW || kind == DSMC_BC_INFLOW) { lc.removed++; return false; }
        lc.wall_hits++;
        if (kind == DSMC_BC_SPECULAR) {
            v[axis] = -v[axis];
            vmask |= 1u << axis;
        } else {
            const uint4 r = draw_bits(c.seed, run, step, place, kWall, (uint32_t)bounce);
            const T sw = (T)Tsd;
            T z0, z1;
            gauss2<T>(u01<T>(r.y), u01<T>(r.z), z0, z1);
            v[axis] = dir * (sw * dsqrt((T)-2.0 * dlog(u01<T>(r.x))));
            v[t0] = sw * z0;
            v[t1] = sw * z1;
            vmask |= 7u;
        }
    }
}

// ---------------------------------------------------------------------------
// warp / block helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Programmatic dependent launch: the step kernels are launched so that each
// may be scheduled while the kernel before it in the stream is finishing.
// Every step kernel calls this first: it lets the next kernel begin its
// launch, then waits until the previous kernel has completed and its memory
// is visible (a no-op for a kernel launched without the attribute).
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// atomicAdd returning the old value, with an L2 evict-last policy: the
// per-cell counters stay cached while the particle streams pass through L2
__device__ __forceinline__ uint32_t atomic_add_l2_keep(uint32_t* p, uint32_t v)
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    uint32_t old;
    asm volatile("atom.global.add.L2::cache_hint.u32 %0, [%1], %2, %3;"
                 : "=r"(old)
                 : "l"(p), "r"(v), "l"(pol)
                 : "memory");
    return old;
}

// atomicAdd without a returned value (red), with the same L2 evict-last
// policy: Motion only counts, nothing waits for the old value
__device__ __forceinline__ void red_add_l2_keep(uint32_t* p, uint32_t v)
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("red.global.add.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
                 : "memory");
}

// Runs of equal cell keys in consecutive lanes: in a cell-ordered pool the
// 32 consecutive slots of a warp hold few cells, each in one or a few runs.
// Live lanes whose key equals the previous lane's (live) key continue that
// lane's run; the first lane of a run is its head.  Gives this lane's head
// and, on the head, the run's length.  (A key that reappears after another
// key starts a second run of its own: runs only aggregate, every lane still
// belongs to exactly one run.)
__device__ __forceinline__ void key_runs(uint32_t key, bool live, uint32_t lane, uint32_t& head,
                                         uint32_t& len)
{
    const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
    const uint32_t live_mask = __ballot_sync(0xFFFFFFFFu, live);
    const bool prev_live = lane > 0u && ((live_mask >> (lane - 1u)) & 1u);
    const uint32_t heads = __ballot_sync(0xFFFFFFFFu, live && (!prev_live || prev != key));
    const uint32_t upto = 0xFFFFFFFFu >> (31u - lane);            // lanes 0 .. lane
    const uint32_t le = heads & upto;
    head = le ? 31u - (uint32_t)__clz(le) : lane;
    const uint32_t stop = (heads | ~live_mask) & ~upto;            // heads or dead lanes above
    const uint32_t end = stop ? (uint32_t)__ffs(stop) - 1u : 32u;
    len = end - head;
}

// load with an L2 evict-last policy (per-cell tables that later kernels of
// the step read again)
__device__ __forceinline__ uint32_t ld_l2_keep(const uint32_t* p)
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    uint32_t v;
    asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, untiled) from global to shared memory,
// completed on an mbarrier.  Addresses and sizes must be multiples of 16
// bytes; every wait is bounded.
constexpr uint32_t kWaitPolls = 1u << 20;   // try_wait polls before a wait is abandoned

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before
// later bulk copies into shared memory
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0u;
}

// wait for the phase with the given parity to complete; false if it did not
// within kWaitPolls polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (uint32_t it = 0; it < kWaitPolls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void flush_counters(Counters* ctr, const LocalCounters& lc)
{
    const uint32_t r = __reduce_add_sync(0xFFFFFFFFu, lc.removed);
    const uint32_t w = __reduce_add_sync(0xFFFFFFFFu, lc.wall_hits);
    const uint32_t b = __reduce_add_sync(0xFFFFFFFFu, lc.bounce);
    if (lane_id() == 0) {
        if (r) atomicAdd(&ctr->removed, (unsigned long long)r);
        if (w) atomicAdd(&ctr->wall_hits, (unsigned long long)w);
        if (b) atomicAdd(&ctr->bounce_limit, (unsigned long long)b);
    }
}

// exclusive scan of one value per thread over the block (blockDim <= 1024)
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* smem_warp, uint32_t& total)
{
    const int lane = lane_id(), warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? smem_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) smem_warp[lane] = s;
    }
    __syncthreads();
    const uint32_t before = warp ? smem_warp[warp - 1] : 0u;
    total = smem_warp[nw - 1];
    __syncthreads();
    return before + x - v;
}

// ---------------------------------------------------------------------------
// Step-0 state
template <typename T>
__global__ void k_init_cells(StepArgs<T> a)
{
    const Cfg& c = *a.cfg;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.total_cells;
         i += (int64_t)gridDim.x * blockDim.x) {
        a.rem[i] = 0.0;
        a.smax[i] = (T)c.smax0;
        a.count[i] = 0u;
    }
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < a.n_runs;
         r += (int64_t)gridDim.x * blockDim.x)
        a.gen_done[r] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctr->step = 1u;
        a.ctr->n_big = 0u;
        a.ctr->n_slow = 0u;
    }
}

// freestream fill, part 1: Poisson-rounded count per cell
template <typename T>
__global__ void k_fill_count(StepArgs<T> a)
{
    const Cfg& c = *a.cfg;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.total_cells;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t rl = (uint32_t)(i / c.ncells), cell = (uint32_t)(i - (int64_t)rl * c.ncells);
        const uint4 r = draw_bits(c.seed, a.run0 + rl, 0u, cell, kFillCount, 0u);
        a.count[i] = c.fill ? (uint32_t)floor(c.fill_lam + u01<double>(r.x)) : 0u;
    }
}

// freestream fill, part 2: one warp per cell writes its particles in
// (cell, k) order; ids (debug mode) count per run in that order
template <typename T, int DIM>
__global__ void k_fill_particles(StepArgs<T> a)
{
    const Cfg& c = *a.cfg;
    const int lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
         i < a.total_cells; i += warps) {
        const uint32_t rl = (uint32_t)(i / c.ncells), cell = (uint32_t)(i - (int64_t)rl * c.ncells);
        const uint32_t beg = a.start[i], N = a.start[i + 1] - beg;
        // the counts start the first step at zero (the scan leaves them)
        if (lane == 0) a.count[i] = 0u;
        if ((int64_t)beg + N > a.cap_old) {
            if (lane == 0) atomicOr(&a.ctr->error, DSMC_ERR_POOL);
            continue;
        }
        const T sd = (T)c.fill_sd;
        for (uint32_t k = lane; k < N; k += 32) {
            const uint4 b0 = draw_bits(c.seed, a.run0 + rl, 0u, cell, kFillPart, 2u * k);
            const uint4 b1 = draw_bits(c.seed, a.run0 + rl, 0u, cell, kFillPart, 2u * k + 1u);
            T z[4];
            gauss2<T>(u01<T>(b0.x), u01<T>(b0.y), z[0], z[1]);
            gauss2<T>(u01<T>(b0.z), u01<T>(b0.w), z[2], z[3]);
            const T ub[3] = {u01<T>(b1.x), u01<T>(b1.y), u01<T>(b1.z)};
            const uint32_t p = beg + k;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) a.xi[ax][p] = ub[ax] * (T)c.d[ax];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) a.vi[ax][p] = (T)c.fill_U[ax] + sd * z[ax];
            if (a.idi) a.idi[p] = (beg - a.run_base[rl]) + k;
            a.ci_i[p] = (uint32_t)i;
        }
    }
}

template <typename T>
__global__ void k_fill_ids(StepArgs<T> a)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.n_runs; r += gridDim.x * blockDim.x)
        a.next_id[r] = a.run_base[r + 1] - a.run_base[r];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.start[a.total_cells + 1] = a.run_base[a.n_runs];
}

// inflow segment that owns element e (elements are numbered segment by
// segment in list order); the caller guarantees 0 <= e < n_elem
__device__ __forceinline__ int inflow_segment_of(const Cfg& c, int64_t e)
{
    int q = 0;
    for (; q < c.n_bc - 1; ++q) {
        const BcDev& b = c.bc[q];
        if (b.kind == DSMC_BC_INFLOW && b.face < 6 && e >= b.elem_base && e < b.elem_base + b.n_elem)
            break;
    }
    return q;
}

// Entrants of inflow element e this step: floor(lambda + R) if its segment
// is active and owns the face cell (the last listed active segment wins),
// else 0.
__device__ __forceinline__ uint32_t element_entrants(const Cfg& c, uint32_t run, uint32_t step,
                                                     int64_t e)
{
    const int q = inflow_segment_of(c, e);
    const BcDev& b = c.bc[q];
    const int64_t loc = e - b.elem_base;
    const int aa = b.lo[0] + (int)(loc % b.elem_w), bb = b.lo[1] + (int)(loc / b.elem_w);
    if (!(bc_active(b, (int)step) && bc_lookup(c, b.face, aa, bb, (int)step) == q)) return 0u;
    const uint4 r = draw_bits(c.seed, run, step, (uint32_t)e, kGenCount, 0u);
    return (uint32_t)floor(b.lam + u01<double>(r.x));
}

// Generation, counting pass (runs with more than kGenElems inflow
// elements): entrants of every group of kGenElems consecutive elements, one
// CTA per (run, group), so that the creating pass can number each group's
// entrants without waiting for the groups before it.
template <typename T>
__device__ __forceinline__ void gen_count_block(const StepArgs<T>& a, uint32_t blk)
{
    const Cfg& c = *a.cfg;
    __shared__ uint32_t s_warp[32];
    const uint32_t G = (uint32_t)a.gen_groups;
    const uint32_t rl = blk / G, grp = blk - rl * G;
    const uint32_t run = a.run0 + rl;
    const uint32_t step = a.ctr->step;
    const int64_t e0 = (int64_t)grp * kGenElems;
    const int64_t e1 = e0 + kGenElems < c.n_elem ? e0 + kGenElems : c.n_elem;
    uint32_t sum = 0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) sum += element_entrants(c, run, step, e);
    uint32_t total;
    block_exclusive_scan(sum, s_warp, total);
    if (threadIdx.x == 0) a.gen_tot[(int64_t)rl * G + grp] = total;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gen_count(StepArgs<T> a)
{
    pdl_enter();
    gen_count_block(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Generation: one CTA per (run, group of kGenElems inflow elements).
// Elements are taken in segment-list order; each element's count is
// floor(lambda + R); a run's entrants are numbered (ids, new-region slots)
// in (element, k) order -- a group starts after the entrants of the groups
// before it -- created from their draws and moved for R_f dt.
template <typename T, int DIM>
__device__ __forceinline__ void generate_block(const StepArgs<T>& a, uint32_t blk)
{
    const Cfg& c = *a.cfg;
    __shared__ uint32_t s_off[257];
    __shared__ uint32_t s_warp[32];
    const uint32_t GG = (uint32_t)a.gen_groups;
    const uint32_t rl = blk / GG, grp = blk - rl * GG;
    const uint32_t run = a.run0 + rl;
    const uint32_t step = a.ctr->step;
    const uint32_t n_old = min(a.run_base[rl + 1], (uint32_t)a.cap_old) -
                           min(a.run_base[rl], (uint32_t)a.cap_old);
    const uint32_t id0 = a.next_id[rl];
    const int64_t gen_base = a.cap_old + (int64_t)rl * a.gcap;
    const int64_t e_begin = (int64_t)grp * kGenElems;
    const int64_t e_end = GG == 1u ? c.n_elem
                                   : (e_begin + kGenElems < c.n_elem ? e_begin + kGenElems : c.n_elem);
    uint32_t prefix = 0;
    for (uint32_t g = 0; g < grp; ++g) prefix += a.gen_tot[(int64_t)rl * GG + g];
    uint32_t running = prefix;
    LocalCounters lc;
    uint32_t rejects = 0;
    bool overflow = false;
    for (int64_t chunk = e_begin; chunk < e_end; chunk += blockDim.x) {
        const int64_t e = chunk + threadIdx.x;
        const uint32_t G = e < e_end ? element_entrants(c, run, step, e) : 0u;
        uint32_t total;
        const uint32_t off = block_exclusive_scan(G, s_warp, total);
        s_off[threadIdx.x] = off;
        if (threadIdx.x == 0) s_off[blockDim.x] = total;
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < total; j += blockDim.x) {
            // element of entrant j: last t with s_off[t] <= j
            int lo = 0, hi = (int)blockDim.x - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= j) lo = mid; else hi = mid - 1;
            }
            const int64_t e2 = chunk + lo;
            const uint32_t k = j - s_off[lo];
            const uint32_t local = running + j;
            if ((int64_t)local >= a.gcap) { overflow = true; continue; }
            const int q = inflow_segment_of(c, e2);
            const BcDev& b = c.bc[q];
            const int64_t loc = e2 - b.elem_base;
            const int aa = b.lo[0] + (int)(loc % b.elem_w), bb = b.lo[1] + (int)(loc / b.elem_w);
            const uint4 b0 = draw_bits(c.seed, run, step, (uint32_t)e2, kGenPart, k * kGenBlocks);
            const uint4 b1 = draw_bits(c.seed, run, step, (uint32_t)e2, kGenPart, k * kGenBlocks + 1u);
            T z0, z1;
            gauss2<T>(u01<T>(b1.x), u01<T>(b1.y), z0, z1);
            // inward normal speed ratio: normal proposals about the mode xm
            // (variance 1/2), kept with probability (x/xm) exp(1 - x/xm)
            const T xm = (T)b.xm;
            T xi = xm;
            bool got = false;
            for (uint32_t blk = 2; blk < (uint32_t)kGenBlocks && !got; ++blk) {
                const uint4 rb = draw_bits(c.seed, run, step, (uint32_t)e2, kGenPart, k * kGenBlocks + blk);
                T zz[2];
                gauss2<T>(u01<T>(rb.x), u01<T>(rb.y), zz[0], zz[1]);
                const T ua[2] = {u01<T>(rb.z), u01<T>(rb.w)};
#pragma unroll
                for (int att = 0; att < 2; ++att) {
                    if (got) break;
                    const T xx = xm + zz[att] * (T)0.70710678118654752440;
                    if (xx > (T)0 && ua[att] < (xx / xm) * dexp((T)1 - xx / xm)) { xi = xx; got = true; }
                }
            }
            if (!got) rejects++;
            T x[3] = {(T)0, (T)0, (T)0}, v[3];
            int ci[3] = {0, 0, 0};
            ci[b.axis] = b.side ? c.n[b.axis] - 1 : 0;
            x[b.axis] = b.side ? (T)c.d[b.axis] : (T)0;
            ci[b.t0] = aa;
            x[b.t0] = u01<T>(b0.x) * (T)c.d[b.t0];
            if (b.t1 < DIM) {
                ci[b.t1] = bb;
                x[b.t1] = u01<T>(b0.y) * (T)c.d[b.t1];
            }
            v[b.axis] = (T)b.dir * (T)b.cmp * xi;
            v[b.t0] = (T)b.U[b.t0] + (T)b.sd * z0;
            v[b.t1] = (T)b.U[b.t1] + (T)b.sd * z1;
            const T tau = u01<T>(b0.z) * (T)c.dt;
            uint32_t vmask = 0;
            // wall draws keyed by the entrant's place in the run's step
            // order: after the n_old old particles, in generation order
            const bool alive = move_particle<T, DIM>(c, ci, x, v, n_old + local, run, step, tau, lc,
                                                     vmask);
            const int64_t slot = gen_base + local;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) a.xi[ax][slot] = x[ax];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) a.vi[ax][slot] = v[ax];
            if (a.idi) a.idi[slot] = id0 + local;
            uint32_t key = kDead;
            if (alive) {
                key = rl * (uint32_t)c.ncells + encode_cell<DIM>(c, ci);
                red_add_l2_keep(&a.count[key], 1u);
            }
            a.gc[slot] = key;
        }
        running += total;
        __syncthreads();
    }
    flush_counters(a.ctr, lc);
    if (rejects) atomicAdd(&a.ctr->reject_limit, (unsigned long long)rejects);
    if (overflow) atomicOr(&a.ctr->error, DSMC_ERR_GEN);
    if (threadIdx.x == 0) {
        const uint32_t cap = (uint32_t)a.gcap;
        const uint32_t made = (running < cap ? running : cap) - (prefix < cap ? prefix : cap);
        atomicAdd(&a.ctr->generated, (unsigned long long)made);
        atomicAdd(&a.ctr->particle_steps, (unsigned long long)((grp == 0 ? n_old : 0u) + made));
        if (GG == 1u) {
            a.next_id[rl] = id0 + running;
        } else {
            // the run's last CTA to finish advances its id counter (every
            // CTA of the run has read id0 by then)
            __threadfence();
            if (atomicAdd(&a.gen_done[rl], 1u) == GG - 1u) {
                uint32_t all = 0;
                for (uint32_t g = 0; g < GG; ++g) all += a.gen_tot[(int64_t)rl * GG + g];
                a.next_id[rl] = id0 + all;
                a.gen_done[rl] = 0u;
            }
        }
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_generate(StepArgs<T> a)
{
    pdl_enter();
    generate_block<T, DIM>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// run of a run-major cell key: key / ncells by a 64-bit multiply-high
// (exact for every 32-bit key, see the host's magic number)
template <class C>
__device__ __forceinline__ uint32_t run_of_key(const C& c, uint32_t key)
{
    return c.ncells_magic ? (uint32_t)__umul64hi((unsigned long long)key, c.ncells_magic) : key;
}

// Motion of the pool, straight-flight part: one particle per thread with
// few registers, so that many warps keep their loads in flight.  Each
// particle's run and cell come from its stored cell key.  The new cell's
// count (Enumeration) takes one atomic add per distinct cell of the warp
// (the pool is cell-ordered, so a warp's particles share few cells), with
// no returned value and an L2 evict-last hint on the counters.  A particle
// whose flight may meet a surface is appended to the slow list (one atomic
// per warp) and moved by k_move_slow.
// pool particles before which Motion stops: after a pool overflow (reported
// through the error word) the recorded size can exceed the buffers, so it
// never walks past them
template <typename T>
__device__ __forceinline__ uint32_t move_total(const StepArgs<T>& a)
{
    return min(a.run_base[a.n_runs], (uint32_t)a.cap_old);
}

// four consecutive values from 16-byte aligned p (one vector load, two for
// doubles), and back
__device__ __forceinline__ void ld4(const float* p, float* o)
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double* o)
{
    const double2 v0 = reinterpret_cast<const double2*>(p)[0];
    const double2 v1 = reinterpret_cast<const double2*>(p)[1];
    o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}
__device__ __forceinline__ void st4(float* p, const float* o)
{
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void st4(double* p, const double* o)
{
    reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(o[2], o[3]);
}

// Motion of the slots [s0, s0 + 4), s0 = base + 4 lane, for the warp bases
// base = first + 128 w of this thread's warp w, advancing by `stride` slots
// while below `end` (first a multiple of 4; end <= move_total): four
// particles per thread with their loads issued together (vector loads
// where all four are in range), so that each thread keeps several loads in
// flight.  The cells' counts take one add per run of equal keys in
// consecutive lanes (per position b of the four).
template <typename T, int DIM>
__device__ __forceinline__ void move_span(const StepArgs<T>& a, uint32_t first, uint32_t end,
                                          uint32_t stride)
{
    const Hot<T>& c = a.hot;
    const T dt = c.dt;
    T* __restrict__ xp0 = a.xi[0];
    T* __restrict__ xp1 = a.xi[1];
    T* __restrict__ xp2 = a.xi[2];
    const T* __restrict__ vp0 = a.vi[0];
    const T* __restrict__ vp1 = a.vi[1];
    const T* __restrict__ vp2 = a.vi[2];
    const uint32_t* __restrict__ cip = a.ci_i;
    uint32_t* __restrict__ count = a.count;
    uint32_t* __restrict__ gc = a.gc;
    const uint32_t lane = lane_id();
    const uint32_t below = (1u << lane) - 1u;
    // warp-uniform trip count (the count and slow-list updates are warp
    // operations)
    for (uint32_t base = first; base < end; base += stride) {
        const uint32_t s0 = base + 4u * lane;
        T x0[4], x1[4], x2[4], v0[4], v1[4], v2[4];
        uint32_t kold[4];
        const bool full = s0 + 4u <= end;
        if (full) {
            const uint4 kv = *reinterpret_cast<const uint4*>(cip + s0);
            kold[0] = kv.x; kold[1] = kv.y; kold[2] = kv.z; kold[3] = kv.w;
            ld4(xp0 + s0, x0);
            ld4(xp1 + s0, x1);
            ld4(vp0 + s0, v0);
            ld4(vp1 + s0, v1);
            if (DIM == 3) { ld4(xp2 + s0, x2); ld4(vp2 + s0, v2); }
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const bool in = s0 + b < end;
                kold[b] = in ? cip[s0 + b] : kDead;
                x0[b] = in ? xp0[s0 + b] : (T)0;
                x1[b] = in ? xp1[s0 + b] : (T)0;
                v0[b] = in ? vp0[s0 + b] : (T)0;
                v1[b] = in ? vp1[s0 + b] : (T)0;
                x2[b] = (DIM == 3 && in) ? xp2[s0 + b] : (T)0;
                v2[b] = (DIM == 3 && in) ? vp2[s0 + b] : (T)0;
            }
        }
        uint32_t key[4];
        bool slow[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            key[b] = kDead;   // not counted here (past the end, or slow)
            slow[b] = false;
            if (s0 + b >= end) continue;
            if (kold[b] >= (uint32_t)a.total_cells) {
                // a slot no kernel wrote (possible only after an error already
                // in the error word): dropped, so no counter outside the table
                // moves
                atomicOr(&a.ctr->error, DSMC_ERR_POOL);
                continue;
            }
            T x[3] = {x0[b], x1[b], DIM == 3 ? x2[b] : (T)0};
            const T v[3] = {v0[b], v1[b], DIM == 3 ? v2[b] : (T)0};
            const uint32_t rl = run_of_key(c, kold[b]);
            int ci[3];
            decode_cell<DIM>(c, kold[b] - rl * (uint32_t)c.ncells, ci);
            if (try_free_flight<T, DIM>(c, ci, x, v, dt)) {
                x0[b] = x[0];
                x1[b] = x[1];
                if (DIM == 3) x2[b] = x[2];
                key[b] = rl * (uint32_t)c.ncells + encode_cell<DIM>(c, ci);
            } else {
                slow[b] = true;
            }
        }
        // a slow particle keeps its offsets; k_move_slow moves it and writes
        // its key
        if (full) {
            st4(xp0 + s0, x0);
            st4(xp1 + s0, x1);
            if (DIM == 3) st4(xp2 + s0, x2);
            *reinterpret_cast<uint4*>(gc + s0) = make_uint4(key[0], key[1], key[2], key[3]);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (s0 + b >= end) continue;
                xp0[s0 + b] = x0[b];
                xp1[s0 + b] = x1[b];
                if (DIM == 3) xp2[s0 + b] = x2[b];
                gc[s0 + b] = key[b];
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            uint32_t head, len;
            key_runs(key[b], key[b] != kDead, lane, head, len);
            if (key[b] != kDead && head == lane) red_add_l2_keep(count + key[b], len);
        }
        uint32_t m[4], tot = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            m[b] = __ballot_sync(0xFFFFFFFFu, slow[b]);
            tot += (uint32_t)__popc(m[b]);
        }
        if (tot) {
            uint32_t base_i = 0;
            if (lane == 0) base_i = atomicAdd(&a.ctr->n_slow, tot);
            base_i = __shfl_sync(0xFFFFFFFFu, base_i, 0);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (slow[b]) a.slow_list[base_i + __popc(m[b] & below)] = s0 + b;
                base_i += (uint32_t)__popc(m[b]);
            }
        }
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_move(StepArgs<T> a)
{
    pdl_enter();
    move_span<T, DIM>(a, 4u * (blockIdx.x * blockDim.x + (threadIdx.x & ~31u)), move_total(a),
                      4u * gridDim.x * blockDim.x);
}

// Motion with surface events for the particles k_move set aside.
template <typename T, int DIM>
__device__ __forceinline__ void move_slow_span(const StepArgs<T>& a, uint32_t first, uint32_t stride)
{
    const Cfg& c = *a.cfg;
    const uint32_t n = min(a.ctr->n_slow, (uint32_t)a.cap_old);
    const uint32_t step = a.ctr->step;
    const T dt = (T)c.dt;
    LocalCounters lc;
    for (uint32_t i = first; i < n; i += stride) {
        const uint32_t s = a.slow_list[i];
        const uint32_t kold = a.ci_i[s];
        T x[3], v[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            x[ax] = ax < DIM ? a.xi[ax][s] : (T)0;
            v[ax] = a.vi[ax][s];
        }
        const uint32_t rl = run_of_key(c, kold);
        int ci[3];
        decode_cell<DIM>(c, kold - rl * (uint32_t)c.ncells, ci);
        uint32_t vmask = 0;
        // wall draws keyed by the particle's place in its run's old pool
        const bool alive = move_particle<T, DIM>(c, ci, x, v, s - a.run_base[rl], a.run0 + rl, step,
                                                 dt, lc, vmask);
        uint32_t key = kDead;
        if (alive) {
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) a.xi[ax][s] = x[ax];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
                if (vmask & (1u << ax)) a.vi[ax][s] = v[ax];
            key = rl * (uint32_t)c.ncells + encode_cell<DIM>(c, ci);
            red_add_l2_keep(a.count + key, 1u);
        }
        a.gc[s] = key;
    }
    // every thread reaches this point: the warp reductions are full-warp
    flush_counters(a.ctr, lc);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_move_slow(StepArgs<T> a)
{
    pdl_enter();
    move_slow_span<T, DIM>(a, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// Indexing, part 1: exclusive prefix over the run-major cell counts, in two
// passes.  (a) Each CTA sums the counts of its kScanTile cells; the CTA that
// finishes last (a ticket counter) turns the block sums into their
// exclusive prefix in place, the total after them.  (b) Each CTA scans its
// cells from its block's prefix: each cell's first pool position, and each
// run's first position.
template <typename T>
__device__ __forceinline__ void scan1_block(const StepArgs<T>& a, uint32_t b)
{
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_last;
    const int total = a.total_cells;
    const uint32_t nblocks = (uint32_t)a.scan_blocks;
    const int64_t base = (int64_t)b * kScanTile;
    uint32_t v = 0;
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
        const int64_t i = base + k;
        if (i < total) v += a.count[i];
    }
    v = __reduce_add_sync(0xFFFFFFFFu, v);
    if (lane_id() == 0) s_warp[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t x = threadIdx.x < (blockDim.x >> 5) ? s_warp[threadIdx.x] : 0u;
        x = __reduce_add_sync(0xFFFFFFFFu, x);
        if (threadIdx.x == 0) {
            a.block_sums[b] = x;
            __threadfence();
            s_last = atomicAdd(&a.ctr->scan_ticket, 1u) == nblocks - 1u ? 1u : 0u;
        }
    }
    __syncthreads();
    if (!s_last) return;
    // the last CTA: every other CTA's block sum is visible (its fence came
    // before its ticket); read them past L1
    __threadfence();
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < nblocks; c0 += blockDim.x) {
        const uint32_t i = c0 + threadIdx.x;
        const uint32_t x = i < nblocks ? __ldcg(a.block_sums + i) : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(x, s_warp, tot);
        if (i < nblocks) a.block_sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        a.block_sums[nblocks] = carry;
        a.ctr->scan_ticket = 0u;
    }
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan1(StepArgs<T> a)
{
    pdl_enter();
    scan1_block(a, blockIdx.x);
}

template <typename T>
__device__ __forceinline__ void scan2_block(const StepArgs<T>& a, uint32_t b)
{
    __shared__ uint32_t s_warp[32];
    const int total = a.total_cells;
    const int ncells = a.cfg->ncells;
    const uint32_t nblocks = (uint32_t)a.scan_blocks;
    const uint32_t prefix = __ldcg(a.block_sums + b);
    // each thread: 4 consecutive cells
    const int64_t i0 = (int64_t)b * kScanTile + threadIdx.x * 4;
    uint32_t v[4];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (i0 + k < total) ? a.count[i0 + k] : 0u;
        sum += v[k];
    }
    uint32_t tile_total;
    uint32_t ex = block_exclusive_scan(sum, s_warp, tile_total) + prefix;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = i0 + k;
        if (i < total) {
            a.start[i] = ex;
            if (i % ncells == 0) a.run_base[i / ncells] = ex;
        }
        ex += v[k];
    }
    if (b == nblocks - 1u && threadIdx.x == 0) {
        const uint32_t all = __ldcg(a.block_sums + nblocks);
        a.start[total] = all;
        a.run_base[a.n_runs] = all;
    }
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan2(StepArgs<T> a)
{
    pdl_enter();
    scan2_block(a, blockIdx.x);
}

// the scatter's index space: the old pool's slots [0, n_old), padded to a
// multiple of 128, then the entrants' region [cap_old, cap_old + cap_new).
// The pool holds run_base[n_runs] particles after this step's scan, but
// the slots to scatter are those of the pre-step pool: its size is kept at
// start[total + 1] by the previous step.
template <typename T>
__device__ __forceinline__ uint64_t scatter_extent(const StepArgs<T>& a, uint64_t* n_old_out,
                                                   uint64_t* pad_out)
{
    const uint64_t n_old = min((uint64_t)a.start[a.total_cells + 1], (uint64_t)a.cap_old);
    const uint64_t pad = (n_old + 127) / 128 * 128;
    *n_old_out = n_old;
    *pad_out = pad;
    return pad + (uint64_t)a.cap_new;
}

// Indexing, part 2: LCR[start[cell] + r] = slot for every live particle, r
// taken from the cell's count, which Motion left at the cell's particle
// count and which this pass counts back down to zero (ready for the next
// step's Motion): one atomic subtract per run of equal keys in consecutive
// lanes, the run's lanes taking consecutive places below the returned
// value.  The order inside a cell is any: the next kernel puts each cell in
// slot order (the order one serial pass over the pool would give).
// Indices v0 .. v0 + 3, v0 = base + 4 lane, for the warp bases base = first
// + 128 w, advancing by `stride` while below `end`; all four slots' loads
// and count updates are issued before their results are used.
__device__ __forceinline__ uint32_t atomic_sub_l2_keep(uint32_t* p, uint32_t v)
{
    return atomic_add_l2_keep(p, 0u - v);
}

template <typename T>
__device__ __forceinline__ void scatter_span(const StepArgs<T>& a, uint64_t first, uint64_t end,
                                             uint64_t stride)
{
    uint64_t n_old, pad;
    scatter_extent(a, &n_old, &pad);
    uint32_t* __restrict__ gc = a.gc;
    uint32_t* __restrict__ count = a.count;
    const uint32_t* __restrict__ start = a.start;
    uint32_t* __restrict__ lcr = a.lcr;
    bool overflow = false;
    const uint32_t lane = lane_id();
    // warp-uniform trip count (the count updates are warp operations)
    for (uint64_t base = first; base < end; base += stride) {
        uint32_t key[4], st[4];
        uint64_t slot[4];
        // index v0 + b -> slot; v0 is a multiple of 4 and so is the padded
        // old-pool size, so the four lie in one region
        const uint64_t v0 = base + 4u * lane;
        const uint64_t s0 = v0 < pad ? v0 : (uint64_t)a.cap_old + (v0 - pad);
        const uint64_t lim = v0 < pad ? n_old : (uint64_t)a.cap_old + (uint64_t)a.cap_new;
        if (v0 + 4 <= end && s0 + 4 <= lim) {
            const uint4 kv = *reinterpret_cast<const uint4*>(gc + s0);
            key[0] = kv.x; key[1] = kv.y; key[2] = kv.z; key[3] = kv.w;
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const bool in = v0 + b < end && s0 + b < lim;
                key[b] = in ? gc[s0 + b] : kDead;
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) slot[b] = s0 + b;
#pragma unroll
        for (int b = 0; b < 4; ++b) st[b] = key[b] != kDead ? ld_l2_keep(start + key[b]) : 0u;
        uint32_t head[4], old[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            uint32_t len;
            key_runs(key[b], key[b] != kDead, lane, head[b], len);
            old[b] = 0u;
            if (key[b] != kDead && head[b] == lane) old[b] = atomic_sub_l2_keep(count + key[b], len);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t o = __shfl_sync(0xFFFFFFFFu, old[b], head[b]);
            if (key[b] == kDead) continue;
            if (slot[b] >= (uint64_t)a.cap_old) gc[slot[b]] = kDead;   // re-kill the entrant's key
            const uint32_t rk = o - 1u - (lane - head[b]);
            const uint64_t pos = (uint64_t)st[b] + rk;
            if (pos >= (uint64_t)a.cap_old || rk >= 0x80000000u) { overflow = true; continue; }
            lcr[pos] = (uint32_t)slot[b];
        }
    }
    if (overflow) atomicOr(&a.ctr->error, DSMC_ERR_POOL);
}

template <typename T>
__global__ void __launch_bounds__(256) k_scatter(StepArgs<T> a)
{
    pdl_enter();
    uint64_t n_old, pad;
    const uint64_t nv = scatter_extent(a, &n_old, &pad);
    scatter_span(a, 4ull * ((uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)), nv,
                 4ull * gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// a Philox draw through the configuration the caller holds: the Cfg
// computes the key schedule, the launch-parameter constants carry it
__device__ __forceinline__ uint4 draw_c(const Cfg& c, uint32_t run, uint32_t step, uint32_t entity,
                                        uint32_t purpose, uint32_t sub)
{
    return draw_bits(c.seed, run, step, entity, purpose, sub);
}
template <typename T>
__device__ __forceinline__ uint4 draw_c(const Hot<T>& c, uint32_t run, uint32_t step,
                                        uint32_t entity, uint32_t purpose, uint32_t sub)
{
    return philox_rk(make_uint4(entity, (purpose << 28) | (sub & 0x0FFFFFFFu), step, run), c.rk);
}

// (sigma_T c_r) of a pair with relative speed squared g2 (and speed g)
template <typename T, class C>
__device__ __forceinline__ T sigma_cr(const C& c, T g, T g2)
{
    if (c.hs) return (T)c.A_hs * g;
    if (g2 == (T)0) return (T)0;
    return (T)c.K_vhs * dpow(g2, (T)c.one_m_omega);
}

// NTC candidate count of a cell with N particles, M = floor(x) with
// x = (1/2) N (N-1) F_N dt / V_c (sigma c_r)_max + rem; the fractional
// remainder rem = x - M is carried across steps in FP64 and N < 2 leaves it
// unchanged.  With FP32 state the product is formed in binary32 (FP32
// collision arithmetic) and only the remainder carry is FP64; with FP64
// state every operation is FP64.
template <typename T, class C>
__device__ __forceinline__ int64_t ntc_count(const C& c, uint32_t N, T smax, double& rem)
{
    if (N < 2) return 0;
    double x;
    if (sizeof(T) == 4) {
        const float p = (0.5f * (float)(N * (N - 1u))) * c.coef_f * (float)smax;
        x = (double)p + rem;
    } else {
        const double nn = (double)N * (double)(N - 1u);
        x = 0.5 * nn * c.coef * (double)smax + rem;
    }
    const double M = floor(x);
    rem = x - M;
    return (int64_t)M;
}

// index floor(u * n) of a uniform u = (m + 1/2) / 2^23, computed exactly
__device__ __forceinline__ uint32_t pick(uint32_t bits, uint32_t n)
{
    const uint64_t m2 = 2ull * (uint64_t)(bits >> 9) + 1ull;
    return (uint32_t)((m2 * (uint64_t)n) >> 24);
}

// Positions of one cell's particles in the next pool (offsets inside the
// cell, LCR order); x[2] is read in 3-D only.
template <typename T>
struct CellPos {
    const T* x[3];
};

// the subcell index along axis a of offset f: floor(n_sub f / d), clamped
// to the cell
template <typename T, class C>
__device__ __forceinline__ uint32_t subcell_axis(const C& c, int a, T f)
{
    const int ns = c.n_sub;
    int k = (int)dfloor(in_cells(c, a, f) * (T)ns);
    k = k < 0 ? 0 : (k > ns - 1 ? ns - 1 : k);
    return (uint32_t)k;
}

// the subcell of particle m from its offsets, axis 0 fastest (positions are
// read-only while the cells collide; the axes are spelt out so that the
// position pointers stay in registers)
template <typename T, class C>
__device__ __forceinline__ uint32_t subcell_of(const C& c, const CellPos<T>& p, uint32_t m)
{
    const uint32_t ns = (uint32_t)c.n_sub;
    uint32_t s = c.dim == 3 ? subcell_axis<T>(c, 2, __ldg(p.x[2] + m)) : 0u;
    s = s * ns + subcell_axis<T>(c, 1, __ldg(p.x[1] + m));
    return s * ns + subcell_axis<T>(c, 0, __ldg(p.x[0] + m));
}

// The second particle of an NTC candidate whose first is i, among the N of
// the cell, by the gas model's choice of partner (the Interaction step of
// Sec. 1.1 leaves the pair selection to the gas model): uniform over the other
// N - 1 (the r-th other in LCR order, r from `bits`); uniform over the other
// particles of i's subcell, or the uniform rule if i is alone there; the
// nearest other particle (squared distance summed over the grid's axes in
// axis order; the first of equal distances).  The cell's positions are read
// from global memory (read-only path), one pass per choice (two for a
// subcell draw); the passes select without branches so that the loads of
// consecutive particles overlap.
template <typename T, class C>
__device__ __forceinline__ uint32_t pick_partner(const C& c, const CellPos<T>& p, uint32_t N,
                                                 uint32_t i, uint32_t bits)
{
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    if (c.partner == DSMC_PARTNER_NEAREST) {
        const T* x0 = p.x[0];
        const T* x1 = p.x[1];
        const T a0 = __ldg(x0 + i), a1 = __ldg(x1 + i);
        T best = (T)0;
        uint32_t j = kNone;
        if (c.dim == 3) {
            const T* x2 = p.x[2];
            const T a2 = __ldg(x2 + i);
#pragma unroll 4
            for (uint32_t m = 0; m < N; ++m) {
                const T e0 = __ldg(x0 + m) - a0;
                const T e1 = __ldg(x1 + m) - a1;
                const T e2 = __ldg(x2 + m) - a2;
                T dd = e0 * e0;
                dd = dd + e1 * e1;
                dd = dd + e2 * e2;
                const bool take = m != i && (j == kNone || dd < best);
                best = take ? dd : best;
                j = take ? m : j;
            }
        } else {
#pragma unroll 4
            for (uint32_t m = 0; m < N; ++m) {
                const T e0 = __ldg(x0 + m) - a0;
                const T e1 = __ldg(x1 + m) - a1;
                T dd = e0 * e0;
                dd = dd + e1 * e1;
                const bool take = m != i && (j == kNone || dd < best);
                best = take ? dd : best;
                j = take ? m : j;
            }
        }
        return j;
    }
    if (c.partner == DSMC_PARTNER_SUBCELL) {
        const uint32_t si = subcell_of<T>(c, p, i);
        uint32_t K = 0;
#pragma unroll 4
        for (uint32_t m = 0; m < N; ++m) K += (m != i && subcell_of<T>(c, p, m) == si) ? 1u : 0u;
        if (K > 0u) {
            const uint32_t r = pick(bits, K);
            uint32_t seen = 0, j = kNone;
#pragma unroll 4
            for (uint32_t m = 0; m < N; ++m) {
                const bool mate = m != i && subcell_of<T>(c, p, m) == si;
                j = (mate && seen == r) ? m : j;
                seen += mate ? 1u : 0u;
            }
            return j;
        }
    }
    uint32_t j = pick(bits, N - 1u);
    if (j >= i) j += 1u;
    return j;
}

// NTC acceptance u < sigma c_r / (sigma c_r)_max: FP64 state divides, as the
// oracle does; FP32 state compares u (sigma c_r)_max < sigma c_r (no
// division; FP32 collision arithmetic)
template <typename T>
__device__ __forceinline__ bool ntc_accept(T u, T sc, T smax) { return u < sc / smax; }
template <>
__device__ __forceinline__ bool ntc_accept<float>(float u, float sc, float smax) { return u * smax < sc; }

// (cos eps, sin eps) of the azimuth eps = 2 pi u (sincospi, accurate in
// both precisions: the azimuth's rounding stays at the working precision's
// unit roundoff, relative to the pair's relative speed)
template <typename T>
__device__ __forceinline__ void azimuth(T u, T* s, T* c) { dsincospi((T)2.0 * u, s, c); }

// one accepted collision: isotropic scattering of the relative velocity
template <typename T>
__device__ __forceinline__ void scatter_pair(T* v1, T* v2, T g, T u3, T ueps)
{
    const T cosx = (T)2.0 * u3 - (T)1.0;
    // sin(chi) = sqrt(1 - cos^2 chi) = 2 sqrt(u3 (1 - u3)): the second form
    // has no cancellation when cos(chi) is near +-1 (u3 and 1 - u3 are exact)
    const T sinx = (T)2.0 * dsqrt(u3 * ((T)1.0 - u3));
    T se, ce;
    azimuth<T>(ueps, &se, &ce);
    const T gr[3] = {g * cosx, g * sinx * ce, g * sinx * se};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const T cm = (T)0.5 * (v1[ax] + v2[ax]);
        v1[ax] = cm + (T)0.5 * gr[ax];
        v2[ax] = cm - (T)0.5 * gr[ax];
    }
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// The draws of NTC candidate k of a cell with N particles: the pair (i, j),
// the acceptance uniform, cos(chi) and the azimuth uniform.  POS: the
// partner j is chosen by pick_partner from the cell's positions xp.
template <bool POS, typename T, class C>
__device__ __forceinline__ void candidate_draws(const C& c, uint32_t run, uint32_t step,
                                                uint32_t cell, int64_t k, uint32_t N,
                                                const CellPos<T>& xp, uint32_t& ci, uint32_t& cj,
                                                T& u2, T& u3, T& ue)
{
    const uint4 r = draw_c(c, run, step, cell, kColl, (uint32_t)(2 * k));
    const uint4 r2 = draw_c(c, run, step, cell, kColl, (uint32_t)(2 * k + 1));
    ci = pick(r.x, N);
    if constexpr (POS) {
        cj = pick_partner<T>(c, xp, N, ci, r.y);
    } else {
        cj = pick(r.y, N - 1u);
        if (cj >= ci) cj += 1u;
    }
    u2 = u01<T>(r.z);
    u3 = u01<T>(r.w);
    ue = u01<T>(r2.x);
}

// One NTC candidate pair (i, j): accept with probability
// sigma_T c_r / (sigma_T c_r)_max, then scatter isotropically; `azimuth_u()`
// gives the azimuth uniform and is called only for an accepted pair.  Every
// cell path uses this arithmetic, so results do not depend on the path.
template <typename T, class C, class AZ>
__device__ __forceinline__ void collide_pair(const C& c, T* sv0, T* sv1, T* sv2, uint32_t i,
                                             uint32_t j, T u2, T u3, AZ azimuth_u, T smax, T& seen,
                                             uint32_t& nacc, uint32_t& nclamp)
{
    T v1[3] = {sv0[i], sv1[i], sv2[i]};
    T v2[3] = {sv0[j], sv1[j], sv2[j]};
    const T gx = v1[0] - v2[0], gy = v1[1] - v2[1], gz = v1[2] - v2[2];
    const T g2 = gx * gx + gy * gy + gz * gz;
    const T g = dsqrt(g2);
    const T sc = sigma_cr<T>(c, g, g2);
    if (sc > seen) seen = sc;
    if (sc > smax) nclamp++;
    if (ntc_accept<T>(u2, sc, smax)) {
        scatter_pair<T>(v1, v2, g, u3, azimuth_u());
        sv0[i] = v1[0]; sv1[i] = v1[1]; sv2[i] = v1[2];
        sv0[j] = v2[0]; sv1[j] = v2[1]; sv2[j] = v2[2];
        nacc++;
    }
}

// the same with all draws made beforehand
template <typename T, class C>
__device__ __forceinline__ void collide_candidate(const C& c, T* sv0, T* sv1, T* sv2, uint32_t i,
                                                  uint32_t j, T u2, T u3, T ue, T smax, T& seen,
                                                  uint32_t& nacc, uint32_t& nclamp)
{
    collide_pair<T>(c, sv0, sv1, sv2, i, j, u2, u3, [&]() { return ue; }, smax, seen, nacc, nclamp);
}

// Interaction of one large cell, velocities in LCR order at sv0..sv2 (shared
// or global memory); all lanes of the warp call it.  The lanes draw 32
// candidates at a time; a candidate is applied as soon as no earlier
// candidate of the batch that shares one of its particles is still pending,
// so candidates with disjoint pairs are applied side by side, and every
// particle still sees its collisions in candidate order: the result equals
// applying the candidates one after another.  On return every lane holds
// the warp's totals.
template <bool POS, typename T, class C>
__device__ void collide_cell_warp(const C& c, T* sv0, T* sv1, T* sv2, const CellPos<T>& xp,
                                  uint32_t N, int64_t M, T smax, uint32_t cell, uint32_t run,
                                  uint32_t step, T& seen, uint32_t& nacc, uint32_t& nclamp)
{
    const uint32_t lane = lane_id();
    T my_seen = (T)0;
    uint32_t my_acc = 0, my_clamp = 0;
    for (int64_t kb = 0; kb < M; kb += 32) {
        const int64_t k = kb + lane;
        uint32_t ci = 0xFFFFFFFFu, cj = 0xFFFFFFFEu;
        T u2 = (T)1, u3 = (T)0, ue = (T)0;
        if (k < M) candidate_draws<POS, T>(c, run, step, cell, k, N, xp, ci, cj, u2, u3, ue);
        uint32_t pending = __ballot_sync(0xFFFFFFFFu, k < M);
        while (pending) {
            bool blocked = false;
#pragma unroll 4
            for (uint32_t q = 0; q < 31u; ++q) {
                const uint32_t qi = __shfl_sync(0xFFFFFFFFu, ci, q);
                const uint32_t qj = __shfl_sync(0xFFFFFFFFu, cj, q);
                if (q < lane && ((pending >> q) & 1u) &&
                    (qi == ci || qi == cj || qj == ci || qj == cj))
                    blocked = true;
            }
            const bool go = ((pending >> lane) & 1u) && !blocked;
            if (go) collide_candidate<T>(c, sv0, sv1, sv2, ci, cj, u2, u3, ue, smax, my_seen, my_acc,
                                         my_clamp);
            __syncwarp();
            pending &= ~__ballot_sync(0xFFFFFFFFu, go);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T other = __shfl_xor_sync(0xFFFFFFFFu, my_seen, o);
        my_seen = other > my_seen ? other : my_seen;
    }
    seen = my_seen;
    nacc = __reduce_add_sync(0xFFFFFFFFu, my_acc);
    nclamp = __reduce_add_sync(0xFFFFFFFFu, my_clamp);
}

// Sampling of one cell: N, sum v_a, sum v_a^2 in FP64, summed in LCR order
// (one fixed order for every path and launch shape).
template <typename T>
__device__ __forceinline__ void cell_moments(const T* sv0, const T* sv1, const T* sv2, uint32_t N,
                                             double* m)
{
    for (int q = 0; q < DSMC_NMOM; ++q) m[q] = 0.0;
    for (uint32_t r = 0; r < N; ++r) {
        const double v0 = (double)sv0[r], v1 = (double)sv1[r], v2 = (double)sv2[r];
        m[0] += 1.0;
        m[1] += v0; m[2] += v1; m[3] += v2;
        m[4] += v0 * v0; m[5] += v1 * v1; m[6] += v2 * v2;
    }
}

// A slot read back from the LCR; anything outside the pool (possible only
// after an overflow already flagged in the error word) is replaced by slot 0
// and flagged, so no access leaves the buffers.
template <typename T>
__device__ __forceinline__ uint32_t checked_slot(const StepArgs<T>& a, uint32_t s)
{
    if ((int64_t)s >= a.cap_old + a.cap_new) {
        atomicOr(&a.ctr->error, DSMC_ERR_POOL);
        return 0u;
    }
    return s;
}

// Entry (sj, j) of a cell's readdressing range comes before (sk, k): slots
// are unique, the position only breaks ties in a state already flagged as
// corrupted, so the ranks always form a permutation.
__device__ __forceinline__ bool slot_before(uint32_t sj, uint32_t j, uint32_t sk, uint32_t k)
{
    return sj < sk || (sj == sk && j < k);
}

struct CellTally {
    unsigned long long cand = 0, acc = 0, clamp = 0;
};

// A cell of more than kWarpMax particles is handled whole (sort, gather,
// collisions, moments) by the big-cell kernel.
template <typename T>
__device__ __forceinline__ void push_big(const StepArgs<T>& a, int64_t gcell)
{
    const uint32_t idx = atomicAdd(&a.ctr->n_big, 1u);
    if (idx < a.max_big) a.big_list[idx] = (uint32_t)gcell;
    else atomicOr(&a.ctr->error, DSMC_ERR_BIGLIST);
}

// Warp path for one cell of up to kWarpMax particles: slot ranks by
// counting, then the particles gathered into the next pool in slot order.
// Used for tiles whose start table is inconsistent (a corrupt state): it
// checks every cell.  `ws` is this warp's scratch: kWarpMax x (u32 + u16).
template <typename T, int DIM>
__device__ void cell_warp_path(const StepArgs<T>& a, const Cfg& c, int64_t gcell, unsigned char* ws)
{
    const uint32_t lane = lane_id();
    uint32_t* sl = reinterpret_cast<uint32_t*>(ws);
    uint16_t* sp = reinterpret_cast<uint16_t*>(sl + kWarpMax);
    const uint32_t beg = a.start[gcell];
    const uint32_t N = a.start[gcell + 1] - beg;
    if ((uint64_t)beg + N > (uint64_t)a.cap_old) {
        if (lane == 0) atomicOr(&a.ctr->error, DSMC_ERR_POOL);
        return;
    }
    if (N > (uint32_t)kWarpMax) {
        if (lane == 0) push_big(a, gcell);
        return;
    }
    for (uint32_t k = lane; k < N; k += 32) sl[k] = checked_slot(a, a.lcr[beg + k]);
    __syncwarp();
    for (uint32_t k = lane; k < N; k += 32) {
        const uint32_t my = sl[k];
        uint32_t r = 0;
        for (uint32_t j = 0; j < N; ++j) r += slot_before(sl[j], j, my, k) ? 1u : 0u;
        sp[r] = (uint16_t)k;
    }
    __syncwarp();
    for (uint32_t r = lane; r < N; r += 32) {
        const uint32_t k = sp[r];
        const uint32_t s = sl[k];
        const uint32_t o = beg + r;
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) a.xo[ax][o] = a.xi[ax][s];
        a.ci_o[o] = (uint32_t)gcell;
        if (a.ido) a.ido[o] = a.idi[s];
        a.vo[0][o] = a.vi[0][s];
        a.vo[1][o] = a.vi[1][s];
        a.vo[2][o] = a.vi[2][s];
        if (a.lcr_dbg) a.lcr_dbg[o] = s;
    }
    __syncwarp();
}

template <typename T>
__host__ __device__ constexpr size_t warp_scratch_bytes()
{
    return (size_t)kWarpMax * (sizeof(uint32_t) + sizeof(uint16_t));
}

constexpr int kGatherBatch = 3;   // positions per thread and pass of the gather (measured: 2 and 4 slower)

// Indexing, part 3 (sort and gather).  One CTA takes kTileCells consecutive
// (run-major) cells, whose particles occupy one contiguous range of the next
// pool and of the LCR.  (1) Thread 0 starts a bulk copy (TMA) of the tile's
// LCR entries (old slots) into shared memory while each thread tags its
// cell's positions.  (2) Thread per position, kGatherBatch positions per
// pass: the particle's rank inside its cell by counting smaller slots, and
// its offsets and velocity (and its id, in debug mode) gathered from the old
// pool into the next pool at cell start + rank.  Cells above kWarpMax go to the one-CTA-per-cell
// kernel; a tile whose particles exceed the budget is taken in consecutive
// cell ranges that fit it.
// shared memory of the sort/gather tile kernel: the tile's start table, its
// LCR entries (eight spare for the 16-byte aligned superset) and cell tags
struct CellSmem {
    uint32_t* s_start;
    uint32_t* s_lcr;
    uint16_t* s_cellof;
    unsigned char* raw;
    uint64_t* bar;
};

__device__ __forceinline__ CellSmem cell_smem(unsigned char* raw, uint64_t* bar, uint32_t budget)
{
    CellSmem m;
    m.raw = raw;
    m.bar = bar;
    m.s_start = reinterpret_cast<uint32_t*>(raw);
    m.s_lcr = reinterpret_cast<uint32_t*>(raw + (kTileCells + 4) * sizeof(uint32_t));
    m.s_cellof = reinterpret_cast<uint16_t*>(m.s_lcr + budget + 8);
    return m;
}

// One tile of kTileCells cells (every thread of the CTA calls it; the
// mbarrier's phase is carried across calls).
template <typename T, int DIM>
__device__ __forceinline__ void cell_tile(const StepArgs<T>& a, int64_t tile, const CellSmem& sm,
                                          uint32_t& phase)
{
    const Cfg& c = *a.cfg;
    const uint32_t budget = (uint32_t)a.tile_budget;
    uint32_t* s_start = sm.s_start;
    uint32_t* s_lcr = sm.s_lcr;
    uint16_t* s_cellof = sm.s_cellof;
    unsigned char* smem_raw = sm.raw;
    uint64_t& s_bar = *sm.bar;
    const int tid = threadIdx.x;
    const int64_t c0 = tile * kTileCells;
    const int nct = (int)min((int64_t)kTileCells, (int64_t)a.total_cells - c0);
    for (int i = tid; i <= kTileCells; i += blockDim.x) s_start[i] = a.start[c0 + min(i, nct)];
    __syncthreads();
    const uint32_t B = s_start[0], E = s_start[nct];
    if (E < B || (uint64_t)E > (uint64_t)a.cap_old) {
        // an inconsistent start table (a state already flagged corrupt):
        // cell by cell through the warp path, which checks every cell
        unsigned char* ws = smem_raw + (kTileCells + 4) * sizeof(uint32_t) +
                            (size_t)(tid >> 5) * warp_scratch_bytes<T>();
        for (int q = tid >> 5; q < nct; q += kTileCells / 32)
            cell_warp_path<T, DIM>(a, c, c0 + q, ws);
        __syncthreads();
        return;
    }
    // the tile's cells in consecutive ranges [q0, q1) of at most `budget`
    // particles, one range when the whole tile fits; a range of one cell
    // above the budget (a cell above kWarpMax) is only listed for the
    // big-cell kernel
    int q0 = 0;
    while (q0 < nct) {
        const uint32_t Bq = s_start[q0];
        int q1 = nct;
        if (E - Bq > budget) {
            q1 = q0 + __syncthreads_count(tid >= q0 && tid < nct && s_start[tid + 1] - Bq <= budget);
            if (q1 == q0) {
                if (tid == q0) push_big(a, c0 + q0);
                q0 += 1;
                continue;
            }
        }
        const uint32_t Eq = s_start[q1];
        const uint32_t Tn = Eq - Bq;
        if (Eq < Bq || Tn > budget) {
            // not a nondecreasing start table: flagged, the rest skipped
            if (tid == 0) atomicOr(&a.ctr->error, DSMC_ERR_POOL);
            __syncthreads();   // every thread has read the table
            break;
        }
        // [lo, hi): the 16-byte aligned superset of [Bq, Eq); the LCR
        // holds cap_old entries, a multiple of 4, so hi stays inside it
        const uint32_t lo = Bq & ~3u;
        const uint32_t sh = Bq - lo;
        if (tid == 0 && Tn > 0) {
            const uint32_t hi = (Eq + 3u) & ~3u;
            const uint32_t bytes = (hi - lo) * (uint32_t)sizeof(uint32_t);
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar, bytes);
            bulk_g2s(s_lcr, a.lcr + lo, bytes, &s_bar);
        }
        if (tid >= q0 && tid < q1) {
            const uint32_t cb = s_start[tid] - Bq, ce = s_start[tid + 1] - Bq;
            const bool big = ce - cb > (uint32_t)kWarpMax;
            if (big) push_big(a, c0 + tid);
            const uint16_t mark = big ? (uint16_t)0xFFFF : (uint16_t)tid;
            for (uint32_t k = cb; k < ce; ++k) s_cellof[k] = mark;
        }
        if (Tn > 0) {
            if (!mbar_wait(&s_bar, phase)) {
                atomicOr(&a.ctr->error, DSMC_ERR_TIMEOUT);
                mbar_wait(&s_bar, phase);
            }
            phase ^= 1u;
        }
        __syncthreads();
        const uint32_t* tl = s_lcr + sh;
        for (uint32_t k0 = tid; k0 < Tn; k0 += kGatherBatch * kTileCells) {
            // kGatherBatch particles per pass, every load issued before any store
            uint32_t kk[kGatherBatch], sl[kGatherBatch], pid[kGatherBatch];
            int lo2[kGatherBatch];
            T px[kGatherBatch][3], pv[kGatherBatch][3];
#pragma unroll
            for (int b = 0; b < kGatherBatch; ++b) {
                kk[b] = k0 + (uint32_t)b * kTileCells;
                lo2[b] = kk[b] < Tn ? (int)s_cellof[kk[b]] : 0xFFFF;
                sl[b] = lo2[b] != 0xFFFF ? checked_slot(a, tl[kk[b]]) : 0u;
            }
#pragma unroll
            for (int b = 0; b < kGatherBatch; ++b) {
                if (lo2[b] == 0xFFFF) continue;
#pragma unroll
                for (int ax = 0; ax < DIM; ++ax) px[b][ax] = a.xi[ax][sl[b]];
                pv[b][0] = a.vi[0][sl[b]];
                pv[b][1] = a.vi[1][sl[b]];
                pv[b][2] = a.vi[2][sl[b]];
                if (a.ido) pid[b] = a.idi[sl[b]];
            }
#pragma unroll
            for (int b = 0; b < kGatherBatch; ++b) {
                if (lo2[b] == 0xFFFF) continue;
                const uint32_t cb = s_start[lo2[b]] - Bq, ce = s_start[lo2[b] + 1] - Bq;
                const uint32_t my = tl[kk[b]];
                // slots are unique; a repeated one (possible only in a state
                // already flagged corrupt) leaves a hole, never an access
                // outside the cell's range
                uint32_t r = 0;
                for (uint32_t j = cb; j < ce; ++j) r += tl[j] < my ? 1u : 0u;
                const uint32_t o = Bq + cb + r;
#pragma unroll
                for (int ax = 0; ax < DIM; ++ax) a.xo[ax][o] = px[b][ax];
                a.ci_o[o] = (uint32_t)(c0 + lo2[b]);
                if (a.ido) a.ido[o] = pid[b];
                a.vo[0][o] = pv[b][0];
                a.vo[1][o] = pv[b][1];
                a.vo[2][o] = pv[b][2];
                if (a.lcr_dbg) a.lcr_dbg[o] = sl[b];
            }
        }
        __syncthreads();
        q0 = q1;
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kTileCells, 4) k_cell(StepArgs<T> a)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    const CellSmem sm = cell_smem(smem_raw, &s_bar, (uint32_t)a.tile_budget);
    if (threadIdx.x == 0) mbar_init(&s_bar, 1u);
    uint32_t phase = 0;
    const int64_t ntiles = ((int64_t)a.total_cells + kTileCells - 1) / kTileCells;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        cell_tile<T, DIM>(a, tile, sm, phase);
}

// Interaction and Sampling: cells of at most kWarpMax particles (larger
// cells are done whole by the big-cell kernels), on the cells' velocities
// in the next pool, now in LCR order.  A CTA takes kCollideCells consecutive
// cells.  (1) Thread 0 starts bulk copies (TMA) of the tile's velocities,
// up to collide_stage particles, into shared memory; meanwhile every thread
// forms its cell's NTC candidate count (coalesced remainder and (sigma
// c_r)_max accesses) and the staged range is cut to whole cells.  (2) The
// cells are handed to the threads grouped by candidate count (a 32-bin
// counting sort), so that the cells of one warp run similar numbers of
// candidates.  (3) Each thread collides its cell -- in shared memory if
// staged, else in place in global memory, with the same arithmetic.  (4)
// The cells' moments at sample steps; the staged velocities are stored back
// with coalesced stores.  The kernel waits on memory and on the slowest
// cell of each tile, so it is sized for CTAs in flight: a stage of 18
// particles a cell lets 7 CTAs share an SM.  (Measured slower: handing each
// thread the next cell of a list in decreasing candidate order as it
// finishes -- a tile has about one cell per thread, so nothing is left to
// balance; two or four cells per thread in snake order over the candidate
// order, and 64-cell tiles -- fewer warps in flight.)
//
// A thread's candidates of one cell, one after another.  The pair draw of
// candidate k + 1 is made while candidate k is applied (it depends on no
// velocity), which gives the thread two independent chains of work; the
// azimuth draw is made only for an accepted pair.  The draws are those of
// candidate_draws.
template <bool POS, typename T, class C>
__device__ __forceinline__ void collide_cell_run(const C& c, T* v0, T* v1, T* v2,
                                                 const CellPos<T>& xp, uint32_t run, uint32_t step,
                                                 uint32_t cell, uint32_t M, uint32_t N, T smax,
                                                 T& seen, uint32_t& nacc, uint32_t& nclamp)
{
    if (M == 0u) return;
    uint4 r = draw_c(c, run, step, cell, kColl, 0u);
    for (uint32_t k = 0; k < M; ++k) {
        // the next candidate's pair draw (the last one draws its own again)
        const uint32_t kn = k + 1u < M ? k + 1u : k;
        const uint4 rn = draw_c(c, run, step, cell, kColl, 2u * kn);
        const uint32_t i = pick(r.x, N);
        uint32_t j;
        if constexpr (POS) {
            j = pick_partner<T>(c, xp, N, i, r.y);
        } else {
            j = pick(r.y, N - 1u);
            if (j >= i) j += 1u;
        }
        collide_pair<T>(c, v0, v1, v2, i, j, u01<T>(r.z), u01<T>(r.w), [&]() {
            return u01<T>(draw_c(c, run, step, cell, kColl, 2u * k + 1u).x);
        }, smax, seen, nacc, nclamp);
        r = rn;
    }
}

// the staged velocities of a collision CTA: three components of `stage` + 8
// elements each (the 16-byte aligned superset of the tile's range)
__host__ __device__ constexpr int collide_stage_pitch(int stage) { return stage + 8; }

// resident CTAs of the collision kernel per SM that its registers must
// allow: a binary32 stage of 18-19 particles a cell (28 KB) fits 7 on an
// SM's 228 KB, a binary64 one 3.  The kernel waits on memory and on its
// slowest cell per tile, so CTAs in flight matter more than registers: 7
// CTAs of 128 threads (at most 73 registers) measured 12% faster than 6
// (85) on the duct ensemble.
// (The multi-part kernel, which also holds its part's arguments, is
// bounded for one CTA fewer: its default stage, for filled grids, lets 6
// share an SM.)
template <typename T>
__host__ __device__ constexpr int collide_min_blocks() { return sizeof(T) == 4 ? 7 : 3; }

// shared memory of the collision kernel: the staged velocities (three
// components, collide_stage + 8 each) and the mbarrier of their bulk copies
template <typename T>
struct CollideSmem {
    T* s0;
    T* s1;
    T* s2;
    uint64_t* bar;
};

// One tile of kCollideCells cells (every thread of the CTA calls it; the
// mbarrier's phase and the thread's tallies are carried across calls).  Each
// of the kCollideThreads threads takes kCollidePerThread cells: for the
// per-cell steps, cells tid, tid + kCollideThreads, ...; for the collisions,
// positions of the tile's ascending candidate order taken in snake order
// (tid, 2 kCollideThreads - 1 - tid, ...), so that a thread's light cells
// offset its heavy ones.  POS: collision partners are chosen by position
// (pick_partner), read from the next pool.
template <typename T, bool POS>
__device__ __forceinline__ void collide_tile(const StepArgs<T>& a, int64_t tile,
                                             const CollideSmem<T>& sm, uint32_t& phase,
                                             CellTally& tl)
{
    constexpr uint32_t kVec = 16u / sizeof(T);   // elements per 16 bytes
    constexpr int CPT = kCollidePerThread;
    constexpr uint32_t TH = (uint32_t)kCollideThreads;
    T* s0 = sm.s0;
    T* s1 = sm.s1;
    T* s2 = sm.s2;
    uint64_t& s_bar = *sm.bar;
    __shared__ uint32_t s_b0, s_n, s_nload, s_sh;
    __shared__ uint32_t s_bin[32];
    __shared__ uint32_t s_beg[kCollideCells], s_N[kCollideCells], s_M[kCollideCells];
    __shared__ uint32_t s_ord[kCollideCells];
    __shared__ T s_smax[kCollideCells];
    const Hot<T>& c = a.hot;
    const uint32_t step = a.ctr->step;
    const int slot_t = step < (uint32_t)a.n_slot ? a.sample_slot[step] : -1;
    const uint32_t tid = threadIdx.x;
    constexpr uint32_t kOff = 0xFFFFFFFFu;   // s_N of a cell this kernel skips
    const int64_t c0 = tile * kCollideCells;
    const int64_t rest = a.total_cells - c0;
    const uint32_t nc = rest < kCollideCells ? (uint32_t)rest : (uint32_t)kCollideCells;
    uint32_t beg[CPT], N[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
        const uint32_t q = tid + (uint32_t)u * TH;
        beg[u] = 0;
        N[u] = 0;
        if (q < nc) {
            beg[u] = a.start[c0 + q];
            N[u] = a.start[c0 + q + 1] - beg[u];
        }
    }
    if (tid == 0) {
        // the tile's particles [b, end), clipped to the stage and the pool
        // (cell 0 of the tile is thread 0's first cell)
        const uint32_t b = beg[0];
        const uint32_t end = a.start[c0 + nc];
        const int64_t room = a.cap_old - (int64_t)b;
        int64_t n = end > b ? (int64_t)(end - b) : 0;
        if (n > a.collide_stage) n = a.collide_stage;
        if (n > room) n = room > 0 ? room : 0;
        s_b0 = b;
        s_n = (uint32_t)n;
        s_nload = (uint32_t)n;
        if (n > 0) {
            // 16-byte aligned superset [lo, hi) of [b, b + n); hi stays
            // inside the pool, whose capacity is a multiple of 256
            const uint32_t lo = b & ~(kVec - 1u);
            const uint32_t hi = (b + (uint32_t)n + kVec - 1u) & ~(kVec - 1u);
            const uint32_t bytes = (hi - lo) * (uint32_t)sizeof(T);
            s_sh = b - lo;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar, 3u * bytes);
            bulk_g2s(s0, a.vo[0] + lo, bytes, &s_bar);
            bulk_g2s(s1, a.vo[1] + lo, bytes, &s_bar);
            bulk_g2s(s2, a.vo[2] + lo, bytes, &s_bar);
        }
    }
    if (tid < 32) s_bin[tid] = 0u;
    __syncthreads();
    const uint32_t b0 = s_b0;
    const uint32_t nload = s_nload;
    uint32_t bin[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
        const uint32_t q = tid + (uint32_t)u * TH;
        const int64_t gcell = c0 + q;
        const bool mine = q < nc;
        // cut the staged range at the first cell that does not fit whole
        if (mine) {
            const uint32_t rel = beg[u] - b0;
            const uint64_t end = (uint64_t)rel + N[u];
            if (beg[u] < b0) atomicMin(&s_n, 0u);
            else if (rel < nload && end > (uint64_t)nload) atomicMin(&s_n, rel);
        }
        // NTC candidate count of the cell; the remainder is final
        const bool act = mine && N[u] <= (uint32_t)kWarpMax &&
                         (uint64_t)beg[u] + N[u] <= (uint64_t)a.cap_old;
        uint32_t M32 = 0;
        if (act) {
            double rem = a.rem[gcell];
            const T smax = a.smax[gcell];
            const int64_t M = ntc_count<T>(c, N[u], smax, rem);
            if (N[u] >= 2) a.rem[gcell] = rem;
            M32 = M > (int64_t)0x7FFFFFFF ? 0x7FFFFFFFu : (uint32_t)M;
            s_smax[q] = smax;
            if (a.cand && M32 == 0u) { a.cand[gcell] = 0u; a.accd[gcell] = 0u; }
        }
        s_beg[q] = beg[u];
        s_N[q] = act ? N[u] : kOff;
        s_M[q] = M32;
        bin[u] = M32 < 31u ? M32 : 31u;
    }
    __syncthreads();
    const uint32_t n_st = s_n;
    const uint32_t sh = s_sh;
    // (2) the cells in ascending candidate count (32 bins), so that the
    // lanes of a warp run similar numbers of candidates
    uint32_t in_bin[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) in_bin[u] = atomicAdd(&s_bin[bin[u]], 1u);
    __syncthreads();
    if (tid < 32) {
        const uint32_t v = s_bin[tid];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (tid >= (uint32_t)o) x += y;
        }
        s_bin[tid] = x - v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < CPT; ++u) s_ord[s_bin[bin[u]] + in_bin[u]] = tid + (uint32_t)u * TH;
    if (nload > 0) {
        if (!mbar_wait(&s_bar, phase)) {
            atomicOr(&a.ctr->error, DSMC_ERR_TIMEOUT);
            mbar_wait(&s_bar, phase);
        }
        phase ^= 1u;
    }
    __syncthreads();
    // (3) the candidates of the thread's cells, in shared memory if staged,
    // else in place in global memory (the same arithmetic)
#pragma unroll 1
    for (int u = 0; u < CPT; ++u) {
        const uint32_t pos = (u & 1) ? ((uint32_t)u + 1u) * TH - 1u - tid : (uint32_t)u * TH + tid;
        const uint32_t q = s_ord[pos];
        const uint32_t Nq = s_N[q];
        if (Nq != kOff && s_M[q] > 0u) {
            const int64_t gq = c0 + q;
            const uint32_t begq = s_beg[q];
            const uint32_t Mq = s_M[q];
            const T smax = s_smax[q];
            const uint32_t rl = run_of_key(c, (uint32_t)gq);
            const uint32_t cell = (uint32_t)gq - rl * (uint32_t)c.ncells;
            const bool stq = begq >= b0 && (uint64_t)(begq - b0) + Nq <= (uint64_t)n_st;
            T seen = (T)0;
            uint32_t nacc = 0, nclamp = 0;
            const uint32_t o = sh + (begq - b0);
            CellPos<T> xp{};
            if constexpr (POS) {
                for (int ax = 0; ax < 3; ++ax) xp.x[ax] = a.xo[ax] ? a.xo[ax] + begq : nullptr;
            }
            // one call per address space, so that staged cells use
            // shared-memory loads and stores
            if (stq)
                collide_cell_run<POS, T>(c, s0 + o, s1 + o, s2 + o, xp, a.run0 + rl, step, cell, Mq,
                                         Nq, smax, seen, nacc, nclamp);
            else
                collide_cell_run<POS, T>(c, a.vo[0] + begq, a.vo[1] + begq, a.vo[2] + begq, xp,
                                         a.run0 + rl, step, cell, Mq, Nq, smax, seen, nacc, nclamp);
            if (seen > smax) a.smax[gq] = seen;
            if (a.cand) { a.cand[gq] = Mq; a.accd[gq] = nacc; }
            tl.cand += Mq;
            tl.acc += nacc;
            tl.clamp += nclamp;
        }
    }
    __syncthreads();
    // (4) moments at sample steps, thread per cell
    if (slot_t >= 0) {
#pragma unroll 1
        for (int u = 0; u < CPT; ++u) {
            const uint32_t q = tid + (uint32_t)u * TH;
            const uint32_t Nq = s_N[q];
            if (Nq == kOff) continue;
            const int64_t gcell = c0 + q;
            const bool staged = beg[u] >= b0 && (uint64_t)(beg[u] - b0) + Nq <= (uint64_t)n_st;
            const uint32_t o = sh + (beg[u] - b0);
            double m[DSMC_NMOM];
            if (staged) cell_moments<T>(s0 + o, s1 + o, s2 + o, Nq, m);
            else cell_moments<T>(a.vo[0] + beg[u], a.vo[1] + beg[u], a.vo[2] + beg[u], Nq, m);
            double* mo = a.mom + gcell * DSMC_NMOM;
            if (slot_t & kSlotFirst)
                for (int qq = 0; qq < DSMC_NMOM; ++qq) mo[qq] = m[qq];
            else
                for (int qq = 0; qq < DSMC_NMOM; ++qq) mo[qq] += m[qq];
        }
    }
    {
        T* g0 = a.vo[0] + b0;
        T* g1 = a.vo[1] + b0;
        T* g2 = a.vo[2] + b0;
        for (uint32_t p = tid; p < n_st; p += TH) {
            g0[p] = s0[sh + p];
            g1[p] = s1[sh + p];
            g2[p] = s2[sh + p];
        }
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void flush_tally(Counters* ctr, const CellTally& tl)
{
    const unsigned long long cs = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)tl.cand);
    const unsigned long long as = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)tl.acc);
    const unsigned long long ks = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)tl.clamp);
    if (lane_id() == 0) {
        if (cs) atomicAdd(&ctr->candidates, cs);
        if (as) atomicAdd(&ctr->collisions, as);
        if (ks) atomicAdd(&ctr->clamps, ks);
    }
}

template <typename T, bool POS>
__global__ void __launch_bounds__(kCollideThreads, collide_min_blocks<T>()) k_collide(StepArgs<T> a)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    const int pitch = collide_stage_pitch(a.collide_stage);
    CollideSmem<T> sm;
    sm.s0 = reinterpret_cast<T*>(smem_raw);
    sm.s1 = sm.s0 + pitch;
    sm.s2 = sm.s1 + pitch;
    sm.bar = &s_bar;
    if (threadIdx.x == 0) mbar_init(&s_bar, 1u);
    uint32_t phase = 0;
    CellTally tl;
    const int64_t ntiles = (a.total_cells + kCollideCells - 1) / kCollideCells;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        collide_tile<T, POS>(a, tile, sm, phase, tl);
    flush_tally<T>(a.ctr, tl);
}

// ---------------------------------------------------------------------------
// Cells above kWarpMax particles, part 1: each cell's particles put in slot
// order and gathered into the next pool.  The order comes from an LSD radix
// sort of compact slot keys (order_cell), 8 bits a pass (as many passes as
// the keys' span needs, at most 4), on 16-bit positions into the cell's
// keys staged in shared memory.  Each pass is a stable counting sort:
// warp w ranks the chunks of its contiguous range in order (match_any
// groups equal digits; the group's first lane advances the warp's count of
// that digit), an exclusive scan of the counts in (digit, warp) order gives
// each (digit, warp) its first destination, and every position moves there
// plus its rank.  Stable passes make every result a permutation.  A CTA of
// kBigThreads takes the cells above kBigThreads particles one at a time,
// then splits into groups of kMidThreads (named barriers) that take the
// smaller ones, a cell per group.
constexpr int kBigThreads = 1024;
constexpr int kMidThreads = 256;
constexpr int kMidGroups = kBigThreads / kMidThreads;
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;

template <typename T>
__host__ __device__ constexpr int big_max_of() { return 8192; }

// shared memory of order_cell for THREADS threads and cells up to KMAX
// particles: sort keys (u32), slots (u32), two position buffers (u16), the
// (digit, warp) counts (u16; one 16-byte word per thread)
template <int THREADS, int KMAX>
__host__ __device__ constexpr size_t order_smem()
{
    return (size_t)KMAX * (4 + 4 + 2 + 2) + (size_t)kRadixBins * (THREADS / 32) * sizeof(uint16_t);
}

__host__ __device__ constexpr size_t big_smem_bytes()
{
    return order_smem<kBigThreads, big_max_of<float>()>() >
                   kMidGroups * order_smem<kMidThreads, kBigThreads>()
               ? order_smem<kBigThreads, big_max_of<float>()>()
               : kMidGroups * order_smem<kMidThreads, kBigThreads>();
}

// barrier of the THREADS threads that order one cell: the whole CTA, or a
// named barrier of one group
template <int THREADS>
__device__ __forceinline__ void order_sync(uint32_t bar)
{
    if (THREADS == kBigThreads) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(THREADS) : "memory");
}

template <typename T, int DIM>
__device__ __forceinline__ void big_put(const StepArgs<T>& a, uint32_t o, uint32_t s, uint32_t gcell)
{
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) a.xo[ax][o] = a.xi[ax][s];
    a.ci_o[o] = gcell;
    if (a.ido) a.ido[o] = a.idi[s];
    a.vo[0][o] = a.vi[0][s];
    a.vo[1][o] = a.vi[1][s];
    a.vo[2][o] = a.vi[2][s];
    if (a.lcr_dbg) a.lcr_dbg[o] = s;
}

// One cell of N particles (KMAX / 8 < N <= KMAX) put in slot order and
// gathered by THREADS threads (t = 0 .. THREADS - 1, barrier `bar`) on `sm`
// (order_smem bytes, 16-byte aligned) and `red` (4 x THREADS / 32 words).
// Every thread of the group calls it with the same cell.  The radix sort
// runs on a compact key of the slot: the old pool's slots relative to their
// smallest, then the entrants' slots (one run's, in their own region)
// relative to theirs, after the old ones -- the same order as the slots,
// with a span of about the cell's source range rather than the pool's.
template <int THREADS, int KMAX, typename T, int DIM>
__device__ __forceinline__ void order_cell(const StepArgs<T>& a, uint32_t gcell, uint32_t beg,
                                           uint32_t N, unsigned char* sm, uint32_t* red, uint32_t t,
                                           uint32_t bar)
{
    constexpr uint32_t W = THREADS / 32;
    static_assert(KMAX <= 8 * THREADS, "at most 8 chunks of 32 per warp (8-bit ranks)");
    static_assert(kRadixBins * W * sizeof(uint16_t) == THREADS * 16,
                  "one 16-byte word of counts per thread");
    uint32_t* s_key = reinterpret_cast<uint32_t*>(sm);
    uint32_t* s_slot = s_key + KMAX;
    uint16_t* pa = reinterpret_cast<uint16_t*>(s_slot + KMAX);
    uint16_t* pb = pa + KMAX;
    uint16_t* cnt = pb + KMAX;   // [digit][warp]
    const uint32_t lane = t & 31u, w = t >> 5;
    const uint32_t cap = (uint32_t)a.cap_old;
    // smallest and largest slot among the old pool's and among the entrants'
    uint32_t lo_o = 0xFFFFFFFFu, hi_o = 0u, lo_n = 0xFFFFFFFFu, hi_n = 0u;
    for (uint32_t k = t; k < N; k += THREADS) {
        const uint32_t sl = checked_slot(a, a.lcr[beg + k]);
        s_slot[k] = sl;
        pa[k] = (uint16_t)k;
        if (sl < cap) { lo_o = min(lo_o, sl); hi_o = max(hi_o, sl); }
        else { lo_n = min(lo_n, sl); hi_n = max(hi_n, sl); }
    }
    lo_o = __reduce_min_sync(0xFFFFFFFFu, lo_o);
    hi_o = __reduce_max_sync(0xFFFFFFFFu, hi_o);
    lo_n = __reduce_min_sync(0xFFFFFFFFu, lo_n);
    hi_n = __reduce_max_sync(0xFFFFFFFFu, hi_n);
    if (lane == 0) { red[w] = lo_o; red[W + w] = hi_o; red[2 * W + w] = lo_n; red[3 * W + w] = hi_n; }
    order_sync<THREADS>(bar);
    lo_o = __reduce_min_sync(0xFFFFFFFFu, lane < W ? red[lane] : 0xFFFFFFFFu);
    hi_o = __reduce_max_sync(0xFFFFFFFFu, lane < W ? red[W + lane] : 0u);
    lo_n = __reduce_min_sync(0xFFFFFFFFu, lane < W ? red[2 * W + lane] : 0xFFFFFFFFu);
    hi_n = __reduce_max_sync(0xFFFFFFFFu, lane < W ? red[3 * W + lane] : 0u);
    const bool any_old = lo_o <= hi_o, any_new = lo_n <= hi_n;
    const uint32_t base_n = any_old ? hi_o - lo_o + 1u : 0u;
    // each thread keys the positions it loaded
    for (uint32_t k = t; k < N; k += THREADS) {
        const uint32_t sl = s_slot[k];
        s_key[k] = sl < cap ? sl - lo_o : base_n + (sl - lo_n);
    }
    const uint32_t span = any_new ? base_n + (hi_n - lo_n) : (any_old ? hi_o - lo_o : 0u);
    const int passes = span == 0u ? 0 : (32 - __clz(span) + kRadixBits - 1) / kRadixBits;
    // warp w owns positions [w * C * 32, (w + 1) * C * 32), C <= 8
    const uint32_t C = (N + THREADS - 1) / THREADS;
    const uint32_t wbase = w * C * 32u;
    const uint32_t below = (1u << lane) - 1u;
    for (int p = 0; p < passes; ++p) {
        const int sh = p * kRadixBits;
        order_sync<THREADS>(bar);   // the previous pass's reads of cnt, pa and red done
        reinterpret_cast<uint4*>(cnt)[t] = make_uint4(0u, 0u, 0u, 0u);
        order_sync<THREADS>(bar);
        // (1) rank of each position among the equal digits of its warp range
        uint32_t rk0 = 0u, rk1 = 0u;
#pragma unroll
        for (uint32_t c = 0; c < 8u; ++c) {
            if (c < C) {
                const uint32_t e = wbase + c * 32u + lane;
                const bool ok = e < N;
                const uint32_t d = ok ? (s_key[pa[e]] >> sh) & (kRadixBins - 1u)
                                      : (uint32_t)kRadixBins;
                const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
                const uint32_t before = ok ? (uint32_t)cnt[d * W + w] : 0u;
                const uint32_t r = before + __popc(peers & below);
                __syncwarp();
                if (ok && (peers & below) == 0u) cnt[d * W + w] = (uint16_t)(before + __popc(peers));
                __syncwarp();
                if (c < 4u) rk0 |= r << (8u * c);
                else rk1 |= r << (8u * (c - 4u));
            }
        }
        order_sync<THREADS>(bar);
        // (2) exclusive scan of the counts in (digit, warp) order: eight
        // consecutive counts per thread, then across the threads
        uint4 q = reinterpret_cast<const uint4*>(cnt)[t];
        uint32_t v[8] = {q.x & 0xFFFFu, q.x >> 16, q.y & 0xFFFFu, q.y >> 16,
                         q.z & 0xFFFFu, q.z >> 16, q.w & 0xFFFFu, q.w >> 16};
        uint32_t tot = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) tot += v[i];
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31u) red[w] = x;
        order_sync<THREADS>(bar);
        if (w == 0) {
            const uint32_t ws = lane < W ? red[lane] : 0u;
            uint32_t z = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
                if (lane >= (uint32_t)o) z += y;
            }
            if (lane < W) red[W + lane] = z - ws;
        }
        order_sync<THREADS>(bar);
        uint32_t run = red[W + w] + x - tot;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t u = v[i];
            v[i] = run;
            run += u;
        }
        q.x = v[0] | (v[1] << 16);
        q.y = v[2] | (v[3] << 16);
        q.z = v[4] | (v[5] << 16);
        q.w = v[6] | (v[7] << 16);
        reinterpret_cast<uint4*>(cnt)[t] = q;
        order_sync<THREADS>(bar);
        // (3) every position to its (digit, warp) start plus its rank
#pragma unroll
        for (uint32_t c = 0; c < 8u; ++c) {
            if (c < C) {
                const uint32_t e = wbase + c * 32u + lane;
                if (e < N) {
                    const uint32_t pe = pa[e];
                    const uint32_t d = (s_key[pe] >> sh) & (kRadixBins - 1u);
                    const uint32_t r = (c < 4u ? rk0 >> (8u * c) : rk1 >> (8u * (c - 4u))) & 0xFFu;
                    pb[cnt[d * W + w] + r] = (uint16_t)pe;
                }
            }
        }
        uint16_t* sw = pa;
        pa = pb;
        pb = sw;
    }
    order_sync<THREADS>(bar);
    for (uint32_t r = t; r < N; r += THREADS) {
        const uint32_t pe = pa[r];
        big_put<T, DIM>(a, beg + r, s_slot[pe], gcell);
    }
    order_sync<THREADS>(bar);   // buffers free for the group's next cell
}

// the big cells of one problem, CTA `blk` of `nblk` (every thread of the
// CTA calls it)
template <typename T, int DIM>
__device__ __forceinline__ void cell_big_part(const StepArgs<T>& a, uint32_t blk, uint32_t nblk,
                                              unsigned char* smem_raw, uint32_t* s_red)
{
    constexpr int kMax = big_max_of<T>();
    const uint32_t tid = threadIdx.x;
    const uint32_t nb = a.ctr->n_big < a.max_big ? a.ctr->n_big : (uint32_t)a.max_big;
    // (1) cells above kBigThreads particles: the whole CTA per cell
    for (uint32_t bi = blk; bi < nb; bi += nblk) {
        const uint32_t gcell = a.big_list[bi];
        const uint32_t beg = a.start[gcell];
        const uint32_t N = a.start[gcell + 1] - beg;
        if (N <= (uint32_t)kBigThreads) continue;
        if ((uint64_t)beg + N > (uint64_t)a.cap_old) {
            if (tid == 0) atomicOr(&a.ctr->error, DSMC_ERR_POOL);
            continue;
        }
        if (tid == 0) atomicAdd(&a.ctr->big_pool_steps, (unsigned long long)N);
        if (N > (uint32_t)kMax) {
            // over the per-cell limit: reported, and the particles are still
            // carried into the next pool (in LCR order), so that the next
            // step reads no unwritten slot
            if (tid == 0) atomicOr(&a.ctr->error, DSMC_ERR_BIGCELL);
            for (uint32_t r = tid; r < N; r += blockDim.x) {
                big_put<T, DIM>(a, beg + r, checked_slot(a, a.lcr[beg + r]), gcell);
            }
            continue;
        }
        order_cell<kBigThreads, kMax, T, DIM>(a, gcell, beg, N, smem_raw, s_red, tid, 0u);
    }
    __syncthreads();
    // (2) cells of kWarpMax + 1 .. kBigThreads particles: a group of
    // kMidThreads per cell, kMidGroups groups side by side
    const uint32_t g = tid / kMidThreads, tg = tid % kMidThreads;
    unsigned char* sm = smem_raw + (size_t)g * order_smem<kMidThreads, kBigThreads>();
    uint32_t* red = s_red + g * 4 * (kMidThreads / 32);
    for (uint32_t bi = blk * kMidGroups + g; bi < nb; bi += nblk * kMidGroups) {
        const uint32_t gcell = a.big_list[bi];
        const uint32_t beg = a.start[gcell];
        const uint32_t N = a.start[gcell + 1] - beg;
        if (N > (uint32_t)kBigThreads) continue;
        if ((uint64_t)beg + N > (uint64_t)a.cap_old) {
            if (tg == 0) atomicOr(&a.ctr->error, DSMC_ERR_POOL);
            continue;
        }
        if (tg == 0) atomicAdd(&a.ctr->big_pool_steps, (unsigned long long)N);
        order_cell<kMidThreads, kBigThreads, T, DIM>(a, gcell, beg, N, sm, red, tg, 1u + g);
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kBigThreads, 2) k_cell_big(StepArgs<T> a)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_red[4 * (kBigThreads / 32)];
    cell_big_part<T, DIM>(a, blockIdx.x, gridDim.x, smem_raw, s_red);
}

// Cells above kWarpMax particles, part 2: one warp per cell, on the cell's
// velocities in the next pool (LCR order): NTC count, candidates applied by
// collide_cell_warp (disjoint pairs side by side, in-order result), and the
// cell's moments at sample steps.  Many large cells proceed at once.
// the big cells of one problem, warp `wid` of `warps` (POS: partners chosen
// by position)
template <typename T, bool POS>
__device__ __forceinline__ void collide_big_part(const StepArgs<T>& a, uint32_t wid, uint32_t warps)
{
    const Cfg& c = *a.cfg;
    constexpr int kMax = big_max_of<T>();
    const uint32_t step = a.ctr->step;
    const int slot_t = step < (uint32_t)a.n_slot ? a.sample_slot[step] : -1;
    const uint32_t nb = a.ctr->n_big < a.max_big ? a.ctr->n_big : (uint32_t)a.max_big;
    const uint32_t lane = lane_id();
    for (uint32_t bi = wid; bi < nb; bi += warps) {
        const uint32_t gcell = a.big_list[bi];
        const uint32_t beg = a.start[gcell];
        const uint32_t N = a.start[gcell + 1] - beg;
        if ((uint64_t)beg + N > (uint64_t)a.cap_old || N > (uint32_t)kMax) continue;   // flagged
        const uint32_t rl = gcell / (uint32_t)c.ncells;
        const uint32_t cell = gcell - rl * (uint32_t)c.ncells;
        double rem = a.rem[gcell];
        const T smax = a.smax[gcell];
        const int64_t M = ntc_count<T>(c, N, smax, rem);
        T* v0 = a.vo[0] + beg;
        T* v1 = a.vo[1] + beg;
        T* v2 = a.vo[2] + beg;
        T seen = (T)0;
        uint32_t nacc = 0, nclamp = 0;
        CellPos<T> xp{};
        if constexpr (POS) {
            for (int ax = 0; ax < 3; ++ax) xp.x[ax] = a.xo[ax] ? a.xo[ax] + beg : nullptr;
        }
        if (M > 0)
            collide_cell_warp<POS, T>(c, v0, v1, v2, xp, N, M, smax, cell, a.run0 + rl, step, seen,
                                      nacc, nclamp);
        if (lane == 0) {
            a.rem[gcell] = rem;
            if (seen > smax) a.smax[gcell] = seen;
            if (a.cand) { a.cand[gcell] = (uint32_t)M; a.accd[gcell] = nacc; }
            if (M) atomicAdd(&a.ctr->candidates, (unsigned long long)M);
            if (nacc) atomicAdd(&a.ctr->collisions, (unsigned long long)nacc);
            if (nclamp) atomicAdd(&a.ctr->clamps, (unsigned long long)nclamp);
        }
        __syncwarp();
        if (slot_t >= 0 && lane == 0) {
            double m[DSMC_NMOM];
            cell_moments<T>(v0, v1, v2, N, m);
            double* mo = a.mom + (uint64_t)gcell * DSMC_NMOM;
            if (slot_t & kSlotFirst)
                for (int q = 0; q < DSMC_NMOM; ++q) mo[q] = m[q];
            else
                for (int q = 0; q < DSMC_NMOM; ++q) mo[q] += m[q];
        }
    }
}

template <typename T, bool POS>
__global__ void __launch_bounds__(256) k_collide_big(StepArgs<T> a)
{
    pdl_enter();
    collide_big_part<T, POS>(a, blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                             gridDim.x * (blockDim.x >> 5));
}

// ---------------------------------------------------------------------------
// Sampling over runs, at the last step of a sample window: acc[k][g] +=
// sum of the launch's runs of group g (each run's sums over the window's
// steps), in increasing run order (the same order in batched and plain
// modes).
template <typename T>
__device__ __forceinline__ void reduce_part(const StepArgs<T>& a, int64_t first, int64_t stride)
{
    const uint32_t step = a.ctr->step;
    const int slot_v = step < (uint32_t)a.n_slot ? a.sample_slot[step] : -1;
    if (slot_v < 0 || !(slot_v & kSlotLast)) return;
    const int slot_t = slot_v & kSlotIndex;
    const int ncells = a.cfg->ncells;
    const int64_t per = (int64_t)ncells * DSMC_NMOM;
    const int64_t n = (int64_t)a.G * per;
    for (int64_t i = first; i < n; i += stride) {
        const int g = (int)(i / per);
        const int64_t ck = i - (int64_t)g * per;
        double* dst = a.acc + ((int64_t)slot_t * a.G + g) * per + ck;
        double s = *dst;
        // first local run r with (run0 + r) mod G == g
        int r = ((g - a.run0 % a.G) % a.G + a.G) % a.G;
        for (; r < a.n_runs; r += a.G) s += a.mom[(int64_t)r * per + ck];
        *dst = s;
    }
}

template <typename T>
__global__ void k_reduce(StepArgs<T> a)
{
    pdl_enter();
    reduce_part(a, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

template <typename T>
__device__ __forceinline__ void step_end_part(const StepArgs<T>& a)
{
    a.ctr->step += 1u;
    a.ctr->n_big = 0u;
    a.ctr->n_slow = 0u;
    a.ctr->pool_steps += (unsigned long long)min(a.run_base[a.n_runs], (uint32_t)a.cap_old);
    // remember this step's pool size for the next scatter (the slot range of
    // the old pool): start[total + 1] = run_base[n_runs]
    a.start[a.total_cells + 1] = a.run_base[a.n_runs];
}

template <typename T>
__global__ void k_step_end(StepArgs<T> a)
{
    pdl_enter();
    step_end_part(a);
}

// Consistency check of the pool after a run (options.checks): every pool
// position p holds a particle whose stored cell key lies inside the table,
// whose cell's range [start[key], start[key + 1]) contains p, whose id (when
// ids are kept) is below its run's next id (ids are handed out in order),
// whose offsets lie
// inside its cell and whose velocity is finite.  Counts the positions that
// fail and keeps the first.
template <typename T, int DIM>
__global__ void k_check(StepArgs<T> a)
{
    const uint32_t n = min(a.run_base[a.n_runs], (uint32_t)a.cap_old);
    const T* x[3] = {a.xi[0], a.xi[1], a.xi[2]};
    uint32_t bad = 0, first = 0xFFFFFFFFu;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint32_t key = a.ci_i[p];
        bool ok = key < (uint32_t)a.total_cells;
        if (ok) {
            const uint32_t cs = a.start[key], ce = a.start[key + 1];
            ok = cs <= p && p < ce;
            if (ok && a.idi) ok = a.idi[p] < a.next_id[run_of_key(a.hot, key)];
        }
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) {
            const T f = x[ax][p];
            const T d = a.hot.d[ax];
            ok = ok && f >= (T)0 && f <= d * (T)(1.0 + 1e-6);
        }
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) ok = ok && isfinite(a.vi[ax][p]);
        if (!ok) {
            ++bad;
            first = min(first, p);
        }
    }
    if (bad) {
        atomicAdd(&a.ctr->check_fail, bad);
        atomicMin(&a.ctr->check_first, first);
    }
}

// moments of the current pool (test hook), one warp per cell
template <typename T>
__global__ void k_sample_now(StepArgs<T> a, const T* v0, const T* v1, const T* v2)
{
    const uint32_t lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t gcell = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
         gcell < a.total_cells; gcell += warps) {
        const uint32_t beg = a.start[gcell];
        const uint32_t end = min(a.start[gcell + 1], (uint32_t)a.cap_old);
        const uint32_t N = end > beg ? end - beg : 0u;
        double m[DSMC_NMOM] = {0, 0, 0, 0, 0, 0, 0};
        for (uint32_t r = lane; r < N; r += 32) {
            const double x0 = v0[beg + r], x1 = v1[beg + r], x2 = v2[beg + r];
            m[0] += 1.0; m[1] += x0; m[2] += x1; m[3] += x2;
            m[4] += x0 * x0; m[5] += x1 * x1; m[6] += x2 * x2;
        }
#pragma unroll
        for (int q = 0; q < DSMC_NMOM; ++q) m[q] = warp_sum(m[q]);
        if (lane == 0)
            for (int q = 0; q < DSMC_NMOM; ++q) a.mom[gcell * DSMC_NMOM + q] = m[q];
    }
}

// macroscopic quantities of sample t from the group sums; out[cell][10] =
// n, u, v, w, T, se_n, se_u, se_v, se_w, se_T
template <typename T>
__global__ void k_macro(StepArgs<T> a, int t, int n_runs, int window, double* out)
{
    const Cfg& c = *a.cfg;
    const int ncells = c.ncells;
    const int G = a.G;
    const double kB = 1.380649e-23;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < ncells;
         cell += gridDim.x * blockDim.x) {
        double pooled[DSMC_NMOM] = {0, 0, 0, 0, 0, 0, 0};
        double est[DSMC_MAX_GROUPS][5];
        for (int g = 0; g < G; ++g) {
            const double* s = a.acc + (((int64_t)t * G + g) * ncells + cell) * DSMC_NMOM;
            for (int q = 0; q < DSMC_NMOM; ++q) pooled[q] += s[q];
            // (run, step) pairs of group g: its runs times the window's steps
            const double nr = (double)((n_runs - g + G - 1) / G) * (double)window;
            const double N = s[0];
            est[g][0] = N * c.F_N / (nr * c.Vc);
            const double vx = s[1] / N, vy = s[2] / N, vz = s[3] / N;
            est[g][1] = vx; est[g][2] = vy; est[g][3] = vz;
            est[g][4] = c.mass / (3.0 * kB) * ((s[4] + s[5] + s[6]) / N - (vx * vx + vy * vy + vz * vz));
        }
        double* o = out + (int64_t)cell * 10;
        const double N = pooled[0];
        const double vx = pooled[1] / N, vy = pooled[2] / N, vz = pooled[3] / N;
        o[0] = N * c.F_N / ((double)n_runs * (double)window * c.Vc);
        o[1] = vx; o[2] = vy; o[3] = vz;
        o[4] = c.mass / (3.0 * kB) * ((pooled[4] + pooled[5] + pooled[6]) / N - (vx * vx + vy * vy + vz * vz));
        for (int q = 0; q < 5; ++q) {
            int m = 0;
            double mean = 0.0;
            for (int g = 0; g < G; ++g)
                if (est[g][q] == est[g][q]) { mean += est[g][q]; ++m; }
            if (m < 2) { o[5 + q] = __longlong_as_double(0x7FF8000000000000ll); continue; }
            mean /= m;
            double ss = 0.0;
            for (int g = 0; g < G; ++g)
                if (est[g][q] == est[g][q]) ss += (est[g][q] - mean) * (est[g][q] - mean);
            o[5 + q] = sqrt(ss / (m - 1)) / sqrt((double)G);
        }
    }
}

#if !defined(DSMC_KERNELS_FP64)
__global__ void k_philox(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = philox(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]),
                               make_uint2(key[2 * i], key[2 * i + 1]));
        out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
    }
}
#endif

// ---------------------------------------------------------------------------
// Several problems per launch (the parts of a mixed-size ensemble).  Every
// kernel below runs the bodies of the single-problem kernels above on each
// part's StepArgs, copied into shared memory when a CTA turns to that part.
// The tile-shaped work -- Motion chunks, scatter chunks, sort/gather tiles,
// collision tiles -- is claimed from a device work-queue counter per kernel
// kind: a CTA takes the next item (part, tile) as soon as it has finished
// its previous one, so CTAs move between the parts' runs as the load
// requires, the way the paper's dynamic scheme hands processors that have
// finished their share to runs with work left (Sec. 3).  The other kernels
// map CTAs to (part, block) statically or loop over the parts.

// part p with base[p] <= i < base[p + 1] (base[0] = 0, nondecreasing)
__device__ __forceinline__ int part_of(const int32_t* base, int n, int64_t i)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)base[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// the CTA's copy of part p's StepArgs (every thread calls it)
template <typename T>
__device__ __forceinline__ void load_part(StepArgs<T>& dst, const StepArgs<T>* parts, int p)
{
    static_assert(sizeof(StepArgs<T>) % 4 == 0, "StepArgs copied in 4-byte words");
    __syncthreads();   // every thread is done with the previous part
    const uint32_t* src = reinterpret_cast<const uint32_t*>(parts + p);
    uint32_t* d = reinterpret_cast<uint32_t*>(&dst);
    for (uint32_t i = threadIdx.x; i < sizeof(StepArgs<T>) / 4; i += blockDim.x) d[i] = src[i];
    __syncthreads();
}

// The work-queue loop of one CTA: item ids from *q until `total`; the next
// claim is issued while the current item is processed, and broadcast
// through two alternating shared words.
template <class F>
__device__ __forceinline__ void claim_items(uint32_t* q, uint32_t total, F&& f)
{
    __shared__ uint32_t s_item[2];
    if (threadIdx.x == 0) s_item[0] = atomicAdd(q, 1u);
    __syncthreads();
    uint32_t buf = 0, item = s_item[0];
    while (item < total) {
        uint32_t nxt = 0;
        if (threadIdx.x == 0) nxt = atomicAdd(q, 1u);
        f(item);
        if (threadIdx.x == 0) s_item[buf ^ 1u] = nxt;
        __syncthreads();
        buf ^= 1u;
        item = s_item[buf];
    }
}

// per-part item counts of a queue-driven kernel with a device-side size,
// as a prefix table in shared memory (thread p counts part p)
template <class F>
__device__ __forceinline__ void item_prefix(int n_parts, int32_t* base, F&& count_of)
{
    if (threadIdx.x < (uint32_t)n_parts) base[threadIdx.x + 1] = (int32_t)count_of((int)threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        base[0] = 0;
        for (int p = 0; p < n_parts; ++p) base[p + 1] += base[p];
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) mk_gen_count(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    const int p = part_of(m.gcount_base, m.n_parts, blockIdx.x);
    load_part(sa, m.parts, p);
    gen_count_block(sa, blockIdx.x - (uint32_t)m.gcount_base[p]);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) mk_generate(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    const int p = part_of(m.gen_base, m.n_parts, blockIdx.x);
    load_part(sa, m.parts, p);
    generate_block<T, DIM>(sa, blockIdx.x - (uint32_t)m.gen_base[p]);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) mk_move(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    __shared__ int32_t s_base[kMaxParts + 1];
    item_prefix(m.n_parts, s_base, [&](int p) {
        return (move_total(m.parts[p]) + kMoveChunk - 1) / kMoveChunk;
    });
    int cur = -1;
    claim_items(m.queue + kQMove, (uint32_t)s_base[m.n_parts], [&](uint32_t item) {
        const int p = part_of(s_base, m.n_parts, item);
        if (p != cur) { load_part(sa, m.parts, p); cur = p; }
        const uint32_t first = (item - (uint32_t)s_base[p]) * kMoveChunk;
        const uint32_t end = min(first + kMoveChunk, move_total(sa));
        move_span<T, DIM>(sa, first + 4u * (threadIdx.x & ~31u), end, 4u * blockDim.x);
    });
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) mk_move_slow(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    for (int p = 0; p < m.n_parts; ++p) {
        load_part(sa, m.parts, p);
        move_slow_span<T, DIM>(sa, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
    }
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) mk_scan1(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    const int p = part_of(m.scan_base, m.n_parts, blockIdx.x);
    load_part(sa, m.parts, p);
    scan1_block(sa, blockIdx.x - (uint32_t)m.scan_base[p]);
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) mk_scan2(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    const int p = part_of(m.scan_base, m.n_parts, blockIdx.x);
    load_part(sa, m.parts, p);
    scan2_block(sa, blockIdx.x - (uint32_t)m.scan_base[p]);
}

template <typename T>
__global__ void __launch_bounds__(256) mk_scatter(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    __shared__ int32_t s_base[kMaxParts + 1];
    item_prefix(m.n_parts, s_base, [&](int p) {
        uint64_t n_old, pad;
        return (uint32_t)((scatter_extent(m.parts[p], &n_old, &pad) + kScatterChunk - 1) /
                          kScatterChunk);
    });
    int cur = -1;
    claim_items(m.queue + kQScatter, (uint32_t)s_base[m.n_parts], [&](uint32_t item) {
        const int p = part_of(s_base, m.n_parts, item);
        if (p != cur) { load_part(sa, m.parts, p); cur = p; }
        uint64_t n_old, pad;
        const uint64_t nv = scatter_extent(sa, &n_old, &pad);
        const uint64_t first = (uint64_t)(item - (uint32_t)s_base[p]) * kScatterChunk;
        const uint64_t end = first + kScatterChunk < nv ? first + kScatterChunk : nv;
        scatter_span(sa, first + 4u * (threadIdx.x & ~31u), end, 4u * blockDim.x);
    });
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kTileCells, 4) mk_cell(MultiArgs<T> m)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ StepArgs<T> sa;
    if (threadIdx.x == 0) mbar_init(&s_bar, 1u);
    uint32_t phase = 0;
    int cur = -1;
    CellSmem sm;
    claim_items(m.queue + kQCell, (uint32_t)m.tile_base[m.n_parts], [&](uint32_t item) {
        const int p = part_of(m.tile_base, m.n_parts, item);
        if (p != cur) {
            load_part(sa, m.parts, p);
            cur = p;
            sm = cell_smem(smem_raw, &s_bar, (uint32_t)sa.tile_budget);
        }
        cell_tile<T, DIM>(sa, (int64_t)(item - (uint32_t)m.tile_base[p]), sm, phase);
    });
}

template <typename T, bool POS>
__global__ void __launch_bounds__(kCollideThreads, collide_min_blocks<T>() - (sizeof(T) == 4 ? 1 : 0))
    mk_collide(MultiArgs<T> m)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ StepArgs<T> sa;
    const int pitch = collide_stage_pitch(m.collide_stage);
    CollideSmem<T> sm;
    sm.s0 = reinterpret_cast<T*>(smem_raw);
    sm.s1 = sm.s0 + pitch;
    sm.s2 = sm.s1 + pitch;
    sm.bar = &s_bar;
    if (threadIdx.x == 0) mbar_init(&s_bar, 1u);
    uint32_t phase = 0;
    int cur = -1;
    CellTally tl;
    claim_items(m.queue + kQCollide, (uint32_t)m.ctile_base[m.n_parts], [&](uint32_t item) {
        const int p = part_of(m.ctile_base, m.n_parts, item);
        if (p != cur) {
            // the tallies belong to the part they were counted in
            if (cur >= 0) { flush_tally<T>(sa.ctr, tl); tl = CellTally(); }
            load_part(sa, m.parts, p);
            cur = p;
        }
        collide_tile<T, POS>(sa, (int64_t)(item - (uint32_t)m.ctile_base[p]), sm, phase, tl);
    });
    if (cur >= 0) flush_tally<T>(sa.ctr, tl);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kBigThreads, 2) mk_cell_big(MultiArgs<T> m)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_red[4 * (kBigThreads / 32)];
    __shared__ StepArgs<T> sa;
    for (int p = 0; p < m.n_parts; ++p) {
        load_part(sa, m.parts, p);
        cell_big_part<T, DIM>(sa, blockIdx.x, gridDim.x, smem_raw, s_red);
    }
}

template <typename T, bool POS>
__global__ void __launch_bounds__(256) mk_collide_big(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    for (int p = 0; p < m.n_parts; ++p) {
        load_part(sa, m.parts, p);
        collide_big_part<T, POS>(sa, blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                                 gridDim.x * (blockDim.x >> 5));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) mk_reduce(MultiArgs<T> m)
{
    __shared__ StepArgs<T> sa;
    for (int p = 0; p < m.n_parts; ++p) {
        load_part(sa, m.parts, p);
        reduce_part(sa, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
    }
}

// the step's end of every part, and the claim counters zeroed for the next
// step (every queue-driven kernel of this step has completed)
template <typename T>
__global__ void mk_step_end(MultiArgs<T> m)
{
    if (threadIdx.x < (uint32_t)m.n_parts) step_end_part(m.parts[threadIdx.x]);
    if (threadIdx.x < (uint32_t)kQueueKinds) m.queue[threadIdx.x] = 0u;
}

// ---------------------------------------------------------------------------
// Host launchers
template <typename T>
static const StepArgs<T>& A(const void* p) { return *static_cast<const StepArgs<T>*>(p); }

// this compilation's precision (see the top of the file)
#define DISPATCH_PREC(prec, ...)                                      \
    do {                                                              \
        (void)(prec);                                                 \
        using T = DSMC_KT;                                            \
        __VA_ARGS__;                                                  \
    } while (0)

#define DISPATCH_DIM(dim, ...)                                        \
    do {                                                              \
        if ((dim) == 3) { constexpr int D = 3; __VA_ARGS__; }         \
        else { constexpr int D = 2; __VA_ARGS__; }                    \
    } while (0)


// A kernel's dynamic shared-memory limit.  (The shared-memory carveout is
// left to the driver: it takes the smallest carveout that holds the
// resident CTAs, which leaves the rest of the SM's 256 KB to the L1 cache
// that the gathers of the sort/gather kernel hit; a larger carveout, or 6
// KB more shared memory per tile CTA, measured 40% slower there.)
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// launch a step kernel with programmatic stream serialisation (see
// pdl_enter) when ls.pdl is set: its launch overlaps the end of the
// previous kernel.  Graph replays are not helped by it (measured slower),
// so captured steps use plain launches.
template <typename... P, typename... Args>
static void launch_pdl(const LaunchShape& ls, void (*kernel)(P...), unsigned grid, unsigned block,
                       size_t smem, cudaStream_t s, const Args&... args)
{
    if (!ls.pdl) {
        kernel<<<grid, block, smem, s>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a launch the attribute makes fail is retried as a plain launch, which
    // reports any error of its own through cudaGetLastError
    if (cudaLaunchKernelEx(&cfg, kernel, args...) != cudaSuccess) {
        (void)cudaGetLastError();
        kernel<<<grid, block, smem, s>>>(args...);
    }
}

void launch_init_cells(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, (k_init_cells<T><<<ls.sms * 4, 256, 0, s>>>(A<T>(args))));
}

void launch_fill(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const StepArgs<T>& a = A<T>(args);
        k_fill_count<T><<<ls.sms * 4, 256, 0, s>>>(a);
        launch_scan(args, ls, s);
        DISPATCH_DIM(ls.dim, (k_fill_particles<T, D><<<ls.sms * 8, 256, 0, s>>>(a)));
        k_fill_ids<T><<<(a.n_runs + 255) / 256, 256, 0, s>>>(a);
    });
}

void launch_generate(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const StepArgs<T>& a = A<T>(args);
        const unsigned grid = (unsigned)a.n_runs * (unsigned)a.gen_groups;
        if (a.gen_groups > 1) launch_pdl(ls, k_gen_count<T>, grid, 256, 0, s, a);
        DISPATCH_DIM(ls.dim, launch_pdl(ls, k_generate<T, D>, grid, 256, 0, s, a));
    });
}

void launch_move(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, DISPATCH_DIM(ls.dim, {
        launch_pdl(ls, k_move<T, D>, ls.move_blocks, ls.move_threads, 0, s, A<T>(args));
        launch_pdl(ls, k_move_slow<T, D>, ls.sms * 2, 256, 0, s, A<T>(args));
    }));
}

void launch_scan(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const StepArgs<T>& a = A<T>(args);
        launch_pdl(ls, k_scan1<T>, a.scan_blocks, kScanThreads, 0, s, a);
        launch_pdl(ls, k_scan2<T>, a.scan_blocks, kScanThreads, 0, s, a);
    });
}

void launch_scatter(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, launch_pdl(ls, k_scatter<T>, ls.scatter_blocks, 256, 0, s, A<T>(args)));
}

size_t cell_smem_bytes(int prec, int budget)
{
    // start table, LCR entries (eight spare for 16-byte alignment), cell tags
    const size_t head = (kTileCells + 4) * sizeof(uint32_t);
    const size_t tile = ((size_t)budget + 8) * sizeof(uint32_t) + (size_t)budget * sizeof(uint16_t);
    const size_t warps = (kTileCells / 32) * (prec == DSMC_FP64 ? warp_scratch_bytes<double>()
                                                                : warp_scratch_bytes<float>());
    return head + (tile > warps ? tile : warps);
}

void launch_cell(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, DISPATCH_DIM(ls.dim, {
        const StepArgs<T>& a = A<T>(args);
        launch_pdl(ls, k_cell<T, D>, ls.cell_blocks, kTileCells, cell_smem_bytes(prec, a.tile_budget), s, a);
    }));
}

static size_t collide_smem(int prec, int stage)
{
    return (size_t)3 * collide_stage_pitch(stage) * (prec == DSMC_FP64 ? 8 : 4);
}

// the collision kernels choose partners by position only when the gas
// model asks for it (pick_partner); the uniform choice keeps its own
// instantiation
void launch_collide(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const StepArgs<T>& a = A<T>(args);
        const size_t sm = collide_smem(prec, a.collide_stage);
        if (a.hot.partner != DSMC_PARTNER_UNIFORM)
            launch_pdl(ls, k_collide<T, true>, ls.collide_blocks, kCollideThreads, sm, s, a);
        else
            launch_pdl(ls, k_collide<T, false>, ls.collide_blocks, kCollideThreads, sm, s, a);
    });
}

int big_cell_limit() { return big_max_of<DSMC_KT>(); }

static size_t big_smem(int) { return big_smem_bytes(); }

void launch_cell_big(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, DISPATCH_DIM(ls.dim, launch_pdl(ls, k_cell_big<T, D>, ls.big_blocks, kBigThreads,
                                                        big_smem(prec), s, A<T>(args))));
}

void launch_collide_big(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const StepArgs<T>& a = A<T>(args);
        if (a.hot.partner != DSMC_PARTNER_UNIFORM)
            launch_pdl(ls, k_collide_big<T, true>, ls.sms * 2, 256, 0, s, a);
        else
            launch_pdl(ls, k_collide_big<T, false>, ls.sms * 2, 256, 0, s, a);
    });
}

void launch_reduce(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, launch_pdl(ls, k_reduce<T>, ls.sms * 4, 256, 0, s, A<T>(args)));
}

void launch_step_end(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, launch_pdl(ls, k_step_end<T>, 1, 1, 0, s, A<T>(args)));
}

void launch_check(const void* args, const LaunchShape& ls, cudaStream_t s)
{
    DISPATCH_DIM(ls.dim, (k_check<DSMC_KT, D><<<ls.sms * 4, 256, 0, s>>>(A<DSMC_KT>(args))));
}

void launch_sample_now(const void* args, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const StepArgs<T>& a = A<T>(args);
        k_sample_now<T><<<128, 256, 0, s>>>(a, a.vi[0], a.vi[1], a.vi[2]);
    });
}

void launch_macro(const void* args, int sample, int n_runs, int window, double* out,
                  cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, (k_macro<T><<<64, 128, 0, s>>>(A<T>(args), sample, n_runs, window, out)));
}

// The tile kernel's dynamic shared-memory limit is a property of the
// function, shared by every context of the process: it only ever rises, so
// that a context whose tile budget is larger than a later context's keeps
// launching.
static cudaError_t raise_cell_smem_limit(int prec, int dim, size_t bytes)
{
    static std::mutex mu;
    static size_t set[2][2] = {{0, 0}, {0, 0}};
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = set[prec == DSMC_FP64 ? 1 : 0][dim == 3 ? 1 : 0];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    DISPATCH_PREC(prec, DISPATCH_DIM(dim, {
        e = set_smem(k_cell<T, D>, bytes);
    }));
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// The collision kernels' dynamic shared-memory limits, raised only (as the
// tile kernel's): [single, multi-part].
static cudaError_t raise_collide_smem_limit(int prec, int multi, size_t bytes)
{
    static std::mutex mu;
    static size_t set[2][2] = {{0, 0}, {0, 0}};
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = set[prec == DSMC_FP64 ? 1 : 0][multi ? 1 : 0];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    DISPATCH_PREC(prec, {
        if (multi) {
            e = set_smem(mk_collide<T, false>, bytes);
            if (e == cudaSuccess) e = set_smem(mk_collide<T, true>, bytes);
        } else {
            e = set_smem(k_collide<T, false>, bytes);
            if (e == cudaSuccess) e = set_smem(k_collide<T, true>, bytes);
        }
    });
    if (e == cudaSuccess) cur = bytes;
    return e;
}

constexpr int kCollideStageMin = 1024, kCollideStageMax = 8192;

// The largest collision stage (a multiple of 64 particles, 1024 .. 8192) at
// which `per_sm` CTAs of the collision kernel (`multi`: the multi-part one)
// are resident on an SM together, by the occupancy calculator; 1024 if none.
int collide_stage_for(int per_sm, int multi)
{
    constexpr int prec = DSMC_KPREC;
    if (per_sm < 1) per_sm = 1;
    raise_collide_smem_limit(prec, multi, collide_smem(prec, kCollideStageMax));
    int stage = kCollideStageMax;
    for (; stage > kCollideStageMin; stage -= 64) {
        int b = 0;
        DISPATCH_PREC(prec, {
            if (multi)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, mk_collide<T, false>,
                                                              kCollideThreads,
                                                              collide_smem(prec, stage));
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_collide<T, false>,
                                                              kCollideThreads,
                                                              collide_smem(prec, stage));
        });
        if (b >= per_sm) break;
    }
    (void)cudaGetLastError();
    return stage;
}

// Default collision shape: the most CTAs per SM (at most 8) whose stage
// still holds ls->collide_ppc particles a cell (22 when unset), the stage
// the largest that lets that many share an SM.
static void pick_collide_shape(int sms, LaunchShape* ls, int multi)
{
    constexpr int prec = DSMC_KPREC;
    const int want = (ls->collide_ppc > 0 ? ls->collide_ppc : 22) * kCollideCells;
    int k = 8, stage = 0;
    for (; k >= 1; --k) {
        stage = collide_stage_for(k, multi);
        if (stage >= want || k == 1) break;
    }
    if (k < 1) k = 1;
    ls->collide_blocks = sms * k;
    ls->collide_stage = stage;
    raise_collide_smem_limit(prec, multi, collide_smem(prec, stage));
}

void compute_launch_shape(int dim, int sms, LaunchShape* ls)
{
    constexpr int prec = DSMC_KPREC;
    ls->dim = dim;
    ls->sms = sms;
    // tile budget: 3072 staged particles (LCR entries and cell tags, 31 KB;
    // measured on the 512-run duct ensemble: 56 ms against 62 ms for 6144 --
    // the smaller stage leaves more of the SM to the L1 cache the gathers
    // hit), at least the warp path's scratch; a multiple of 8 keeps the
    // staged arrays 16-byte aligned
    int budget = 3072;
    if (ls->tile_budget <= 0) ls->tile_budget = budget;
    ls->tile_budget = (ls->tile_budget + 7) / 8 * 8;
    int bm = 0, bc = 0;
    raise_cell_smem_limit(prec, dim, cell_smem_bytes(prec, ls->tile_budget));
    DISPATCH_PREC(prec, DISPATCH_DIM(dim, {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bm, k_move<T, D>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bc, k_cell<T, D>, kTileCells,
                                                      cell_smem_bytes(prec, ls->tile_budget));
    }));
    ls->move_threads = 256;
    ls->move_blocks = sms * (bm > 0 ? bm : 4);
    ls->scatter_blocks = sms * 8;
    ls->cell_blocks = sms * (bc > 0 ? bc : 2);
    pick_collide_shape(sms, ls, 0);
    ls->big_blocks = sms * 2;
}

cudaError_t prepare_kernels(int dim, int tile_budget, int collide_stage)
{
    constexpr int prec = DSMC_KPREC;
    cudaError_t e = cudaSuccess;
    DISPATCH_PREC(prec, DISPATCH_DIM(dim, {
        e = set_smem(k_cell_big<T, D>, big_smem(prec));
    }));
    if (e == cudaSuccess) e = raise_collide_smem_limit(prec, 0, collide_smem(prec, collide_stage));
    if (e == cudaSuccess) e = raise_cell_smem_limit(prec, dim, cell_smem_bytes(prec, tile_budget));
    return e;
}

// ---- several problems per launch ----------------------------------------
template <typename T>
static const MultiArgs<T>& MA(const void* p) { return *static_cast<const MultiArgs<T>*>(p); }

void launch_m_generate(const void* margs, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const MultiArgs<T>& m = MA<T>(margs);
        if (m.gcount_base[m.n_parts] > 0) mk_gen_count<T><<<m.gcount_base[m.n_parts], 256, 0, s>>>(m);
        DISPATCH_DIM(ls.dim, (mk_generate<T, D><<<m.gen_base[m.n_parts], 256, 0, s>>>(m)));
    });
}

void launch_m_move(const void* margs, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, DISPATCH_DIM(ls.dim, {
        const MultiArgs<T>& m = MA<T>(margs);
        mk_move<T, D><<<ls.move_blocks, 256, 0, s>>>(m);
        mk_move_slow<T, D><<<ls.sms * 2, 256, 0, s>>>(m);
    }));
}

void launch_m_scan(const void* margs, const LaunchShape&, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const MultiArgs<T>& m = MA<T>(margs);
        mk_scan1<T><<<m.scan_base[m.n_parts], kScanThreads, 0, s>>>(m);
        mk_scan2<T><<<m.scan_base[m.n_parts], kScanThreads, 0, s>>>(m);
    });
}

void launch_m_scatter(const void* margs, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, (mk_scatter<T><<<ls.scatter_blocks, 256, 0, s>>>(MA<T>(margs))));
}

void launch_m_cell(const void* margs, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, DISPATCH_DIM(ls.dim, (mk_cell<T, D><<<ls.cell_blocks, kTileCells,
                                                             cell_smem_bytes(prec, ls.tile_budget), s>>>(
                                                   MA<T>(margs)))));
}

void launch_m_cell_big(const void* margs, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, DISPATCH_DIM(ls.dim, (mk_cell_big<T, D><<<ls.big_blocks, kBigThreads,
                                                                 big_smem(prec), s>>>(MA<T>(margs)))));
}

void launch_m_collide_big(const void* margs, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        if (MA<T>(margs).positional)
            mk_collide_big<T, true><<<ls.sms * 2, 256, 0, s>>>(MA<T>(margs));
        else
            mk_collide_big<T, false><<<ls.sms * 2, 256, 0, s>>>(MA<T>(margs));
    });
}

void launch_m_collide(const void* margs, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, {
        const MultiArgs<T>& m = MA<T>(margs);
        const size_t sm = collide_smem(prec, m.collide_stage);
        if (m.positional)
            mk_collide<T, true><<<ls.collide_blocks, kCollideThreads, sm, s>>>(m);
        else
            mk_collide<T, false><<<ls.collide_blocks, kCollideThreads, sm, s>>>(m);
    });
}

void launch_m_reduce(const void* margs, const LaunchShape& ls, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, (mk_reduce<T><<<ls.sms * 4, 256, 0, s>>>(MA<T>(margs))));
}

void launch_m_step_end(const void* margs, const LaunchShape&, cudaStream_t s)
{
    constexpr int prec = DSMC_KPREC;
    DISPATCH_PREC(prec, (mk_step_end<T><<<1, kMaxParts, 0, s>>>(MA<T>(margs))));
}

cudaError_t prepare_multi_kernels(int dim, int tile_budget, int collide_stage)
{
    constexpr int prec = DSMC_KPREC;
    cudaError_t e = cudaSuccess;
    DISPATCH_PREC(prec, DISPATCH_DIM(dim, {
        e = set_smem(mk_cell_big<T, D>, big_smem(prec));
        if (e == cudaSuccess)
            e = set_smem(mk_cell<T, D>, cell_smem_bytes(prec, tile_budget));
    }));
    if (e == cudaSuccess) e = raise_collide_smem_limit(prec, 1, collide_smem(prec, collide_stage));
    return e;
}

// grids of the queue-driven kernels: as many CTAs as fit on the GPU at once
void compute_multi_shape(int dim, int sms, LaunchShape* ls)
{
    constexpr int prec = DSMC_KPREC;
    ls->dim = dim;
    ls->sms = sms;
    if (ls->tile_budget <= 0) ls->tile_budget = 3072;
    ls->tile_budget = (ls->tile_budget + 7) / 8 * 8;
    pick_collide_shape(sms, ls, 1);
    prepare_multi_kernels(dim, ls->tile_budget, ls->collide_stage);
    int bm = 0, bs = 0, bc = 0;
    DISPATCH_PREC(prec, DISPATCH_DIM(dim, {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bm, mk_move<T, D>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, mk_scatter<T>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bc, mk_cell<T, D>, kTileCells,
                                                      cell_smem_bytes(prec, ls->tile_budget));
    }));
    ls->move_threads = 256;
    ls->move_blocks = sms * (bm > 0 ? bm : 4);
    ls->scatter_blocks = sms * (bs > 0 ? bs : 4);
    ls->cell_blocks = sms * (bc > 0 ? bc : 2);
    ls->big_blocks = sms * 2;
    ls->pdl = 0;
}

#if !defined(DSMC_KERNELS_FP64)
// Test hook for the bounded waits: an mbarrier expects 16 bytes that no
// copy will deliver, so its wait gives up after `polls` polls and sets
// DSMC_ERR_TIMEOUT (in the hook's own word, not the run's error word), as a
// bulk-copy wait of the step kernels would.  No asynchronous operation is
// left in flight.
__global__ void k_timeout_probe(Counters* ctr, uint32_t polls)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1u);
        mbar_arrive_expect_tx(&bar, 16u);
        bool done = false;
        for (uint32_t it = 0; it < polls && !done; ++it) done = mbar_try_wait(&bar, 0u);
        if (!done) atomicOr(&ctr->probe, DSMC_ERR_TIMEOUT);
    }
}
#endif

}  // namespace DSMC_KNS

#if !defined(DSMC_KERNELS_FP64)

cudaError_t timeout_probe(Counters* ctr, uint32_t polls, cudaStream_t s)
{
    f32::k_timeout_probe<<<1, 32, 0, s>>>(ctr, polls);
    return cudaGetLastError();
}

cudaError_t philox_device(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                          cudaStream_t s)
{
    f32::k_philox<<<64, 256, 0, s>>>(n, ctr, key, out);
    return cudaGetLastError();
}

#endif

}  // namespace dsmc
