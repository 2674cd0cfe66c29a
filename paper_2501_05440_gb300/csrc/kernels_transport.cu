// kernels_transport.cu -- transport kernels.
//
// Event mode (the field-standard event-based design the paper's Sec. 2 says
// MC/DC is moving to): one kernel per event type over compacted index queues,
// so every warp runs one kind of event; the queues are built by warp-ballot
// compaction with one atomic per warp.
//
// Persistent mode: one grid-resident kernel per cycle; each thread keeps a
// particle in registers and runs its events, refilling from a device work
// counter when it dies (no host round trip, no per-event launches).
#include "kernels.h"
#include "steps.cuh"

namespace mcgb {

__device__ __forceinline__ void load_ps(const Particles &P, int i, PS &p)
{
    p.x = P.x[i]; p.y = P.y[i]; p.z = P.z[i];
    p.u = P.u[i]; p.v = P.v[i]; p.w = P.w[i];
    p.iu = P.iu[i]; p.iv = P.iv[i]; p.iw = P.iw[i];
    p.E = P.E[i];
    p.t = P.t[i];
    p.s = P.s[i];
    p.g = P.g[i]; p.cell = P.cell[i]; p.ix = P.ix[i]; p.iy = P.iy[i]; p.ucell = P.ucell[i];
    p.mat = P.mat[i]; p.prob = P.prob[i]; p.root = P.root[i];
    p.nfis = P.nfis[i]; p.ncoll = P.ncoll[i]; p.ncross = P.ncross[i];
    p.fate = P.fate[i];
}

__device__ __forceinline__ void store_ps(const Particles &P, int i, const PS &p)
{
    P.x[i] = p.x; P.y[i] = p.y; P.z[i] = p.z;
    P.u[i] = p.u; P.v[i] = p.v; P.w[i] = p.w;
    P.iu[i] = p.iu; P.iv[i] = p.iv; P.iw[i] = p.iw;
    P.E[i] = p.E;
    P.t[i] = p.t;
    P.s[i] = p.s;
    P.g[i] = p.g; P.cell[i] = p.cell; P.ix[i] = p.ix; P.iy[i] = p.iy; P.ucell[i] = p.ucell;
    P.mat[i] = p.mat; P.prob[i] = p.prob; P.root[i] = p.root;
    P.nfis[i] = p.nfis; P.ncoll[i] = p.ncoll; P.ncross[i] = p.ncross;
    P.fate[i] = (signed char)p.fate;
}

// One kernel per event: each kernel moves only the state fields its step reads
// and the ones it can change (event_advance_bytes counts those of k_advance).
// Fields a world does not use are neither read nor written: 1/w without
// z-planes, E without continuous-energy problems, t without time dependence.
__device__ __forceinline__ void load_geom(const World &W, const Particles &P, int i, PS &p)
{
    p.x = P.x[i]; p.y = P.y[i]; p.z = P.z[i];
    p.u = P.u[i]; p.v = P.v[i]; p.w = P.w[i];
    p.iu = P.iu[i]; p.iv = P.iv[i]; p.iw = W.need_iw ? P.iw[i] : 0.0;
    p.cell = P.cell[i]; p.ix = P.ix[i]; p.iy = P.iy[i]; p.ucell = P.ucell[i]; p.mat = P.mat[i];
}

__device__ __forceinline__ void store_dir(const World &W, const Particles &P, int i, const PS &p)
{
    P.u[i] = p.u; P.v[i] = p.v; P.w[i] = p.w;
    P.iu[i] = p.iu; P.iv[i] = p.iv;
    if (W.need_iw) P.iw[i] = p.iw;
}

__device__ __forceinline__ int find_problem(const int64_t *base, int nprob, int64_t j)
{
    int lo = 0, hi = nprob;   // base[lo] <= j < base[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (base[mid] <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int accum_replica(const World &W)
{
    return (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % (unsigned)W.nrep);
}

// ---------------------------------------------------------------------------
// CE = false: instantiations for worlds without continuous-energy problems
// (that physics compiled out; chosen by launch_* from W.ce_any).
template <bool CE>
__global__ void k_source(World W, Particles P, Bank Bsrc, RunBufs R, int gen, int64_t total,
                         const int64_t *gen_base, const int *src_idx, int eigen, const int *gen_dev)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= total) return;
    if (gen_dev) gen = *gen_dev;
    int prob = find_problem(gen_base, W.nprob, j);
    const ProblemDev &Pd = W.prob[prob];
    PS p;
    bool ok = init_particle<CE>(W, Pd, Bsrc, p, prob, j - gen_base[prob], gen,
                                src_idx ? src_idx[j] : -1, eigen != 0);
    if (!ok) {
        atomicOr(R.err, ERR_SOURCE);
        p.fate = FATE_LOST;
        p.cell = 0;
        p.mat = 0;
    }
    store_ps(P, (int)j, p);
    P.kt[j] = 0.0;
    P.kc[j] = 0.0;
}

// n_dev (when set) holds the list's length on the device; the grid covers a
// host-known upper bound, so the host need not wait for the count.
template <bool CE>
__global__ void __launch_bounds__(256, 4) k_advance(World W, Particles P, RunBufs R, const int *list,
                                                 int n, const int *n_dev, int *q_cross, int *q_coll)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (n_dev) n = *n_dev;
    int i = -1, ev = EV_DEAD;
    if (t < n) {
        i = list ? list[t] : t;
        PS p;
        // every field is requested before the fate is tested, so that one round
        // trip to memory serves them all (slot i is always in bounds)
        p.fate = P.fate[i];
        load_geom(W, P, i, p);
        p.E = W.ce_any ? P.E[i] : 0.0;
        p.t = W.time_any ? P.t[i] : 0.0;
        p.s = P.s[i];
        p.g = P.g[i]; p.prob = P.prob[i]; p.root = P.root[i];
        p.ncoll = P.ncoll[i]; p.ncross = P.ncross[i];
        double kt = P.kt[i];
        if (p.fate == FATE_ALIVE) {
            const ProblemDev &Pd = W.prob[p.prob];
            int kind, which, uk = 0;
            ev = step_advance<false, true, CE>(W, Pd, p, i, R, accum_replica(W), kind, which, uk, kt);
            P.x[i] = p.x; P.y[i] = p.y; P.z[i] = p.z;
            if (W.time_any) P.t[i] = p.t;
            P.s[i] = p.s;
            if (p.fate != FATE_ALIVE) P.fate[i] = (signed char)p.fate;
            P.kt[i] = kt;
            P.bkind[i] = (signed char)kind;
            P.bwhich[i] = which;
            P.uk[i] = uk;
        }
    }
    enqueue2(ev == EV_CROSS, ev == EV_COLLIDE, i, q_cross, R.q_n + 0, q_coll, R.q_n + 1);
}

__global__ void __launch_bounds__(256) k_cross(World W, Particles P, RunBufs R, const int *q_cross,
                                               int *next, int *next_n)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int n = R.q_n[0];
    int i = -1;
    bool alive = false;
    if (t < n) {
        i = q_cross[t];
        PS p;
        load_geom(W, P, i, p);
        p.ncross = P.ncross[i];
        p.fate = FATE_ALIVE;
        const double u = p.u, v = p.v, w = p.w;
        alive = step_cross(W, p, P.bkind[i], P.bwhich[i]) == EV_ADVANCE;
        P.ncross[i] = p.ncross;
        P.cell[i] = p.cell; P.ix[i] = p.ix; P.iy[i] = p.iy; P.ucell[i] = p.ucell; P.mat[i] = p.mat;
        if (!alive) P.fate[i] = (signed char)p.fate;
        // a reflection changed the direction
        if (__double_as_longlong(u) != __double_as_longlong(p.u) ||
            __double_as_longlong(v) != __double_as_longlong(p.v) ||
            __double_as_longlong(w) != __double_as_longlong(p.w))
            store_dir(W, P, i, p);
    }
    enqueue(alive, i, next, next_n);
}

template <bool CE>
__global__ void __launch_bounds__(256, 4) k_collide(World W, Particles P, Bank Bdst, RunBufs R,
                                                 const int *q_coll, int *next, int *next_n)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int n = R.q_n[1];
    int i = -1;
    bool alive = false;
    if (t < n) {
        i = q_coll[t];
        PS p;
        p.x = P.x[i]; p.y = P.y[i]; p.z = P.z[i];
        p.u = P.u[i]; p.v = P.v[i]; p.w = P.w[i];
        p.t = W.time_any ? P.t[i] : 0.0;
        p.E = W.ce_any ? P.E[i] : 0.0;
        p.s = P.s[i];
        p.g = P.g[i]; p.cell = P.cell[i]; p.ix = P.ix[i]; p.iy = P.iy[i]; p.ucell = P.ucell[i];
        p.mat = P.mat[i]; p.prob = P.prob[i]; p.root = P.root[i];
        p.nfis = P.nfis[i]; p.ncoll = P.ncoll[i];
        p.fate = FATE_ALIVE;
        const ProblemDev &Pd = W.prob[p.prob];
        double kc = P.kc[i];
        alive = step_collide<false, true, CE>(W, Pd, p, i, Bdst, R, P.uk[i], kc) == EV_ADVANCE;
        P.ncoll[i] = p.ncoll;
        P.nfis[i] = p.nfis;
        P.g[i] = p.g;
        if (W.ce_any) P.E[i] = p.E;
        P.s[i] = p.s;
        if (alive) store_dir(W, P, i, p);
        else P.fate[i] = (signed char)p.fate;
        P.kc[i] = kc;
    }
    enqueue(alive, i, next, next_n);
}

// Monolithic segment (Sec. 2: every transport operation of one segment in a
// single kernel, no sorting or grouping of like operations): flight, then the
// crossing or collision it ends in; survivors go to the other list.
template <bool CE>
__global__ void __launch_bounds__(256, 3) k_segment(World W, Particles P, Bank Bdst, RunBufs R,
                                                 const int *list, int n, const int *n_dev,
                                                 int *next, int *next_n)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (n_dev) n = *n_dev;
    int i = -1;
    bool alive = false;
    if (t < n) {
        i = list ? list[t] : t;
        PS p;
        // the fields the segment's steps read (as in k_advance, plus the
        // fission-site count a collision continues), all requested before the
        // fate is tested
        p.fate = P.fate[i];
        load_geom(W, P, i, p);
        p.E = W.ce_any ? P.E[i] : 0.0;
        p.t = W.time_any ? P.t[i] : 0.0;
        p.s = P.s[i];
        p.g = P.g[i]; p.prob = P.prob[i]; p.root = P.root[i];
        p.ncoll = P.ncoll[i]; p.ncross = P.ncross[i]; p.nfis = P.nfis[i];
        double kt = P.kt[i];
        if (p.fate == FATE_ALIVE) {
            const double u = p.u, v = p.v, w = p.w;
            const ProblemDev &Pd = W.prob[p.prob];
            int kind, which, uk = 0;
            double xt = 0.0, xn = 0.0;
            int ev = step_advance<false, true, CE>(W, Pd, p, i, R, accum_replica(W), kind, which, uk, kt,
                                                   nullptr, nullptr, nullptr, &xt, &xn);
            P.kt[i] = kt;
            if (ev == EV_CROSS) {
                ev = step_cross(W, p, kind, which);
                P.ncross[i] = p.ncross;
                P.cell[i] = p.cell; P.ix[i] = p.ix; P.iy[i] = p.iy; P.ucell[i] = p.ucell;
                P.mat[i] = p.mat;
            } else if (ev == EV_COLLIDE) {
                double kc = P.kc[i];
                ev = step_collide<false, true, CE>(W, Pd, p, i, Bdst, R, uk, kc, nullptr, true, xt, xn);
                P.kc[i] = kc;
                P.ncoll[i] = p.ncoll;
                P.nfis[i] = p.nfis;
                P.g[i] = p.g;
                if (W.ce_any) P.E[i] = p.E;
            }
            // what every segment changes: position, clock, random state; the
            // direction after a scattering or reflection; the fate at the end
            P.x[i] = p.x; P.y[i] = p.y; P.z[i] = p.z;
            if (W.time_any) P.t[i] = p.t;
            P.s[i] = p.s;
            if (__double_as_longlong(u) != __double_as_longlong(p.u) ||
                __double_as_longlong(v) != __double_as_longlong(p.v) ||
                __double_as_longlong(w) != __double_as_longlong(p.w))
                store_dir(W, P, i, p);
            if (p.fate != FATE_ALIVE) P.fate[i] = (signed char)p.fate;
            alive = ev == EV_ADVANCE;
        }
    }
    enqueue(alive, i, next, next_n);
}

static inline int nblocks(int64_t n, int block) { return (int)((n + block - 1) / block); }

double event_advance_bytes(const World &W)
{
    const double d = 8.0, i4 = 4.0;
    // loads: fate; x y z u v w 1/u 1/v [1/w] [E] [t] s; g cell ix iy ucell mat
    // prob root ncoll ncross; kt
    double rd = 1.0 + d * (8 + (W.need_iw ? 1 : 0) + (W.ce_any ? 1 : 0) + (W.time_any ? 1 : 0) + 1) +
                i4 * 10 + d;
    // stores: x y z [t] s kt; kind (1 B), crossed surface, union index; the
    // queue entry of the event that follows
    double wr = d * (3 + (W.time_any ? 1 : 0) + 1 + 1) + 1.0 + i4 * 2 + i4;
    return rd + wr;
}

void launch_source(const World &W, const Particles &P, const Bank &Bsrc, const RunBufs &R, int gen,
                   int64_t total, const int64_t *gen_base, const int *src_idx, int eigen, int block,
                   cudaStream_t st, const int *gen_dev)
{
    if (total <= 0) return;
    if (W.ce_any)
        k_source<true><<<nblocks(total, block), block, 0, st>>>(W, P, Bsrc, R, gen, total, gen_base,
                                                                src_idx, eigen, gen_dev);
    else
        k_source<false><<<nblocks(total, block), block, 0, st>>>(W, P, Bsrc, R, gen, total, gen_base,
                                                                 src_idx, eigen, gen_dev);
}

void launch_advance(const World &W, const Particles &P, const RunBufs &R, const int *list, int n,
                    const int *n_dev, int *q_cross, int *q_coll, int block, cudaStream_t st)
{
    if (n <= 0) return;
    if (W.ce_any)
        k_advance<true><<<nblocks(n, block), block, 0, st>>>(W, P, R, list, n, n_dev, q_cross, q_coll);
    else
        k_advance<false><<<nblocks(n, block), block, 0, st>>>(W, P, R, list, n, n_dev, q_cross, q_coll);
}

void launch_cross(const World &W, const Particles &P, const RunBufs &R, const int *q_cross,
                  int n_bound, int *next, int *next_n, int block, cudaStream_t st)
{
    if (n_bound <= 0) return;
    k_cross<<<nblocks(n_bound, block), block, 0, st>>>(W, P, R, q_cross, next, next_n);
}

void launch_collide(const World &W, const Particles &P, const Bank &Bdst, const RunBufs &R,
                    const int *q_coll, int n_bound, int *next, int *next_n, int block,
                    cudaStream_t st)
{
    if (n_bound <= 0) return;
    if (W.ce_any)
        k_collide<true><<<nblocks(n_bound, block), block, 0, st>>>(W, P, Bdst, R, q_coll, next, next_n);
    else
        k_collide<false><<<nblocks(n_bound, block), block, 0, st>>>(W, P, Bdst, R, q_coll, next, next_n);
}

void launch_segment(const World &W, const Particles &P, const Bank &Bdst, const RunBufs &R,
                    const int *list, int n, const int *n_dev, int *next, int *next_n, int block,
                    cudaStream_t st)
{
    if (n <= 0) return;
    if (W.ce_any)
        k_segment<true><<<nblocks(n, block), block, 0, st>>>(W, P, Bdst, R, list, n, n_dev, next, next_n);
    else
        k_segment<false><<<nblocks(n, block), block, 0, st>>>(W, P, Bdst, R, list, n, n_dev, next,
                                                              next_n);
}

// ---------------------------------------------------------------------------
// Persistent event loop.  All lanes of a warp stay in the loop until every
// lane has run out of work, so the warp-wide ballot/shuffle calls are always
// made by the full warp.
__device__ __forceinline__ void write_dead(const Particles &P, int slot, const PS &p, double kt,
                                           double kc)
{
    P.nfis[slot] = p.nfis;
    P.ncoll[slot] = p.ncoll;
    P.ncross[slot] = p.ncross;
    P.fate[slot] = (signed char)p.fate;
    P.s[slot] = p.s;
    P.g[slot] = p.g;
    P.kt[slot] = kt;
    P.kc[slot] = kc;
}

template <bool TIME, bool CE>
__global__ void __launch_bounds__(256) k_persistent(World W, Particles P, Bank Bsrc, Bank Bdst,
                                                    RunBufs R, PersistentArgs a)
{
    const int64_t total = a.gen_n ? (int64_t)*a.gen_n : a.total;
    const int lane = threadIdx.x & 31;
    const int rep = accum_replica(W);
    PS p;
    p.fate = FATE_LOST;
    int slot = -1;
    bool alive = false, done = false;
    double kt = 0.0, kc = 0.0;
    const ProblemDev *Pd = W.prob;
    long long passes = 0;
    for (;;) {
        if (a.max_passes > 0 && ++passes > a.max_passes) {   // warp-uniform
            if (lane == 0) atomicOr(R.err, ERR_ITER);
            break;
        }
        bool need = !alive && !done;
        unsigned m = __ballot_sync(0xffffffffu, need);
        if (m) {
            int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(a.work, __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (need) {
                int64_t j = (int64_t)base + __popc(m & ((1u << lane) - 1u));
                if (j >= total) {
                    done = true;
                } else {
                    slot = (int)j;
                    kt = 0.0;
                    kc = 0.0;
                    const bool ok = load_born<TIME, CE>(W, P, j, p);   // made by launch_source
                    Pd = W.prob + p.prob;
                    if (ok) {
                        alive = true;
                    } else {
                        atomicOr(R.err, ERR_SOURCE);
                        p.fate = FATE_LOST;
                        write_dead(P, slot, p, kt, kc);
                    }
                }
            }
        }
        if (__all_sync(0xffffffffu, done)) break;
        if (alive) {
            int kind, which, uk = 0;
            double xt = 0.0, xn = 0.0;
            int ev = step_advance<false, TIME, CE>(W, *Pd, p, slot, R, rep, kind, which, uk, kt, nullptr,
                                                   nullptr, nullptr, &xt, &xn);
            if (ev == EV_CROSS) ev = step_cross(W, p, kind, which);
            else if (ev == EV_COLLIDE)
                ev = step_collide<false, TIME, CE>(W, *Pd, p, slot, Bdst, R, uk, kc, nullptr, true, xt, xn);
            if (ev == EV_DEAD) {
                alive = false;
                write_dead(P, slot, p, kt, kc);
            }
        }
    }
}

void launch_persistent(const World &W, const Particles &P, const Bank &Bsrc, const Bank &Bdst,
                       const RunBufs &R, const PersistentArgs &a, int grid, int block,
                       cudaStream_t st)
{
    if (W.ce_any) {
        if (W.time_any) k_persistent<true, true><<<grid, block, 0, st>>>(W, P, Bsrc, Bdst, R, a);
        else k_persistent<false, true><<<grid, block, 0, st>>>(W, P, Bsrc, Bdst, R, a);
    } else {
        if (W.time_any) k_persistent<true, false><<<grid, block, 0, st>>>(W, P, Bsrc, Bdst, R, a);
        else k_persistent<false, false><<<grid, block, 0, st>>>(W, P, Bsrc, Bdst, R, a);
    }
}

int persistent_max_blocks_per_sm(int block)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persistent<false, true>, block, 0);
    return n;
}

}  // namespace mcgb
