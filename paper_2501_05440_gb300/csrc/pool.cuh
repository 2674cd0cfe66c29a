// pool.cuh -- persistent event loop with block-sorted events (templates; each
// kernels_pool_*.cu translation unit instantiates one combination of
// continuous-energy physics and time dependence, so that they compile in
// parallel).
//
// Each block keeps a pool of P particles in shared memory (structure of
// arrays) and repeats: refill empty slots from the device work counter; run
// the flight (advance) of every newborn and live particle; run the surface
// crossings, then the collisions.  Twice a pass the block builds a compacted
// list: the empty slots, then the live particles by material, for the refill
// and the flights; the crossings, then the collisions by material, for the
// events -- so that consecutive threads, whole warps, run the same event on
// the same kind of data.  The
// grid stays resident for the whole cycle; no particle state goes through HBM
// between events.  When no history is left to start and a block holds at most
// a warp's worth of particles, each runs to its end in registers.  Results do
// not depend on which thread runs which slot: every history draws from its own
// random stream.
#pragma once
#include "kernels.h"
#include "steps.cuh"

namespace mcgb {

namespace {

constexpr int POOL_T = 256;          // threads per block
constexpr int NBUCKET = 33;          // list buckets (flights: 1 + material % 32; events: 0 lattice
                                     // steps, 1 surface crossings, 2 + material % 31 collisions)
constexpr int SLOT_EMPTY = -2;

struct Pool {
    double *x, *y, *z, *u, *v, *w, *kt, *kc, *iu, *iv, *iw;
    double *E, *sg, *nf;   // continuous energy only: energy, the last flight's Sigma_t, nuSigma_f
    double *t;             // time-dependent only: the clock
    unsigned long long *s;
    int *g, *cell, *ix, *iy, *ucell, *mat, *prob, *root, *nfis, *ncoll, *ncross, *gslot, *fate;
    int *evw;              // the flight's outcome: event | kind << 4 | (surface + 1) << 8
    int *uk;               // continuous energy only: union-grid index
    int *list;
};

// Fields per particle: 12 doubles and 15 ints always, 3 doubles and an int
// more with continuous energy, a double more with time.  A multigroup pool of
// 256 particles (156 B each) leaves four blocks per SM room for a larger L1.
__host__ __device__ constexpr size_t pool_bytes(int P, bool TIME, bool CE)
{
    return (size_t)P * ((12 + (CE ? 3 : 0) + (TIME ? 1 : 0)) * 8 + (15 + (CE ? 1 : 0)) * 4);
}

__device__ __forceinline__ int pack_ev(int ev, int kind, int which)
{
    return ev | (kind << 4) | ((which + 1) << 8);
}
__device__ __forceinline__ int ev_kind(int e) { return (e >> 4) & 15; }
__device__ __forceinline__ int ev_which(int e) { return (int)((unsigned)e >> 8) - 1; }

template <bool TIME, bool CE>
__device__ __forceinline__ Pool carve(unsigned char *base, int P)
{
    Pool q;
    double *d = reinterpret_cast<double *>(base);
    int k = 0;
    auto nd = [&]() { return d + (size_t)(k++) * P; };
    q.x = nd(); q.y = nd(); q.z = nd(); q.u = nd(); q.v = nd(); q.w = nd();
    q.kt = nd(); q.kc = nd(); q.iu = nd(); q.iv = nd(); q.iw = nd();
    q.s = reinterpret_cast<unsigned long long *>(nd());
    q.E = CE ? nd() : nullptr;
    q.sg = CE ? nd() : nullptr;
    q.nf = CE ? nd() : nullptr;
    q.t = TIME ? nd() : nullptr;
    int *i = reinterpret_cast<int *>(d + (size_t)k * P);
    int m = 0;
    auto ni = [&]() { return i + (size_t)(m++) * P; };
    q.g = ni(); q.cell = ni(); q.ix = ni(); q.iy = ni(); q.ucell = ni(); q.mat = ni();
    q.prob = ni(); q.root = ni(); q.nfis = ni(); q.ncoll = ni(); q.ncross = ni();
    q.gslot = ni(); q.fate = ni(); q.evw = ni();
    q.uk = CE ? ni() : nullptr;
    q.list = ni();
    return q;
}

// TIME = false: the particle clock is neither loaded nor kept; CE = false: nor the energy
template <bool TIME, bool CE>
__device__ __forceinline__ void pool_load(const Pool &q, int i, PS &p)
{
    p.x = q.x[i]; p.y = q.y[i]; p.z = q.z[i]; p.u = q.u[i]; p.v = q.v[i]; p.w = q.w[i];
    p.iu = q.iu[i]; p.iv = q.iv[i]; p.iw = q.iw[i];
    p.E = CE ? q.E[i] : 0.0;
    p.s = q.s[i];
    p.t = TIME ? q.t[i] : 0.0;
    p.g = q.g[i]; p.cell = q.cell[i]; p.ix = q.ix[i]; p.iy = q.iy[i]; p.ucell = q.ucell[i];
    p.mat = q.mat[i]; p.prob = q.prob[i]; p.root = q.root[i]; p.nfis = q.nfis[i];
    p.ncoll = q.ncoll[i]; p.ncross = q.ncross[i]; p.fate = q.fate[i];
}

template <bool TIME, bool CE>
__device__ __forceinline__ void pool_store(const Pool &q, int i, const PS &p)
{
    q.x[i] = p.x; q.y[i] = p.y; q.z[i] = p.z; q.u[i] = p.u; q.v[i] = p.v; q.w[i] = p.w;
    q.iu[i] = p.iu; q.iv[i] = p.iv; q.iw[i] = p.iw;
    if (CE) q.E[i] = p.E;
    q.s[i] = p.s;
    if (TIME) q.t[i] = p.t;
    q.g[i] = p.g; q.cell[i] = p.cell; q.ix[i] = p.ix; q.iy[i] = p.iy; q.ucell[i] = p.ucell;
    q.mat[i] = p.mat; q.prob[i] = p.prob; q.root[i] = p.root; q.nfis[i] = p.nfis;
    q.ncoll[i] = p.ncoll; q.ncross[i] = p.ncross; q.fate[i] = p.fate;
}

// history over: its record goes to the global slot, the pool slot becomes empty
__device__ __forceinline__ void retire(const Pool &q, const Particles &G, int i, const PS &p)
{
    int j = q.gslot[i];
    G.nfis[j] = p.nfis;
    G.ncoll[j] = p.ncoll;
    G.ncross[j] = p.ncross;
    G.fate[j] = (signed char)p.fate;
    G.s[j] = p.s;
    G.g[j] = p.g;
    G.kt[j] = q.kt[i];
    G.kc[j] = q.kc[i];
    q.fate[i] = SLOT_EMPTY;
}

// Bucketed compaction of the pool: slots with key >= 0 go to q.list, grouped
// by key in increasing order; counts per key in cnt[NBUCKET], the total in
// cnt[NBUCKET] and returned.  All threads call.  The lanes of a warp with equal
// keys find each other (match), and one of them reserves their places in the
// bucket with a single shared-memory atomic; after one barrier every warp
// scans the bucket counts itself and places its own slots, so a second barrier
// ends the call.  Two count arrays are used in turn (hb selects), each zeroed
// during the other's call.  REFILL: bucket 0 holds the empty slots, and
// thread 0 also takes the block's share of the device work counter for them
// (s_base, s_take; s_exhausted when it runs out).
template <int P, int T, bool REFILL = false, class KeyFn>
__device__ __forceinline__ int build_list(const Pool &q, int *hist2, int &hb, int *cnt, KeyFn key,
                                          int *work = nullptr, int64_t total_work = 0,
                                          int *s_base = nullptr, int *s_take = nullptr,
                                          int *s_exhausted = nullptr)
{
    static_assert(P % T == 0, "every lane of a warp takes the same number of slots");
    static_assert(NBUCKET == 33, "32 buckets scanned by the lanes of a warp, one more after them");
    constexpr int R = P / T;
    const int lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    int *hist = hist2 + hb * (NBUCKET + 1);
    int *other = hist2 + (hb ^ 1) * (NBUCKET + 1);
    hb ^= 1;
    int kr[R], rank[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        int k = key(threadIdx.x + r * T);
        unsigned m = __match_any_sync(0xffffffffu, k);
        int first = __ffs(m) - 1;
        int base = 0;
        if (k >= 0 && lane == first) base = atomicAdd(hist + k, __popc(m));
        base = __shfl_sync(0xffffffffu, base, first);
        kr[r] = k;
        rank[r] = base + __popc(m & lower);
    }
    __syncthreads();
    // exclusive scan of the 33 bucket counts, in every warp
    int v = hist[lane];
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const int last = hist[32];
    const int base32 = __shfl_sync(0xffffffffu, x, 31);
    const int total = base32 + last;
    const int excl = x - v;
#pragma unroll
    for (int r = 0; r < R; r++) {
        int off = __shfl_sync(0xffffffffu, excl, kr[r] & 31);
        if (kr[r] == 32) off = base32;
        if (kr[r] >= 0) q.list[off + rank[r]] = threadIdx.x + r * T;
    }
    if (threadIdx.x < 32) {
        cnt[lane] = v;
        other[lane] = 0;
        if (lane == 0) {
            cnt[32] = last;
            cnt[NBUCKET] = total;
            other[32] = 0;
            if (REFILL) {   // bucket 0 holds the empty slots: v of lane 0
                int take = 0, b = 0;
                if (v > 0) {
                    b = atomicAdd(work, v);
                    int64_t left = total_work - (int64_t)b;
                    take = left <= 0 ? 0 : (left < v ? (int)left : v);
                    if (take < v) *s_exhausted = 1;
                }
                *s_base = b;
                *s_take = take;
            }
        }
    }
    __syncthreads();
    return total;
}

// P particles per block of T threads; the register budget is planned for
// pool_min_blocks(P, T, TIME, CE) resident blocks (128 registers per thread at
// 2 blocks of 256 threads; a pool of one particle per thread trades spilled
// registers for a fourth resident block -- measured faster -- which the shared
// memory allows, or a third for the time-dependent continuous-energy physics,
// where the fourth was slower).
__host__ __device__ constexpr int pool_min_blocks(int P, int T, bool TIME, bool CE)
{
    return (P <= T && T == 256) ? ((CE && TIME) ? 3 : 4) : 65536 / (T * 128);
}

template <int P, int T, bool TIME, bool CE>
__global__ void __launch_bounds__(T, pool_min_blocks(P, T, TIME, CE)) k_pool(World W, Particles G, Bank Bsrc,
                                                               Bank Bdst, RunBufs R,
                                                               PersistentArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int hist[2 * (NBUCKET + 1)], cnt[NBUCKET + 1];
    __shared__ int s_base, s_take, s_exhausted;
    const Pool q = carve<TIME, CE>(smem, P);
    int hb = 0;
    for (int k = threadIdx.x; k < 2 * (NBUCKET + 1); k += T) hist[k] = 0;
    const int64_t total = a.gen_n ? (int64_t)*a.gen_n : a.total;
    const int rep = (int)(blockIdx.x % (unsigned)W.nrep);
    for (int i = threadIdx.x; i < P; i += T) q.fate[i] = SLOT_EMPTY;
    if (threadIdx.x == 0) s_exhausted = 0;
    __syncthreads();
    long long passes = 0;
    for (;;) {
        if (a.max_passes > 0 && ++passes > a.max_passes) {   // block-uniform
            if (threadIdx.x == 0) atomicOr(R.err, ERR_ITER);
            break;
        }
        // ---- one sorted list per pass: while histories are left to start, the
        // empty slots (bucket 0, refilled from the work counter), then the live
        // particles grouped by material; the newborn fly first, unsorted
        const bool refill = !s_exhausted;   // block-uniform
        int n_all;
        if (refill)
            n_all = build_list<P, T, true>(q, hist, hb, cnt, [&](int i) {
                const int f = q.fate[i];
                return f == SLOT_EMPTY ? 0 : (f == FATE_ALIVE ? 1 + (q.mat[i] & 31) : -1);
            }, a.work, total, &s_base, &s_take, &s_exhausted);
        else
            n_all = build_list<P, T>(q, hist, hb, cnt, [&](int i) {
                return q.fate[i] == FATE_ALIVE ? 1 + (q.mat[i] & 31) : -1;
            });
        const int n0 = refill ? cnt[0] : 0;   // empty slots, listed first
        const int nb = refill ? s_take : 0;   // of which born this pass
        if (refill) {
            for (int k = threadIdx.x; k < nb; k += T) {
                int i = q.list[k];
                int64_t j = (int64_t)s_base + k;
                PS p;
                const bool ok = load_born<TIME, CE>(W, G, j, p);   // made by launch_source
                q.gslot[i] = (int)j;
                q.kt[i] = 0.0;
                q.kc[i] = 0.0;
                if (!ok) {
                    atomicOr(R.err, ERR_SOURCE);
                    p.fate = FATE_LOST;
                    p.cell = 0;
                    p.mat = 0;
                    pool_store<TIME, CE>(q, i, p);
                    retire(q, G, i, p);
                } else {
                    pool_store<TIME, CE>(q, i, p);
                }
            }
            // no barrier: list entry k below nb is born and then flown by the
            // same thread (k mod T), and the births touch no other slot
        }
        // ---- flights: the newborn (list entries below nb), then every live particle
        const int n_adv = nb + (n_all - n0);
        if (n_adv == 0 && s_exhausted) break;
        if (s_exhausted && n_adv <= 32) {
            // the block's last few histories (no more to start, one warp's worth):
            // each runs to its end in a thread of warp 0, with no block barrier,
            // list building or shared-memory round trip between its events
            const int t = threadIdx.x;
            const int i = t < n_adv ? q.list[t < nb ? t : t - nb + n0] : 0;
            if (t < n_adv && q.fate[i] == FATE_ALIVE) {
                PS p;
                pool_load<TIME, CE>(q, i, p);
                const ProblemDev &Pd = W.prob[p.prob];
                const int slot = q.gslot[i];
                double kt = q.kt[i], kc = q.kc[i];
                for (;;) {
                    int kind, which, uk = 0;
                    double xt = 0.0, xn = 0.0;
                    int ev = step_advance<false, TIME, CE>(W, Pd, p, slot, R, rep, kind, which, uk, kt,
                                                           nullptr, nullptr, nullptr, &xt, &xn);
                    if (ev == EV_CROSS) ev = step_cross(W, p, kind, which);
                    else if (ev == EV_COLLIDE)
                        ev = step_collide<false, TIME, CE>(W, Pd, p, slot, Bdst, R, uk, kc, nullptr,
                                                           true, xt, xn);
                    if (ev == EV_DEAD) break;
                }
                q.kt[i] = kt;
                q.kc[i] = kc;
                retire(q, G, i, p);
            }
            break;
        }
        for (int k = threadIdx.x; k < n_adv; k += T) {
            const int i = q.list[k < nb ? k : k - nb + n0];
            if (q.fate[i] != FATE_ALIVE) continue;   // a birth the source could not place
            PS p;
            pool_load<TIME, CE>(q, i, p);
            int kind, which, uk = 0;
            double kt = q.kt[i];
            double xt = 0.0, xn = 0.0;
            int ev = step_advance<false, TIME, CE>(W, W.prob[p.prob], p, q.gslot[i], R, rep, kind, which,
                                                uk, kt, nullptr, nullptr, nullptr, &xt, &xn);
            if (CE) {
                q.sg[i] = xt;
                q.nf[i] = xn;
            }
            q.x[i] = p.x;
            q.y[i] = p.y;
            q.z[i] = p.z;
            if (TIME) q.t[i] = p.t;
            q.s[i] = p.s;
            q.kt[i] = kt;
            q.evw[i] = pack_ev(ev, kind, which);
            if (CE) q.uk[i] = uk;
            if (ev == EV_DEAD) {
                q.fate[i] = p.fate;
                retire(q, G, i, p);
            }
        }
        __syncthreads();
        // ---- crossings (lattice steps in bucket 0, surface crossings in 1), then
        // collisions grouped by material
        int n_ev = build_list<P, T>(q, hist, hb, cnt, [&](int i) {
            if (q.fate[i] != FATE_ALIVE) return -1;
            const int e = q.evw[i];
            if ((e & 15) != EV_CROSS) return 2 + (q.mat[i] % 31);
            const int kind = ev_kind(e);   // lattice steps apart from surface crossings
            return (kind == B_LATX || kind == B_LATY) ? 0 : 1;
        });
        int n_cross = cnt[0] + cnt[1];
        for (int k = threadIdx.x; k < n_ev; k += T) {
            int i = q.list[k];
            PS p;
            pool_load<TIME, CE>(q, i, p);
            int ev;
            if (k < n_cross) {
                ev = step_cross(W, p, ev_kind(q.evw[i]), ev_which(q.evw[i]));
            } else {
                double kc = q.kc[i];
                ev = step_collide<false, TIME, CE>(W, W.prob[p.prob], p, q.gslot[i], Bdst, R, CE ? q.uk[i] : 0, kc,
                                                   nullptr, CE, CE ? q.sg[i] : 0.0, CE ? q.nf[i] : 0.0);
                q.kc[i] = kc;
            }
            pool_store<TIME, CE>(q, i, p);
            if (ev == EV_DEAD) retire(q, G, i, p);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Warp-level variant: each warp owns PW slots of the shared pool and sorts its
// own events with ballots (no block barrier; warps progress independently).
constexpr int WPOOL_T = 128;   // threads (4 warps) per block

// compacts the slots of the warp's pool for which pred(i) holds into `list`
template <int PW, class Pred>
__device__ __forceinline__ int warp_list(int *list, Pred pred)
{
    const int lane = threadIdx.x & 31;
    int n = 0;
#pragma unroll
    for (int r = 0; r < PW / 32; r++) {
        int i = r * 32 + lane;
        bool b = pred(i);
        unsigned m = __ballot_sync(0xffffffffu, b);
        if (b) list[n + __popc(m & ((1u << lane) - 1u))] = i;
        n += __popc(m);
    }
    __syncwarp();
    return n;
}

// resident blocks per SM the register budget is planned for (smem allows as many)
template <int PW> struct WpoolMinBlocks { static constexpr int value = PW <= 32 ? 6 : (PW <= 64 ? 5 : 2); };

template <int PW, bool TIME, bool CE>
__global__ void __launch_bounds__(WPOOL_T, WpoolMinBlocks<PW>::value) k_wpool(World W, Particles G, Bank Bsrc, Bank Bdst,
                                                      RunBufs R, PersistentArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Pool q = carve<TIME, CE>(smem + (size_t)warp * pool_bytes(PW, TIME, CE), PW);
    const int64_t total = a.gen_n ? (int64_t)*a.gen_n : a.total;
    const int rep = (int)((blockIdx.x * (WPOOL_T / 32) + warp) % (unsigned)W.nrep);
    for (int i = lane; i < PW; i += 32) q.fate[i] = SLOT_EMPTY;
    __syncwarp();
    bool exhausted = false;
    long long passes = 0;
    for (;;) {
        if (a.max_passes > 0 && ++passes > a.max_passes) {   // warp-uniform
            if (lane == 0) atomicOr(R.err, ERR_ITER);
            break;
        }
        if (!exhausted) {
            int n_empty = warp_list<PW>(q.list, [&](int i) { return q.fate[i] == SLOT_EMPTY; });
            int base = 0;
            if (lane == 0 && n_empty > 0) base = atomicAdd(a.work, n_empty);
            base = __shfl_sync(0xffffffffu, base, 0);
            int take = 0;
            if (n_empty > 0) {
                int64_t left = total - (int64_t)base;
                take = left <= 0 ? 0 : (left < n_empty ? (int)left : n_empty);
                if (take < n_empty) exhausted = true;
            }
            for (int k = lane; k < take; k += 32) {
                int i = q.list[k];
                int64_t j = (int64_t)base + k;
                PS p;
                const bool ok = load_born<TIME, CE>(W, G, j, p);   // made by launch_source
                q.gslot[i] = (int)j;
                q.kt[i] = 0.0;
                q.kc[i] = 0.0;
                if (!ok) {
                    atomicOr(R.err, ERR_SOURCE);
                    p.fate = FATE_LOST;
                    p.cell = 0;
                    p.mat = 0;
                    pool_store<TIME, CE>(q, i, p);
                    retire(q, G, i, p);
                } else {
                    pool_store<TIME, CE>(q, i, p);
                }
            }
            __syncwarp();
        }
        int n_adv = warp_list<PW>(q.list, [&](int i) { return q.fate[i] == FATE_ALIVE; });
        if (n_adv == 0 && exhausted) break;
        for (int k = lane; k < n_adv; k += 32) {
            int i = q.list[k];
            PS p;
            pool_load<TIME, CE>(q, i, p);
            int kind, which, uk = 0;
            double kt = q.kt[i];
            double xt = 0.0, xn = 0.0;
            int ev = step_advance<false, TIME, CE>(W, W.prob[p.prob], p, q.gslot[i], R, rep, kind, which,
                                                uk, kt, nullptr, nullptr, nullptr, &xt, &xn);
            if (CE) {
                q.sg[i] = xt;
                q.nf[i] = xn;
            }
            q.x[i] = p.x;
            q.y[i] = p.y;
            q.z[i] = p.z;
            if (TIME) q.t[i] = p.t;
            q.s[i] = p.s;
            q.kt[i] = kt;
            q.evw[i] = pack_ev(ev, kind, which);
            if (CE) q.uk[i] = uk;
            if (ev == EV_DEAD) {
                q.fate[i] = p.fate;
                retire(q, G, i, p);
            }
        }
        __syncwarp();
        int n_x = warp_list<PW>(q.list, [&](int i) {
            return q.fate[i] == FATE_ALIVE && (q.evw[i] & 15) == EV_CROSS;
        });
        for (int k = lane; k < n_x; k += 32) {
            int i = q.list[k];
            PS p;
            pool_load<TIME, CE>(q, i, p);
            int ev = step_cross(W, p, ev_kind(q.evw[i]), ev_which(q.evw[i]));
            pool_store<TIME, CE>(q, i, p);
            if (ev == EV_DEAD) retire(q, G, i, p);
        }
        __syncwarp();
        int n_c = warp_list<PW>(q.list, [&](int i) {
            return q.fate[i] == FATE_ALIVE && (q.evw[i] & 15) == EV_COLLIDE;
        });
        for (int k = lane; k < n_c; k += 32) {
            int i = q.list[k];
            PS p;
            pool_load<TIME, CE>(q, i, p);
            double kc = q.kc[i];
            int ev = step_collide<false, TIME, CE>(W, W.prob[p.prob], p, q.gslot[i], Bdst, R, CE ? q.uk[i] : 0, kc,
                                                   nullptr, CE, CE ? q.sg[i] : 0.0, CE ? q.nf[i] : 0.0);
            q.kc[i] = kc;
            q.evw[i] = EV_ADVANCE;
            pool_store<TIME, CE>(q, i, p);
            if (ev == EV_DEAD) retire(q, G, i, p);
        }
        __syncwarp();
    }
}

template <int PW, bool TIME, bool CE>
void launch_wpool_t(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                    const RunBufs &R, const PersistentArgs &a, int grid, cudaStream_t st)
{
    size_t sm = pool_bytes(PW, TIME, CE) * (WPOOL_T / 32);
    cudaFuncSetAttribute(k_wpool<PW, TIME, CE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_wpool<PW, TIME, CE><<<grid, WPOOL_T, sm, st>>>(W, G, Bsrc, Bdst, R, a);
}

template <int PW, bool CE> int wpool_occupancy()
{
    int n = 0;
    size_t sm = pool_bytes(PW, false, CE) * (WPOOL_T / 32);
    cudaFuncSetAttribute(k_wpool<PW, false, CE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_wpool<PW, false, CE>, WPOOL_T, sm);
    return n;
}

template <int P, int T, bool TIME, bool CE>
void launch_pool_t(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                   const RunBufs &R, const PersistentArgs &a, int grid, cudaStream_t st)
{
    size_t sm = pool_bytes(P, TIME, CE);
    cudaFuncSetAttribute(k_pool<P, T, TIME, CE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_pool<P, T, TIME, CE><<<grid, T, sm, st>>>(W, G, Bsrc, Bdst, R, a);
}

template <int P, int T, bool CE> int pool_occupancy()
{
    int n = 0;
    size_t sm = pool_bytes(P, false, CE);
    cudaFuncSetAttribute(k_pool<P, T, false, CE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pool<P, T, false, CE>, T, sm);
    return n;
}

// pool codes: 32, 64, 128 = particles per warp (warp-level lists, 128-thread
// blocks); 256, 512, 1024 = particles per 256-thread block; 2256, 2512 = 256 or
// 512 particles per 128-thread block
template <bool CE> int pool_occupancy_of(int P)
{
    switch (P) {
    case 32: return wpool_occupancy<32, CE>();
    case 64: return wpool_occupancy<64, CE>();
    case 128: return wpool_occupancy<128, CE>();
    case 256: return pool_occupancy<256, 256, CE>();
    case 512: return pool_occupancy<512, 256, CE>();
    case 1024: return pool_occupancy<1024, 256, CE>();
    case 2256: return pool_occupancy<256, 128, CE>();
    case 2512: return pool_occupancy<512, 128, CE>();
    default: return 0;
    }
}

template <bool TIME, bool CE>
bool launch_pool_of(const World &W, const Particles &G, const Bank &Bsrc, const Bank &Bdst,
                    const RunBufs &R, const PersistentArgs &a, int pool, int grid, cudaStream_t st)
{
    switch (pool) {
    case 32: launch_wpool_t<32, TIME, CE>(W, G, Bsrc, Bdst, R, a, grid, st); return true;
    case 64: launch_wpool_t<64, TIME, CE>(W, G, Bsrc, Bdst, R, a, grid, st); return true;
    case 128: launch_wpool_t<128, TIME, CE>(W, G, Bsrc, Bdst, R, a, grid, st); return true;
    case 256: launch_pool_t<256, 256, TIME, CE>(W, G, Bsrc, Bdst, R, a, grid, st); return true;
    case 512: launch_pool_t<512, 256, TIME, CE>(W, G, Bsrc, Bdst, R, a, grid, st); return true;
    case 1024: launch_pool_t<1024, 256, TIME, CE>(W, G, Bsrc, Bdst, R, a, grid, st); return true;
    case 2256: launch_pool_t<256, 128, TIME, CE>(W, G, Bsrc, Bdst, R, a, grid, st); return true;
    case 2512: launch_pool_t<512, 128, TIME, CE>(W, G, Bsrc, Bdst, R, a, grid, st); return true;
    default: return false;
    }
}

}  // namespace

}  // namespace mcgb
