// kernels_domain.cu -- spatial domain decomposition of a power iteration.
//
// Each rank owns a slab of space along one axis and transports only the
// particles inside it (Sec. 1: MC/DC decomposes the domain over MPI ranks).
// Particle state lives in slot j of the Particles arrays, j the history's
// source index in its cycle, on every rank; a flight that reaches the slab's
// boundary stops there (EV_EXPORT) with the rest of its sampled collision
// distance, and the particle's record goes to the neighbouring rank, which
// continues the same flight without a new random draw.  Fission sites keep
// (parent j, child) so that the ranks' sites put together give the single
// device's (parent, child)-ordered bank.
#include "kernels.h"
#include "steps.cuh"

namespace mcgb {

namespace {

// the rank whose slab holds coordinate c: the largest r with cuts[r] <= c
__device__ __forceinline__ int slab_of(const double *cuts, int nd, double c)
{
    int r = 0;
    while (r + 1 < nd && !(c < cuts[r + 1])) r++;
    return r;
}

__device__ __forceinline__ double axis_coord(int axis, double x, double y, double z)
{
    return axis == 0 ? x : (axis == 1 ? y : z);
}

__device__ __forceinline__ void append(int *list, int *n, int j)
{
    list[atomicAdd(n, 1)] = j;
}

__device__ __forceinline__ void store_state(const Particles &P, int j, const PS &p, double drem,
                                            double kt, double kc)
{
    P.x[j] = p.x; P.y[j] = p.y; P.z[j] = p.z;
    P.u[j] = p.u; P.v[j] = p.v; P.w[j] = p.w;
    P.iu[j] = p.iu; P.iv[j] = p.iv; P.iw[j] = p.iw;
    P.E[j] = p.E;
    P.s[j] = p.s;
    P.g[j] = p.g; P.cell[j] = p.cell; P.ix[j] = p.ix; P.iy[j] = p.iy; P.ucell[j] = p.ucell;
    P.mat[j] = p.mat; P.prob[j] = p.prob; P.root[j] = p.root;
    P.nfis[j] = p.nfis; P.ncoll[j] = p.ncoll; P.ncross[j] = p.ncross;
    P.fate[j] = (signed char)p.fate;
    P.drem[j] = drem;
    P.kt[j] = kt;
    P.kc[j] = kc;
}

__device__ __forceinline__ void load_state(const Particles &P, int j, PS &p)
{
    p.x = P.x[j]; p.y = P.y[j]; p.z = P.z[j];
    p.u = P.u[j]; p.v = P.v[j]; p.w = P.w[j];
    p.iu = P.iu[j]; p.iv = P.iv[j]; p.iw = P.iw[j];
    p.E = P.E[j];
    p.t = 0.0;
    p.s = P.s[j];
    p.g = P.g[j]; p.cell = P.cell[j]; p.ix = P.ix[j]; p.iy = P.iy[j]; p.ucell = P.ucell[j];
    p.mat = P.mat[j]; p.prob = P.prob[j]; p.root = P.root[j];
    p.nfis = P.nfis[j]; p.ncoll = P.ncoll[j]; p.ncross = P.ncross[j];
    p.fate = FATE_ALIVE;
}

// Sources of cycle `gen` for every history j: the source definition (cycle
// 0), or the global ordered bank resampled systematically (site_index_of, the
// same rule as a single device), born with the history's own stream.  Every
// rank evaluates the position of every source; only the owner of the slab
// holding it births it (the draws of a birth are the history's own) and
// lists it; the others mark the slot as elsewhere.  All slots' k partial sums
// are cleared.
template <bool CE>
__global__ void k_dom_sources(World W, Particles P, Bank none, int gen, int64_t N,
                              const ShardSite *bank, int64_t M, double xi, DomainCut dom,
                              const double *cuts, int nd, int rank, int *list, int *n_list,
                              int *err)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    P.kt[j] = 0.0;
    P.kc[j] = 0.0;
    P.drem[j] = -1.0;
    const ProblemDev &Pd = W.prob[0];
    PS p;
    if (!bank) {
        bool ok = init_particle<CE>(W, Pd, none, p, 0, j, gen, -1, true);
        if (!ok) {   // reported to the host by every rank; the run stops
            atomicOr(err, ERR_SOURCE);
            P.fate[j] = FATE_ELSEWHERE;
            return;
        }
        if (slab_of(cuts, nd, axis_coord(dom.axis, p.x, p.y, p.z)) != rank) {
            P.fate[j] = FATE_ELSEWHERE;
            return;
        }
    } else {
        // the birth of init_particle from a bank site, read from a record
        const ShardSite &b = bank[site_index_of(j, xi, M, N)];
        if (slab_of(cuts, nd, axis_coord(dom.axis, b.x, b.y, b.z)) != rank) {
            P.fate[j] = FATE_ELSEWHERE;
            return;
        }
        p.s = rng_stream(Pd.seed, ((uint64_t)gen << 32) + (uint64_t)j);
        p.prob = 0;
        p.nfis = 0;
        p.ncoll = 0;
        p.ncross = 0;
        p.fate = FATE_ALIVE;
        p.g = 0;
        p.E = 0.0;
        p.root = (int)j;
        p.x = b.x;
        p.t = 0.0;
        p.y = b.y;
        p.z = b.z;
        p.cell = b.cell;
        p.ix = b.ix;
        p.iy = b.iy;
        p.ucell = b.ucell;
        p.mat = b.mat;
        birth_energy<CE>(W, Pd, p);
        iso_dir(p.s, p.u, p.v, p.w);
        set_recip(W, p);
    }
    store_state(P, (int)j, p, -1.0, 0.0, 0.0);
    append(list, n_list, (int)j);
}

// Transport every listed particle until it dies or leaves the slab: one
// thread runs one history at a time, taking the next from a work counter.
template <bool CE>
__global__ void __launch_bounds__(256) k_dom_sweep(World W, Particles P, Bank Bdst, RunBufs R,
                                                   const int *list, int n, int *work,
                                                   DomainCut dom, int *outbox, int *n_out)
{
    const int rep = (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) % (unsigned)W.nrep);
    for (;;) {
        int k = atomicAdd(work, 1);
        if (k >= n) break;
        const int j = list[k];
        PS p;
        load_state(P, j, p);
        double drem = P.drem[j], kt = P.kt[j], kc = P.kc[j];
        const ProblemDev &Pd = W.prob[p.prob];
        int ev;
        for (;;) {
            int kind, which, uk = 0;
            double xt = 0.0, xn = 0.0;
            ev = step_advance<false, false, CE, true>(W, Pd, p, j, R, rep, kind, which, uk, kt,
                                                      nullptr, &dom, &drem, &xt, &xn);
            if (ev == EV_CROSS) ev = step_cross(W, p, kind, which);
            else if (ev == EV_COLLIDE)
                ev = step_collide<false, false, CE>(W, Pd, p, j, Bdst, R, uk, kc, nullptr, true, xt, xn);
            if (ev == EV_DEAD || ev == EV_EXPORT) break;
        }
        if (ev == EV_EXPORT) {
            p.fate = FATE_MOVED;
            append(outbox, n_out, j);
        }
        store_state(P, j, p, drem, kt, kc);
    }
}

// Records of the particles leaving: addressed to the neighbour ahead along
// the axis (the particle stopped on the slab's boundary moving outward).
__global__ void k_dom_pack(Particles P, const int *outbox, int n, DomainCut dom, int rank,
                           FlightRec *out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int j = outbox[k];
    FlightRec r;
    r.x = P.x[j]; r.y = P.y[j]; r.z = P.z[j];
    r.u = P.u[j]; r.v = P.v[j]; r.w = P.w[j];
    r.E = P.E[j];
    r.drem = P.drem[j];
    r.s = P.s[j];
    r.hist = j;
    r.g = P.g[j]; r.cell = P.cell[j]; r.ix = P.ix[j]; r.iy = P.iy[j]; r.ucell = P.ucell[j];
    r.mat = P.mat[j]; r.prob = P.prob[j]; r.root = P.root[j];
    r.nfis = P.nfis[j]; r.ncoll = P.ncoll[j]; r.ncross = P.ncross[j];
    const double dir = dom.axis == 0 ? r.u : (dom.axis == 1 ? r.v : r.w);
    r.dest = dir > 0.0 ? rank + 1 : rank - 1;
    out[k] = r;
}

// Particles arriving: the records addressed to this rank go to their slots
// (direction reciprocals rounded again from the direction: the same values)
// and onto the list.  The k partial sums of the slot continue what this rank
// ran up on an earlier visit of the history (0 on its first).
__global__ void k_dom_unpack(World W, Particles P, const FlightRec *in, int64_t n, int rank,
                             int *list, int *n_list)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const FlightRec &r = in[k];
    if (r.dest != rank) return;
    PS p;
    p.x = r.x; p.y = r.y; p.z = r.z;
    p.u = r.u; p.v = r.v; p.w = r.w;
    set_recip(W, p);
    if (!W.need_iw) p.iw = 0.0;
    p.E = r.E;
    p.t = 0.0;
    p.s = r.s;
    p.g = r.g; p.cell = r.cell; p.ix = r.ix; p.iy = r.iy; p.ucell = r.ucell; p.mat = r.mat;
    p.prob = r.prob; p.root = r.root; p.nfis = r.nfis; p.ncoll = r.ncoll; p.ncross = r.ncross;
    p.fate = FATE_ALIVE;
    const int j = (int)r.hist;
    store_state(P, j, p, r.drem, P.kt[j], P.kc[j]);
    append(list, n_list, j);
}

// The rank's share of the cycle end: the k partial sums of every slot (those
// a particle ran up while in this slab), the event counters and the site
// counts of the histories that ended here (0 for the others).
__global__ void k_dom_reduce(Particles P, int64_t N, double *ksum, unsigned long long *cnt,
                             int *nfis_out)
{
    double kt = 0.0, kc = 0.0;
    unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int f = P.fate[i];
        if (f != FATE_ELSEWHERE) {
            kt += P.kt[i];
            kc += P.kc[i];
        }
        const bool ended = f >= FATE_ABSORBED && f <= FATE_TIME;
        nfis_out[i] = ended ? P.nfis[i] : 0;
        if (ended) {
            c[0] += P.ncoll[i];
            c[1] += P.ncross[i];
            c[2] += f == FATE_LEAKED;
            c[3] += f == FATE_LOST;
            c[4] += f == FATE_CAPPED;
            c[5] += f == FATE_TIME;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kt += __shfl_down_sync(0xffffffffu, kt, o);
        kc += __shfl_down_sync(0xffffffffu, kc, o);
#pragma unroll
        for (int q = 0; q < 6; q++) c[q] += __shfl_down_sync(0xffffffffu, c[q], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(ksum, kt);
        atomicAdd(ksum + 1, kc);
#pragma unroll
        for (int q = 0; q < 6; q++)
            if (c[q]) atomicAdd(cnt + q, c[q]);
    }
}

// The sites banked in this slab as records (append order), parents global
__global__ void k_dom_sites(Bank B, int64_t m, ShardSite *out)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    ShardSite s;
    s.x = B.x[k]; s.y = B.y[k]; s.z = B.z[k]; s.t = B.t[k];
    s.cell = B.cell[k]; s.ix = B.ix[k]; s.iy = B.iy[k]; s.ucell = B.ucell[k]; s.mat = B.mat[k];
    s.child = B.child[k];
    s.parent = B.parent[k];
    out[k] = s;
}

// Every rank's sites in (parent, child) order: site (j, c) goes to off[j] + c,
// off the exclusive scan of the histories' site counts.
__global__ void k_dom_place(const ShardSite *in, int64_t m, const int *off, ShardSite *glob,
                            int64_t cap, int *err)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const ShardSite &s = in[k];
    int64_t pos = (int64_t)off[s.parent] + s.child;
    if (pos < 0 || pos >= cap) {
        atomicOr(err, ERR_BANK_OVERFLOW);
        return;
    }
    glob[pos] = s;
}

// Per-history records of the histories that ended in this slab (0 elsewhere)
__global__ void k_dom_records(Particles P, int64_t N, int *nc, int *nx, int *nf, int *fate, int *g,
                              unsigned long long *rng)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int f = P.fate[i];
    const bool ended = f >= FATE_ABSORBED && f <= FATE_TIME;
    nc[i] = ended ? P.ncoll[i] : 0;
    nx[i] = ended ? P.ncross[i] : 0;
    nf[i] = ended ? P.nfis[i] : 0;
    fate[i] = ended ? f : 0;
    g[i] = ended ? P.g[i] : 0;
    rng[i] = ended ? (unsigned long long)P.s[i] : 0ULL;
}

inline int blocks_for(int64_t n) { return (int)((n + 255) / 256); }

}  // namespace

void launch_dom_sources(const World &W, const Particles &P, int gen, int64_t N,
                        const ShardSite *bank, int64_t M, double xi, const DomainCut &dom,
                        const double *cuts, int nd, int rank, int *list, int *n_list, int *err,
                        cudaStream_t st)
{
    Bank none{};
    if (W.ce_any)
        k_dom_sources<true><<<blocks_for(N), 256, 0, st>>>(W, P, none, gen, N, bank, M, xi, dom,
                                                           cuts, nd, rank, list, n_list, err);
    else
        k_dom_sources<false><<<blocks_for(N), 256, 0, st>>>(W, P, none, gen, N, bank, M, xi, dom,
                                                            cuts, nd, rank, list, n_list, err);
}

void launch_dom_sweep(const World &W, const Particles &P, const Bank &Bdst, const RunBufs &R,
                      const int *list, int n, int *work, const DomainCut &dom, int *outbox,
                      int *n_out, int grid, cudaStream_t st)
{
    if (n <= 0) return;
    if (W.ce_any)
        k_dom_sweep<true><<<grid, 256, 0, st>>>(W, P, Bdst, R, list, n, work, dom, outbox, n_out);
    else
        k_dom_sweep<false><<<grid, 256, 0, st>>>(W, P, Bdst, R, list, n, work, dom, outbox, n_out);
}

void launch_dom_pack(const Particles &P, const int *outbox, int n, const DomainCut &dom, int rank,
                     FlightRec *out, cudaStream_t st)
{
    if (n > 0) k_dom_pack<<<blocks_for(n), 256, 0, st>>>(P, outbox, n, dom, rank, out);
}

void launch_dom_unpack(const World &W, const Particles &P, const FlightRec *in, int64_t n, int rank,
                       int *list, int *n_list, cudaStream_t st)
{
    if (n > 0) k_dom_unpack<<<blocks_for(n), 256, 0, st>>>(W, P, in, n, rank, list, n_list);
}

void launch_dom_reduce(const Particles &P, int64_t N, double *ksum, unsigned long long *cnt,
                       int *nfis_out, cudaStream_t st)
{
    k_dom_reduce<<<608, 256, 0, st>>>(P, N, ksum, cnt, nfis_out);
}

void launch_dom_sites(const Bank &B, int64_t m, ShardSite *out, cudaStream_t st)
{
    if (m > 0) k_dom_sites<<<blocks_for(m), 256, 0, st>>>(B, m, out);
}

void launch_dom_place(const ShardSite *in, int64_t m, const int *off, ShardSite *glob, int64_t cap,
                      int *err, cudaStream_t st)
{
    if (m > 0) k_dom_place<<<blocks_for(m), 256, 0, st>>>(in, m, off, glob, cap, err);
}

void launch_dom_records(const Particles &P, int64_t N, int *nc, int *nx, int *nf, int *fate, int *g,
                        unsigned long long *rng, cudaStream_t st)
{
    if (N > 0) k_dom_records<<<blocks_for(N), 256, 0, st>>>(P, N, nc, nx, nf, fate, g, rng);
}

}  // namespace mcgb
