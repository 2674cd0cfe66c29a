// steps.cuh -- the three events of a particle (Sec. 2: a segment of transport
// is a flight to the next event, then a surface crossing or a collision),
// written once and used by both the one-kernel-per-event path and the
// persistent event loop.
#pragma once
#include "transport.cuh"

namespace mcgb {

enum { EV_ADVANCE = 0, EV_CROSS = 1, EV_COLLIDE = 2, EV_DEAD = 3, EV_EXPORT = 4 };


__device__ __forceinline__ int tally_batch(const ProblemDev &P, const PS &p)
{
    return P.batches > 1 ? (int)(((int64_t)p.root * P.batches) / P.n) : 0;
}

// Flight: distance to collision d_c = -ln(xi) / Sigma_t (one draw, always taken),
// distance to the nearest boundary d_s, move by min(d_c, d_s) (ties cross),
// score the track length.  Returns EV_CROSS, EV_COLLIDE or EV_DEAD (lost or cut).
// REPLAY: same draws and moves, no tallies; the flight length is returned in d.
// TIME = false: the world has no time dependence (the clock is compiled out).
// CE = false: the world has no continuous-energy problem (that physics is
// compiled out: a smaller kernel with fewer registers and spills).
// DOM: the flight also stops where it leaves the slab *dom (EV_EXPORT), and
// *drem carries the rest of the sampled collision distance to the next flight
// (which then takes no draw; *drem < 0: sample as usual).
// xs_t, xs_nf (continuous energy): receive the flight's Sigma_t and its
// collision estimate of k, nuSigma_f (1/Sigma_t), which a collision at the
// flight's end takes instead of looking them up again.
template <bool REPLAY = false, bool TIME = true, bool CE = true, bool DOM = false>
__device__ __forceinline__ int step_advance(const World &W, const ProblemDev &P, PS &p, int slot,
                                            const RunBufs &R, int rep, int &kind, int &which,
                                            int &uk, double &kt, double *d_out = nullptr,
                                            const DomainCut *dom = nullptr, double *drem = nullptr,
                                            double *xs_t = nullptr, double *xs_nf = nullptr)
{
    if (p.ncoll + p.ncross >= MAX_EVENTS) {
        p.fate = FATE_CAPPED;
        return EV_DEAD;
    }
    double sigt, mfp, nusf;
    if (CE && P.ce) {
        ce_macro(W, p.mat, p.E, sigt, nusf);
        mfp = is_pos(sigt) ? rcp_rn(sigt) : MCGB_INF;   // correctly rounded 1 / sigt
        if (xs_t) {
            *xs_t = sigt;
            *xs_nf = nusf * mfp;
        }
    } else {
        int go = __ldg(W.m_goff + p.mat) + p.g;
        sigt = __ldg(W.g_sigt + go);
        nusf = __ldg(W.g_nusf + go);
        mfp = __ldg(W.g_mfp + go);
    }
    double dc;
    if (DOM && !is_neg(*drem)) {
        dc = *drem;     // the rest of a flight cut at the slab's boundary
    } else {
        uint64_t n = draw_n(p.s);
        dc = is_pos(sigt) ? -log_n(W, n) * mfp : MCGB_INF;
    }
    if (DOM) *drem = -1.0;
    double ds = boundary(W, p, kind, which);
    const bool timed = TIME && P.time_on;
    if (!timed && is_inf(dc) && is_inf(ds)) {
        p.fate = FATE_LOST;
        return EV_DEAD;
    }
    bool coll = lt_mag(dc, ds);     // both are +-0, positive or +inf
    double d = coll ? dc : ds;
    bool leaves = false;
    if (DOM) {
        // distance to the slab's boundary ahead along its axis; strictly
        // nearer than the collision and the surface: the particle stops there
        const double c = dom->axis == 0 ? p.x : (dom->axis == 1 ? p.y : p.z);
        const double dir = dom->axis == 0 ? p.u : (dom->axis == 1 ? p.v : p.w);
        double tdom = MCGB_INF;
        if (is_pos(dir) && !is_inf(dom->hi)) tdom = div_rn(dom->hi - c, dir);
        else if (is_neg(dir) && !is_inf(-dom->lo)) tdom = div_rn(dom->lo - c, dir);
        if (is_neg(tdom)) tdom = 0.0;
        if (lt_mag(tdom, d)) {
            leaves = true;
            *drem = dc - tdom;    // +inf stays +inf
            d = tdom;
        }
    }
    // time dependence: the flight ends where the clock reaches tcut, at the
    // distance (tcut - t) / (1/v); a tie goes to the collision or crossing
    bool tcut = false;
    const double ta = p.t;
    double tb = p.t;
    if (timed) {
        double iv = (CE && P.ce) ? rcp_rn(W.kv * sqrt_rn(p.E)) : __ldg(W.g_invv + P.invv_off + p.g);
        double dt = div_rn(P.tcut - p.t, iv);
        if (is_neg(dt)) dt = 0.0;
        if (lt_mag(dt, d)) {
            tcut = true;
            d = dt;
        }
        if (!tcut && is_inf(d)) {
            p.fate = FATE_LOST;
            return EV_DEAD;
        }
        tb = tcut ? P.tcut : fma(d, iv, p.t);
    }
    p.x = fma(d, p.u, p.x);
    p.y = fma(d, p.v, p.y);
    p.z = fma(d, p.w, p.z);
    if (REPLAY) {
        *d_out = d;
    } else {
        score<TIME, CE>(W, P, p, d, tally_batch(P, p), R.tacc, rep, ta, tb);
        kt = fma(d, nusf, kt);   // a sum over histories: agreement within rounding only
        if (R.own && (p.ucell >= 0 ? p.ucell : p.cell) == R.own_cell)
            R.own[(int64_t)slot * R.own_G + p.g] += d;
    }
    if (TIME) p.t = tb;
    if (tcut) {
        p.fate = FATE_TIME;
        return EV_DEAD;
    }
    if (DOM && leaves) return EV_EXPORT;
    return coll ? EV_COLLIDE : EV_CROSS;
}

__device__ __forceinline__ int step_cross(const World &W, PS &p, int kind, int which)
{
    p.ncross++;
    int r = cross(W, p, kind, which);
    if (r == 1) {
        p.fate = FATE_LEAKED;
        return EV_DEAD;
    }
    if (r < 0) {
        p.fate = FATE_LOST;
        return EV_DEAD;
    }
    return EV_ADVANCE;
}

// Collision (analog, weight 1).  Multigroup: fission sites floor(mu) + [xi1 <=
// frac mu], mu = nuSigma_f/Sigma_t (no division by k); scatter when xi2 <=
// Sigma_s,tot/Sigma_t with outgoing group the first g' where xi3 <= cdf(g');
// isotropic direction; otherwise absorbed.  Continuous energy: nuclide by
// xi Sigma_t against the running sum, fission sites as above with nu sigma_f /
// sigma_t of that nuclide, scatter (elastic, target at rest) when
// xi sigma_t <= sigma_s.
// REPLAY (multigroup only): same draws, no bank; *nf_out = sites banked.
// xs_given (continuous energy): xs_t, xs_nf are Sigma_t and nuSigma_f (1/Sigma_t)
// of the flight that ended here (same material and energy), not looked up again.
template <bool REPLAY = false, bool TIME = true, bool CE = true>
__device__ __forceinline__ int step_collide(const World &W, const ProblemDev &P, PS &p, int slot,
                                            const Bank &B, const RunBufs &R, int uk, double &kc,
                                            int *nf_out = nullptr, bool xs_given = false,
                                            double xs_t = 0.0, double xs_nf = 0.0)
{
    p.ncoll++;
    if (!CE || !P.ce) {
        int go = __ldg(W.m_goff + p.mat);
        int G = __ldg(W.m_G + p.mat);
        int g = p.g;
        kc = kc + __ldg(W.g_mu + go + g);
        double xi = draw(p.s);
        int nf = (int)__ldg(W.g_mufl + go + g) + (lt_mag(__ldg(W.g_mufr + go + g), xi) ? 0 : 1);
        if (REPLAY) {
            *nf_out = nf;
            p.nfis += nf;
        } else {
            bank_append<TIME>(B, R.bank_n, R.err, p, slot, nf);
        }
        xi = draw(p.s);
        if (!lt_mag(__ldg(W.g_ps + go + g), xi)) {
            xi = draw(p.s);
            p.g = sample_cdf(W.gg_scdf + __ldg(W.m_ggoff + p.mat) + g * G, G, xi);
            iso_dir(p.s, p.u, p.v, p.w);
            set_recip(W, p);
        } else {
            p.fate = FATE_ABSORBED;
            return EV_DEAD;
        }
    } else {
        double sigt, kterm;   // k_c scores nuSigma_f / Sigma_t as nuSigma_f (1/Sigma_t)
        if (xs_given) {
            sigt = xs_t;
            kterm = xs_nf;
        } else {
            double nusf;
            ce_macro(W, p.mat, p.E, sigt, nusf);
            kterm = nusf * rcp_rn(sigt);
        }
        uk = union_index(W, p.E);   // per-nuclide values for the reaction
        kc = kc + kterm;
        int off = __ldg(W.mc_off + p.mat), n = __ldg(W.mc_n + p.mat);
        // nuclide: first whose running sum of N_i sigma_t,i (each term fused into
        // the sum) reaches xi Sigma_t
        double target = draw(p.s) * sigt;
        double cum = 0.0;
        int sel = n - 1;
        double st = 0.0, ss = 0.0, sf = 0.0;
        for (int q = 0; q < n; q++) {
            double a, b, c;
            ce_micro(W, __ldg(W.mc_nuc + off + q), uk, p.E, a, b, c);
            cum = fma(__ldg(W.mc_dens + off + q), a, cum);
            st = a;
            ss = b;
            sf = c;
            if (!lt_mag(cum, target)) {
                sel = q;
                break;
            }
        }
        int nuc = __ldg(W.mc_nuc + off + sel);
        double mu = div_rn(__ldg(W.n_nu + nuc) * sf, st);
        double fl;
        const int nfl = floor_nonneg(mu, fl);
        double xi = draw(p.s);
        int nf = nfl + (lt_mag(mu - fl, xi) ? 0 : 1);
        bank_append<TIME>(B, R.bank_n, R.err, p, slot, nf);
        xi = draw(p.s);
        if (!lt_mag(ss, xi * st)) {
            if (is_pos(P.fg_kT) && lt_mag(p.E, P.fg_emax))
                p.E = free_gas(W, p.E, W.n_kin + 6 * nuc, P.fg_kT, P.fg_ikT, p.s, p.u, p.v, p.w);
            else
                p.E = elastic(p.E, W.n_kin + 6 * nuc, p.s, p.u, p.v, p.w);
            set_recip(W, p);
        } else {
            p.fate = FATE_ABSORBED;
            return EV_DEAD;
        }
    }
    if (P.max_coll && p.ncoll >= P.max_coll) {
        p.fate = FATE_CUT;
        return EV_DEAD;
    }
    return EV_ADVANCE;
}

// New particle for slot `slot` (local index `local` of its problem) of
// generation/cycle `gen`: stream gen 2^32 + local; from the source definition
// (site < 0) or born at bank site `site`.
template <bool CE = true>
__device__ __forceinline__ bool init_particle(const World &W, const ProblemDev &P, const Bank &B,
                                              PS &p, int prob, int64_t local, int gen, int site,
                                              bool eigen)
{
    p.s = rng_stream(P.seed, ((uint64_t)gen << 32) + (uint64_t)local);
    p.prob = prob;
    p.nfis = 0;
    p.ncoll = 0;
    p.ncross = 0;
    p.fate = FATE_ALIVE;
    p.g = 0;
    p.E = 0.0;
    p.ix = -1;
    p.iy = -1;
    p.ucell = -1;
    if (site < 0) {
        p.root = (int)local;
        return sample_source<CE>(W, P, p);
    }
    p.root = eigen ? (int)local : B.root[site];
    birth_from_site<CE>(W, P, B, site, p);
    return true;
}

// The birth of slot j that launch_source stored in the particle arrays (fields
// a world does not use are not read); false when the source could not place
// the particle (k_source raised the error and stored it as lost).
template <bool TIME = true, bool CE = true>
__device__ __forceinline__ bool load_born(const World &W, const Particles &G, int64_t j, PS &p)
{
    p.x = G.x[j]; p.y = G.y[j]; p.z = G.z[j];
    p.u = G.u[j]; p.v = G.v[j]; p.w = G.w[j];
    p.iu = G.iu[j]; p.iv = G.iv[j]; p.iw = W.need_iw ? G.iw[j] : 0.0;
    p.E = CE ? G.E[j] : 0.0;
    p.t = TIME ? G.t[j] : 0.0;
    p.s = G.s[j];
    p.g = G.g[j]; p.cell = G.cell[j]; p.ix = G.ix[j]; p.iy = G.iy[j]; p.ucell = G.ucell[j];
    p.mat = G.mat[j]; p.prob = G.prob[j]; p.root = G.root[j];
    p.nfis = 0;
    p.ncoll = 0;
    p.ncross = 0;
    p.fate = G.fate[j];
    return p.fate == FATE_ALIVE;
}

// Block-aggregated append of `val` to queue a when pa holds and to queue b when
// pb holds: each warp counts its lanes with a ballot, the warps reserve their
// places in the block's share with shared-memory atomics, and one thread takes
// the block's share of each queue with a single global atomic (one per block
// instead of one per warp: the queue counters are the only addresses every
// block of the launch updates).  Every thread of the block must call it, with
// a block size a multiple of 32; qb may be null (one queue).
__device__ __forceinline__ void enqueue2(bool pa, bool pb, int val, int *qa, int *na, int *qb, int *nb)
{
    __shared__ int s_n[2], s_base[2];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_n[0] = 0;
        s_n[1] = 0;
    }
    __syncthreads();
    const unsigned ma = __ballot_sync(0xffffffffu, pa), mb = __ballot_sync(0xffffffffu, pb);
    int wa = 0, wb = 0;
    if (lane == 0) {
        if (ma) wa = atomicAdd(&s_n[0], __popc(ma));
        if (mb) wb = atomicAdd(&s_n[1], __popc(mb));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_base[0] = s_n[0] ? atomicAdd(na, s_n[0]) : 0;
        s_base[1] = s_n[1] ? atomicAdd(nb, s_n[1]) : 0;
    }
    __syncthreads();
    wa = __shfl_sync(0xffffffffu, wa, 0);
    wb = __shfl_sync(0xffffffffu, wb, 0);
    const unsigned lt = (1u << lane) - 1u;
    if (pa) qa[s_base[0] + wa + __popc(ma & lt)] = val;
    if (pb) qb[s_base[1] + wb + __popc(mb & lt)] = val;
}

__device__ __forceinline__ void enqueue(bool pred, int val, int *queue, int *count)
{
    enqueue2(pred, false, val, queue, count, nullptr, nullptr);
}

}  // namespace mcgb
