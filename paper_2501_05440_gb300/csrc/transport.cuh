// transport.cuh -- device functions of event-based Monte Carlo transport.
//
// One particle's steps (Sec. 2 of the paper lists them as sampling a
// direction, moving the particle, and so on; Sec. 1 names the physics):
//   sample a distance to collision, find the nearest CSG boundary, move and
//   score the track length, then cross the boundary or collide.
// The paper gives no formulas.  The choices made here (random-number
// generator, draw order, root selection, tie-breaks, estimators) are stated
// beside each function; every floating-point expression is evaluated in the
// order written, without contraction (the library is built with -fmad=false),
// so that each history is bit-reproducible on any conforming IEEE machine.
#pragma once
#include <cooperative_groups.h>

#include <cstdint>

#include "fpint.cuh"
#include "world.h"

namespace mcgb {

#define MCGB_INF __longlong_as_double(0x7FF0000000000000LL)

// Comparisons done on the bit patterns (integer pipe) instead of the FP64 pipe.
// Exact for all non-NaN values: is_neg(x) == (x < 0.0), is_pos(x) == (x > 0.0);
// lt_mag(a, b) == (a < b) when a and b are +-0, positive or +inf.
__device__ __forceinline__ bool is_neg(double x)
{
    long long b = __double_as_longlong(x);
    return b < 0 && b != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool is_pos(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool lt_mag(double a, double b)
{
    return (__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFLL) <
           (__double_as_longlong(b) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ bool is_inf(double x)
{
    return __double_as_longlong(x) == 0x7FF0000000000000LL;
}
// x > c for a positive constant c: exact for every non-NaN x (negative x have
// negative bit patterns).
__device__ __forceinline__ bool gt_pos(double x, double c)
{
    return __double_as_longlong(x) > __double_as_longlong(c);
}

// floor(mu) for a finite mu >= 0, as a double and as an integer, from the bits
// (no FP64 instruction): the fraction bits below the units place cleared.
__device__ __forceinline__ int floor_nonneg(double mu, double &fl)
{
    const uint64_t b = (uint64_t)__double_as_longlong(mu);
    const int e = (int)(b >> 52) - 1023;
    if (e < 0) {
        fl = 0.0;
        return 0;
    }
    if (e > 30) {   // beyond any fission yield; kept exact all the same
        fl = floor(mu);
        return (int)fl;
    }
    fl = __longlong_as_double((long long)(b & ~((1ULL << (52 - e)) - 1)));
    return (int)((((b & ((1ULL << 52) - 1)) | (1ULL << 52)) >> (52 - e)));
}

// ---------------------------------------------------------------------------
// Random numbers (Sec. 1: replicable on CPU and GPU).  63-bit LCG
// s' = (g s + 1) mod 2^63, g = 2806196910506780709; stream i starts at
// skip(seed, 152917 i) (Brown's skip-ahead); a draw advances the state and
// returns xi = n 2^-53 with n = (s >> 10) + 1 in [1, 2^53].
constexpr uint64_t LCG_G = 2806196910506780709ULL;
constexpr uint64_t LCG_MASK = 0x7FFFFFFFFFFFFFFFULL;
constexpr uint64_t LCG_STRIDE = 152917ULL;

__host__ __device__ __forceinline__ uint64_t rng_next(uint64_t s)
{
    return (LCG_G * s + 1ULL) & LCG_MASK;
}

__host__ __device__ __forceinline__ uint64_t rng_skip(uint64_t s, uint64_t n)
{
    uint64_t G = 1, C = 0, h = LCG_G, f = 1;
    n &= LCG_MASK;
    while (n) {
        if (n & 1) {
            G = G * h;
            C = C * h + f;
        }
        f = f * (h + 1);
        h = h * h;
        n >>= 1;
    }
    return (G * (s & LCG_MASK) + C) & LCG_MASK;
}

__host__ __device__ __forceinline__ uint64_t rng_stream(uint64_t seed, uint64_t id)
{
    return rng_skip(seed, id * LCG_STRIDE);
}

__device__ __forceinline__ uint64_t draw_n(uint64_t &s)
{
    s = rng_next(s);
    return (s >> 10) + 1;
}

// n 2^-53 for 1 <= n <= 2^53, built from the bits (exact; no FP64 instruction).
__device__ __forceinline__ double n_to_xi(uint64_t n)
{
    int lz = __clzll((long long)n);
    uint64_t frac = ((n << lz) << 1) >> 12;
    uint64_t bits = ((uint64_t)(1023 - 53 + 63 - lz) << 52) | frac;
    return __longlong_as_double((long long)bits);
}

// 2 xi - 1 = (2n - 2^53) 2^-53 exactly (no FP64 instruction).
__device__ __forceinline__ double n_to_sym(uint64_t n)
{
    long long k = (long long)(2 * n) - (1LL << 53);
    if (k == 0) return 0.0;
    uint64_t a = k < 0 ? (uint64_t)(-k) : (uint64_t)k;
    int lz = __clzll((long long)a);
    uint64_t frac = ((a << lz) << 1) >> 12;
    uint64_t bits = ((uint64_t)(1023 - 53 + 63 - lz) << 52) | frac;
    if (k < 0) bits |= 0x8000000000000000ULL;
    return __longlong_as_double((long long)bits);
}

// 2 (2 xi - 1) = (2n - 2^53) 2^-52 exactly (no FP64 instruction).
__device__ __forceinline__ double n_to_sym2(uint64_t n)
{
    long long k = (long long)(2 * n) - (1LL << 53);
    if (k == 0) return 0.0;
    uint64_t a = k < 0 ? (uint64_t)(-k) : (uint64_t)k;
    int lz = __clzll((long long)a);
    uint64_t frac = ((a << lz) << 1) >> 12;
    uint64_t bits = ((uint64_t)(1023 - 52 + 63 - lz) << 52) | frac;
    if (k < 0) bits |= 0x8000000000000000ULL;
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double draw(uint64_t &s) { return n_to_xi(draw_n(s)); }
__device__ __forceinline__ double draw_sym(uint64_t &s) { return n_to_sym(draw_n(s)); }
__device__ __forceinline__ double draw_sym2(uint64_t &s) { return n_to_sym2(draw_n(s)); }

// ---------------------------------------------------------------------------
// ln xi for xi = n 2^-53, n in [1, 2^53], on the integer pipe: the table-driven
// reduction of Tang (ACM TOMS 1990) in fixed point.  n = 2^e m with m in
// [1, 2); c = 1 + j/256 from the top 8 fraction bits of m; r = (m - c)(1/c)
// in [0, 2^-8); ln xi = (e - 53) ln 2 + ln c + ln(1 + r), with
// ln(1 + r) = r (1 - r (1/2 - r (1/3 - r (1/4 - r (1/5 - r/6))))) by Horner's
// rule on 64-bit fractions (each product truncated), the sum in 57 fraction
// bits (|ln xi| < 37), then rounded once to a double.  Tables (built on the
// host): ln c and (e - 53) ln 2 rounded to 57 fraction bits, 1/c to 63.
// Error: below 2^-56 absolute and 1.2 ulp relative where |ln xi| >= 1/32.
__device__ __forceinline__ double log_n(const World &W, uint64_t n)
{
    const int lz = __clzll((long long)n);
    const uint64_t frac = ((n << lz) << 1) >> 12;   // the 52 fraction bits of m
    const int j = (int)(frac >> 44);
    const uint64_t d = frac & ((1ULL << 44) - 1);    // (m - c) 2^52, exact
    // r 2^64 = d (1/c) 2^(64 - 52), from the 107-bit product d (2^63/c)
    const uint64_t ic = __ldg(W.invc_q + j);
    const uint64_t r = (__umul64hi(d, ic) << 13) | ((d * ic) >> 51);
    uint64_t q = 0x1555555555555555ULL;               // 1/6 (63 fraction bits)
    q = 0x1999999999999999ULL - __umul64hi(r, q);     // 1/5 - r q
    q = 0x2000000000000000ULL - __umul64hi(r, q);     // 1/4
    q = 0x2AAAAAAAAAAAAAAAULL - __umul64hi(r, q);     // 1/3
    q = 0x4000000000000000ULL - __umul64hi(r, q);     // 1/2
    q = 0x8000000000000000ULL - __umul64hi(r, q);     // 1
    const uint64_t p = __umul64hi(r, q);              // ln(1 + r), 63 fraction bits
    const int64_t L = __ldg(W.eln2_q + (63 - lz)) + __ldg(W.lnc_q + j) + (int64_t)(p >> 6);
    if (L == 0) return 0.0;                           // xi = 1
    // -L 2^-57 to a double, rounded to nearest (ties to even)
    const uint64_t a = (uint64_t)(-L);
    const int z = __clzll((long long)a);
    const uint64_t x = a << z;
    uint64_t mant = x >> 11;
    const uint64_t rem = x & 0x7FF;
    mant += (rem > 0x400 || (rem == 0x400 && (mant & 1))) ? 1 : 0;
    const uint64_t bits = ((uint64_t)(63 - z - 57 + 1022) << 52) + mant;   // carries into the exponent
    return -__longlong_as_double((long long)bits);
}

// ---------------------------------------------------------------------------
// Isotropic direction by Marsaglia's disk rejection (no trigonometry): (a, b)
// uniform in the unit disk, S = a^2 + b^2 < 1, Omega = (2a sqrt(1 - S),
// 2b sqrt(1 - S), 1 - 2S).  Computed from 2a, 2b and 4S, which are exact
// scalings: the doublings fold into the draws and the fused constants, and
// every value is the one of the formula as written (S = fma(a, a, b b)).
__device__ __forceinline__ void iso_dir(uint64_t &s, double &u, double &v, double &w)
{
    // the loop repeats only the rejection test; the accepted point is used once
    double a2, b2, S4;
    int k = 0;
    do {
        a2 = draw_sym2(s);
        b2 = draw_sym2(s);
        S4 = fma(a2, a2, b2 * b2);
        k++;
    } while (!lt_mag(S4, 4.0) && k < 64);
    if (!lt_mag(S4, 4.0)) {
        u = 0.0;
        v = 0.0;
        w = 1.0;
        return;
    }
    double t = sqrt_rn(fma(-0.25, S4, 1.0));
    u = a2 * t;
    v = b2 * t;
    w = fma(-0.5, S4, 1.0);
}

// Azimuth as (cos, sin) of the doubled angle of a point uniform in the unit disk.
__device__ __forceinline__ void azimuth(uint64_t &s, double &cphi, double &sphi)
{
    double a, b, r2;
    int k = 0;
    bool ok;
    do {
        a = draw_sym(s);
        b = draw_sym(s);
        r2 = fma(a, a, b * b);
        ok = !lt_mag(1.0, r2) && is_pos(r2);
        k++;
    } while (!ok && k < 64);
    if (!ok) {
        cphi = 1.0;
        sphi = 0.0;
        return;
    }
    const double inv = rcp_rn(r2);   // correctly rounded 1 / r2
    cphi = fma(a, a, -(b * b)) * inv;
    sphi = 2.0 * a * b * inv;
}

// Rotate (u,v,w) by polar cosine mu with a sampled azimuth (polar axis z, or x near |w| = 1).
__device__ __forceinline__ void rotate(double mu, uint64_t &s, double &u, double &v, double &w)
{
    double cphi, sphi;
    azimuth(s, cphi, sphi);
    double st2 = fma(-mu, mu, 1.0);
    double st = sqrt_rn(is_pos(st2) ? st2 : 0.0);
    double u0 = u, v0 = v, w0 = w;
    double ww = fma(-w0, w0, 1.0);
    if (gt_pos(ww, 1.0e-10)) {
        double q = sqrt_rn(ww);
        double f = div_rn(st, q);
        u = fma(mu, u0, f * fma(u0 * w0, cphi, -(v0 * sphi)));
        v = fma(mu, v0, f * fma(v0 * w0, cphi, u0 * sphi));
        w = fma(mu, w0, -(st * q * cphi));
    } else {
        double uu = fma(-u0, u0, 1.0);
        double q = sqrt_rn(uu);
        double f = div_rn(st, q);
        v = fma(mu, v0, f * fma(v0 * u0, cphi, -(w0 * sphi)));
        w = fma(mu, w0, f * fma(w0 * u0, cphi, v0 * sphi));
        u = fma(mu, u0, -(st * q * cphi));
    }
}

// Elastic scattering off a target at rest; energy floored at E_MIN.  kin holds
// the nuclide's constants {A, 2A, A^2 + 1 (one rounding), 1 / (A + 1)^2, ...}:
// q = 2A mu_cm + (A^2 + 1), E' = (E q) / (A + 1)^2, mu_lab = (A mu_cm + 1) / sqrt(q).
__device__ __forceinline__ double elastic(double E, const double *kin, uint64_t &s, double &u,
                                          double &v, double &w)
{
    const double2 k01 = __ldg(reinterpret_cast<const double2 *>(kin));
    const double2 k23 = __ldg(reinterpret_cast<const double2 *>(kin) + 1);
    double mucm = draw_sym(s);
    double q = fma(k01.y, mucm, k23.x);
    double Ep = E * q * k23.y;
    double mul = div_rn(fma(k01.x, mucm, 1.0), sqrt_rn(q));
    if (lt_mag(1.0, mul)) mul = is_neg(mul) ? -1.0 : 1.0;   // |mul| > 1: clamped
    rotate(mul, s, u, v, w);
    return lt_mag(Ep, E_MIN) ? E_MIN : Ep;
}

// Maxwellian fission spectrum (T = 1.33 MeV): E = -T (ln xi1 + ln xi2 a^2/(a^2+b^2)),
// (a, b) uniform in the unit disk; resampled above 20 MeV; floored at E_MIN.
__device__ __forceinline__ double maxwell(const World &W, uint64_t &s)
{
    for (int k = 0; k < 64; k++) {
        double L1 = log_n(W, draw_n(s));
        double L2 = log_n(W, draw_n(s));
        double a = 1.0, r2 = 1.0;
        {
            double aa, bb, rr;
            int t = 0;
            bool ok;
            do {
                aa = draw_sym(s);
                bb = draw_sym(s);
                rr = fma(aa, aa, bb * bb);
                ok = !lt_mag(1.0, rr) && is_pos(rr);
                t++;
            } while (!ok && t < 64);
            if (ok) {
                a = aa;
                r2 = rr;
            }
        }
        double c2 = div_rn(a * a, r2);
        double E = -1.33e6 * (L1 + L2 * c2);
        if (!lt_mag(E_MAX, E)) return lt_mag(E, E_MIN) ? E_MIN : E;
    }
    return E_MAX;
}

// cos^2 of an angle uniform on [0, pi/2]: a^2 / (a^2 + b^2) of a point uniform
// in the unit disk (rejection, at most 64 tries; 1 if none is accepted)
__device__ __forceinline__ double disk_cos2(uint64_t &s)
{
    double aa, bb, rr;
    int t = 0;
    bool ok;
    do {
        aa = draw_sym(s);
        bb = draw_sym(s);
        rr = fma(aa, aa, bb * bb);
        ok = !lt_mag(1.0, rr) && is_pos(rr);
        t++;
    } while (!ok && t < 64);
    return ok ? div_rn(aa * aa, rr) : 1.0;
}

// Elastic scattering off a free-gas target with a constant cross section (the
// model Sec. 4 assumes for its continuous-energy pin).  Speeds in units of the
// target's thermal speed sqrt(2 kT / (A m)); the neutron's is y = sqrt(A E / kT).
// The target speed x and cosine mu (target vs neutron direction) follow the
// relative speed r = |y Omega - x Omega_T| times the Maxwellian x^2 exp(-x^2):
// proposals from (x + y) x^2 exp(-x^2) -- with probability y sqrt(pi) /
// (y sqrt(pi) + 2) from x^2 exp(-x^2) (x^2 = -(ln xi1 + ln xi2 c), c = cos^2 of
// a uniform angle), else from x^3 exp(-x^2) (x^2 = -(ln xi1 + ln xi2)) -- with
// mu = 2 xi - 1, accepted when xi (x + y) <= r.  The target direction is the
// neutron's rotated by mu.  The centre-of-mass velocity V = (y Omega +
// A x Omega_T) / (A + 1) is kept, the neutron's speed in that frame A r / (A + 1)
// is kept and its direction there is isotropic; E' = E |v'|^2 / y^2 (floored at
// 1e-5 eV), Omega' = v' / |v'|.  Rounding: y^2 = (A E)(1/kT); each product
// that is added to another term is fused into that addition; 1/(A + 1) and
// 1/A come from the nuclide's constants kin = {A, 2A, A^2 + 1, 1/(A+1)^2,
// 1/(A+1), 1/A}; E' = |v'|^2 (kT (1/A)), which is E |v'|^2 / y^2.
__device__ __forceinline__ double free_gas(const World &W, double E, const double *kin, double kT,
                                           double ikT, uint64_t &s, double &u, double &v, double &w)
{
    const double SQRT_PI = 1.7724538509055160273;
    const double A = __ldg(kin);
    const double2 k45 = __ldg(reinterpret_cast<const double2 *>(kin) + 2);   // 1/(A+1), 1/A
    const double y2 = A * E * ikT;
    const double y = sqrt_rn(y2);
    double py = y * SQRT_PI;
    double x = 0.0, mu = 1.0, r = y;
    for (int k = 0; k < MAX_TRIES; k++) {
        double x2;
        if (lt_mag(draw(s) * (py + 2.0), py)) {
            double L1 = log_n(W, draw_n(s));
            double L2 = log_n(W, draw_n(s));
            double c2 = disk_cos2(s);
            x2 = -fma(L2, c2, L1);
        } else {
            double L1 = log_n(W, draw_n(s));
            double L2 = log_n(W, draw_n(s));
            x2 = -(L1 + L2);
        }
        x = sqrt_rn(x2);
        mu = draw_sym(s);
        double r2 = fma(-(2.0 * x * y), mu, x2 + y2);
        r = sqrt_rn(is_pos(r2) ? r2 : 0.0);
        if (!lt_mag(r, draw(s) * (x + y))) break;
    }
    double tu = u, tv = v, tw = w;
    rotate(mu, s, tu, tv, tw);
    const double inv = k45.x;
    const double Ax = A * x;
    double Vx = fma(y, u, Ax * tu) * inv;
    double Vy = fma(y, v, Ax * tv) * inv;
    double Vz = fma(y, w, Ax * tw) * inv;
    double cu, cv, cw;
    iso_dir(s, cu, cv, cw);
    double wc = A * r * inv;
    double px = fma(wc, cu, Vx), py2 = fma(wc, cv, Vy), pz = fma(wc, cw, Vz);
    double p2 = fma(px, px, fma(py2, py2, pz * pz));
    double ip = rcp_rn(sqrt_rn(p2));   // correctly rounded, the same as 1.0 / sqrt(p2)
    u = px * ip;
    v = py2 * ip;
    w = pz * ip;
    double Ep = p2 * (kT * k45.y);
    return lt_mag(Ep, E_MIN) ? E_MIN : Ep;
}

// First k with xi <= cdf[k] (cdf nondecreasing, ending with exactly 1): the count
// of entries below xi, taken over the whole table (no divergent early exit).
__device__ __forceinline__ int sample_cdf(const double *cdf, int n, double xi)
{
    int k = 0;
    for (int q = 0; q < n - 1; q++) k += lt_mag(__ldg(cdf + q), xi) ? 1 : 0;
    return k;
}

// ---------------------------------------------------------------------------
// Particle held in registers
struct PS {
    double x, y, z, u, v, w, E;
    double iu, iv, iw;   // 1/u, 1/v, 1/w, rounded whenever the direction is set
    double t;            // time (s) when the problem is time dependent
    uint64_t s;
    int g, cell, ix, iy, ucell, mat, prob, root, nfis, ncoll, ncross, fate;
};

// 1/w is read only by z-planes; a world without them never computes it.
// rcp_rn is the correctly rounded reciprocal, the same value as 1.0 / x.
__device__ __forceinline__ void set_recip(const World &W, PS &p)
{
    p.iu = rcp_rn(p.u);
    p.iv = rcp_rn(p.v);
    if (W.need_iw) p.iw = rcp_rn(p.w);
}

// ---------------------------------------------------------------------------
// CSG geometry (Sec. 1: constructive solid geometry with surface tracking)
__device__ __forceinline__ double surf_f(const World &W, int sid, double x, double y, double z)
{
    const double *c = W.s_coef + 4 * sid;
    switch (__ldg(W.s_type + sid)) {
    case SURF_PX: return x - __ldg(c);
    case SURF_PY: return y - __ldg(c);
    case SURF_PZ: return z - __ldg(c);
    case SURF_PLANE: return __ldg(c) * x + __ldg(c + 1) * y + __ldg(c + 2) * z - __ldg(c + 3);
    case SURF_CYLZ: {
        double dx = x - __ldg(c), dy = y - __ldg(c + 1);
        return fma(dx, dx, dy * dy) - __ldg(W.s_r2 + sid);
    }
    default: {
        double dx = x - __ldg(c), dy = y - __ldg(c + 1), dz = z - __ldg(c + 2);
        return fma(dx, dx, fma(dy, dy, dz * dz)) - __ldg(W.s_r2 + sid);
    }
    }
}

__device__ __forceinline__ double surf_gdot(const World &W, int sid, double x, double y, double z,
                                            double u, double v, double w)
{
    const double *c = W.s_coef + 4 * sid;
    switch (__ldg(W.s_type + sid)) {
    case SURF_PX: return u;
    case SURF_PY: return v;
    case SURF_PZ: return w;
    case SURF_PLANE: return __ldg(c) * u + __ldg(c + 1) * v + __ldg(c + 2) * w;
    case SURF_CYLZ: return (x - __ldg(c)) * u + (y - __ldg(c + 1)) * v;
    default: return (x - __ldg(c)) * u + (y - __ldg(c + 1)) * v + (z - __ldg(c + 2)) * w;
    }
}

// Distance to leaving the half-space of the given sense.  The root is chosen
// from the sense (so a surface just crossed is never re-hit), quadratic roots
// use cancellation-free forms, and round-off negatives become 0.  Axis planes
// (and lattice walls) use the direction's reciprocal, t = (x0 - x)(1/u);
// quadratic terms are evaluated with fused multiply-adds.
__device__ __forceinline__ double surf_dist(const World &W, int sid, int sense, double x, double y,
                                            double z, double u, double v, double w, double iu,
                                            double iv, double iw)
{
    const double *c = W.s_coef + 4 * sid;
    int type = __ldg(W.s_type + sid);
    double t;
    if (type <= SURF_PLANE) {
        double dn, f, inv;
        switch (type) {
        case SURF_PX: dn = u; f = x - __ldg(c); inv = iu; break;
        case SURF_PY: dn = v; f = y - __ldg(c); inv = iv; break;
        case SURF_PZ: dn = w; f = z - __ldg(c); inv = iw; break;
        default:
            dn = __ldg(c) * u + __ldg(c + 1) * v + __ldg(c + 2) * w;
            f = __ldg(c) * x + __ldg(c + 1) * y + __ldg(c + 2) * z - __ldg(c + 3);
            inv = 0.0;
        }
        if ((sense > 0 && is_neg(dn)) || (sense < 0 && is_pos(dn))) {
            // axis planes use the direction's reciprocal, other planes divide
            t = type == SURF_PLANE ? div_rn(-f, dn) : -f * inv;
            return is_neg(t) ? 0.0 : t;
        }
        return MCGB_INF;
    }
    double a, b, cc;
    if (type == SURF_CYLZ) {
        double dx = x, dy = y;   // a cylinder on the axis: x - 0.0 is x
        if (!__ldg(W.s_zc + sid)) {
            dx = x - __ldg(c);
            dy = y - __ldg(c + 1);
        }
        a = fma(u, u, v * v);
        b = fma(dx, u, dy * v);
        cc = fma(dx, dx, fma(dy, dy, -__ldg(W.s_r2 + sid)));
    } else {
        double dx = x - __ldg(c), dy = y - __ldg(c + 1), dz = z - __ldg(c + 2);
        a = fma(u, u, fma(v, v, w * w));
        b = fma(dx, u, fma(dy, v, dz * w));
        cc = fma(dx, dx, fma(dy, dy, fma(dz, dz, -__ldg(W.s_r2 + sid))));
    }
    if (!is_pos(a)) return MCGB_INF;
    double disc = fma(b, b, -(a * cc));
    // Inside: the far root by the cancellation-free form chosen by the sign of
    // b, (|b| + sq) / a for b <= 0, -cc / (|b| + sq) for b > 0; outside, when
    // approaching and hit: the near root cc / (|b| + sq).  The operands are
    // selected first so that one square root, one addition and one division
    // serve every lane of a warp, whichever of the cases its lanes are in.
    const bool inside = sense < 0;
    if (!inside && (!is_neg(b) || is_neg(disc))) return MCGB_INF;
    if (is_neg(disc)) disc = 0.0;
    double s1 = fabs(b) + sqrt_rn(disc);
    const bool far_plus = inside && !is_pos(b);
    double num = far_plus ? s1 : (inside ? -cc : cc);
    double den = far_plus ? a : s1;
    t = div_rn(num, den);
    return is_neg(t) ? 0.0 : t;
}

// Does cell `ci` hold the point?  Sense from the sign of f; exactly on a surface
// from the sign of (gradient . direction), 0 counting as +.  `forced` (a surface
// just crossed) takes `forced_sense`.
__device__ __forceinline__ bool cell_holds(const World &W, int ci, double x, double y, double z,
                                           double u, double v, double w, int forced,
                                           int forced_sense)
{
    int off = __ldg(W.c_off + ci), nh = __ldg(W.c_nhs + ci);
    for (int h = 0; h < nh; h++) {
        int sid = __ldg(W.hs_surf + off + h);
        int sense;
        if (sid == forced) {
            sense = forced_sense;
        } else {
            double f = surf_f(W, sid, x, y, z);
            if (is_pos(f)) sense = 1;
            else if (is_neg(f)) sense = -1;
            else sense = is_neg(surf_gdot(W, sid, x, y, z, u, v, w)) ? -1 : 1;
        }
        if (sense != __ldg(W.hs_sense + off + h)) return false;
    }
    return true;
}

// First cell of universe U (definition order) holding the point, -1 if none.
__device__ __forceinline__ int locate_univ(const World &W, int U, double x, double y, double z,
                                           double u, double v, double w, int forced,
                                           int forced_sense)
{
    int b = __ldg(W.u_off + U), e = __ldg(W.u_off + U + 1);
    for (int k = b; k < e; k++) {
        int ci = __ldg(W.u_cells + k);
        if (cell_holds(W, ci, x, y, z, u, v, w, forced, forced_sense)) return ci;
    }
    return -1;
}

// After crossing half-space `hs` (global index) of a cell in universe U: scan the
// precomputed candidates (cells of U bounded by the same surface with the other
// sense), then the whole universe.  Cells must partition space, so the answer is
// the same as a full scan's.
__device__ __forceinline__ int relocate(const World &W, int U, int hs, double x, double y, double z,
                                        double u, double v, double w)
{
    int forced = __ldg(W.hs_surf + hs);
    int fs = -__ldg(W.hs_sense + hs);
    int b = __ldg(W.hs_coff + hs), e = __ldg(W.hs_coff + hs + 1);
    for (int k = b; k < e; k++) {
        int ci = __ldg(W.hs_cand + k);
        if (cell_holds(W, ci, x, y, z, u, v, w, forced, fs)) return ci;
    }
    return locate_univ(W, U, x, y, z, u, v, w, forced, fs);
}

__device__ __forceinline__ void local_xy(const World &W, int L, int ix, int iy, double x, double y,
                                         double &xl, double &yl)
{
    // x - (x0 + (ix + 0.5) pitch), the centre precomputed with that expression
    const double *ctr = W.l_ctr + __ldg(W.l_woff + L);
    xl = x - __ldg(ctr + ix);
    yl = y - __ldg(ctr + __ldg(W.l_nx + L) + 1 + iy);
}

__device__ __forceinline__ void lattice_index(const World &W, int L, double x, double y, int &ix,
                                              int &iy)
{
    double p = __ldg(W.l_pitch + L);
    int i = (int)floor(div_rn(x - __ldg(W.l_x0 + L), p));
    int j = (int)floor(div_rn(y - __ldg(W.l_y0 + L), p));
    int nx = __ldg(W.l_nx + L), ny = __ldg(W.l_ny + L);
    ix = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
    iy = j < 0 ? 0 : (j >= ny ? ny - 1 : j);
}

// Below the root cell: lattice element universe cell and material.
// `wall`: the particle has just stepped across a lattice wall, so it lies on the
// new element's boundary, where the universe's edge cell (if proven) holds it.
__device__ __forceinline__ bool descend(const World &W, PS &p, int hs_forced, bool wall = false)
{
    if (__ldg(W.c_fillk + p.cell) == FILL_LAT) {
        int L = __ldg(W.c_fill + p.cell);
        int U = __ldg(W.l_univ + __ldg(W.l_uoff + L) + p.ix + __ldg(W.l_nx + L) * p.iy);
        int uc;
        int edge = wall ? __ldg(W.u_edge + U) : -1;
        if (edge >= 0) {
            uc = edge;
        } else {
            // element-local coordinates only where a cell test needs them
            double xl, yl;
            local_xy(W, L, p.ix, p.iy, p.x, p.y, xl, yl);
            uc = hs_forced >= 0 ? relocate(W, U, hs_forced, xl, yl, p.z, p.u, p.v, p.w)
                                : locate_univ(W, U, xl, yl, p.z, p.u, p.v, p.w, -1, 0);
        }
        if (uc < 0) return false;
        p.ucell = uc;
        p.mat = __ldg(W.c_fill + uc);
    } else {
        p.ucell = -1;
        p.ix = -1;
        p.iy = -1;
        p.mat = __ldg(W.c_fill + p.cell);
    }
    return true;
}

__device__ __forceinline__ bool locate_full(const World &W, int root_univ, PS &p)
{
    int rc = locate_univ(W, root_univ, p.x, p.y, p.z, p.u, p.v, p.w, -1, 0);
    if (rc < 0) return false;
    p.cell = rc;
    if (__ldg(W.c_fillk + rc) == FILL_LAT)
        lattice_index(W, __ldg(W.c_fill + rc), p.x, p.y, p.ix, p.iy);
    return descend(W, p, -1);
}

// Nearest boundary: root cell surfaces, then interior lattice walls (x, y), then
// the element universe cell's surfaces; ties go to the earliest (strict <).
__device__ __forceinline__ double boundary(const World &W, const PS &p, int &kind, int &which)
{
    double best = MCGB_INF;
    kind = B_NONE;
    which = -1;
    int off = __ldg(W.c_off + p.cell), nh = __ldg(W.c_nhs + p.cell);
    // a root plane on a lattice side is reached first only from the outer
    // column or row on that side: from elsewhere a lattice wall ahead is
    // strictly nearer (proven per cell when the world is built)
    unsigned sides = 0xFu;
    const bool skip = __ldg(W.c_skiproot + p.cell) != 0;
    // inside a surface strictly inside the element: no lattice wall is reached
    // first, and no root surface either when all of them lie on or beyond the
    // lattice's edges
    const bool inner = p.ucell >= 0 && __ldg(W.c_inner + p.ucell) != 0;
    if (inner && __ldg(W.c_rootfar + p.cell) != 0) {
        nh = 0;
    } else if (skip) {
        int L = __ldg(W.c_fill + p.cell);
        sides = (p.ix == 0 ? 1u : 0u) | (p.ix == __ldg(W.l_nx + L) - 1 ? 2u : 0u) |
                (p.iy == 0 ? 4u : 0u) | (p.iy == __ldg(W.l_ny + L) - 1 ? 8u : 0u);
        if (!sides) nh = 0;
    }
    for (int h = 0; h < nh; h++) {
        if (skip && !((sides >> (__ldg(W.hs_side + off + h) - 1)) & 1u)) continue;
        double t = surf_dist(W, __ldg(W.hs_surf + off + h), __ldg(W.hs_sense + off + h), p.x, p.y,
                             p.z, p.u, p.v, p.w, p.iu, p.iv, p.iw);
        if (lt_mag(t, best)) {
            best = t;
            kind = B_ROOT;
            which = off + h;
        }
    }
    if (__ldg(W.c_fillk + p.cell) == FILL_LAT) {
        int L = __ldg(W.c_fill + p.cell);
        int nx = __ldg(W.l_nx + L), ny = __ldg(W.l_ny + L);
        // walls x0 + i pitch, precomputed with that expression; the wall ahead is
        // chosen first, then t = (wall - x)(1/u)
        const double *xw = W.l_wall + __ldg(W.l_woff + L);
        const double *yw = xw + nx + 1;
        int wx = inner ? -1 : (is_pos(p.u) ? (p.ix < nx - 1 ? p.ix + 1 : -1) : (is_neg(p.u) && p.ix > 0 ? p.ix : -1));
        if (wx >= 0) {
            double t = (__ldg(xw + wx) - p.x) * p.iu;
            if (is_neg(t)) t = 0.0;
            if (lt_mag(t, best)) {
                best = t;
                kind = B_LATX;
            }
        }
        int wy = inner ? -1 : (is_pos(p.v) ? (p.iy < ny - 1 ? p.iy + 1 : -1) : (is_neg(p.v) && p.iy > 0 ? p.iy : -1));
        if (wy >= 0) {
            double t = (__ldg(yw + wy) - p.y) * p.iv;
            if (is_neg(t)) t = 0.0;
            if (lt_mag(t, best)) {
                best = t;
                kind = B_LATY;
            }
        }
        double xl, yl;
        local_xy(W, L, p.ix, p.iy, p.x, p.y, xl, yl);
        int uoff = __ldg(W.c_off + p.ucell), unh = __ldg(W.c_nhs + p.ucell);
        for (int h = 0; h < unh; h++) {
            double tt = surf_dist(W, __ldg(W.hs_surf + uoff + h), __ldg(W.hs_sense + uoff + h), xl,
                                  yl, p.z, p.u, p.v, p.w, p.iu, p.iv, p.iw);
            if (lt_mag(tt, best)) {
                best = tt;
                kind = B_UNIV;
                which = uoff + h;
            }
        }
    }
    return best;
}

// Surface crossing: vacuum -> leak (returns 1); reflective plane -> mirror the
// direction, keep the cell; interior -> relocate with the crossed surface's
// sense flipped; lattice wall -> step the element.  Returns -1 when no cell
// holds the particle (lost).
__device__ __forceinline__ int cross(const World &W, PS &p, int kind, int which)
{
    if (kind == B_ROOT) {
        int sid = __ldg(W.hs_surf + which);
        int bc = __ldg(W.s_bc + sid);
        if (bc == BC_VACUUM) return 1;
        if (bc == BC_REFLECT) {
            switch (__ldg(W.s_type + sid)) {
            case SURF_PX: p.u = -p.u; p.iu = -p.iu; break;
            case SURF_PY: p.v = -p.v; p.iv = -p.iv; break;
            case SURF_PZ: p.w = -p.w; p.iw = -p.iw; break;
            default: {
                const double *c = W.s_coef + 4 * sid;
                double a = __ldg(c), b = __ldg(c + 1), cz = __ldg(c + 2);
                double dn = a * p.u + b * p.v + cz * p.w;
                double nn = a * a + b * b + cz * cz;
                double k = div_rn(2.0 * dn, nn);
                p.u = p.u - k * a;
                p.v = p.v - k * b;
                p.w = p.w - k * cz;
                set_recip(W, p);
            }
            }
            return 0;
        }
        int nc = relocate(W, __ldg(W.c_univ + p.cell), which, p.x, p.y, p.z, p.u, p.v, p.w);
        if (nc < 0) return -1;
        p.cell = nc;
        if (__ldg(W.c_fillk + nc) == FILL_LAT)
            lattice_index(W, __ldg(W.c_fill + nc), p.x, p.y, p.ix, p.iy);
        return descend(W, p, -1) ? 0 : -1;
    }
    if (kind == B_LATX || kind == B_LATY) {
        if (kind == B_LATX) p.ix += is_pos(p.u) ? 1 : -1;
        else p.iy += is_pos(p.v) ? 1 : -1;
        return descend(W, p, -1, true) ? 0 : -1;
    }
    return descend(W, p, which) ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Continuous-energy lookup: union-grid binary search, then each nuclide's
// interval from the precomputed map (equal to that nuclide's own largest
// E_j <= E); sigma = sigma_j + f (sigma_{j+1} - sigma_j), f = (E - E_j)(1/dE_j).
// The search starts from the bracket of E's bucket: buckets are keyed by the
// top bits of E's bit pattern (exponent and 8 fraction bits, monotone in E for
// E > 0), and bucket b holds the search result at its lower edge, so the
// result at E lies between the results at its bucket's edges; the loop is the
// plain one and returns the same index as a search over the whole grid.
__device__ __forceinline__ int union_index(const World &W, double E)
{
    long long key = (__double_as_longlong(E) >> 44) - W.ukey0;
    key = key < 0 ? 0 : (key > W.nukey - 1 ? W.nukey - 1 : key);
    int lo = __ldg(W.ukey_lo + key);
    int hi = __ldg(W.ukey_lo + key + 1) + 1;
    if (hi > W.nunion - 1) hi = W.nunion - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (!lt_mag(E, __ldg(W.Eu + mid))) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One nuclide at union interval k: sigma_t (= (s + c) + f), sigma_s, sigma_f.
__device__ __forceinline__ void ce_micro(const World &W, int nuc, int k, double E, double &st,
                                         double &ss, double &sf)
{
    int j = __ldg(W.umap + (int64_t)nuc * W.nunion + k);
    const double2 *iv =
        reinterpret_cast<const double2 *>(W.n_iv + 8 * ((int64_t)__ldg(W.n_ivoff + nuc) + j));
    double2 e_inv = __ldg(iv), s = __ldg(iv + 1), c = __ldg(iv + 2), f = __ldg(iv + 3);
    double fr = (E - e_inv.x) * e_inv.y;
    ss = fma(fr, s.y, s.x);
    double sc = fma(fr, c.y, c.x);
    sf = fma(fr, f.y, f.x);
    st = ss + sc + sf;
}

// Macroscopic Sigma_t and nuSigma_f: sums of N_i sigma_i in the material's nuclide order.
// Macroscopic flight cross sections of a CE material: the material's table on
// its own union grid (sums of the per-nuclide lin-lin values at its points),
// interpolated, Sigma = S_k + ((E - E_k)(1/dE_k)) dS_k, k from the bracketed
// search (largest k <= n-2 with E_k <= E, else 0).
__device__ __forceinline__ void ce_macro(const World &W, int mat, double E, double &sigt,
                                         double &nusf)
{
    const int off = __ldg(W.cm_off + mat), n = __ldg(W.cm_n + mat);
    const int nkey = __ldg(W.cm_nkey + mat);
    long long key = (__double_as_longlong(E) >> 44) - __ldg(W.cm_key0 + mat);
    key = key < 0 ? 0 : (key > nkey - 1 ? nkey - 1 : key);
    const int *klo = W.cm_klo + __ldg(W.cm_koff + mat);
    int lo = __ldg(klo + key);
    int hi = __ldg(klo + key + 1) + 1;
    if (hi > n - 1) hi = n - 1;
    const double *Eg = W.cm_E + off;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (!lt_mag(E, __ldg(Eg + mid))) lo = mid;
        else hi = mid;
    }
    const double2 *r = reinterpret_cast<const double2 *>(W.cm_rec + 6 * ((int64_t)off + lo));
    double2 e_inv = __ldg(r), t = __ldg(r + 1), f = __ldg(r + 2);
    double fr = (E - e_inv.x) * e_inv.y;
    sigt = fma(fr, t.y, t.x);
    nusf = fma(fr, f.y, f.x);
}

// ---------------------------------------------------------------------------
// Track-length tallies: score d into [batch][bin][energy] of every tally of the
// particle's problem (accumulator replica `rep` spreads atomic traffic).
// Times are finite and >= 0, so the magnitude compare orders them exactly.
__device__ __forceinline__ bool lt_time(double a, double b) { return lt_mag(a, b); }

// Track-length tallies; a tally with time bins scores instead, per bin, the
// time the segment [ta, tb] spends in the bin times 1 / bin width (population).
// TIME = false compiles the time bins out (worlds without time dependence).
template <bool TIME, bool CE = true>
__device__ __forceinline__ void score(const World &W, const ProblemDev &P, const PS &p, double d,
                                      int batch, double *acc, int rep, double ta, double tb)
{
    for (int t = P.tally_first; t < P.tally_first + P.tally_count; t++) {
        int filter = __ldg(W.t_filter + t);
        int bin;
        if (filter == FILTER_CELL) {
            bin = (p.ucell >= 0 ? p.ucell : p.cell) - P.cell0;
        } else if (filter == FILTER_LATTICE) {
            if (p.ucell < 0) continue;
            bin = p.ix + __ldg(W.l_nx + P.lattice0) * p.iy;
        } else {
            bin = p.mat - P.mat0;
        }
        int e;
        if (CE && P.ce) {
            const double *ed = W.t_edges + __ldg(W.t_eoff + t);
            int ne = __ldg(W.t_nedges + t);
            if (lt_mag(p.E, __ldg(ed)) || lt_mag(__ldg(ed + ne - 1), p.E)) continue;
            e = 0;
            while (e + 1 < ne - 1 && !lt_mag(p.E, __ldg(ed + e + 1))) e++;
        } else {
            e = p.g;
        }
        int nb = __ldg(W.t_nbins + t), ne_ = __ldg(W.t_ne + t);
        int ntb = TIME ? __ldg(W.t_ntb + t) : 0;
        const int64_t base = (int64_t)rep * W.acc_size + __ldg(W.t_off + t);
        const int64_t cell = ((int64_t)batch * nb + bin) * ne_ + e;   // [batch][bin][e]
        if (ntb == 0) {
            atomicAdd(acc + base + cell, d);
            continue;
        }
        // [batch][bin][e][time bin].  Only bins with e_k < tb and ta < e_{k+1}
        // can score (the edges increase): the first is found by bisection,
        // the loop stops at the first edge >= tb.
        const int64_t idx = base + cell * ntb;
        const double *te = W.t_tedges + __ldg(W.t_toff + t);
        const double *tw = W.t_tinvw + __ldg(W.t_toff + t);
        int k0 = 0, k1 = ntb;   // first k with ta < e_{k+1}
        while (k0 < k1) {
            int mid = (k0 + k1) >> 1;
            if (lt_time(ta, __ldg(te + mid + 1))) k1 = mid;
            else k0 = mid + 1;
        }
        for (int k = k0; k < ntb; k++) {
            double e0 = __ldg(te + k);
            if (!lt_time(e0, tb)) break;
            double e1 = __ldg(te + k + 1);
            double lo = lt_time(e0, ta) ? ta : e0;   // max(ta, e0)
            double hi = lt_time(tb, e1) ? tb : e1;   // min(tb, e1)
            if (lt_time(lo, hi)) atomicAdd(acc + idx + k, (hi - lo) * __ldg(tw + k));
        }
    }
}

// ---------------------------------------------------------------------------
// Fission sites (parent slot, child index) are appended in any order and put in
// (parent, child) order at the end of the cycle.  The lanes that bank together
// reserve their sites with one atomic: counts are summed and prefix-summed from
// three ballots of their bit planes (a count of 8 or more takes its own atomic).
template <bool TIME = true>
__device__ __forceinline__ void bank_append(const Bank &B, int *bank_n, int *err, PS &p, int slot,
                                            int nf)
{
    cooperative_groups::coalesced_group g = cooperative_groups::coalesced_threads();
    const unsigned lt = (1u << g.thread_rank()) - 1u;
    int small = nf < 8 ? nf : 0;
    unsigned b0 = g.ballot(small & 1), b1 = g.ballot(small & 2), b2 = g.ballot(small & 4);
    int total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
    int before = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
    int base = 0;
    if (g.thread_rank() == 0 && total > 0) base = atomicAdd(bank_n, total);
    base = g.shfl(base, 0);
    int pos0 = nf < 8 ? base + before : atomicAdd(bank_n, nf);
    for (int k = 0; k < nf; k++) {
        int pos = pos0 + k;
        if (pos >= B.cap) {
            atomicOr(err, ERR_BANK_OVERFLOW);
        } else {
            B.x[pos] = p.x;
            B.t[pos] = TIME ? p.t : 0.0;
            B.y[pos] = p.y;
            B.z[pos] = p.z;
            B.cell[pos] = p.cell;
            B.ix[pos] = p.ix;
            B.iy[pos] = p.iy;
            B.ucell[pos] = p.ucell;
            B.mat[pos] = p.mat;
            B.parent[pos] = slot;
            B.child[pos] = p.nfis;
            B.root[pos] = p.root;
            B.prob[pos] = p.prob;
        }
        p.nfis++;
    }
}

// Systematic resampling: source j of N takes bank site floor((j + xi) M / N),
// at most M - 1.  xi = n 2^-53 exactly (n in [1, 2^53]), so the floor of the
// rational is exact in integers: (j + n 2^-53) M / N = (j M + n M 2^-53) / N,
// and floor((K + f) / N) = floor(K / N) for an integer K and 0 <= f < 1, with
// K = j M + floor(n M / 2^53).  (j M < 2^63 for j < N <= 2^31, M <= 2^32.)
__device__ __forceinline__ int64_t site_index_of(int64_t j, double xi, int64_t M, int64_t N)
{
    uint64_t n = (uint64_t)(xi * 0x1p53);
    uint64_t m = (uint64_t)M;
    uint64_t lo = n * m, hi = __umul64hi(n, m);
    uint64_t K = (uint64_t)j * m + ((hi << 11) | (lo >> 53));
    int64_t idx = (int64_t)(K / (uint64_t)N);
    return idx >= M ? M - 1 : idx;
}

// ---------------------------------------------------------------------------
// Sources: draw order is position (3 draws per rejection attempt), energy, direction.
__device__ __forceinline__ bool mat_fissile(const World &W, const ProblemDev &P, int mat)
{
    return P.ce ? __ldg(W.mc_fissile + mat) != 0 : __ldg(W.m_fissile + mat) != 0;
}

template <bool CE = true>
__device__ __forceinline__ void birth_energy(const World &W, const ProblemDev &P, PS &p)
{
    if (CE && P.ce) p.E = maxwell(W, p.s);
    else p.g = sample_cdf(W.g_chicdf + __ldg(W.m_goff + p.mat), __ldg(W.m_G + p.mat), draw(p.s));
}

template <bool CE = true>
__device__ __forceinline__ bool sample_source(const World &W, const ProblemDev &P, PS &p)
{
    p.u = p.v = p.w = 0.0;
    p.t = P.time_on ? P.t0 : 0.0;
    if (P.src_kind == SRC_BOX) {
        bool ok = false;
        for (int t = 0; t < MAX_TRIES && !ok; t++) {
            p.x = P.src_p[0] + draw(p.s) * (P.src_p[1] - P.src_p[0]);
            p.y = P.src_p[2] + draw(p.s) * (P.src_p[3] - P.src_p[2]);
            p.z = P.src_p[4] + draw(p.s) * (P.src_p[5] - P.src_p[4]);
            if (!locate_full(W, P.root_univ, p)) continue;
            ok = P.src_accept == 0 || mat_fissile(W, P, p.mat);
        }
        if (!ok) return false;
    } else {
        p.x = P.src_p[0];
        p.y = P.src_p[1];
        p.z = P.src_p[2];
        if (!locate_full(W, P.root_univ, p)) return false;
    }
    switch (P.src_ekind) {
    case E_CHI: birth_energy<CE>(W, P, p); break;
    case E_PDF: p.g = sample_cdf(W.src_cdf + P.src_cdf_off, P.src_ncdf, draw(p.s)); break;
    case E_FIXED: p.E = P.src_E; break;
    default: if (CE) p.E = maxwell(W, p.s);
    }
    if (P.src_dkind == DIR_BEAM) {
        p.u = P.src_beam[0];
        p.v = P.src_beam[1];
        p.w = P.src_beam[2];
    } else {
        iso_dir(p.s, p.u, p.v, p.w);
    }
    set_recip(W, p);
    return true;
}

template <bool CE = true>
__device__ __forceinline__ void birth_from_site(const World &W, const ProblemDev &P, const Bank &B,
                                                int b, PS &p)
{
    p.x = B.x[b];
    p.t = B.t[b];
    p.y = B.y[b];
    p.z = B.z[b];
    p.cell = B.cell[b];
    p.ix = B.ix[b];
    p.iy = B.iy[b];
    p.ucell = B.ucell[b];
    p.mat = B.mat[b];
    birth_energy<CE>(W, P, p);
    iso_dir(p.s, p.u, p.v, p.w);
    set_recip(W, p);
}

}  // namespace mcgb
