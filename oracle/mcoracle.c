/*
 * mcoracle.c -- plain history-based CPU reference for event-based Monte Carlo
 * neutral-particle transport.  TEST INFRASTRUCTURE: only the tests, the smoke
 * check and the benchmark's CPU-baseline leg use this file.
 *
 * What is computed follows the paper's description of the transport code
 * (Sec. 1: multigroup and continuous-energy physics, CSG geometry with surface
 * tracking, k-eigenvalue and fully dynamic/fixed-source runs, replicable
 * random numbers; Sec. 2: particles advance, cross surfaces and collide).  The
 * paper gives no formulas, so every step is the textbook one, taken one
 * particle at a time (history-based), with secondaries deferred to the next
 * cycle or generation.  Wherever the paper is silent the choice is stated in a
 * comment beginning "Reading:".
 *
 * Arithmetic.  The default (plain) mode writes each quantity as its definition
 * reads: ln xi from libm, d = (distance along the normal) / (direction cosine),
 * sums and products in the order written with no fused multiply-add (compile
 * with -ffp-contract=off), continuous-energy cross sections summed over
 * nuclides at the particle's energy, discrete outcomes sampled against
 * unnormalised running sums.  The strict mode exists only to compare against
 * the CUDA library bit for bit; it adopts that library's rounding conventions,
 * each marked "Strict:" below.  The two modes draw the same random numbers in
 * the same order and differ only in rounding.
 */
#include "mcoracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define INF HUGE_VAL
#define MAX_EVENTS 1000000   /* events per history before it is cut (counted as capped) */
#define MAX_TRIES 10000      /* source rejection attempts */
#define MAX_GEN 200          /* fixed-source generations */

/* ------------------------------------------------------------------------- */
/* Random numbers.  The paper (Sec. 1) states only that streams are replicable
 * on CPU and GPU.  Reading: the 63-bit congruential generator of the MCNP /
 * OpenMC family, s' = (g s + c) mod 2^63 with g = 2806196910506780709, c = 1;
 * stream i starts 152917 i steps after the seed; a draw advances the state and
 * returns xi = ((s >> 10) + 1) 2^-53, in (0, 1].                              */
#define LCG_MULT 2806196910506780709ULL
#define LCG_ADD 1ULL
#define LCG_BITS 0x7FFFFFFFFFFFFFFFULL
#define STREAM_STRIDE 152917ULL

uint64_t orc_rng_next(uint64_t s) { return (LCG_MULT * s + LCG_ADD) & LCG_BITS; }

double orc_rng_xi(uint64_t s) { return (double)((s >> 10) + 1) * 0x1p-53; }

/* n steps at once (Brown, "Random number generation with arbitrary strides",
 * 1994).  k steps are the affine map s -> A_k s + B_k (mod 2^63).  Reading the
 * bits of n from the most significant down: k -> 2k composes the map with
 * itself, A_2k = A_k^2, B_2k = (A_k + 1) B_k; k -> k + 1 appends one step,
 * A_k+1 = g A_k, B_k+1 = g B_k + c.  Unsigned arithmetic wraps mod 2^64, and
 * only the low 63 bits are kept at the end.                                   */
uint64_t orc_rng_skip(uint64_t s, uint64_t n)
{
    uint64_t A = 1, B = 0;
    n &= LCG_BITS;
    for (int bit = 62; bit >= 0; bit--) {
        B = (A + 1) * B;
        A = A * A;
        if ((n >> bit) & 1) {
            A = LCG_MULT * A;
            B = LCG_MULT * B + LCG_ADD;
        }
    }
    return (A * (s & LCG_BITS) + B) & LCG_BITS;
}

uint64_t orc_rng_stream(uint64_t seed, uint64_t id) { return orc_rng_skip(seed, id * STREAM_STRIDE); }

static uint64_t draw_n(uint64_t *s)
{
    *s = orc_rng_next(*s);
    return (*s >> 10) + 1;          /* the integer n of xi = n 2^-53 */
}

static double draw(uint64_t *s) { return (double)draw_n(s) * 0x1p-53; }

/* ------------------------------------------------------------------------- */
/* ln xi for the flight distance and the spectra.  Plain: libm's log.
 * Strict: the CUDA library's fixed-point form of the table-driven method of
 * Tang ("Table-driven implementation of the logarithm function in IEEE
 * floating-point arithmetic", ACM TOMS 1990): xi = 2^(e-53) m with m in
 * [1, 2); c = 1 + j/256 from the top 8 bits of m's fraction; r = (m - c)(1/c)
 * as a 64-bit fraction; ln xi = (e - 53) ln 2 + ln c + log1p(r), log1p by its
 * Taylor polynomial to r^6 by Horner's rule on 63-bit fractions (every
 * product truncated), the three terms added in 57 fraction bits and the sum
 * rounded once to a double.  The tables hold ln c and ln 2 to 57 fraction
 * bits, rounded to nearest (computed here from the Mercator series of
 * -ln(1 - t) in 120-bit fixed point), and 1/c to 63 bits rounded down.      */
typedef unsigned __int128 orc_u128;
static int64_t FX_LNC[256], FX_ELN2[64];
static uint64_t FX_INVC[256];
static int tang_ready;

/* a b / 2^120 for a, b < 2^121: the 256-bit product from 64-bit limbs */
static orc_u128 fx_mul120(orc_u128 a, orc_u128 b)
{
    uint64_t a1 = (uint64_t)(a >> 64), a0 = (uint64_t)a, b1 = (uint64_t)(b >> 64), b0 = (uint64_t)b;
    orc_u128 p00 = (orc_u128)a0 * b0, p01 = (orc_u128)a0 * b1, p10 = (orc_u128)a1 * b0,
             p11 = (orc_u128)a1 * b1;
    /* product = p11 2^128 + (p01 + p10) 2^64 + p00; keep bits 120 and up */
    orc_u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;   /* bits 64..191, low part */
    orc_u128 hi = p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);  /* bits 128 and up */
    return (hi << 8) | ((uint64_t)mid >> 56);
}

/* -ln(1 - t) = t + t^2/2 + t^3/3 + ... for t = num/den < 1/2, 120 fraction bits */
static orc_u128 fx_mercator120(uint64_t num, uint64_t den)
{
    orc_u128 t = ((orc_u128)num << 120) / den, pw = t, sum = 0;
    for (int k = 1; k <= 400 && pw; k++) {
        sum += pw / (orc_u128)k;
        pw = fx_mul120(pw, t);
    }
    return sum;
}

static int64_t fx_round57(orc_u128 v) { return (int64_t)((v + ((orc_u128)1 << 62)) >> 63); }

static void tang_init(void)
{
    if (tang_ready) return;
    for (int j = 0; j < 256; j++) {
        /* ln(1 + j/256) = -ln(1 - j/(256 + j)) */
        FX_LNC[j] = fx_round57(fx_mercator120((uint64_t)j, (uint64_t)(256 + j)));
        FX_INVC[j] = (uint64_t)(((orc_u128)1 << 71) / (orc_u128)(256 + j));
    }
    int64_t ln2 = fx_round57(fx_mercator120(1, 2));   /* -ln(1 - 1/2) */
    for (int e = 0; e < 64; e++) FX_ELN2[e] = (int64_t)(e - 53) * ln2;
    tang_ready = 1;
}

int64_t orc_log_table_q57(int j)
{
    tang_init();
    return j >= 0 && j < 256 ? FX_LNC[j] : INT64_MIN;
}

/* n in [1, 2^53]: xi = n 2^-53 */
static double tang_log(uint64_t n)
{
    int e = 0;
    while ((n >> e) > 1) e++;                         /* 2^e <= n < 2^(e+1) */
    uint64_t fr = (n << (52 - e)) & ((1ULL << 52) - 1);   /* m's 52 fraction bits */
    int j = (int)(fr >> 44);
    uint64_t d = fr & ((1ULL << 44) - 1);             /* (m - c) 2^52 */
    uint64_t r = (uint64_t)(((orc_u128)d * FX_INVC[j]) >> 51);   /* r 2^64 */
    static const uint64_t inv_k[6] = {0x8000000000000000ULL, 0x4000000000000000ULL,
                                      0x2AAAAAAAAAAAAAAAULL, 0x2000000000000000ULL,
                                      0x1999999999999999ULL, 0x1555555555555555ULL};   /* 2^63 / k */
    uint64_t h = inv_k[5];
    for (int k = 4; k >= 0; k--) h = inv_k[k] - (uint64_t)(((orc_u128)r * h) >> 64);
    uint64_t lp = (uint64_t)(((orc_u128)r * h) >> 64);   /* log1p(r) 2^63 */
    int64_t L = FX_ELN2[e] + FX_LNC[j] + (int64_t)(lp >> 6);
    if (L == 0) return 0.0;
    /* -L 2^-57, rounded to the nearest double (ties to even) by the FPU's
     * conversion of the integer: |L| < 2^63 */
    return -ldexp((double)(uint64_t)(-L), -57);
}

double orc_log(double xi)
{
    tang_init();
    if (!(xi > 0.0) || xi > 1.0) return NAN;
    return tang_log((uint64_t)(xi * 0x1p53));
}

/* ln of xi = n 2^-53 in the given mode */
static double ln_xi(uint64_t n, int strict)
{
    return strict ? tang_log(n) : log((double)n * 0x1p-53);
}

/* a^2 + b^2.  Strict: the first product is fused into the addition. */
static double sumsq2(double a, double b, int strict)
{
    return strict ? fma(a, a, b * b) : a * a + b * b;
}

/* ------------------------------------------------------------------------- */
/* Isotropic direction (Marsaglia, "Choosing a point from the surface of a
 * sphere", 1972): (a, b) uniform in the unit disk by rejection, S = a^2 + b^2,
 * Omega = (2a sqrt(1-S), 2b sqrt(1-S), 1 - 2S).  No trigonometric function.   */
static void iso_dir(uint64_t *s, double *u, double *v, double *w, int strict)
{
    for (int k = 0; k < 64; k++) {
        double a = 2.0 * draw(s) - 1.0;
        double b = 2.0 * draw(s) - 1.0;
        double S = sumsq2(a, b, strict);
        if (S < 1.0) {
            double t = 2.0 * sqrt(1.0 - S);
            *u = a * t;
            *v = b * t;
            *w = 1.0 - 2.0 * S;
            return;
        }
    }
    *u = 0.0; *v = 0.0; *w = 1.0;
}

int orc_iso_dir(uint64_t *s, double out[3], int mode)
{
    iso_dir(s, &out[0], &out[1], &out[2], mode == ORC_STRICT);
    return 0;
}

/* A point uniform in the unit disk minus its centre, by rejection (at most 64
 * tries): returns 1 with (a, b) and r2 = a^2 + b^2 in (0, 1], else 0.        */
static int disk_point(uint64_t *s, double *a, double *b, double *r2, int strict)
{
    for (int k = 0; k < 64; k++) {
        double x = 2.0 * draw(s) - 1.0;
        double y = 2.0 * draw(s) - 1.0;
        double q = sumsq2(x, y, strict);
        if (q <= 1.0 && q > 0.0) {
            *a = x; *b = y; *r2 = q;
            return 1;
        }
    }
    return 0;
}

/* Uniform azimuth as (cos phi, sin phi) without trigonometry: the doubled
 * angle of a disk point (a, b) is uniform, cos = (a^2 - b^2)/r2,
 * sin = 2ab/r2.                                                               */
static void azimuth(uint64_t *s, double *cphi, double *sphi, int strict)
{
    double a, b, r2;
    if (!disk_point(s, &a, &b, &r2, strict)) { *cphi = 1.0; *sphi = 0.0; return; }
    if (strict) {           /* one reciprocal, rounded once, for both */
        double inv = 1.0 / r2;
        *cphi = fma(a, a, -(b * b)) * inv;
        *sphi = 2.0 * a * b * inv;
        return;
    }
    *cphi = (a * a - b * b) / r2;
    *sphi = 2.0 * a * b / r2;
}

/* Rotate direction (u,v,w) by polar cosine mu about itself, azimuth sampled
 * (textbook rotation, polar axis z, or x when |w| is near 1).  Strict: each
 * product that is added to another term is fused into that addition.        */
static void rotate(double mu, uint64_t *s, double *u, double *v, double *w, int strict)
{
    double cphi, sphi;
    azimuth(s, &cphi, &sphi, strict);
    if (strict) {
        double st2 = fma(-mu, mu, 1.0);
        double st = sqrt(st2 > 0.0 ? st2 : 0.0);
        double u0 = *u, v0 = *v, w0 = *w;
        double ww = fma(-w0, w0, 1.0);
        if (ww > 1.0e-10) {
            double q = sqrt(ww);
            double f = st / q;
            *u = fma(mu, u0, f * fma(u0 * w0, cphi, -(v0 * sphi)));
            *v = fma(mu, v0, f * fma(v0 * w0, cphi, u0 * sphi));
            *w = fma(mu, w0, -(st * q * cphi));
        } else {
            double q = sqrt(fma(-u0, u0, 1.0));
            double f = st / q;
            *v = fma(mu, v0, f * fma(v0 * u0, cphi, -(w0 * sphi)));
            *w = fma(mu, w0, f * fma(w0 * u0, cphi, v0 * sphi));
            *u = fma(mu, u0, -(st * q * cphi));
        }
        return;
    }
    double st2 = 1.0 - mu * mu;
    double st = sqrt(st2 > 0.0 ? st2 : 0.0);
    double u0 = *u, v0 = *v, w0 = *w;
    double ww = 1.0 - w0 * w0;
    if (ww > 1.0e-10) {
        double q = sqrt(ww);
        double f = st / q;
        *u = mu * u0 + f * (u0 * w0 * cphi - v0 * sphi);
        *v = mu * v0 + f * (v0 * w0 * cphi + u0 * sphi);
        *w = mu * w0 - st * q * cphi;
    } else {
        double uu = 1.0 - u0 * u0;
        double q = sqrt(uu);
        double f = st / q;
        *v = mu * v0 + f * (v0 * u0 * cphi - w0 * sphi);
        *w = mu * w0 + f * (w0 * u0 * cphi + v0 * sphi);
        *u = mu * u0 - st * q * cphi;
    }
}

/* Elastic scattering off a target at rest (textbook two-body kinematics):
 * mu_cm = 2 xi - 1, q = A^2 + 2 A mu_cm + 1, E' = E q / (A+1)^2,
 * mu_lab = (1 + A mu_cm) / sqrt(q).  Strict: q = (2A) mu_cm + (A^2 + 1) with
 * A^2 + 1 rounded once and the product fused, E' = (E q) (1/(A+1)^2) with the
 * reciprocal rounded once, mu_lab's numerator fused.
 * Reading: E' is floored at 1e-5 eV (the paper's data start there).           */
#define E_MIN 1.0e-5
#define E_MAX 2.0e7
static double elastic(double E, double A, uint64_t *s, double *u, double *v, double *w, int strict)
{
    double mucm = 2.0 * draw(s) - 1.0;
    double q, Ep, mul;
    if (strict) {
        q = fma(2.0 * A, mucm, fma(A, A, 1.0));
        Ep = E * q * (1.0 / ((A + 1.0) * (A + 1.0)));
        mul = fma(A, mucm, 1.0) / sqrt(q);
    } else {
        q = A * A + 2.0 * A * mucm + 1.0;
        Ep = E * q / ((A + 1.0) * (A + 1.0));
        mul = (1.0 + A * mucm) / sqrt(q);
    }
    if (mul > 1.0) mul = 1.0;
    if (mul < -1.0) mul = -1.0;
    rotate(mul, s, u, v, w, strict);
    return Ep < E_MIN ? E_MIN : Ep;
}

int orc_elastic(double E, double A, const double dir[3], uint64_t *s, double out[4], int mode)
{
    double u = dir[0], v = dir[1], w = dir[2];
    out[0] = elastic(E, A, s, &u, &v, &w, mode == ORC_STRICT);
    out[1] = u; out[2] = v; out[3] = w;
    return 0;
}

/* cos^2 of an angle uniform on [0, pi/2]: a^2 / (a^2 + b^2) of a disk point
 * (1 if no point is accepted in 64 tries)                                     */
static double disk_cos2(uint64_t *s, int strict)
{
    double a, b, r2;
    if (!disk_point(s, &a, &b, &r2, strict)) return 1.0;
    return a * a / r2;
}

/* Fission spectrum.  Reading: Maxwellian with T = 1.33 MeV sampled by the
 * Everett-Cashwell rule E = -T (ln xi1 + ln xi2 cos^2 theta) with theta uniform;
 * cos^2 theta is a^2 / (a^2 + b^2) of a point uniform in the unit disk (no
 * trigonometry); energies above 20 MeV are resampled.                         */
static double maxwell(uint64_t *s, int strict)
{
    for (int k = 0; k < 64; k++) {
        double L1 = ln_xi(draw_n(s), strict);
        double L2 = ln_xi(draw_n(s), strict);
        double c2 = disk_cos2(s, strict);
        double E = -1.33e6 * (L1 + L2 * c2);
        if (E <= E_MAX) return E < E_MIN ? E_MIN : E;
    }
    return E_MAX;
}

double orc_maxwell(uint64_t *s, int mode)
{
    tang_init();
    return maxwell(s, mode == ORC_STRICT);
}

/* Elastic scattering off a free-gas target with a constant cross section (the
 * model Sec. 4 assumes for its continuous-energy pin).  Speeds are in units of
 * the target's thermal speed sqrt(2 kT / (A m)): the neutron's is
 * y = sqrt(A E / kT).  The target's speed x and the cosine mu between its
 * direction and the neutron's follow the density proportional to the relative
 * speed r = |y Omega - x Omega_T| times the Maxwellian x^2 exp(-x^2):
 * proposals from (x + y) x^2 exp(-x^2) -- with probability
 * y sqrt(pi) / (y sqrt(pi) + 2) from x^2 exp(-x^2), x^2 = -(ln xi1 + ln xi2 c),
 * c = cos^2 of a uniform angle, else from x^3 exp(-x^2), x^2 = -(ln xi1 + ln xi2)
 * -- with mu = 2 xi - 1, accepted when xi (x + y) <= r.  The target direction is
 * the neutron's rotated by mu.  Two-body kinematics: the centre-of-mass velocity
 * V = (y Omega + A x Omega_T) / (A + 1) is kept, the neutron's speed in that
 * frame A r / (A + 1) is kept and its direction there is isotropic; then
 * E' = E |v'|^2 / y^2 (floored at 1e-5 eV) and Omega' = v' / |v'|.           */
static double free_gas(double E, double A, double kT, uint64_t *s, double *u, double *v,
                       double *w, int strict)
{
    const double SQRT_PI = 1.7724538509055160273;
    /* strict: y^2 = (A E)(1/kT), products fused into the additions that
     * follow them, E' = |v'|^2 (kT (1/A)) (= E |v'|^2 / y^2) */
    double y2 = strict ? A * E * (1.0 / kT) : A * E / kT;
    double y = sqrt(y2);
    double py = y * SQRT_PI;
    double x = 0.0, mu = 1.0, r = y;
    for (int k = 0; k < MAX_TRIES; k++) {
        double x2;
        if (draw(s) * (py + 2.0) < py) {
            double L1 = ln_xi(draw_n(s), strict);
            double L2 = ln_xi(draw_n(s), strict);
            double c2 = disk_cos2(s, strict);
            x2 = strict ? -fma(L2, c2, L1) : -(L1 + L2 * c2);
        } else {
            double L1 = ln_xi(draw_n(s), strict);
            double L2 = ln_xi(draw_n(s), strict);
            x2 = -(L1 + L2);
        }
        x = sqrt(x2);
        mu = 2.0 * draw(s) - 1.0;
        double r2 = strict ? fma(-(2.0 * x * y), mu, x2 + y2) : x2 + y * y - 2.0 * x * y * mu;
        r = sqrt(r2 > 0.0 ? r2 : 0.0);
        if (draw(s) * (x + y) <= r) break;
    }
    double tu = *u, tv = *v, tw = *w;
    rotate(mu, s, &tu, &tv, &tw, strict);
    double inv = 1.0 / (A + 1.0);
    double Vx, Vy, Vz, px, py2, pz, p2;
    double cu, cv, cw;
    if (strict) {
        double Ax = A * x;
        Vx = fma(y, *u, Ax * tu) * inv;
        Vy = fma(y, *v, Ax * tv) * inv;
        Vz = fma(y, *w, Ax * tw) * inv;
        iso_dir(s, &cu, &cv, &cw, strict);
        double wc = A * r * inv;
        px = fma(wc, cu, Vx); py2 = fma(wc, cv, Vy); pz = fma(wc, cw, Vz);
        p2 = fma(px, px, fma(py2, py2, pz * pz));
    } else {
        Vx = (y * *u + A * x * tu) * inv;
        Vy = (y * *v + A * x * tv) * inv;
        Vz = (y * *w + A * x * tw) * inv;
        iso_dir(s, &cu, &cv, &cw, strict);
        double wc = A * r * inv;
        px = Vx + wc * cu; py2 = Vy + wc * cv; pz = Vz + wc * cw;
        p2 = px * px + py2 * py2 + pz * pz;
    }
    double ip = 1.0 / sqrt(p2);
    *u = px * ip; *v = py2 * ip; *w = pz * ip;
    double Ep = strict ? p2 * (kT * (1.0 / A)) : E * (p2 / (y * y));
    return Ep < E_MIN ? E_MIN : Ep;
}

int orc_free_gas(double E, double A, double kT, const double dir[3], uint64_t *s, double out[4],
                 int mode)
{
    tang_init();
    double u = dir[0], v = dir[1], w = dir[2];
    out[0] = free_gas(E, A, kT, s, &u, &v, &w, mode == ORC_STRICT);
    out[1] = u; out[2] = v; out[3] = w;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Resampling site (power iteration, Sec. 4).  Reading: systematic sampling --
 * source j of N takes bank site floor((j + xi) M / N), xi = n 2^-53 the
 * cycle's draw, clamped to M - 1 (reached only at xi = 1, j = N - 1).  The
 * floor of the rational is taken exactly in integers: (j + n 2^-53) M / N =
 * (j M 2^53 + n M) / (N 2^53).                                                */
int64_t orc_site_index(int64_t j, uint64_t n, int64_t M, int64_t N)
{
    unsigned __int128 num = ((unsigned __int128)(uint64_t)j << 53) + n;
    num *= (uint64_t)M;
    unsigned __int128 den = (unsigned __int128)(uint64_t)N << 53;
    int64_t k = (int64_t)(num / den);
    return k >= M ? M - 1 : k;
}

/* ------------------------------------------------------------------------- */
/* problem description                                                        */
typedef struct { int type, bc; double c[4]; double r2; } Surface;
typedef struct { int universe, nhs, off, fill_kind, fill; } Cell;
typedef struct { double x0, y0, pitch; int nx, ny; int *univ; } Lattice;
typedef struct {
    double *sigt, *sigs, *nusf, *chi;          /* input */
    double *stot, *chitot;                     /* row sums of sigma_s; sum of chi */
    double *mfp, *ps, *scdf, *chicdf;          /* strict mode's rounded-once constants */
    int fissile;
} MatMG;
typedef struct { double A, nu; int n; double *E, *s, *c, *f; } Nuclide;
typedef struct { int n; int *nuc; double *dens; int fissile; } MatCE;
/* macroscopic total and nu-fission cross sections of a CE material at the
 * points of its own union grid (the merged grids of its nuclides) */
typedef struct { int n; double *E, *St, *Sf; } MacroCE;
typedef struct {
    int kind, accept, ekind, dkind, ne;
    double p[6], beam[3];
    double *edata, *ecdf, etot;
} Source;
typedef struct {
    int filter, nedges; double *edges; int nbins, ne;
    int ntb;                     /* time bins (0: track length, no time binning) */
    double *tedges, *tinvw;      /* time edges and 1 / bin width */
} Tally;

typedef struct {
    double x, y, z, t;
    int cell, ix, iy, ucell, mat;
    int64_t parent, root;
    int32_t child;
} Site;

struct orc_ctx {
    char err[256];
    int strict;                  /* ORC_STRICT: the CUDA library's rounding conventions */
    int ns, nc, nhs, nl, G, nm, nn, nmc, nt, ce, max_coll;
    Surface *surf;
    Cell *cell;
    int *hs_surf, *hs_sense;
    Lattice *lat;
    int nuniv, *uoff, *ulist;
    MatMG *mg;
    Nuclide *nuc;
    MatCE *mce;
    Source src;
    int src_set;
    Tally *tally;
    MacroCE *macro;              /* per CE material, built when a run starts */
    /* free-gas elastic scattering below fg_emax (kT > 0 enables it) */
    double fg_kT, fg_emax;
    /* time dependence: source time, cutoff, 1/v per group, CE speed constant */
    int time_on;
    double t0, tcut, kv;
    double *invv;
    /* results */
    double k[6];
    int ncyc;
    double *cyc_ktl, *cyc_kc;
    int64_t *cyc_m;
    double **t_sum, **t_sum2, **t_mean, **t_sd;
    int64_t counters[8];
    int64_t nhist;
    int32_t *h_coll, *h_cross, *h_fis, *h_fate, *h_g;
    uint64_t *h_rng;
    int64_t nbank;
    Site *bank;
};

static int fail(orc_ctx *c, int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof c->err, fmt, ap);
    va_end(ap);
    return code;
}

static void *xgrow(void *p, size_t n, size_t sz) { return realloc(p, (n ? n : 1) * sz); }

static double *dup_d(const double *a, int n)
{
    double *r = malloc((size_t)(n ? n : 1) * sizeof(double));
    if (n) memcpy(r, a, (size_t)n * sizeof(double));
    return r;
}

orc_ctx *orc_create(void)
{
    tang_init();
    orc_ctx *c = calloc(1, sizeof(orc_ctx));
    c->G = 0;
    c->ce = -1;
    return c;
}

static void free_results(orc_ctx *c)
{
    for (int t = 0; c->t_sum && t < c->nt; t++) {
        free(c->t_sum[t]); free(c->t_sum2[t]); free(c->t_mean[t]); free(c->t_sd[t]);
    }
    free(c->t_sum); free(c->t_sum2); free(c->t_mean); free(c->t_sd);
    c->t_sum = c->t_sum2 = c->t_mean = c->t_sd = NULL;
    free(c->cyc_ktl); free(c->cyc_kc); free(c->cyc_m);
    c->cyc_ktl = c->cyc_kc = NULL; c->cyc_m = NULL;
    free(c->h_coll); free(c->h_cross); free(c->h_fis); free(c->h_rng);
    free(c->h_fate); free(c->h_g);
    c->h_coll = c->h_cross = c->h_fis = c->h_fate = c->h_g = NULL; c->h_rng = NULL;
    free(c->bank); c->bank = NULL; c->nbank = 0; c->nhist = 0;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free_results(c);
    for (int i = 0; i < c->nl; i++) free(c->lat[i].univ);
    for (int i = 0; i < c->nm; i++) {
        MatMG *m = &c->mg[i];
        free(m->sigt); free(m->sigs); free(m->nusf); free(m->chi); free(m->stot); free(m->chitot);
        free(m->mfp); free(m->ps); free(m->scdf); free(m->chicdf);
    }
    for (int i = 0; i < c->nn; i++) {
        free(c->nuc[i].E); free(c->nuc[i].s); free(c->nuc[i].c); free(c->nuc[i].f);
    }
    for (int i = 0; i < c->nmc; i++) { free(c->mce[i].nuc); free(c->mce[i].dens); }
    if (c->macro)
        for (int i = 0; i < c->nmc; i++) { free(c->macro[i].E); free(c->macro[i].St); free(c->macro[i].Sf); }
    free(c->macro);
    for (int i = 0; i < c->nt; i++) {
        free(c->tally[i].edges); free(c->tally[i].tedges); free(c->tally[i].tinvw);
    }
    free(c->invv);
    free(c->src.edata); free(c->src.ecdf);
    free(c->surf); free(c->cell); free(c->hs_surf); free(c->hs_sense); free(c->lat);
    free(c->uoff); free(c->ulist); free(c->mg); free(c->nuc); free(c->mce); free(c->tally);
    free(c);
}

const char *orc_error(const orc_ctx *c) { return c ? c->err : "null context"; }

int orc_set_arith(orc_ctx *c, int mode)
{
    if (mode != ORC_PLAIN && mode != ORC_STRICT) return fail(c, ORC_EINVAL, "bad arithmetic mode");
    c->strict = mode == ORC_STRICT;
    return 0;
}

int orc_add_surface(orc_ctx *c, int type, const double coef[4], int bc)
{
    if (type < ORC_PX || type > ORC_SPHERE || bc < 0 || bc > 2)
        return fail(c, ORC_EINVAL, "bad surface type/bc");
    if (bc == ORC_BC_REFLECT && type > ORC_PLANE)
        return fail(c, ORC_EINVAL, "reflective boundaries must be planes");
    c->surf = xgrow(c->surf, c->ns + 1, sizeof(Surface));
    Surface *s = &c->surf[c->ns];
    s->type = type;
    s->bc = bc;
    memcpy(s->c, coef, sizeof s->c);
    double R = type == ORC_CYLZ ? coef[2] : coef[3];
    s->r2 = R * R;
    return c->ns++;
}

int orc_add_cell(orc_ctx *c, int universe, int n, const int *surf, const int *sense,
                 int fill_kind, int fill)
{
    if (universe < 0 || n < 0 || fill < 0) return fail(c, ORC_EINVAL, "bad cell");
    for (int k = 0; k < n; k++)
        if (surf[k] < 0 || surf[k] >= c->ns || (sense[k] != 1 && sense[k] != -1))
            return fail(c, ORC_EINVAL, "bad half-space in cell %d", c->nc);
    c->cell = xgrow(c->cell, c->nc + 1, sizeof(Cell));
    c->hs_surf = xgrow(c->hs_surf, c->nhs + n, sizeof(int));
    c->hs_sense = xgrow(c->hs_sense, c->nhs + n, sizeof(int));
    Cell *e = &c->cell[c->nc];
    e->universe = universe;
    e->nhs = n;
    e->off = c->nhs;
    e->fill_kind = fill_kind;
    e->fill = fill;
    for (int k = 0; k < n; k++) {
        c->hs_surf[c->nhs + k] = surf[k];
        c->hs_sense[c->nhs + k] = sense[k];
    }
    c->nhs += n;
    return c->nc++;
}

int orc_add_lattice(orc_ctx *c, double x0, double y0, double pitch, int nx, int ny,
                    const int *universes)
{
    if (nx <= 0 || ny <= 0 || !(pitch > 0.0)) return fail(c, ORC_EINVAL, "bad lattice");
    c->lat = xgrow(c->lat, c->nl + 1, sizeof(Lattice));
    Lattice *L = &c->lat[c->nl];
    L->x0 = x0; L->y0 = y0; L->pitch = pitch; L->nx = nx; L->ny = ny;
    L->univ = malloc(sizeof(int) * (size_t)nx * ny);
    memcpy(L->univ, universes, sizeof(int) * (size_t)nx * ny);
    return c->nl++;
}

int orc_set_groups(orc_ctx *c, int G)
{
    if (G <= 0 || c->nm) return fail(c, ORC_EINVAL, "bad group count");
    c->G = G;
    c->ce = 0;
    return 0;
}

/* Discrete sampling from non-negative weights w[0..n-1] with total W: the
 * outcome is the first k whose running sum w[0] + ... + w[k] reaches xi W.
 * Plain: exactly that comparison.  Strict: the CUDA library's table of the
 * running sums each divided by W (the last set to exactly 1), searched for the
 * first entry >= xi.                                                         */
static double weight_total(const double *w, int n)
{
    double W = 0.0;
    for (int k = 0; k < n; k++) W = W + w[k];
    return W;
}

static void strict_cdf(const double *w, int n, double *tab)
{
    double W = weight_total(w, n);
    double run = 0.0;
    for (int k = 0; k < n; k++) {
        run = run + w[k];
        tab[k] = k == n - 1 ? 1.0 : run / W;
    }
}

static int sample_discrete(const double *w, double W, const double *tab, int n, double xi,
                           int strict)
{
    if (strict) {
        for (int k = 0; k < n - 1; k++)
            if (xi <= tab[k]) return k;
        return n - 1;
    }
    double target = xi * W, run = 0.0;
    for (int k = 0; k < n - 1; k++) {
        run = run + w[k];
        if (target <= run) return k;
    }
    return n - 1;
}

int orc_add_material_mg(orc_ctx *c, const double *sigma_t, const double *sigma_s,
                        const double *nu_sigma_f, const double *chi)
{
    int G = c->G;
    if (c->ce != 0 || G <= 0) return fail(c, ORC_ESTATE, "set groups first");
    c->mg = xgrow(c->mg, c->nm + 1, sizeof(MatMG));
    MatMG *m = &c->mg[c->nm];
    m->sigt = dup_d(sigma_t, G);
    m->sigs = dup_d(sigma_s, G * G);
    m->nusf = dup_d(nu_sigma_f, G);
    m->chi = dup_d(chi, G);
    m->stot = malloc(sizeof(double) * G);
    m->chitot = malloc(sizeof(double));
    m->mfp = malloc(sizeof(double) * G);
    m->ps = malloc(sizeof(double) * G);
    m->scdf = malloc(sizeof(double) * G * G);
    m->chicdf = malloc(sizeof(double) * G);
    m->fissile = 0;
    for (int g = 0; g < G; g++) {
        if (sigma_t[g] < 0.0 || nu_sigma_f[g] < 0.0) return fail(c, ORC_EINVAL, "negative XS");
        for (int h = 0; h < G; h++)
            if (sigma_s[g * G + h] < 0.0) return fail(c, ORC_EINVAL, "negative XS");
        m->stot[g] = weight_total(&sigma_s[g * G], G);
        if (m->stot[g] > sigma_t[g]) return fail(c, ORC_EINVAL, "scattering exceeds total");
        /* Strict: the mean free path 1/Sigma_t and the scattering probability
         * Sigma_s,tot/Sigma_t are rounded once per group (0 and inf in a void). */
        m->mfp[g] = sigma_t[g] > 0.0 ? 1.0 / sigma_t[g] : INF;
        m->ps[g] = sigma_t[g] > 0.0 ? m->stot[g] / sigma_t[g] : 0.0;
        if (m->stot[g] > 0.0) strict_cdf(&sigma_s[g * G], G, &m->scdf[g * G]);
        else for (int h = 0; h < G; h++) m->scdf[g * G + h] = 1.0;
        if (nu_sigma_f[g] > 0.0) m->fissile = 1;
    }
    m->chitot[0] = weight_total(chi, G);
    if (m->chitot[0] > 0.0) strict_cdf(chi, G, m->chicdf);
    else for (int g = 0; g < G; g++) m->chicdf[g] = 1.0;
    return c->nm++;
}

int orc_add_nuclide(orc_ctx *c, double A, int n, const double *E, const double *sig_s,
                    const double *sig_c, const double *sig_f, double nu)
{
    if (c->ce == 0) return fail(c, ORC_ESTATE, "problem is multigroup");
    if (n < 2 || !(A > 0.0)) return fail(c, ORC_EINVAL, "bad nuclide");
    for (int k = 1; k < n; k++)
        if (!(E[k] > E[k - 1])) return fail(c, ORC_EINVAL, "energy grid not increasing");
    c->ce = 1;
    c->nuc = xgrow(c->nuc, c->nn + 1, sizeof(Nuclide));
    Nuclide *u = &c->nuc[c->nn];
    u->A = A; u->nu = nu; u->n = n;
    u->E = dup_d(E, n); u->s = dup_d(sig_s, n); u->c = dup_d(sig_c, n); u->f = dup_d(sig_f, n);
    return c->nn++;
}

int orc_add_material_ce(orc_ctx *c, int n, const int *nuclides, const double *density)
{
    if (c->ce != 1) return fail(c, ORC_ESTATE, "add nuclides first");
    c->mce = xgrow(c->mce, c->nmc + 1, sizeof(MatCE));
    MatCE *m = &c->mce[c->nmc];
    m->n = n;
    m->nuc = malloc(sizeof(int) * (n ? n : 1));
    m->dens = dup_d(density, n);
    m->fissile = 0;
    for (int k = 0; k < n; k++) {
        if (nuclides[k] < 0 || nuclides[k] >= c->nn) return fail(c, ORC_EINVAL, "bad nuclide id");
        m->nuc[k] = nuclides[k];
        const Nuclide *u = &c->nuc[nuclides[k]];
        if (u->nu > 0.0)
            for (int j = 0; j < u->n; j++)
                if (u->f[j] > 0.0) { m->fissile = 1; break; }
    }
    return c->nmc++;
}

int orc_set_source(orc_ctx *c, int kind, const double *params, int accept, int energy_kind,
                   const double *energy, int n_energy, int dir_kind, const double *beam)
{
    Source *s = &c->src;
    free(s->edata); free(s->ecdf);
    memset(s, 0, sizeof *s);
    s->kind = kind; s->accept = accept; s->ekind = energy_kind; s->dkind = dir_kind;
    memcpy(s->p, params, sizeof(double) * (kind == ORC_SRC_BOX ? 6 : 3));
    if (dir_kind == ORC_DIR_BEAM) memcpy(s->beam, beam, sizeof s->beam);
    s->ne = n_energy;
    s->edata = dup_d(energy, n_energy);
    s->ecdf = malloc(sizeof(double) * (n_energy ? n_energy : 1));
    if (energy_kind == ORC_E_PDF) {
        s->etot = weight_total(energy, n_energy);
        strict_cdf(energy, n_energy, s->ecdf);
    }
    c->src_set = 1;
    return 0;
}

int orc_add_tally(orc_ctx *c, int filter, int n_edges, const double *edges)
{
    c->tally = xgrow(c->tally, c->nt + 1, sizeof(Tally));
    Tally *t = &c->tally[c->nt];
    t->filter = filter;
    t->nedges = n_edges;
    t->edges = dup_d(edges, n_edges);
    t->ntb = 0;
    t->tedges = t->tinvw = NULL;
    return c->nt++;
}

int orc_set_free_gas(orc_ctx *c, double kT, double cut)
{
    if (!(kT > 0.0) || !(kT < INF) || cut < 0.0) return fail(c, ORC_EINVAL, "bad free-gas settings");
    c->fg_kT = kT;
    c->fg_emax = (cut > 0.0 ? cut : 400.0) * kT;
    return 0;
}

int orc_set_time(orc_ctx *c, double t0, double t_cut)
{
    if (!(t_cut > t0) || !(t_cut < INF) || !(t0 >= 0.0))
        return fail(c, ORC_EINVAL, "need 0 <= t0 < t_cut < inf");
    c->time_on = 1;
    c->t0 = t0;
    c->tcut = t_cut;
    return 0;
}

int orc_set_inverse_speeds(orc_ctx *c, int G, const double *inv_v)
{
    if (G != c->G || G <= 0) return fail(c, ORC_EINVAL, "one inverse speed per group");
    for (int g = 0; g < G; g++)
        if (!(inv_v[g] > 0.0) || !(inv_v[g] < INF)) return fail(c, ORC_EINVAL, "bad inverse speed");
    free(c->invv);
    c->invv = dup_d(inv_v, G);
    return 0;
}

int orc_set_tally_time_bins(orc_ctx *c, int tally, int n_edges, const double *edges)
{
    if (tally < 0 || tally >= c->nt || n_edges < 2 || !(edges[0] >= 0.0))
        return fail(c, ORC_EINVAL, "bad time bins");
    for (int k = 0; k + 1 < n_edges; k++)
        if (!(edges[k + 1] > edges[k])) return fail(c, ORC_EINVAL, "time edges must increase");
    Tally *t = &c->tally[tally];
    free(t->tedges); free(t->tinvw);
    t->ntb = n_edges - 1;
    t->tedges = dup_d(edges, n_edges);
    t->tinvw = malloc(sizeof(double) * (size_t)t->ntb);
    for (int k = 0; k < t->ntb; k++) t->tinvw[k] = 1.0 / (edges[k + 1] - edges[k]);
    return 0;
}

int orc_set_max_collisions(orc_ctx *c, int max_collisions)
{
    c->max_coll = max_collisions;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* geometry                                                                   */
/* Surface functions f(r): f < 0 on the negative side.  Planes n.r - d, a
 * z-cylinder (x-x0)^2 + (y-y0)^2 - R^2, a sphere likewise in three
 * coordinates.  Strict: the sums of squares are evaluated with fused
 * multiply-adds.                                                              */
static double surf_f(const Surface *s, double x, double y, double z, int strict)
{
    switch (s->type) {
    case ORC_PX: return x - s->c[0];
    case ORC_PY: return y - s->c[0];
    case ORC_PZ: return z - s->c[0];
    case ORC_PLANE: return s->c[0] * x + s->c[1] * y + s->c[2] * z - s->c[3];
    case ORC_CYLZ: {
        double dx = x - s->c[0], dy = y - s->c[1];
        return sumsq2(dx, dy, strict) - s->r2;
    }
    default: {
        double dx = x - s->c[0], dy = y - s->c[1], dz = z - s->c[2];
        double q = strict ? fma(dx, dx, fma(dy, dy, dz * dz)) : dx * dx + dy * dy + dz * dz;
        return q - s->r2;
    }
    }
}

/* gradient of the surface function dotted with the direction (sign only used) */
static double surf_gdot(const Surface *s, double x, double y, double z, double u, double v,
                        double w)
{
    switch (s->type) {
    case ORC_PX: return u;
    case ORC_PY: return v;
    case ORC_PZ: return w;
    case ORC_PLANE: return s->c[0] * u + s->c[1] * v + s->c[2] * w;
    case ORC_CYLZ: return (x - s->c[0]) * u + (y - s->c[1]) * v;
    default: return (x - s->c[0]) * u + (y - s->c[1]) * v + (z - s->c[2]) * w;
    }
}

/* Distance along the direction to where the particle leaves the half-space of
 * the given sense.  Reading (the paper names surface tracking, Sec. 1, without
 * rules): the root is chosen from the sense, not from evaluating the position,
 * so a particle sitting on a surface it just crossed never re-hits it; a
 * negative root from round-off is taken as 0.
 * Plane: t = -f(r) / (n.Omega) when the particle moves towards the other side.
 * Quadric: f(r + t Omega) = a t^2 + 2 b t + cc with a = |Omega_perp|^2,
 * b = (r - r0).Omega_perp, cc = f(r), disc = b^2 - a cc; roots by the
 * cancellation-free forms: inside (sense -1) the far root, (-b + sqrt(disc))/a
 * for b <= 0 and -cc/(b + sqrt(disc)) for b > 0; outside, when approaching
 * (b < 0) and hit (disc >= 0), the near root cc/(-b + sqrt(disc)).
 * Strict: axis planes multiply by the direction's reciprocal carried with the
 * particle, t = -f (1/u); quadric terms use fused multiply-adds.             */
static double surf_dist(const Surface *s, int sense, double x, double y, double z, double u,
                        double v, double w, double iu, double iv, double iw, int strict)
{
    double t;
    if (s->type <= ORC_PLANE) {
        double dn, f, inv;
        switch (s->type) {
        case ORC_PX: dn = u; f = x - s->c[0]; inv = iu; break;
        case ORC_PY: dn = v; f = y - s->c[0]; inv = iv; break;
        case ORC_PZ: dn = w; f = z - s->c[0]; inv = iw; break;
        default:
            dn = s->c[0] * u + s->c[1] * v + s->c[2] * w;
            f = s->c[0] * x + s->c[1] * y + s->c[2] * z - s->c[3];
            inv = 0.0;
        }
        if ((sense > 0 && dn < 0.0) || (sense < 0 && dn > 0.0)) {
            t = (strict && s->type != ORC_PLANE) ? -f * inv : -f / dn;
            return t < 0.0 ? 0.0 : t;
        }
        return INF;
    }
    double a, b, cc;
    if (s->type == ORC_CYLZ) {
        double dx = x - s->c[0], dy = y - s->c[1];
        if (strict) {
            a = fma(u, u, v * v);
            b = fma(dx, u, dy * v);
            cc = fma(dx, dx, fma(dy, dy, -s->r2));
        } else {
            a = u * u + v * v;
            b = dx * u + dy * v;
            cc = dx * dx + dy * dy - s->r2;
        }
    } else {
        double dx = x - s->c[0], dy = y - s->c[1], dz = z - s->c[2];
        if (strict) {
            a = fma(u, u, fma(v, v, w * w));
            b = fma(dx, u, fma(dy, v, dz * w));
            cc = fma(dx, dx, fma(dy, dy, fma(dz, dz, -s->r2)));
        } else {
            a = u * u + v * v + w * w;
            b = dx * u + dy * v + dz * w;
            cc = dx * dx + dy * dy + dz * dz - s->r2;
        }
    }
    if (a == 0.0) return INF;
    double disc = strict ? fma(b, b, -(a * cc)) : b * b - a * cc;
    if (sense < 0) {
        if (disc < 0.0) disc = 0.0;
        if (b <= 0.0) t = (-b + sqrt(disc)) / a;
        else t = -cc / (b + sqrt(disc));
        return t < 0.0 ? 0.0 : t;
    }
    if (b >= 0.0 || disc < 0.0) return INF;
    t = cc / (-b + sqrt(disc));
    return t < 0.0 ? 0.0 : t;
}

static void build_universes(orc_ctx *c)
{
    int nu = 0;
    for (int i = 0; i < c->nc; i++)
        if (c->cell[i].universe + 1 > nu) nu = c->cell[i].universe + 1;
    free(c->uoff); free(c->ulist);
    c->nuniv = nu;
    c->uoff = calloc((size_t)nu + 1, sizeof(int));
    c->ulist = malloc(sizeof(int) * (c->nc ? c->nc : 1));
    for (int i = 0; i < c->nc; i++) c->uoff[c->cell[i].universe + 1]++;
    for (int u = 0; u < nu; u++) c->uoff[u + 1] += c->uoff[u];
    int *fill = calloc((size_t)nu, sizeof(int));
    for (int i = 0; i < c->nc; i++) {
        int u = c->cell[i].universe;
        c->ulist[c->uoff[u] + fill[u]++] = i;
    }
    free(fill);
}

/* The cell of universe U containing the point: every half-space must agree.
 * The sense of a surface is the sign of its function; exactly on a surface the
 * sign of (gradient . direction) decides, 0 counting as +.  `forced` (a
 * surface just crossed) takes `forced_sense` instead.  Cells are scanned in
 * definition order; the first match is returned (cells must partition space). */
static int locate_univ(const orc_ctx *c, int U, double x, double y, double z, double u, double v,
                       double w, int forced, int forced_sense)
{
    if (U < 0 || U >= c->nuniv) return -1;
    for (int k = c->uoff[U]; k < c->uoff[U + 1]; k++) {
        const Cell *e = &c->cell[c->ulist[k]];
        int ok = 1;
        for (int h = 0; h < e->nhs && ok; h++) {
            int sid = c->hs_surf[e->off + h];
            int sense;
            if (sid == forced) {
                sense = forced_sense;
            } else {
                const Surface *s = &c->surf[sid];
                double f = surf_f(s, x, y, z, c->strict);
                if (f > 0.0) sense = 1;
                else if (f < 0.0) sense = -1;
                else sense = surf_gdot(s, x, y, z, u, v, w) >= 0.0 ? 1 : -1;
            }
            if (sense != c->hs_sense[e->off + h]) ok = 0;
        }
        if (ok) return c->ulist[k];
    }
    return -1;
}

typedef struct {
    double x, y, z, u, v, w, E;
    double iu, iv, iw;           /* 1/u, 1/v, 1/w, rounded when the direction is set */
    double t;                    /* time (s), when the problem is time dependent */
    int g;
    uint64_t s;
    int cell, ix, iy, ucell, mat;
    int64_t index, root;
    int nfis, ncoll, ncross, alive, fate;
} Particle;

/* history fates */
enum { FATE_ABSORBED = 0, FATE_LEAKED = 1, FATE_CUT = 2, FATE_LOST = 3, FATE_CAPPED = 4,
       FATE_TIME = 5 };

/* Strict: the particle carries 1/u, 1/v, 1/w, rounded whenever its direction
 * is set (axis-plane and lattice-wall distances multiply by them). */
static void set_recip(Particle *p)
{
    p->iu = 1.0 / p->u;
    p->iv = 1.0 / p->v;
    p->iw = 1.0 / p->w;
}

static void local_xy(const Lattice *L, int ix, int iy, double x, double y, double *xl, double *yl)
{
    *xl = x - (L->x0 + ((double)ix + 0.5) * L->pitch);
    *yl = y - (L->y0 + ((double)iy + 0.5) * L->pitch);
}

/* Lattice element from a position: floor((x - x0)/pitch), clamped to the lattice. */
static void lattice_index(const Lattice *L, double x, double y, int *ix, int *iy)
{
    int i = (int)floor((x - L->x0) / L->pitch);
    int j = (int)floor((y - L->y0) / L->pitch);
    *ix = i < 0 ? 0 : (i >= L->nx ? L->nx - 1 : i);
    *iy = j < 0 ? 0 : (j >= L->ny ? L->ny - 1 : j);
}

/* Below the root cell: if it holds a lattice, find the element and the cell of
 * the element's universe (in element-centred coordinates); set the material. */
static int descend(const orc_ctx *c, Particle *p, int forced, int forced_sense)
{
    const Cell *rc = &c->cell[p->cell];
    if (rc->fill_kind == ORC_FILL_LATTICE) {
        const Lattice *L = &c->lat[rc->fill];
        double xl, yl;
        local_xy(L, p->ix, p->iy, p->x, p->y, &xl, &yl);
        int U = L->univ[p->ix + L->nx * p->iy];
        int uc = locate_univ(c, U, xl, yl, p->z, p->u, p->v, p->w, forced, forced_sense);
        if (uc < 0) return -1;
        p->ucell = uc;
        p->mat = c->cell[uc].fill;
    } else {
        p->ucell = -1;
        p->ix = p->iy = -1;
        p->mat = rc->fill;
    }
    return 0;
}

static int locate_full(const orc_ctx *c, Particle *p)
{
    int rc = locate_univ(c, 0, p->x, p->y, p->z, p->u, p->v, p->w, -1, 0);
    if (rc < 0) return -1;
    p->cell = rc;
    if (c->cell[rc].fill_kind == ORC_FILL_LATTICE)
        lattice_index(&c->lat[c->cell[rc].fill], p->x, p->y, &p->ix, &p->iy);
    return descend(c, p, -1, 0);
}

enum { B_NONE = 0, B_ROOT = 1, B_LATX = 2, B_LATY = 3, B_UNIV = 4 };

/* Nearest boundary: the root cell's surfaces, then the lattice element walls
 * (interior walls only), then the element universe cell's surfaces.  Reading:
 * ties go to the earliest in that order (strict <).                          */
static double boundary(const orc_ctx *c, const Particle *p, int *kind, int *which)
{
    double best = INF;
    *kind = B_NONE;
    *which = -1;
    const Cell *rc = &c->cell[p->cell];
    for (int h = 0; h < rc->nhs; h++) {
        double t = surf_dist(&c->surf[c->hs_surf[rc->off + h]], c->hs_sense[rc->off + h], p->x,
                             p->y, p->z, p->u, p->v, p->w, p->iu, p->iv, p->iw, c->strict);
        if (t < best) { best = t; *kind = B_ROOT; *which = rc->off + h; }
    }
    if (rc->fill_kind == ORC_FILL_LATTICE) {
        const Lattice *L = &c->lat[rc->fill];
        /* the wall ahead, x0 + i pitch; t = (wall - x) / u (strict: times 1/u) */
        double t = INF;
        int wx = p->u > 0.0 && p->ix < L->nx - 1 ? p->ix + 1 : (p->u < 0.0 && p->ix > 0 ? p->ix : -1);
        if (wx >= 0) {
            double gap = L->x0 + (double)wx * L->pitch - p->x;
            t = c->strict ? gap * p->iu : gap / p->u;
        }
        if (t < 0.0) t = 0.0;
        if (t < best) { best = t; *kind = B_LATX; }
        t = INF;
        int wy = p->v > 0.0 && p->iy < L->ny - 1 ? p->iy + 1 : (p->v < 0.0 && p->iy > 0 ? p->iy : -1);
        if (wy >= 0) {
            double gap = L->y0 + (double)wy * L->pitch - p->y;
            t = c->strict ? gap * p->iv : gap / p->v;
        }
        if (t < 0.0) t = 0.0;
        if (t < best) { best = t; *kind = B_LATY; }
        double xl, yl;
        local_xy(L, p->ix, p->iy, p->x, p->y, &xl, &yl);
        const Cell *uc = &c->cell[p->ucell];
        for (int h = 0; h < uc->nhs; h++) {
            double tt = surf_dist(&c->surf[c->hs_surf[uc->off + h]], c->hs_sense[uc->off + h], xl,
                                  yl, p->z, p->u, p->v, p->w, p->iu, p->iv, p->iw, c->strict);
            if (tt < best) { best = tt; *kind = B_UNIV; *which = uc->off + h; }
        }
    }
    return best;
}

/* Surface crossing (Sec. 1, surface tracking).  Vacuum: the particle leaks.
 * Reflective plane: Omega -= 2 (Omega.n) n / |n|^2, the cell is kept.
 * Interior: the new cell is the one holding the point with the crossed
 * surface's sense flipped.  Lattice wall: step the element index, relocate in
 * the new element's universe.  Returns 0, 1 (leaked) or -1 (lost).           */
static int cross(const orc_ctx *c, Particle *p, int kind, int which)
{
    if (kind == B_ROOT) {
        int sid = c->hs_surf[which];
        const Surface *s = &c->surf[sid];
        if (s->bc == ORC_BC_VACUUM) return 1;
        if (s->bc == ORC_BC_REFLECT) {
            switch (s->type) {
            case ORC_PX: p->u = -p->u; p->iu = -p->iu; break;
            case ORC_PY: p->v = -p->v; p->iv = -p->iv; break;
            case ORC_PZ: p->w = -p->w; p->iw = -p->iw; break;
            default: {
                double dn = s->c[0] * p->u + s->c[1] * p->v + s->c[2] * p->w;
                double nn = s->c[0] * s->c[0] + s->c[1] * s->c[1] + s->c[2] * s->c[2];
                double k = 2.0 * dn / nn;
                p->u = p->u - k * s->c[0];
                p->v = p->v - k * s->c[1];
                p->w = p->w - k * s->c[2];
                set_recip(p);
            }
            }
            return 0;
        }
        int nc = locate_univ(c, 0, p->x, p->y, p->z, p->u, p->v, p->w, sid, -c->hs_sense[which]);
        if (nc < 0) return -1;
        p->cell = nc;
        if (c->cell[nc].fill_kind == ORC_FILL_LATTICE)
            lattice_index(&c->lat[c->cell[nc].fill], p->x, p->y, &p->ix, &p->iy);
        return descend(c, p, -1, 0);
    }
    if (kind == B_LATX || kind == B_LATY) {
        if (kind == B_LATX) p->ix += p->u > 0.0 ? 1 : -1;
        else p->iy += p->v > 0.0 ? 1 : -1;
        return descend(c, p, -1, 0);
    }
    /* universe-level surface */
    return descend(c, p, c->hs_surf[which], -c->hs_sense[which]);
}

int orc_probe(orc_ctx *c, const double pos[3], const double dir[3], int out_path[5],
              double *dist, int *kind)
{
    build_universes(c);
    Particle p;
    memset(&p, 0, sizeof p);
    p.x = pos[0]; p.y = pos[1]; p.z = pos[2];
    p.u = dir[0]; p.v = dir[1]; p.w = dir[2];
    set_recip(&p);
    if (locate_full(c, &p) < 0) return fail(c, ORC_ELOST, "point outside geometry");
    out_path[0] = p.cell; out_path[1] = p.ix; out_path[2] = p.iy; out_path[3] = p.ucell;
    out_path[4] = p.mat;
    int which;
    *dist = boundary(c, &p, kind, &which);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* continuous-energy lookup.  Reading: for each nuclide, the interval is the
 * largest grid index j with E_j <= E (binary search, clamped to the last
 * interval); cross sections are linear in E on it (lin-lin interpolation):
 * f = (E - E_j) / (E_{j+1} - E_j), sigma = sigma_j + f (sigma_{j+1} - sigma_j).
 * Macroscopic values are N_i sigma_i summed in the material's nuclide order;
 * sigma_t,i = (sigma_s + sigma_c) + sigma_f.  Strict: the interval's
 * reciprocal width is rounded once, f = (E - E_j) (1/(E_{j+1} - E_j)), and
 * for a reaction (fused) the product is fused into the addition,
 * sigma = fma(f, sigma_{j+1} - sigma_j, sigma_j); the tables of the strict
 * macroscopic lookup take the unfused form.                                 */
typedef struct {
    double sigt, nusf;
    double st[16], ss[16], sf[16];
} CEXS;

static int nuc_interval(const Nuclide *u, double E)
{
    int lo = 0, hi = u->n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (u->E[mid] <= E) lo = mid;
        else hi = mid;
    }
    return lo;
}

static void ce_lookup(const orc_ctx *c, int mat, double E, CEXS *x, int fused)
{
    const MatCE *m = &c->mce[mat];
    x->sigt = 0.0;
    x->nusf = 0.0;
    for (int k = 0; k < m->n; k++) {
        const Nuclide *u = &c->nuc[m->nuc[k]];
        int j = nuc_interval(u, E);
        double f = c->strict ? (E - u->E[j]) * (1.0 / (u->E[j + 1] - u->E[j]))
                             : (E - u->E[j]) / (u->E[j + 1] - u->E[j]);
        double ss, sc, sf;
        if (fused) {
            ss = fma(f, u->s[j + 1] - u->s[j], u->s[j]);
            sc = fma(f, u->c[j + 1] - u->c[j], u->c[j]);
            sf = fma(f, u->f[j + 1] - u->f[j], u->f[j]);
        } else {
            ss = u->s[j] + f * (u->s[j + 1] - u->s[j]);
            sc = u->c[j] + f * (u->c[j + 1] - u->c[j]);
            sf = u->f[j] + f * (u->f[j + 1] - u->f[j]);
        }
        double st = ss + sc + sf;
        x->st[k] = st; x->ss[k] = ss; x->sf[k] = sf;
        x->sigt = x->sigt + m->dens[k] * st;
        x->nusf = x->nusf + m->dens[k] * (u->nu * sf);
    }
}

/* Strict: macroscopic cross sections for a flight come from a per-material
 * table, as in the CUDA library.  Every nuclide is lin-lin on each interval of
 * the material's union grid (its own points are union points), so the sums
 * Sigma_t = sum_i N_i sigma_t,i and nuSigma_f are linear there too; they are
 * tabulated at the union points (each per-nuclide value as in ce_lookup,
 * summed in the material's order) and interpolated,
 * Sigma(E) = fma((E - E_k) (1 / (E_k+1 - E_k)), S_k+1 - S_k, S_k), with k the
 * largest union index <= n - 2 whose point is <= E (0 if none).  Equal to the
 * per-nuclide sum in exact arithmetic (and exactly at the union points); the
 * plain mode sums the nuclides at the particle's energy instead.            */
static int dbl_cmp(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y);
}

static void build_macro(orc_ctx *c)
{
    if (c->macro)
        for (int i = 0; i < c->nmc; i++) { free(c->macro[i].E); free(c->macro[i].St); free(c->macro[i].Sf); }
    free(c->macro);
    c->macro = calloc(c->nmc ? c->nmc : 1, sizeof(MacroCE));
    for (int m = 0; m < c->nmc; m++) {
        const MatCE *mc = &c->mce[m];
        int tot = 0;
        for (int k = 0; k < mc->n; k++) tot += c->nuc[mc->nuc[k]].n;
        double *E = malloc(sizeof(double) * (size_t)(tot ? tot : 1));
        int q = 0;
        for (int k = 0; k < mc->n; k++) {
            const Nuclide *u = &c->nuc[mc->nuc[k]];
            for (int j = 0; j < u->n; j++) E[q++] = u->E[j];
        }
        qsort(E, (size_t)tot, sizeof(double), dbl_cmp);
        int n = 0;
        for (int k = 0; k < tot; k++)
            if (n == 0 || E[k] != E[n - 1]) E[n++] = E[k];
        MacroCE *M = &c->macro[m];
        M->n = n;
        M->E = E;
        M->St = malloc(sizeof(double) * (size_t)(n ? n : 1));
        M->Sf = malloc(sizeof(double) * (size_t)(n ? n : 1));
        for (int k = 0; k < n; k++) {
            CEXS x;
            ce_lookup(c, m, E[k], &x, 0);
            M->St[k] = x.sigt;
            M->Sf[k] = x.nusf;
        }
    }
}

static void macro_xs(const orc_ctx *c, int mat, double E, double *sigt, double *nusf)
{
    const MacroCE *M = &c->macro[mat];
    int lo = 0, hi = M->n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (M->E[mid] <= E) lo = mid;
        else hi = mid;
    }
    if (M->n < 2) { *sigt = M->St[0]; *nusf = M->Sf[0]; return; }
    double f = (E - M->E[lo]) * (1.0 / (M->E[lo + 1] - M->E[lo]));
    *sigt = fma(f, M->St[lo + 1] - M->St[lo], M->St[lo]);
    *nusf = fma(f, M->Sf[lo + 1] - M->Sf[lo], M->Sf[lo]);
}

/* flight cross sections Sigma_t, nuSigma_f of a CE material in the context's mode */
static void flight_xs(const orc_ctx *c, int mat, double E, double *sigt, double *nusf)
{
    if (c->strict) {
        macro_xs(c, mat, E, sigt, nusf);
        return;
    }
    CEXS x;
    ce_lookup(c, mat, E, &x, 0);
    *sigt = x.sigt;
    *nusf = x.nusf;
}

int orc_ce_lookup(orc_ctx *c, int material, double E, double out[4])
{
    if (c->ce != 1 || material < 0 || material >= c->nmc) return fail(c, ORC_EINVAL, "bad material");
    CEXS x;
    ce_lookup(c, material, E, &x, c->strict);
    if (c->strict && !c->macro) build_macro(c);
    flight_xs(c, material, E, &out[0], &out[1]);
    double ss = 0.0, sf = 0.0;
    for (int k = 0; k < c->mce[material].n; k++) {
        ss = ss + c->mce[material].dens[k] * x.ss[k];
        sf = sf + c->mce[material].dens[k] * x.sf[k];
    }
    out[2] = ss; out[3] = sf;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* transport of one history                                                   */
typedef struct {
    double **acc;           /* per tally: [batch][bin * ne + e] */
    double ktl, kc;
    Site *bank;
    int64_t nbank, capbank;
    int64_t coll, crossn, leak, lost, capped, timecut;
} Acc;

typedef struct {            /* gradient records (one per score) */
    int64_t n, cap;
    int *param;
    double *val, *ownb;
    int *nfb;
    int64_t *pid;
    double *own;            /* own detector tally per particle (global index) */
    int det_cell;
    const double *weights;
    int64_t pid_base;
} Grad;

static void bank_push(Acc *a, const Particle *p)
{
    if (a->nbank == a->capbank) {
        a->capbank = a->capbank ? 2 * a->capbank : 1024;
        a->bank = realloc(a->bank, sizeof(Site) * (size_t)a->capbank);
    }
    Site *s = &a->bank[a->nbank++];
    s->x = p->x; s->y = p->y; s->z = p->z; s->t = p->t;
    s->cell = p->cell; s->ix = p->ix; s->iy = p->iy; s->ucell = p->ucell; s->mat = p->mat;
    s->parent = p->index; s->root = p->root; s->child = p->nfis;
}

static void grad_rec(Grad *gr, int param, double val, double ownb, int nfb, int64_t pid)
{
    if (gr->n == gr->cap) {
        gr->cap = gr->cap ? 2 * gr->cap : 4096;
        gr->param = realloc(gr->param, sizeof(int) * gr->cap);
        gr->val = realloc(gr->val, sizeof(double) * gr->cap);
        gr->ownb = realloc(gr->ownb, sizeof(double) * gr->cap);
        gr->nfb = realloc(gr->nfb, sizeof(int) * gr->cap);
        gr->pid = realloc(gr->pid, sizeof(int64_t) * gr->cap);
    }
    gr->param[gr->n] = param; gr->val[gr->n] = val; gr->ownb[gr->n] = ownb;
    gr->nfb[gr->n] = nfb; gr->pid[gr->n] = pid;
    gr->n++;
}

/* values per batch of a tally: bins x energy bins x time bins */
static size_t tally_len(const Tally *T)
{
    return (size_t)T->nbins * (size_t)T->ne * (size_t)(T->ntb ? T->ntb : 1);
}

static int tally_bin(const orc_ctx *c, const Tally *t, const Particle *p, int *bin, int *e)
{
    switch (t->filter) {
    case ORC_FILTER_CELL: *bin = p->ucell >= 0 ? p->ucell : p->cell; break;
    case ORC_FILTER_LATTICE:
        if (p->ucell < 0) return 0;
        *bin = p->ix + c->lat[0].nx * p->iy;
        break;
    default: *bin = p->mat;
    }
    if (c->ce) {
        /* energy bin: largest b with edges[b] <= E, the top edge closing the last bin */
        if (p->E < t->edges[0] || p->E > t->edges[t->nedges - 1]) return 0;
        int b = 0;
        while (b + 1 < t->nedges - 1 && t->edges[b + 1] <= p->E) b++;
        *e = b;
    } else {
        *e = p->g;
    }
    return 1;
}

static void transport(const orc_ctx *c, Particle *p, Acc *a, int batch, Grad *gr, int64_t pid)
{
    const int G = c->G;
    double own = 0.0;
    for (;;) {
        if (p->ncoll + p->ncross >= MAX_EVENTS) { a->capped++; p->fate = FATE_CAPPED; break; }
        /* cross sections at the particle's material and energy */
        const int strict = c->strict;
        double sigt, nusf;
        CEXS x;
        const MatMG *m = NULL;
        if (c->ce) {
            flight_xs(c, p->mat, p->E, &sigt, &nusf);
        } else {
            m = &c->mg[p->mat];
            sigt = m->sigt[p->g];
            nusf = m->nusf[p->g];
        }
        /* distance to collision: d_c = -ln(xi) / Sigma_t (a draw is always
         * taken).  Strict: -ln(xi) times 1/Sigma_t rounded once (per group in
         * multigroup data, per lookup in continuous energy). */
        uint64_t n = draw_n(&p->s);
        double dc = INF;
        if (sigt > 0.0) {
            if (!strict) dc = -ln_xi(n, 0) / sigt;
            else dc = -ln_xi(n, 1) * (c->ce ? 1.0 / sigt : m->mfp[p->g]);
        }
        int kind, which;
        double ds = boundary(c, p, &kind, &which);
        if (!c->time_on && dc == INF && ds == INF) { a->lost++; p->fate = FATE_LOST; break; }
        int coll = dc < ds;              /* ties: surface crossing */
        double d = coll ? dc : ds;
        /* time dependence: the flight ends where the clock reaches t_cut, at the
         * distance (t_cut - t) / (1/v); a tie goes to the collision or crossing */
        int tcut = 0;
        double ta = p->t, tb = p->t;
        if (c->time_on) {
            /* multigroup: 1/v given per group; continuous energy: v = K sqrt(E).
             * Plain: flight time d / v, distance to the cutoff (t_cut - t) v.
             * Strict: 1/v rounded once per flight, (t_cut - t) / (1/v), and the
             * clock advanced by one fused multiply-add t + d (1/v). */
            if (c->ce && !strict) {
                double vel = c->kv * sqrt(p->E);
                double dt = (c->tcut - p->t) * vel;
                if (dt < 0.0) dt = 0.0;
                if (dt < d) { tcut = 1; d = dt; }
                if (!tcut && d == INF) { a->lost++; p->fate = FATE_LOST; break; }
                tb = tcut ? c->tcut : p->t + d / vel;
            } else {
                double iv = c->ce ? 1.0 / (c->kv * sqrt(p->E)) : c->invv[p->g];
                double dt = (c->tcut - p->t) / iv;
                if (dt < 0.0) dt = 0.0;
                if (dt < d) { tcut = 1; d = dt; }
                if (!tcut && d == INF) { a->lost++; p->fate = FATE_LOST; break; }
                tb = tcut ? c->tcut : (strict ? fma(d, iv, p->t) : p->t + d * iv);
            }
        }
        /* move: r + d Omega (strict: one fused multiply-add per coordinate) */
        if (strict) {
            p->x = fma(d, p->u, p->x);
            p->y = fma(d, p->v, p->y);
            p->z = fma(d, p->w, p->z);
        } else {
            p->x = p->x + d * p->u;
            p->y = p->y + d * p->v;
            p->z = p->z + d * p->w;
        }
        /* track-length estimators; with time bins, the time spent in each bin
         * over the bin width (population) */
        for (int t = 0; t < c->nt; t++) {
            const Tally *T = &c->tally[t];
            int bin, e;
            if (!tally_bin(c, T, p, &bin, &e)) continue;
            if (T->ntb == 0) {
                a->acc[t][(size_t)batch * T->nbins * T->ne + (size_t)bin * T->ne + e] += d;
                continue;
            }
            double *row = a->acc[t] + ((size_t)batch * T->nbins * T->ne + (size_t)bin * T->ne + e) *
                                          (size_t)T->ntb;
            /* overlap of [ta, tb] with the bin over the bin width (strict: times
             * the width's reciprocal rounded once) */
            for (int k = 0; k < T->ntb; k++) {
                double lo = ta > T->tedges[k] ? ta : T->tedges[k];
                double hi = tb < T->tedges[k + 1] ? tb : T->tedges[k + 1];
                if (lo < hi)
                    row[k] += strict ? (hi - lo) * T->tinvw[k]
                                     : (hi - lo) / (T->tedges[k + 1] - T->tedges[k]);
            }
        }
        p->t = tb;
        a->ktl += d * nusf;
        if (tcut) { a->timecut++; p->fate = FATE_TIME; break; }
        double ownb = own;
        if (gr && (p->ucell >= 0 ? p->ucell : p->cell) == gr->det_cell)
            own = own + gr->weights[p->g] * d;
        if (!coll) {
            p->ncross++;
            if (gr && sigt != 0.0) grad_rec(gr, p->mat * G + p->g, -d, ownb, p->nfis, pid);
            int r = cross(c, p, kind, which);
            if (r == 1) { a->leak++; p->fate = FATE_LEAKED; break; }
            if (r < 0) { a->lost++; p->fate = FATE_LOST; break; }
            continue;
        }
        /* collision */
        p->ncoll++;
        int nfb = p->nfis;
        if (!c->ce) {
            int g = p->g;
            const double rsig = 1.0 / sigt;           /* 1/Sigma_t (Sigma_t > 0 here) */
            const double mu = m->nusf[g] / sigt;      /* expected fission sites */
            const double mufl = floor(mu), mufr = mu - mufl;
            a->kc += mu;
            if (gr) grad_rec(gr, p->mat * G + g, rsig - d, ownb, nfb, pid);
            /* fission sites: floor(mu) + [xi <= frac(mu)], mu = nuSigma_f/Sigma_t.
             * Reading: no division by k; the population is controlled by resampling. */
            double xi = draw(&p->s);
            int nf = (int)mufl + (xi <= mufr ? 1 : 0);
            if (gr && m->nusf[g] != 0.0 && mufr != 0.0) {
                double fac = nf > (int)mufl ? 1.0 / mufr : -1.0 / (1.0 - mufr);
                int nm = c->nm;
                grad_rec(gr, nm * G + nm * G * G + p->mat * G + g, rsig * fac, ownb, nfb, pid);
                grad_rec(gr, p->mat * G + g, -(mu * rsig) * fac, ownb, nfb, pid);
            }
            for (int k = 0; k < nf; k++) { bank_push(a, p); p->nfis++; }
            /* analog reaction: scatter with probability Sigma_s,tot / Sigma_t, i.e.
             * when xi Sigma_t <= Sigma_s,tot (strict: xi <= the ratio rounded once) */
            xi = draw(&p->s);
            int scatter = strict ? xi <= m->ps[g] : xi * sigt <= m->stot[g];
            if (scatter) {
                xi = draw(&p->s);
                int gp = sample_discrete(&m->sigs[g * G], m->stot[g], &m->scdf[g * G], G, xi, strict);
                if (gr) {
                    int nm = c->nm;
                    grad_rec(gr, nm * G + (p->mat * G + g) * G + gp, 1.0 / m->sigs[g * G + gp], ownb,
                             nfb, pid);
                    grad_rec(gr, p->mat * G + g, -rsig, ownb, nfb, pid);
                }
                p->g = gp;
                iso_dir(&p->s, &p->u, &p->v, &p->w, strict);   /* isotropic (P0) scattering */
                set_recip(p);
            } else {
                if (gr) {
                    double sa = m->sigt[g] - m->stot[g];
                    if (sa > 0.0) {
                        int nm = c->nm;
                        grad_rec(gr, p->mat * G + g, 1.0 / sa - rsig, ownb, nfb, pid);
                        for (int h = 0; h < G; h++)
                            if (m->sigs[g * G + h] != 0.0)
                                grad_rec(gr, nm * G + (p->mat * G + g) * G + h, -1.0 / sa, ownb, nfb,
                                         pid);
                    }
                }
                p->alive = 0;
            }
        } else {
            const MatCE *mc = &c->mce[p->mat];
            ce_lookup(c, p->mat, p->E, &x, strict);   /* per-nuclide values for the reaction */
            /* strict: nuSigma_f times the flight's reciprocal 1/Sigma_t, rounded once */
            a->kc += strict ? nusf * (1.0 / sigt) : nusf / sigt;
            /* nuclide by xi Sigma_t against the running sum of N_i sigma_t,i */
            double target = draw(&p->s) * sigt;
            double cum = 0.0;
            int sel = mc->n - 1;
            for (int k = 0; k < mc->n; k++) {
                cum = strict ? fma(mc->dens[k], x.st[k], cum) : cum + mc->dens[k] * x.st[k];
                if (target <= cum) { sel = k; break; }
            }
            const Nuclide *u = &c->nuc[mc->nuc[sel]];
            double mu = u->nu * x.sf[sel] / x.st[sel];
            double fl = floor(mu);
            double xi = draw(&p->s);
            int nf = (int)fl + (xi <= mu - fl ? 1 : 0);
            for (int k = 0; k < nf; k++) { bank_push(a, p); p->nfis++; }
            /* scatter (elastic, target at rest) with probability sigma_s,i/sigma_t,i */
            xi = draw(&p->s);
            if (xi * x.st[sel] <= x.ss[sel]) {
                if (c->fg_kT > 0.0 && p->E < c->fg_emax)
                    p->E = free_gas(p->E, u->A, c->fg_kT, &p->s, &p->u, &p->v, &p->w, strict);
                else
                    p->E = elastic(p->E, u->A, &p->s, &p->u, &p->v, &p->w, strict);
                set_recip(p);
            } else {
                p->alive = 0;
            }
        }
        if (!p->alive) { p->fate = FATE_ABSORBED; break; }
        if (c->max_coll && p->ncoll >= c->max_coll) { p->alive = 0; p->fate = FATE_CUT; break; }
    }
    if (gr) gr->own[pid] = own;
    a->coll += p->ncoll;
    a->crossn += p->ncross;
}

/* ------------------------------------------------------------------------- */
/* sources                                                                    */
static int birth_energy(const orc_ctx *c, Particle *p)
{
    if (c->ce) {
        p->E = maxwell(&p->s, c->strict);
    } else {
        const MatMG *m = &c->mg[p->mat];
        p->g = sample_discrete(m->chi, m->chitot[0], m->chicdf, c->G, draw(&p->s), c->strict);
    }
    return 0;
}

static int mat_fissile(const orc_ctx *c, int mat)
{
    return c->ce ? c->mce[mat].fissile : c->mg[mat].fissile;
}

/* Draw order: position (3 draws per rejection attempt for a box), energy
 * (group or E), direction.  The point is located with a zero direction.     */
static int sample_source(const orc_ctx *c, Particle *p)
{
    const Source *s = &c->src;
    p->u = p->v = p->w = 0.0;
    p->t = c->time_on ? c->t0 : 0.0;
    if (s->kind == ORC_SRC_BOX) {
        int ok = 0;
        for (int t = 0; t < MAX_TRIES && !ok; t++) {
            p->x = s->p[0] + draw(&p->s) * (s->p[1] - s->p[0]);
            p->y = s->p[2] + draw(&p->s) * (s->p[3] - s->p[2]);
            p->z = s->p[4] + draw(&p->s) * (s->p[5] - s->p[4]);
            if (locate_full(c, p) < 0) continue;
            ok = s->accept == ORC_ACCEPT_ANY || mat_fissile(c, p->mat);
        }
        if (!ok) return -1;
    } else {
        p->x = s->p[0]; p->y = s->p[1]; p->z = s->p[2];
        if (locate_full(c, p) < 0) return -1;
    }
    switch (s->ekind) {
    case ORC_E_CHI: birth_energy(c, p); break;
    case ORC_E_PDF:
        p->g = sample_discrete(s->edata, s->etot, s->ecdf, s->ne, draw(&p->s), c->strict);
        break;
    case ORC_E_FIXED: p->E = s->edata[0]; break;
    default: p->E = maxwell(&p->s, c->strict);
    }
    if (s->dkind == ORC_DIR_BEAM) { p->u = s->beam[0]; p->v = s->beam[1]; p->w = s->beam[2]; }
    else iso_dir(&p->s, &p->u, &p->v, &p->w, c->strict);
    set_recip(p);
    return 0;
}

static void from_site(const orc_ctx *c, Particle *p, const Site *b)
{
    p->x = b->x; p->y = b->y; p->z = b->z; p->t = b->t;
    p->cell = b->cell; p->ix = b->ix; p->iy = b->iy; p->ucell = b->ucell; p->mat = b->mat;
    birth_energy(c, p);
    iso_dir(&p->s, &p->u, &p->v, &p->w, c->strict);
    set_recip(p);
}

static int site_cmp(const void *a, const void *b)
{
    const Site *x = a, *y = b;
    if (x->parent != y->parent) return x->parent < y->parent ? -1 : 1;
    return x->child < y->child ? -1 : (x->child > y->child);
}

/* ------------------------------------------------------------------------- */
static int prepare(orc_ctx *c)
{
    if (!c->src_set) return fail(c, ORC_ESTATE, "no source");
    if (c->nc == 0) return fail(c, ORC_ESTATE, "no cells");
    if (c->ce < 0) return fail(c, ORC_ESTATE, "no materials");
    build_universes(c);
    for (int t = 0; t < c->nt; t++) {
        Tally *T = &c->tally[t];
        T->nbins = T->filter == ORC_FILTER_CELL ? c->nc
                 : T->filter == ORC_FILTER_LATTICE ? (c->nl ? c->lat[0].nx * c->lat[0].ny : 0)
                 : (c->ce ? c->nmc : c->nm);
        T->ne = c->ce ? T->nedges - 1 : c->G;
        if (c->ce && T->nedges < 2) return fail(c, ORC_EINVAL, "CE tally needs energy edges");
    }
    if (c->time_on && !c->ce && !c->invv) return fail(c, ORC_ESTATE, "no inverse speeds");
    if (c->ce && c->strict) build_macro(c);
    c->kv = sqrt(2.0 * 1.602176634e-19 / 1.67492749804e-27) * 100.0;
    free_results(c);
    memset(c->counters, 0, sizeof c->counters);
    c->t_sum = calloc(c->nt ? c->nt : 1, sizeof(double *));
    c->t_sum2 = calloc(c->nt ? c->nt : 1, sizeof(double *));
    c->t_mean = calloc(c->nt ? c->nt : 1, sizeof(double *));
    c->t_sd = calloc(c->nt ? c->nt : 1, sizeof(double *));
    for (int t = 0; t < c->nt; t++) {
        size_t nb = tally_len(&c->tally[t]);
        c->t_sum[t] = calloc(nb ? nb : 1, sizeof(double));
        c->t_sum2[t] = calloc(nb ? nb : 1, sizeof(double));
        c->t_mean[t] = calloc(nb ? nb : 1, sizeof(double));
        c->t_sd[t] = calloc(nb ? nb : 1, sizeof(double));
    }
    return 0;
}

static Acc *make_accs(const orc_ctx *c, int nthr, int nbatch)
{
    Acc *A = calloc((size_t)nthr, sizeof(Acc));
    for (int i = 0; i < nthr; i++) {
        A[i].acc = calloc(c->nt ? c->nt : 1, sizeof(double *));
        for (int t = 0; t < c->nt; t++)
            A[i].acc[t] = calloc((size_t)nbatch * tally_len(&c->tally[t]) + 1,
                                 sizeof(double));
    }
    return A;
}

static void free_accs(const orc_ctx *c, Acc *A, int nthr)
{
    for (int i = 0; i < nthr; i++) {
        for (int t = 0; t < c->nt; t++) free(A[i].acc[t]);
        free(A[i].acc);
        free(A[i].bank);
    }
    free(A);
}

/* merge per-thread banks and sort them by (parent, child): the order is unique */
static Site *merge_banks(Acc *A, int nthr, int64_t *M)
{
    int64_t tot = 0;
    for (int i = 0; i < nthr; i++) tot += A[i].nbank;
    Site *b = malloc(sizeof(Site) * (size_t)(tot ? tot : 1));
    int64_t k = 0;
    for (int i = 0; i < nthr; i++) {
        memcpy(b + k, A[i].bank, sizeof(Site) * (size_t)A[i].nbank);
        k += A[i].nbank;
        A[i].nbank = 0;
    }
    qsort(b, (size_t)tot, sizeof(Site), site_cmp);
    *M = tot;
    return b;
}

static int nthreads(int threads)
{
#ifdef _OPENMP
    return threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

static void record_histories(orc_ctx *c, const Particle *P, int64_t n)
{
    free(c->h_coll); free(c->h_cross); free(c->h_fis); free(c->h_rng);
    free(c->h_fate); free(c->h_g);
    c->nhist = n;
    c->h_fate = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    c->h_g = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    c->h_coll = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    c->h_cross = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    c->h_fis = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    c->h_rng = malloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
    for (int64_t j = 0; j < n; j++) {
        c->h_coll[j] = P[j].ncoll; c->h_cross[j] = P[j].ncross;
        c->h_fis[j] = P[j].nfis; c->h_rng[j] = P[j].s;
        c->h_fate[j] = P[j].fate; c->h_g[j] = P[j].g;
    }
}

static void sum_counters(orc_ctx *c, Acc *A, int nthr)
{
    for (int i = 0; i < nthr; i++) {
        c->counters[1] += A[i].coll; c->counters[2] += A[i].crossn; c->counters[3] += A[i].leak;
        c->counters[4] += A[i].lost; c->counters[5] += A[i].capped;
        c->counters[7] += A[i].timecut;
        A[i].coll = A[i].crossn = A[i].leak = A[i].lost = A[i].capped = A[i].timecut = 0;
    }
}

static void mean_sd(double sum, double sum2, int n, double *mean, double *sd)
{
    *mean = sum / n;
    if (n > 1) {
        double var = (sum2 - n * (*mean) * (*mean)) / (n - 1);
        *sd = sqrt(var > 0.0 ? var / n : 0.0);
    } else {
        *sd = 0.0;
    }
}

/* Power iteration (Sec. 4 runs 50 inactive + 100 active cycles).  Reading:
 * cycle c's particle j uses stream c 2^32 + j; after a cycle the bank (sorted
 * by parent and child) of M sites is resampled systematically to N:
 * site j <- bank[floor((j + xi) M / N)] (orc_site_index), xi the first draw of
 * stream c 2^32 + 2^32 - 1.  Per cycle k_analog = M/N, k_TL = sum d nuSigma_f / N,
 * k_C = sum nuSigma_f/Sigma_t / N; k and tallies are means over active
 * cycles with sd = s / sqrt(n_active).                                        */
int orc_run_eigen(orc_ctx *c, int64_t n, int inactive, int active, uint64_t seed, int threads)
{
    if (c->time_on) return fail(c, ORC_EINVAL, "time dependence is for fixed-source runs");
    int r = prepare(c);
    if (r) return r;
    if (n <= 0 || active < 1 || inactive < 0) return fail(c, ORC_EINVAL, "bad run size");
    int nthr = nthreads(threads);
    int ncyc = inactive + active;
    Acc *A = make_accs(c, nthr, 1);
    Particle *P = calloc((size_t)n, sizeof(Particle));
    int64_t *site = malloc(sizeof(int64_t) * (size_t)n);
    Site *bank = NULL;
    int64_t M = 0;
    c->ncyc = ncyc;
    c->cyc_ktl = calloc((size_t)ncyc, sizeof(double));
    c->cyc_kc = calloc((size_t)ncyc, sizeof(double));
    c->cyc_m = calloc((size_t)ncyc, sizeof(int64_t));
    double ks[3] = {0, 0, 0}, ks2[3] = {0, 0, 0};
    int err = 0;
    for (int cyc = 0; cyc < ncyc && !err; cyc++) {
        int bad = 0;
#pragma omp parallel for num_threads(nthr) schedule(static) reduction(+ : bad)
        for (int64_t j = 0; j < n; j++) {
            Particle *p = &P[j];
            memset(p, 0, sizeof *p);
            p->s = orc_rng_stream(seed, ((uint64_t)cyc << 32) + (uint64_t)j);
            p->index = j;
            p->root = j;
            p->alive = 1;
            if (cyc == 0) {
                if (sample_source(c, p) < 0) { bad++; continue; }
            } else {
                from_site(c, p, &bank[site[j]]);
            }
#ifdef _OPENMP
            Acc *a = &A[omp_get_thread_num()];
#else
            Acc *a = &A[0];
#endif
            transport(c, p, a, 0, NULL, j);
        }
        if (bad) { err = fail(c, ORC_ESTATE, "source sampling failed"); break; }
        free(bank);
        bank = merge_banks(A, nthr, &M);
        double ktl = 0.0, kc = 0.0;
        for (int i = 0; i < nthr; i++) { ktl += A[i].ktl; kc += A[i].kc; A[i].ktl = A[i].kc = 0.0; }
        ktl /= (double)n;
        kc /= (double)n;
        double ka = (double)M / (double)n;
        c->cyc_ktl[cyc] = ktl; c->cyc_kc[cyc] = kc; c->cyc_m[cyc] = M;
        for (int t = 0; t < c->nt; t++) {
            size_t nb = tally_len(&c->tally[t]);
            for (size_t b = 0; b < nb; b++) {
                double v = 0.0;
                for (int i = 0; i < nthr; i++) { v += A[i].acc[t][b]; A[i].acc[t][b] = 0.0; }
                v /= (double)n;
                if (cyc >= inactive) { c->t_sum[t][b] += v; c->t_sum2[t][b] += v * v; }
            }
        }
        if (cyc >= inactive) {
            double kv[3] = {ktl, kc, ka};
            for (int q = 0; q < 3; q++) { ks[q] += kv[q]; ks2[q] += kv[q] * kv[q]; }
        }
        sum_counters(c, A, nthr);
        c->counters[0] += n;
        if (cyc == ncyc - 1) record_histories(c, P, n);
        if (M == 0) { err = fail(c, ORC_ESTATE, "fission bank empty after cycle %d", cyc); break; }
        uint64_t rs = orc_rng_stream(seed, ((uint64_t)cyc << 32) + 0xFFFFFFFFULL);
        uint64_t xn = draw_n(&rs);
        for (int64_t j = 0; j < n; j++) site[j] = orc_site_index(j, xn, M, n);
    }
    if (!err) {
        for (int q = 0; q < 3; q++) mean_sd(ks[q], ks2[q], active, &c->k[2 * q], &c->k[2 * q + 1]);
        for (int t = 0; t < c->nt; t++) {
            size_t nb = tally_len(&c->tally[t]);
            for (size_t b = 0; b < nb; b++)
                mean_sd(c->t_sum[t][b], c->t_sum2[t][b], active, &c->t_mean[t][b], &c->t_sd[t][b]);
        }
        c->nbank = M;
        c->bank = bank;
        bank = NULL;
        if (c->counters[4] > 0 && (double)c->counters[4] > 1e-6 * (double)c->counters[0])
            err = fail(c, ORC_ELOST, "lost particles: %lld", (long long)c->counters[4]);
    }
    c->counters[6] = ncyc;
    free(bank); free(site); free(P);
    free_accs(c, A, nthr);
    return err;
}

/* Fixed source: generation 0 from the source (stream j), generation g+1 is the
 * whole sorted bank of generation g (stream (g+1) 2^32 + j), until the bank is
 * empty.  Reading: source particle j belongs to batch floor(j B / N) and its
 * descendants inherit it; tallies are batch means per source particle.       */
static int run_fixed(orc_ctx *c, int64_t n, int batches, uint64_t seed, int threads, Grad *gr)
{
    int r = prepare(c);
    if (r) return r;
    if (n <= 0 || batches < 1 || batches > n) return fail(c, ORC_EINVAL, "bad run size");
    int nthr = gr ? 1 : nthreads(threads);
    Acc *A = make_accs(c, nthr, batches);
    Site *bank = NULL;
    int64_t M = 0, ngen_n = n;
    int err = 0, gen;
    int64_t *gen_base = NULL, *gen_n = NULL;
    int64_t **gen_off = NULL;   /* per generation: first child index of each particle */
    for (gen = 0; gen < MAX_GEN; gen++) {
        Particle *P = calloc((size_t)ngen_n, sizeof(Particle));
        int bad = 0;
        int64_t base = 0;
        if (gr) {
            gen_base = realloc(gen_base, sizeof(int64_t) * (gen + 1));
            gen_n = realloc(gen_n, sizeof(int64_t) * (gen + 1));
            gen_off = realloc(gen_off, sizeof(int64_t *) * (gen + 1));
            base = gen ? gen_base[gen - 1] + gen_n[gen - 1] : 0;
            gen_base[gen] = base;
            gen_n[gen] = ngen_n;
            gr->own = realloc(gr->own, sizeof(double) * (size_t)(base + ngen_n));
        }
#pragma omp parallel for num_threads(nthr) schedule(static) reduction(+ : bad)
        for (int64_t j = 0; j < ngen_n; j++) {
            Particle *p = &P[j];
            p->s = orc_rng_stream(seed, ((uint64_t)gen << 32) + (uint64_t)j);
            p->index = j;
            p->alive = 1;
            if (gen == 0) {
                p->root = j;
                if (sample_source(c, p) < 0) { bad++; continue; }
            } else {
                p->root = bank[j].root;
                from_site(c, p, &bank[j]);
            }
#ifdef _OPENMP
            Acc *a = &A[omp_get_thread_num()];
#else
            Acc *a = &A[0];
#endif
            int batch = (int)((p->root * (int64_t)batches) / n);
            transport(c, p, a, batch, gr, gr ? base + j : j);
        }
        if (bad) { free(P); err = fail(c, ORC_ESTATE, "source sampling failed"); break; }
        if (gen == 0) record_histories(c, P, ngen_n);
        sum_counters(c, A, nthr);
        c->counters[0] += ngen_n;
        Site *nb = merge_banks(A, nthr, &M);
        if (gen == 0) {
            c->bank = malloc(sizeof(Site) * (size_t)(M ? M : 1));
            memcpy(c->bank, nb, sizeof(Site) * (size_t)M);
            c->nbank = M;
        }
        if (gr) {
            int64_t *off = malloc(sizeof(int64_t) * (size_t)(ngen_n + 1));
            for (int64_t j = 0; j <= ngen_n; j++) off[j] = 0;
            for (int64_t k = 0; k < M; k++) off[nb[k].parent + 1]++;
            for (int64_t j = 0; j < ngen_n; j++) off[j + 1] += off[j];
            gen_off[gen] = off;
        }
        free(P);
        free(bank);
        bank = nb;
        ngen_n = M;
        if (M == 0) break;
    }
    if (!err && gen == MAX_GEN) err = fail(c, ORC_ETIMEOUT, "generation limit reached");
    c->counters[6] = gen + 1;
    if (!err) {
        /* batch statistics */
        int64_t *nb = calloc((size_t)batches, sizeof(int64_t));
        for (int64_t j = 0; j < n; j++) nb[(j * batches) / n]++;
        for (int t = 0; t < c->nt; t++) {
            size_t ns = tally_len(&c->tally[t]);
            for (size_t b = 0; b < ns; b++) {
                double s = 0.0, s2 = 0.0;
                for (int q = 0; q < batches; q++) {
                    double v = 0.0;
                    for (int i = 0; i < nthr; i++) v += A[i].acc[t][(size_t)q * ns + b];
                    v /= (double)nb[q];
                    s += v;
                    s2 += v * v;
                }
                mean_sd(s, s2, batches, &c->t_mean[t][b], &c->t_sd[t][b]);
            }
        }
        free(nb);
        if (c->counters[4] > 0 && (double)c->counters[4] > 1e-6 * (double)c->counters[0])
            err = fail(c, ORC_ELOST, "lost particles: %lld", (long long)c->counters[4]);
    }
    if (gr && !err) {
        /* subtree totals, last generation first */
        int ng = gen + 1 <= MAX_GEN ? gen + 1 : MAX_GEN;
        int64_t tot = gen_base[ng - 1] + gen_n[ng - 1];
        double *sub = malloc(sizeof(double) * (size_t)(tot ? tot : 1));
        for (int g = ng - 1; g >= 0; g--) {
            for (int64_t j = 0; j < gen_n[g]; j++) {
                double s = gr->own[gen_base[g] + j];
                if (g + 1 < ng)
                    for (int64_t k = gen_off[g][j]; k < gen_off[g][j + 1]; k++)
                        s += sub[gen_base[g + 1] + k];
                sub[gen_base[g] + j] = s;
            }
        }
        /* combine every score with its downstream tally D */
        int npar = c->nm * c->G * (2 + c->G);
        double *acc = calloc((size_t)npar, sizeof(double));
        for (int64_t q = 0; q < gr->n; q++) {
            int64_t pid = gr->pid[q];
            int g = 0;
            while (g + 1 < ng && pid >= gen_base[g + 1]) g++;
            int64_t j = pid - gen_base[g];
            double D = gr->own[pid] - gr->ownb[q];
            if (g + 1 < ng)
                for (int64_t k = gen_off[g][j] + gr->nfb[q]; k < gen_off[g][j + 1]; k++)
                    D += sub[gen_base[g + 1] + k];
            acc[gr->param[q]] += gr->val[q] * D;
        }
        for (int k = 0; k < npar; k++) acc[k] /= (double)n;
        gr->val = realloc(gr->val, sizeof(double) * (size_t)(npar > gr->cap ? npar : gr->cap));
        memcpy(gr->val, acc, sizeof(double) * (size_t)npar);
        free(acc);
        free(sub);
    }
    if (gr) {
        for (int g = 0; g <= gen && g < MAX_GEN; g++) free(gen_off[g]);
        free(gen_off); free(gen_base); free(gen_n);
    }
    free(bank);
    free_accs(c, A, nthr);
    return err;
}

int orc_run_fixed(orc_ctx *c, int64_t n, int batches, uint64_t seed, int threads)
{
    return run_fixed(c, n, batches, seed, threads, NULL);
}

/* Likelihood-ratio derivative of a cell's track-length tally (fixed source,
 * multigroup).  The paper has no derivative; this is the textbook score
 * function estimator: dE[T]/dtheta = E[sum_e s_e D_e], where s_e is the
 * derivative of the log-probability of event e and D_e is the tally scored
 * from the start of e's flight onward by the particle plus the full subtree
 * tallies of the secondaries it banks at or after e.  Scores (weight 1):
 *  flight ending at a surface        dSigma_t: -d
 *  flight ending in a collision      dSigma_t: 1/Sigma_t - d
 *  scatter g -> g'                   dSigma_s[g,g']: 1/Sigma_s[g,g'], dSigma_t: -1/Sigma_t
 *  absorption (Sigma_a = Sigma_t - Sigma_s,tot)
 *                                    dSigma_t: 1/Sigma_a - 1/Sigma_t, dSigma_s[g,*]: -1/Sigma_a
 *  fission count, mu = nuSigma_f/Sigma_t, P(floor mu + 1) = frac mu
 *                                    d log P = mu'/frac (n = floor+1) or -mu'/(1-frac),
 *                                    mu'_nuSigma_f = 1/Sigma_t, mu'_Sigma_t = -mu/Sigma_t
 * Parameters whose value is 0 (and fission counts with frac mu = 0) take no
 * score.  This oracle stores every score with its context during the forward
 * pass and combines them afterwards (no replay).                              */
int orc_grad_fixed(orc_ctx *c, int64_t n, uint64_t seed, int cell, const double *weights,
                   double *d_sigt, double *d_sigs, double *d_nusf, double *tally)
{
    if (c->ce) return fail(c, ORC_EINVAL, "derivatives are multigroup only");
    if (c->time_on) return fail(c, ORC_EINVAL, "derivatives are for time-independent runs");
    Grad gr;
    memset(&gr, 0, sizeof gr);
    gr.det_cell = cell;
    gr.weights = weights;
    int mc = c->max_coll;
    int r = run_fixed(c, n, 1, seed, 1, &gr);
    c->max_coll = mc;
    if (!r) {
        int G = c->G, nm = c->nm;
        memcpy(d_sigt, gr.val, sizeof(double) * nm * G);
        memcpy(d_sigs, gr.val + nm * G, sizeof(double) * nm * G * G);
        memcpy(d_nusf, gr.val + nm * G + nm * G * G, sizeof(double) * nm * G);
        for (int t = 0; t < c->nt; t++)
            if (c->tally[t].filter == ORC_FILTER_CELL) {
                for (int g = 0; g < G; g++) tally[g] = c->t_mean[t][(size_t)cell * G + g];
                break;
            }
    }
    free(gr.param); free(gr.val); free(gr.ownb); free(gr.nfb); free(gr.pid); free(gr.own);
    return r;
}

/* Histories j = idx[k] of the first cycle / generation 0 (sources from the
 * source definition, stream j), each run alone: for checking single histories
 * of a large run without running all of it. */
int orc_histories_by_index(orc_ctx *c, uint64_t seed, int64_t n_idx, const int64_t *idx,
                           int32_t *n_coll, int32_t *n_cross, uint64_t *rng_end, int32_t *n_fis,
                           int32_t *fate, int32_t *g_end)
{
    int r = prepare(c);
    if (r) return r;
    Acc *A = make_accs(c, 1, 1);
    for (int64_t k = 0; k < n_idx; k++) {
        Particle p;
        memset(&p, 0, sizeof p);
        p.s = orc_rng_stream(seed, (uint64_t)idx[k]);
        p.index = idx[k];
        p.root = 0;
        p.alive = 1;
        if (sample_source(c, &p) < 0) {
            free_accs(c, A, 1);
            return fail(c, ORC_ESTATE, "source sampling failed");
        }
        transport(c, &p, &A[0], 0, NULL, 0);
        A[0].nbank = 0;
        n_coll[k] = p.ncoll; n_cross[k] = p.ncross; rng_end[k] = p.s; n_fis[k] = p.nfis;
        fate[k] = p.fate; g_end[k] = p.g;
    }
    free_accs(c, A, 1);
    return 0;
}

/* ------------------------------------------------------------------------- */
int orc_get_k(const orc_ctx *c, double out[6])
{
    memcpy(out, c->k, sizeof c->k);
    return 0;
}

int orc_get_cycle_k(const orc_ctx *c, int n_cycles, double *k_tl, double *k_c, int64_t *bank_size)
{
    for (int i = 0; i < n_cycles && i < c->ncyc; i++) {
        k_tl[i] = c->cyc_ktl[i]; k_c[i] = c->cyc_kc[i]; bank_size[i] = c->cyc_m[i];
    }
    return 0;
}

int orc_tally_size(const orc_ctx *c, int tally, int *n_bins, int *n_ebins, int *n_tbins)
{
    if (tally < 0 || tally >= c->nt) return ORC_EINVAL;
    *n_bins = c->tally[tally].nbins;
    *n_ebins = c->tally[tally].ne;
    *n_tbins = c->tally[tally].ntb ? c->tally[tally].ntb : 1;
    return 0;
}

int orc_get_tally(const orc_ctx *c, int tally, double *mean, double *sd)
{
    if (tally < 0 || tally >= c->nt || !c->t_mean) return ORC_EINVAL;
    size_t nb = tally_len(&c->tally[tally]);
    memcpy(mean, c->t_mean[tally], sizeof(double) * nb);
    memcpy(sd, c->t_sd[tally], sizeof(double) * nb);
    return 0;
}

int orc_get_counters(const orc_ctx *c, int64_t out[8])
{
    memcpy(out, c->counters, sizeof c->counters);
    return 0;
}

int64_t orc_history_count(const orc_ctx *c) { return c->nhist; }

int orc_get_histories(const orc_ctx *c, int32_t *n_coll, int32_t *n_cross, uint64_t *rng_end,
                      int32_t *n_fis, int32_t *fate, int32_t *g_end)
{
    for (int64_t j = 0; j < c->nhist; j++) {
        n_coll[j] = c->h_coll[j]; n_cross[j] = c->h_cross[j];
        rng_end[j] = c->h_rng[j]; n_fis[j] = c->h_fis[j];
        fate[j] = c->h_fate[j]; g_end[j] = c->h_g[j];
    }
    return 0;
}

int64_t orc_bank_count(const orc_ctx *c) { return c->nbank; }

int orc_get_bank(const orc_ctx *c, double *xyz, int64_t *parent, int32_t *child, int32_t *mat)
{
    for (int64_t k = 0; k < c->nbank; k++) {
        xyz[3 * k] = c->bank[k].x; xyz[3 * k + 1] = c->bank[k].y; xyz[3 * k + 2] = c->bank[k].z;
        parent[k] = c->bank[k].parent; child[k] = c->bank[k].child; mat[k] = c->bank[k].mat;
    }
    return 0;
}
