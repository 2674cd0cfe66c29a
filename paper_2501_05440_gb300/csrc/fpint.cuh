// fpint.cuh -- correctly rounded float64 square root, quotient and reciprocal
// computed on the integer and float32 pipes.
//
// On this chip a float64 instruction occupies the SM's float64 unit for 16
// cycles and has 64 cycles of latency, so the hardware square root and
// division (chains of dependent float64 operations) cost the transport loop
// both throughput and latency.  The functions here return the same values --
// the IEEE round-to-nearest results, like sqrt(), x / y and 1.0 / y -- from
// integer arithmetic on the 53-bit significands:
//
//   * a float32 approximation of the root or reciprocal (the PTX
//     rsqrt.approx / rcp.approx instructions, relative error below 2^-22)
//     of the significand, built from its bits (no conversion instruction:
//     conversions between 64-bit integers and floats run on the float64
//     pipe),
//   * two Newton corrections, each from an exact integer residual
//     (N - Q^2 for the root, N - Q D for the quotient) scaled by that
//     float32 approximation (the Newton-Raphson refinement with residual
//     correction of Markstein, IBM J. Res. Dev. 34(1), 1990; the integer
//     root with remainder of Brent and Zimmermann, Modern Computer
//     Arithmetic, 2010, Sec. 1.5),
//   * a last exact residual that moves the candidate by at most one unit to
//     the nearest value (no ties can occur for a square root or a quotient
//     of 53-bit significands).
//
// The error bounds of the two corrections and the ranges of the 64-bit
// products leave a factor of more than ten to the approximations' error
// bound (checked with approximations perturbed by up to 2^-18.3).  Operands
// whose result or inputs are zero, subnormal, infinite or NaN take the
// hardware operation (a branch that transport arithmetic practically never
// takes).
#pragma once
#include <cstdint>

namespace mcgb {

__device__ __forceinline__ float rsqrt_approx_f32(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx_f32(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The hardware operations for the operands the integer paths leave out, kept
// out of line: inlined at every call site, their code (taken practically
// never) made the transport loops larger and slowed their instruction fetch.
// A translation unit that defines MCGB_FALLBACK_INLINE before including this
// header inlines them instead (the derivative replay's per-history loop ran
// 25% slower with the calls).
#ifdef MCGB_FALLBACK_INLINE
#define MCGB_FALLBACK __forceinline__
#else
#define MCGB_FALLBACK __noinline__
#endif
static __device__ MCGB_FALLBACK double sqrt_hw(double x) { return sqrt(x); }
static __device__ MCGB_FALLBACK double div_hw(double n, double d) { return n / d; }

constexpr uint64_t FP_FRAC = (1ULL << 52) - 1;
constexpr uint64_t FP_HIDDEN = 1ULL << 52;
constexpr uint64_t FP_SIGN = 0x8000000000000000ULL;

// y 2^25 as an integer, for a float y in [0.25, 2) (the approximations below
// lie in (0.5, 1] up to their error)
__device__ __forceinline__ uint32_t f32_fixed25(float y)
{
    const uint32_t b = __float_as_uint(y);
    return ((b & 0x7FFFFFu) | 0x800000u) << ((b >> 23) - 125u);
}

// sqrt(x), correctly rounded.  x = M2 2^e2 with e2 even and M2 in [2^52, 2^54);
// the result significand is R = round(sqrt(N)), N = M2 2^52 in [2^104, 2^106).
__device__ __forceinline__ double sqrt_rn(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t E = (uint32_t)(b >> 52);          // sign bit included: negatives fall back
    if (E - 1u >= 2046u) return sqrt_hw(x);
    const uint64_t F = b & FP_FRAC;
    const uint32_t odd = (~E) & 1u;                   // E even <=> E - 1075 odd
    const uint64_t M2 = (F | FP_HIDDEN) << odd;
    const int Er = (((int)E - 1075 - (int)odd) >> 1) + 1049;   // biased exponent of the root
    // m = M2 / 2^52 in [1, 4) as a float built from the bits (fraction truncated);
    // y ~ m^-1/2 (Y = y 2^25), s = m y ~ m^1/2 with significand ms: Q0 = ms 2^sh
    const float mf = __uint_as_float(((127u + odd) << 23) | (uint32_t)(F >> 29));
    const float y = rsqrt_approx_f32(mf);
    const int64_t Y = f32_fixed25(y);
    const uint32_t sb = __float_as_uint(mf * y);
    const uint64_t ms = (sb & 0x7FFFFFu) | 0x800000u;
    const int sh = (int)(sb >> 23) - 98;
    // (N - Q0^2) / 2^52 = M2 - ms^2 2^(2 sh - 52), exact in 64 bits
    const int64_t R0 = (int64_t)M2 - (int64_t)((ms * ms) << (2 * sh - 52));
    // Q1 = Q0 + (N - Q0^2) / (2 Q0), with 1 / Q0 ~ y 2^-52
    const int64_t Q1 = (int64_t)(ms << sh) + (((R0 >> 4) * Y) >> 22);
    // R1 = N - Q1^2 in 128 bits (|R1| < 2^67), then Q2 = Q1 + R1 / (2 Q1), rounded
    const uint64_t Nhi = M2 >> 12, Nlo = M2 << 52;
    const uint64_t qlo = (uint64_t)Q1 * (uint64_t)Q1, qhi = __umul64hi((uint64_t)Q1, (uint64_t)Q1);
    const uint64_t rlo = Nlo - qlo;
    const uint64_t rhi = Nhi - qhi - (Nlo < qlo ? 1ULL : 0ULL);
    const int64_t R1s = (int64_t)((rhi << 32) | (rlo >> 32));      // R1 / 2^32, rounded down
    int64_t Q2 = Q1 + ((R1s * Y + (1LL << 45)) >> 46);
    // |Q2 - sqrt(N)| < 1: N - Q2^2 is below 2^55 in magnitude, exact from the low words;
    // the nearest R satisfies -R < N - R^2 <= R
    const int64_t r = (int64_t)(Nlo - (uint64_t)Q2 * (uint64_t)Q2);
    Q2 += (r > Q2 ? 1 : 0) - (r <= -Q2 ? 1 : 0);
    return __longlong_as_double((long long)(((uint64_t)(Er - 1) << 52) + (uint64_t)Q2));
}

// n / d, correctly rounded.  The quotient significand is q = round(Mn 2^K / Md),
// K = 52 or 53 so that q lies in [2^52, 2^53).
__device__ __forceinline__ double div_rn(double n, double d)
{
    const uint64_t bn = (uint64_t)__double_as_longlong(n), bd = (uint64_t)__double_as_longlong(d);
    const uint32_t En = (uint32_t)(bn >> 52) & 0x7FFu, Ed = (uint32_t)(bd >> 52) & 0x7FFu;
    const uint64_t Fn = bn & FP_FRAC, Fd = bd & FP_FRAC;
    const uint64_t Mn = Fn | FP_HIDDEN, Md = Fd | FP_HIDDEN;
    const int lt = Mn < Md ? 1 : 0;
    const int Er = (int)En - (int)Ed + 1023 - lt;
    if (En - 1u >= 2046u || Ed - 1u >= 2046u || (uint32_t)(Er - 1) >= 2046u) return div_hw(n, d);
    const int K = 52 + lt;
    // significands in [1, 2) as floats built from the bits; y ~ 1 / d_m (Y = y 2^25);
    // n_m y ~ n_m / d_m with significand mq: Q0 = mq 2^sh ~ q
    const float df = __uint_as_float((127u << 23) | (uint32_t)(Fd >> 29));
    const float nf = __uint_as_float((127u << 23) | (uint32_t)(Fn >> 29));
    const float y = rcp_approx_f32(df);
    const int64_t Y = f32_fixed25(y);
    const uint32_t qb = __float_as_uint(nf * y);
    const uint64_t mq = (qb & 0x7FFFFFu) | 0x800000u;
    const int sh = (int)(qb >> 23) - 150 + K;
    // (N - Q0 Md) / 2^sh = Mn 2^(K - sh) - mq Md, below 2^58 in magnitude: exact from the low words
    const int64_t R0 = (int64_t)((Mn << (K - sh)) - mq * Md);
    // Q1 = Q0 + (N - Q0 Md) / Md, with 1 / Md ~ y 2^-52
    const int64_t Q1 = (int64_t)(mq << sh) + (((R0 >> 24) * Y) >> (53 - sh));
    // R1 = N - Q1 Md in 128 bits (|R1| < 2^64), then Q2 = Q1 + R1 / Md, rounded
    const uint64_t Nlo = Mn << K, Nhi = Mn >> (64 - K);
    const uint64_t plo = (uint64_t)Q1 * Md, phi = __umul64hi((uint64_t)Q1, Md);
    const uint64_t rlo = Nlo - plo;
    const uint64_t rhi = Nhi - phi - (Nlo < plo ? 1ULL : 0ULL);
    const int64_t R1s = (int64_t)((rhi << 32) | (rlo >> 32));
    int64_t Q2 = Q1 + ((R1s * Y + (1LL << 44)) >> 45);
    // |Q2 - q| < 1: the nearest q satisfies |N - q Md| < Md / 2 (never equal)
    const int64_t r = (int64_t)(Nlo - (uint64_t)Q2 * Md);
    Q2 += (2 * r > (int64_t)Md ? 1 : 0) - (2 * r < -(int64_t)Md ? 1 : 0);
    return __longlong_as_double(
        (long long)(((bn ^ bd) & FP_SIGN) | (((uint64_t)(Er - 1) << 52) + (uint64_t)Q2)));
}

// 1 / d, correctly rounded (the quotient above with n = 1).
__device__ __forceinline__ double rcp_rn(double d) { return div_rn(1.0, d); }

}  // namespace mcgb
