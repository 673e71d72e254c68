// Correctly rounded reciprocal of a binary64 value (round to nearest) on the
// integer pipes.
//
// Why: the collision needs 1/rho once per cell update; the FP64 division
// occupies the FP64 pipe -- the sweep's bottleneck on B300 -- for several
// operation slots, while the integer pipes are mostly idle.  The result is
// the same bits as the IEEE division 1.0 / x, so the canonical arithmetic
// (and bitwise parity with the oracle) is unchanged.
//
// Method: Newton-Raphson iteration for the reciprocal (Brent & Zimmermann,
// Modern Computer Arithmetic, Sec. 3.4.1) carried out in integer fixed
// point, followed by an exact remainder test for the final rounding.  For
// x = M 2^(E - 1075) with the 53-bit significand M in (2^52, 2^53), 1/x =
// (2^105 / M) 2^(1022 - E - 53); the significand of the result is
// Q = round(2^105 / M), which lies in [2^52, 2^53).
//  1. A seed Q0 ~ 2^105 / M with relative error below 2^-20 (on the device
//     from the FP32 reciprocal approximation of M's leading 24 bits).
//  2. Two Newton steps Q <- Q + Q T / 2^105 with T = 2^105 - Q M computed
//     exactly in 128-bit integers: the relative error goes from e to about
//     e^2, so after two steps Q is within a few units of 2^105 / M.
//  3. Exact correction: with T = 2^105 - Q M, step Q until 0 <= T < M
//     (then Q = floor(2^105 / M) and T is the remainder), and round up when
//     2 T > M.  A tie 2 T = M would need M to divide 2^106, i.e. M a power
//     of two, which is the exact case handled apart.
// Every value outside the handled range (zero, negative, subnormal,
// infinite or NaN x, or a reciprocal that would be subnormal) and any
// correction that does not settle within its bound take the division
// itself, so every input gives the IEEE answer.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define RCP_HD __host__ __device__ __forceinline__
#else
#define RCP_HD inline
#endif

namespace vlbm {

typedef __int128 rcp_i128;

// Steps 2-3 for a significand M in (2^52, 2^53) and a seed Q of relative
// error below 2^-20; ok = false when the correction did not settle.
RCP_HD unsigned long long rcp_significand(unsigned long long M, unsigned long long Q, bool& ok) {
    const rcp_i128 ONE = (rcp_i128)1 << 105;
    const rcp_i128 m = (rcp_i128)M;
    // |T| < 2^86: scaled by 2^-32 so that Q (T / 2^32) fits in 127 bits
    rcp_i128 T = ONE - (rcp_i128)Q * m;
    Q = (unsigned long long)((rcp_i128)Q + (((rcp_i128)Q * (T >> 32)) >> 73));
    // |T| < 2^67 now
    T = ONE - (rcp_i128)Q * m;
    Q = (unsigned long long)((rcp_i128)Q + (((rcp_i128)Q * T) >> 105));
    T = ONE - (rcp_i128)Q * m;
    for (int i = 0; i < 4 && T < 0; i++) {
        Q--;
        T += m;
    }
    for (int i = 0; i < 4 && T >= m; i++) {
        Q++;
        T -= m;
    }
    ok = T >= 0 && T < m;
    return Q + (2 * T > m ? 1ull : 0ull);
}

// 1/x, with `seed` mapping the significand M to the seed Q0.
template <class Seed>
RCP_HD double rcp_rn_with(double x, Seed seed) {
    unsigned long long B;
#ifdef __CUDA_ARCH__
    B = (unsigned long long)__double_as_longlong(x);
#else
    std::memcpy(&B, &x, sizeof B);
#endif
    const unsigned E = (unsigned)(B >> 52);  // includes the sign bit: negative x gives E >= 2048
    if (E - 1u > 2043u) return 1.0 / x;      // E in [1, 2044]: the reciprocal is normal
    const unsigned long long F = B & 0x000FFFFFFFFFFFFFull;
    unsigned long long R;
    if (F == 0) {
        R = (unsigned long long)(2046u - E) << 52;  // x a power of two
    } else {
        const unsigned long long M = F | 0x0010000000000000ull;
        bool ok = true;
        const unsigned long long Q = rcp_significand(M, seed(M), ok);
        if (!ok) return 1.0 / x;
        R = ((unsigned long long)(2045u - E) << 52) | (Q - 0x0010000000000000ull);
    }
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)R);
#else
    double r;
    std::memcpy(&r, &R, sizeof r);
    return r;
#endif
}

#ifdef __CUDACC__
// The device seed: the FP32 reciprocal approximation of f = M's leading 24
// bits as a value in [1, 2) (relative error of f below 2^-23, of the
// approximation about 2^-23), scaled to 2^53 / f ~ 2^105 / M.
__device__ __forceinline__ unsigned long long rcp_seed_dev(unsigned long long M) {
    const float f = __uint_as_float(0x3F800000u | (unsigned)((M >> 29) & 0x7FFFFFu));
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));
    const unsigned rb = __float_as_uint(r);  // r in [0.5, 1]
    return (unsigned long long)((rb & 0x7FFFFFu) | 0x800000u) << (30 + (int)(rb >> 23) - 127);
}

__device__ __forceinline__ double rcp_rn(double x) { return rcp_rn_with(x, rcp_seed_dev); }

// a / b correctly rounded (the IEEE quotient), given y = RN(1/b): one FP64
// multiply and four fma in place of the division's longer sequence.
// q0 = RN(a y) lies within two ulps of a / b; a correction q <- RN(q + r y)
// with the remainder r = a - b q (one fma) then leaves q within one ulp, so
// the next remainder is exact, and with y within half an ulp of 1/b the
// second correction gives RN(a / b) (Markstein's theorem; Muller et al.,
// Handbook of Floating-Point Arithmetic, on division by Newton-Raphson
// iteration).  Operands of magnitude outside [2^-500, 2^501) -- zero,
// subnormal, huge, infinite, NaN -- where a remainder or the quotient could
// leave the normal range take the division itself.
__device__ __forceinline__ double div_rn_y(double a, double b, double y) {
    const unsigned ea = (unsigned)((unsigned long long)__double_as_longlong(a) >> 52) & 0x7FFu;
    const unsigned eb = (unsigned)((unsigned long long)__double_as_longlong(b) >> 52) & 0x7FFu;
    if (ea - 523u > 1000u || eb - 523u > 1000u) return a / b;
    double q = a * y;
    double r = fma(-q, b, a);
    q = fma(r, y, q);
    r = fma(-q, b, a);
    return fma(r, y, q);
}

// a / b with the reciprocal of b on the integer pipes.
__device__ __forceinline__ double div_rn(double a, double b) { return div_rn_y(a, b, rcp_rn(b)); }
#endif

}  // namespace vlbm
