// Exact accumulation of binary64 values in 192-bit two's-complement fixed
// point (resolution 2^-128, magnitude below 2^63), on the integer pipes.
//
// Integer addition is associative, so a sum does not depend on the order in
// which cells, tiles or thread groups contribute: the conservation totals
// come out identical for every launch configuration and equal to the exactly
// rounded sum of the addends (a value below 2^-75 loses the bits of its
// significand that fall under 2^-128).  The conversions are the plain
// definition of the formats: unpack sign, exponent and significand, shift
// the significand into place, negate; back to binary64 by locating the
// leading one and rounding to nearest even from the dropped bits.
#pragma once
#include <cstdint>

namespace vlbm {

struct Fix192 {
    unsigned long long w[3];  // little-endian words
};

__device__ __forceinline__ Fix192 fix_zero() { return Fix192{{0ull, 0ull, 0ull}}; }

__device__ __forceinline__ void fix_add(Fix192& a, const Fix192& b) {
    const unsigned long long s0 = a.w[0] + b.w[0];
    const unsigned long long c0 = s0 < a.w[0] ? 1ull : 0ull;
    const unsigned long long s1 = a.w[1] + b.w[1];
    unsigned long long c1 = s1 < a.w[1] ? 1ull : 0ull;
    const unsigned long long s1c = s1 + c0;
    c1 += s1c < s1 ? 1ull : 0ull;
    a.w[2] = a.w[2] + b.w[2] + c1;
    a.w[1] = s1c;
    a.w[0] = s0;
}

__device__ __forceinline__ void fix_neg(Fix192& a) {
    a.w[0] = ~a.w[0];
    a.w[1] = ~a.w[1];
    a.w[2] = ~a.w[2];
    const Fix192 one{{1ull, 0ull, 0ull}};
    fix_add(a, one);
}

__device__ __forceinline__ void fix_sub(Fix192& a, const Fix192& b) {
    const unsigned long long d0 = a.w[0] - b.w[0];
    const unsigned long long b0 = a.w[0] < b.w[0] ? 1ull : 0ull;
    const unsigned long long d1 = a.w[1] - b.w[1];
    unsigned long long b1 = a.w[1] < b.w[1] ? 1ull : 0ull;
    b1 += d1 < b0 ? 1ull : 0ull;
    a.w[2] = a.w[2] - b.w[2] - b1;
    a.w[1] = d1 - b0;
    a.w[0] = d0;
}

// |v| * 2^scale_exp as fixed point, from the bits B of v (truncated below
// 2^-128; NaN/inf give 0, the sweep reports them separately).  The words are
// chosen by selects, not by indexing, so everything stays in registers.
__device__ __forceinline__ Fix192 fix_from_mag(unsigned long long B, int scale_exp) {
    int E = (int)((B >> 52) & 0x7FFull);
    unsigned long long m = B & 0x000FFFFFFFFFFFFFull;
    Fix192 r = fix_zero();
    if (E == 2047) return r;
    if (E) m |= 0x0010000000000000ull;
    else E = 1;
    // |v| = m * 2^(E - 1075 + scale_exp); fixed = |v| * 2^128
    const int sh = E - 1075 + scale_exp + 128;
    if (sh >= 0) {
        if (sh >= 192) return r;  // out of range: the caller's magnitudes never get here
        const int wi = sh >> 6, b = sh & 63;
        const unsigned long long lo = m << b;
        const unsigned long long hi = b ? m >> (64 - b) : 0ull;
        r.w[0] = wi == 0 ? lo : 0ull;
        r.w[1] = wi == 1 ? lo : (wi == 0 ? hi : 0ull);
        r.w[2] = wi == 2 ? lo : (wi == 1 ? hi : 0ull);
    } else if (sh > -64) {
        r.w[0] = m >> (-sh);
    }
    return r;
}

// v * 2^scale_exp as fixed point.
__device__ __forceinline__ Fix192 fix_from_double(double v, int scale_exp) {
    const unsigned long long B = (unsigned long long)__double_as_longlong(v);
    Fix192 r = fix_from_mag(B, scale_exp);
    if (B >> 63) fix_neg(r);
    return r;
}

// sum += v * 2^scale_exp and abs_sum += |v| * 2^scale_exp, exactly.
__device__ __forceinline__ void fix_accumulate(Fix192& sum, Fix192& abs_sum, double v, int scale_exp) {
    const unsigned long long B = (unsigned long long)__double_as_longlong(v);
    const Fix192 a = fix_from_mag(B, scale_exp);
    fix_add(abs_sum, a);
    if (B >> 63) fix_sub(sum, a);
    else fix_add(sum, a);
}

__device__ __forceinline__ Fix192 fix_shfl_down(const Fix192& a, int off) {
    Fix192 r;
    for (int i = 0; i < 3; i++) r.w[i] = __shfl_down_sync(0xffffffffu, a.w[i], off);
    return r;
}

// Word i of a (0 beyond the top), by selects.
__device__ __forceinline__ unsigned long long fix_word(const Fix192& a, int i) {
    return i == 0 ? a.w[0] : i == 1 ? a.w[1] : i == 2 ? a.w[2] : 0ull;
}

// The 64 bits of a starting at bit position pos (0 <= pos < 192).
__device__ __forceinline__ unsigned long long fix_bits64(const Fix192& a, int pos) {
    const int wi = pos >> 6, b = pos & 63;
    const unsigned long long lo = fix_word(a, wi) >> b;
    return b ? lo | (fix_word(a, wi + 1) << (64 - b)) : lo;
}

// Correctly rounded (nearest, ties to even) binary64 value of a * 2^-128.
__device__ __forceinline__ double fix_to_double(Fix192 a) {
    const bool neg = (a.w[2] >> 63) != 0;
    if (neg) fix_neg(a);
    int p = -1;  // index of the leading one
    if (a.w[2]) p = 128 + 63 - __clzll((long long)a.w[2]);
    else if (a.w[1]) p = 64 + 63 - __clzll((long long)a.w[1]);
    else if (a.w[0]) p = 63 - __clzll((long long)a.w[0]);
    if (p < 0) return 0.0;
    unsigned long long m;
    if (p <= 52) {
        m = a.w[0];  // exact
    } else {
        const int s = p - 52;  // keep bits [s, s + 53)
        m = fix_bits64(a, s) & 0x001FFFFFFFFFFFFFull;
        const int t = s - 1;  // rounding bit; sticky = any bit below it
        const bool rnd = (fix_bits64(a, t) & 1ull) != 0;
        const int tw = t >> 6, tb = t & 63;
        bool sticky = (fix_word(a, tw) & ((1ull << tb) - 1ull)) != 0;
        if (tw >= 1) sticky = sticky || a.w[0] != 0;
        if (tw >= 2) sticky = sticky || a.w[1] != 0;
        if (rnd && (sticky || (m & 1ull))) {
            m += 1;
            if (m >> 53) {
                m >>= 1;
                p += 1;
            }
        }
    }
    // m < 2^53 is exact in binary64; scaling by powers of two is exact
    double r = (double)m;
    if (p > 52) r = ldexp(r, p - 52);
    r = ldexp(r, -128);
    return neg ? -r : r;
}

}  // namespace vlbm
