// Bit-exact IEEE-754 binary64 addition and multiplication (round to nearest,
// ties to even) computed on the integer pipes.
//
// Why: on B300 the FP64 pipe retires about 1.6 lane-operations per clock per
// SM, while the integer/FP32 pipes retire up to 128.  A sweep of the VLBM
// collision is bound by the FP64 pipe; moving part of its additions and
// multiplications to these integer routines lets both pipes work at once.
// The results are the same bits the FP64 unit produces, so the canonical
// arithmetic (and bitwise parity with the oracle) is unchanged.
//
// Method (the textbook one for binary floating point): unpack sign, biased
// exponent and the 53-bit significand with its hidden bit; align the smaller
// operand keeping a sticky bit; add or subtract; renormalise; round to
// nearest even from the dropped bits; repack.  Products use the full 106-bit
// significand product (64x64 -> 128 bit).  Operands or results outside the
// normal range (zeros of the multiplication excepted, zeros of the addition
// included) fall back to the hardware instruction, so every input gives the
// hardware answer.
#pragma once
#include <cstdint>

namespace vlbm {

constexpr unsigned long long EMU_SIGN = 0x8000000000000000ull;
constexpr unsigned long long EMU_ABS = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long EMU_MANT = 0x000FFFFFFFFFFFFFull;
constexpr unsigned long long EMU_HID = 0x0010000000000000ull;

__device__ __forceinline__ double emu_add(double a, double b) {
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const unsigned long long Am = A & EMU_ABS, Bm = B & EMU_ABS;
    const bool sw = Bm > Am;
    const unsigned long long X = sw ? B : A, Y = sw ? A : B;  // |x| >= |y|
    const unsigned long long Xm = sw ? Bm : Am, Ym = sw ? Am : Bm;
    const unsigned ex = (unsigned)(Xm >> 52), ey = (unsigned)(Ym >> 52);
    if (Ym == 0)  // y = +-0: x + y = x, and -0 only when both are -0
        return __longlong_as_double((long long)(Xm == 0 ? (X & Y) : X));
    if (ey == 0 || ex >= 2047u) return a + b;
    const unsigned long long mx = ((Xm & EMU_MANT) | EMU_HID) << 10;  // hidden bit at 62
    const unsigned long long my = ((Ym & EMU_MANT) | EMU_HID) << 10;
    const unsigned d = ex - ey;
    unsigned long long mys;
    if (d == 0) mys = my;
    else if (d < 64) mys = (my >> d) | (unsigned long long)((my << (64 - d)) != 0);
    else mys = 1;
    int e = (int)ex;
    unsigned long long m;
    if (((X ^ Y) & EMU_SIGN) == 0) {
        m = mx + mys;
        if (m >> 63) {
            m = (m >> 1) | (m & 1);
            e += 1;
        }
    } else {
        m = mx - mys;
        if (m == 0) return 0.0;
        const int lz = __clzll((long long)m) - 1;
        m <<= lz;
        e -= lz;
    }
    const unsigned rem = (unsigned)m & 0x3FFu;
    m >>= 10;
    if (rem > 0x200u || (rem == 0x200u && (m & 1))) m += 1;
    if (m >> 53) {
        m >>= 1;
        e += 1;
    }
    if (e <= 0 || e >= 2047) return a + b;
    return __longlong_as_double((long long)((X & EMU_SIGN) | ((unsigned long long)e << 52) | (m & EMU_MANT)));
}

__device__ __forceinline__ double emu_sub(double a, double b) {
    return emu_add(a, __longlong_as_double(__double_as_longlong(b) ^ (long long)EMU_SIGN));
}

__device__ __forceinline__ double emu_mul(double a, double b) {
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const unsigned long long S = (A ^ B) & EMU_SIGN;
    const unsigned ea = (unsigned)(A >> 52) & 0x7FFu, eb = (unsigned)(B >> 52) & 0x7FFu;
    if (ea == 2047u || eb == 2047u) return a * b;
    if ((A & EMU_ABS) == 0 || (B & EMU_ABS) == 0) return __longlong_as_double((long long)S);
    if (ea == 0 || eb == 0) return a * b;
    const unsigned long long ma = ((A & EMU_MANT) | EMU_HID) << 11;  // bit 63 set
    const unsigned long long mb = ((B & EMU_MANT) | EMU_HID) << 11;
    unsigned long long hi = __umul64hi(ma, mb);
    unsigned long long lo = ma * mb;
    int e = (int)ea + (int)eb - 1023;
    if (hi >> 63) {
        e += 1;
    } else {
        hi = (hi << 1) | (lo >> 63);
        lo <<= 1;
    }
    const unsigned rem = (unsigned)hi & 0x7FFu;
    unsigned long long m = hi >> 11;
    if (rem > 0x400u || (rem == 0x400u && (lo != 0 || (m & 1)))) m += 1;
    if (m >> 53) {
        m >>= 1;
        e += 1;
    }
    if (e <= 0 || e >= 2047) return a * b;
    return __longlong_as_double((long long)(S | ((unsigned long long)e << 52) | (m & EMU_MANT)));
}

// x * 2^-1 for a value whose halving is exact (normal, exponent > 1);
// anything else takes the hardware multiplication.
__device__ __forceinline__ double emu_half(double a) {
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned e = (unsigned)(A >> 52) & 0x7FFu;
    if (e > 1u && e < 2047u) return __longlong_as_double((long long)(A - (1ull << 52)));
    return a * 0.5;
}

}  // namespace vlbm
