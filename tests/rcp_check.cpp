// Host check of the integer-pipe reciprocal (rcp_rn.cuh): on seeded random
// doubles (all exponents, values near 1, significands next to 1 and 2,
// exponent extremes, zeros, subnormals, infinities, NaNs, negatives) the
// result must be the IEEE division 1.0 / x bit for bit, for the host seed
// (FP32 division of the leading 24 bits) and for seeds perturbed by up to
// +-3 * 2^-21 relative, and inside the handled range the exact correction
// must settle every time (no fallback to the division).
//
//   rcp_check [--n N] [--seed S]
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#include "rcp_rn.cuh"

using namespace vlbm;

static unsigned long long bits(double x) {
    unsigned long long b;
    std::memcpy(&b, &x, sizeof b);
    return b;
}
static double from_bits(unsigned long long b) {
    double x;
    std::memcpy(&x, &b, sizeof x);
    return x;
}

// FP32 reciprocal of M's leading 24 bits as a value in [1, 2), scaled by 2^53
static unsigned long long host_seed(unsigned long long M) {
    const unsigned fb = 0x3F800000u | (unsigned)((M >> 29) & 0x7FFFFFu);
    float f;
    std::memcpy(&f, &fb, sizeof f);
    const float r = 1.0f / f;
    unsigned rb;
    std::memcpy(&rb, &r, sizeof rb);
    return (unsigned long long)((rb & 0x7FFFFFu) | 0x800000u) << (30 + (int)(rb >> 23) - 127);
}

int main(int argc, char** argv) {
    long long n = 4000000;
    unsigned long long seed = 5;
    for (int i = 1; i < argc; i++) {
        if (!strcmp(argv[i], "--n") && i + 1 < argc) n = atoll(argv[++i]);
        else if (!strcmp(argv[i], "--seed") && i + 1 < argc) seed = strtoull(argv[++i], nullptr, 10);
    }
    std::mt19937_64 rng(seed);
    long long bad = 0, unsettled = 0, tested = 0;
    auto check = [&](double x) {
        const double ref = 1.0 / x;
        for (int k = -3; k <= 3; k++) {
            auto seedk = [k](unsigned long long M) {
                const unsigned long long q = host_seed(M);
                return (unsigned long long)((long long)q + k * (long long)(q >> 21));
            };
            const double got = rcp_rn_with(x, seedk);
            const bool same = (ref != ref && got != got) || bits(ref) == bits(got);
            if (!same) {
                if (bad < 5) printf("MISMATCH x=%a seed shift %d: %a vs %a\n", x, k, ref, got);
                bad++;
            }
            // inside the handled range the correction must settle
            const unsigned E = (unsigned)(bits(x) >> 52);
            const unsigned long long F = bits(x) & 0x000FFFFFFFFFFFFFull;
            if (E - 1u <= 2043u && F) {
                bool ok = true;
                rcp_significand(F | 0x0010000000000000ull, seedk(F | 0x0010000000000000ull), ok);
                if (!ok) unsettled++;
            }
        }
        tested++;
    };
    const unsigned long long MANT = 0x000FFFFFFFFFFFFFull;
    for (long long i = 0; i < n; i++) {
        const unsigned long long r = rng(), r2 = rng();
        const unsigned kind = (unsigned)(r2 % 100);
        unsigned long long e, mant = r & MANT, sign = 0;
        if (kind < 50) e = 1023 - 8 + (r2 >> 8) % 16;  // densities and energies
        else if (kind < 60) {                          // significands next to 1 and next to 2
            e = 1 + (r2 >> 8) % 2046;
            mant = (r2 >> 20) & 1 ? (r & 0xFFFFF) : MANT - (r & 0xFFFFF);
        } else if (kind < 70) e = ((r2 >> 8) & 1) ? 1 + (r2 >> 9) % 4 : 2040 + (r2 >> 9) % 8;  // extremes
        else if (kind < 75) {
            const unsigned long long sp[7] = {0ull, 1ull, MANT, 0x0010000000000000ull, 0x7FEFFFFFFFFFFFFFull,
                                              0x7FF0000000000000ull, 0x7FF8000000000000ull};
            const double v = from_bits(sp[(r2 >> 8) % 7]);
            check(v);
            check(-v);
            continue;
        } else if (kind < 80) {
            e = (r2 >> 8) % 2048;
            sign = 1;
        } else e = (r2 >> 8) % 2048;
        check(from_bits((sign << 63) | (e << 52) | mant));
    }
    // every power of two and its neighbours
    for (unsigned long long e = 0; e < 2048; e++)
        for (long long d = -2; d <= 2; d++) check(from_bits((e << 52) + (unsigned long long)d));
    printf("%s %lld values, %lld mismatches, %lld unsettled\n", bad || unsettled ? "FAIL" : "OK", tested, bad,
           unsettled);
    return bad || unsettled ? 1 : 0;
}
