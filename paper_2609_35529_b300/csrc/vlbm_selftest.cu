// Self-tests of the correctly rounded reciprocal on the integer pipes (used
// by the collision for 1/rho) and of the division built on it (the
// relaxation sensor's quotients), against the FP64 division.
#include <cuda_runtime.h>
#include <cstdint>

#include "rcp_rn.cuh"
#include "vlbm.h"

namespace vlbm {

constexpr unsigned long long EMU_MANT = 0x000FFFFFFFFFFFFFull;  // binary64 significand field
constexpr unsigned long long EMU_HID = 0x0010000000000000ull;   // its hidden bit

// SplitMix64 (Steele, Lea & Flood 2014): counter-based 64-bit generator.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ bool same(double x, double y) {
    if (x != x && y != y) return true;  // both NaN
    return __double_as_longlong(x) == __double_as_longlong(y);
}

}  // namespace vlbm

namespace vlbm {

// A reciprocal test value: mostly densities near 1, plus significands next
// to 1 and 2, exponent extremes, specials, negatives and raw bit patterns.
__device__ double rcp_operand(unsigned long long r, unsigned long long r2) {
    const unsigned kind = (unsigned)(r2 % 100);
    unsigned long long mant = r & EMU_MANT, e, sign = 0;
    if (kind < 60) e = 1023 - 8 + (r2 >> 8) % 16;
    else if (kind < 70) {
        e = 1 + (r2 >> 8) % 2046;
        mant = (r2 >> 20) & 1 ? (r & 0xFFFFF) : EMU_MANT - (r & 0xFFFFF);
    } else if (kind < 78) e = ((r2 >> 8) & 1) ? 1 + (r2 >> 9) % 4 : 2040 + (r2 >> 9) % 8;
    else if (kind < 82) {
        const unsigned long long sp[7] = {0ull, 1ull, EMU_MANT, 0x0010000000000000ull, 0x7FEFFFFFFFFFFFFFull,
                                          0x7FF0000000000000ull, 0x7FF8000000000000ull};
        return __longlong_as_double((long long)(sp[(r2 >> 8) % 7] | (((r2 >> 40) & 1ull) << 63)));
    } else if (kind < 86) {
        e = (r2 >> 8) % 2048;
        sign = 1;
    } else if (kind < 93) e = (r2 >> 8) % 2048;
    else return __longlong_as_double((long long)r);
    return __longlong_as_double((long long)((sign << 63) | (e << 52) | mant));
}

// bad[0]: results that differ from 1.0 / x; bad[1]: handled inputs whose
// exact correction did not settle (they take the division).
__global__ void selftest_rcp_kernel(unsigned long long seed, long long n, unsigned long long* bad, double* first) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = rcp_operand(splitmix64(seed ^ (2 * i)), splitmix64(seed ^ (2 * i + 1)));
        const double ref = 1.0 / x, got = rcp_rn(x);
        if (!same(ref, got) && atomicAdd(&bad[0], 1ull) == 0) {
            first[0] = x;
            first[1] = got;
        }
        const unsigned long long B = (unsigned long long)__double_as_longlong(x);
        const unsigned E = (unsigned)(B >> 52);
        const unsigned long long F = B & EMU_MANT;
        if (E - 1u <= 2043u && F) {
            bool ok = true;
            const unsigned long long M = F | EMU_HID;
            rcp_significand(M, rcp_seed_dev(M), ok);
            if (!ok) atomicAdd(&bad[1], 1ull);
        }
    }
}

// A division test pair: quotients of the relaxation sensor's kinds (a
// compression gate d / (d + e), beta / c), operands over the whole normal
// range with random signs, exponents next to the guard's bounds, specials,
// and raw bit patterns.
__device__ void div_operands(unsigned long long r, unsigned long long r2, unsigned long long r3, double& a,
                             double& b) {
    const unsigned kind = (unsigned)(r3 % 100);
    auto mk = [](unsigned long long sign, unsigned long long e, unsigned long long mant) {
        return __longlong_as_double((long long)((sign << 63) | (e << 52) | (mant & EMU_MANT)));
    };
    if (kind < 35) {
        a = mk(0, 1023 - 60 + (r3 >> 8) % 70, r);
        b = a + mk(0, 1023 - 70 + (r3 >> 16) % 80, r2);
    } else if (kind < 55) {
        a = mk(0, 1021 + (r3 >> 8) % 2, r);
        b = mk(0, 1022 + (r3 >> 16) % 3, r2);
    } else if (kind < 80) {
        a = mk((r3 >> 8) & 1, 1 + (r3 >> 9) % 2046, r);
        b = mk((r3 >> 20) & 1, 1 + (r3 >> 21) % 2046, r2);
    } else if (kind < 90) {
        const unsigned long long edge[4] = {521, 524, 1522, 1525};
        a = mk((r3 >> 8) & 1, edge[(r3 >> 9) % 4] - (r3 >> 11) % 3, r);
        b = mk((r3 >> 13) & 1, edge[(r3 >> 14) % 4] - (r3 >> 16) % 3, r2);
    } else if (kind < 95) {
        const unsigned long long sp[6] = {0ull, 1ull, EMU_MANT, 0x7FF0000000000000ull, 0x7FF8000000000000ull,
                                          0x3FF0000000000000ull};
        a = (r3 >> 8) & 1 ? __longlong_as_double((long long)sp[(r3 >> 9) % 6]) : mk(0, 1023, r);
        b = (r3 >> 12) & 1 ? __longlong_as_double((long long)sp[(r3 >> 13) % 6]) : mk(0, 1023, r2);
    } else {
        a = __longlong_as_double((long long)r);
        b = __longlong_as_double((long long)r2);
    }
}

// bad: quotients that differ from a / b (div_rn, or div_rn_y with the
// reciprocal 1.0 / b).
__global__ void selftest_div_kernel(unsigned long long seed, long long n, unsigned long long* bad, double* first) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double a, b;
        div_operands(splitmix64(seed ^ (3 * i)), splitmix64(seed ^ (3 * i + 1)), splitmix64(seed ^ (3 * i + 2)), a, b);
        const double ref = a / b;
        const double g1 = div_rn(a, b), g2 = div_rn_y(a, b, 1.0 / b);
        if ((!same(ref, g1) || !same(ref, g2)) && atomicAdd(bad, 1ull) == 0) {
            first[0] = a;
            first[1] = b;
            first[2] = same(ref, g1) ? g2 : g1;
        }
    }
}

}  // namespace vlbm

extern "C" vlbm_status vlbm_selftest_div(uint64_t seed, int64_t n, uint64_t* mismatches, double first_bad[3]) {
    if (n < 0 || !mismatches) return VLBM_ERR_ARG;
    unsigned long long* dbad = nullptr;
    double* dfirst = nullptr;
    if (cudaMalloc(&dbad, sizeof(unsigned long long)) != cudaSuccess) return VLBM_ERR_OOM;
    if (cudaMalloc(&dfirst, 3 * sizeof(double)) != cudaSuccess) {
        cudaFree(dbad);
        return VLBM_ERR_OOM;
    }
    cudaMemset(dbad, 0, sizeof(unsigned long long));
    cudaMemset(dfirst, 0, 3 * sizeof(double));
    vlbm::selftest_div_kernel<<<148 * 8, 256>>>(seed, n, dbad, dfirst);
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long hb = 0;
    double hf[3] = {0.0, 0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpy(&hb, dbad, sizeof hb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hf, dfirst, sizeof hf, cudaMemcpyDeviceToHost);
    cudaFree(dbad);
    cudaFree(dfirst);
    if (e != cudaSuccess) return VLBM_ERR_CUDA;
    *mismatches = hb;
    if (first_bad)
        for (int i = 0; i < 3; i++) first_bad[i] = hf[i];
    return VLBM_OK;
}

extern "C" vlbm_status vlbm_selftest_rcp(uint64_t seed, int64_t n, uint64_t* mismatches, uint64_t* unsettled,
                                         double first_bad[2]) {
    if (n < 0 || !mismatches || !unsettled) return VLBM_ERR_ARG;
    unsigned long long* dbad = nullptr;
    double* dfirst = nullptr;
    if (cudaMalloc(&dbad, 2 * sizeof(unsigned long long)) != cudaSuccess) return VLBM_ERR_OOM;
    if (cudaMalloc(&dfirst, 2 * sizeof(double)) != cudaSuccess) {
        cudaFree(dbad);
        return VLBM_ERR_OOM;
    }
    cudaMemset(dbad, 0, 2 * sizeof(unsigned long long));
    cudaMemset(dfirst, 0, 2 * sizeof(double));
    vlbm::selftest_rcp_kernel<<<148 * 8, 256>>>(seed, n, dbad, dfirst);
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long hb[2] = {0, 0};
    double hf[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpy(hb, dbad, sizeof hb, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hf, dfirst, sizeof hf, cudaMemcpyDeviceToHost);
    cudaFree(dbad);
    cudaFree(dfirst);
    if (e != cudaSuccess) return VLBM_ERR_CUDA;
    *mismatches = hb[0];
    *unsettled = hb[1];
    if (first_bad) first_bad[0] = hf[0], first_bad[1] = hf[1];
    return VLBM_OK;
}
