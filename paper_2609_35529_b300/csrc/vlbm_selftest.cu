// Self-test of the correctly rounded reciprocal on the integer pipes (used
// by the collision for 1/rho) against the FP64 division.
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

}  // namespace vlbm

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
