// Conservation totals of a population array without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want a
// conservation check: an application that reserves all of its GPU memory up
// front and forbids later allocations (a real-time loop, an embedding host
// that owns the memory pool), or a caller that holds only raw device
// pointers to populations it manages itself.  vlbm_audit needs a hierarchy
// handle, whose creation allocates; this entry point takes the caller's
// population array and output buffer and keeps its only scratch (the
// per-CTA partial sums of the two-pass reduction) in a fixed file-scope
// device array.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "vlbm.h"

namespace {

constexpr int kStaticThreads = 256;
constexpr int kCellsPerBlock = 4096;
constexpr int kMaxBlocks = VLBM_STATIC_MAX_BLOCKS;

// Partial sums of the reduction: kMaxBlocks slots of 8 (sum, compensation)
// pairs.  Every device that loads the library holds this array until the
// process exits.  In host code the symbol is only a handle: its device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_partials[kMaxBlocks * 16];

struct CSum {
    double s, c;
};

__device__ __forceinline__ void cadd(CSum& a, double x) {
    const double t = a.s + x;
    if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}

__device__ __forceinline__ CSum cjoin(CSum a, CSum b) {
    CSum r;
    r.s = a.s;
    r.c = a.c + b.c;
    cadd(r, b.s);
    return r;
}

// Pass 1: block b sums cells [b * kCellsPerBlock, (b + 1) * kCellsPerBlock)
// of the nx x ny grid into partials[b].  W_k = (f_+x + f_-x) + (f_+y + f_-y).
__global__ void __launch_bounds__(kStaticThreads) static_partials(const double* __restrict__ f, long long ld, int nx,
                                                                  int ny, double weight, double* partials) {
    CSum acc[8];
    for (int m = 0; m < 8; m++) acc[m] = {0.0, 0.0};
    const long long ncell = (long long)nx * ny;
    const long long plane = ld * ny;
    const long long c0 = (long long)blockIdx.x * kCellsPerBlock;
    for (long long i = c0 + threadIdx.x; i < c0 + kCellsPerBlock && i < ncell; i += kStaticThreads) {
        const long long x = i % nx, y = i / nx;
        const long long o = y * ld + x;
        for (int k = 0; k < 4; k++) {
            const double w = ((f[(0 + k) * plane + o] + f[(4 + k) * plane + o]) +
                              (f[(8 + k) * plane + o] + f[(12 + k) * plane + o])) * weight;
            cadd(acc[k], w);
            cadd(acc[4 + k], fabs(w));
        }
    }
    __shared__ CSum sh[kStaticThreads / 32][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int m = 0; m < 8; m++) {
        CSum a = acc[m];
        for (int off = 16; off > 0; off >>= 1) {
            CSum b;
            b.s = __shfl_down_sync(0xffffffffu, a.s, off);
            b.c = __shfl_down_sync(0xffffffffu, a.c, off);
            if (lane < off) a = cjoin(a, b);
        }
        if (lane == 0) sh[wid][m] = a;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int m = threadIdx.x;
        CSum a = sh[0][m];
        for (int w2 = 1; w2 < kStaticThreads / 32; w2++) a = cjoin(a, sh[w2][m]);
        partials[blockIdx.x * 16 + 2 * m] = a.s;
        partials[blockIdx.x * 16 + 2 * m + 1] = a.c;
    }
}

// Pass 2: the partial sums of this call's blocks, in block order.
__global__ void static_final(const double* __restrict__ partials, int nblk, double* __restrict__ out) {
    const int m = threadIdx.x;
    if (m >= 8) return;
    CSum a = {0.0, 0.0};
    for (int b = 0; b < nblk; b++) a = cjoin(a, CSum{partials[b * 16 + 2 * m], partials[b * 16 + 2 * m + 1]});
    out[m] = a.s + a.c;
}

// Device address of g_partials per device: looked up again (with that device
// current) on every call made outside a stream capture, so that a context
// created anew (after cudaDeviceReset) is followed; the last address is
// kept for calls made while `stream` is being captured, which must not load
// modules.
std::mutex g_mu;
double* g_addr[64] = {};

}  // namespace

extern "C" vlbm_status vlbm_totals_static(const double* f, int64_t ld, int32_t nx, int32_t ny, double weight,
                                          double* out, void* stream) {
    if (!f || !out || nx < 1 || ny < 1 || ld < nx) return VLBM_ERR_ARG;
    const long long ncell = (long long)nx * ny;
    const long long nblk = (ncell + kCellsPerBlock - 1) / kCellsPerBlock;
    if (nblk > kMaxBlocks) return VLBM_ERR_ARG;  // more cells than the fixed scratch covers
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VLBM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return VLBM_ERR_CUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return VLBM_ERR_CUDA;
            g_addr[dev] = (double*)p;
        }
        scratch = g_addr[dev];
    }
    if (!scratch) return VLBM_ERR_CUDA;  // first call on this device made during a capture
    static_partials<<<(unsigned)nblk, kStaticThreads, 0, s>>>(f, ld, nx, ny, weight, scratch);
    static_final<<<1, 32, 0, s>>>(scratch, (int)nblk, out);
    return cudaGetLastError() == cudaSuccess ? VLBM_OK : VLBM_ERR_CUDA;
}
