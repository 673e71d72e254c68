// CUDA kernels of the refined VLBM (sm_103a, FP64).
//
// Canonical arithmetic: every floating-point expression below is evaluated
// as written, with fma() only where spelled out (the library is built with
// --fmad=false).  The expression order is fixed so that results do not
// depend on the launch configuration.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <cstdint>

#include "fix192.cuh"
#include "rcp_rn.cuh"
#include "vlbm_dev.cuh"
#include "vlbm_launch.h"

namespace vlbm {

__device__ __constant__ int kCX[4] = {1, -1, 0, 0};
__device__ __constant__ int kCY[4] = {0, 0, 1, -1};

// ---------------------------------------------------------------------------
// single-cell operators (Sec. 2.1-2.2)
// ---------------------------------------------------------------------------

// Euler flux Q(W) with the ideal-gas closure (Sec. 2.1, Eq. 1).
__device__ __forceinline__ void euler_flux(double gm1, const double W[4], double Qx[4], double Qy[4],
                                           double& p_out) {
    const double inv = rcp_rn(W[0]);  // = 1.0 / W[0], on the integer pipes
    const double u = W[1] * inv;
    const double v = W[2] * inv;
    const double ruu = W[1] * u;
    const double rvv = W[2] * v;
    const double p = gm1 * fma(-0.5, ruu + rvv, W[3]);
    const double H = W[3] + p;
    Qx[0] = W[1];
    Qx[1] = ruu + p;
    Qx[2] = W[2] * u;
    Qx[3] = H * u;
    Qy[0] = W[2];
    Qy[1] = W[1] * v;
    Qy[2] = rvv + p;
    Qy[3] = H * v;
    p_out = p;
}

__device__ __forceinline__ bool physical(double rho, double p) {
    const long long rb = __double_as_longlong(rho);
    const long long pb = __double_as_longlong(p);
    const long long inf = 0x7FF0000000000000LL;
    return rb > 0 && rb < inf && pb > 0 && pb < inf;
}

// Launch-shape bit of a variant (no effect on the arithmetic): the
// persistent task kernel runs half tiles per warp (task_kernel_half).
enum : int { TK_HALF = 512 };
// The sweep reads the relaxation parameter of each cell from the sensor
// planes (sensor-driven relaxation).
enum : int { SW_SENSOR = 1024 };

// BGK relaxation (Eq. 6) in place: f <- 2 beta f^eq(W) + (1 - 2 beta) f with
// 2 beta f^eq_{+-alpha} = (beta/2) W +- (beta/c) Q_alpha (Eq. 4, D = 2):
// f* = fma(+-beta/c, Q_alpha, fma(1 - 2 beta, f, (beta/2) W)), for given
// moments W and fluxes Q.
__device__ __forceinline__ void relax(double f[16], const double W[4], const double Qx[4], const double Qy[4],
                                      double om, double hb, double bcs) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const double A = hb * W[k];
        f[k] = fma(bcs, Qx[k], fma(om, f[k], A));
        f[4 + k] = fma(-bcs, Qx[k], fma(om, f[4 + k], A));
        f[8 + k] = fma(bcs, Qy[k], fma(om, f[8 + k], A));
        f[12 + k] = fma(-bcs, Qy[k], fma(om, f[12 + k], A));
    }
}

// The collision of a cell: moments and Euler flux of its populations, then
// the relaxation.  The one division 1/rho is the correctly rounded
// reciprocal on the integer pipes (the same bits as 1.0 / rho).  Returns
// whether the state is physical.
__device__ __forceinline__ bool collide(double f[16], double om, double hb, double bcs, double gm1,
                                        double* Wout = nullptr) {
    double W[4], Qx[4], Qy[4];
#pragma unroll
    for (int k = 0; k < 4; k++) W[k] = (f[k] + f[4 + k]) + (f[8 + k] + f[12 + k]);
    if (Wout)
        for (int k = 0; k < 4; k++) Wout[k] = W[k];
    const double inv = rcp_rn(W[0]);  // = 1.0 / W[0], on the integer pipes
    const double u = W[1] * inv;
    const double v = W[2] * inv;
    const double ruu = W[1] * u;
    const double rvv = W[2] * v;
    const double p = gm1 * fma(-0.5, ruu + rvv, W[3]);
    const double H = W[3] + p;
    Qx[0] = W[1];
    Qx[1] = ruu + p;
    Qx[2] = W[2] * u;
    Qx[3] = H * u;
    Qy[0] = W[2];
    Qy[1] = W[1] * v;
    Qy[2] = rvv + p;
    Qy[3] = H * v;
    relax(f, W, Qx, Qy, om, hb, bcs);
    return physical(W[0], p);
}

__device__ __forceinline__ double minmod(double a, double b) {
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

// Loads of data that may have been written earlier in the same launch (the
// persistent task kernel) go to L2 (ld.global.cg), never to a possibly stale
// L1 line; the per-phase kernels read data from earlier launches.
template <bool COH, class T>
__device__ __forceinline__ T ld(const T* p) {
    if constexpr (COH) return __ldcg(p);
    else return __ldg(p);
}

// Source and destination buffers of a level's step.  Level 0 ping-pongs on
// the hierarchy's parity word (advanced by `step` inside a multi-step
// launch); level l >= 1 takes two steps per parent step: sub-step 1 reads
// buffer 0 and writes buffer 1, sub-step 2 the reverse.
__device__ __forceinline__ void level_bufs(const LevelDev& L, int kk, int step, const double*& src, double*& dst) {
    if (L.level == 0) {
        const int par = (*L.par0 + step) & 1;
        src = L.buf[par];
        dst = L.buf[par ^ 1];
    } else {
        src = L.buf[kk == 1 ? 0 : 1];
        dst = L.buf[kk == 1 ? 1 : 0];
    }
}

// state / scratch buffer of a level at a sync point
__device__ __forceinline__ int state_buf(const LevelDev& L) { return L.level == 0 ? *L.par0 : 0; }

// ---------------------------------------------------------------------------
// sensor-driven relaxation (Sec. 2.2, Eq. sensor-B)
// ---------------------------------------------------------------------------
// Per level step, on the level's active cells, from the pre-collision state:
//   s_k   = g_k / (2 qmax_k), g_k = (Qx_k(E) - Qx_k(W)) + (Qy_k(N) - Qy_k(S))
//           (dx (div Q)_k / max |Q_k| with central differences)
//   s     = (0.25 ((s_0^2 + s_3^2) + (s_1^2 + s_2^2)))^(1/2)
//   theta = dil^2 / (dil^2 + vort^2 + eps) where dil < 0, else 0, with the
//           undivided dil = (u(E) - u(W)) + (v(N) - v(S)) and
//           vort = (v(E) - v(W)) - (u(N) - u(S))
//   beta  = beta_max - (beta_max - beta_min) clip(C s_bar theta_bar, 0, 1)
//           with 3 x 3 box filters s_bar, theta_bar (sums grouped so that
//           swapping x and y gives the same rounding)
// A neighbour that is not an active cell of the level (covered, off the
// level, beyond a non-periodic side) takes the centre cell's value.

// Cell index of neighbour (x + dx, y + dy) when it is an active cell of the
// level, else the centre's.
__device__ __forceinline__ long long sens_nb(const LevelDev& L, int x, int y, int dx, int dy, long long c) {
    int xx = x + dx, yy = y + dy;
    if (xx < 0) { if (!L.px) return c; xx += L.nx; }
    if (xx >= L.nx) { if (!L.px) return c; xx -= L.nx; }
    if (yy < 0) { if (!L.py) return c; yy += L.ny; }
    if (yy >= L.ny) { if (!L.py) return c; yy -= L.ny; }
    const long long cn = (long long)yy * L.pitch + xx;
    return (L.flags[cn] & (F_IN | F_COV)) == F_IN ? cn : c;
}

// Pass 1 on cell (x, y): W, Q, u, v from the level step's source buffer
// (the sweep relaxes with these W and Q), and the state's check.  COH:
// loads through L2 (data written earlier in the same launch).
template <bool COH>
__device__ __forceinline__ void sensor_prep_cell(const LevelDev& L, int x, int y, int kk, int step) {
    if (x >= L.nx || y >= L.ny) return;
    const long long c = (long long)y * L.pitch + x;
    if ((L.flags[c] & (F_IN | F_COV)) != F_IN) return;
    const double* src;
    double* dst;
    level_bufs(L, kk, step, src, dst);
    const long long P = L.plane;
    double W[4], Qx[4], Qy[4], p;
#pragma unroll
    for (int k = 0; k < 4; k++)
        W[k] = (ld<COH>(src + qoff(0 + k, P, c)) + ld<COH>(src + qoff(4 + k, P, c))) +
               (ld<COH>(src + qoff(8 + k, P, c)) + ld<COH>(src + qoff(12 + k, P, c)));
    euler_flux(L.gm1, W, Qx, Qy, p);
    const double inv = rcp_rn(W[0]);  // = 1.0 / W[0]
#pragma unroll
    for (int k = 0; k < 4; k++) {
        L.sens[k * P + c] = Qx[k];
        L.sens[(4 + k) * P + c] = Qy[k];
        L.sens[(12 + k) * P + c] = W[k];
    }
    L.sens[8 * P + c] = W[1] * inv;
    L.sens[9 * P + c] = W[2] * inv;
    // the sweep takes W and Q from here: the state's check is made here
    if (!physical(W[0], p)) atomicOr(L.status, ST_NONPHYS);
}

// Pass 2 on cell (x, y): s and theta.
template <bool COH>
__device__ __forceinline__ void sensor_rate_cell(const LevelDev& L, int x, int y) {
    if (x >= L.nx || y >= L.ny) return;
    const long long c = (long long)y * L.pitch + x;
    if ((L.flags[c] & (F_IN | F_COV)) != F_IN) return;
    const long long e = sens_nb(L, x, y, 1, 0, c), ww = sens_nb(L, x, y, -1, 0, c);
    const long long n = sens_nb(L, x, y, 0, 1, c), so = sens_nb(L, x, y, 0, -1, c);
    const double* S = L.sens;
    const long long P = L.plane;
    double sh[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const double g = (ld<COH>(S + k * P + e) - ld<COH>(S + k * P + ww)) +
                         (ld<COH>(S + (4 + k) * P + n) - ld<COH>(S + (4 + k) * P + so));
        sh[k] = g * L.iq[k];
    }
    // fields paired (rho, rho E), (rho u, rho v): invariant under x <-> y
    L.sens[10 * P + c] = sqrt(0.25 * ((sh[0] * sh[0] + sh[3] * sh[3]) + (sh[1] * sh[1] + sh[2] * sh[2])));
    const double ue = ld<COH>(S + 8 * P + e), uw = ld<COH>(S + 8 * P + ww);
    const double un = ld<COH>(S + 8 * P + n), us = ld<COH>(S + 8 * P + so);
    const double ve = ld<COH>(S + 9 * P + e), vw = ld<COH>(S + 9 * P + ww);
    const double vn = ld<COH>(S + 9 * P + n), vs = ld<COH>(S + 9 * P + so);
    const double dil = (ue - uw) + (vn - vs);
    const double vort = (ve - vw) - (un - us);
    const double d2 = dil * dil;
    L.sens[11 * P + c] = dil < 0.0 ? div_rn(d2, (d2 + vort * vort) + L.eps) : 0.0;
}

__global__ void sensor_prep_kernel(const LevelDev* __restrict__ levs, const Item* __restrict__ items, int nitems,
                                   int kk, const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6, cx = threadIdx.x & 7, cy = (threadIdx.x >> 3) & 7;
    for (int it = blockIdx.x * TILES_PER_CTA + sub; it < nitems; it += gridDim.x * TILES_PER_CTA) {
        const Item w = items[it];
        const LevelDev& L = levs[w.lid];
        if (L.sens) sensor_prep_cell<false>(L, w.tx * TILE + cx, w.ty * TILE + cy, kk, 0);
    }
}

__global__ void sensor_rate_kernel(const LevelDev* __restrict__ levs, const Item* __restrict__ items, int nitems,
                                   const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6, cx = threadIdx.x & 7, cy = (threadIdx.x >> 3) & 7;
    for (int it = blockIdx.x * TILES_PER_CTA + sub; it < nitems; it += gridDim.x * TILES_PER_CTA) {
        const Item w = items[it];
        const LevelDev& L = levs[w.lid];
        if (L.sens) sensor_rate_cell<false>(L, w.tx * TILE + cx, w.ty * TILE + cy);
    }
}

// The relaxation parameter of active cell (x, y) from the 3 x 3 filters.
template <bool COH>
__device__ double sensor_beta_at(const LevelDev& L, int x, int y) {
    const long long c = (long long)y * L.pitch + x;
    const double* Ss = L.sens + 10 * L.plane;
    const double* St = L.sens + 11 * L.plane;
    // centre + ((E + W) + (N + S)) + ((NE + SW) + (NW + SE)): the same
    // rounding after swapping x and y
    const long long e = sens_nb(L, x, y, 1, 0, c), w = sens_nb(L, x, y, -1, 0, c);
    const long long n = sens_nb(L, x, y, 0, 1, c), so = sens_nb(L, x, y, 0, -1, c);
    const long long ne = sens_nb(L, x, y, 1, 1, c), sw = sens_nb(L, x, y, -1, -1, c);
    const long long nw = sens_nb(L, x, y, -1, 1, c), se = sens_nb(L, x, y, 1, -1, c);
    auto S = [&](long long i) { return ld<COH>(Ss + i); };
    auto T = [&](long long i) { return ld<COH>(St + i); };
    const double as = (S(c) + ((S(e) + S(w)) + (S(n) + S(so)))) + ((S(ne) + S(sw)) + (S(nw) + S(se)));
    const double at = (T(c) + ((T(e) + T(w)) + (T(n) + T(so)))) + ((T(ne) + T(sw)) + (T(nw) + T(se)));
    double z = (L.csens * (L.ninth * as)) * (L.ninth * at);
    if (z < 0.0) z = 0.0;
    if (z > 1.0) z = 1.0;
    return L.beta_max - (L.beta_max - L.beta_min) * z;
}

// ---------------------------------------------------------------------------
// the fused level sweep: collide, push-stream, boundary and coarse-to-fine
// ---------------------------------------------------------------------------

// Boundary values for the incoming populations of a cell whose upwind
// neighbour lies beyond a non-periodic side of the domain; f holds the
// cell's post-collision populations (constant indices only, so they stay in
// registers).
__device__ __forceinline__ void sweep_boundary(const LevelDev& L, int x, int y, long long c, const double (&f)[16],
                                               double* dst) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
        // side i: west (i = 0, x == 0), east, south, north
        const bool on = i == 0 ? (x == 0 && !L.px)
                                : i == 1 ? (x == L.nx - 1 && !L.px) : i == 2 ? (y == 0 && !L.py) : (y == L.ny - 1 && !L.py);
        if (!on) continue;
        const int bc = L.bc[i];
        const int normal = i < 2 ? 1 : 2;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            double v;
            if (bc == BC_OUTFLOW) {
                v = f[4 * i + k];
            } else if (bc == BC_INFLOW) {
                v = L.feqb[i][4 * i + k];
            } else {
                const double m = f[4 * (i ^ 1) + k];
                v = (k == normal) ? -m : m;
            }
            dst[qoff(4 * i + k, L.plane, c)] = v;
        }
    }
}

// Reconstructed coarse-to-fine values for the incoming populations of a
// cell whose upwind neighbour lies in coarser territory.
template <bool COH>
__device__ __forceinline__ void sweep_recon(const LevelDev* __restrict__ levs, const LevelDev& L, int x, int y,
                                        long long c, uint32_t fl, double* dst, int kk, int kkp, int step) {
    // coarse-to-fine reconstruction (Sec. 3.3, Eqs. 22-23)
    const uint32_t rec = (fl & F_RECON_MASK) >> F_RECON_SHIFT;
    if (!rec) return;
    const LevelDev& P = levs[L.parent];
    const double* psrc;
    double* pdst;
    level_bufs(P, kkp, step, psrc, pdst);
    const double wk = (kk == 1) ? -0.25 : 0.25;
    for (int i = 0; i < 4; i++) {
        if (!(rec & (1u << i))) continue;
        int ux = x - kCX[i], uy = y - kCY[i];
        if (ux < 0) ux += L.nx;
        if (ux >= L.nx) ux -= L.nx;
        if (uy < 0) uy += L.ny;
        if (uy >= L.ny) uy -= L.ny;
        const int l0x = ux >> 1, l0y = uy >> 1;  // coarse cell L0
        const int hx = x >> 1, hy = y >> 1;      // covered cell C = L0 + c_d
        const int d = i;
        const int tx = d < 2 ? 0 : 1, ty = d < 2 ? 1 : 0;
        int mx = l0x - tx, my = l0y - ty, qx = l0x + tx, qy = l0y + ty;
        int hmx = hx - tx, hmy = hy - ty, hpx = hx + tx, hpy = hy + ty;
        bool okm = true, okp = true;
        if (tx) {
            if (mx < 0) { if (P.px) { mx += P.nx; hmx += P.nx; } else okm = false; }
            if (qx >= P.nx) { if (P.px) { qx -= P.nx; hpx -= P.nx; } else okp = false; }
        } else {
            if (my < 0) { if (P.py) { my += P.ny; hmy += P.ny; } else okm = false; }
            if (qy >= P.ny) { if (P.py) { qy -= P.ny; hpy -= P.ny; } else okp = false; }
        }
        if (okm) okm = (ld<COH>(P.flags + (long long)my * P.pitch + mx) & (F_IN | F_COV)) == F_IN;
        if (okp) okp = (ld<COH>(P.flags + (long long)qy * P.pitch + qx) & (F_IN | F_COV)) == F_IN;
        const bool fresh = (ld<COH>(P.flags + (long long)l0y * P.pitch + l0x) >> (F_FRESH_SHIFT + d)) & 1u;
        const long long ch = (long long)hy * P.pitch + hx;
        const long long cm = (long long)hmy * P.pitch + hmx;
        const long long cp = (long long)hpy * P.pitch + hpx;
        const int j = d < 2 ? (y & 1) : (x & 1);
        const double wj = j ? 0.25 : -0.25;
        for (int k = 0; k < 4; k++) {
            const int q = 4 * d + k;
            const double a = ld<COH>(pdst + qoff(q, P.plane, ch));
            const double ap = fresh ? a : ld<COH>(psrc + qoff(q, P.plane, ch));
            double s = 0.0;
            if (okm && okp) s = minmod(a - ld<COH>(pdst + qoff(q, P.plane, cm)), ld<COH>(pdst + qoff(q, P.plane, cp)) - a);
            dst[qoff(4 * i + k, L.plane, c)] = fma(s, wj, fma(a - ap, wk, a));
        }
    }
}

// One cell of one level step: load the 16 populations, collide, push, then
// the boundary / reconstruction slow path.  kk: this level's sub-step (1, 2)
// within its parent's step (ignored on level 0); kkp: the parent's
// sub-step; step: coarse step index inside a multi-step launch.
template <int P, bool COH>
__device__ __forceinline__ void sweep_cell(const LevelDev* __restrict__ levs, const LevelDev& L, int x, int y, int kk,
                                           int kkp, int step, double* Wout = nullptr) {
    const int nx = L.nx, ny = L.ny;
    if (x >= nx || y >= ny) return;
    const long long c = (long long)y * L.pitch + x;
    const uint32_t fl = ld<COH>(L.flags + c);
    if ((fl & (F_IN | F_COV)) != F_IN) return;
    const double* src;
    double* dst;
    level_bufs(L, kk, step, src, dst);
    const long long plane = L.plane;
    double f[16];
#pragma unroll
    for (int pr = 0; pr < 8; pr++) {  // 16-byte loads of the field pairs
        const double2 v = ld<COH>(reinterpret_cast<const double2*>(src + qoff(2 * pr, plane, c)));
        f[2 * pr] = v.x;
        f[2 * pr + 1] = v.y;
    }
    bool ok;
    if constexpr ((P & SW_SENSOR) != 0) {
        if (L.sens) {
            // the moments and fluxes of the sensor's first pass (the same
            // populations, the same expressions) and the cell's own beta
            const double b = sensor_beta_at<COH>(L, x, y);
            double W[4], Qx[4], Qy[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                W[k] = ld<COH>(L.sens + (12 + k) * plane + c);
                Qx[k] = ld<COH>(L.sens + k * plane + c);
                Qy[k] = ld<COH>(L.sens + (4 + k) * plane + c);
            }
            if (Wout)
                for (int k = 0; k < 4; k++) Wout[k] = W[k];
            relax(f, W, Qx, Qy, 1.0 - 2.0 * b, 0.5 * b, div_rn_y(b, L.c, L.rc));  // b / c
            ok = true;  // the first pass checked the state
        } else {
            ok = collide(f, L.om, L.hb, L.bcs, L.gm1, Wout);
        }
    } else {
        ok = collide(f, L.om, L.hb, L.bcs, L.gm1, Wout);
    }
    if (!ok) atomicOr(L.status, ST_NONPHYS);
    // push streaming (Eq. 5): f*_i lands on x + c_i
    long long cxp = c + 1, cxm = c - 1, cyp = c + L.pitch, cym = c - L.pitch;
    bool oxp = true, oxm = true, oyp = true, oym = true;
    if (x == nx - 1) { if (L.px) cxp = c - (nx - 1); else oxp = false; }
    if (x == 0) { if (L.px) cxm = c + (nx - 1); else oxm = false; }
    if (y == ny - 1) { if (L.py) cyp = c - (long long)(ny - 1) * L.pitch; else oyp = false; }
    if (y == 0) { if (L.py) cym = c + (long long)(ny - 1) * L.pitch; else oym = false; }
    // 16-byte stores of the field pairs
    auto push = [&](int i, long long t) {
        *reinterpret_cast<double2*>(dst + qoff(4 * i, plane, t)) = make_double2(f[4 * i], f[4 * i + 1]);
        *reinterpret_cast<double2*>(dst + qoff(4 * i + 2, plane, t)) = make_double2(f[4 * i + 2], f[4 * i + 3]);
    };
    if (oxp) push(0, cxp);
    if (oxm) push(1, cxm);
    if (oyp) push(2, cyp);
    if (oym) push(3, cym);
    if (fl & F_BND) sweep_boundary(L, x, y, c, f, dst);
    if (fl & F_RECON_MASK) sweep_recon<COH>(levs, L, x, y, c, fl, dst, kk, kkp, step);
}

// One step of one level for every tile in `items` (all of the same level
// index within their hierarchies).
template <int P, int MINB>
__global__ void __launch_bounds__(CTA_THREADS, MINB)
sweep_kernel(const LevelDev* __restrict__ levs, const Item* __restrict__ items, int nitems, int kk, int kkp,
             const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6;
    const int cx = threadIdx.x & 7;
    const int cy = (threadIdx.x >> 3) & 7;
    for (int it = blockIdx.x * TILES_PER_CTA + sub; it < nitems; it += gridDim.x * TILES_PER_CTA) {
        const Item w = items[it];
        sweep_cell<P, false>(levs, levs[w.lid], w.tx * TILE + cx, w.ty * TILE + cy, kk, kkp, 0);
    }
}

// Reflux (Sec. 3.3, Eq. 24) for one cell: the pending incoming population of
// a coarse ring cell is the plain average of the four post-collision values
// the fine edge cells sent towards it during the cycle, summed (k = 1:
// j = 0, 1), then (k = 2: j = 0, 1).  Also retires the "no previous sample"
// marks.
template <bool COH>
__device__ __forceinline__ void close_cell(const LevelDev* __restrict__ levs, const LevelDev& L, int x, int y, int kk,
                                           int step) {
    if (x >= L.nx || y >= L.ny) return;
    const long long c = (long long)y * L.pitch + x;
    const uint32_t fl = ld<COH>(L.flags + c);
    const uint32_t pend = (fl & F_PEND_MASK) >> F_PEND_SHIFT;
    if ((fl & (F_IN | F_COV)) != F_IN || !pend) return;
    const double* src;
    double* dst;
    level_bufs(L, kk, step, src, dst);
    const LevelDev& F = levs[L.child];
    const double* s1 = F.buf[1];  // fine sub-step 1 wrote buffer 1
    const double* s2 = F.buf[0];  // fine sub-step 2 wrote buffer 0
    for (int i = 0; i < 4; i++) {
        if (!(pend & (1u << i))) continue;
        const int d = i ^ 1;  // from this cell towards the covered one
        int gx0, gy0, gx1, gy1;
        if (d == 0) { gx0 = gx1 = 2 * x + 1; gy0 = 2 * y; gy1 = 2 * y + 1; }
        else if (d == 1) { gx0 = gx1 = 2 * x; gy0 = 2 * y; gy1 = 2 * y + 1; }
        else if (d == 2) { gy0 = gy1 = 2 * y + 1; gx0 = 2 * x; gx1 = 2 * x + 1; }
        else { gy0 = gy1 = 2 * y; gx0 = 2 * x; gx1 = 2 * x + 1; }
        const long long g0 = (long long)gy0 * F.pitch + gx0;
        const long long g1 = (long long)gy1 * F.pitch + gx1;
        for (int k = 0; k < 4; k++) {
            const int q = 4 * i + k;
            const long long o0 = qoff(q, F.plane, g0), o1 = qoff(q, F.plane, g1);
            const double v = ((ld<COH>(s1 + o0) + ld<COH>(s1 + o1)) + (ld<COH>(s2 + o0) + ld<COH>(s2 + o1))) * 0.25;
            dst[qoff(q, L.plane, c)] = v;
        }
    }
    if (fl & F_FRESH_MASK) L.flags[c] = (uint16_t)(fl & ~F_FRESH_MASK);
}

__global__ void close_kernel(const LevelDev* __restrict__ levs, const Item* __restrict__ items, int nitems, int kk,
                             const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6;
    const int cx = threadIdx.x & 7;
    const int cy = (threadIdx.x >> 3) & 7;
    for (int it = blockIdx.x * TILES_PER_CTA + sub; it < nitems; it += gridDim.x * TILES_PER_CTA) {
        const Item w = items[it];
        close_cell<false>(levs, levs[w.lid], w.tx * TILE + cx, w.ty * TILE + cy, kk, 0);
    }
}

// Exact sums of the audited moments.  An audit slot holds W_k of the 64
// cells of one tile, layout [k][cell], at weight 2^scale[slot]; a thread
// reads one (field, cell) column across a range of slots and keeps two
// sums (W and |W|).
//
// Fast path: the values a thread sees have nearly the same exponent, so
// they are added as integers m * 2^d (m the 53-bit significand) into a
// two's-complement 128-bit window whose least significant bit sits at
// position `base` of the 192-bit fixed point (0 <= base <= 64, chosen from
// the thread's first value).  A value whose bits fit the window exactly
// (0 <= d < 64) takes the fast path; zeros are skipped; anything else
// (subnormal, tiny, huge, NaN) takes the general 192-bit path.  Below 2^10
// fast additions the window cannot overflow (|m 2^d| < 2^117); it is
// folded into the 192-bit sums before that and at the end, so the result
// is the same exact sum either way.
struct Win128 {
    unsigned long long lo, hi;
};

__device__ __forceinline__ void win_fold(Fix192& acc, Win128& w, int base) {
    const unsigned long long ext = (w.hi >> 63) ? ~0ull : 0ull;
    Fix192 f;
    if (base == 0) {
        f.w[0] = w.lo;
        f.w[1] = w.hi;
        f.w[2] = ext;
    } else if (base == 64) {
        f.w[0] = 0ull;
        f.w[1] = w.lo;
        f.w[2] = w.hi;
    } else {
        f.w[0] = w.lo << base;
        f.w[1] = (w.hi << base) | (w.lo >> (64 - base));
        f.w[2] = (ext << base) | (w.hi >> (64 - base));
    }
    fix_add(acc, f);
    w.lo = w.hi = 0ull;
}

// A thread's running exact sums (sum, abs_sum) with the 128-bit window in
// front of them: add(v, sc) takes v * 2^sc, flush() folds the window in.
struct WinSum {
    Win128 ws{0ull, 0ull}, wa{0ull, 0ull};
    int base = -1, nfast = 0;

    __device__ __forceinline__ void add(double v, int sc, Fix192& sum, Fix192& abs_sum) {
        const unsigned long long B = (unsigned long long)__double_as_longlong(v);
        if ((B << 1) == 0ull) return;  // +-0
        const int E = (int)((B >> 52) & 0x7FFull);
        const int sh = E - 947 + sc;  // position of the significand's lsb (2^-128 units)
        if (base < 0 && E != 0 && E != 2047) base = min(max(sh - 32, 0), 64);
        const int d = sh - base;
        if (E == 0 || E == 2047 || base < 0 || d < 0 || d > 63) {
            fix_accumulate(sum, abs_sum, v, sc);
            return;
        }
        const unsigned long long m = (B & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
        const unsigned long long lo = m << d;
        const unsigned long long hi = d ? m >> (64 - d) : 0ull;
        // |v| into the magnitude window
        const unsigned long long a0 = wa.lo + lo;
        wa.hi += hi + (a0 < lo ? 1ull : 0ull);
        wa.lo = a0;
        // +-|v| into the signed window
        if (B >> 63) {
            const unsigned long long brw = ws.lo < lo ? 1ull : 0ull;
            ws.lo -= lo;
            ws.hi -= hi + brw;
        } else {
            const unsigned long long s0 = ws.lo + lo;
            ws.hi += hi + (s0 < lo ? 1ull : 0ull);
            ws.lo = s0;
        }
        if (++nfast == 1023) flush(sum, abs_sum);
    }

    __device__ __forceinline__ void flush(Fix192& sum, Fix192& abs_sum) {
        if (base < 0) return;
        win_fold(sum, ws, base);
        win_fold(abs_sum, wa, base);
        nfast = 0;
    }
};

// Exact per-thread sums of v_j * 2^scale[j] for v_j = aw[j * AUDIT_SLOT +
// col], slots j in [j0, j1), into sum and abs_sum (192-bit), through the
// 128-bit window; COH: loads through L2 (data written in the same launch).
template <bool COH>
__device__ __forceinline__ void audit_thread_sums(const double* __restrict__ aw, const int* __restrict__ scale,
                                                  int j0, int j1, int col, Fix192& sum, Fix192& abs_sum) {
    WinSum acc;
    // AUDIT_BATCH loads in flight per thread, then their accumulation
    constexpr int AUDIT_BATCH = 8;
    for (int jb = j0; jb < j1; jb += AUDIT_BATCH) {
        double vb[AUDIT_BATCH];
        int sb[AUDIT_BATCH];
#pragma unroll
        for (int u = 0; u < AUDIT_BATCH; u++) {
            const int j = jb + u;
            const double* q = aw + (size_t)j * AUDIT_SLOT + col;
            vb[u] = j < j1 ? (COH ? __ldcg(q) : __ldcs(q)) : 0.0;
            sb[u] = j < j1 ? (COH ? __ldcg(scale + j) : __ldg(scale + j)) : 0;
        }
#pragma unroll
        for (int u = 0; u < AUDIT_BATCH; u++) acc.add(vb[u], sb[u], sum, abs_sum);
    }
    acc.flush(sum, abs_sum);
}

// Barrier of one 64-thread group (named barrier 1 + g).
__device__ __forceinline__ void group_bar(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(64) : "memory");
}

// Audit task (kind 2) run by one 64-thread group: field T.kk over the audit
// block T.aslot; thread lt reads column (field, cell lt) of every slot of the
// block (written earlier in the same launch: loads through L2).  The block's
// sums of W_k and |W_k| go to words 3 k .. 3 k + 2 and 3 (4 + k) .. of its
// 24-word partial.
__device__ __forceinline__ void audit_task(const Segment& S, const Task& T, int g, int lt) {
    __shared__ Fix192 s_ap[TILES_PER_CTA][2][2];
    const int k = T.kk;
    const int2 r = S.arng[T.aslot];
    Fix192 sum = fix_zero(), abs_sum = fix_zero();
    audit_thread_sums<true>(S.aw, S.ascale, r.x, r.y, k * 64 + lt, sum, abs_sum);
    for (int off = 16; off > 0; off >>= 1) {
        const Fix192 o1 = fix_shfl_down(sum, off);
        const Fix192 o2 = fix_shfl_down(abs_sum, off);
        fix_add(sum, o1);
        fix_add(abs_sum, o2);
    }
    if ((lt & 31) == 0) {
        s_ap[g][lt >> 5][0] = sum;
        s_ap[g][lt >> 5][1] = abs_sum;
    }
    group_bar(g);
    if (lt == 0) {
        Fix192 a = s_ap[g][0][0], b = s_ap[g][0][1];
        fix_add(a, s_ap[g][1][0]);
        fix_add(b, s_ap[g][1][1]);
        unsigned long long* o = S.apart + (size_t)T.aslot * 24;
        for (int i = 0; i < 3; i++) {
            o[3 * k + i] = a.w[i];
            o[3 * (4 + k) + i] = b.w[i];
        }
    }
}

// The same by one warp alone (two columns per lane).
__device__ __forceinline__ void audit_task_warp(const Segment& S, const Task& T, int lane) {
    const int k = T.kk;
    const int2 r = S.arng[T.aslot];
    Fix192 sum = fix_zero(), abs_sum = fix_zero();
    audit_thread_sums<true>(S.aw, S.ascale, r.x, r.y, k * 64 + lane, sum, abs_sum);
    audit_thread_sums<true>(S.aw, S.ascale, r.x, r.y, k * 64 + 32 + lane, sum, abs_sum);
    for (int off = 16; off > 0; off >>= 1) {
        const Fix192 o1 = fix_shfl_down(sum, off);
        const Fix192 o2 = fix_shfl_down(abs_sum, off);
        fix_add(sum, o1);
        fix_add(abs_sum, o2);
    }
    if (lane == 0) {
        unsigned long long* o = S.apart + (size_t)T.aslot * 24;
        for (int i = 0; i < 3; i++) {
            o[3 * k + i] = sum.w[i];
            o[3 * (4 + k) + i] = abs_sum.w[i];
        }
    }
}

// ---------------------------------------------------------------------------
// the persistent task kernel: every tile of every phase of G coarse steps,
// of every hierarchy of the batch, in one launch
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Completion marks: a task of launch epoch e is complete when its mark holds
// 2 e.  Marks only grow (a mark left by an earlier launch, of this task list
// or of one built before it, is at most 2 (e - 1)), so a kernel never
// mistakes a stale mark for completion and no mark is ever reset between
// launches, whichever task kernel ran them.
//
// Bounded wait on a task's completion mark: gives up after ~2^21 polls
// (about a second), records a timeout in the hierarchy's status word and
// returns, so that a broken schedule can never hang the GPU.
__device__ __forceinline__ void wait_done(const unsigned* p, unsigned mark, int* status) {
    unsigned ns = 32;
    for (int it = 0; it < (1 << 21); it++) {
        if ((int)(ld_acquire(p) - mark) >= 0) return;
        // once any wait of this hierarchy has given up, stop waiting at all
        if ((it & 255) == 255 && (*(volatile int*)status & ST_TIMEOUT)) return;
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
    }
    atomicOr(status, ST_TIMEOUT);
}

// The chunk holding ticket t: prefix[c] <= t < prefix[c + 1].
__device__ __forceinline__ int find_segment(const int* __restrict__ prefix, int nseg, int t) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Tasks are claimed in list order -- segment by segment, each segment in a
// topological order of its dependencies -- so every task a claimed task
// waits for was claimed earlier by a running thread group: the schedule
// cannot deadlock, whatever the number of resident CTAs.  A group claims its
// next ticket once the waits of its current task are over, so a claimed but
// unstarted task only ever waits behind a task that no longer waits.
//
// Memory ordering: the group's lane 0 publishes a task with a gpu-scope
// fence and a release store after a group barrier (the writes of all 64
// threads precede the barrier); waiting lanes read the marks with acquire
// loads before the group barrier that precedes the task's reads, which go
// through L2 (ld.global.cg, cp.async.cg).


// Iterations: a launch runs its task list `iters` times in a row, one coarse
// step per iteration (iters > 1 only for a one-step list of one hierarchy).
// Ticket t is task t % total of iteration t / total; iteration it of launch
// epoch e completes a task with mark 2 (e + it).  A dependency entry d >= 0
// is task d of the same iteration; d < 0 is task ~d of the previous
// iteration, satisfied by stream order in the launch's first iteration.
__device__ __forceinline__ void wait_deps(const Segment& S, const Task& T, int it, unsigned mark, int lane, int width,
                                          int* status) {
    for (int j = lane; j < T.ndep; j += width) {
        const int d = S.deps[T.dep0 + j];
        if (d >= 0) wait_done(S.done + d, mark, status);
        else if (it > 0) wait_done(S.done + ~d, mark - 2u, status);
    }
}

template <int P, int MINB>
__global__ void __launch_bounds__(CTA_THREADS, MINB)
task_kernel(const LevelDev* __restrict__ levs, const Segment* __restrict__ segs, const int* __restrict__ prefix,
            const int2* __restrict__ chunks, int* ctl, int iters) {
    __shared__ int s_task[TILES_PER_CTA][2];
    const int g = threadIdx.x >> 6;
    const int lt = threadIdx.x & 63;
    const int cx = lt & 7, cy = lt >> 3;
    const unsigned epoch = (unsigned)ctl[CTL_EPOCH];
    const int total = ctl[CTL_TOTAL], nseg = ctl[CTL_NSEG], nchunk = ctl[CTL_NCHUNK];
    const bool audit = ctl[CTL_AUDIT] != 0;
    const int cyc = total * iters;
    const int tickets = cyc + (audit ? ctl[CTL_NAUD] : 0);
    if (lt == 0) s_task[g][0] = atomicAdd(&ctl[CTL_CLAIM], 1);
    group_bar(g);
    for (int par = 0;; par ^= 1) {
        const int t = s_task[g][par];
        if (t >= tickets) break;
        int it, i;
        Segment S;
        if (t < cyc) {
            it = t / total;
            const int tt = t - it * total;
            const int ck = find_segment(prefix, nchunk, tt);
            const int2 chunk = chunks[ck];
            S = segs[chunk.x];
            i = chunk.y + (tt - prefix[ck]);
        } else {  // an audited launch's reduction tasks (one list), after every iteration
            it = 0;
            S = segs[0];
            i = total + (t - cyc);
        }
        const Task T = S.tasks[i];
        const LevelDev& L = levs[T.lid + S.lid_base];
        const unsigned mark = 2u * (epoch + (unsigned)it);
        const int step = T.step + it;
        // audit work (moments kept, reduction tasks) in the first iteration
        // of an audited launch only; a reduction task is empty otherwise
        const bool aud = audit && it == 0;
        if (T.kind != 2 || aud) wait_deps(S, T, it, mark, lt, 64, L.status);
        if (lt == 0) s_task[g][par ^ 1] = atomicAdd(&ctl[CTL_CLAIM], 1);
        group_bar(g);
        if (T.kind == 0) {
            if (aud && S.aw && T.aslot >= 0) {
                // audited sweep: keep the moments of the cell (0 off the
                // active set) for the exact reduction after the launch
                double W[4] = {0.0, 0.0, 0.0, 0.0};
                sweep_cell<P, true>(levs, L, T.tx * TILE + cx, T.ty * TILE + cy, T.kk, T.kkp, step, W);
                double* o = S.aw + (size_t)T.aslot * AUDIT_SLOT + lt;
                for (int k = 0; k < 4; k++) o[k * 64] = W[k];
            } else {
                sweep_cell<P, true>(levs, L, T.tx * TILE + cx, T.ty * TILE + cy, T.kk, T.kkp, step);
            }
        } else if (T.kind == 1) {
            close_cell<true>(levs, L, T.tx * TILE + cx, T.ty * TILE + cy, T.kk, step);
        } else if (T.kind == 2) {
            if (aud) audit_task(S, T, g, lt);
        } else if constexpr ((P & SW_SENSOR) != 0) {
            // the relaxation sensor's passes of the level step (kinds 3, 4)
            if (T.kind == 3) sensor_prep_cell<true>(L, T.tx * TILE + cx, T.ty * TILE + cy, T.kk, step);
            else sensor_rate_cell<true>(L, T.tx * TILE + cx, T.ty * TILE + cy);
        }
        group_bar(g);
        if (lt == 0) {
            __threadfence();
            st_release(S.done + i, mark);
            if (atomicAdd(&ctl[CTL_FIN], 1) == tickets - 1) {
                // every task of the launch is complete: advance the parity of
                // each hierarchy by the launch's step count, open the next epoch
                if (ctl[CTL_FLIP] && (iters & 1))
                    for (int m = 0; m < nseg; m++) *segs[m].par0 ^= 1;
                ctl[CTL_EPOCH] = (int)(epoch + (unsigned)iters);
            }
        }
    }
}

// TK_HALF: the same schedule with every warp on its own -- a task (tile) is
// two half-tasks of four rows, claimed as tickets 2 t and 2 t + 1 by any
// two warps; each warp waits for the task's dependencies itself.  The first
// half to finish raises the task's mark to 2 e - 1, the second (which sees
// 2 e - 1 there) publishes 2 e.  No group barrier is left in the loop.
// Deadlock freedom is unchanged: the halves of every task a half waits for
// were claimed before it.
template <int P, int MINB>
__global__ void __launch_bounds__(CTA_THREADS, MINB)
task_kernel_half(const LevelDev* __restrict__ levs, const Segment* __restrict__ segs,
                 const int* __restrict__ prefix, const int2* __restrict__ chunks, int* ctl, int iters) {
    const int lane = threadIdx.x & 31;
    const unsigned epoch = (unsigned)ctl[CTL_EPOCH];
    const int total = ctl[CTL_TOTAL], nseg = ctl[CTL_NSEG], nchunk = ctl[CTL_NCHUNK];
    const bool audit = ctl[CTL_AUDIT] != 0;
    const int cyc = total * iters;
    const int tickets = 2 * (cyc + (audit ? ctl[CTL_NAUD] : 0));
    for (;;) {
        int h = 0;
        if (lane == 0) h = atomicAdd(&ctl[CTL_CLAIM], 1);
        h = __shfl_sync(0xffffffffu, h, 0);
        if (h >= tickets) break;
        const int t = h >> 1, half = h & 1;
        int it, i;
        Segment S;
        if (t < cyc) {
            it = t / total;
            const int tt = t - it * total;
            const int ck = find_segment(prefix, nchunk, tt);
            const int2 chunk = chunks[ck];
            S = segs[chunk.x];
            i = chunk.y + (tt - prefix[ck]);
        } else {  // an audited launch's reduction tasks (one list), after every iteration
            it = 0;
            S = segs[0];
            i = total + (t - cyc);
        }
        const Task T = S.tasks[i];
        const LevelDev& L = levs[T.lid + S.lid_base];
        const unsigned mark = 2u * (epoch + (unsigned)it);
        const int step = T.step + it;
        const bool aud = audit && it == 0;
        if (T.kind != 2 || aud) wait_deps(S, T, it, mark, lane, 32, L.status);
        __syncwarp();
        const int cx = lane & 7, cy = half * 4 + (lane >> 3), lt = cy * 8 + cx;
        if (T.kind == 0) {
            if (aud && S.aw && T.aslot >= 0) {
                double W[4] = {0.0, 0.0, 0.0, 0.0};
                sweep_cell<P, true>(levs, L, T.tx * TILE + cx, T.ty * TILE + cy, T.kk, T.kkp, step, W);
                double* o = S.aw + (size_t)T.aslot * AUDIT_SLOT + lt;
                for (int k = 0; k < 4; k++) o[k * 64] = W[k];
            } else {
                sweep_cell<P, true>(levs, L, T.tx * TILE + cx, T.ty * TILE + cy, T.kk, T.kkp, step);
            }
        } else if (T.kind == 1) {
            close_cell<true>(levs, L, T.tx * TILE + cx, T.ty * TILE + cy, T.kk, step);
        } else if (T.kind == 2) {
            if (aud && half == 0) audit_task_warp(S, T, lane);  // the first half does the whole audit task
        } else if constexpr ((P & SW_SENSOR) != 0) {
            if (T.kind == 3) sensor_prep_cell<true>(L, T.tx * TILE + cx, T.ty * TILE + cy, T.kk, step);
            else sensor_rate_cell<true>(L, T.tx * TILE + cx, T.ty * TILE + cy);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            if (atomicMax(S.done + i, mark - 1u) == mark - 1u) {
                __threadfence();
                st_release(S.done + i, mark);
            }
            if (atomicAdd(&ctl[CTL_FIN], 1) == tickets - 1) {
                if (ctl[CTL_FLIP] && (iters & 1))
                    for (int m = 0; m < nseg; m++) *segs[m].par0 ^= 1;
                ctl[CTL_EPOCH] = (int)(epoch + (unsigned)iters);
            }
        }
    }
}

__global__ void end_step_kernel(int* const* par, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) *par[t] ^= 1;
}

// Totals from exact partial sums: segment b covers partials [seg[b],
// seg[b+1]) (seg == nullptr: one segment [0, n)); out[b][0..3] = sum w W_k,
// out[b][4..7] = sum w |W_k|, each the correctly rounded exact sum.
__global__ void __launch_bounds__(256) audit_segments_kernel(const unsigned long long* __restrict__ slots,
                                                             const int* __restrict__ seg, int n,
                                                             double* __restrict__ out) {
    __shared__ Fix192 part[256 / 32][8];
    const int b = blockIdx.x;
    const int i0 = seg ? seg[b] : 0, i1 = seg ? seg[b + 1] : n;
    Fix192 acc[8];
    for (int k = 0; k < 8; k++) acc[k] = fix_zero();
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
        for (int k = 0; k < 8; k++) {
            Fix192 v;
            for (int j = 0; j < 3; j++) v.w[j] = __ldcg(slots + (size_t)i * 24 + 3 * k + j);
            fix_add(acc[k], v);
        }
    for (int off = 16; off > 0; off >>= 1)
        for (int k = 0; k < 8; k++) {
            const Fix192 o = fix_shfl_down(acc[k], off);
            fix_add(acc[k], o);
        }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 8; k++) part[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < 8) {
        const int k = threadIdx.x;
        Fix192 a = part[0][k];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) fix_add(a, part[w][k]);
        out[(size_t)b * 8 + k] = fix_to_double(a);
    }
}

// ---------------------------------------------------------------------------
// initialisation and read-back
// ---------------------------------------------------------------------------

// f = f^eq(W) on every cell of the level (Eq. 4): W/4 +- Q_alpha/(2c).
__global__ void feq_init_kernel(LevelDev L, const double* __restrict__ W, long long ld, double hc) {
    const long long n = (long long)L.nx * L.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % L.nx), y = (int)(t / L.nx);
        const long long c = (long long)y * L.pitch + x;
        if (!(L.flags[c] & F_IN)) continue;
        double w[4], Qx[4], Qy[4], p;
        const long long pl = ld * L.ny;
        for (int k = 0; k < 4; k++) w[k] = W[k * pl + (long long)y * ld + x];
        euler_flux(L.gm1, w, Qx, Qy, p);
        double* out = L.buf[state_buf(L)];
        for (int k = 0; k < 4; k++) {
            const double qw = 0.25 * w[k];
            out[qoff(0 + k, L.plane, c)] = fma(hc, Qx[k], qw);
            out[qoff(4 + k, L.plane, c)] = fma(-hc, Qx[k], qw);
            out[qoff(8 + k, L.plane, c)] = fma(hc, Qy[k], qw);
            out[qoff(12 + k, L.plane, c)] = fma(-hc, Qy[k], qw);
        }
    }
}

// population planes <-> a dense [16][ny][ld] array (state buffer)
__global__ void copy_pop_kernel(LevelDev L, double* __restrict__ ext, long long ld, int to_ext) {
    const long long n = (long long)L.nx * L.ny;
    double* st = L.buf[state_buf(L)];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % L.nx), y = (int)(t / L.nx);
        const long long c = (long long)y * L.pitch + x;
        for (int q = 0; q < 16; q++) {
            const long long e = (long long)q * ld * L.ny + (long long)y * ld + x;
            if (to_ext) ext[e] = st[qoff(q, L.plane, c)];
            else st[qoff(q, L.plane, c)] = ext[e];
        }
    }
}

// W = sum_i f_i (same order as the collision) and the active mask.
__global__ void gather_W_kernel(LevelDev L, double* __restrict__ W, long long ld, uint8_t* __restrict__ valid) {
    const long long n = (long long)L.nx * L.ny;
    const double* st = L.buf[state_buf(L)];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % L.nx), y = (int)(t / L.nx);
        const long long c = (long long)y * L.pitch + x;
        const uint32_t fl = L.flags[c];
        const long long pl = ld * L.ny;
        const long long o = (long long)y * ld + x;
        for (int k = 0; k < 4; k++) {
            double v = 0.0;
            if (fl & F_IN)
                v = (st[qoff(0 + k, L.plane, c)] + st[qoff(4 + k, L.plane, c)]) +
                    (st[qoff(8 + k, L.plane, c)] + st[qoff(12 + k, L.plane, c)]);
            W[k * pl + o] = v;
        }
        if (valid) valid[(long long)y * L.nx + x] = (fl & (F_IN | F_COV)) == F_IN;
    }
}

// ---------------------------------------------------------------------------
// conservation audit: exact sums
// ---------------------------------------------------------------------------

// Exact per-CTA sums over the cells of the listed active tiles (a tile is
// entirely active, entirely covered or entirely off its level, so every
// cell of an active tile within the domain is active; the cell flags are
// not read): part[blk][0..23] = sum w W_k (k = 0..3), then sum w |W_k|,
// w = 4^-level, as 192-bit fixed point (three words each).  A CTA takes one
// tile at a time; its 64-thread group g adds up field k = g of the tile's
// cells, so a thread holds two accumulators and many CTAs fit on an SM.
// The last CTA to finish writes the rounded totals out[0..7] (ticket: a
// zeroed counter, left zeroed).

// One thread's view of one tile: whether its cell lies in the domain, and
// the four populations of its (field, cell), loaded without waiting for them.
struct AuditCell {
    bool on;
    int lev;
    double f0, f1, f2, f3;
};

__device__ __forceinline__ AuditCell audit_load(const LevelDev* __restrict__ levs, const Item* __restrict__ items,
                                                int it, int nitems, int k, int cx, int cy) {
    AuditCell a{false, 0, 0.0, 0.0, 0.0, 0.0};
    if (it >= nitems) return a;
    const Item w = items[it];
    const LevelDev& L = levs[w.lid];
    const int x = w.tx * TILE + cx, y = w.ty * TILE + cy;
    if (x >= L.nx || y >= L.ny) return a;
    const long long c = (long long)y * L.pitch + x;
    const double* st = L.buf[state_buf(L)];
    a.on = true;
    a.lev = L.level;
    a.f0 = __ldcs(st + qoff(0 + k, L.plane, c));
    a.f1 = __ldcs(st + qoff(4 + k, L.plane, c));
    a.f2 = __ldcs(st + qoff(8 + k, L.plane, c));
    a.f3 = __ldcs(st + qoff(12 + k, L.plane, c));
    return a;
}

// The CTA that finishes last: out[m] = the correctly rounded sum of quantity
// m over the partials of the launch's nb blocks; warp m of the CTA takes
// quantity m.
__device__ __noinline__ void audit_finish(const unsigned long long* part, int nb, double* out) {
    const int lane = threadIdx.x & 31, m = threadIdx.x >> 5;
    if (m >= 8) return;
    Fix192 a = fix_zero();
    for (int i = lane; i < nb; i += 32) {
        Fix192 v;
        for (int j = 0; j < 3; j++) v.w[j] = __ldcg(part + (size_t)i * 24 + 3 * m + j);
        fix_add(a, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const Fix192 b = fix_shfl_down(a, o);
        fix_add(a, b);
    }
    if (lane == 0) out[m] = fix_to_double(a);
}

__global__ void __launch_bounds__(256) audit_kernel(const LevelDev* __restrict__ levs, const Item* __restrict__ items,
                                                    int nitems, unsigned long long* __restrict__ part,
                                                    double* __restrict__ out, unsigned* __restrict__ ticket,
                                                    const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int k = threadIdx.x >> 6;
    const int cx = threadIdx.x & 7;
    const int cy = (threadIdx.x >> 3) & 7;
    Fix192 sum = fix_zero(), abs_sum = fix_zero();
    WinSum acc;
    // the next tile's flags and populations are in flight while this tile's
    // are added up
    AuditCell cur = audit_load(levs, items, blockIdx.x, nitems, k, cx, cy);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const AuditCell nxt = audit_load(levs, items, it + gridDim.x, nitems, k, cx, cy);
        if (cur.on) acc.add((cur.f0 + cur.f1) + (cur.f2 + cur.f3), -2 * cur.lev, sum, abs_sum);
        cur = nxt;
    }
    acc.flush(sum, abs_sum);
    __shared__ Fix192 sh[8][2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const Fix192 a = fix_shfl_down(sum, o);
        const Fix192 b = fix_shfl_down(abs_sum, o);
        fix_add(sum, a);
        fix_add(abs_sum, b);
    }
    if (lane == 0) {
        sh[wid][0] = sum;
        sh[wid][1] = abs_sum;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        // m < 4: sum of field m (warps 2m, 2m + 1); m >= 4: its absolute sum
        const int m = threadIdx.x, f = m & 3, j = m >> 2;
        Fix192 a = sh[2 * f][j];
        fix_add(a, sh[2 * f + 1][j]);
        for (int i = 0; i < 3; i++) part[(size_t)blockIdx.x * 24 + 3 * m + i] = a.w[i];
    }
    // the last CTA to finish adds up every CTA's partials and resets the ticket
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    audit_finish(part, gridDim.x, out);
    if (threadIdx.x == 0) *ticket = 0u;
}

// Totals of an audited persistent launch: out[m] = the correctly rounded sum
// of quantity m over the *nblk reduction blocks' partials (24 words each);
// then closes the launch's audit gate (*gate = 0).  One CTA of 1024
// threads: warp w adds up quantity w % 8 over every fourth run of 32
// blocks, and the four warps of a quantity are combined at the end.
__global__ void __launch_bounds__(1024) audit_blocks_kernel(const unsigned long long* __restrict__ part,
                                                            const int* __restrict__ nblk, double* __restrict__ out,
                                                            int* gate) {
    __shared__ Fix192 red[4][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, m = w & 7, j = w >> 3;
    const int nb = *nblk;
    Fix192 a = fix_zero();
    for (int i = j * 32 + lane; i < nb; i += 128) {
        Fix192 v;
        for (int q = 0; q < 3; q++) v.w[q] = part[(size_t)i * 24 + 3 * m + q];
        fix_add(a, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const Fix192 b = fix_shfl_down(a, o);
        fix_add(a, b);
    }
    if (lane == 0) red[j][m] = a;
    __syncthreads();
    if (threadIdx.x < 8) {
        Fix192 t = red[0][threadIdx.x];
        for (int q = 1; q < 4; q++) fix_add(t, red[q][threadIdx.x]);
        out[threadIdx.x] = fix_to_double(t);
    }
    if (threadIdx.x == 0) *gate = 0;
}

// ---------------------------------------------------------------------------
// adaptive refinement (Sec. 3.4)
// ---------------------------------------------------------------------------

__device__ __forceinline__ const double* composite_src(const LevelDev& L, uint32_t fl) {
    // active cells: state buffer; covered cells: the average of their
    // children, kept in the other buffer by avgdown_kernel
    const int sb = state_buf(L);
    return ((fl & (F_IN | F_COV)) == (F_IN | F_COV)) ? L.buf[sb ^ 1] : L.buf[sb];
}

// Average-down (Eq. 25) of every covered cell of level C from its children
// on level F: ((c00 + c11) + (c10 + c01)) / 4, into C's scratch buffer.
__global__ void avgdown_kernel(LevelDev C, LevelDev F, const Item* __restrict__ items, int nitems,
                               const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6, cx = threadIdx.x & 7, cy = (threadIdx.x >> 3) & 7;
    // work item: (tile, field) -- the four populations of one field
    for (int wi = blockIdx.x * TILES_PER_CTA + sub; wi < 4 * nitems; wi += gridDim.x * TILES_PER_CTA) {
        const Item w = items[wi >> 2];
        const int k = wi & 3;
        const int x = w.tx * TILE + cx, y = w.ty * TILE + cy;
        if (x >= C.nx || y >= C.ny) continue;
        const long long c = (long long)y * C.pitch + x;
        if ((C.flags[c] & (F_IN | F_COV)) != (F_IN | F_COV)) continue;
        double* out = C.buf[state_buf(C) ^ 1];
        const long long k00 = (long long)(2 * y) * F.pitch + 2 * x;
        const long long k10 = k00 + 1, k01 = k00 + F.pitch, k11 = k01 + 1;
        const double* p00 = composite_src(F, F.flags[k00]);
        const double* p10 = composite_src(F, F.flags[k10]);
        const double* p01 = composite_src(F, F.flags[k01]);
        const double* p11 = composite_src(F, F.flags[k11]);
        for (int q = 4 * k; q < 4 * k + 4; q++)
            out[qoff(q, C.plane, c)] = ((p00[qoff(q, F.plane, k00)] + p11[qoff(q, F.plane, k11)]) +
                                        (p10[qoff(q, F.plane, k10)] + p01[qoff(q, F.plane, k01)])) * 0.25;
    }
}

// Flags every block (8 x 8 cells) holding a cell within `buffer` cells
// (square neighbourhood) of tagged cell (x, y): cells beyond a periodic side
// wrap, beyond another side they do not exist.  Several threads may flag one
// block; they all store 1.
__device__ __forceinline__ void flag_blocks_near(int x, int y, int nx, int ny, int px, int py, int buffer, int bxn,
                                                 uint8_t* __restrict__ out) {
    for (int ya = y - buffer; ya <= y + buffer;) {
        int yy = ya;
        if (yy < 0 || yy >= ny) {
            if (!py) {
                ya = yy < 0 ? 0 : y + buffer + 1;
                continue;
            }
            yy = ((yy % ny) + ny) % ny;
        }
        const int jb = yy / TILE;
        for (int xa = x - buffer; xa <= x + buffer;) {
            int xx = xa;
            if (xx < 0 || xx >= nx) {
                if (!px) {
                    xa = xx < 0 ? 0 : x + buffer + 1;
                    continue;
                }
                xx = ((xx % nx) + nx) % nx;
            }
            const int ib = xx / TILE;
            out[(long long)jb * bxn + ib] = 1;
            xa += min((ib + 1) * TILE, nx) - xx;  // on to the next block
        }
        ya += min((jb + 1) * TILE, ny) - yy;
    }
}

// The composite moments W_0 .. W_{NK-1} of the 10 x 10 window around tile
// w (the tile and a one-cell ring; sides wrap where periodic) into Ws[k],
// with on = 1 where the cell is on the level: thread lt of the tile's group
// stages its own cell and, for lt < 36, one cell of the ring.  Whether a
// cell is on the level, and covered (its composite value then sits in the
// scratch buffer), is read from the block maps bin / bcov (one byte per
// 8 x 8 block, cached) rather than from the cell flags, so the population
// loads do not wait for a flag load.
constexpr int WIN = TILE + 2;
template <int NK>
__device__ __forceinline__ void stage_window(const LevelDev& L, const uint8_t* __restrict__ bin,
                                             const uint8_t* __restrict__ bcov, const Item& w, int lt,
                                             double (*Ws)[WIN * WIN], uint8_t* on) {
    const int bx = (L.nx + TILE - 1) / TILE;
    const int sb = state_buf(L);
    for (int pass = 0; pass < 2; pass++) {
        int hx, hy;
        if (pass == 0) {
            hx = (lt & 7) + 1;
            hy = (lt >> 3) + 1;
        } else {
            if (lt >= 4 * (TILE + 1)) break;
            if (lt < WIN) { hx = lt; hy = 0; }
            else if (lt < 2 * WIN) { hx = lt - WIN; hy = WIN - 1; }
            else if (lt < 2 * WIN + TILE) { hx = 0; hy = lt - 2 * WIN + 1; }
            else { hx = WIN - 1; hy = lt - 2 * WIN - TILE + 1; }
        }
        int x = w.tx * TILE + hx - 1, y = w.ty * TILE + hy - 1;
        bool ok = true;
        if (x < 0) { if (L.px) x += L.nx; else ok = false; }
        if (x >= L.nx) { if (L.px) x -= L.nx; else ok = false; }
        if (y < 0) { if (L.py) y += L.ny; else ok = false; }
        if (y >= L.ny) { if (L.py) y -= L.ny; else ok = false; }
        ok = ok && x >= 0 && x < L.nx && y >= 0 && y < L.ny;  // cells past a narrow domain's side
        uint8_t in = 0;
        if (ok) {
            const long long b = (long long)(y / TILE) * bx + x / TILE;
            if (bin[b]) {
                in = 1;
                const long long c = (long long)y * L.pitch + x;
                const double* src = L.buf[bcov[b] ? sb ^ 1 : sb];
                for (int k = 0; k < NK; k++)
                    Ws[k][hy * WIN + hx] = (src[qoff(0 + k, L.plane, c)] + src[qoff(4 + k, L.plane, c)]) +
                                           (src[qoff(8 + k, L.plane, c)] + src[qoff(12 + k, L.plane, c)]);
            }
        }
        on[hy * WIN + hx] = in;
    }
}

// Binary exponent of |x| from its bits (biased: 0 for zero and subnormals,
// 2047 for infinities and NaN).
__device__ __forceinline__ int bexp(double x) {
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFull);
}

// Whether d1^2 + d2^2 > tol2 (2 rc)^2 is false by the exponents alone: with
// |d| < 2^(Ed + 1) for the larger difference and tol2 >= 2^Et, rc >= 2^Ec,
// the left side is below 2^(2 Ed + 3) and the right side at least
// 2^(Et + 2 Ec + 2); when 2 Ed + 3 <= Et + 2 Ec + 1 the left side is below
// half the right side, far outside the few ulps by which the rounded
// products and sum can move either side, so the rounded comparison is false
// too.  Only for moderate exponents (|Ed|, |Ec|, |Et| <= 200 unbiased, or a
// zero or subnormal difference), where no product under- or overflows;
// otherwise the full test decides.  et: the unbiased exponent of tol2, or a
// value below -200 to disable.
__device__ __forceinline__ bool tag_below_by_exponents(double d1, double d2, double rc, int et) {
    const int ec = bexp(rc) - 1023, ed = max(bexp(d1), bexp(d2)) - 1023;
    if (et < -200 || et > 200 || ec < -200 || ec > 200 || ed > 200) return false;
    return 2 * ed + 3 <= et + 2 * ec + 1;
}

// Normalised density-gradient indicator: tag when
// (rho_E - rho_W)^2 + (rho_N - rho_S)^2 > tol^2 (2 rho_C)^2; neighbours off
// the level or beyond a non-periodic side take rho_C.  A tagged cell flags
// the blocks within `buffer` cells of it in bflag (zeroed beforehand).
// Cells whose differences are far below the threshold are settled by their
// exponents (tag_below_by_exponents); the rest by the test as written.
__global__ void __launch_bounds__(CTA_THREADS, 6)
tag_kernel(LevelDev L, BlockMaps M, const Item* __restrict__ items, int nitems, double tol2, int buffer,
           uint8_t* __restrict__ bflag, const int* __restrict__ ncount) {
    __shared__ double sW[TILES_PER_CTA][1][WIN * WIN];
    __shared__ uint8_t son[TILES_PER_CTA][WIN * WIN];
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63, cx = lt & 7, cy = lt >> 3;
    // the exponent of tol2 for the shortcut (normal tol2 only)
    const int et = (bexp(tol2) == 0 || bexp(tol2) == 2047 || !(tol2 > 0.0)) ? -1000 : bexp(tol2) - 1023;
    for (int it = blockIdx.x * TILES_PER_CTA + sub; it < nitems; it += gridDim.x * TILES_PER_CTA) {
        const Item w = items[it];
        group_bar(sub);  // the group's previous window is read
        stage_window<1>(L, M.bin, M.bcov, w, lt, sW[sub], son[sub]);
        group_bar(sub);
        const int x = w.tx * TILE + cx, y = w.ty * TILE + cy;
        const int hc = (cy + 1) * WIN + cx + 1;
        if (x >= L.nx || y >= L.ny || !son[sub][hc]) continue;
        const double rc = sW[sub][0][hc];
        const int nb[4] = {hc + 1, hc - 1, hc + WIN, hc - WIN};  // E, W, N, S
        double rn[4];
        for (int d = 0; d < 4; d++) rn[d] = son[sub][nb[d]] ? sW[sub][0][nb[d]] : rc;
        const double d1 = rn[0] - rn[1];
        const double d2 = rn[2] - rn[3];
        if (tag_below_by_exponents(d1, d2, rc, et)) continue;
        const double num = d1 * d1 + d2 * d2;
        const double t = 2.0 * rc;
        if (num > tol2 * (t * t)) flag_blocks_near(x, y, L.nx, L.ny, L.px, L.py, buffer, (L.nx + TILE - 1) / TILE, bflag);
    }
}

// Moments of the composite state at cell c.
__device__ __forceinline__ void comp_W(const LevelDev& L, long long c, double W[4]) {
    const double* s = composite_src(L, L.flags[c]);
    for (int k = 0; k < 4; k++)
        W[k] = (s[qoff(0 + k, L.plane, c)] + s[qoff(4 + k, L.plane, c)]) +
               (s[qoff(8 + k, L.plane, c)] + s[qoff(12 + k, L.plane, c)]);
}

// Flux-jump sensor of Sec. 3.4, Eq. amr-sigma, first pass: the maxima
// qmax_k = max |Q_{alpha,k}| over the composite cells of the listed tiles,
// merged into qmax[k] as bit patterns (non-negative binary64 values order
// like their bits).
__global__ void qmax_kernel(LevelDev L, const Item* __restrict__ items, int nitems,
                            unsigned long long* __restrict__ qmax, const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6, cx = threadIdx.x & 7, cy = (threadIdx.x >> 3) & 7;
    unsigned long long m[4] = {0ull, 0ull, 0ull, 0ull};
    for (int it = blockIdx.x * TILES_PER_CTA + sub; it < nitems; it += gridDim.x * TILES_PER_CTA) {
        const Item w = items[it];
        const int x = w.tx * TILE + cx, y = w.ty * TILE + cy;
        if (x >= L.nx || y >= L.ny) continue;
        const long long c = (long long)y * L.pitch + x;
        if (!(L.flags[c] & F_IN)) continue;
        double W[4], Qx[4], Qy[4], p;
        comp_W(L, c, W);
        euler_flux(L.gm1, W, Qx, Qy, p);
        for (int k = 0; k < 4; k++) {
            const unsigned long long a = (unsigned long long)__double_as_longlong(fabs(Qx[k]));
            const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(Qy[k]));
            m[k] = max(m[k], max(a, b));
        }
    }
    for (int k = 0; k < 4; k++) {
        unsigned long long v = m[k];
        for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, off));
        if ((threadIdx.x & 31) == 0 && v) atomicMax(qmax + k, v);
    }
}

// Second pass: a cell is tagged when s = max_k |s_k| > tol with
// s_k = dx (div Q)_k / qmax_k, i.e. when |g_k| > (2 tol) qmax_k for some k,
// g_k = (Qx_k(E) - Qx_k(W)) + (Qy_k(N) - Qy_k(S)) (central differences;
// neighbours off the level or beyond a non-periodic side take the cell's
// own flux).  A tagged cell flags the blocks within `buffer` cells of it.
__global__ void __launch_bounds__(CTA_THREADS, 4)
tag_flux_kernel(LevelDev L, BlockMaps M, const Item* __restrict__ items, int nitems,
                const unsigned long long* __restrict__ qmax, double tol, int buffer, uint8_t* __restrict__ bflag,
                const int* __restrict__ ncount) {
    __shared__ double sW[TILES_PER_CTA][4][WIN * WIN];
    __shared__ uint8_t son[TILES_PER_CTA][WIN * WIN];
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63, cx = lt & 7, cy = lt >> 3;
    for (int it = blockIdx.x * TILES_PER_CTA + sub; it < nitems; it += gridDim.x * TILES_PER_CTA) {
        const Item w = items[it];
        group_bar(sub);  // the group's previous window is read
        stage_window<4>(L, M.bin, M.bcov, w, lt, sW[sub], son[sub]);
        group_bar(sub);
        const int x = w.tx * TILE + cx, y = w.ty * TILE + cy;
        const int hc = (cy + 1) * WIN + cx + 1;
        if (x >= L.nx || y >= L.ny || !son[sub][hc]) continue;
        double W[4], Qcx[4], Qcy[4], p;
        for (int k = 0; k < 4; k++) W[k] = sW[sub][k][hc];
        euler_flux(L.gm1, W, Qcx, Qcy, p);
        const int nb[4] = {hc + 1, hc - 1, hc + WIN, hc - WIN};  // E, W, N, S
        double Qx[4][4], Qy[4][4];
        for (int d = 0; d < 4; d++) {
            if (son[sub][nb[d]]) {
                double Wn[4];
                for (int k = 0; k < 4; k++) Wn[k] = sW[sub][k][nb[d]];
                euler_flux(L.gm1, Wn, Qx[d], Qy[d], p);
            } else {
                for (int k = 0; k < 4; k++) {
                    Qx[d][k] = Qcx[k];
                    Qy[d][k] = Qcy[k];
                }
            }
        }
        bool t = false;
        for (int k = 0; k < 4; k++) {
            const double g = (Qx[0][k] - Qx[1][k]) + (Qy[2][k] - Qy[3][k]);
            const double lim = (2.0 * tol) * __longlong_as_double((long long)qmax[k]);
            t = t || fabs(g) > lim;
        }
        if (t) flag_blocks_near(x, y, L.nx, L.ny, L.px, L.py, buffer, (L.nx + TILE - 1) / TILE, bflag);
    }
}

__global__ void merge_kernel(LevelDev L, const Item* __restrict__ items, int nitems, const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6, cx = threadIdx.x & 7, cy = (threadIdx.x >> 3) & 7;
    // work item: (tile, field) -- the four populations of one field
    for (int wi = blockIdx.x * TILES_PER_CTA + sub; wi < 4 * nitems; wi += gridDim.x * TILES_PER_CTA) {
        const Item w = items[wi >> 2];
        const int k = wi & 3;
        const int x = w.tx * TILE + cx, y = w.ty * TILE + cy;
        if (x >= L.nx || y >= L.ny) continue;
        const long long c = (long long)y * L.pitch + x;
        const int sb = state_buf(L);
        for (int q = 4 * k; q < 4 * k + 4; q++) L.buf[sb][qoff(q, L.plane, c)] = L.buf[sb ^ 1][qoff(q, L.plane, c)];
    }
}

// Cells entering refinement are split (Eqs. 26-27): per population,
// sigma_x = minmod(f - f_W, f_E - f), sigma_y likewise, child (a, b) =
// f + (sigma_x xi_a + sigma_y xi_b), xi = -1/4, +1/4.  Neighbours that were
// covered before the regrid contribute their children's average; beyond a
// non-periodic side the slope is zero.  Uses the layout from before the
// regrid (flags are rebuilt afterwards).
__global__ void split_kernel(LevelDev C, LevelDev F, const Item* __restrict__ items, int nitems,
                             const int* __restrict__ ncount) {
    if (ncount) nitems = *ncount;
    const int sub = threadIdx.x >> 6, cx = threadIdx.x & 7, cy = (threadIdx.x >> 3) & 7;
    // work item: (tile, field) -- the four populations of one field
    for (int wi = blockIdx.x * TILES_PER_CTA + sub; wi < 4 * nitems; wi += gridDim.x * TILES_PER_CTA) {
        const Item w = items[wi >> 2];
        const int k = wi & 3;
        const int x = w.tx * TILE + cx, y = w.ty * TILE + cy;
        if (x >= C.nx || y >= C.ny) continue;
        const long long c = (long long)y * C.pitch + x;
        long long nb[4];
        bool ok[4];
        for (int d = 0; d < 4; d++) {
            int xx = x + kCX[d], yy = y + kCY[d];
            ok[d] = true;
            if (xx < 0) { if (C.px) xx += C.nx; else ok[d] = false; }
            if (xx >= C.nx) { if (C.px) xx -= C.nx; else ok[d] = false; }
            if (yy < 0) { if (C.py) yy += C.ny; else ok[d] = false; }
            if (yy >= C.ny) { if (C.py) yy -= C.ny; else ok[d] = false; }
            nb[d] = ok[d] ? (long long)yy * C.pitch + xx : c;
        }
        const double* st = C.buf[state_buf(C)];
        const double* nsrc[4];
        for (int d = 0; d < 4; d++) nsrc[d] = ok[d] ? composite_src(C, C.flags[nb[d]]) : st;
        double* fo = F.buf[state_buf(F)];
        const long long k00 = (long long)(2 * y) * F.pitch + 2 * x;
        for (int q = 4 * k; q < 4 * k + 4; q++) {
            const double fc = st[qoff(q, C.plane, c)];
            const double vE = nsrc[0][qoff(q, C.plane, nb[0])], vW = nsrc[1][qoff(q, C.plane, nb[1])];
            const double vN = nsrc[2][qoff(q, C.plane, nb[2])], vS = nsrc[3][qoff(q, C.plane, nb[3])];
            const double sx = (ok[0] && ok[1]) ? minmod(fc - vW, vE - fc) : 0.0;
            const double sy = (ok[2] && ok[3]) ? minmod(fc - vS, vN - fc) : 0.0;
            fo[qoff(q, F.plane, k00)] = fc + (sx * -0.25 + sy * -0.25);
            fo[qoff(q, F.plane, k00 + 1)] = fc + (sx * 0.25 + sy * -0.25);
            fo[qoff(q, F.plane, k00 + F.pitch)] = fc + (sx * -0.25 + sy * 0.25);
            fo[qoff(q, F.plane, k00 + F.pitch + 1)] = fc + (sx * 0.25 + sy * 0.25);
        }
    }
}

// Per-cell flags of a level from its block maps (blk_in, blk_cov: one byte
// per 8 x 8 block).  Faces that exist now but did not exist under the old
// flags have no previous sample.
template <class Lv>
__device__ __forceinline__ uint16_t cell_flags(const Lv& L, int x, int y, long long t, int bx,
                                               const uint8_t* __restrict__ blk_in,
                                               const uint8_t* __restrict__ blk_cov,
                                               const uint16_t* __restrict__ oldf) {
    if (x >= L.nx) return 0;
    const long long b = (long long)(y / TILE) * bx + x / TILE;
    const bool in = blk_in[b], cov = in && blk_cov[b];
    uint32_t fl = (in ? F_IN : 0u) | (cov ? F_COV : 0u);
    if (in && !cov) {
        const uint32_t ofl = oldf[t];
        const bool oact = (ofl & (F_IN | F_COV)) == F_IN;
        for (int i = 0; i < 4; i++) {
            // upwind neighbour of direction i (the one that feeds it)
            int ux = x - kCX[i], uy = y - kCY[i];
            bool inside = true;
            if (ux < 0) { if (L.px) ux += L.nx; else inside = false; }
            if (ux >= L.nx) { if (L.px) ux -= L.nx; else inside = false; }
            if (uy < 0) { if (L.py) uy += L.ny; else inside = false; }
            if (uy >= L.ny) { if (L.py) uy -= L.ny; else inside = false; }
            if (!inside) { fl |= F_BND; continue; }
            const long long ub = (long long)(uy / TILE) * bx + ux / TILE;
            const bool uin = blk_in[ub], ucov = uin && blk_cov[ub];
            if (!uin) fl |= 1u << (F_RECON_SHIFT + i);
            else if (ucov) {
                fl |= 1u << (F_PEND_SHIFT + i);
                // face (x, d) with d = i ^ 1 points at the covered cell u
                const int d = i ^ 1;
                const long long uc = (long long)uy * L.pitch + ux;
                const bool existed = oact && ((oldf[uc] & (F_IN | F_COV)) == (F_IN | F_COV));
                const bool was_fresh = (ofl >> (F_FRESH_SHIFT + d)) & 1u;
                if (!existed || was_fresh) fl |= 1u << (F_FRESH_SHIFT + d);
            }
        }
    }
    return (uint16_t)fl;
}

__global__ void flags_kernel(LevelDev L, const uint8_t* __restrict__ blk_in, const uint8_t* __restrict__ blk_cov,
                             const uint16_t* __restrict__ oldf, uint16_t* __restrict__ newf) {
    const int bx = (L.nx + TILE - 1) / TILE;
    const long long n = (long long)L.pitch * L.ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(t % L.pitch), y = (int)(t / L.pitch);
        newf[t] = cell_flags(L, x, y, t, bx, blk_in, blk_cov, oldf);
    }
}

// The same for the listed blocks of every level (those on the level before
// or after a change of layout; length at *nc), into newf; copy = 1 then
// copies those blocks of newf back into oldf.  Every other block is off the
// level on both sides: its flags are zero and stay zero.
__global__ void flags_blocks_kernel(FlagsSet F, int copy) {
    const int sub = threadIdx.x >> 6, cx = threadIdx.x & 7, cy = (threadIdx.x >> 3) & 7;
    for (int l = 0; l < F.nl; l++) {
        const FlagsSet::Geom& L = F.g[l];
        const int bx = (L.nx + TILE - 1) / TILE;
        const int n = *F.nc[l];
        const Item* __restrict__ items = F.items[l];
        uint16_t* __restrict__ oldf = F.oldf[l];
        uint16_t* __restrict__ newf = F.newf[l];
        for (int it = blockIdx.x * TILES_PER_CTA + sub; it < n; it += gridDim.x * TILES_PER_CTA) {
            const Item w = items[it];
            const int x = w.tx * TILE + cx, y = w.ty * TILE + cy;
            if (y >= L.ny) continue;
            const long long t = (long long)y * L.pitch + x;
            if (copy) oldf[t] = newf[t];
            else newf[t] = cell_flags(L, x, y, t, bx, F.bin[l], F.bcov[l], oldf);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static inline int tile_grid(int nitems, int max_ctas) {
    int g = (nitems + TILES_PER_CTA - 1) / TILES_PER_CTA;
    if (max_ctas > 0 && g > max_ctas) g = max_ctas;
    return g < 1 ? 1 : g;
}

// CTAs of CTA_THREADS threads of kernel fn that the device holds at once.
static int resident_ctas(const void* fn) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto f = cache.find(fn);
    if (f != cache.end()) return f->second;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, CTA_THREADS, 0);
    const int r = std::max(1, sms * std::max(1, per));
    cache[fn] = r;
    return r;
}

// Grid of a launch of `kernel` over a tile list: n tiles, or -- when the
// list's length lives in device memory (nc != nullptr) -- one wave of the
// CTAs the device holds at once, looping over at most n tiles.
template <class K>
static inline int list_grid(K* kernel, int n, const int* nc, int max_ctas = 0) {
    int g = tile_grid(n, max_ctas);
    if (nc) g = std::min(g, resident_ctas((const void*)kernel));
    return g;
}

static inline int flat_grid(long long n) {
    long long g = (n + 255) / 256;
    if (g > 148LL * 16) g = 148LL * 16;
    return (int)(g < 1 ? 1 : g);
}

// Sweep variants: (launch shape, minimum resident CTAs per SM): whole
// 8 x 8 tiles per group of 64 threads at 2, 3 or 4 CTAs per SM, or (the
// persistent kernel only) half tiles per warp at 3 or 2.
#define VLBM_SWEEP_VARIANTS(X) X(0, 0, 2) X(1, 0, 3) X(2, 0, 4) X(3, TK_HALF, 3) X(4, TK_HALF, 2)

int sweep_variants() { return 5; }

cudaError_t launch_sensor(const LevelDev* levs, const Item* items, int n, int kk, cudaStream_t s, const int* nc) {
    if (n <= 0) return cudaSuccess;
    sensor_prep_kernel<<<list_grid(sensor_prep_kernel, n, nc), CTA_THREADS, 0, s>>>(levs, items, n, kk, nc);
    sensor_rate_kernel<<<list_grid(sensor_rate_kernel, n, nc), CTA_THREADS, 0, s>>>(levs, items, n, nc);
    return cudaGetLastError();
}

cudaError_t launch_sweep(const LevelDev* levs, const Item* items, int n, int kk, int kkp, int max_ctas, int variant,
                         cudaStream_t s, bool sensor, const int* nc) {
    if (n <= 0) return cudaSuccess;
    if (sensor) {  // per-cell relaxation parameters: one form of the sweep
        sweep_kernel<SW_SENSOR, 2><<<list_grid(sweep_kernel<SW_SENSOR, 2>, n, nc, max_ctas), CTA_THREADS, 0, s>>>(
            levs, items, n, kk, kkp, nc);
        return cudaGetLastError();
    }
    switch (variant) {
#define X(id, P, B)                                                                                       \
    case id:                                                                                              \
        sweep_kernel<P, B><<<list_grid(sweep_kernel<P, B>, n, nc, max_ctas), CTA_THREADS, 0, s>>>(levs, items, n, kk, \
                                                                                                 kkp, nc); \
        break;
        VLBM_SWEEP_VARIANTS(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Resident CTAs per SM of one task-kernel variant (sets its shared-memory
// attributes first), and its launch.
template <int P, int B>
int task_variant_per_sm() {
    int per = 0;
    if constexpr ((P & TK_HALF) != 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, task_kernel_half<P, B>, CTA_THREADS, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, task_kernel<P, B>, CTA_THREADS, 0);
    }
    return per;
}

template <int P, int B>
void task_variant_launch(int g, const LevelDev* levs, const Segment* segs, const int* prefix, const int2* chunks,
                         int* ctl, int iters, cudaStream_t s) {
    if constexpr ((P & TK_HALF) != 0)
        task_kernel_half<P, B><<<g, CTA_THREADS, 0, s>>>(levs, segs, prefix, chunks, ctl, iters);
    else
        task_kernel<P, B><<<g, CTA_THREADS, 0, s>>>(levs, segs, prefix, chunks, ctl, iters);
}

int task_kernel_ctas(int variant) {
    static int cache[16] = {0};
    if (variant < 0 || variant >= 16) return 0;
    if (cache[variant]) return cache[variant];
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    switch (variant) {
#define X(id, P, B) case id: per = task_variant_per_sm<P, B>(); break;
        VLBM_SWEEP_VARIANTS(X)
#undef X
    }
    cache[variant] = sms * (per > 0 ? per : 1);
    return cache[variant];
}

cudaError_t launch_tasks(const LevelDev* levs, const Segment* segs, const int* prefix, const int2* chunks, int* ctl,
                         int variant, int ctas, int iters, cudaStream_t s, bool sensor) {
    if (iters < 1) return cudaErrorInvalidValue;
    if (sensor) {
        // lists with the relaxation sensor's passes: the variant's launch
        // shape, in the kernel form that runs them
        static int full_s[16] = {0};
        if (variant < 0 || variant >= 16) return cudaErrorInvalidValue;
        if (!full_s[variant]) {
            int dev = 0, sms = 0, per = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            switch (variant) {
#define X(id, P, B) case id: per = task_variant_per_sm<(P) | SW_SENSOR, B>(); break;
                VLBM_SWEEP_VARIANTS(X)
#undef X
                default: return cudaErrorInvalidValue;
            }
            full_s[variant] = sms * std::max(1, per);
        }
        const int gs = ctas > 0 ? std::min(ctas, full_s[variant]) : full_s[variant];
        switch (variant) {
#define X(id, P, B) case id: task_variant_launch<(P) | SW_SENSOR, B>(gs, levs, segs, prefix, chunks, ctl, iters, s); break;
            VLBM_SWEEP_VARIANTS(X)
#undef X
        }
        return cudaGetLastError();
    }
    const int full = task_kernel_ctas(variant);  // also sets the kernel's shared-memory attributes
    const int g = ctas > 0 ? std::min(ctas, full) : full;
    switch (variant) {
#define X(id, P, B) case id: task_variant_launch<P, B>(g, levs, segs, prefix, chunks, ctl, iters, s); break;
        VLBM_SWEEP_VARIANTS(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_audit_blocks(const unsigned long long* part, const int* nblk, double* out, int* gate,
                                cudaStream_t s) {
    audit_blocks_kernel<<<1, 1024, 0, s>>>(part, nblk, out, gate);
    return cudaGetLastError();
}

cudaError_t launch_audit_segments(const unsigned long long* slots, const int* seg, int nseg, double* out,
                                  cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    audit_segments_kernel<<<nseg, 256, 0, s>>>(slots, seg, 0, out);
    return cudaGetLastError();
}


cudaError_t launch_close(const LevelDev* levs, const Item* items, int n, int kk, cudaStream_t s, const int* nc) {
    if (n <= 0) return cudaSuccess;
    close_kernel<<<list_grid(close_kernel, n, nc), CTA_THREADS, 0, s>>>(levs, items, n, kk, nc);
    return cudaGetLastError();
}

cudaError_t launch_end_step(int* const* par, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    end_step_kernel<<<(n + 127) / 128, 128, 0, s>>>(par, n);
    return cudaGetLastError();
}

cudaError_t launch_feq_init(const LevelDev& L, const double* W, long long ld, double hc, cudaStream_t s) {
    feq_init_kernel<<<flat_grid((long long)L.nx * L.ny), 256, 0, s>>>(L, W, ld, hc);
    return cudaGetLastError();
}

cudaError_t launch_copy_pop(const LevelDev& L, double* ext, long long ld, int to_ext, cudaStream_t s) {
    copy_pop_kernel<<<flat_grid((long long)L.nx * L.ny), 256, 0, s>>>(L, ext, ld, to_ext);
    return cudaGetLastError();
}

cudaError_t launch_gather_W(const LevelDev& L, double* W, long long ld, uint8_t* valid, cudaStream_t s) {
    gather_W_kernel<<<flat_grid((long long)L.nx * L.ny), 256, 0, s>>>(L, W, ld, valid);
    return cudaGetLastError();
}

// One wave: the CTAs that fit on the device at once loop over the tiles.
int audit_blocks(int nitems) {
    static int resident = 0;
    if (!resident) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, audit_kernel, 256, 0);
        resident = std::max(1, sms * std::max(1, per));
    }
    return std::max(1, std::min(nitems, resident));  // a CTA per tile at a time
}

cudaError_t launch_audit(const LevelDev* levs, const Item* items, int n, unsigned long long* part, double* out,
                         unsigned* ticket, cudaStream_t s, const int* nc) {
    const int g = audit_blocks(n);
    audit_kernel<<<g, 256, 0, s>>>(levs, items, n, part, out, ticket, nc);
    return cudaGetLastError();
}

cudaError_t launch_avgdown(const LevelDev& C, const LevelDev& F, const Item* items, int n, cudaStream_t s,
                           const int* nc) {
    if (n <= 0) return cudaSuccess;
    avgdown_kernel<<<list_grid(avgdown_kernel, 4 * n, nc), CTA_THREADS, 0, s>>>(C, F, items, n, nc);
    return cudaGetLastError();
}

cudaError_t launch_tag(const LevelDev& L, const BlockMaps& M, const Item* items, int n, double tol2, int buffer,
                       uint8_t* bflag, cudaStream_t s, const int* nc) {
    if (n <= 0) return cudaSuccess;
    tag_kernel<<<list_grid(tag_kernel, n, nc), CTA_THREADS, 0, s>>>(L, M, items, n, tol2, buffer, bflag, nc);
    return cudaGetLastError();
}

cudaError_t launch_qmax(const LevelDev& L, const Item* items, int n, unsigned long long* qmax, cudaStream_t s,
                        const int* nc) {
    if (n <= 0) return cudaSuccess;
    qmax_kernel<<<list_grid(qmax_kernel, n, nc), CTA_THREADS, 0, s>>>(L, items, n, qmax, nc);
    return cudaGetLastError();
}

cudaError_t launch_tag_flux(const LevelDev& L, const BlockMaps& M, const Item* items, int n,
                            const unsigned long long* qmax, double tol, int buffer, uint8_t* bflag, cudaStream_t s,
                            const int* nc) {
    if (n <= 0) return cudaSuccess;
    tag_flux_kernel<<<list_grid(tag_flux_kernel, n, nc), CTA_THREADS, 0, s>>>(L, M, items, n, qmax, tol, buffer, bflag,
                                                                            nc);
    return cudaGetLastError();
}

cudaError_t launch_merge(const LevelDev& L, const Item* items, int n, cudaStream_t s, const int* nc) {
    if (n <= 0) return cudaSuccess;
    merge_kernel<<<list_grid(merge_kernel, 4 * n, nc), CTA_THREADS, 0, s>>>(L, items, n, nc);
    return cudaGetLastError();
}

cudaError_t launch_split(const LevelDev& C, const LevelDev& F, const Item* items, int n, cudaStream_t s,
                         const int* nc) {
    if (n <= 0) return cudaSuccess;
    split_kernel<<<list_grid(split_kernel, 4 * n, nc), CTA_THREADS, 0, s>>>(C, F, items, n, nc);
    return cudaGetLastError();
}

cudaError_t launch_flags(const LevelDev& L, const uint8_t* blk_in, const uint8_t* blk_cov, const uint16_t* oldf,
                         uint16_t* newf, cudaStream_t s) {
    flags_kernel<<<flat_grid((long long)L.pitch * L.ny), 256, 0, s>>>(L, blk_in, blk_cov, oldf, newf);
    return cudaGetLastError();
}

cudaError_t launch_flags_update(const FlagsSet& F, int cap, cudaStream_t s) {
    const int g = list_grid(flags_blocks_kernel, cap, F.nc[0]);
    flags_blocks_kernel<<<g, CTA_THREADS, 0, s>>>(F, 0);
    flags_blocks_kernel<<<g, CTA_THREADS, 0, s>>>(F, 1);
    return cudaGetLastError();
}

}  // namespace vlbm
