// Device-resident layouts and task lists (see vlbm_amr.h).
#include <cuda_runtime.h>

#include <cstdint>

#include "vlbm_amr.h"

namespace vlbm {

namespace {

// ---------------------------------------------------------------------------
// CTA-wide prefix sums
// ---------------------------------------------------------------------------

__device__ __forceinline__ int warp_incl(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one value per thread over the CTA (blockDim.x a
// multiple of 32, at most 1024); returns the thread's offset, *total the
// CTA's sum.
__device__ int cta_excl(int v, int* sm, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const int inc = warp_incl(v);
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
        int x = lane < nw ? sm[lane] : 0;
        x = warp_incl(x);
        if (lane < nw) sm[lane] = x;
    }
    __syncthreads();
    const int base = w ? sm[w - 1] : 0;
    *total = sm[nw - 1];
    __syncthreads();
    return base + inc - v;
}

// ---------------------------------------------------------------------------
// layout rule, derived maps, nesting
// ---------------------------------------------------------------------------

__device__ __forceinline__ int wrap_or(int v, int n, int per, bool& ok) {
    if (v < 0 || v >= n) {
        if (!per) {
            ok = false;
            return 0;
        }
        v = ((v % n) + n) % n;
    }
    return v;
}

// Whether the one-cell-widened extent of child block ib (child level of n
// cells, periodic or not) holds a cell whose parent cell lies in parent block
// pb: the cells 8 ib - 1 .. min(n, 8 ib + 8), wrapped or dropped at the
// sides, parent cell x >> 1, its block (x >> 1) / 8.
__device__ bool widened_touches(int ib, int n, int per, int pb) {
    const int x0 = ib * TILE - 1, x1 = min(n, ib * TILE + TILE) + 1;
    for (int x = x0; x < x1; x++) {
        int xx = x;
        if (xx < 0 || xx >= n) {
            if (!per) continue;
            xx = (xx + n) % n;
        }
        if (((xx >> 1) / TILE) == pb) return true;
    }
    return false;
}

__global__ void layout_rule_kernel(LayoutDev L, LayoutDev F, int has_f, const uint8_t* __restrict__ bflag) {
    const long long nb = (long long)L.bx * L.by;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
        const int ib = (int)(b % L.bx), jb = (int)(b / L.bx);
        uint8_t cov = bflag[b] ? 1 : 0;
        if (has_f && !cov) {
            // candidate child blocks: a window around the children of this
            // block, wrapped on periodic sides (duplicates do not matter)
            for (int dj = -3; dj <= 4 && !cov; dj++) {
                bool oky = true;
                const int cj = wrap_or(2 * jb + dj, F.by, F.py, oky);
                if (!oky) continue;
                if (!widened_touches(cj, F.ny, F.py, jb)) continue;
                for (int di = -3; di <= 4; di++) {
                    bool okx = true;
                    const int ci = wrap_or(2 * ib + di, F.bx, F.px, okx);
                    if (!okx) continue;
                    if (!F.ncov[(long long)cj * F.bx + ci]) continue;
                    if (widened_touches(ci, F.nx, F.px, ib)) {
                        cov = 1;
                        break;
                    }
                }
            }
        }
        L.ncov[b] = cov;
    }
}

// The level of flat block index b of a set and the block's index on it.
__device__ __forceinline__ int set_level(const LayoutSet& S, long long& b) {
    int l = 0;
    while (l + 1 < S.nl && b >= S.b0[l + 1]) l++;
    b -= S.b0[l];
    return l;
}

// New on-level maps of every level of the set: level 0 holds every block; a
// block of level l >= 1 is on it when its parent is on level l - 1 and
// covered there, i.e. when every ancestor's block is covered in the new maps.
__global__ void derive_in_kernel(LayoutSet S) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < S.b0[S.nl];
         g += (long long)gridDim.x * blockDim.x) {
        long long b = g;
        const int l = set_level(S, b);
        const LayoutDev& L = S.L[l];
        int ib = (int)(b % L.bx), jb = (int)(b / L.bx);
        bool in = true;
        for (int q = l - 1; q >= 0 && in; q--) {
            ib >>= 1;
            jb >>= 1;
            in = S.L[q].ncov[(long long)jb * S.L[q].bx + ib] != 0;
        }
        L.nin[b] = in ? 1 : 0;
    }
}

__global__ void nest_check_kernel(LayoutSet S, int* status) {
    bool bad = false;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < S.b0[S.nl];
         g += (long long)gridDim.x * blockDim.x) {
        long long b = g;
        const int l = set_level(S, b);
        const LayoutDev& L = S.L[l];
        if (!L.ncov[b]) continue;
        if (l == S.nl - 1 || !L.nin[b]) {
            bad = true;
            continue;
        }
        if (L.level == 0) continue;
        const int ib = (int)(b % L.bx), jb = (int)(b / L.bx);
        const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
        for (int d = 0; d < 4; d++) {
            bool ok = true;
            const int i2 = wrap_or(ib + di[d], L.bx, L.px, ok), j2 = wrap_or(jb + dj[d], L.by, L.py, ok);
            if (ok && !L.nin[(long long)j2 * L.bx + i2]) bad = true;
        }
    }
    if (bad) atomicOr(status, ST_NESTING);
}

__global__ void commit_maps_kernel(LayoutSet S) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < S.b0[S.nl];
         g += (long long)gridDim.x * blockDim.x) {
        long long b = g;
        const LayoutDev& L = S.L[set_level(S, b)];
        L.bin[b] = L.nin[b];
        L.bcov[b] = L.ncov[b];
    }
}

// ---------------------------------------------------------------------------
// tile lists by compaction (row-major block order)
// ---------------------------------------------------------------------------

constexpr int LIST_T = 256, LIST_E = LAY_CHUNK / LIST_T;

struct Member {
    uint8_t bits;   // 1 << LST_*
    uint8_t recon;  // active with a face neighbour off the level
};

// Whether block b changes its on-level or covered state with the new maps.
__device__ __forceinline__ bool block_changed(const LayoutDev& L, long long b) {
    const bool in = L.bin[b] != 0, nin = L.nin[b] != 0;
    return in != nin || (in && L.bcov[b] != 0) != (nin && L.ncov[b] != 0);
}

__device__ __forceinline__ Member member(const LayoutDev& L, long long b) {
    Member m{0, 0};
    const int ib = (int)(b % L.bx), jb = (int)(b / L.bx);
    const bool in = L.bin[b] != 0, covb = L.bcov[b] != 0;
    const bool cov = in && covb, act = in && !covb;
    if (in) m.bits |= 1u << LST_IN;
    if (cov) m.bits |= 1u << LST_COV;
    if (act) {
        m.bits |= 1u << LST_ACT;
        bool ring = false, rec = false;
        const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
        for (int d = 0; d < 4; d++) {
            bool ok = true;
            const int i2 = wrap_or(ib + di[d], L.bx, L.px, ok), j2 = wrap_or(jb + dj[d], L.by, L.py, ok);
            if (!ok) continue;
            const long long b2 = (long long)j2 * L.bx + i2;
            ring = ring || (L.bin[b2] && L.bcov[b2]);
            rec = rec || !L.bin[b2];
        }
        if (ring) m.bits |= 1u << LST_RING;
        m.recon = rec;
    }
    if (L.nin && L.ncov) {
        const bool ncov = L.nin[b] && L.ncov[b];
        if (cov && !ncov) m.bits |= 1u << LST_EXIT;
        if (ncov && !cov) m.bits |= 1u << LST_ENTER;
        // a cell's flags depend on its own block and its face-neighbour
        // blocks (the upwind cell of a face may lie in either): they change
        // only where one of those changes its on-level or covered state
        if (in || L.nin[b]) {
            bool ch = block_changed(L, b);
            const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
            for (int d = 0; d < 4 && !ch; d++) {
                bool ok = true;
                const int i2 = wrap_or(ib + di[d], L.bx, L.px, ok), j2 = wrap_or(jb + dj[d], L.by, L.py, ok);
                if (ok) ch = block_changed(L, (long long)j2 * L.bx + i2);
            }
            if (ch) m.bits |= 1u << LST_TOUCH;
        }
    }
    return m;
}

// The level of the set's chunk (CTA) c and the chunk's index on it.
__device__ __forceinline__ int chunk_level(const LayoutSet& S, int& c) {
    int l = 0;
    while (l + 1 < S.nl && c >= S.c0[l + 1]) l++;
    c -= S.c0[l];
    return l;
}

__global__ void lists_count_kernel(LayoutSet S) {
    __shared__ int sm[32];
    int c = blockIdx.x;
    const int l = chunk_level(S, c);
    const LayoutDev& L = S.L[l];
    const int mask = S.mask[l];
    const long long nb = (long long)L.bx * L.by;
    int n[NLST] = {};
    for (int e = 0; e < LIST_E; e++) {
        const long long b = (long long)c * LAY_CHUNK + threadIdx.x * LIST_E + e;
        if (b >= nb) break;
        const Member m = member(L, b);
        for (int k = 0; k < NLST; k++) n[k] += (m.bits & mask) >> k & 1;
    }
    for (int k = 0; k < NLST; k++) {
        if (!(mask >> k & 1)) continue;
        int tot;
        cta_excl(n[k], sm, &tot);
        if (threadIdx.x == 0) L.chunk[k * L.nchunk + c] = tot;
    }
}

// one CTA per (level, list): exclusive chunk offsets, the list length, and
// (act) the reset of the active cell count
__global__ void lists_scan_kernel(LayoutSet S) {
    __shared__ int sm[32];
    const int l = blockIdx.x / NLST, k = blockIdx.x % NLST;
    const LayoutDev& L = S.L[l];
    if (!(S.mask[l] >> k & 1)) return;
    int carry = 0;
    for (int b = 0; b < L.nchunk; b += blockDim.x) {
        const int i = b + threadIdx.x;
        const int v = i < L.nchunk ? L.chunk[k * L.nchunk + i] : 0;
        int tot;
        const int off = cta_excl(v, sm, &tot);
        if (i < L.nchunk) L.chunk[k * L.nchunk + i] = carry + off;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        L.cnt[k] = carry;
        if (k == LST_ACT) *L.cells = 0ull;
    }
}

__global__ void lists_scatter_kernel(LayoutSet S) {
    __shared__ int sm[32];
    int c = blockIdx.x;
    const int lid = chunk_level(S, c);
    const LayoutDev& L = S.L[lid];
    const int mask = S.mask[lid];
    const long long nb = (long long)L.bx * L.by;
    Member m[LIST_E];
    int n[NLST] = {};
    for (int e = 0; e < LIST_E; e++) {
        const long long b = (long long)c * LAY_CHUNK + threadIdx.x * LIST_E + e;
        m[e] = b < nb ? member(L, b) : Member{0, 0};
        for (int k = 0; k < NLST; k++) n[k] += (m[e].bits & mask) >> k & 1;
    }
    int off[NLST];
    for (int k = 0; k < NLST; k++) {
        off[k] = 0;
        if (!(mask >> k & 1)) continue;
        int tot;
        off[k] = L.chunk[k * L.nchunk + c] + cta_excl(n[k], sm, &tot);
    }
    const bool maps = (mask >> LST_ACT) & 1;
    unsigned long long cells = 0;
    for (int e = 0; e < LIST_E; e++) {
        const long long b = (long long)c * LAY_CHUNK + threadIdx.x * LIST_E + e;
        if (b >= nb) break;
        const int ib = (int)(b % L.bx), jb = (int)(b / L.bx);
        const Item it{L.level, (unsigned short)ib, (unsigned short)jb};
        const uint8_t bits = m[e].bits & mask;
        for (int k = 0; k < NLST; k++)
            if (bits >> k & 1) L.list[k][off[k]++] = it;
        if (maps) {
            const bool act = bits >> LST_ACT & 1;
            L.act_idx[b] = act ? off[LST_ACT] - 1 : -1;
            L.ring_idx[b] = (bits >> LST_RING & 1) ? off[LST_RING] - 1 : -1;
            L.recon[b] = m[e].recon;
            if (act)
                cells += (unsigned long long)(min(L.nx, ib * TILE + TILE) - ib * TILE) *
                         (unsigned long long)(min(L.ny, jb * TILE + TILE) - jb * TILE);
        }
    }
    if (maps) {
        for (int o = 16; o > 0; o >>= 1) cells += __shfl_down_sync(0xffffffffu, cells, o);
        if ((threadIdx.x & 31) == 0 && cells) atomicAdd(L.cells, cells);
    }
}

// parent tiles under the reconstruction footprint of child tile (tx, ty):
// the parent cells 4 t - 1 .. 4 t + 4 on each axis, wrapped or dropped
__device__ int foot_keys(const LayoutDev& P, int tx, int ty, int* keys) {
    int ns = 0;
    for (int cy2 = ty * TILE / 2 - 1; cy2 <= ty * TILE / 2 + TILE / 2; cy2++)
        for (int cx2 = tx * TILE / 2 - 1; cx2 <= tx * TILE / 2 + TILE / 2; cx2++) {
            bool ok = true;
            const int xx = wrap_or(cx2, P.nx, P.px, ok), yy = wrap_or(cy2, P.ny, P.py, ok);
            if (!ok) continue;
            const int key = (yy / TILE) * P.bx + xx / TILE;
            bool dup = false;
            for (int q = 0; q < ns; q++) dup = dup || keys[q] == key;
            if (dup || ns == 16) continue;
            keys[ns++] = key;
        }
    return ns;
}

// Reverse footprints of every refinable level of the set: for each
// reconstructing tile i of level l >= 1 and each tile of level l - 1 under
// its footprint, i joins that tile's entries (counts past FOOT_CAP are kept,
// and the readers take at most FOOT_CAP of them).
__global__ void footprints_kernel(LayoutSet S, int* status) {
    int off[9];  // S.nl <= 8
    off[0] = off[1] = 0;
    for (int l = 1; l < S.nl; l++) off[l + 1] = off[l] + S.L[l].cnt[LST_ACT];
    bool ovf = false;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < off[S.nl]; g += gridDim.x * blockDim.x) {
        int l = 1;
        while (g >= off[l + 1]) l++;
        const LayoutDev& C = S.L[l];
        const LayoutDev& P = S.L[l - 1];
        const int i = g - off[l];
        const Item it = C.list[LST_ACT][i];
        if (!C.recon[(long long)it.ty * C.bx + it.tx]) continue;
        int keys[16];
        const int nk = foot_keys(P, it.tx, it.ty, keys);
        for (int q = 0; q < nk; q++) {
            const int slot = atomicAdd(P.fcnt + keys[q], 1);
            if (slot < FOOT_CAP) P.fidx[(long long)keys[q] * FOOT_CAP + slot] = i;
            else ovf = true;
        }
    }
    if (ovf) atomicOr(status, ST_TASKCAP);
}

struct ActRef {
    const Item* list[4];
    const int* cnt[4];
    int cap[4];
};

__global__ void concat_act_kernel(ActRef R, int nl, Item* __restrict__ out, int* __restrict__ n_out) {
    int off[5];
    off[0] = 0;
    for (int l = 0; l < nl; l++) off[l + 1] = off[l] + R.cnt[l][LST_ACT];
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = off[nl];
    for (int l = 0; l < nl; l++) {
        const int n = R.cnt[l][LST_ACT];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            Item it = R.list[l][i];
            it.lid = l;
            out[off[l] + i] = it;
        }
    }
}

__global__ void count_lups_kernel(const unsigned long long* c0, const unsigned long long* c1,
                                  const unsigned long long* c2, const unsigned long long* c3, int nl, long long steps,
                                  unsigned long long* counter) {
    const unsigned long long* c[4] = {c0, c1, c2, c3};
    unsigned long long s = 0;
    for (int l = 0; l < nl; l++) s += *c[l] << l;
    *counter += s * (unsigned long long)steps;
}

static inline int flat_blocks(long long n) {
    long long g = (n + 255) / 256;
    if (g > 148LL * 16) g = 148LL * 16;
    return (int)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------------------
// task lists (the device form of build_tasks in vlbm_tasks.h)
// ---------------------------------------------------------------------------

// Dependencies per task: up to TB_SMALL in the task's fixed slot, more in
// the overflow area.  The work is chains of table lookups (latency bound),
// so a warp walks one task's accesses in parallel (tb_warp_kernel).
// Adversarial layouts (most cells refined, checkerboard coverage) reached
// 98 distinct dependencies; the fallback pass holds TB_MAXDEP, beyond which
// the build raises ST_TASKCAP (reported as VLBM_ERR_OOM).
constexpr int TB_SMALL = TASK_DEP_SLOT;
constexpr int TB_MAXDEP = 256;
constexpr int TB_BUILD_THREADS = 128;
__constant__ int kSDI[5] = {0, 1, -1, 0, 0};
__constant__ int kSDJ[5] = {0, 0, 0, 1, -1};

__device__ __forceinline__ int src_of(int level, int kk, int step) { return level == 0 ? (step & 1) : (kk == 1 ? 0 : 1); }

// A task's dependency set for the fallback pass (in local memory): at most
// `cap` distinct task indices, entry i at v[i * stride].
struct DepSet {
    int* v;      // entry i at v[i * stride]
    int stride;
    int cap;
    int n;
    bool ovf;
    __device__ void store(int* out) const {
        for (int i = 0; i < n; i++) out[i] = at(i);
    }
    __device__ void add(int q) {
        for (int i = 0; i < n; i++)
            if (v[i * stride] == q) return;
        if (n < cap) v[(n++) * stride] = q;
        else ovf = true;
    }
    __device__ int at(int i) const { return v[i * stride]; }
    __device__ void put(int i, int q) { v[i * stride] = q; }
    // ascending, like the host builder
    __device__ void sort() {
        for (int a = 1; a < n; a++) {
            const int x = at(a);
            int b = a - 1;
            while (b >= 0 && at(b) > x) {
                put(b + 1, at(b));
                b--;
            }
            put(b + 1, x);
        }
    }
};

// parent tiles read by the reconstruction of fine tile (tx, ty): the coarse
// tiles under the coarse cells [4 t - 1, 4 t + 4] in each direction
__device__ int footprint(const TBLevel& P, int tx, int ty, int* keys) {
    int ns = 0;
    const int c0x = tx * TILE / 2 - 1, c1x = tx * TILE / 2 + TILE / 2;
    const int c0y = ty * TILE / 2 - 1, c1y = ty * TILE / 2 + TILE / 2;
    for (int cy2 = c0y; cy2 <= c1y; cy2++)
        for (int cx2 = c0x; cx2 <= c1x; cx2++) {
            bool ok = true;
            const int xx = wrap_or(cx2, P.nx, P.px, ok), yy = wrap_or(cy2, P.ny, P.py, ok);
            if (!ok) continue;
            const int key = (yy / TILE) * P.bx + xx / TILE;
            bool dup = false;
            for (int q = 0; q < ns; q++) dup = dup || keys[q] == key;
            if (dup || ns == 16) continue;
            keys[ns++] = key;
        }
    return ns;
}

// The builder's view of a plan: the static tables (phases, accesses,
// offsets) read from shared memory, everything else from the plan.
struct TB {
    const TBPlan& P;
    const TBPhase* ph;
    const TBAcc* acc;
    const int* acc_beg;
    const int* acc_pos;
    const int* off;
    __device__ explicit TB(const TBPlan& p) : P(p) {}

    template <class F>
    __device__ void touching(const TBAcc& a, int l, int tx, int ty, F&& emit) const {
        const int base = off[a.phase];
        switch (a.pat) {
            case TB_OWN: {
                const int i = P.lev[l].act_idx[ty * P.lev[l].bx + tx];
                if (i >= 0) emit(base + i);
                break;
            }
            case TB_STENCIL: {
                const TBLevel& V = P.lev[l];
                for (int d = 0; d < 5; d++) {
                    bool ok = true;
                    const int sx = wrap_or(tx - kSDI[d], V.bx, V.px, ok), sy = wrap_or(ty - kSDJ[d], V.by, V.py, ok);
                    if (!ok) continue;
                    bool ok2 = true;
                    const int rx = wrap_or(sx + kSDI[d], V.bx, V.px, ok2), ry = wrap_or(sy + kSDJ[d], V.by, V.py, ok2);
                    if (!ok2 || rx != tx || ry != ty) continue;
                    const int i = V.act_idx[sy * V.bx + sx];
                    if (i >= 0) emit(base + i);
                }
                break;
            }
            case TB_FOOT: {  // reconstructing tiles of level l + 1 whose footprint holds (tx, ty)
                const TBLevel& Pl = P.lev[l];
                const int key = ty * Pl.bx + tx;
                const int n = min(Pl.fcnt[key], FOOT_CAP);
                for (int j = 0; j < n; j++) emit(base + Pl.fidx[key * FOOT_CAP + j]);
                break;
            }
            case TB_CHILD4: {
                const TBLevel& Pl = P.lev[l - 1];
                const int i = Pl.ring_idx[(ty / 2) * Pl.bx + tx / 2];
                if (i >= 0) emit(base + i);
                break;
            }
            case TB_OWNRING: {
                const int i = P.lev[l].ring_idx[ty * P.lev[l].bx + tx];
                if (i >= 0) emit(base + i);
                break;
            }
            case TB_BOX9: {
                const TBLevel& V = P.lev[l];
                for (int d = 0; d < 9; d++) {
                    const int dx = d % 3 - 1, dy = d / 3 - 1;
                    bool ok = true;
                    const int sx = wrap_or(tx - dx, V.bx, V.px, ok), sy = wrap_or(ty - dy, V.by, V.py, ok);
                    if (!ok) continue;
                    const int i = V.act_idx[sy * V.bx + sx];
                    if (i >= 0) emit(base + i);
                }
                break;
            }
        }
    }

    // bit 0: some sweep of level l pushes into the tile (an active tile among
    // it and its four face neighbours, by the push targets); bit 1: a close
    // writes it (a ring tile of a refinable level)
    __device__ int wmask(int l, int tx, int ty) const {
        const TBLevel& V = P.lev[l];
        int m = 0;
        for (int d = 0; d < 5 && !m; d++) {
            bool ok = true;
            const int sx = wrap_or(tx - kSDI[d], V.bx, V.px, ok), sy = wrap_or(ty - kSDJ[d], V.by, V.py, ok);
            if (!ok) continue;
            bool ok2 = true;
            const int rx = wrap_or(sx + kSDI[d], V.bx, V.px, ok2), ry = wrap_or(sy + kSDJ[d], V.by, V.py, ok2);
            if (!ok2 || rx != tx || ry != ty) continue;
            if (V.act_idx[sy * V.bx + sx] >= 0) m = 1;
        }
        if (l + 1 < P.nlev && V.ring_idx[ty * V.bx + tx] >= 0) m |= 2;
        return m;
    }

    // The tasks that the access (write or read, level l, resource kind, tile
    // (tx, ty)) of phase p depends on, each passed to emit (possibly more
    // than once): a read waits for the last earlier writer of the tile; a
    // write waits for every reader since that writer, or for the writer
    // itself when there was none.  A cyclic list's walk goes on through the
    // whole previous iteration (entries ~q): every tile a step reads or
    // writes is written within one step, so the walk ends there.  Level 0
    // alternates its buffers from step to step, so there its buffer kinds
    // swap across the wrap.
    template <class Emit>
    __device__ __forceinline__ void deps_of(int p, bool write, int l, int kind, int tx, int ty, Emit&& emit) const {
        if (!write && kind < 3) {
            const int m = wmask(l, tx, ty);
            if (kind == 2 ? !(m & 2) : !m) return;
        }
        bool readers = false;
        for (int pass = 0; pass < 1 + P.cyclic; pass++) {
            const int rc = l * TB_NRES + (pass && l == 0 && kind < 2 ? kind ^ 1 : kind);
            const int a0 = acc_beg[rc];
            const int e0 = pass ? acc_beg[rc + 1] : acc_pos[rc * (P.nphase + 1) + p];
            for (int e = e0 - 1; e >= a0; e--) {
                const TBAcc a = acc[e];
                if (a.write) {
                    bool any = false;
                    touching(a, l, tx, ty, [&](int q) {
                        any = true;
                        if (!readers) emit(pass ? ~q : q);
                    });
                    if (any) return;
                } else if (write) {
                    touching(a, l, tx, ty, [&](int q) {
                        readers = true;
                        emit(pass ? ~q : q);
                    });
                }
            }
        }
    }

    // Access q (0 <= q < nq) of a task of phase ph on tile it: false when
    // the access falls off a non-periodic side or outside the finer level.
    // Sweeps: q = 0 reads the tile's source buffer, q = 1..5 write the
    // destination buffer of the tile and its four neighbours (push), a
    // reconstructing tile reads both buffers and the flags of each of its nk
    // coarse footprint tiles (q = 6 + 3 k + r), and with the sensor the
    // sweep reads its tile's first-pass planes (q = 6 + 3 nk) and the
    // second-pass planes of the 3 x 3 tiles around it; closes: q = 0..7 read
    // the two buffers of the four child tiles, q = 8, 9 write the tile's
    // destination buffer and flags; the sensor's first pass reads the
    // source buffer and writes its planes (q = 0, 1), its second pass reads
    // the first-pass planes of the tile and its four neighbours and writes
    // its own planes (q = 0..4, 5).
    __device__ __forceinline__ bool query(const TBPhase& ph, const Item& it, const int* keys, int nk, int q,
                                          bool& write, int& l, int& kind, int& tx, int& ty) const {
        l = ph.l;
        if (ph.kind == 3 || ph.kind == 4 || (ph.kind == 0 && q >= 6 + 3 * nk)) {
            const TBLevel& L = P.lev[l];
            int dx = 0, dy = 0;
            if (ph.kind == 3) {
                write = q == 1;
                kind = q == 0 ? src_of(l, ph.kk, ph.step) : 3;
            } else if (ph.kind == 4) {
                write = q == 5;
                kind = q == 5 ? 4 : 3;
                if (q < 5) dx = kSDI[q], dy = kSDJ[q];
            } else {
                const int j = q - (6 + 3 * nk);
                write = false;
                kind = j == 0 ? 3 : 4;
                if (j > 0) dx = (j - 1) % 3 - 1, dy = (j - 1) / 3 - 1;
            }
            bool ok = true;
            tx = wrap_or(it.tx + dx, L.bx, L.px, ok);
            ty = wrap_or(it.ty + dy, L.by, L.py, ok);
            return ok;
        }
        if (ph.kind == 0) {
            const int bs = src_of(l, ph.kk, ph.step);
            if (q == 0) {
                write = false;
                kind = bs;
                tx = it.tx;
                ty = it.ty;
                return true;
            }
            if (q <= 5) {
                const TBLevel& L = P.lev[l];
                bool ok = true;
                tx = wrap_or(it.tx + kSDI[q - 1], L.bx, L.px, ok);
                ty = wrap_or(it.ty + kSDJ[q - 1], L.by, L.py, ok);
                write = true;
                kind = bs ^ 1;
                return ok;
            }
            const int k = (q - 6) / 3, r = (q - 6) % 3;
            const int pbs = src_of(l - 1, ph.kkp, ph.step);
            const int bx = P.lev[l - 1].bx;
            l -= 1;
            write = false;
            kind = r == 0 ? pbs : (r == 1 ? pbs ^ 1 : 2);
            tx = keys[k] % bx;
            ty = keys[k] / bx;
            return true;
        }
        if (q < 8) {
            const TBLevel& C = P.lev[l + 1];
            const int c = q >> 1;
            tx = 2 * it.tx + (c & 1);
            ty = 2 * it.ty + (c >> 1);
            l += 1;
            write = false;
            kind = q & 1;
            return tx < C.bx && ty < C.by;
        }
        write = true;
        kind = q == 8 ? (src_of(l, ph.kk, ph.step) ^ 1) : 2;
        tx = it.tx;
        ty = it.ty;
        return true;
    }

    // the dependencies of task t of phase p into the set S (the fallback
    // pass: one thread per task)
    template <class Set>
    __device__ __forceinline__ void deps(int p, int t, Set& S, Item& it) const {
        const TBPhase ph = this->ph[p];
        const int l = ph.l;
        const TBLevel& L = P.lev[l];
        const int i = t - off[p];
        it = ph.kind == 1 ? L.ring[i] : L.act[i];
        S.n = 0;
        S.ovf = false;
        int keys[16];
        const int nk = (ph.kind == 0 && l > 0 && L.recon[it.ty * L.bx + it.tx]) ? footprint(P.lev[l - 1], it.tx, it.ty, keys) : 0;
        const int nq = num_queries(ph, nk);
        for (int q = 0; q < nq; q++) {
            bool wr;
            int ql, qk, qx, qy;
            if (query(ph, it, keys, nk, q, wr, ql, qk, qx, qy)) deps_of(p, wr, ql, qk, qx, qy, [&](int d) { S.add(d); });
        }
    }

    // accesses of a task of phase ph with nk footprint tiles
    __device__ __forceinline__ int num_queries(const TBPhase& ph, int nk) const {
        switch (ph.kind) {
            case 0: return 6 + 3 * nk + (P.sensor ? 10 : 0);
            case 1: return 10;
            case 3: return 2;
            case 4: return 6;
            default: return 0;
        }
    }

    __device__ int phase_of(int t) const {
        int lo = 0, hi = P.nphase - 1;  // largest p with off[p] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        return lo;  // off[lo] <= t < off[lo + 1]: never an empty phase
    }
};

// Audit slot of task i of phase ph (-1: not an audited sweep): the slots of
// level l follow those of levels 0 .. l - 1.
__device__ __forceinline__ int tb_slot_base(const TBPlan& P, int l) {
    int b = 0;
    for (int q = 0; q < l; q++) b += P.lev[q].cnt[LST_ACT];
    return b;
}

__device__ __forceinline__ int tb_aslot(const TBPlan& P, const TBPhase& ph, int i) {
    return (P.audit && ph.kind == 0 && ph.first && ph.l < P.nlev) ? tb_slot_base(P, ph.l) + i : -1;
}

// Phase offsets by a scan over the phases in rounds of the CTA's threads
// (one CTA), and the build's counters reset.
__global__ void tb_offsets_kernel(TBPlan P) {
    __shared__ int sm[32];
    const int slots = P.audit ? tb_slot_base(P, P.nlev) : 0;
    const int nblk = (slots + TB_AUDIT_BLOCK - 1) / TB_AUDIT_BLOCK;
    int carry = 0;
    for (int r = 0; r < P.nphase; r += blockDim.x) {
        const int p = r + threadIdx.x;
        int c = 0;
        if (p < P.nphase) {
            const TBPhase ph = P.ph[p];
            if (ph.kind == 0 || ph.kind >= 3) c = ph.l < P.nlev ? P.lev[ph.l].cnt[LST_ACT] : 0;
            else if (ph.kind == 1) c = ph.l + 1 < P.nlev ? P.lev[ph.l].cnt[LST_RING] : 0;
            else c = 4 * nblk;
        }
        int tot;
        const int x = cta_excl(c, sm, &tot);
        if (p < P.nphase) P.off[p] = carry + x;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        P.off[P.nphase] = carry;
        P.need[0] = carry;
        P.need[1] = 0;
        P.need[2] = 0;
        P.need[3] = 0;
        P.need[4] = 0;
        P.need[5] = slots;
        P.need[6] = nblk;
        P.need[7] = 0;  // tb_big_kernel's finishing ticket
    }
}

// Reduction task t (phase p, kind 2) by one warp: block b = i / 4, field
// k = i % 4; its dependencies are the sweeps owning the block's slots
// (ascending: levels in phase order, each in list order); the field-0 task
// also writes the block's slot range and its slots' weights.
__device__ void tb_audit_task(const TBPlan& P, const int* off, int p, int t, int lane) {
    const int i = t - off[p];
    const int b = i >> 2, k = i & 3;
    const int j0 = b * TB_AUDIT_BLOCK, j1 = min(j0 + TB_AUDIT_BLOCK, P.need[5]);
    const int j = j0 + lane;
    if (j < j1) {
        int l = 0, base = 0;
        while (l + 1 < P.nlev && j >= base + P.lev[l].cnt[LST_ACT]) base += P.lev[l++].cnt[LST_ACT];
        P.deps[(long long)t * TB_SMALL + lane] = off[P.pfirst[l]] + (j - base);
        if (k == 0) P.ascale[j] = -2 * l;
    }
    if (lane == 0) {
        if (k == 0) P.arng[b] = make_int2(j0, j1);
        Task T;
        T.lid = 0;
        T.tx = 0;
        T.ty = 0;
        T.kind = 2;
        T.kk = (signed char)k;
        T.kkp = 0;
        T.step = 0;
        T.dep0 = t * TB_SMALL;
        T.ndep = j1 - j0;
        T.aslot = b;
        P.tasks[t] = T;
    }
}

// Copies the plan's static tables into shared memory; returns the view.
__device__ TB tb_global(const TBPlan& P) {
    TB tb(P);
    tb.ph = P.ph;
    tb.acc = P.acc;
    tb.acc_beg = P.acc_beg;
    tb.acc_pos = P.acc_pos;
    tb.off = P.off;
    return tb;
}


// Writes a task and its sorted dependencies (at deps[d0 ..]).
template <class Set>
__device__ __forceinline__ void tb_write(const TBPlan& P, const TB& tb, int p, int t, const Item& it, Set& S,
                                         long long d0) {
    S.sort();
    S.store(P.deps + d0);
    const TBPhase ph = tb.ph[p];
    Task T;
    T.lid = ph.l;
    T.tx = it.tx;
    T.ty = it.ty;
    T.kind = (signed char)ph.kind;
    T.kk = (signed char)ph.kk;
    T.kkp = (signed char)(ph.kind != 1 ? ph.kkp : 0);
    T.step = (signed char)ph.step;
    T.dep0 = (int)d0;
    T.ndep = S.n;
    T.aslot = tb_aslot(P, ph, t - tb.off[p]);
    P.tasks[t] = T;
}

// Ascending sort of 64 keys held two per lane (element lane in a, element
// lane + 32 in b) by a bitonic network: each 32-key half by warp shuffles,
// then one merge of the halves.
__device__ __forceinline__ void warp_bitonic32(int& v, int lane, bool ascending_last) {
    for (int k = 2; k <= 32; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool up = k == 32 ? ascending_last : ((lane & k) == 0);
            const bool lower = (lane & j) == 0;
            v = (lower == up) ? min(v, o) : max(v, o);
        }
}

__device__ __forceinline__ void warp_merge32(int& v, int lane) {
    for (int j = 16; j > 0; j >>= 1) {
        const int o = __shfl_xor_sync(0xffffffffu, v, j);
        v = ((lane & j) == 0) ? min(v, o) : max(v, o);
    }
}

__device__ __forceinline__ void warp_sort64(int& a, int& b, int lane) {
    warp_bitonic32(a, lane, true);   // ascending
    warp_bitonic32(b, lane, false);  // descending: a then b is bitonic
    const int lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
    warp_merge32(a, lane);
    warp_merge32(b, lane);
}

// Four tasks per warp: each quarter-warp walks one task's accesses in
// parallel (a sweep has six, a close ten, so eight lanes per task keep the
// warp busy) and appends what it finds (duplicates included) to the task's
// shared buffer; then the whole warp sorts each task's entries and keeps the
// distinct ones, ascending, in the task's fixed TB_SMALL slot of the
// dependency array (deps[t * TB_SMALL ..]), or in the overflow area after
// the slots when there are more.  A task whose raw entries exceed its
// buffer is left to the fallback pass.
constexpr int TBW_WARPS = 4;
constexpr int TBW_TASKS = 4;   // tasks per warp
constexpr int TBW_LANES = 32 / TBW_TASKS;
constexpr int TBW_RAW = 256;   // raw entries per task

__global__ void __launch_bounds__(TBW_WARPS * 32) tb_warp_kernel(TBPlan P) {
    __shared__ int raw[TBW_WARPS][TBW_TASKS][TBW_RAW];
    __shared__ unsigned char keep[TBW_WARPS][TBW_RAW];
    __shared__ int nraw[TBW_WARPS][TBW_TASKS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = lane / TBW_LANES, hl = lane % TBW_LANES;
    const int total = P.off[P.nphase];
    if (total > P.task_cap) return;
    const TB tb = tb_global(P);
    unsigned char* K = keep[w];
    const long long base = (long long)P.task_cap * TB_SMALL;
    for (int tp = TBW_TASKS * (blockIdx.x * TBW_WARPS + w); tp < total; tp += TBW_TASKS * gridDim.x * TBW_WARPS) {
        // the walks: lane group h on task tp + h
        {
            const int t = tp + half;
            __syncwarp();  // the previous tasks' buffers are read
            if (hl == 0) nraw[w][half] = 0;
            __syncwarp();
            const int pw = t < total ? tb.phase_of(t) : 0;
            if (t < total && tb.ph[pw].kind != 2) {
                const int p = pw;
                const TBPhase ph = tb.ph[p];
                const TBLevel& L = P.lev[ph.l];
                const int i = t - tb.off[p];
                const Item it = ph.kind == 1 ? L.ring[i] : L.act[i];
                int keys[16];
                const int nk = (ph.kind == 0 && ph.l > 0 && L.recon[it.ty * L.bx + it.tx])
                                   ? footprint(P.lev[ph.l - 1], it.tx, it.ty, keys) : 0;
                const int nq = tb.num_queries(ph, nk);
                int* R = raw[w][half];
                int* cnt = &nraw[w][half];
                for (int q = hl; q < nq; q += TBW_LANES) {
                    bool wr;
                    int ql, qk, qx, qy;
                    if (!tb.query(ph, it, keys, nk, q, wr, ql, qk, qx, qy)) continue;
                    tb.deps_of(p, wr, ql, qk, qx, qy, [&](int d) {
                        const int at = atomicAdd(cnt, 1);
                        if (at < TBW_RAW) R[at] = d;
                    });
                }
            }
            __syncwarp();
        }
        for (int u = 0; u < TBW_TASKS; u++) {
            const int t = tp + u;
            if (t >= total) break;
            const int pt = tb.phase_of(t);
            if (tb.ph[pt].kind == 2) {
                tb_audit_task(P, tb.off, pt, t, lane);
                continue;
            }
            const int* R = raw[w][u];
            const int n = nraw[w][u];
            if (n > TBW_RAW) {
                if (lane == 0) P.big[atomicAdd(P.need + 2, 1)] = t;
                continue;
            }
            // up to 64 entries: sorted in registers (two per lane), kept where
            // they differ from their predecessor; more: by ranks in shared memory
            const bool small = n <= 64;
            int va = 0x7fffffff, vb = 0x7fffffff;
            unsigned keep_a = 0u, keep_b = 0u;
            int nu = 0;
            if (small) {
                if (lane < n) va = R[lane];
                if (lane + 32 < n) vb = R[lane + 32];
                warp_sort64(va, vb, lane);
                const int pa = __shfl_up_sync(0xffffffffu, va, 1), pb = __shfl_up_sync(0xffffffffu, vb, 1);
                const int a31 = __shfl_sync(0xffffffffu, va, 31);
                keep_a = __ballot_sync(0xffffffffu, lane < n && (lane == 0 || va != pa));
                keep_b = __ballot_sync(0xffffffffu, lane + 32 < n && vb != (lane == 0 ? a31 : pb));
                nu = __popc(keep_a) + __popc(keep_b);
            } else {
                // entry j is kept when no earlier entry holds its value
                int kept = 0;
                for (int j = lane; j < n; j += 32) {
                    const int v = R[j];
                    bool first = true;
                    for (int k = 0; k < j && first; k++) first = R[k] != v;
                    K[j] = first;
                    kept += first;
                }
                nu = __reduce_add_sync(0xffffffffu, kept);
            }
            __syncwarp();
            long long at = (long long)t * TB_SMALL;
            if (nu > TB_SMALL) {
                long long a2 = 0;
                if (lane == 0) {
                    a2 = base + atomicAdd(P.need + 1, nu);
                    atomicAdd(P.need + 4, 1);
                    if (a2 + nu > P.dep_cap) {
                        atomicOr(P.need + 3, 1);
                        a2 = -1;
                    }
                }
                at = __shfl_sync(0xffffffffu, a2, 0);
            }
            if (at >= 0) {
                if (small) {
                    const unsigned below = (1u << lane) - 1u;
                    if (keep_a >> lane & 1u) P.deps[at + __popc(keep_a & below)] = va;
                    if (keep_b >> lane & 1u) P.deps[at + __popc(keep_a) + __popc(keep_b & below)] = vb;
                } else {
                    // a kept entry's place: the kept entries with smaller values
                    for (int j = lane; j < n; j += 32) {
                        if (!K[j]) continue;
                        const int v = R[j];
                        int r = 0;
                        for (int k = 0; k < n; k++) r += (K[k] && R[k] < v);
                        P.deps[at + r] = v;
                    }
                }
                if (lane == 0) {
                    const int p = pt;
                    const TBPhase ph = tb.ph[p];
                    const TBLevel& L = P.lev[ph.l];
                    const int i = t - tb.off[p];
                    const Item it = ph.kind == 1 ? L.ring[i] : L.act[i];
                    Task T;
                    T.lid = ph.l;
                    T.tx = it.tx;
                    T.ty = it.ty;
                    T.kind = (signed char)ph.kind;
                    T.kk = (signed char)ph.kk;
                    T.kkp = (signed char)(ph.kind != 1 ? ph.kkp : 0);
                    T.step = (signed char)ph.step;
                    T.dep0 = (int)at;
                    T.ndep = nu;
                    T.aslot = tb_aslot(P, ph, i);
                    P.tasks[t] = T;
                }
            }
            __syncwarp();
        }
    }
}

// The launch's counts: the list's tasks up to the audit phase (run once per
// iteration) and the audit phase's reduction tasks after them (run once, by
// an audited launch).
__device__ void tb_finish(const TBPlan& P) {
    const bool ap = P.nphase > 0 && P.ph[P.nphase - 1].kind == 2;
    int total = ap ? P.off[P.nphase - 1] : P.off[P.nphase];
    int naud = P.off[P.nphase] - total;
    if (P.need[3] != 0 || P.off[P.nphase] > P.task_cap) {
        atomicOr(P.status, ST_TASKCAP);
        total = naud = 0;
    }
    P.seg->ntasks = total;
    P.prefix[0] = 0;
    P.prefix[1] = total;
    P.ctl[CTL_TOTAL] = total;
    P.ctl[CTL_NAUD] = naud;
}

// Fallback pass: the tasks whose raw entries overflowed the warp buffer,
// one thread each with a local-memory set of up to TB_MAXDEP distinct
// dependencies, into the overflow area; the last CTA to finish writes the
// launch's counts (tb_finish).
__global__ void __launch_bounds__(TB_BUILD_THREADS) tb_big_kernel(TBPlan P) {
    const int nbig = P.need[2];
    if (nbig > 0) {
        const TB tb = tb_global(P);
        int buf[TB_MAXDEP];
        DepSet S{buf, 1, TB_MAXDEP, 0, false};
        const long long base = (long long)P.task_cap * TB_SMALL;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbig; i += gridDim.x * blockDim.x) {
            const int t = P.big[i];
            const int p = tb.phase_of(t);
            Item it;
            tb.deps(p, t, S, it);
            const long long at = base + atomicAdd(P.need + 1, S.n);
            if (S.ovf || at + S.n > P.dep_cap) {
                atomicOr(P.need + 3, 1);
                continue;
            }
            if (S.n > TB_SMALL) atomicAdd(P.need + 4, 1);
            tb_write(P, tb, p, t, it, S, at);
        }
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(P.need + 7, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        tb_finish(P);
    }
}

// The chunk table of a persistent launch over several one-step task lists
// (segments), phase-major: for each phase p, for each segment m, the run of
// m's tasks of phase p (`offs[m][p] .. offs[m][p + 1]`).  A segment whose
// build failed (its own task counts, mctl[m][CTL_TOTAL] + mctl[m][CTL_NAUD],
// are not its phase total) contributes nothing.  One CTA; entries p * nm + m in rounds of the
// CTA's threads, two scans per round (tickets and non-empty chunks).
__global__ void merge_chunks_kernel(const int* const* __restrict__ offs, const int* const* __restrict__ mctl, int nm,
                                    int nphase, int* __restrict__ prefix, int2* __restrict__ chunks, int* ctl) {
    __shared__ int sm[32];
    __shared__ int carry_t, carry_c;
    if (threadIdx.x == 0) carry_t = carry_c = 0;
    __syncthreads();
    const int ne = nphase * nm;
    for (int r = 0; r < ne; r += blockDim.x) {
        const int e = r + threadIdx.x;
        int cnt = 0, a = 0, m = 0;
        if (e < ne) {
            const int p = e / nm;
            m = e - p * nm;
            const int* o = offs[m];
            if (mctl[m][CTL_TOTAL] + mctl[m][CTL_NAUD] == o[nphase]) {
                a = o[p];
                cnt = o[p + 1] - a;
            }
        }
        int tt, tc;
        const int xt = cta_excl(cnt, sm, &tt);
        const int xc = cta_excl(cnt > 0 ? 1 : 0, sm, &tc);
        if (cnt > 0) {
            prefix[carry_c + xc] = carry_t + xt;
            chunks[carry_c + xc] = make_int2(m, a);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_t += tt;
            carry_c += tc;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        prefix[carry_c] = carry_t;
        ctl[CTL_CLAIM] = 0;
        ctl[CTL_FIN] = 0;
        ctl[CTL_TOTAL] = carry_t;
        ctl[CTL_NSEG] = nm;
        ctl[CTL_NCHUNK] = carry_c;
    }
}

}  // namespace


cudaError_t launch_layout_rule(const LayoutDev& L, const LayoutDev* F, const uint8_t* bflag, cudaStream_t s) {
    layout_rule_kernel<<<flat_blocks((long long)L.bx * L.by), 256, 0, s>>>(L, F ? *F : L, F != nullptr, bflag);
    return cudaGetLastError();
}


LayoutSet layout_set(const LayoutDev* const* levs, const int* masks, int nl) {
    LayoutSet S{};
    S.nl = nl;
    for (int l = 0; l < nl; l++) {
        S.L[l] = *levs[l];
        S.mask[l] = masks ? masks[l] : 0;
        S.c0[l + 1] = S.c0[l] + levs[l]->nchunk;
        S.b0[l + 1] = S.b0[l] + (long long)levs[l]->bx * levs[l]->by;
    }
    return S;
}

cudaError_t launch_derive_in(const LayoutDev* const* levs, int nl, cudaStream_t s) {
    const LayoutSet S = layout_set(levs, nullptr, nl);
    derive_in_kernel<<<flat_blocks(S.b0[nl]), 256, 0, s>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_nest_check(const LayoutDev* const* levs, int nl, int* status, cudaStream_t s) {
    const LayoutSet S = layout_set(levs, nullptr, nl);
    nest_check_kernel<<<flat_blocks(S.b0[nl]), 256, 0, s>>>(S, status);
    return cudaGetLastError();
}

cudaError_t launch_commit_maps(const LayoutDev* const* levs, int nl, cudaStream_t s) {
    const LayoutSet S = layout_set(levs, nullptr, nl);
    commit_maps_kernel<<<flat_blocks(S.b0[nl]), 256, 0, s>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_lists(const LayoutDev* const* levs, const int* masks, int nl, cudaStream_t s) {
    const LayoutSet S = layout_set(levs, masks, nl);
    if (S.c0[nl] <= 0) return cudaSuccess;
    lists_count_kernel<<<S.c0[nl], LIST_T, 0, s>>>(S);
    lists_scan_kernel<<<NLST * nl, 1024, 0, s>>>(S);
    lists_scatter_kernel<<<S.c0[nl], LIST_T, 0, s>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_footprints(const LayoutDev* const* levs, int nl, int* status, cudaStream_t s) {
    if (nl < 2) return cudaSuccess;
    long long nc = 0;
    for (int l = 0; l + 1 < nl; l++) {
        cudaMemsetAsync(levs[l]->fcnt, 0, (size_t)levs[l]->bx * levs[l]->by * sizeof(int), s);
        nc += (long long)levs[l + 1]->bx * levs[l + 1]->by;
    }
    const LayoutSet S = layout_set(levs, nullptr, nl);
    footprints_kernel<<<flat_blocks(nc), 256, 0, s>>>(S, status);
    return cudaGetLastError();
}

cudaError_t launch_concat_act(const LayoutDev* levs, int n, Item* out, int* n_out, cudaStream_t s) {
    ActRef R{};
    long long cap = 0;
    for (int l = 0; l < n; l++) {
        R.list[l] = levs[l].list[LST_ACT];
        R.cnt[l] = levs[l].cnt;
        R.cap[l] = levs[l].bx * levs[l].by;
        cap = cap > R.cap[l] ? cap : R.cap[l];
    }
    concat_act_kernel<<<flat_blocks(cap), 256, 0, s>>>(R, n, out, n_out);
    return cudaGetLastError();
}

cudaError_t launch_count_lups(const LayoutDev* levs, int n, long long steps, unsigned long long* counter,
                              cudaStream_t s) {
    const unsigned long long* c[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int l = 0; l < n; l++) c[l] = levs[l].cells;
    count_lups_kernel<<<1, 1, 0, s>>>(c[0], c[1], c[2], c[3], n, steps, counter);
    return cudaGetLastError();
}

cudaError_t launch_merge_chunks(const int* const* offs, const int* const* mctl, int nm, int nphase, int* prefix,
                                int2* chunks, int* ctl, cudaStream_t s) {
    merge_chunks_kernel<<<1, 1024, 0, s>>>(offs, mctl, nm, nphase, prefix, chunks, ctl);
    return cudaGetLastError();
}

cudaError_t launch_task_build(const TBPlan& P, cudaStream_t s) {
    static bool attrs = false;
    if (!attrs) {  // the fallback's sets live in local memory: the whole L1 for them
        cudaFuncSetAttribute(tb_big_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        attrs = true;
    }
    tb_offsets_kernel<<<1, 256, 0, s>>>(P);
    const long long gl = ((long long)P.task_cap + TBW_TASKS * TBW_WARPS - 1) / (TBW_TASKS * TBW_WARPS);
    const int g = (int)(gl < 1 ? 1 : (gl > 148 * 12 ? 148 * 12 : gl));
    tb_warp_kernel<<<g, TBW_WARPS * 32, 0, s>>>(P);
    tb_big_kernel<<<148, TB_BUILD_THREADS, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace vlbm
