// Device-side data model of the VLBM library (sm_103a).
//
// Storage: every level l of a hierarchy owns two dense population buffers
// over its whole index space, population q = 4 i + k (direction i in
// +x,-x,+y,-y; field k in rho, rho u, rho v, rho E) of cell y * pitch + x at
// qoff(q, plane, cell) (pairs of fields interleaved), plus a 16-bit flag
// word per cell.  Work is organised in 8 x 8 tiles that coincide
// with the refinement blocks, so a tile is entirely active, entirely covered
// by the next level, or entirely off the level.
//
// Streaming is "push": the thread of cell x writes its post-collision
// population f*_i into the destination buffer at x + c_i, whatever lies
// there.  Two facts of the refinement coupling fall out of that for free:
//   * a coarse ring cell L0 pushes f*_d(L0) into the covered cell C = L0 + c_d
//     of its own level, so after a coarse step dst[C] holds the current
//     sample of Eq. 20 and src[C] the previous one (the buffers ping-pong);
//   * a fine edge cell R0 pushes its outgoing f* into the fine-level cell that
//     lies inside the coarse cell L0; the two fine sub-steps of a cycle write
//     the two buffers, so the four values averaged by Eq. 24 are there when
//     the cycle closes.
// No face tables, ghost copies or register arrays are needed.
#pragma once
#include <cstdint>
#ifdef __CUDACC__
#include <vector_types.h>
#else
struct int2 {
    int x, y;
};
#endif

namespace vlbm {

constexpr int NQ = 16;
constexpr int TILE = 8;          // tile edge = refinement block edge (cells)
constexpr int TILES_PER_CTA = 4; // 4 x 64 threads
constexpr int AUDIT_SLOT = 4 * 64; // doubles per audit slot: W_k of a tile's cells, [k][cell]
constexpr int CTA_THREADS = TILES_PER_CTA * TILE * TILE;

// per-cell flag bits
enum : uint32_t {
    F_IN = 1u << 0,         // cell belongs to the level
    F_COV = 1u << 1,        // cell is covered by the next finer level
    F_RECON_SHIFT = 2,      // bits 2..5: upwind of direction i is coarser land
    F_PEND_SHIFT = 6,       // bits 6..9: upwind of direction i is covered
    F_FRESH_SHIFT = 10,     // bits 10..13: face (cell, d) has no previous sample
    F_BND = 1u << 14,       // an upwind neighbour lies beyond a non-periodic side
};
constexpr uint32_t F_RECON_MASK = 0xFu << F_RECON_SHIFT;
constexpr uint32_t F_PEND_MASK = 0xFu << F_PEND_SHIFT;
constexpr uint32_t F_FRESH_MASK = 0xFu << F_FRESH_SHIFT;

// status bits of a hierarchy
// ST_NESTING: a layout computed on the device is not properly nested;
// ST_TASKCAP: a task list built on the device did not fit its buffers
enum : int { ST_NONPHYS = 1, ST_TIMEOUT = 2, ST_NESTING = 4, ST_TASKCAP = 8 };

enum : int { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW = 2, BC_REFLECT = 3 };

// One level of one hierarchy, as the kernels see it.
struct LevelDev {
    double* buf[2];
    uint16_t* flags;
    int* par0;        // level-0 buffer parity of the hierarchy (device word)
    int* status;      // status word of the hierarchy (device)
    long long plane;  // pitch * ny
    int nx, ny, pitch, level;
    int parent;       // index of the parent level in the table, -1 on level 0
    int child;        // index of the child level in the table, -1 on the finest
    int px, py;       // periodic in x / y
    int bc[4];        // W, E, S, N
    double om, hb, bcs, gm1;
    double wscale;    // area weight 4^-level
    double feqb[4][16];
    // sensor-driven relaxation (sens == nullptr: constant beta): planes of
    // sens: 0-3 Qx, 4-7 Qy, 8 u, 9 v, 12-15 W (from the pre-collision state
    // of the level step), 10 s, 11 theta; plane stride `plane`.  rc = 1 / c
    // (rounded to nearest).
    double* sens;
    double beta_max, beta_min, csens, eps, ninth, c, rc, iq[4];
};
constexpr int SENS_PLANES = 16;

#ifdef __CUDACC__
#define VLBM_HD __host__ __device__
#else
#define VLBM_HD
#endif

// Offset of population q = 4 i + k of cell c in a level buffer: the planes
// of fields (0, 1) and of fields (2, 3) of each direction are interleaved,
// [q / 2][cell][q % 2], so one 16-byte access moves a pair of them (same
// direction, same destination cell).  16 * plane doubles in all.
VLBM_HD inline long long qoff(int q, long long plane, long long c) {
    return (long long)(q >> 1) * (2 * plane) + 2 * c + (q & 1);
}

// A unit of work: one 8 x 8 tile of one level.
struct Item {
    int lid;
    unsigned short tx, ty;
};

// A task of the persistent kernel: one tile of one phase (kind 0 = level
// sweep, kind 1 = reflux close) of one coarse step, or (kind 2) the exact
// sums of one field (kk) over one block of audit slots; its dependencies are
// deps[dep0 .. dep0 + ndep), indices of earlier tasks.
struct Task {
    int lid;
    unsigned short tx, ty;
    signed char kind, kk, kkp, step;
    int dep0, ndep;
    int aslot;  // kind 0: the slot of its moments when audited, else -1; kind 2: the audit block
};

// One hierarchy's task list as the persistent kernel sees it.  Task level
// indices and dependency indices are local to the segment; lid_base maps
// the level indices into the batch's level table.  done[] holds the launch
// epoch in which each task completed (never cleared between launches).
struct Segment {
    const Task* tasks;
    const int* deps;
    unsigned* done;
    double* aw;                  // audited moments, AUDIT_SLOT per slot (nullptr: no audit)
    const int2* arng;            // slot range of each audit block
    const int* ascale;           // weight exponent of each slot
    unsigned long long* apart;   // exact sums of each audit block, 24 words
    int* par0;                   // the hierarchy's level-0 parity word
    int ntasks, lid_base;
};

// control words of a persistent launch
// Control words of a persistent launch: ticket and finish counters, launch
// epoch, tasks per iteration, segments (hierarchies), flip of the level-0
// parity after an odd number of one-step iterations, and chunks -- runs of
// consecutive tickets that are consecutive tasks of one segment.
enum : int {
    CTL_CLAIM = 0,
    CTL_FIN = 1,
    CTL_EPOCH = 2,
    CTL_TOTAL = 3,
    CTL_NSEG = 4,
    CTL_FLIP = 5,
    CTL_NCHUNK = 6,
    // nonzero: the launch's first iteration is audited -- its first sweep
    // of each level keeps the moments, and the CTL_NAUD reduction tasks
    // stored after the list's CTL_TOTAL tasks add them up, once, after the
    // last iteration's tickets; zero: neither
    CTL_AUDIT = 7,
    CTL_NAUD = 8,
    CTL_WORDS = 16
};

}  // namespace vlbm
