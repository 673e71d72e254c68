// Device-resident layouts: the adaptive regrid of Sec. 3.4 (Fig. 2) and the
// persistent schedule's task lists, computed on the GPU so that a regrid
// never waits for the host.
//
// A level's layout is a pair of block maps (one byte per 8 x 8 block: on the
// level, covered by the next level) and the tile lists derived from them --
// active, ring (active with a covered face neighbour), covered, on the level,
// and during a regrid the blocks leaving and entering refinement -- with
// their lengths in device memory.  Kernels that walk a list read its length
// from device memory, so the host never needs it: a tag-driven regrid is a
// fixed sequence of launches (indicator, block flags, layout rule, merge,
// split, flags, lists, task lists) whose sizes are all decided on the GPU.
// The lists keep the row-major block order of the host's tile lists, and the
// task lists are the same, task for task and dependency for dependency, as
// the host builder's (build_tasks in vlbm_tasks.h), which a self-test checks.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "vlbm_dev.cuh"

namespace vlbm {

// lists: active, ring, covered, on the level; during a regrid the blocks
// leaving and entering refinement and those on the level before or after
// (whose per-cell flags are rebuilt)
enum : int { LST_ACT = 0, LST_RING = 1, LST_COV = 2, LST_IN = 3, LST_EXIT = 4, LST_ENTER = 5, LST_TOUCH = 6, NLST = 7 };
constexpr int LAY_CHUNK = 1024;  // blocks per compaction chunk (one CTA)
constexpr int FOOT_CAP = 32;     // reverse-footprint entries per block

// One level's device layout.  Capacities: every list and map holds bx * by
// blocks; chunk holds NLST * nchunk ints.
struct LayoutDev {
    int nx = 0, ny = 0, bx = 0, by = 0, px = 0, py = 0, level = 0;
    uint8_t *bin = nullptr, *bcov = nullptr;  // current block maps
    uint8_t *nin = nullptr, *ncov = nullptr;  // the layout being installed
    uint8_t* recon = nullptr;                 // active block with a face neighbour off the level
    int *act_idx = nullptr, *ring_idx = nullptr;  // block -> index in the act / ring list, or -1
    // refinable levels: per block, the indices in the next level's act list
    // of the reconstructing tiles whose footprint holds the block (at most
    // FOOT_CAP, fidx[b * FOOT_CAP + j], j < min(fcnt[b], FOOT_CAP))
    int* fcnt = nullptr;
    int* fidx = nullptr;
    Item* list[NLST] = {};
    int* cnt = nullptr;                       // [NLST] list lengths
    unsigned long long* cells = nullptr;      // active cells of the level
    int* chunk = nullptr;                     // compaction scratch
    int nchunk = 0;
};

// Up to eight layouts for one launch (the levels, or also the new-map views
// of the same levels): chunk (CTA) and block offsets of each in the set.
struct LayoutSet {
    LayoutDev L[8];
    int mask[8];
    int c0[9];
    long long b0[9];
    int nl;
};

// New covered map of level L (l <= nlev - 2): the flagged blocks plus the
// blocks holding the parents of the one-cell neighbourhood of the next
// level's new covered blocks (F: level l + 1 when it is refinable, else
// nullptr).  The same rule as the host's layout_rule.
cudaError_t launch_layout_rule(const LayoutDev& L, const LayoutDev* F, const uint8_t* bflag, cudaStream_t s);
// New on-level maps of levels 0 .. nl - 1 from the new covered maps (level
// 0: all blocks; level l: the blocks whose ancestors are all covered), in
// one launch.
cudaError_t launch_derive_in(const LayoutDev* const* levs, int nl, cudaStream_t s);
// Proper nesting of the new maps of every level (covered blocks on the
// level, none on the finest level -- the last of the set --, covered blocks
// of levels >= 1 with their four face neighbours on the level); a violation
// sets ST_NESTING in *status.
cudaError_t launch_nest_check(const LayoutDev* const* levs, int nl, int* status, cudaStream_t s);
// Lists of each layout l of levs[0 .. nl) (nl <= 8; a level may appear twice,
// as its current maps and as a view of its new maps, with disjoint masks)
// selected by masks[l] (bits 1 << LST_*): act, ring,
// cov, in from the current maps (with recon, act_idx, ring_idx and cells),
// exit and enter from the current against the new maps, touch (on the
// level under either, with the block or a face neighbour changing its
// on-level or covered state: the blocks whose cell flags can change).
// Items carry the level index.  Every layout in the same three launches.
cudaError_t launch_lists(const LayoutDev* const* levs, const int* masks, int nl, cudaStream_t s);
// Copies the new maps over the current ones, every level.
cudaError_t launch_commit_maps(const LayoutDev* const* levs, int nl, cudaStream_t s);
// Reverse footprints of every refinable level of levs[0 .. nl) from the
// reconstructing tiles of the level below it (after the lists), in one
// launch; an overflow of FOOT_CAP sets ST_TASKCAP (and readers take at most
// FOOT_CAP entries).
cudaError_t launch_footprints(const LayoutDev* const* levs, int nl, int* status, cudaStream_t s);
// Concatenates the act lists of levels 0..n-1 into out (lid = level), with
// the total in *n_out.
cudaError_t launch_concat_act(const LayoutDev* levs, int n, Item* out, int* n_out, cudaStream_t s);
// counter += steps * sum_l cells_l 2^l
cudaError_t launch_count_lups(const LayoutDev* levs, int n, long long steps, unsigned long long* counter,
                              cudaStream_t s);

// ---- device task lists ----------------------------------------------------

// access patterns of the task builder: which tasks of a phase touch a tile
// of a resource (the same patterns as vlbm_tasks.h)
// (TB_BOX9: the 3 x 3 tiles around each task's tile, the relaxation
// sensor's filters)
enum : int { TB_OWN = 0, TB_STENCIL = 1, TB_FOOT = 2, TB_CHILD4 = 3, TB_OWNRING = 4, TB_BOX9 = 5 };

// kind 0: sweeps of level l (sub-step kk of the parent's sub-step kkp; first:
// the level's first sweep of the step), 1: closes of level l, 2: the audit
// phase of a cyclic list (reduction tasks, see TBPlan::audit), 3 and 4: the
// relaxation sensor's two passes before each sweep phase (W, Q, u, v; then
// s and theta), on the sweep's tiles
struct TBPhase {
    int kind, l, kk, kkp, step, first;
};
struct TBAcc {
    int phase, write, pat;
};
struct TBLevel {
    int nx, ny, bx, by, px, py;
    const Item* act;
    const Item* ring;
    const int* act_idx;
    const int* ring_idx;
    const uint8_t* recon;
    const int* fcnt;  // reverse footprints (refinable levels)
    const int* fidx;
    const int* cnt;  // [NLST]
};
// resources of a level: buffer 0, buffer 1, flags, the sensor's first-pass
// planes, its second-pass planes
constexpr int TB_NRES = 5;
constexpr int TASK_RC = 4 * TB_NRES;  // resource classes (level, resource)
// dependencies of task t at deps[t * TASK_DEP_SLOT ..] when they fit, else
// in the overflow area after task_cap * TASK_DEP_SLOT entries
constexpr int TASK_DEP_SLOT = 32;
// audit slots per reduction block of a device-built list (its reduction
// tasks' dependencies fit their fixed slots)
constexpr int TB_AUDIT_BLOCK = 32;

// Static tables of a phase sequence (depend on the level count and the steps
// per launch only) and the buffers of one task list.
struct TBPlan {
    int nlev = 0, nphase = 0, nacc = 0;
    // cyclic: the list is one coarse step that the kernel runs once per
    // step, and a task's walk continues through the previous iteration
    // (dependencies there stored as ~index); otherwise the list starts from
    // a synchronised state
    int cyclic = 0;
    TBLevel lev[4] = {};
    const TBPhase* ph = nullptr;       // [nphase]
    const TBAcc* acc = nullptr;        // per resource class (l * TB_NRES + kind), in phase order
    const int* acc_beg = nullptr;      // [TASK_RC + 1]
    const int* acc_pos = nullptr;      // [(l * TB_NRES + kind) * (nphase + 1) + p]: first entry at or after phase p
    int* off = nullptr;                // [nphase + 1] task offsets of the phases (computed)
    Task* tasks = nullptr;             // [task_cap]
    int* deps = nullptr;               // [dep_cap]: fixed slots, then the overflow area
    unsigned* done = nullptr;          // completion marks (left as they are)
    int task_cap = 0;
    long long dep_cap = 0;
    int* need = nullptr;               // [8]: tasks of the last build, overflow area used, tasks of the
                                       // fallback pass, overflow flag, tasks in the overflow area, audit
                                       // slots, audit blocks, the fallback pass's finishing ticket
    // Audited cyclic list: the first sweep of each level in the step gives
    // each of its tiles an audit slot (levels in order, each in act-list
    // order), and the audit phase holds four reduction tasks (one per field)
    // per block of TB_AUDIT_BLOCK consecutive slots, each depending on the
    // sweeps of its block's slots.  The kernel does this work only in the
    // first iteration of a launch whose CTL_AUDIT word is set.
    int audit = 0;
    // the relaxation sensor's passes are in the list: the sweeps also read
    // their tile's first-pass planes and the second-pass planes of the 3 x 3
    // tiles around it
    int sensor = 0;
    int pfirst[4] = {-1, -1, -1, -1};  // the first-sweep phase of each level
    int* ascale = nullptr;             // [slots] weight exponent of the slot's level (-2 l)
    int2* arng = nullptr;              // [blocks] slot range of each block
    int* big = nullptr;                // [task_cap] tasks of the fallback pass
    int* status = nullptr;             // hierarchy status word (ST_TASKCAP on overflow)
    Segment* seg = nullptr;            // the single-member segment of the launch
    int* prefix = nullptr;             // [2]
    int* ctl = nullptr;                // CTL_WORDS
};
// Builds the task list of the plan's phase sequence on the current lists:
// phase offsets, then every task with its sorted dependencies (four tasks
// per warp; a one-thread fallback pass for tasks whose raw dependency
// entries overflow the warp's buffer, whose last CTA writes the launch's
// task count into seg, prefix and ctl).  When the overflow area is
// exhausted the list is left empty (the launch does nothing) and
// ST_TASKCAP is set in *status.
cudaError_t launch_task_build(const TBPlan& P, cudaStream_t s);
// The chunk table of one persistent launch over nm one-step task lists with
// the same phase sequence (nphase phases), phase-major: per phase, each
// list's tasks of that phase in turn.  offs[m]: list m's phase offsets
// (device, nphase + 1 ints); mctl[m]: its own control words (a list whose
// build failed is left out).  Writes prefix (<= nphase * nm + 1), chunks
// (<= nphase * nm) and the launch's control words (counters reset; the
// epoch and the parity flip are left as they are).
cudaError_t launch_merge_chunks(const int* const* offs, const int* const* mctl, int nm, int nphase, int* prefix,
                                int2* chunks, int* ctl, cudaStream_t s);

}  // namespace vlbm
