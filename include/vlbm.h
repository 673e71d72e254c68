/*
 * vlbm.h -- C ABI of the B300 (sm_103a) implementation of the conservative
 * locally refined vectorial lattice Boltzmann method for the 2-D compressible
 * Euler equations (Hosseini, Strassle & Karlin, "Conservative local grid
 * refinement for the vectorial lattice Boltzmann method").
 *
 * What one coarse step computes (all FP64, all on the GPU):
 *   - per level, the fused D2Q4 stream-and-collide update: each conserved
 *     field (rho, rho u, rho v, rho E) has its own four populations, the
 *     vector equilibrium f_i^eq = W/4 + c_i.Q(W)/(2c^2) is fixed by the Euler
 *     flux, the BGK relaxation is f* = 2 beta f^eq + (1 - 2 beta) f
 *     (Sec. 2.2, Eqs. 4-6) and streaming is an exact one-cell shift (Eq. 5);
 *   - sub-cycling: level l+1 takes two steps per level-l step at the same
 *     link speed c (acoustic scaling, Sec. 3.2, Eq. 15);
 *   - coarse-to-fine: the mean-preserving reconstruction in time with the
 *     tangential minmod correction (Sec. 3.3, Eqs. 20, 22, 23);
 *   - fine-to-coarse: the reflux average of the r*r = 4 post-collision
 *     values leaving the fine side (Sec. 3.3, Eq. 24);
 *   - at regrids: merge (plain average, Eq. 25) and split (minmod-limited
 *     linear reconstruction, Eqs. 26-27), Sec. 3.4.
 *
 * Conventions
 *   - Every call returns a vlbm_status; no C++ exception crosses the ABI.
 *   - Level l has (nx0 << l) x (ny0 << l) cells; cell (i, j) of level l has
 *     its centre at ((i + 0.5) dx0 / 2^l, (j + 0.5) dx0 / 2^l).  Refinement
 *     ratio 2 per level, at most VLBM_MAX_LEVELS levels.
 *   - Refinement is decided per 8 x 8 block of cells of the refined level
 *     (VLBM_BLOCK): boxes and masks must be block aligned.
 *   - Host arrays are owned by the caller and copied; device arrays passed
 *     with on_device = 1 must live on the handle's device and are read on
 *     the handle's stream.
 *   - Conserved-field arrays are W[4][ny_l][ld] (x fastest, ld >= nx_l),
 *     fields in the order rho, rho u, rho v, rho E.
 *   - Population arrays are f[16][ny_l][ld] with population q = 4 i + k:
 *     direction i in (+x, -x, +y, -y), field k as above.
 *   - The library owns all device memory of a handle; it comes from the
 *     caller's allocator when one is given, else from cudaMallocAsync on
 *     the handle's stream.
 *   - Handles are not thread safe; distinct handles are independent.
 *   - vlbm_advance is asynchronous.  A non-physical state (rho <= 0,
 *     p <= 0 or not finite) met by a kernel is reported by the next
 *     synchronising call (vlbm_sync, vlbm_get_conserved, vlbm_audit,
 *     vlbm_regrid) as VLBM_ERR_NONPHYSICAL; the handle then answers
 *     VLBM_ERR_STATE to every call but vlbm_last_error and vlbm_destroy.
 */
#ifndef VLBM_H
#define VLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VLBM_MAX_LEVELS 4
#define VLBM_BLOCK 8

typedef struct vlbm_hier vlbm_hier;     /* opaque, owned by the library */
typedef struct vlbm_engine vlbm_engine; /* opaque batching/serving engine */

typedef enum {
    VLBM_OK = 0,
    VLBM_ERR_ARG = 1,          /* an argument is out of range or malformed */
    VLBM_ERR_NESTING = 2,      /* a refinement layout is not properly nested */
    VLBM_ERR_OOM = 3,          /* allocation failed, or the engine is full */
    VLBM_ERR_CUDA = 4,         /* a CUDA call failed (see vlbm_last_error) */
    VLBM_ERR_NONPHYSICAL = 5,  /* rho <= 0, p <= 0 or NaN met by a kernel */
    VLBM_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    VLBM_ERR_STATE = 7         /* the handle is poisoned by an earlier error */
} vlbm_status;

typedef enum {
    VLBM_BC_PERIODIC = 0,  /* both sides of an axis must be periodic */
    VLBM_BC_OUTFLOW = 1,   /* zero gradient: the ghost repeats the edge cell */
    VLBM_BC_INFLOW = 2,    /* ghost in equilibrium at the side's inflow_W */
    VLBM_BC_REFLECT = 3    /* slip wall: mirror state, normal momentum negated */
} vlbm_bc;

/* A rectangle of cells of `level` that is covered by level + 1. */
typedef struct {
    int32_t level, i0, j0, ni, nj;
} vlbm_box;

typedef struct {
    int32_t nx0, ny0;          /* coarse grid size (cells), >= 1 each */
    double dx0;                /* coarse spacing (only reported back) */
    int32_t max_levels;        /* 1..VLBM_MAX_LEVELS */
    int32_t bc[4];             /* vlbm_bc of the W, E, S, N sides */
    double inflow_W[4][4];     /* W of the ghost state, per side (INFLOW only) */
    double gamma;              /* ideal-gas ratio of specific heats, > 1 */
    double c;                  /* link speed c = dx/dt (same on every level), > 0 */
    double beta;               /* BGK relaxation parameter, 0 <= beta <= 1 */
    const vlbm_box* boxes;     /* initial static refinement, may be NULL */
    int32_t nboxes;
    double tag_tol;            /* adaptive regrid: indicator tolerance */
    int32_t tag_buffer;        /* adaptive regrid: dilation (cells) */
    int32_t tag_sensor;        /* adaptive regrid indicator: VLBM_SENSOR_* */
} vlbm_config;

/* Tagging indicators of the adaptive regrid (both on the composite state,
 * covered cells holding the average of their children; neighbours off the
 * level or beyond a non-periodic side take the cell's own value):
 *   DENSITY  (rho_E - rho_W)^2 + (rho_N - rho_S)^2 > tol^2 (2 rho_C)^2
 *   FLUX     the flux-jump estimate of Sec. 3.4 (Eq. amr-sigma),
 *            s = max_k |dx (div Q)_k| / max_{x,alpha} |Q_{alpha,k}| > tol,
 *            central differences, maxima over every cell of every level */
enum { VLBM_SENSOR_DENSITY = 0, VLBM_SENSOR_FLUX = 1 };

typedef struct {
    /* returns device memory of `bytes` usable on `stream`, or NULL */
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} vlbm_allocator;

typedef struct {
    int32_t nlev;                          /* levels allocated */
    int32_t nx[VLBM_MAX_LEVELS], ny[VLBM_MAX_LEVELS];
    int64_t active_cells[VLBM_MAX_LEVELS]; /* cells updated per level step */
    int64_t lups_per_step;                 /* sum_l active_cells_l * 2^l */
    int64_t device_bytes;                  /* device memory held */
    int64_t steps;                         /* coarse steps taken */
    double c, beta, gamma, dx0;
} vlbm_info;

/* ---- hierarchy life cycle ---------------------------------------------- */

/* Creates a hierarchy: levels 0 .. max_levels-1 at refinement ratio 2 with
 * one link speed c on every level (acoustic scaling, Sec. 3.2, Eq. 15: the
 * time step halves from level to level), ideal gas of ratio gamma
 * (Sec. 2.1, Eq. 1), BGK parameter beta (Sec. 2.2, Eq. 6), with the initial
 * static layout cfg->boxes (validated: block aligned, inside the domain,
 * properly nested -- every cell covered on level l >= 1 has its four face
 * neighbours on level l; the paper's levels are nested, Sec. 4.3).  The
 * populations are zero until vlbm_set_state.  alloc (may be NULL: stream
 * ordered cudaMallocAsync) provides all of the handle's device memory;
 * stream is a cudaStream_t (NULL = legacy default stream) used by every
 * later call on the handle.
 * Errors: ERR_ARG, ERR_NESTING, ERR_OOM, ERR_CUDA; *out is NULL then. */
vlbm_status vlbm_create_hierarchy(const vlbm_config* cfg, const vlbm_allocator* alloc,
                                  void* stream, vlbm_hier** out);

/* Sets f = f^eq(W) (Eq. 4) on every cell of `level` (covered cells included)
 * from W[4][ny_l][ld].  on_device = 0: host array (copied, synchronous);
 * 1: device array.  Faces seen for the first time have no previous sample.
 * Errors: ERR_ARG (level, ld), ERR_CUDA, ERR_STATE. */
vlbm_status vlbm_set_state(vlbm_hier* h, int32_t level, const double* W, int64_t ld,
                           int32_t on_device);

/* Raw population access for tests and checkpoints: f[16][ny_l][ld]. */
vlbm_status vlbm_set_populations(vlbm_hier* h, int32_t level, const double* f, int64_t ld,
                                 int32_t on_device);
vlbm_status vlbm_get_populations(vlbm_hier* h, int32_t level, double* f, int64_t ld,
                                 int32_t on_device);

/* Advances `coarse_steps` coarse steps (each: one level-0 step, two level-1
 * steps per level-0 step, and so on, with reconstruction and reflux at every
 * interface; Sec. 3.2, Fig. 1 and Eq. 15 for the sub-cycle, Sec. 3.3, Eqs.
 * 20-24 for the coupling, Sec. 2.2, Eqs. 4-6 for the level update).
 * Asynchronous on the handle's stream: launches captured CUDA graphs, and
 * after a layout change first builds the persistent schedule's task lists
 * on the device.  Deferred errors (non-physical state, a timed-out wait, a
 * device layout or task list that did not fit) are reported by the next
 * synchronising call.  Errors: ERR_ARG (negative), ERR_CUDA, ERR_STATE. */
vlbm_status vlbm_advance(vlbm_hier* h, int64_t coarse_steps);

/* Regrid (Sec. 3.4, Fig. 2).  boxes != NULL: the new layout is the union of
 * the boxes (validated like vlbm_create_hierarchy); synchronises the
 * stream.  boxes == NULL: the layout is derived from the indicator
 * cfg->tag_sensor (VLBM_SENSOR_*) with cfg->tag_tol and cfg->tag_buffer,
 * rounded to blocks and grown so that every level nests; for a hierarchy
 * outside an engine this runs on the device alone and is asynchronous (the
 * indicator, block flags, layout rule, merge, split, flags and tile lists
 * are queued on the stream and the host never waits), a nesting violation
 * then being reported as ERR_NESTING by the next synchronising call.  Cells
 * leaving refinement take the merge of their children (Eq. 25), cells
 * entering refinement are split (Eqs. 26-27) -- finest level first for
 * merges, coarsest first for splits.
 * Errors: ERR_ARG, ERR_NESTING (layout unchanged), ERR_CUDA, ERR_STATE,
 * ERR_NONPHYSICAL (from an earlier advance). */
vlbm_status vlbm_regrid(vlbm_hier* h, const vlbm_box* boxes, int32_t nboxes);

/* Same as vlbm_regrid with a per-cell refinement mask for every level
 * l < nlev-1 (ref[l] is uint8[ny_l][nx_l], 1 = covered by level l+1); the
 * masks must be block aligned. */
vlbm_status vlbm_regrid_masks(vlbm_hier* h, const uint8_t* const* ref);

/* Per-cell layout of `level`: in[c] = 1 on the level, ref[c] = 1 covered by
 * the next level (host arrays of ny_l * nx_l bytes, either may be NULL). */
vlbm_status vlbm_get_layout(vlbm_hier* h, int32_t level, uint8_t* in, uint8_t* ref);

/* Conserved fields W = sum_i f_i (the zeroth moment of the populations,
 * Sec. 2.2, Eq. 4) of `level` into W[4][ny_l][ld] (host, may be NULL);
 * valid[ny_l*nx_l] (may be NULL) = 1 on active cells.  totals and
 * abs_totals (may be NULL) receive sum_l 4^-l sum_active W_k and the same
 * of |W_k| over the whole hierarchy -- the paper's conservation monitors
 * (total over the coarse cells outside the patch holes plus the fine cells,
 * area weighted; Sec. 4.1.2, 4.1.3, 4.2) -- as the exact sums (192-bit
 * fixed point, resolution 2^-128) rounded once to nearest binary64.
 * Synchronises.  Errors: ERR_ARG, ERR_CUDA, ERR_NONPHYSICAL, ERR_STATE. */
vlbm_status vlbm_get_conserved(vlbm_hier* h, int32_t level, double* W, int64_t ld,
                               uint8_t* valid, double totals[4], double abs_totals[4]);

/* Totals only: the conservation monitors of Sec. 4.1.2, 4.1.3 and 4.2 as
 * exact sums (see vlbm_get_conserved).  Synchronises.
 * Errors: ERR_ARG, ERR_CUDA, ERR_NONPHYSICAL, ERR_STATE. */
vlbm_status vlbm_audit(vlbm_hier* h, double totals[4], double abs_totals[4]);

/* Waits for the stream and reports deferred device errors. */
vlbm_status vlbm_sync(vlbm_hier* h);

/* Sizes, active cells per level and cell updates per coarse step of the
 * current layout.  After a tag-driven regrid (which runs on the device
 * alone) this synchronises the stream to fetch the new layout.
 * Errors: ERR_ARG, ERR_CUDA, ERR_STATE. */
vlbm_status vlbm_get_info(const vlbm_hier* h, vlbm_info* info);

/* Cell updates done since the hierarchy was created: the sum over every
 * coarse step taken of sum_l active_cells_l * 2^l, counted on the device at
 * the layout each step ran on (so it stays exact across regrids that the
 * host never waited for).  Synchronises.
 * Errors: ERR_ARG, ERR_CUDA, ERR_NONPHYSICAL, ERR_STATE. */
vlbm_status vlbm_lups_done(vlbm_hier* h, int64_t* lups);

/* Kernels this library has queued for the hierarchy since its creation
 * (every kernel of every captured graph launch, and each eager launch of a
 * step, regrid, audit or task-list build), counted on the host when they
 * are queued.  Errors: ERR_ARG. */
vlbm_status vlbm_kernels_launched(const vlbm_hier* h, int64_t* n);

/* The cell-update counter (vlbm_lups_done) copied, in stream order and
 * without waiting, into *dst
 * (host memory: pinned for a truly asynchronous copy; valid once the stream
 * has reached this point).  Errors: ERR_ARG, ERR_CUDA, ERR_STATE. */
vlbm_status vlbm_lups_mark(vlbm_hier* h, int64_t* dst);

/* Conservation across regrids (Sec. 3.4: merge and split add or remove
 * nothing).  on = 1: every tag-driven regrid that runs on the device
 * records, on the device and without synchronising, the exact totals of
 * vlbm_audit immediately before and immediately after it, into a ring of
 * the last 4096 regrids.  The totals after a regrid are those of the state
 * the regrid leaves: when the next steps run on the persistent schedule
 * they come from that launch's first sweeps (which form every active
 * cell's moments anyway) and a reduction in the same launch; otherwise, or
 * when another call changes the state or reads the rows first, from a
 * separate audit queued then -- the same values either way.
 * vlbm_get_regrid_audits copies the rows recorded since the previous read
 * (at most cap, oldest first) into out[n][16]: totals before (4), |W|
 * totals before (4), totals after (4), |W| totals after (4); it
 * synchronises.  Errors: ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE (and
 * deferred errors on the read). */
vlbm_status vlbm_set_regrid_audit(vlbm_hier* h, int32_t on);
vlbm_status vlbm_get_regrid_audits(vlbm_hier* h, double* out, int64_t cap, int64_t* n);

/* Host-side time the library has spent on a hierarchy since its creation,
 * in milliseconds (wall clock, cumulative), by activity:
 *   TAG       adaptive regrid: average-down, indicator and block flags on the
 *             device and their copy to the host queued, and (vlbm_regrid)
 *             the wait for them
 *   LAYOUT    new block maps from flags or boxes (grading, nesting)
 *   REGRID    merge/split launches, per-cell flags, tile lists, uploads
 *   BUILD     level tables of the launch (after a layout change)
 *   TASKS     task lists with their dependencies (one coarse step or
 *             graph_steps coarse steps), uploaded
 *   CAPTURE   CUDA graph capture and instantiation
 * and the counts NREGRIDS (vlbm_regrid calls) and NTASKLISTS (task lists
 * built).  Device time of the sweeps is not included (see vlbm_profile).
 * Errors: ERR_ARG. */
enum {
    VLBM_T_TAG = 0,
    VLBM_T_LAYOUT = 1,
    VLBM_T_REGRID = 2,
    VLBM_T_BUILD = 3,
    VLBM_T_TASKS = 4,
    VLBM_T_CAPTURE = 5,
    VLBM_T_NREGRIDS = 6,
    VLBM_T_NTASKLISTS = 7,
    VLBM_T_COUNT = 8
};
vlbm_status vlbm_host_times(const vlbm_hier* h, double out[VLBM_T_COUNT]);

/* Per-kernel timing of the sub-cycle.  Runs `coarse_steps` coarse steps
 * launch by launch (not through the graph) with CUDA events around every
 * kernel on the handle's stream, and reports one record per kernel kind:
 * kind 0 = level sweep (fused collide + stream + boundary + coarse-to-fine)
 * of `level`, kind 1 = reflux close into `level`, kind 2 = end of step.
 * `cells` counts the cell updates the launches performed.  The state
 * advances exactly as with vlbm_advance.  cap >= 2 * VLBM_MAX_LEVELS + 1
 * records suffice.  Errors: ERR_ARG, ERR_CUDA, ERR_STATE. */
typedef struct {
    int32_t kind, level;
    int64_t launches;
    int64_t cells;
    double ms;
} vlbm_kernel_time;

vlbm_status vlbm_profile(vlbm_hier* h, int64_t coarse_steps, vlbm_kernel_time* out, int32_t cap, int32_t* n);

/* Launch tuning of the sweep.  variant (0 .. vlbm_num_variants() - 1)
 * selects one compiled launch shape of the level sweep: 0, 1, 2 -- 64-thread
 * groups on whole 8x8 tiles at 2, 3 or 4 CTAs per SM; 3, 4 -- for the
 * persistent kernel of schedule 1, warps working alone on half-tile tasks at
 * 3 or 2 CTAs per SM (the per-phase sweep runs whole tiles).  Results are
 * identical bit for bit in every variant.
 * schedule 0 issues one kernel launch per phase of the sub-cycle (level
 * sweeps, reflux closes); schedule 1 runs graph_steps coarse steps of every
 * phase in one persistent launch whose 8x8-tile tasks start as soon as the
 * tasks they depend on (read-after-write, write-after-read and
 * write-after-write on populations and flags) are done -- the waits are
 * bounded and report VLBM_ERR_TIMEOUT; the task lists are built on the
 * device after every layout change (on the host when per-step totals are
 * on); schedule 2 (auto) uses schedule 0 until the current layout has lived
 * persist_after coarse steps (default 2) and schedule 1 from then on, and
 * schedule 1 whenever per-step totals are on (a device task-list build costs
 * less than a coarse step of schedule 0 loses to schedule 1 on multi-level
 * layouts, so only layouts that change every step or two keep schedule 0).
 * The default tuning is variant 1, schedule 1, graph_steps 8.  max_ctas
 * caps the grid (0 = no cap: schedule 0 takes one CTA per four tiles, or one
 * wave of resident CTAs looping over a list whose length lives on the
 * device; schedule 1 all resident CTAs);
 * graph_steps (1..64) is the number of coarse steps captured per CUDA graph.
 * vlbm_set_tuning returns ERR_ARG for an unknown variant or out-of-range
 * values (the tuning is then unchanged).  Results do not depend on the
 * tuning. */
typedef struct {
    int32_t variant, max_ctas, graph_steps, schedule;
    int64_t persist_after; /* schedule 2 only, >= 0 */
} vlbm_tuning;

int32_t vlbm_num_variants(void);
vlbm_status vlbm_set_tuning(vlbm_hier* h, const vlbm_tuning* t);
vlbm_status vlbm_get_tuning(const vlbm_hier* h, vlbm_tuning* t);


/* Self-test of the integer-pipe reciprocal that the collision uses for
 * 1/rho (the Euler flux of Sec. 2.1, Eq. 1; Newton-Raphson in integer
 * fixed point with an exact remainder test): on n seeded values
 * (SplitMix64 stream from `seed`; densities near 1, significands next to 1
 * and 2, exponent extremes, zeros, subnormals, infinities, NaNs,
 * negatives, raw bit patterns) *mismatches counts results whose bits
 * differ from the FP64 division 1.0 / x, *unsettled the inputs of the
 * handled range (positive normal x with a normal reciprocal) whose exact
 * correction did not settle (they would take the division); first_bad
 * (may be NULL) receives the first offending (x, result).  Runs on the
 * current device and synchronises it.  Errors: ERR_ARG, ERR_OOM, ERR_CUDA. */
vlbm_status vlbm_selftest_rcp(uint64_t seed, int64_t n, uint64_t* mismatches, uint64_t* unsettled,
                              double first_bad[2]);

/* Self-test of the correctly rounded division a / b that the relaxation
 * sensor uses (the reciprocal above, then two remainder corrections by
 * fused multiply-add): over n test pairs (SplitMix64 stream from `seed`;
 * quotients of the sensor's kinds, operands over the whole binary64 range
 * with random signs, exponents next to the fast path's bounds, zeros,
 * subnormals, infinities, NaNs, raw bit patterns) *mismatches counts
 * quotients whose bits differ from the FP64 division; first_bad (may be
 * NULL) receives the first offending (a, b, result).  Runs on the current
 * device and synchronises it.  Errors: ERR_ARG, ERR_OOM, ERR_CUDA. */
vlbm_status vlbm_selftest_div(uint64_t seed, int64_t n, uint64_t* mismatches, double first_bad[3]);

/* Sensor-driven relaxation (Sec. 2.2, Eq. sensor-B).  on = 1: every level
 * step first evaluates, on the level's pre-collision state,
 *   s_k   = dx (div Q)_k / qmax_k (central differences), qmax_k =
 *           max |Q_{alpha,k}| over the active cells of every level of the
 *           state at this call (kept fixed, like the link speed),
 *   s     = (sum_k s_k^2 / 4)^(1/2),
 *   theta = dil^2 / (dil^2 + vort^2 + eps) where dil = div u < 0, else 0
 *           (undivided central differences),
 * then relaxes each active cell with
 *   beta  = beta_max - (beta_max - beta_min) clip(c_sensor s_bar theta_bar, 0, 1)
 * where s_bar, theta_bar are 3 x 3 box filters and beta_max is cfg->beta;
 * neighbours that are not active cells of the level take the cell's own
 * value.  W remains a collision invariant cell by cell, so conservation is
 * unchanged.  Two sensor passes precede each level sweep: two launches on
 * schedule 0; on schedule 1 tasks of the persistent launch that depend on
 * the tiles they read (one kernel form: the tuning's variant does not
 * apply).  Per-step totals are not available with the sensor.  on = 0: constant
 * beta again.  Synchronises.  Errors: ERR_ARG (parameters: 0 <= beta_min
 * <= beta, c_sensor >= 0, eps >= 0; resident in an engine; per-step totals
 * on), ERR_OOM, ERR_CUDA, ERR_STATE. */
vlbm_status vlbm_set_sensor(vlbm_hier* h, int32_t on, double beta_min, double c_sensor, double eps);

/* Self-test of the device-resident layouts (no counterpart in the paper:
 * it checks this library's own machinery).  `cases` seeded random
 * hierarchies (2-4 levels, ragged sizes, periodic or not per axis), each
 * regridded three times from random block flags on the device alone; after
 * each regrid the device's block maps, tile lists (active, ring, covered,
 * on-level, in row-major order), reconstruction map and active cell counts
 * must equal those the host computes from the same flags with its layout
 * rule, and the persistent schedule's task list built on the device for
 * 1-3 coarse steps must equal the host builder's task for task and
 * dependency for dependency.  *mismatches counts differences;
 * *second_pass (may be NULL) the tasks with more dependencies than their
 * fixed slot holds (stored in the overflow area); first_bad (may
 * be NULL, `cap` bytes) describes the first difference.  Runs on the
 * current device, synchronises.  Errors: ERR_ARG, ERR_OOM, ERR_CUDA. */
vlbm_status vlbm_selftest_layout(uint64_t seed, int32_t cases, int64_t* mismatches, int64_t* second_pass,
                                 char* first_bad, int32_t cap);

/* Self-test of the bounded waits of the persistent task kernel (schedule
 * 1): launches it on one task that depends on a completion mark nothing
 * sets.  The wait gives up after its poll limit (about a second), the
 * kernel records the timeout in its status word and returns.  Returns
 * VLBM_ERR_TIMEOUT when that happened (the expected outcome), VLBM_OK if
 * the wait ended otherwise, ERR_CUDA on a CUDA error; *elapsed_ms is the
 * kernel's duration and *status_word the raw status bits (2 = timeout).
 * Uses its own stream and memory; synchronises. */
vlbm_status vlbm_selftest_timeout(double* elapsed_ms, int32_t* status_word);

/* Checkpoint / resume.  The blob (host memory, versioned) holds what a
 * coarse step needs at a sync point: the configuration it was made under,
 * the step count and level-0 parity, every level's block maps, per-cell
 * flags and state buffer over the whole index space (covered cells keep the
 * previous coarse samples of Eq. 20).  Loading it into a hierarchy created
 * with the same nx0, ny0, max_levels, boundaries, gamma, c and beta resumes
 * the run bit for bit.  save/load synchronise.  Errors: ERR_ARG (size,
 * magic or configuration mismatch), ERR_CUDA, ERR_STATE. */
vlbm_status vlbm_checkpoint_size(vlbm_hier* h, size_t* bytes);
vlbm_status vlbm_checkpoint_save(vlbm_hier* h, void* blob, size_t bytes);
vlbm_status vlbm_checkpoint_load(vlbm_hier* h, const void* blob, size_t bytes);

/* Per-step conservation audit fused into the sweep (Sec. 4.1.2, 4.1.3, 4.2
 * report conservation to round-off; this checks it at every coarse step).
 * With `on`, every coarse step taken by vlbm_advance records the totals of
 * the state at the START of that step: sum_l 4^-l sum_active W_k and the
 * same of |W_k| (k = rho, rho u, rho v, rho E).  The sweep's first
 * sub-step on every level keeps the moments of its cells; reduction tasks of
 * the same persistent launch, scheduled between the later sweeps, sum them
 * in 192-bit fixed point on the integer pipes (resolution 2^-128), so the
 * totals are exact, independent of the launch configuration, and rounded
 * once to binary64 (the correctly rounded sum); no extra pass over the
 * populations is made.  Requires the
 * persistent schedule (vlbm_tuning.schedule = 1), else ERR_ARG.
 * vlbm_get_step_totals synchronises and returns, oldest first, the rows
 * recorded since the previous call (at most the 4096 most recent), each
 * 8 doubles (totals[4], abs_totals[4]); *n receives the row count.
 * Errors: ERR_ARG, ERR_CUDA, ERR_NONPHYSICAL, ERR_STATE. */
vlbm_status vlbm_set_step_totals(vlbm_hier* h, int32_t on);
vlbm_status vlbm_get_step_totals(vlbm_hier* h, double* out, int64_t cap, int64_t* n);

/* Conservation totals of a caller-owned population array, allocating
 * nothing.  The paper has no counterpart: this serves callers that cannot
 * allocate device memory when they want the check (an application that
 * reserves all of its GPU memory up front and forbids later allocations, or
 * one that holds only raw device pointers to populations it manages) and
 * so cannot create a hierarchy for vlbm_audit.
 *   f      device array [16][ny][ld] in the layout of vlbm_get_populations
 *   out    device array of 8 doubles: weight * sum W_k and weight * sum |W_k|
 *          over all nx * ny cells, k = rho, rho u, rho v, rho E
 *   stream cudaStream_t the two kernels run on (NULL = legacy default)
 * The reduction's partial sums live in one fixed device array of
 * VLBM_STATIC_MAX_BLOCKS slots (2 MiB, held by every device that loads the
 * library until exit); each slot covers 4096 cells, so nx * ny is limited to
 * VLBM_STATIC_MAX_BLOCKS * 4096 cells and larger grids get ERR_ARG.  CUDA
 * loads modules lazily: the first call on a device loads this code and the
 * array onto it, which takes device memory once -- make that first call (a
 * warm-up on a small array will do) before reserving the rest of the
 * device's memory, and before any stream capture; later calls take none.
 * A call made outside a capture looks the array's device address up afresh
 * (a context recreated after a device reset is followed); a call made while
 * `stream` is captured uses the address of the last call on that device.
 * Every call shares the array: calls whose kernels overlap on the GPU
 * (other streams) race and must be serialised by the caller.  No
 * cudaMalloc, cudaFree or allocating library routine is used.
 * Asynchronous: read `out` after synchronising `stream`.
 * Errors: ERR_ARG (null pointers, sizes), ERR_CUDA (also: first call on the
 * device made during a stream capture). */
#define VLBM_STATIC_MAX_BLOCKS 16384
vlbm_status vlbm_totals_static(const double* f, int64_t ld, int32_t nx, int32_t ny, double weight, double* out,
                               void* stream);

/* Human-readable description of the last error on the handle (never NULL). */
const char* vlbm_last_error(const vlbm_hier* h);

void vlbm_destroy(vlbm_hier* h);

/* ---- batching / serving engine ------------------------------------------ */

/* An engine advances many resident hierarchies together: the k coarse
 * steps of one call run for every resident as one launch per phase of the
 * sub-cycle covering the tiles of all residents (schedule 0, the default),
 * or in one persistent launch of the task kernel (schedule 1: each
 * resident's one-step task list, built on the device when its layout
 * changes, merged phase-major with the others -- every resident's tasks of a
 * phase before any resident's tasks of the next -- so no thread group waits
 * at a small resident's phase boundary while others have ready work; the
 * per-phase launches serve while a resident runs the sensor-driven
 * relaxation).  mem_budget bounds the summed
 * device memory of the residents (0 = no bound).  alloc (may be NULL:
 * stream-ordered cudaMallocAsync) provides the engine's own device memory
 * (its launch tables); the residents' memory comes from their own handles.
 * stream (NULL: a stream of its own) carries every engine launch.
 * Errors: ERR_ARG, ERR_CUDA, ERR_OOM; *out is NULL then. */
vlbm_status vlbm_engine_create(size_t mem_budget, const vlbm_allocator* alloc, void* stream, vlbm_engine** out);

/* Admits h (created on the same device; the engine borrows it until release)
 * for coarse_steps steps (0: reported finished, unchanged, by the next
 * vlbm_engine_advance); adaptive hierarchies (tag_tol > 0) regrid every
 * regrid_every coarse steps (0 = never).  Errors: ERR_OOM when admitting
 * would exceed the budget (not admitted, try later), ERR_ARG. */
vlbm_status vlbm_engine_admit(vlbm_engine* e, vlbm_hier* h, int64_t coarse_steps,
                              int32_t regrid_every, int32_t* slot);

/* Queues the next k coarse steps of every resident that can step, 1 <= k
 * <= max_steps (at most 64), as many as no resident reaches its step count
 * or an adaptive resident its next regrid in between, on the engine's
 * schedule (vlbm_engine_set_schedule); each resident's result is the same
 * as when it is advanced alone.  An adaptive resident due for a regrid pauses: the
 * first half of its regrid is queued on a high-priority stream, a later
 * call finishes it once its block flags are on the host.  Asynchronous:
 * the call waits only for the steps it queued four calls before, and for
 * pending regrids or finishing residents when no resident can step.
 * finished_slots (capacity = the largest slot + 1) receives the residents
 * whose step count is met and whose last step has completed on the GPU --
 * reported by the first call after that; their results can then be read
 * without waiting, and a finished resident whose state turned non-physical
 * is poisoned (its handle then returns ERR_STATE, vlbm_last_error says
 * why).  *steps = k (0 when no resident can step).  Errors: ERR_ARG,
 * ERR_CUDA, errors of a resident's regrid. */
vlbm_status vlbm_engine_advance(vlbm_engine* e, int32_t max_steps, int32_t* finished_slots, int32_t* nfinished,
                                int32_t* steps);

/* The engine's schedule: 0 (default) one launch per phase shared by all
 * residents; 1 one persistent launch per call over every resident's
 * device-built task list, phase-major.  Results do not depend on it.
 * Errors: ERR_ARG (unknown schedule). */
vlbm_status vlbm_engine_set_schedule(vlbm_engine* e, int32_t schedule);

/* vlbm_engine_advance with max_steps = 1. */
vlbm_status vlbm_engine_step(vlbm_engine* e, int32_t* finished_slots, int32_t* nfinished);

/* Removes a resident (its hierarchy returns to the caller, unchanged).
 * Waits for the engine's queued work unless the resident was reported
 * finished. */
vlbm_status vlbm_engine_release(vlbm_engine* e, int32_t slot);

/* Coarse steps taken and cell updates done by a resident since admission. */
vlbm_status vlbm_engine_slot_stats(const vlbm_engine* e, int32_t slot, int64_t* steps_done, int64_t* lups_done);

/* Number of residents and their summed device bytes. */
vlbm_status vlbm_engine_usage(const vlbm_engine* e, int32_t* residents, int64_t* bytes);

/* Host time of the engine's calls, in milliseconds (wall clock,
 * cumulative), by activity:
 *   REGRID_FINISH  second halves of residents' regrids (layout rule,
 *                  merge/split queued), including waits when no resident
 *                  could step
 *   FINISH         finishing residents: event checks, status words, waits
 *                  when no resident could step
 *   REBUILD        batch tables, task lists and graphs after a change of
 *                  members or layouts
 *   LAUNCH         queueing the steps (graph and per-phase launches)
 *   LEAD           waiting for the steps queued four calls before
 *   REGRID_BEGIN   first halves of residents' regrids queued
 * and the counts CALLS (engine calls) and STEPS (coarse steps queued, the
 * sum of k).  Errors: ERR_ARG. */
enum {
    VLBM_ET_REGRID_FINISH = 0,
    VLBM_ET_FINISH = 1,
    VLBM_ET_REBUILD = 2,
    VLBM_ET_LAUNCH = 3,
    VLBM_ET_LEAD = 4,
    VLBM_ET_REGRID_BEGIN = 5,
    VLBM_ET_CALLS = 6,
    VLBM_ET_STEPS = 7,
    VLBM_ET_COUNT = 8
};
vlbm_status vlbm_engine_host_times(const vlbm_engine* e, double out[VLBM_ET_COUNT]);

void vlbm_engine_destroy(vlbm_engine* e);

#ifdef __cplusplus
}
#endif
#endif /* VLBM_H */
