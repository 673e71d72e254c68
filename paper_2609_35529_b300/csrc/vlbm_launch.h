// Host-side declarations of the kernel launchers (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "vlbm_dev.cuh"

namespace vlbm {

// Launchers over a tile list take its length n, or -- with nc != nullptr --
// its capacity n and the length in device memory at nc.
cudaError_t launch_sweep(const LevelDev* levs, const Item* items, int n, int kk, int kkp, int max_ctas, int variant,
                         cudaStream_t s, bool sensor = false, const int* nc = nullptr);
cudaError_t launch_sensor(const LevelDev* levs, const Item* items, int n, int kk, cudaStream_t s,
                          const int* nc = nullptr);
int sweep_variants();
int task_kernel_ctas(int variant);
// The persistent task kernel over the segments' task lists, `iters` times in
// a row (one coarse step per iteration of one-step lists; 1 otherwise).
// Within an iteration, ticket t lies in chunk c (prefix[c] <= t <
// prefix[c + 1]) and is task chunks[c].y + t - prefix[c] of segment
// chunks[c].x; every segment's tasks appear in its own list order.
// sensor: the lists hold the relaxation sensor's passes (task kinds 3, 4)
// and the sweeps take each cell's beta from them (the variant's launch
// shape, in the kernel form that runs them).
cudaError_t launch_tasks(const LevelDev* levs, const Segment* segs, const int* prefix, const int2* chunks, int* ctl,
                         int variant, int ctas, int iters, cudaStream_t s, bool sensor = false);
cudaError_t launch_audit_segments(const unsigned long long* slots, const int* seg, int nseg, double* out,
                                  cudaStream_t s);
// Totals of an audited persistent launch from its reduction blocks' exact
// partials (*nblk blocks of 24 words, device count) into out[0..7]; clears
// *gate (the launch's CTL_AUDIT word) afterwards.
cudaError_t launch_audit_blocks(const unsigned long long* part, const int* nblk, double* out, int* gate,
                                cudaStream_t s);
cudaError_t launch_close(const LevelDev* levs, const Item* items, int n, int kk, cudaStream_t s,
                         const int* nc = nullptr);
cudaError_t launch_end_step(int* const* par, int n, cudaStream_t s);
cudaError_t launch_feq_init(const LevelDev& L, const double* W, long long ld, double hc, cudaStream_t s);
cudaError_t launch_copy_pop(const LevelDev& L, double* ext, long long ld, int to_ext, cudaStream_t s);
cudaError_t launch_gather_W(const LevelDev& L, double* W, long long ld, uint8_t* valid, cudaStream_t s);
int audit_blocks(int nitems);
// Exact totals of the cells of the listed active tiles into out[0..7] in one
// launch (part: 24 words per CTA of audit_blocks(n); ticket: a zeroed word,
// left zeroed).  Reads the tiles' populations and the level table only.
cudaError_t launch_audit(const LevelDev* levs, const Item* items, int n, unsigned long long* part, double* out,
                         unsigned* ticket, cudaStream_t s, const int* nc = nullptr);
cudaError_t launch_avgdown(const LevelDev& C, const LevelDev& F, const Item* items, int n, cudaStream_t s,
                           const int* nc = nullptr);
// A level's block maps (one byte per 8 x 8 block): on the level, covered.
struct BlockMaps {
    const uint8_t* bin;
    const uint8_t* bcov;
};
// The tag kernels flag, in bflag (zeroed by the caller), every block within
// `buffer` cells of a tagged cell of the listed tiles.
cudaError_t launch_tag(const LevelDev& L, const BlockMaps& M, const Item* items, int n, double tol2, int buffer,
                       uint8_t* bflag, cudaStream_t s, const int* nc = nullptr);
cudaError_t launch_qmax(const LevelDev& L, const Item* items, int n, unsigned long long* qmax, cudaStream_t s,
                        const int* nc = nullptr);
cudaError_t launch_tag_flux(const LevelDev& L, const BlockMaps& M, const Item* items, int n,
                            const unsigned long long* qmax, double tol, int buffer, uint8_t* bflag, cudaStream_t s,
                            const int* nc = nullptr);
cudaError_t launch_merge(const LevelDev& L, const Item* items, int n, cudaStream_t s, const int* nc = nullptr);
cudaError_t launch_split(const LevelDev& C, const LevelDev& F, const Item* items, int n, cudaStream_t s,
                         const int* nc = nullptr);
cudaError_t launch_flags(const LevelDev& L, const uint8_t* blk_in, const uint8_t* blk_cov, const uint16_t* oldf,
                         uint16_t* newf, cudaStream_t s);
// Per level: the listed blocks (on the level before or after a layout
// change; length at *nc[l]), the new block maps, the flags (rebuilt in
// place) and their scratch (overwritten).
struct FlagsSet {
    struct Geom {
        int nx, ny, pitch, px, py;
    } g[4];
    const Item* items[4];
    const int* nc[4];
    const uint8_t* bin[4];
    const uint8_t* bcov[4];
    uint16_t* oldf[4];
    uint16_t* newf[4];
    int nl;
};
// The flags of every level's listed blocks from the new block maps, in two
// launches (cap: the largest list's capacity).
cudaError_t launch_flags_update(const FlagsSet& F, int cap, cudaStream_t s);

}  // namespace vlbm
