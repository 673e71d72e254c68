// Self-test of the persistent kernel's bounded waits: one task whose
// dependency mark nothing ever sets.  The wait gives up after its poll
// limit, the kernel records VLBM_ERR_TIMEOUT in the status word and
// returns; the context stays usable.  No fault, trap or endless loop is
// involved: this is the documented failure path of a broken schedule.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "vlbm.h"
#include "vlbm_dev.cuh"
#include "vlbm_launch.h"

using namespace vlbm;

extern "C" vlbm_status vlbm_selftest_timeout(double* elapsed_ms, int32_t* status_word) {
    if (!elapsed_ms || !status_word) return VLBM_ERR_ARG;
    // device block: [words: par0, status][flags 8x8][done 2][deps 1][prefix 2][chunk][ctl]
    // followed by the task, the segment and the level table
    struct Blob {
        int words[2];
        uint16_t flags[64];
        unsigned done[2];
        int deps[1];
        int prefix[2];
        int2 chunk[1];
        int ctl[CTL_WORDS];
        Task task;
        Segment seg;
        LevelDev lev;
    };
    Blob* d = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    vlbm_status st = VLBM_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && st == VLBM_OK) st = VLBM_ERR_CUDA;
        return e == cudaSuccess;
    };
    if (ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) && ck(cudaMalloc((void**)&d, sizeof(Blob))) &&
        ck(cudaEventCreate(&e0)) && ck(cudaEventCreate(&e1))) {
        Blob h;
        std::memset(&h, 0, sizeof h);  // flags 0: the task's tile holds no cell of the level
        h.deps[0] = 1;                 // mark 1 belongs to no task: it stays 0
        h.prefix[0] = 0;
        h.prefix[1] = 1;
        h.ctl[CTL_EPOCH] = 1;
        h.ctl[CTL_TOTAL] = 1;
        h.ctl[CTL_NSEG] = 1;
        h.ctl[CTL_NCHUNK] = 1;
        h.chunk[0] = make_int2(0, 0);
        h.task.lid = 0;
        h.task.kind = 1;  // reflux close: a no-op on a tile without level cells
        h.task.dep0 = 0;
        h.task.ndep = 1;
        h.task.aslot = -1;
        h.seg.tasks = &d->task;
        h.seg.deps = d->deps;
        h.seg.done = d->done;
        h.seg.aw = nullptr;
        h.seg.par0 = &d->words[0];
        h.seg.ntasks = 1;
        h.seg.lid_base = 0;
        h.lev.flags = d->flags;
        h.lev.par0 = &d->words[0];
        h.lev.status = &d->words[1];
        h.lev.nx = h.lev.ny = TILE;
        h.lev.pitch = TILE;
        h.lev.plane = TILE * TILE;
        h.lev.parent = h.lev.child = -1;
        if (ck(cudaMemcpyAsync(d, &h, sizeof h, cudaMemcpyHostToDevice, s)) && ck(cudaEventRecord(e0, s)) &&
            ck(launch_tasks(&d->lev, &d->seg, d->prefix, d->chunk, d->ctl, 1, 1, 1, s)) && ck(cudaEventRecord(e1, s)) &&
            ck(cudaStreamSynchronize(s))) {
            int w[2] = {0, 0};
            float ms = 0.f;
            if (ck(cudaMemcpy(w, d->words, sizeof w, cudaMemcpyDeviceToHost)) && ck(cudaEventElapsedTime(&ms, e0, e1))) {
                *elapsed_ms = ms;
                *status_word = w[1];
                st = (w[1] & ST_TIMEOUT) ? VLBM_ERR_TIMEOUT : VLBM_OK;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d) cudaFree(d);
    if (s) cudaStreamDestroy(s);
    return st;
}
