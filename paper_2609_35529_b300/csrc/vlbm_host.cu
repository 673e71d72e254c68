// Host runtime of the VLBM library: hierarchies, layouts, batches, CUDA-graph
// capture of the sub-cycle, the C ABI and the batching/serving engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "vlbm.h"
#include "vlbm_amr.h"
#include "vlbm_dev.cuh"
#include "vlbm_launch.h"
#include "vlbm_tasks.h"

using namespace vlbm;

namespace {

// audit slots (tiles) summed by one block of the per-step audit reduction
constexpr int AUDIT_BLOCK_SLOTS = 32;
// distance (in tasks) between an audit reduction and the last sweep it reads:
// about twice the thread groups resident at 3 CTAs per SM (148 x 3 x 4)
constexpr int AUDIT_LAG = 4096;

// Kernel nodes of every instantiated graph, so that a launch can be counted
// as the kernels it runs (vlbm_kernels_launched).
std::mutex g_nk_mu;
std::vector<std::pair<cudaGraphExec_t, long long>> g_nk;

long long kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    long long k = 0;
    for (cudaGraphNode_t v : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(v, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
    }
    return k;
}

// cudaGraphInstantiate, recording the graph's kernel count for the exec.
cudaError_t instantiate(cudaGraphExec_t* ex, cudaGraph_t g) {
    const cudaError_t e = cudaGraphInstantiate(ex, g, 0);
    if (e == cudaSuccess) {
        const long long k = kernel_nodes(g);
        std::lock_guard<std::mutex> lk(g_nk_mu);
        for (auto& p : g_nk)
            if (p.first == *ex) {
                p.second = k;
                return e;
            }
        g_nk.emplace_back(*ex, k);
    }
    return e;
}

long long graph_kernels(cudaGraphExec_t ex) {
    std::lock_guard<std::mutex> lk(g_nk_mu);
    for (const auto& p : g_nk)
        if (p.first == ex) return p.second;
    return 0;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

struct Fail {
    vlbm_status st;
    std::string msg;
};

#define VCK(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            throw Fail{VLBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// ---- canonical host arithmetic (built with -ffp-contract=off) --------------

// Euler flux and vector equilibrium of Eq. 4 (D = 2), identical in expression
// order to the device code: used for the inflow ghost populations.
void host_feq(double gamma, double c, const double W[4], double feq[16]) {
    const double gm1 = gamma - 1.0;
    const double inv = 1.0 / W[0];
    const double u = W[1] * inv;
    const double v = W[2] * inv;
    const double ruu = W[1] * u;
    const double rvv = W[2] * v;
    const double p = gm1 * std::fma(-0.5, ruu + rvv, W[3]);
    const double H = W[3] + p;
    const double Qx[4] = {W[1], ruu + p, W[2] * u, H * u};
    const double Qy[4] = {W[2], W[1] * v, rvv + p, H * v};
    const double hc = 0.5 / c;
    for (int k = 0; k < 4; k++) {
        const double qw = 0.25 * W[k];
        feq[k] = std::fma(hc, Qx[k], qw);
        feq[4 + k] = std::fma(-hc, Qx[k], qw);
        feq[8 + k] = std::fma(hc, Qy[k], qw);
        feq[12 + k] = std::fma(-hc, Qy[k], qw);
    }
}

// The library's own stream-ordered memory pool on the current device, which
// keeps freed memory for reuse (release threshold: unlimited) instead of
// returning it to the driver at every synchronisation -- hierarchies of
// several GB and task lists come and go with every request and regrid.
cudaMemPool_t library_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

// Pinned host memory for the library's staging buffers, from a process-wide
// pool with power-of-two size classes: blocks are returned to the pool, not
// to the driver, because freeing pinned memory (cudaFreeHost) waits for the
// whole device -- a hierarchy destroyed while an engine's steps are queued
// would drain them.  The pool keeps what it holds until the process exits.
std::mutex pin_pool_mu;
std::vector<std::vector<void*>> pin_pool(64);
size_t pin_class(size_t n) {
    size_t c = 12;  // 4 KiB at least
    while (((size_t)1 << c) < n) c++;
    return c;
}
void* pin_alloc(size_t n) {
    const size_t c = pin_class(n);
    {
        std::lock_guard<std::mutex> g(pin_pool_mu);
        if (!pin_pool[c].empty()) {
            void* p = pin_pool[c].back();
            pin_pool[c].pop_back();
            return p;
        }
    }
    void* p = nullptr;
    VCK(cudaMallocHost(&p, (size_t)1 << c));
    return p;
}
// n must be the size given to pin_alloc; no copy may still use the block
void pin_free(void* p, size_t n) {
    if (!p) return;
    std::lock_guard<std::mutex> g(pin_pool_mu);
    pin_pool[pin_class(n)].push_back(p);
}

// Pinned staging of host-to-device uploads inside a region (begin .. end):
// a copy from pageable memory can make the host wait until the stream
// reaches it, one from pinned memory never does.  Chunks are reused once the
// event recorded at the end of the previous region has completed.
struct PinArena {
    std::vector<std::pair<uint8_t*, size_t>> chunks;
    size_t ci = 0, off = 0;
    cudaEvent_t ev = nullptr;
    cudaStream_t s = nullptr;
    bool pending = false, on = false;
    void begin(cudaStream_t stream) {
        if (on) VCK(cudaStreamSynchronize(s));  // a region left by an error: its copies may be in flight
        if (pending) VCK(cudaEventSynchronize(ev));
        pending = false;
        on = true;
        ci = off = 0;
        s = stream;
    }
    const void* put(const void* src, size_t n) {
        off = (off + 15) & ~size_t(15);
        while (ci < chunks.size() && off + n > chunks[ci].second) {
            ci++;
            off = 0;
        }
        if (ci == chunks.size()) {
            const size_t sz = std::max<size_t>(n, size_t(1) << 20);
            uint8_t* p = (uint8_t*)pin_alloc(sz);
            chunks.push_back({p, sz});
            off = 0;
        }
        uint8_t* d = chunks[ci].first + off;
        std::memcpy(d, src, n);
        off += n;
        return d;
    }
    void end() {
        if (!on) return;
        on = false;
        if (!ev) VCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        VCK(cudaEventRecord(ev, s));
        pending = true;
    }
    void release() {
        if (on && s) cudaStreamSynchronize(s);
        if (pending && ev) cudaEventSynchronize(ev);
        for (auto& c : chunks) pin_free(c.first, c.second);
        chunks.clear();
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
        pending = on = false;
    }
};

struct DevMem {
    PinArena* pin = nullptr;  // uploads are staged through it while it is on
    const vlbm_allocator* alloc = nullptr;
    vlbm_allocator a{};
    bool has = false;
    cudaStream_t s = nullptr;
    size_t bytes = 0;
    void* get(size_t n) {
        if (n == 0) n = 16;
        n = (n + 255) & ~size_t(255);
        void* p = nullptr;
        if (has) {
            p = a.alloc(n, (void*)s, a.ctx);
            if (!p) throw Fail{VLBM_ERR_OOM, "allocator returned NULL"};
        } else {
            cudaMemPool_t pool = library_pool();
            cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, n, pool, s) : cudaMallocAsync(&p, n, s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                throw Fail{VLBM_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e)};
            }
        }
        bytes += n;
        return p;
    }
    void put(void* p, size_t n) {
        if (!p) return;
        if (n == 0) n = 16;
        n = (n + 255) & ~size_t(255);
        if (has) a.free(p, (void*)s, a.ctx);
        else cudaFreeAsync(p, s);
        bytes -= std::min(bytes, n);
    }
};

template <class T>
struct DArr {
    T* p = nullptr;
    size_t cap = 0;  // elements
    size_t n = 0;
    void ensure(DevMem& m, size_t need) {
        if (need <= cap && p) return;
        if (p) m.put(p, cap * sizeof(T));
        cap = std::max<size_t>(need, 16);
        p = (T*)m.get(cap * sizeof(T));
    }
    void upload(DevMem& m, const std::vector<T>& v, cudaStream_t s) {
        ensure(m, v.size());
        n = v.size();
        if (!n) return;
        const void* src = v.data();
        if (m.pin && m.pin->on) src = m.pin->put(src, n * sizeof(T));
        VCK(cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void release(DevMem& m) {
        if (p) m.put(p, cap * sizeof(T));
        p = nullptr;
        cap = n = 0;
    }
};

struct Level {
    int nx = 0, ny = 0, pitch = 0, bx = 0, by = 0;
    long long plane = 0;
    double* buf[2] = {nullptr, nullptr};
    uint16_t* flags = nullptr;
    uint16_t* flags_tmp = nullptr;
    std::vector<uint8_t> bin, bcov;  // block maps (current layout; host copy, see vlbm_hier::host_ok)
    LayoutDev dl;                      // the layout on the device (always current)
    std::vector<Item> act, ring, cov, in;  // tiles (lid = level index)
    std::vector<uint8_t> recon;             // per tile: a face neighbour is coarser land
    long long active_cells = 0;
};

}  // namespace

struct Batch;

struct vlbm_hier {
    vlbm_config cfg{};
    std::vector<vlbm_box> boxes;
    int nlev = 1;
    double om = 0, hb = 0, bcs = 0, gm1 = 0, hc = 0;
    double feqb[4][16] = {};
    Level lev[VLBM_MAX_LEVELS];
    int* words = nullptr;  // [0] level-0 parity, [1] status
    DevMem mem;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Batch* own = nullptr;
    vlbm_engine* engine = nullptr;
    long long steps = 0;
    bool poisoned = false;
    std::string err = "no error";
    // scratch
    DArr<double> stage;     // W / f staging
    DArr<uint8_t> stage8;   // valid masks
    DArr<unsigned long long> qmax;  // flux-jump sensor: max |Q_k| (bit patterns)
    DArr<unsigned long long> partial;  // audit partial sums (exact, 24 words per block)
    DArr<unsigned> aticket;            // the audit's finishing counter (zero between audits)
    DArr<double> tot;      // audit result
    DArr<Item> listbuf;    // item lists for regrid kernels
    DArr<uint8_t> bflag;   // block flags
    DArr<LevelDev> atab;   // level table for audits (rebuilt with the layout)
    double* hout = nullptr;  // pinned host copy of the audit result
    // tag-driven regrid in two halves: the status words and the block flags
    // land in pinned memory (rg_pin), rg_ev marks their arrival
    PinArena pin;  // staging of the regrids' uploads
    uint8_t* rg_pin = nullptr;
    size_t rg_cap = 0;
    cudaEvent_t rg_ev = nullptr;
    // task-list builds run on aux, after ev_layout (recorded when a device
    // regrid's layout is complete, for layout ev_layout_version); the main
    // stream waits for ev_built before the persistent launch.  The audit
    // before a device regrid runs on aux2, beside the regrid's first part
    // and the build.
    cudaStream_t aux = nullptr, aux2 = nullptr;
    // the side branch of the captured regrid graph (tagging of levels >= 1)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_layout = nullptr, ev_built = nullptr;
    long long ev_layout_version = -1;
    vlbm_tuning tune{1, 0, 8, 1, 2};
    long long layout_steps = 0;  // coarse steps taken on the current layout
    // The layout lives on the device (Level::dl, always current); the host
    // copies (Level::bin, bcov and the tile lists) are current while host_ok.
    // A tag-driven regrid runs on the device alone and clears host_ok; calls
    // that need the host copies fetch them first (ensure_host).
    bool host_ok = true;
    long long layout_version = 0;    // bumped at every layout change
    Item* ditems = nullptr;          // active tiles of every level (audits), length at dcount[0]
    size_t ditems_cap = 0;
    int* dcount = nullptr;           // [0] ditems length
    unsigned long long* lupc = nullptr;  // cell updates done so far
    int** parp = nullptr;                // device array holding `words` (the level-0 parity)
    long long foot_version = -1;         // layout of the last reverse footprints (task builds)
    // exact totals recorded on the device before and after every device
    // regrid (vlbm_set_regrid_audit): ring of RA_CAP rows of 16 doubles
    long long klaunch = 0;  // kernels launched for this hierarchy (vlbm_kernels_launched)
    bool regrid_audit = false;
    double* raud = nullptr;
    long long ra_n = 0, ra_read = 0;
    // ring row whose totals after the regrid are still to come (-1: none):
    // from the first step of the next persistent launch, or from a separate
    // audit before anything else changes the state
    long long after_pending = -1;
    static constexpr long long RA_CAP = 4096;
    // the device regrid, captured in two parts: [0] indicator to new maps
    // and move lists (reads the populations), [1] merge / split, flags and
    // lists (writes them)
    cudaGraphExec_t rg_exec[2] = {nullptr, nullptr};
    std::vector<uintptr_t> rg_key;
    cudaEvent_t ev_rg0 = nullptr, ev_audit = nullptr;
    // Task lists built on the device for the persistent schedule (no
    // per-step audit): [0] one coarse step, [1] tune.graph_steps steps
    struct DevPlan {
        int steps = -1;
        long long version = -1;
        int nphase = 0, nacc = 0;
        DArr<TBPhase> ph;
        DArr<TBAcc> acc;
        DArr<int> acc_beg, acc_pos, off, deps, need, prefix, ctl, big;
        DArr<int2> chunks;
        DArr<Task> tasks;
        DArr<unsigned> done;
        DArr<Segment> seg;
        int task_cap = 0;
        long long dep_cap = 0;
        int build_kernels = 0;  // kernels the last dev_plan call queued (a task list build)
        // audited cyclic list (regrid audits on): the totals after a regrid
        // come from the next launch's first sweeps (see TBPlan::audit)
        bool audit = false;
        bool sensor = false;  // the relaxation sensor's passes are tasks of the list
        int pfirst[4] = {-1, -1, -1, -1};
        DArr<double> aw;
        DArr<int> ascale;
        DArr<int2> arng;
        DArr<unsigned long long> apart;
        // graphs of its persistent launch: [0] one iteration, [1] G iterations
        cudaGraphExec_t exec[2] = {nullptr, nullptr};
        std::vector<uintptr_t> key[2];
    } dp[2];  // [0] the cyclic one-step list the device path runs; [1] a k-step list (self-test)
    // per-phase launches over the device lists: [0] one step, [1] G steps
    struct PhaseGraph {
        cudaGraphExec_t exec = nullptr;
        std::vector<uintptr_t> key;
    } pg[2];
    // per-step conservation totals recorded by vlbm_advance (pinned ring)
    bool step_audit = false;
    double times[VLBM_T_COUNT] = {};  // host-side time, see vlbm_host_times
    // sensor-driven relaxation (vlbm_set_sensor): parameters and, per level,
    // SENS_PLANES planes of the level's index space
    bool sensor_on = false;
    double s_beta_min = 0.5, s_csens = 0.0, s_eps = 0.0, s_iq[4] = {0, 0, 0, 0};
    double* sens[VLBM_MAX_LEVELS] = {};
    double* hist = nullptr;
    long long hist_cap = 4096, hist_n = 0, hist_read = 0;
    // cached task lists of this hierarchy alone: [0] one step, [1] G steps
    struct TaskList {
        std::vector<Task> t;
        std::vector<int> d;
        int steps = -1;
        bool audit = false;
        // device copies (the hierarchy's memory): tasks, dependencies,
        // completion epochs; for the per-step audit the audited moments
        // (AUDIT_SLOT doubles per slot), each slot's weight exponent, the
        // slot range of each reduction block, the blocks' exact partial
        // sums, each step's block range and the per-step totals
        DArr<Task> dt;
        DArr<int> dd;
        DArr<unsigned> done;
        DArr<double> aw;
        DArr<int> ascale;
        DArr<int2> arng;
        DArr<unsigned long long> apart;
        DArr<int> abseg;
        DArr<double> aout;
        int nseg = 0, nblk = 0;
    } tl[2];

    LevelDev dev(int l, int parent, int child) const {
        LevelDev d{};
        const Level& L = lev[l];
        d.buf[0] = L.buf[0];
        d.buf[1] = L.buf[1];
        d.flags = L.flags;
        d.par0 = words;
        d.status = words + 1;
        d.plane = L.plane;
        d.nx = L.nx;
        d.ny = L.ny;
        d.pitch = L.pitch;
        d.level = l;
        d.parent = parent;
        d.child = child;
        d.px = cfg.bc[0] == VLBM_BC_PERIODIC;
        d.py = cfg.bc[2] == VLBM_BC_PERIODIC;
        for (int s = 0; s < 4; s++) d.bc[s] = cfg.bc[s];
        d.om = om;
        d.hb = hb;
        d.bcs = bcs;
        d.gm1 = gm1;
        d.wscale = std::ldexp(1.0, -2 * l);
        std::memcpy(d.feqb, feqb, sizeof feqb);
        d.sens = sensor_on ? sens[l] : nullptr;
        d.beta_max = cfg.beta;
        d.beta_min = s_beta_min;
        d.csens = s_csens;
        d.eps = s_eps;
        d.ninth = 1.0 / 9.0;
        d.c = cfg.c;
        d.rc = 1.0 / cfg.c;
        for (int k = 0; k < 4; k++) d.iq[k] = s_iq[k];
        return d;
    }
    size_t device_bytes() const { return mem.bytes; }
};

// A set of hierarchies advanced together; every phase of the sub-cycle is one
// launch over the tiles of all members.
struct Batch {
    std::vector<vlbm_hier*> members;
    int maxlev = 0;
    DevMem* mem = nullptr;
    DArr<LevelDev> levs;
    DArr<Item> sweep[VLBM_MAX_LEVELS], close[VLBM_MAX_LEVELS];
    DArr<int*> par;
    cudaGraphExec_t exec1 = nullptr, execG = nullptr;
    int G = 8;
    bool sensor = false;  // some member runs the sensor-driven relaxation (per-phase schedule)
    bool valid = false;
    int max_ctas = 0;  // sweep grid cap (0 = one CTA per 4 tiles)
    int variant = 0;   // sweep kernel variant

    void release() {
        if (exec1) cudaGraphExecDestroy(exec1);
        if (execG) cudaGraphExecDestroy(execG);
        exec1 = execG = nullptr;
        for (StageBuf& b : sbufs) {
            if (b.pending) cudaEventSynchronize(b.ev);
            pin_free(b.p, b.cap);
            if (b.ev) cudaEventDestroy(b.ev);
        }
        sbufs.clear();
        scur = -1;
        levs.release(*mem);
        for (int l = 0; l < VLBM_MAX_LEVELS; l++) {
            sweep[l].release(*mem);
            close[l].release(*mem);
        }
        par.release(*mem);
        dsegs.release(*mem);
        doffs.release(*mem);
        dmctl.release(*mem);
        dprefix.release(*mem);
        dctl.release(*mem);
        dchunks.release(*mem);
        for (int w = 0; w < 2; w++) {
            segs[w].release(*mem);
            prefix[w].release(*mem);
            chunks[w].release(*mem);
            ctl[w].release(*mem);
            captured[w].clear();
            seg_ok[w] = false;
        }
        valid = false;
    }

    void schedule(int l, int kk, int kkp, cudaStream_t s) {
        if (sensor) VCK(launch_sensor(levs.p, sweep[l].p, (int)sweep[l].n, kk, s));
        VCK(launch_sweep(levs.p, sweep[l].p, (int)sweep[l].n, kk, kkp, max_ctas, variant, s, sensor));
        if (l + 1 < maxlev && sweep[l + 1].n > 0) {
            schedule(l + 1, 1, kk, s);
            schedule(l + 1, 2, kk, s);
            VCK(launch_close(levs.p, close[l].p, (int)close[l].n, kk, s));
        }
    }

    void one_step(cudaStream_t s) {
        schedule(0, 0, 0, s);
        VCK(launch_end_step(par.p, (int)par.n, s));
    }

    cudaGraphExec_t capture(int nsteps, cudaStream_t s) {
        cudaGraph_t g = nullptr;
        VCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            for (int i = 0; i < nsteps; i++) one_step(s);
        } catch (...) {
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        VCK(cudaStreamEndCapture(s, &g));
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = instantiate(&ex, g);
        cudaGraphDestroy(g);
        VCK(e);
        return ex;
    }

    // rebuilds the tables of all members; graphs are re-captured on use
    void build(cudaStream_t s) {
        if (schedule_mode != 1) {
            if (exec1) cudaGraphExecDestroy(exec1);
            if (execG) cudaGraphExecDestroy(execG);
            exec1 = execG = nullptr;
            for (auto& c : captured) c.clear();
        }
        // sizes first, then every table written once, straight into a pinned
        // staging buffer, and copied from there (no stream synchronisation:
        // the engine's queue keeps running while a batch is rebuilt)
        size_t ntab = 0, nsw[VLBM_MAX_LEVELS] = {}, ncl[VLBM_MAX_LEVELS] = {};
        maxlev = 0;
        sensor = false;
        for (vlbm_hier* h : members) {
            ntab += h->nlev;
            for (int l = 0; l < h->nlev; l++) {
                nsw[l] += h->lev[l].act.size();
                if (l + 1 < h->nlev) ncl[l] += h->lev[l].ring.size();
            }
            maxlev = std::max(maxlev, h->nlev);
            sensor = sensor || h->sensor_on;
        }
        size_t need = ntab * sizeof(LevelDev) + members.size() * sizeof(int*);
        for (int l = 0; l < VLBM_MAX_LEVELS; l++) need += (nsw[l] + ncl[l]) * sizeof(Item);
        stage_begin(need);
        LevelDev* tab = stage_part(levs, ntab);
        int** pw = stage_part(par, members.size());
        Item *sw[VLBM_MAX_LEVELS], *cl[VLBM_MAX_LEVELS];
        for (int l = 0; l < VLBM_MAX_LEVELS; l++) {
            sw[l] = stage_part(sweep[l], nsw[l]);
            cl[l] = stage_part(close[l], ncl[l]);
        }
        int base = 0;
        for (size_t m = 0; m < members.size(); m++) {
            vlbm_hier* h = members[m];
            for (int l = 0; l < h->nlev; l++) {
                *tab++ = h->dev(l, l ? base + l - 1 : -1, l + 1 < h->nlev ? base + l + 1 : -1);
                for (Item it : h->lev[l].act) {
                    it.lid = base + l;
                    *sw[l]++ = it;
                }
                if (l + 1 < h->nlev)
                    for (Item it : h->lev[l].ring) {
                        it.lid = base + l;
                        *cl[l]++ = it;
                    }
            }
            pw[m] = h->words;
            base += h->nlev;
        }
        stage_copies(s);
        stage_end(s);
        // the one-step and G-step graphs (and task lists) are built when first used
        seg_ok[0] = seg_ok[1] = false;
        valid = true;
    }

    // Pinned staging of the table uploads: a small ring of buffers, each
    // reused once the copies queued from it have completed, so that a
    // rebuild never waits for the steps queued on the engine's stream (the
    // copies are ordered after them).
    struct StageBuf {
        char* p = nullptr;
        size_t cap = 0;
        cudaEvent_t ev = nullptr;
        bool pending = false;
    };
    std::vector<StageBuf> sbufs;
    int scur = -1, slast = -1;
    size_t stage_off = 0;
    void stage_begin(size_t need) {
        need += 16 * 256;  // alignment of the parts
        int pick = -1;
        for (int i = 0; i < (int)sbufs.size() && pick < 0; i++) {
            StageBuf& b = sbufs[i];
            if (b.cap < need) continue;
            if (b.pending) {
                const cudaError_t q = cudaEventQuery(b.ev);
                if (q == cudaErrorNotReady) continue;
                VCK(q);
                b.pending = false;
            }
            pick = i;
        }
        if (pick < 0 && sbufs.size() < 8) {
            sbufs.emplace_back();
            pick = (int)sbufs.size() - 1;
        }
        if (pick < 0) {  // all eight in flight: wait for the one after the last used
            pick = (slast + 1) % (int)sbufs.size();
            VCK(cudaEventSynchronize(sbufs[pick].ev));
            sbufs[pick].pending = false;
        }
        StageBuf& b = sbufs[pick];
        if (b.cap < need) {  // idle here
            pin_free(b.p, b.cap);
            b.p = nullptr;
            b.cap = std::max(2 * b.cap, need + (size_t)(1 << 20));
            b.p = (char*)pin_alloc(b.cap);
        }
        if (!b.ev) VCK(cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming));
        scur = pick;
        stage_off = 0;
    }
    template <class T>
    void staged(DArr<T>& d, const std::vector<T>& v, cudaStream_t s) {
        d.ensure(*mem, v.size());
        d.n = v.size();
        const size_t b = v.size() * sizeof(T);
        if (!b) return;
        StageBuf& sb = sbufs[scur];
        const size_t off = (stage_off + 255) & ~size_t(255);
        if (off + b > sb.cap) throw Fail{VLBM_ERR_ARG, "staging buffer too small"};  // sized by the caller
        std::memcpy(sb.p + off, v.data(), b);
        VCK(cudaMemcpyAsync(d.p, sb.p + off, b, cudaMemcpyHostToDevice, s));
        stage_off = off + b;
    }
    // A part of n elements of the current staging buffer for d (resized to
    // n), to be filled by the caller and copied by stage_copies.
    std::vector<std::tuple<void*, size_t, size_t>> stage_pending_copies;
    template <class T>
    T* stage_part(DArr<T>& d, size_t n) {
        d.ensure(*mem, n);
        d.n = n;
        StageBuf& sb = sbufs[scur];
        const size_t off = (stage_off + 255) & ~size_t(255);
        const size_t b = n * sizeof(T);
        if (off + b > sb.cap) throw Fail{VLBM_ERR_ARG, "staging buffer too small"};  // sized by the caller
        stage_off = off + b;
        if (b) stage_pending_copies.emplace_back((void*)d.p, off, b);
        return (T*)(sb.p + off);
    }
    void stage_copies(cudaStream_t s) {
        StageBuf& sb = sbufs[scur];
        for (auto& c : stage_pending_copies)
            VCK(cudaMemcpyAsync(std::get<0>(c), sb.p + std::get<1>(c), std::get<2>(c), cudaMemcpyHostToDevice, s));
        stage_pending_copies.clear();
    }
    void stage_end(cudaStream_t s) {
        StageBuf& sb = sbufs[scur];
        VCK(cudaEventRecord(sb.ev, s));
        sb.pending = true;
        slast = scur;
        scur = -1;
    }

    // eager launches with events around each kernel (profiling)
    struct Rec {
        int kind, level;
        long long launches = 0, cells = 0;
        double ms = 0;
    };
    void timed(int kind, int level, long long cells, std::vector<Rec>& recs, cudaStream_t s,
               const std::function<cudaError_t()>& fn) {
        cudaEvent_t a, b;
        VCK(cudaEventCreate(&a));
        VCK(cudaEventCreate(&b));
        VCK(cudaEventRecord(a, s));
        VCK(fn());
        VCK(cudaEventRecord(b, s));
        VCK(cudaEventSynchronize(b));
        float ms = 0;
        VCK(cudaEventElapsedTime(&ms, a, b));
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        for (Rec& r : recs)
            if (r.kind == kind && r.level == level) {
                r.launches++;
                r.cells += cells;
                r.ms += ms;
                return;
            }
        Rec r;
        r.kind = kind;
        r.level = level;
        r.launches = 1;
        r.cells = cells;
        r.ms = ms;
        recs.push_back(r);
    }
    void schedule_timed(int l, int kk, int kkp, const long long* cells, std::vector<Rec>& recs, cudaStream_t s) {
        if (sweep[l].n)
            timed(0, l, cells[l], recs, s, [&] {
                if (sensor) {
                    cudaError_t e = launch_sensor(levs.p, sweep[l].p, (int)sweep[l].n, kk, s);
                    if (e != cudaSuccess) return e;
                }
                return launch_sweep(levs.p, sweep[l].p, (int)sweep[l].n, kk, kkp, max_ctas, variant, s, sensor);
            });
        if (l + 1 < maxlev && sweep[l + 1].n > 0) {
            schedule_timed(l + 1, 1, kk, cells, recs, s);
            schedule_timed(l + 1, 2, kk, cells, recs, s);
            if (close[l].n)
                timed(1, l, 0, recs, s, [&] { return launch_close(levs.p, close[l].p, (int)close[l].n, kk, s); });
        }
    }
    void profile(long long n, const long long* cells, std::vector<Rec>& recs, cudaStream_t s) {
        for (long long i = 0; i < n; i++) {
            schedule_timed(0, 0, 0, cells, recs, s);
            timed(2, 0, 0, recs, s, [&] { return launch_end_step(par.p, (int)par.n, s); });
        }
    }

    // ---- one persistent launch over every member's device-built list ------
    // (the engine): per call, each member's one-step list (rebuilt on the
    // device when its layout changed), a segment table, and the chunk table
    // that orders the members' tasks phase-major -- every member's phase-p
    // tasks before any member's phase p + 1 -- so that no thread group waits
    // at one small member's phase boundary while others have ready work
    DArr<Segment> dsegs;
    DArr<const int*> doffs, dmctl;
    DArr<int> dprefix, dctl;
    DArr<int2> dchunks;
    void device_steps(long long k, cudaStream_t s);

    // ---- persistent task schedule -----------------------------------------
    int schedule_mode = 1;  // 0: one launch per phase, 1: persistent task kernel
    bool audit = false;     // fused per-step audit (single-member batches)
    // segment tables of the persistent launches: [0] one step, [1] G steps
    DArr<Segment> segs[2];
    DArr<int> prefix[2];
    DArr<int2> chunks[2];
    DArr<int> ctl[2];
    int ntotal[2] = {0, 0};
    bool seg_ok[2] = {false, false};
    // everything a captured task graph holds by value (pointers, sizes,
    // grid), so that it is re-captured exactly when one of them changes
    std::vector<uintptr_t> captured[2];
    std::vector<uintptr_t> launch_key(int which) const;

    // Task list of one hierarchy alone (local level indices), cached and
    // uploaded to the hierarchy's memory until its layout, its steps per
    // launch or its audit setting change.
    void member_tasks(vlbm_hier* h, int which, int nsteps, bool aud);

    // Segment table of a persistent launch over all members.
    void build_segments(int which, int nsteps, cudaStream_t s);
    DevMem* mem_ptr() { return mem; }

    void task_launch(int which, cudaStream_t s) {
        VCK(cudaMemsetAsync(ctl[which].p, 0, 2 * sizeof(int), s));  // claim and finish counters
        VCK(launch_tasks(levs.p, segs[which].p, prefix[which].p, chunks[which].p, ctl[which].p, variant, max_ctas, 1,
                         s));
        if (audit && members.size() == 1) {
            auto& T = members[0]->tl[which];
            VCK(launch_audit_segments(T.apart.p, T.abseg.p, T.nseg, T.aout.p, s));
        }
    }

    cudaGraphExec_t capture_tasks(int which, cudaStream_t s) {
        cudaGraph_t g = nullptr;
        VCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        try {
            task_launch(which, s);
        } catch (...) {
            cudaStreamEndCapture(s, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        VCK(cudaStreamEndCapture(s, &g));
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = instantiate(&ex, g);
        cudaGraphDestroy(g);
        VCK(e);
        return ex;
    }

    // The graph of one step (which = 0) or of G steps (which = 1), with its
    // task lists built and captured on first use.
    cudaGraphExec_t exec_for(int which, cudaStream_t s);

    long long* klaunch = nullptr;  // kernel counter of the batch's hierarchy (own batches)
    void count(cudaGraphExec_t ex) {
        if (klaunch) *klaunch += graph_kernels(ex);
    }
    void advance(long long n, cudaStream_t s) {
        if (n >= G) {
            cudaGraphExec_t ex = exec_for(1, s);
            for (; n >= G; n -= G) {
                VCK(cudaGraphLaunch(ex, s));
                count(ex);
            }
        }
        if (n > 0) {
            cudaGraphExec_t ex = exec_for(0, s);
            for (; n > 0; n--) {
                VCK(cudaGraphLaunch(ex, s));
                count(ex);
            }
        }
    }
};

void Batch::member_tasks(vlbm_hier* h, int which, int nsteps, bool aud) {
    vlbm_hier::TaskList& L = h->tl[which];
    if (L.steps == nsteps && L.audit == aud) return;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<TaskLevel> lv(h->nlev);
    for (int l = 0; l < h->nlev; l++) {
        const Level& HL = h->lev[l];
        lv[l].nx = HL.nx;
        lv[l].ny = HL.ny;
        lv[l].bx = HL.bx;
        lv[l].by = HL.by;
        lv[l].px = h->cfg.bc[0] == VLBM_BC_PERIODIC;
        lv[l].py = h->cfg.bc[2] == VLBM_BC_PERIODIC;
        lv[l].act = &HL.act;
        lv[l].ring = &HL.ring;
        lv[l].recon = &HL.recon;
    }
    TaskLists tl;
    build_tasks(lv, nsteps, tl);
    L.t.swap(tl.t);
    L.d.swap(tl.d);
    // audit slots, reduction blocks and their tasks
    std::vector<int> scale, bseg;
    std::vector<int2> rng;
    const int nslots = assign_audit(L.t, L.d, nsteps, aud ? AUDIT_BLOCK_SLOTS : 0, scale, rng, bseg, AUDIT_LAG);
    cudaStream_t s = h->stream;
    L.dt.upload(h->mem, L.t, s);
    std::vector<int> d = L.d;
    if (d.empty()) d.push_back(0);
    L.dd.upload(h->mem, d, s);
    L.done.ensure(h->mem, std::max<size_t>(1, L.t.size()));
    if (aud) {
        L.nseg = nsteps;
        L.nblk = (int)rng.size();
        L.aw.ensure(h->mem, (size_t)std::max(1, nslots) * AUDIT_SLOT);
        L.ascale.upload(h->mem, scale, s);
        if (rng.empty()) rng.push_back(make_int2(0, 0));
        L.arng.upload(h->mem, rng, s);
        L.apart.ensure(h->mem, (size_t)std::max(1, L.nblk) * 24);
        L.abseg.upload(h->mem, bseg, s);
        L.aout.ensure(h->mem, (size_t)nsteps * 8);
    } else {
        L.nseg = L.nblk = 0;
    }
    VCK(cudaStreamSynchronize(s));
    L.steps = nsteps;
    L.audit = aud;
    h->times[VLBM_T_TASKS] += ms_since(t0);
    h->times[VLBM_T_NTASKLISTS] += 1;
}

std::vector<uintptr_t> Batch::launch_key(int which) const {
    std::vector<uintptr_t> k = {(uintptr_t)levs.p, (uintptr_t)segs[which].p, (uintptr_t)prefix[which].p,
                                (uintptr_t)chunks[which].p, (uintptr_t)ctl[which].p, (uintptr_t)variant,
                                (uintptr_t)max_ctas,
                                (uintptr_t)(audit && members.size() == 1)};
    if (audit && members.size() == 1) {
        const auto& T = members[0]->tl[which];
        for (uintptr_t v : {(uintptr_t)T.aw.p, (uintptr_t)T.arng.p, (uintptr_t)T.ascale.p, (uintptr_t)T.nblk,
                            (uintptr_t)T.apart.p, (uintptr_t)T.abseg.p, (uintptr_t)T.nseg, (uintptr_t)T.aout.p})
            k.push_back(v);
    }
    return k;
}

cudaGraphExec_t Batch::exec_for(int which, cudaStream_t s) {
    cudaGraphExec_t& ex = which ? execG : exec1;
    if (schedule_mode != 1) {
        if (!ex) ex = capture(which ? G : 1, s);
        return ex;
    }
    if (!seg_ok[which]) {
        build_segments(which, which ? G : 1, s);
        seg_ok[which] = true;
    }
    std::vector<uintptr_t> key = launch_key(which);
    if (!ex || key != captured[which]) {
        const auto t0 = std::chrono::steady_clock::now();
        if (ex) cudaGraphExecDestroy(ex);
        ex = nullptr;
        captured[which].clear();
        ex = capture_tasks(which, s);
        captured[which] = key;
        for (vlbm_hier* h : members) h->times[VLBM_T_CAPTURE] += ms_since(t0) / (double)members.size();
    }
    return ex;
}

void Batch::build_segments(int which, int nsteps, cudaStream_t s) {
    const bool aud = audit && members.size() == 1;
    std::vector<Segment> sg;
    std::vector<int> pre(1, 0);
    int base = 0;
    for (vlbm_hier* h : members) {
        member_tasks(h, which, nsteps, aud);
        vlbm_hier::TaskList& L = h->tl[which];
        // completion marks restart with this batch's epochs
        VCK(cudaMemsetAsync(L.done.p, 0, std::max<size_t>(1, L.t.size()) * sizeof(unsigned), s));
        Segment S{};
        S.tasks = L.dt.p;
        S.deps = L.dd.p;
        S.done = L.done.p;
        S.aw = aud ? L.aw.p : nullptr;
        S.arng = aud ? L.arng.p : nullptr;
        S.ascale = aud ? L.ascale.p : nullptr;
        S.apart = aud ? L.apart.p : nullptr;
        S.par0 = h->words;
        S.ntasks = (int)L.t.size();
        S.lid_base = base;
        sg.push_back(S);
        pre.push_back(pre.back() + S.ntasks);
        base += h->nlev;
    }
    if (sg.empty()) {
        sg.push_back(Segment{});
        pre.push_back(0);
    }
    ntotal[which] = pre.back();
    std::vector<int> c(CTL_WORDS, 0);
    c[CTL_EPOCH] = 1;
    c[CTL_TOTAL] = pre.back();
    c[CTL_NSEG] = (int)members.size();
    c[CTL_FLIP] = nsteps & 1;
    c[CTL_NCHUNK] = (int)sg.size();  // one chunk per segment: member by member
    c[CTL_AUDIT] = 1;                // a segment with audit slots audits every launch (one-pass lists)
    std::vector<int2> ch(sg.size());
    for (size_t m = 0; m < sg.size(); m++) ch[m] = make_int2((int)m, 0);
    // pinned staging: the engine's queued steps keep running meanwhile
    stage_begin(sg.size() * sizeof(Segment) + (pre.size() + c.size()) * sizeof(int) + ch.size() * sizeof(int2));
    staged(segs[which], sg, s);
    staged(prefix[which], pre, s);
    staged(ctl[which], c, s);
    staged(chunks[which], ch, s);
    stage_end(s);
}

namespace {

// ---- layouts ----------------------------------------------------------------

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// in-maps of levels >= 1 from the covered maps (children of covered blocks)
void derive_in(vlbm_hier* h, std::vector<uint8_t>* bin, const std::vector<uint8_t>* bcov) {
    for (int l = 0; l < h->nlev; l++) {
        Level& L = h->lev[l];
        bin[l].assign((size_t)L.bx * L.by, l == 0 ? 1 : 0);
        if (l == 0) continue;
        const Level& P = h->lev[l - 1];
        for (int jb = 0; jb < L.by; jb++)
            for (int ib = 0; ib < L.bx; ib++) {
                const size_t pb = (size_t)(jb >> 1) * P.bx + (ib >> 1);
                bin[l][(size_t)jb * L.bx + ib] = bin[l - 1][pb] && bcov[l - 1][pb];
            }
    }
}

// Proper nesting: covered blocks lie on their level, none on the finest
// level, and on levels >= 1 every covered block's four face-neighbour blocks
// (inside the domain) are on the level.
bool nested(vlbm_hier* h, const std::vector<uint8_t>* bin, const std::vector<uint8_t>* bcov, std::string& why) {
    const bool px = h->cfg.bc[0] == VLBM_BC_PERIODIC, py = h->cfg.bc[2] == VLBM_BC_PERIODIC;
    for (int l = 0; l < h->nlev; l++) {
        const Level& L = h->lev[l];
        for (int jb = 0; jb < L.by; jb++)
            for (int ib = 0; ib < L.bx; ib++) {
                const size_t b = (size_t)jb * L.bx + ib;
                if (!bcov[l][b]) continue;
                if (l == h->nlev - 1) { why = "finest level cannot be refined"; return false; }
                if (!bin[l][b]) { why = "refined block outside its level (level " + std::to_string(l) + ")"; return false; }
                if (l == 0) continue;
                const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
                for (int d = 0; d < 4; d++) {
                    int i2 = ib + di[d], j2 = jb + dj[d];
                    if (i2 < 0 || i2 >= L.bx) { if (!px) continue; i2 = (i2 + L.bx) % L.bx; }
                    if (j2 < 0 || j2 >= L.by) { if (!py) continue; j2 = (j2 + L.by) % L.by; }
                    if (!bin[l][(size_t)j2 * L.bx + i2]) {
                        why = "level " + std::to_string(l + 1) + " touches level " + std::to_string(l - 1);
                        return false;
                    }
                }
            }
    }
    return true;
}

void boxes_to_maps(vlbm_hier* h, const vlbm_box* boxes, int nboxes, std::vector<uint8_t>* bcov) {
    for (int l = 0; l < h->nlev; l++) bcov[l].assign((size_t)h->lev[l].bx * h->lev[l].by, 0);
    for (int b = 0; b < nboxes; b++) {
        const vlbm_box& x = boxes[b];
        if (x.level < 0 || x.level >= h->nlev) throw Fail{VLBM_ERR_ARG, "box level out of range"};
        const Level& L = h->lev[x.level];
        if (x.ni <= 0 || x.nj <= 0 || x.i0 < 0 || x.j0 < 0 || x.i0 + x.ni > L.nx || x.j0 + x.nj > L.ny)
            throw Fail{VLBM_ERR_ARG, "box outside the level"};
        auto aligned = [](int a, int n) { return a % TILE == 0 || a == n; };
        if (!aligned(x.i0, L.nx) || !aligned(x.j0, L.ny) || !aligned(x.i0 + x.ni, L.nx) || !aligned(x.j0 + x.nj, L.ny))
            throw Fail{VLBM_ERR_ARG, "box not aligned to 8-cell blocks"};
        if (x.level == h->nlev - 1) throw Fail{VLBM_ERR_NESTING, "finest level cannot be refined"};
        for (int j = x.j0 / TILE; j < ceil_div(x.j0 + x.nj, TILE); j++)
            for (int i = x.i0 / TILE; i < ceil_div(x.i0 + x.ni, TILE); i++) bcov[x.level][(size_t)j * L.bx + i] = 1;
    }
}

void masks_to_maps(vlbm_hier* h, const uint8_t* const* ref, std::vector<uint8_t>* bcov) {
    for (int l = 0; l < h->nlev; l++) {
        const Level& L = h->lev[l];
        bcov[l].assign((size_t)L.bx * L.by, 0);
        if (l == h->nlev - 1 || !ref || !ref[l]) continue;
        for (int jb = 0; jb < L.by; jb++)
            for (int ib = 0; ib < L.bx; ib++) {
                int ones = 0, cells = 0;
                for (int y = jb * TILE; y < std::min(L.ny, jb * TILE + TILE); y++)
                    for (int x = ib * TILE; x < std::min(L.nx, ib * TILE + TILE); x++) {
                        cells++;
                        ones += ref[l][(size_t)y * L.nx + x] ? 1 : 0;
                    }
                if (ones != 0 && ones != cells) throw Fail{VLBM_ERR_ARG, "refinement mask not aligned to 8-cell blocks"};
                bcov[l][(size_t)jb * L.bx + ib] = ones ? 1 : 0;
            }
    }
}

// Layout rule for adaptive regrids, on blocks: bflag[l] marks the blocks
// that hold a tagged cell within `buffer` cells; from the finest refinable
// level down, add the blocks holding the parents of the 8-neighbourhood of
// the next finer refined set (proper nesting).
void layout_rule(vlbm_hier* h, const std::vector<uint8_t>* bflag, std::vector<uint8_t>* bcov) {
    const bool px = h->cfg.bc[0] == VLBM_BC_PERIODIC, py = h->cfg.bc[2] == VLBM_BC_PERIODIC;
    for (int l = h->nlev - 1; l >= 0; l--) {
        Level& L = h->lev[l];
        bcov[l].assign((size_t)L.bx * L.by, 0);
        if (l == h->nlev - 1) continue;
        for (size_t b = 0; b < bcov[l].size(); b++) bcov[l][b] = bflag[l][b];
        if (l + 1 <= h->nlev - 2) {
            const Level& C = h->lev[l + 1];
            for (int jb = 0; jb < C.by; jb++)
                for (int ib = 0; ib < C.bx; ib++) {
                    if (!bcov[l + 1][(size_t)jb * C.bx + ib]) continue;
                    // the block's cells on level l+1, widened by one cell
                    const int x0 = ib * TILE - 1, x1 = std::min(C.nx, ib * TILE + TILE) + 1;
                    const int y0 = jb * TILE - 1, y1 = std::min(C.ny, jb * TILE + TILE) + 1;
                    for (int y = y0; y < y1; y++) {
                        int yy = y;
                        if (yy < 0 || yy >= C.ny) { if (!py) continue; yy = (yy + C.ny) % C.ny; }
                        for (int x = x0; x < x1; x++) {
                            int xx = x;
                            if (xx < 0 || xx >= C.nx) { if (!px) continue; xx = (xx + C.nx) % C.nx; }
                            const int cxp = xx >> 1, cyp = yy >> 1;  // parent cell on level l
                            bcov[l][(size_t)(cyp / TILE) * L.bx + cxp / TILE] = 1;
                        }
                    }
                }
        }
    }
}

void build_lists(vlbm_hier* h) {
    const bool px = h->cfg.bc[0] == VLBM_BC_PERIODIC, py = h->cfg.bc[2] == VLBM_BC_PERIODIC;
    for (int l = 0; l < h->nlev; l++) {
        Level& L = h->lev[l];
        TileLists o;
        tile_lists(l, L.nx, L.ny, L.bx, L.by, px, py, L.bin.data(), L.bcov.data(), o);
        L.act.swap(o.act);
        L.ring.swap(o.ring);
        L.cov.swap(o.cov);
        L.in.swap(o.in);
        L.recon.swap(o.recon);
        L.active_cells = o.active_cells;
    }
}

LevelDev lvdev(vlbm_hier* h, int l) { return h->dev(l, -1, -1); }

constexpr int LISTS_ALL = (1 << LST_ACT) | (1 << LST_RING) | (1 << LST_COV) | (1 << LST_IN);
constexpr int LISTS_MOVE = (1 << LST_EXIT) | (1 << LST_ENTER) | (1 << LST_TOUCH);

int lcap(const LayoutDev& D) { return D.bx * D.by; }

// The hierarchy's level table (parent / child links) as the kernels see it.
void refresh_atab(vlbm_hier* h) {
    std::vector<LevelDev> tab;
    for (int l = 0; l < h->nlev; l++) tab.push_back(h->dev(l, l ? l - 1 : -1, l + 1 < h->nlev ? l + 1 : -1));
    h->atab.upload(h->mem, tab, h->stream);
}

void layout_changed(vlbm_hier* h) {
    h->layout_version++;
    h->tl[0].steps = h->tl[1].steps = -1;
    h->layout_steps = 0;
}

// The device lists of every level from the current device maps, and the
// concatenated active tiles of the audits.
void device_lists(vlbm_hier* h) {
    LayoutDev dls[VLBM_MAX_LEVELS];
    const LayoutDev* lp[VLBM_MAX_LEVELS];
    int masks[VLBM_MAX_LEVELS];
    for (int l = 0; l < h->nlev; l++) {
        dls[l] = h->lev[l].dl;
        lp[l] = &h->lev[l].dl;
        masks[l] = LISTS_ALL;
    }
    VCK(launch_lists(lp, masks, h->nlev, h->stream));
    VCK(launch_concat_act(dls, h->nlev, h->ditems, h->dcount, h->stream));
}

void upload_bytes(vlbm_hier* h, void* dst, const void* src, size_t n) {
    if (!n) return;
    if (h->pin.on) src = h->pin.put(src, n);
    VCK(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, h->stream));
}

// Installs new block maps: uploads them, rebuilds the per-cell flags (old
// flags decide which faces are new) and the tile lists, on the host and on
// the device.
void install_layout(vlbm_hier* h, std::vector<uint8_t>* bin, std::vector<uint8_t>* bcov) {
    cudaStream_t s = h->stream;
    for (int l = 0; l < h->nlev; l++) {
        Level& L = h->lev[l];
        L.bin = bin[l];
        L.bcov = bcov[l];
        upload_bytes(h, L.dl.bin, L.bin.data(), L.bin.size());
        upload_bytes(h, L.dl.bcov, L.bcov.data(), L.bcov.size());
        VCK(launch_flags(lvdev(h, l), L.dl.bin, L.dl.bcov, L.flags, L.flags_tmp, s));
        std::swap(L.flags, L.flags_tmp);
    }
    build_lists(h);
    h->host_ok = true;
    layout_changed(h);
    device_lists(h);
    refresh_atab(h);
}

// The host copies of the layout (maps and tile lists), fetched from the
// device after a regrid that ran there.  Synchronises the stream.
void ensure_host(vlbm_hier* h) {
    if (h->host_ok) return;
    VCK(cudaStreamSynchronize(h->stream));
    for (int l = 0; l < h->nlev; l++) {
        Level& L = h->lev[l];
        const size_t nb = (size_t)L.bx * L.by;
        L.bin.resize(nb);
        L.bcov.resize(nb);
        VCK(cudaMemcpy(L.bin.data(), L.dl.bin, nb, cudaMemcpyDeviceToHost));
        VCK(cudaMemcpy(L.bcov.data(), L.dl.bcov, nb, cudaMemcpyDeviceToHost));
    }
    build_lists(h);
    h->host_ok = true;
    h->tl[0].steps = h->tl[1].steps = -1;
    if (h->own) h->own->valid = false;
}

// Device layout of level l: block maps, lists and their lengths, sized for
// the whole level.
void alloc_layout(vlbm_hier* h, int l) {
    Level& L = h->lev[l];
    LayoutDev& D = L.dl;
    D.nx = L.nx;
    D.ny = L.ny;
    D.bx = L.bx;
    D.by = L.by;
    D.px = h->cfg.bc[0] == VLBM_BC_PERIODIC;
    D.py = h->cfg.bc[2] == VLBM_BC_PERIODIC;
    D.level = l;
    const size_t nb = (size_t)L.bx * L.by;
    D.nchunk = (int)((nb + LAY_CHUNK - 1) / LAY_CHUNK);
    cudaStream_t s = h->stream;
    D.bin = (uint8_t*)h->mem.get(nb);
    D.bcov = (uint8_t*)h->mem.get(nb);
    D.nin = (uint8_t*)h->mem.get(nb);
    D.ncov = (uint8_t*)h->mem.get(nb);
    D.recon = (uint8_t*)h->mem.get(nb);
    D.act_idx = (int*)h->mem.get(nb * sizeof(int));
    D.ring_idx = (int*)h->mem.get(nb * sizeof(int));
    if (l + 1 < h->nlev) {
        D.fcnt = (int*)h->mem.get(nb * sizeof(int));
        D.fidx = (int*)h->mem.get(nb * FOOT_CAP * sizeof(int));
        VCK(cudaMemsetAsync(D.fcnt, 0, nb * sizeof(int), s));
    }
    for (int k = 0; k < NLST; k++) D.list[k] = (Item*)h->mem.get(nb * sizeof(Item));
    D.cnt = (int*)h->mem.get(NLST * sizeof(int));
    D.cells = (unsigned long long*)h->mem.get(sizeof(unsigned long long));
    D.chunk = (int*)h->mem.get((size_t)NLST * D.nchunk * sizeof(int));
    for (uint8_t* m : {D.bin, D.bcov, D.nin, D.ncov, D.recon}) VCK(cudaMemsetAsync(m, 0, nb, s));
    VCK(cudaMemsetAsync(D.act_idx, 0xff, nb * sizeof(int), s));
    VCK(cudaMemsetAsync(D.ring_idx, 0xff, nb * sizeof(int), s));
    VCK(cudaMemsetAsync(D.cnt, 0, NLST * sizeof(int), s));
    VCK(cudaMemsetAsync(D.cells, 0, sizeof(unsigned long long), s));
}

void free_layout(vlbm_hier* h, int l) {
    Level& L = h->lev[l];
    LayoutDev& D = L.dl;
    if (!D.bin) return;
    const size_t nb = (size_t)L.bx * L.by;
    for (uint8_t* m : {D.bin, D.bcov, D.nin, D.ncov, D.recon}) h->mem.put(m, nb);
    h->mem.put(D.act_idx, nb * sizeof(int));
    h->mem.put(D.ring_idx, nb * sizeof(int));
    if (D.fcnt) {
        h->mem.put(D.fcnt, nb * sizeof(int));
        h->mem.put(D.fidx, nb * FOOT_CAP * sizeof(int));
    }
    for (int k = 0; k < NLST; k++) h->mem.put(D.list[k], nb * sizeof(Item));
    h->mem.put(D.cnt, NLST * sizeof(int));
    h->mem.put(D.cells, sizeof(unsigned long long));
    h->mem.put(D.chunk, (size_t)NLST * D.nchunk * sizeof(int));
    D = LayoutDev{};
}

void check_status(vlbm_hier* h) {
    int st[2] = {0, 0};
    VCK(cudaMemcpyAsync(st, h->words, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    VCK(cudaStreamSynchronize(h->stream));
    if (st[1] & ST_NONPHYS) throw Fail{VLBM_ERR_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or NaN)"};
    if (st[1] & ST_TIMEOUT) throw Fail{VLBM_ERR_TIMEOUT, "a bounded device wait timed out"};
    if (st[1] & ST_NESTING) throw Fail{VLBM_ERR_NESTING, "a layout computed on the device is not properly nested"};
    if (st[1] & ST_TASKCAP) throw Fail{VLBM_ERR_OOM, "a task list built on the device did not fit its buffers"};
}

// Conservative regrid to the covered maps newcov (Sec. 3.4, Fig. 2).
void regrid_to(vlbm_hier* h, std::vector<uint8_t>* newcov, bool averaged) {
    ensure_host(h);
    cudaStream_t s = h->stream;
    std::vector<uint8_t> newin[VLBM_MAX_LEVELS];
    derive_in(h, newin, newcov);
    std::string why;
    if (!nested(h, newin, newcov, why)) throw Fail{VLBM_ERR_NESTING, why};
    h->pin.begin(s);  // the uploads below come from pinned staging
    // 1. average-down, finest level first (merge values and slope data)
    // (one stream: each upload into listbuf is ordered after the kernel that
    // read the previous list, so no host synchronisation is needed)
    if (!averaged)
        for (int l = h->nlev - 2; l >= 0; l--) {
            h->listbuf.upload(h->mem, h->lev[l].cov, s);
            VCK(launch_avgdown(lvdev(h, l), lvdev(h, l + 1), h->listbuf.p, (int)h->listbuf.n, s));
        }
    // 2. merge: cells covered before and not now
    for (int l = h->nlev - 2; l >= 0; l--) {
        Level& L = h->lev[l];
        std::vector<Item> ex;
        for (const Item& it : L.cov) {
            const size_t b = (size_t)it.ty * L.bx + it.tx;
            if (!(newin[l][b] && newcov[l][b])) ex.push_back(it);
        }
        h->listbuf.upload(h->mem, ex, s);
        VCK(launch_merge(lvdev(h, l), h->listbuf.p, (int)ex.size(), s));
    }
    // 3. split: cells covered now and not before, coarsest level first
    for (int l = 0; l <= h->nlev - 2; l++) {
        Level& L = h->lev[l];
        std::vector<Item> en;
        for (int jb = 0; jb < L.by; jb++)
            for (int ib = 0; ib < L.bx; ib++) {
                const size_t b = (size_t)jb * L.bx + ib;
                if (newin[l][b] && newcov[l][b] && !(L.bin[b] && L.bcov[b]))
                    en.push_back(Item{l, (unsigned short)ib, (unsigned short)jb});
            }
        h->listbuf.upload(h->mem, en, s);
        VCK(launch_split(lvdev(h, l), lvdev(h, l + 1), h->listbuf.p, (int)en.size(), s));
    }
    install_layout(h, newin, newcov);
    h->pin.end();
}

// Tag-driven regrid (Sec. 3.4), first half, queued on h->stream:
// average-down, the sensor on every refinable level, the block flags, and
// their copy -- with the hierarchy's status words -- into pinned host
// memory; h->rg_ev completes when they have arrived.  Nothing waits here.
void tag_begin(vlbm_hier* h) {
    if (!(h->cfg.tag_tol > 0.0) || h->cfg.tag_buffer < 0) throw Fail{VLBM_ERR_ARG, "no tagging parameters"};
    if (h->cfg.tag_sensor != VLBM_SENSOR_DENSITY && h->cfg.tag_sensor != VLBM_SENSOR_FLUX)
        throw Fail{VLBM_ERR_ARG, "unknown tagging sensor"};
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = h->stream;
    h->pin.begin(s);  // the uploads below come from pinned staging
    for (int l = h->nlev - 2; l >= 0; l--) {
        h->listbuf.upload(h->mem, h->lev[l].cov, s);
        VCK(launch_avgdown(lvdev(h, l), lvdev(h, l + 1), h->listbuf.p, (int)h->listbuf.n, s));
    }
    const double tol2 = h->cfg.tag_tol * h->cfg.tag_tol;
    const bool fluxs = h->cfg.tag_sensor == VLBM_SENSOR_FLUX;
    if (fluxs) {
        // the flux maxima over every cell of every level
        h->qmax.ensure(h->mem, 4);
        VCK(cudaMemsetAsync(h->qmax.p, 0, 4 * sizeof(unsigned long long), s));
        for (int l = 0; l < h->nlev; l++) {
            h->listbuf.upload(h->mem, h->lev[l].in, s);
            VCK(launch_qmax(lvdev(h, l), h->listbuf.p, (int)h->listbuf.n, h->qmax.p, s));
        }
    }
    size_t nb = 0;
    for (int l = 0; l <= h->nlev - 2; l++) nb += (size_t)h->lev[l].bx * h->lev[l].by;
    h->bflag.ensure(h->mem, std::max<size_t>(1, nb));
    VCK(cudaMemsetAsync(h->bflag.p, 0, nb, s));
    size_t off = 0;
    for (int l = 0; l <= h->nlev - 2; l++) {
        Level& L = h->lev[l];
        h->listbuf.upload(h->mem, L.in, s);
        const BlockMaps M{L.dl.bin, L.dl.bcov};
        if (fluxs)
            VCK(launch_tag_flux(lvdev(h, l), M, h->listbuf.p, (int)L.in.size(), h->qmax.p, h->cfg.tag_tol,
                                h->cfg.tag_buffer, h->bflag.p + off, s));
        else
            VCK(launch_tag(lvdev(h, l), M, h->listbuf.p, (int)L.in.size(), tol2, h->cfg.tag_buffer, h->bflag.p + off,
                           s));
        off += (size_t)L.bx * L.by;
    }
    // status words first (8 bytes), then the flags
    if (h->rg_cap < 8 + nb) {
        if (h->rg_pin) {
            if (h->rg_ev) VCK(cudaEventSynchronize(h->rg_ev));  // a copy into the old buffer may be in flight
            pin_free(h->rg_pin, h->rg_cap);
            h->rg_pin = nullptr;
            h->rg_cap = 0;
        }
        h->rg_pin = (uint8_t*)pin_alloc(8 + nb);
        h->rg_cap = 8 + nb;
    }
    if (!h->rg_ev) VCK(cudaEventCreateWithFlags(&h->rg_ev, cudaEventDisableTiming));
    VCK(cudaMemcpyAsync(h->rg_pin, h->words, 8, cudaMemcpyDeviceToHost, s));
    if (nb) VCK(cudaMemcpyAsync(h->rg_pin + 8, h->bflag.p, nb, cudaMemcpyDeviceToHost, s));
    h->pin.end();
    VCK(cudaEventRecord(h->rg_ev, s));
    h->times[VLBM_T_TAG] += ms_since(t0);
}

// Second half, once h->rg_ev has completed: the status check, the layout
// rule on the block flags, and the conservative regrid (queued on h->stream).
void tag_finish(vlbm_hier* h) {
    int st[2];
    std::memcpy(st, h->rg_pin, sizeof st);
    if (st[1] & ST_NONPHYS) throw Fail{VLBM_ERR_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or NaN)"};
    if (st[1] & ST_TIMEOUT) throw Fail{VLBM_ERR_TIMEOUT, "a bounded device wait timed out"};
    auto t0 = std::chrono::steady_clock::now();
    std::vector<uint8_t> bflag[VLBM_MAX_LEVELS], bcov[VLBM_MAX_LEVELS];
    size_t off = 0;
    for (int l = 0; l <= h->nlev - 2; l++) {
        const size_t n = (size_t)h->lev[l].bx * h->lev[l].by;
        bflag[l].assign(h->rg_pin + 8 + off, h->rg_pin + 8 + off + n);
        off += n;
    }
    layout_rule(h, bflag, bcov);
    h->times[VLBM_T_LAYOUT] += ms_since(t0);
    t0 = std::chrono::steady_clock::now();
    regrid_to(h, bcov, true);
    h->times[VLBM_T_REGRID] += ms_since(t0);
}

// ---- the adaptive regrid on the device (Sec. 3.4, Fig. 2) --------------------

// Indicator and block flags of every refinable level into h->bflag (level l
// at offset sum_{m < l} bx_m by_m), from the composite state.
void check_tagging(const vlbm_hier* h) {
    if (!(h->cfg.tag_tol > 0.0) || h->cfg.tag_buffer < 0) throw Fail{VLBM_ERR_ARG, "no tagging parameters"};
    if (h->cfg.tag_sensor != VLBM_SENSOR_DENSITY && h->cfg.tag_sensor != VLBM_SENSOR_FLUX)
        throw Fail{VLBM_ERR_ARG, "unknown tagging sensor"};
}

// The scratch of a device regrid at its final size (allocated outside any
// stream capture).
void regrid_buffers(vlbm_hier* h) {
    size_t nb = 0;
    for (int l = 0; l <= h->nlev - 2; l++) nb += (size_t)h->lev[l].bx * h->lev[l].by;
    h->bflag.ensure(h->mem, std::max<size_t>(1, nb));
    h->qmax.ensure(h->mem, 4);
}

void device_tags(vlbm_hier* h) {
    check_tagging(h);
    cudaStream_t s = h->stream;
    const int nl = h->nlev;
    const bool fluxs = h->cfg.tag_sensor == VLBM_SENSOR_FLUX;
    size_t nb = 0;
    for (int l = 0; l <= nl - 2; l++) nb += (size_t)h->lev[l].bx * h->lev[l].by;
    h->bflag.ensure(h->mem, std::max<size_t>(1, nb));
    VCK(cudaMemsetAsync(h->bflag.p, 0, nb, s));
    const double tol2 = h->cfg.tag_tol * h->cfg.tag_tol;
    size_t off[VLBM_MAX_LEVELS] = {};
    for (int l = 1; l <= nl - 2; l++) off[l] = off[l - 1] + (size_t)h->lev[l - 1].bx * h->lev[l - 1].by;
    auto tag = [&](int l, cudaStream_t st) {
        const LayoutDev& D = h->lev[l].dl;
        VCK(launch_tag(lvdev(h, l), BlockMaps{D.bin, D.bcov}, D.list[LST_IN], lcap(D), tol2, h->cfg.tag_buffer,
                       h->bflag.p + off[l], st, D.cnt + LST_IN));
    };
    // composite state: the average of the children in every covered cell,
    // finest level first.  With the density indicator a level l >= 1 is
    // tagged on the side stream as soon as its composite state is complete,
    // beside the averaging and tagging of the coarser levels (a fork and a
    // join of the captured graph).
    bool forked = false;
    for (int l = nl - 2; l >= 0; l--) {
        const LayoutDev& D = h->lev[l].dl;
        VCK(launch_avgdown(lvdev(h, l), lvdev(h, l + 1), D.list[LST_COV], lcap(D), s, D.cnt + LST_COV));
        if (!fluxs && l >= 1) {
            VCK(cudaEventRecord(h->ev_fork, s));
            VCK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            tag(l, h->side);
            forked = true;
        }
    }
    if (!fluxs) {
        tag(0, s);
        if (forked) {
            VCK(cudaEventRecord(h->ev_join, h->side));
            VCK(cudaStreamWaitEvent(s, h->ev_join, 0));
        }
        return;
    }
    // the flux-jump indicator: the flux maxima over every level first
    h->qmax.ensure(h->mem, 4);
    VCK(cudaMemsetAsync(h->qmax.p, 0, 4 * sizeof(unsigned long long), s));
    for (int l = 0; l < nl; l++) {
        const LayoutDev& D = h->lev[l].dl;
        VCK(launch_qmax(lvdev(h, l), D.list[LST_IN], lcap(D), h->qmax.p, s, D.cnt + LST_IN));
    }
    for (int l = 0; l <= nl - 2; l++) {
        const LayoutDev& D = h->lev[l].dl;
        VCK(launch_tag_flux(lvdev(h, l), BlockMaps{D.bin, D.bcov}, D.list[LST_IN], lcap(D), h->qmax.p,
                            h->cfg.tag_tol, h->cfg.tag_buffer, h->bflag.p + off[l], s, D.cnt + LST_IN));
    }
}

// From block flags to the new layout, on the device.  Part 0 (reads the
// populations only): the layout rule (finest refinable level first), the
// new on-level maps, the nesting check, the exit / enter / touch lists and
// the new layout's tile lists and index maps; part 1: merge (finest first)
// and split (coarsest first) of the cells that change, the per-cell flags,
// the new maps committed and the audit's tile list; part -1: both.  Expects
// the composite state of the current layout (device_tags).
void device_apply_flags(vlbm_hier* h, const uint8_t* bflag, int part = -1) {
    cudaStream_t s = h->stream;
    const int nl = h->nlev;
    size_t off[VLBM_MAX_LEVELS] = {};
    for (int l = 1; l < nl; l++) off[l] = off[l - 1] + (size_t)h->lev[l - 1].bx * h->lev[l - 1].by;
    LayoutDev* D[VLBM_MAX_LEVELS];
    for (int l = 0; l < nl; l++) D[l] = &h->lev[l].dl;
    const LayoutDev* const* DL = D;
    if (part != 1) {
        VCK(cudaMemsetAsync(D[nl - 1]->ncov, 0, (size_t)lcap(*D[nl - 1]), s));
        for (int l = nl - 2; l >= 0; l--)
            VCK(launch_layout_rule(*D[l], l + 1 <= nl - 2 ? D[l + 1] : nullptr, bflag + off[l], s));
        VCK(launch_derive_in(DL, nl, s));
        VCK(launch_nest_check(DL, nl, h->words + 1, s));
        // in the same three launches: the exit / enter / touch lists from the
        // current against the new maps, and the tile lists and index maps of
        // the new layout from a view of the new maps (the current ones are
        // committed in the second part): everything a task-list build reads
        // is final once this part is done
        int masks[2 * VLBM_MAX_LEVELS];
        LayoutDev NL[VLBM_MAX_LEVELS];
        const LayoutDev* SL[2 * VLBM_MAX_LEVELS];
        for (int l = 0; l < nl; l++) {
            SL[l] = D[l];
            masks[l] = l <= nl - 2 ? LISTS_MOVE : (1 << LST_TOUCH);
            NL[l] = *D[l];
            NL[l].bin = D[l]->nin;
            NL[l].bcov = D[l]->ncov;
            NL[l].nin = NL[l].ncov = nullptr;
            SL[nl + l] = &NL[l];
            masks[nl + l] = LISTS_ALL;
        }
        VCK(launch_lists(SL, masks, 2 * nl, s));
    }
    if (part == 0) return;
    // the new maps committed and the audit's tile list concatenated touch
    // nothing that merge, split and the flags read or write: a parallel
    // branch (the maps and lists of the new layout are final after part 0)
    if (!h->side) VCK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    for (cudaEvent_t* ev : {&h->ev_fork, &h->ev_join})
        if (!*ev) VCK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    VCK(cudaEventRecord(h->ev_fork, s));
    VCK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    VCK(launch_commit_maps(DL, nl, h->side));
    {
        LayoutDev dls[VLBM_MAX_LEVELS];
        for (int l = 0; l < nl; l++) dls[l] = *D[l];
        VCK(launch_concat_act(dls, nl, h->ditems, h->dcount, h->side));
    }
    VCK(cudaEventRecord(h->ev_join, h->side));
    for (int l = nl - 2; l >= 0; l--)
        VCK(launch_merge(lvdev(h, l), D[l]->list[LST_EXIT], lcap(*D[l]), s, D[l]->cnt + LST_EXIT));
    for (int l = 0; l <= nl - 2; l++)
        VCK(launch_split(lvdev(h, l), lvdev(h, l + 1), D[l]->list[LST_ENTER], lcap(*D[l]), s, D[l]->cnt + LST_ENTER));
    FlagsSet F{};
    F.nl = nl;
    int cap = 0;
    for (int l = 0; l < nl; l++) {
        Level& L = h->lev[l];
        const LevelDev V = lvdev(h, l);
        F.g[l] = FlagsSet::Geom{V.nx, V.ny, V.pitch, V.px, V.py};
        F.items[l] = D[l]->list[LST_TOUCH];
        F.nc[l] = D[l]->cnt + LST_TOUCH;
        F.bin[l] = D[l]->nin;
        F.bcov[l] = D[l]->ncov;
        F.oldf[l] = L.flags;
        F.newf[l] = L.flags_tmp;
        cap = std::max(cap, lcap(*D[l]));
    }
    VCK(launch_flags_update(F, cap, s));
    VCK(cudaStreamWaitEvent(s, h->ev_join, 0));
}

// The totals after the last regrid, when still to come, by a separate
// audit of the current state (nothing has changed it since the regrid).
void settle_after_audit(vlbm_hier* h) {
    if (h->after_pending < 0) return;
    const long long slot = h->after_pending;
    h->after_pending = -1;
    const int icap = (int)std::min<size_t>(h->ditems_cap, 1u << 30);
    VCK(launch_audit(h->atab.p, h->ditems, icap, h->partial.p, h->raud + 16 * slot + 8, h->aticket.p, h->stream,
                     h->dcount));
    h->klaunch += 1;
}

// A tag-driven regrid on the device: indicator, block flags, new layout,
// merge / split, flags and lists, replayed as two captured graphs (every
// size involved is decided on the device, so the graphs stay valid).
void device_regrid(vlbm_hier* h) {
    check_tagging(h);
    regrid_buffers(h);
    std::vector<uintptr_t> key = {(uintptr_t)h->bflag.p, (uintptr_t)h->qmax.p,
                                  (uintptr_t)h->cfg.tag_sensor, (uintptr_t)h->ditems, (uintptr_t)h->words};
    for (int l = 0; l < h->nlev; l++) {
        key.push_back((uintptr_t)h->lev[l].flags);
        key.push_back((uintptr_t)h->lev[l].flags_tmp);
        key.push_back((uintptr_t)h->lev[l].buf[0]);
    }
    cudaStream_t s = h->stream;
    if (!h->rg_exec[0] || !h->rg_exec[1] || key != h->rg_key) {
        const auto t0 = std::chrono::steady_clock::now();
        if (!h->side) VCK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        for (cudaEvent_t* ev : {&h->ev_fork, &h->ev_join})
            if (!*ev) VCK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
        for (int part = 0; part < 2; part++) {
            cudaGraphExec_t& ex = h->rg_exec[part];
            if (ex) cudaGraphExecDestroy(ex);
            ex = nullptr;
            cudaGraph_t g = nullptr;
            VCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            try {
                if (part == 0) device_tags(h);
                device_apply_flags(h, h->bflag.p, part);
            } catch (...) {
                cudaStreamEndCapture(s, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            VCK(cudaStreamEndCapture(s, &g));
            cudaError_t e = instantiate(&ex, g);
            cudaGraphDestroy(g);
            VCK(e);
        }
        h->rg_key = key;
        h->times[VLBM_T_CAPTURE] += ms_since(t0);
    }
    for (cudaEvent_t* ev : {&h->ev_layout, &h->ev_rg0, &h->ev_audit})
        if (!*ev) VCK(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    if (!h->aux) VCK(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
    if (!h->aux2) VCK(cudaStreamCreateWithFlags(&h->aux2, cudaStreamNonBlocking));
    settle_after_audit(h);  // the previous regrid's totals after, if still to come
    const long long slot = h->ra_n % vlbm_hier::RA_CAP;
    const int icap = (int)std::min<size_t>(h->ditems_cap, 1u << 30);
    if (h->regrid_audit) {
        // the audit before the regrid reads the active cells' state, which
        // the first part (indicator, maps, move lists) leaves alone: it runs
        // on a stream of its own beside that part and the task-list build
        // that follows it, and the second part (merge, split: writes) waits
        // for it
        VCK(cudaEventRecord(h->ev_rg0, s));
        VCK(cudaStreamWaitEvent(h->aux2, h->ev_rg0, 0));
        VCK(launch_audit(h->atab.p, h->ditems, icap, h->partial.p, h->raud + 16 * slot, h->aticket.p, h->aux2,
                         h->dcount));
        VCK(cudaEventRecord(h->ev_audit, h->aux2));
    }
    VCK(cudaGraphLaunch(h->rg_exec[0], s));
    VCK(cudaEventRecord(h->ev_layout, s));  // the new layout's maps and lists are complete here
    if (h->regrid_audit) VCK(cudaStreamWaitEvent(s, h->ev_audit, 0));
    VCK(cudaGraphLaunch(h->rg_exec[1], s));
    h->klaunch += graph_kernels(h->rg_exec[0]) + graph_kernels(h->rg_exec[1]);
    if (h->regrid_audit) {
        // the totals after the regrid come later: from the first sweeps of
        // the next persistent launch, which read every active cell's state
        // anyway, or from a separate audit before anything else changes it
        h->ra_n++;
        h->klaunch += 1;
        h->after_pending = slot;
    }
    h->host_ok = false;
    layout_changed(h);
    h->ev_layout_version = h->layout_version;
}

// ---- the sub-cycle over the device lists ---------------------------------------

// Static tables of the phase sequence of `nsteps` coarse steps (the same
// recursion as phases() in vlbm_tasks.h, then the audit phase of a cyclic
// list) and the accesses of its phases per resource class (level, buffer
// 0 / 1 / flags), in phase order.
void plan_tables(int nlev, int nsteps, bool audit_phase, bool sensor, std::vector<TBPhase>& ph,
                 std::vector<TBAcc>& acc, std::vector<int>& beg, std::vector<int>& pos) {
    ph.clear();
    struct Rec {
        static void run(std::vector<TBPhase>& ph, bool sensor, int l, int kk, int kkp, int step, bool first) {
            if (sensor) {  // the relaxation sensor's two passes over the level's state
                ph.push_back(TBPhase{3, l, kk, kkp, step, 0});
                ph.push_back(TBPhase{4, l, kk, kkp, step, 0});
            }
            ph.push_back(TBPhase{0, l, kk, kkp, step, first ? 1 : 0});
            if (l + 1 < TASK_MAX_LEVELS) {
                run(ph, sensor, l + 1, 1, kk, step, first);
                run(ph, sensor, l + 1, 2, kk, step, false);
                ph.push_back(TBPhase{1, l, kk, 0, step, 0});
            }
        }
    };
    for (int st = 0; st < nsteps; st++) Rec::run(ph, sensor, 0, 0, 0, st, true);
    // the audit phase (reductions of the first sweeps' moments) touches no
    // buffer: it orders nothing but its own tasks after their sweeps
    if (audit_phase) ph.push_back(TBPhase{2, 0, 0, 0, 0, 0});
    auto src_of = [](int level, int kk, int step) { return level == 0 ? (step & 1) : (kk == 1 ? 0 : 1); };
    // resources per level: buffer 0, buffer 1, flags, the sensor's
    // first-pass planes (3), its second-pass planes (4)
    std::vector<TBAcc> per[TASK_MAX_LEVELS][TB_NRES];
    for (int p = 0; p < (int)ph.size(); p++) {
        const TBPhase& P = ph[p];
        const int l = P.l;
        if (P.kind == 2) continue;
        if (P.kind >= 3) {
            if (l >= nlev) continue;
            if (P.kind == 3) {
                per[l][src_of(l, P.kk, P.step)].push_back({p, 0, TB_OWN});
                per[l][3].push_back({p, 1, TB_OWN});
            } else {
                per[l][3].push_back({p, 0, TB_STENCIL});
                per[l][4].push_back({p, 1, TB_OWN});
            }
        } else if (P.kind == 0) {
            if (l >= nlev) continue;
            const int bs = src_of(l, P.kk, P.step);
            per[l][bs].push_back({p, 0, TB_OWN});
            per[l][bs ^ 1].push_back({p, 1, TB_STENCIL});
            if (l > 0) {
                const int pbs = src_of(l - 1, P.kkp, P.step);
                per[l - 1][pbs].push_back({p, 0, TB_FOOT});
                per[l - 1][pbs ^ 1].push_back({p, 0, TB_FOOT});
                per[l - 1][2].push_back({p, 0, TB_FOOT});
            }
            if (sensor) {
                per[l][3].push_back({p, 0, TB_OWN});
                per[l][4].push_back({p, 0, TB_BOX9});
            }
        } else {
            if (l + 1 >= nlev) continue;
            const int bd = src_of(l, P.kk, P.step) ^ 1;
            per[l + 1][0].push_back({p, 0, TB_CHILD4});
            per[l + 1][1].push_back({p, 0, TB_CHILD4});
            per[l][bd].push_back({p, 1, TB_OWNRING});
            per[l][2].push_back({p, 1, TB_OWNRING});
        }
    }
    const int np = (int)ph.size();
    acc.clear();
    beg.assign(TASK_RC + 1, 0);
    pos.assign((size_t)TASK_RC * (np + 1), 0);
    for (int rc = 0; rc < TASK_RC; rc++) {
        const std::vector<TBAcc>& A = per[rc / TB_NRES][rc % TB_NRES];
        beg[rc] = (int)acc.size();
        int e = 0;
        for (int p = 0; p <= np; p++) {
            while (e < (int)A.size() && A[e].phase < p) e++;
            pos[(size_t)rc * (np + 1) + p] = beg[rc] + e;
        }
        acc.insert(acc.end(), A.begin(), A.end());
    }
    beg[TASK_RC] = (int)acc.size();
}

// The task list on the current layout, built on the device when the layout
// changed: cyclic -- one coarse step that the persistent kernel repeats once
// per step (dp[0]); otherwise `k` coarse steps from a synchronised state
// (dp[1]).
vlbm_hier::DevPlan& dev_plan(vlbm_hier* h, int k, bool cyclic) {
    vlbm_hier::DevPlan& D = h->dp[cyclic ? 0 : 1];
    if (cyclic) k = 1;
    // regrid audits of a hierarchy on its own: the totals after each regrid
    // come from the next launch (the engine audits separately)
    const bool audit = cyclic && h->regrid_audit && !h->engine;
    const bool sensor = cyclic && h->sensor_on;
    D.build_kernels = 0;
    cudaStream_t s = h->stream;
    bool plan_fresh_ok = true;  // no upload queued on the main stream since the layout event
    if (D.steps != k || D.audit != audit || D.sensor != sensor) {
        plan_fresh_ok = false;
        std::vector<TBPhase> ph;
        std::vector<TBAcc> acc;
        std::vector<int> beg, pos;
        plan_tables(h->nlev, k, cyclic, sensor, ph, acc, beg, pos);
        long long cap = 0, slot_cap = 0;
        for (int l = 0; l < h->nlev; l++) slot_cap += (long long)h->lev[l].bx * h->lev[l].by;
        const long long blk_cap = (slot_cap + TB_AUDIT_BLOCK - 1) / TB_AUDIT_BLOCK;
        for (int l = 0; l < 4; l++) D.pfirst[l] = -1;
        for (int p = 0; p < (int)ph.size(); p++) {
            const TBPhase& P = ph[p];
            if ((P.kind == 0 || P.kind >= 3) && P.l < h->nlev) cap += (long long)h->lev[P.l].bx * h->lev[P.l].by;
            if (P.kind == 1 && P.l + 1 < h->nlev) cap += (long long)h->lev[P.l].bx * h->lev[P.l].by;
            if (P.kind == 2 && audit) cap += 4 * blk_cap;
            if (P.kind == 0 && P.first && P.l < 4 && D.pfirst[P.l] < 0) D.pfirst[P.l] = p;
        }
        if (audit) {
            D.aw.ensure(h->mem, (size_t)slot_cap * AUDIT_SLOT);
            D.ascale.ensure(h->mem, (size_t)slot_cap);
            D.arng.ensure(h->mem, (size_t)blk_cap);
            D.apart.ensure(h->mem, (size_t)blk_cap * 24);
        } else {
            D.aw.release(h->mem);
            D.ascale.release(h->mem);
            D.arng.release(h->mem);
            D.apart.release(h->mem);
        }
        D.audit = audit;
        D.sensor = sensor;
        // a cyclic list's tickets (tasks x iterations, up to 64) are ints too
        if (cap >= ((1LL << 31) - 1) / (cyclic ? 64 : 1)) throw Fail{VLBM_ERR_ARG, "hierarchy too large for one task list"};
        if (acc.empty()) acc.push_back(TBAcc{0, 0, 0});
        D.ph.upload(h->mem, ph, s);
        D.acc.upload(h->mem, acc, s);
        D.acc_beg.upload(h->mem, beg, s);
        D.acc_pos.upload(h->mem, pos, s);
        D.nphase = (int)ph.size();
        D.nacc = (int)acc.size();
        D.off.ensure(h->mem, ph.size() + 1);
        D.task_cap = (int)cap;
        // fixed slots of TASK_DEP_SLOT dependencies per task and an overflow
        // area for the tasks with more: measured at most about 12
        // dependencies per task slot on average and 98 for one task on
        // adversarial layouts (most cells refined, checkerboard coverage); an
        // exhausted area raises VLBM_ERR_OOM at the next synchronising call
        D.dep_cap = (long long)TASK_DEP_SLOT * cap + std::max<long long>(1 << 22, 8 * cap);
        if (D.dep_cap >= (1LL << 31)) throw Fail{VLBM_ERR_ARG, "hierarchy too large for one task list"};
        D.tasks.ensure(h->mem, (size_t)cap + 1);
        D.deps.ensure(h->mem, (size_t)D.dep_cap);
        D.need.ensure(h->mem, 8);
        D.big.ensure(h->mem, (size_t)cap + 1);
        // completion marks restart with the epoch below: a mark left from
        // before the restart could otherwise pass for a later epoch's
        D.done.ensure(h->mem, (size_t)cap + 1);
        VCK(cudaMemsetAsync(D.done.p, 0, D.done.cap * sizeof(unsigned), s));
        // the launch's segment and control words (the builder fills in the
        // task count; from here on the epoch only grows, so the marks that
        // launches of this plan leave stay below every later launch's)
        Segment sg{};
        sg.tasks = D.tasks.p;
        sg.deps = D.deps.p;
        sg.done = D.done.p;
        sg.aw = audit ? D.aw.p : nullptr;
        sg.arng = audit ? D.arng.p : nullptr;
        sg.ascale = audit ? D.ascale.p : nullptr;
        sg.apart = audit ? D.apart.p : nullptr;
        sg.par0 = h->words;
        sg.lid_base = 0;
        D.seg.upload(h->mem, std::vector<Segment>{sg}, s);
        D.prefix.upload(h->mem, std::vector<int>{0, 0}, s);
        D.chunks.upload(h->mem, std::vector<int2>{make_int2(0, 0)}, s);
        std::vector<int> c(CTL_WORDS, 0);
        c[CTL_EPOCH] = 1;
        c[CTL_NSEG] = 1;
        c[CTL_NCHUNK] = 1;
        c[CTL_FLIP] = k & 1;
        D.ctl.upload(h->mem, c, s);
        D.steps = k;
        D.version = -1;
    }
    if (D.version != h->layout_version) {
        const auto t0 = std::chrono::steady_clock::now();
        // The build reads only the layout: it runs on the auxiliary stream
        // from the moment the regrid that made the layout is done, beside
        // what the main stream does after it (the post-regrid audit), and
        // the main stream waits for it.  Under a capture of the main stream,
        // or when the layout came another way, it starts from the main
        // stream's current end.
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        VCK(cudaStreamIsCapturing(s, &cs));
        cudaStream_t bs = s;
        if (cs == cudaStreamCaptureStatusNone) {
            if (!h->aux) VCK(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
            if (!h->ev_layout) VCK(cudaEventCreateWithFlags(&h->ev_layout, cudaEventDisableTiming));
            if (!h->ev_built) VCK(cudaEventCreateWithFlags(&h->ev_built, cudaEventDisableTiming));
            if (h->ev_layout_version != h->layout_version || !plan_fresh_ok) {
                VCK(cudaEventRecord(h->ev_layout, s));
                h->ev_layout_version = h->layout_version;
            }
            VCK(cudaStreamWaitEvent(h->aux, h->ev_layout, 0));
            bs = h->aux;
        }
        // the reverse footprints of the current layout (shared by both plans)
        if (h->foot_version != h->layout_version) {
            const LayoutDev* FL[VLBM_MAX_LEVELS];
            for (int l = 0; l < h->nlev; l++) FL[l] = &h->lev[l].dl;
            VCK(launch_footprints(FL, h->nlev, h->words + 1, bs));
            h->foot_version = h->layout_version;
            D.build_kernels += h->nlev > 1 ? 1 : 0;
        }
        TBPlan P;
        P.nlev = h->nlev;
        P.nphase = D.nphase;
        P.nacc = D.nacc;
        P.cyclic = cyclic ? 1 : 0;
        for (int l = 0; l < h->nlev; l++) {
            const LayoutDev& L = h->lev[l].dl;
            P.lev[l] = TBLevel{L.nx, L.ny, L.bx, L.by, L.px, L.py, L.list[LST_ACT], L.list[LST_RING],
                               L.act_idx, L.ring_idx, L.recon, L.fcnt, L.fidx, L.cnt};
        }
        P.ph = D.ph.p;
        P.acc = D.acc.p;
        P.acc_beg = D.acc_beg.p;
        P.acc_pos = D.acc_pos.p;
        P.off = D.off.p;
        P.tasks = D.tasks.p;
        P.deps = D.deps.p;
        P.done = D.done.p;
        P.task_cap = D.task_cap;
        P.dep_cap = D.dep_cap;
        P.need = D.need.p;
        P.big = D.big.p;
        P.status = h->words + 1;
        P.seg = D.seg.p;
        P.prefix = D.prefix.p;
        P.ctl = D.ctl.p;
        P.audit = D.audit ? 1 : 0;
        P.sensor = D.sensor ? 1 : 0;
        for (int l = 0; l < 4; l++) P.pfirst[l] = D.pfirst[l];
        P.ascale = D.ascale.p;
        P.arng = D.arng.p;
        VCK(launch_task_build(P, bs));
        if (bs != s) {
            VCK(cudaEventRecord(h->ev_built, bs));
            VCK(cudaStreamWaitEvent(s, h->ev_built, 0));
        }
        D.build_kernels += 3;  // offsets, the warp pass, the fallback pass
        D.version = h->layout_version;
        h->times[VLBM_T_TASKS] += ms_since(t0);
        h->times[VLBM_T_NTASKLISTS] += 1;
    }
    return D;
}

// ... and the graph of its persistent launch: the cyclic list, `iters`
// coarse steps ([which]: 0 one step, 1 G steps).
cudaGraphExec_t dev_task_graph(vlbm_hier* h, int which, int iters) {
    vlbm_hier::DevPlan& D = dev_plan(h, 1, true);
    cudaStream_t s = h->stream;
    std::vector<uintptr_t> key = {(uintptr_t)h->atab.p,   (uintptr_t)D.seg.p,          (uintptr_t)D.prefix.p,
                                  (uintptr_t)D.chunks.p, (uintptr_t)D.ctl.p,          (uintptr_t)h->tune.variant,
                                  (uintptr_t)h->tune.max_ctas, (uintptr_t)iters,     (uintptr_t)D.sensor};
    cudaGraphExec_t& ex = D.exec[which];
    if (!ex || key != D.key[which]) {
        const auto t0 = std::chrono::steady_clock::now();
        if (ex) cudaGraphExecDestroy(ex);
        ex = nullptr;
        cudaGraph_t g = nullptr;
        VCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemsetAsync(D.ctl.p, 0, 2 * sizeof(int), s);  // claim and finish counters
        if (e == cudaSuccess)
            e = launch_tasks(h->atab.p, D.seg.p, D.prefix.p, D.chunks.p, D.ctl.p, h->tune.variant, h->tune.max_ctas,
                             iters, s, D.sensor);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = instantiate(&ex, g);
        if (g) cudaGraphDestroy(g);
        VCK(e);
        D.key[which] = key;
        h->times[VLBM_T_CAPTURE] += ms_since(t0);
    }
    return ex;
}

// One launch per level phase over the device lists (the per-phase schedule,
// and the one the relaxation sensor runs on).
void dev_schedule(vlbm_hier* h, int l, int kk, int kkp, cudaStream_t s) {
    const LayoutDev& D = h->lev[l].dl;
    if (h->sensor_on) VCK(launch_sensor(h->atab.p, D.list[LST_ACT], lcap(D), kk, s, D.cnt + LST_ACT));
    VCK(launch_sweep(h->atab.p, D.list[LST_ACT], lcap(D), kk, kkp, h->tune.max_ctas, h->tune.variant, s, h->sensor_on,
                     D.cnt + LST_ACT));
    if (l + 1 < h->nlev) {
        dev_schedule(h, l + 1, 1, kk, s);
        dev_schedule(h, l + 1, 2, kk, s);
        VCK(launch_close(h->atab.p, D.list[LST_RING], lcap(D), kk, s, D.cnt + LST_RING));
    }
}

cudaGraphExec_t dev_phase_graph(vlbm_hier* h, int which, int k) {
    vlbm_hier::PhaseGraph& P = h->pg[which];
    std::vector<uintptr_t> key = {(uintptr_t)h->atab.p, (uintptr_t)h->tune.variant, (uintptr_t)h->tune.max_ctas,
                                  (uintptr_t)h->sensor_on, (uintptr_t)k, (uintptr_t)h->parp};
    if (P.exec && key == P.key) return P.exec;
    const auto t0 = std::chrono::steady_clock::now();
    if (P.exec) cudaGraphExecDestroy(P.exec);
    P.exec = nullptr;
    cudaStream_t s = h->stream;
    cudaGraph_t g = nullptr;
    VCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
        for (int i = 0; i < k; i++) {
            dev_schedule(h, 0, 0, 0, s);
            VCK(launch_end_step(h->parp, 1, s));
        }
    } catch (...) {
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    VCK(cudaStreamEndCapture(s, &g));
    cudaError_t e = instantiate(&P.exec, g);
    cudaGraphDestroy(g);
    VCK(e);
    P.key = key;
    h->times[VLBM_T_CAPTURE] += ms_since(t0);
    return P.exec;
}

void count_lups(vlbm_hier* h, long long n) {
    if (n <= 0) return;
    LayoutDev dls[VLBM_MAX_LEVELS];
    for (int l = 0; l < h->nlev; l++) dls[l] = h->lev[l].dl;
    VCK(launch_count_lups(dls, h->nlev, n, h->lupc, h->stream));
}

// n coarse steps on the device lists: the persistent task kernel (sched 1)
// or one launch per phase (sched 0), G steps per graph launch.
void dev_advance(vlbm_hier* h, long long n, int sched) {
    cudaStream_t s = h->stream;
    const int G = h->tune.graph_steps;
    // totals after the last regrid still to come: from the first launch's
    // first step on the persistent schedule, else by a separate audit now
    if (h->after_pending >= 0 && (sched != 1 || n <= 0)) settle_after_audit(h);
    auto launch = [&](cudaGraphExec_t ex, long long nk) {
        vlbm_hier::DevPlan& D = h->dp[0];
        const bool fused = sched == 1 && h->after_pending >= 0 && D.audit;
        if (h->after_pending >= 0 && !fused) settle_after_audit(h);
        if (fused) VCK(cudaMemsetAsync(D.ctl.p + CTL_AUDIT, 1, sizeof(int), s));  // nonzero: audited
        VCK(cudaGraphLaunch(ex, s));
        h->klaunch += nk;
        if (fused) {
            VCK(launch_audit_blocks(D.apart.p, D.need.p + 6, h->raud + 16 * h->after_pending + 8,
                                    D.ctl.p + CTL_AUDIT, s));
            h->after_pending = -1;
            h->klaunch += 1;
        }
    };
    long long left = n;
    if (left >= G) {
        cudaGraphExec_t ex = sched == 1 ? dev_task_graph(h, 1, G) : dev_phase_graph(h, 1, G);
        if (sched == 1) h->klaunch += h->dp[0].build_kernels;  // a task list build, if one was queued
        const long long nk = graph_kernels(ex);
        for (; left >= G; left -= G) launch(ex, nk);
    }
    if (left > 0) {
        cudaGraphExec_t ex = sched == 1 ? dev_task_graph(h, 0, 1) : dev_phase_graph(h, 0, 1);
        if (sched == 1) h->klaunch += h->dp[0].build_kernels;
        const long long nk = graph_kernels(ex);
        for (; left > 0; left--) launch(ex, nk);
    }
    count_lups(h, n);
    h->klaunch += 1;
}

void release_dev_plans(vlbm_hier* h) {
    for (auto& D : h->dp) {
        for (int w = 0; w < 2; w++) {
            if (D.exec[w]) cudaGraphExecDestroy(D.exec[w]);
            D.exec[w] = nullptr;
            D.key[w].clear();
        }
        for (DArr<int>* a : {&D.acc_beg, &D.acc_pos, &D.off, &D.deps, &D.need, &D.prefix, &D.ctl, &D.big, &D.ascale})
            a->release(h->mem);
        D.aw.release(h->mem);
        D.arng.release(h->mem);
        D.apart.release(h->mem);
        D.audit = false;
        D.chunks.release(h->mem);
        D.ph.release(h->mem);
        D.acc.release(h->mem);
        D.tasks.release(h->mem);
        D.done.release(h->mem);
        D.seg.release(h->mem);
        D.steps = -1;
        D.version = -1;
    }
    for (auto& P : h->pg) {
        if (P.exec) cudaGraphExecDestroy(P.exec);
        P.exec = nullptr;
        P.key.clear();
    }
    for (auto& x : h->rg_exec) {
        if (x) cudaGraphExecDestroy(x);
        x = nullptr;
    }
    h->rg_key.clear();
}

void invalidate(vlbm_hier* h);

}  // namespace

// k coarse steps of every member in one persistent launch (the engine).
void Batch::device_steps(long long k, cudaStream_t s) {
    const int nm = (int)members.size();
    if (nm == 0 || k <= 0) return;
    if (k > 64) throw Fail{VLBM_ERR_ARG, "at most 64 steps per persistent launch"};
    // every member's one-step list on its current layout, built on the
    // device (on the member's auxiliary stream; this stream waits for it)
    for (vlbm_hier* h : members) {
        cudaStream_t own = h->stream;
        h->stream = s;
        h->mem.s = s;
        try {
            dev_plan(h, 1, true);
        } catch (...) {
            h->stream = own;
            h->mem.s = own;
            throw;
        }
        h->stream = own;
        h->mem.s = own;
    }
    std::vector<Segment> sg(nm);
    std::vector<const int*> offs(nm), mctl(nm);
    int base = 0, nphase = 0;
    for (int m = 0; m < nm; m++) {
        vlbm_hier* h = members[m];
        const vlbm_hier::DevPlan& D = h->dp[0];
        Segment S{};
        S.tasks = D.tasks.p;
        S.deps = D.deps.p;
        S.done = D.done.p;
        S.par0 = h->words;
        S.lid_base = base;
        sg[m] = S;
        offs[m] = D.off.p;
        mctl[m] = D.ctl.p;
        base += h->nlev;
        nphase = D.nphase;  // one phase sequence for every hierarchy (all levels up to the maximum)
    }
    if (!dctl.p) {
        std::vector<int> c(CTL_WORDS, 0);
        c[CTL_EPOCH] = 1;
        c[CTL_FLIP] = 1;  // one-step lists
        dctl.upload(*mem, c, s);
    }
    dprefix.ensure(*mem, (size_t)nphase * nm + 1);
    dchunks.ensure(*mem, (size_t)nphase * nm + 1);
    stage_begin(sg.size() * sizeof(Segment) + 2 * offs.size() * sizeof(const int*));
    staged(dsegs, sg, s);
    staged(doffs, offs, s);
    staged(dmctl, mctl, s);
    stage_end(s);
    VCK(launch_merge_chunks(doffs.p, dmctl.p, nm, nphase, dprefix.p, dchunks.p, dctl.p, s));
    VCK(launch_tasks(levs.p, dsegs.p, dprefix.p, dchunks.p, dctl.p, variant, max_ctas, (int)k, s));
}

// ----------------------------------------------------------------------------
// engine
// ----------------------------------------------------------------------------

struct vlbm_engine {
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevMem mem;
    // schedule 0 (default): shared per-phase launches, one launch per level
    // phase covering the tiles of all residents; schedule 1: one persistent
    // launch per call over every resident's device-built one-step task list,
    // merged phase-major (measured slower on the serving trace: 4912 against
    // 5710 MLUPS capacity, its per-call list builds and short launches of
    // many small residents cost more than the launch gaps they save)
    Batch batch;
    int schedule = 0;
    struct Res {
        vlbm_hier* h = nullptr;
        long long target = 0, done = 0, lups = 0;
        int regrid_every = 0;
        bool live = false;
        bool adaptive() const { return regrid_every > 0 && h->cfg.tag_tol > 0; }
        bool paused = false;           // waiting for its regrid (not in a batch)
        bool tagging = false;          // the first half of its regrid is queued
        bool finishing = false;        // step count met, last step maybe still running (ev)
        bool reported = false;         // reported finished
        long long regridded_at = -1;   // step count of its last regrid
        cudaEvent_t ev = nullptr;      // end of its last step, then of its regrid
    };
    std::vector<Res> res;
    bool dirty = true;
    bool regridded = false;  // an adaptive resident changed its layout since the last rebuild
    bool admitted = true;    // a resident was admitted or released since the last rebuild
    cudaStream_t hi = nullptr;  // high-priority stream of the residents' regrids
    // the ends of the steps queued by the last LEAD calls: a call waits for
    // the steps queued LEAD calls before, so the host stays at most LEAD
    // calls ahead of the GPU
    static constexpr int LEAD = 4;  // deep enough to cover a burst of admissions
    cudaEvent_t lead[LEAD] = {};
    bool lead_set[LEAD] = {};
    int lead_i = 0;
    double times[VLBM_ET_COUNT] = {};  // host time by activity, see vlbm_engine_host_times
    std::string err = "no error";
};

namespace {

void invalidate(vlbm_hier* h) {
    if (h->own) h->own->valid = false;
    if (h->engine) h->engine->dirty = true;
}

// Runs fn with the hierarchy's queue and memory pool stream set to s; a
// failure poisons the hierarchy as its own calls would.
template <class F>
void on_stream(vlbm_hier* h, cudaStream_t s, F&& fn) {
    cudaStream_t own = h->stream;
    h->stream = s;
    h->mem.s = s;
    try {
        fn();
    } catch (const Fail& f) {
        h->stream = own;
        h->mem.s = own;
        h->err = f.msg;
        if (f.st == VLBM_ERR_NONPHYSICAL || f.st == VLBM_ERR_TIMEOUT || f.st == VLBM_ERR_CUDA) h->poisoned = true;
        throw Fail{f.st, "regrid: " + f.msg};
    }
    h->stream = own;
    h->mem.s = own;
}

vlbm_status finish(vlbm_hier* h, const Fail& f) {
    h->err = f.msg;
    if (f.st == VLBM_ERR_NONPHYSICAL || f.st == VLBM_ERR_TIMEOUT || f.st == VLBM_ERR_CUDA) h->poisoned = true;
    return f.st;
}

template <class F>
vlbm_status run(vlbm_hier* h, F&& fn) {
    if (!h) return VLBM_ERR_ARG;
    if (h->poisoned) return VLBM_ERR_STATE;
    try {
        fn();
        return VLBM_OK;
    } catch (const Fail& f) {
        return finish(h, f);
    } catch (const std::bad_alloc&) {
        h->err = "host allocation failed";
        return VLBM_ERR_OOM;
    }
}

void destroy_levels(vlbm_hier* h) {
    for (int l = 0; l < h->nlev; l++) {
        Level& L = h->lev[l];
        const size_t pb = (size_t)16 * L.plane * sizeof(double);
        h->mem.put(L.buf[0], pb);
        h->mem.put(L.buf[1], pb);
        h->mem.put(L.flags, (size_t)L.plane * 2);
        h->mem.put(L.flags_tmp, (size_t)L.plane * 2);
        free_layout(h, l);
        L.buf[0] = L.buf[1] = nullptr;
        L.flags = L.flags_tmp = nullptr;
    }
    for (int l = 0; l < VLBM_MAX_LEVELS; l++) {
        if (h->sens[l]) h->mem.put(h->sens[l], (size_t)SENS_PLANES * h->lev[l].plane * sizeof(double));
        h->sens[l] = nullptr;
    }
    h->mem.put(h->words, 64);
    h->words = nullptr;
    h->stage.release(h->mem);
    h->stage8.release(h->mem);
    h->qmax.release(h->mem);
    h->partial.release(h->mem);
    h->aticket.release(h->mem);
    h->tot.release(h->mem);
    h->listbuf.release(h->mem);
    h->bflag.release(h->mem);
    h->atab.release(h->mem);
    release_dev_plans(h);
    h->mem.put(h->ditems, h->ditems_cap * sizeof(Item));
    h->mem.put(h->dcount, 4 * sizeof(int));
    h->mem.put(h->lupc, sizeof(unsigned long long));
    h->mem.put(h->parp, sizeof(int*));
    h->mem.put(h->raud, (size_t)vlbm_hier::RA_CAP * 16 * sizeof(double));
    h->raud = nullptr;
    h->ditems = nullptr;
    h->dcount = nullptr;
    h->lupc = nullptr;
    h->parp = nullptr;
    pin_free(h->hout, 8 * sizeof(double));
    h->hout = nullptr;
    h->pin.release();
    pin_free(h->rg_pin, h->rg_cap);
    h->rg_pin = nullptr;
    h->rg_cap = 0;
    if (h->rg_ev) cudaEventDestroy(h->rg_ev);
    h->rg_ev = nullptr;
    for (cudaStream_t* st : {&h->aux, &h->aux2, &h->side}) {
        if (*st) {
            cudaStreamSynchronize(*st);
            cudaStreamDestroy(*st);
        }
        *st = nullptr;
    }
    for (cudaEvent_t* ev : {&h->ev_layout, &h->ev_built, &h->ev_rg0, &h->ev_audit, &h->ev_fork, &h->ev_join}) {
        if (*ev) cudaEventDestroy(*ev);
        *ev = nullptr;
    }
    pin_free(h->hist, (size_t)h->hist_cap * 8 * sizeof(double));
    h->hist = nullptr;
    for (auto& L : h->tl) {
        L.dt.release(h->mem);
        L.dd.release(h->mem);
        L.done.release(h->mem);
        L.aw.release(h->mem);
        L.ascale.release(h->mem);
        L.arng.release(h->mem);
        L.apart.release(h->mem);
        L.abseg.release(h->mem);
        L.aout.release(h->mem);
        L.steps = -1;
    }
}

// Schedule of the next steps on the host-built lists (per-step totals,
// profiling): 2 (auto) takes the per-phase launches on a layout younger than
// persist_after coarse steps -- an adaptive run that regrids often never
// pays for a task list -- and the persistent task kernel after that, or
// whenever per-step totals are on.
int effective_schedule(const vlbm_hier* h) {
    if (h->sensor_on) return 0;  // host-built lists hold no sensor passes
    if (h->tune.schedule != 2) return h->tune.schedule;
    return (h->step_audit || h->layout_steps >= h->tune.persist_after) ? 1 : 0;
}

// Schedule of the steps on the device lists.  Auto (2) keeps the per-phase
// launches on a layout younger than persist_after coarse steps, as on the
// host lists.  A device build of a layout's one-step task list costs about
// 0.1 ms on the 2048 x 1024 shock-bubble, less than the persistent kernel
// saves in one coarse step (regridding every 4 steps: 5650 MLUPS
// persistent, 5104 per phase), hence the default of 2.
int dev_schedule_mode(const vlbm_hier* h) {
    if (h->tune.schedule != 2) return h->tune.schedule;
    return h->layout_steps >= h->tune.persist_after ? 1 : 0;
}

void ensure_own_batch(vlbm_hier* h, int sched) {
    ensure_host(h);
    if (!h->own) {
        h->own = new Batch();
        h->own->mem = &h->mem;
        h->own->klaunch = &h->klaunch;
        h->own->members.push_back(h);
    }
    if (h->own->valid && h->own->schedule_mode != sched) h->own->valid = false;
    if (!h->own->valid) {
        h->own->variant = h->tune.variant;
        h->own->max_ctas = h->tune.max_ctas;
        h->own->G = h->tune.graph_steps;
        h->own->schedule_mode = sched;
        h->own->audit = h->step_audit && sched == 1;
        const auto t0 = std::chrono::steady_clock::now();
        h->own->build(h->stream);
        h->times[VLBM_T_BUILD] += ms_since(t0);
    }
}

}  // namespace

// ----------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------

extern "C" {

vlbm_status vlbm_create_hierarchy(const vlbm_config* cfg, const vlbm_allocator* alloc, void* stream, vlbm_hier** out) {
    if (!out) return VLBM_ERR_ARG;
    *out = nullptr;
    if (!cfg) return VLBM_ERR_ARG;
    if (cfg->nx0 < 1 || cfg->ny0 < 1 || cfg->max_levels < 1 || cfg->max_levels > VLBM_MAX_LEVELS) return VLBM_ERR_ARG;
    if (!(cfg->gamma > 1.0) || !(cfg->c > 0.0) || !(cfg->beta >= 0.0 && cfg->beta <= 1.0)) return VLBM_ERR_ARG;
    for (int s = 0; s < 4; s++)
        if (cfg->bc[s] < 0 || cfg->bc[s] > 3) return VLBM_ERR_ARG;
    if ((cfg->bc[0] == VLBM_BC_PERIODIC) != (cfg->bc[1] == VLBM_BC_PERIODIC)) return VLBM_ERR_ARG;
    if ((cfg->bc[2] == VLBM_BC_PERIODIC) != (cfg->bc[3] == VLBM_BC_PERIODIC)) return VLBM_ERR_ARG;
    const long long nxmax = (long long)cfg->nx0 << (cfg->max_levels - 1);
    const long long nymax = (long long)cfg->ny0 << (cfg->max_levels - 1);
    if (nxmax / TILE >= 65535 || nymax / TILE >= 65535) return VLBM_ERR_ARG;
    if (cfg->nboxes < 0 || (cfg->nboxes > 0 && !cfg->boxes)) return VLBM_ERR_ARG;
    vlbm_hier* h = new (std::nothrow) vlbm_hier();
    if (!h) return VLBM_ERR_OOM;
    h->cfg = *cfg;
    if (cfg->nboxes) h->boxes.assign(cfg->boxes, cfg->boxes + cfg->nboxes);
    h->cfg.boxes = nullptr;
    h->nlev = cfg->max_levels;
    h->gm1 = cfg->gamma - 1.0;
    h->om = 1.0 - 2.0 * cfg->beta;
    h->hb = 0.5 * cfg->beta;
    h->bcs = cfg->beta / cfg->c;
    h->hc = 0.5 / cfg->c;
    for (int s = 0; s < 4; s++)
        if (cfg->bc[s] == VLBM_BC_INFLOW) host_feq(cfg->gamma, cfg->c, cfg->inflow_W[s], h->feqb[s]);
    if (alloc) {
        if (!alloc->alloc || !alloc->free) {
            delete h;
            return VLBM_ERR_ARG;
        }
        h->mem.a = *alloc;
        h->mem.has = true;
    }
    try {
        if (stream) {
            h->stream = (cudaStream_t)stream;
        } else {
            VCK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
            h->own_stream = true;
        }
        h->mem.s = h->stream;
        h->mem.pin = &h->pin;
        h->words = (int*)h->mem.get(64);
        VCK(cudaMemsetAsync(h->words, 0, 64, h->stream));
        for (int l = 0; l < h->nlev; l++) {
            Level& L = h->lev[l];
            L.nx = cfg->nx0 << l;
            L.ny = cfg->ny0 << l;
            L.pitch = (L.nx + 15) & ~15;
            L.plane = (long long)L.pitch * L.ny;
            L.bx = ceil_div(L.nx, TILE);
            L.by = ceil_div(L.ny, TILE);
            const size_t pb = (size_t)16 * L.plane * sizeof(double);
            L.buf[0] = (double*)h->mem.get(pb);
            L.buf[1] = (double*)h->mem.get(pb);
            L.flags = (uint16_t*)h->mem.get((size_t)L.plane * 2);
            L.flags_tmp = (uint16_t*)h->mem.get((size_t)L.plane * 2);
            VCK(cudaMemsetAsync(L.buf[0], 0, pb, h->stream));
            VCK(cudaMemsetAsync(L.buf[1], 0, pb, h->stream));
            VCK(cudaMemsetAsync(L.flags, 0, (size_t)L.plane * 2, h->stream));
            VCK(cudaMemsetAsync(L.flags_tmp, 0, (size_t)L.plane * 2, h->stream));
            alloc_layout(h, l);
            h->ditems_cap += (size_t)L.bx * L.by;
        }
        h->ditems = (Item*)h->mem.get(h->ditems_cap * sizeof(Item));
        h->dcount = (int*)h->mem.get(4 * sizeof(int));
        h->lupc = (unsigned long long*)h->mem.get(sizeof(unsigned long long));
        h->parp = (int**)h->mem.get(sizeof(int*));
        VCK(cudaMemsetAsync(h->dcount, 0, 4 * sizeof(int), h->stream));
        VCK(cudaMemsetAsync(h->lupc, 0, sizeof(unsigned long long), h->stream));
        VCK(cudaMemcpyAsync(h->parp, &h->words, sizeof(int*), cudaMemcpyHostToDevice, h->stream));
        h->partial.ensure(h->mem, (size_t)24 * audit_blocks((int)std::min<size_t>(h->ditems_cap, 1u << 30)));
        h->aticket.ensure(h->mem, 1);
        VCK(cudaMemsetAsync(h->aticket.p, 0, sizeof(unsigned), h->stream));
        h->tot.ensure(h->mem, 8);
        std::vector<uint8_t> bin[VLBM_MAX_LEVELS], bcov[VLBM_MAX_LEVELS];
        boxes_to_maps(h, h->boxes.data(), (int)h->boxes.size(), bcov);
        derive_in(h, bin, bcov);
        std::string why;
        if (!nested(h, bin, bcov, why)) throw Fail{VLBM_ERR_NESTING, why};
        install_layout(h, bin, bcov);
        VCK(cudaStreamSynchronize(h->stream));
    } catch (const Fail& f) {
        vlbm_status st = f.st;
        destroy_levels(h);
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        delete h;
        return st;
    }
    *out = h;
    return VLBM_OK;
}

void vlbm_destroy(vlbm_hier* h) {
    if (!h) return;
    if (h->engine) {
        // still resident: detach
        vlbm_engine* e = h->engine;
        for (size_t i = 0; i < e->res.size(); i++)
            if (e->res[i].live && e->res[i].h == h) vlbm_engine_release(e, (int)i);
    }
    cudaStreamSynchronize(h->stream);
    if (h->own) {
        h->own->release();
        delete h->own;
    }
    destroy_levels(h);
    cudaStreamSynchronize(h->stream);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char* vlbm_last_error(const vlbm_hier* h) { return h ? h->err.c_str() : "null handle"; }

vlbm_status vlbm_set_state(vlbm_hier* h, int32_t level, const double* W, int64_t ld, int32_t on_device) {
    return run(h, [&] {
        if (level < 0 || level >= h->nlev || !W) throw Fail{VLBM_ERR_ARG, "bad level or W"};
        settle_after_audit(h);
        Level& L = h->lev[level];
        if (ld < L.nx) throw Fail{VLBM_ERR_ARG, "ld < nx"};
        const double* src = W;
        if (!on_device) {
            const size_t n = (size_t)4 * ld * L.ny;
            h->stage.ensure(h->mem, n);
            VCK(cudaMemcpyAsync(h->stage.p, W, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            src = h->stage.p;
        }
        VCK(launch_feq_init(lvdev(h, level), src, ld, h->hc, h->stream));
        h->klaunch += 1;
        if (!on_device) VCK(cudaStreamSynchronize(h->stream));
    });
}

static vlbm_status pop_copy(vlbm_hier* h, int32_t level, double* f, int64_t ld, int32_t on_device, int to_ext) {
    return run(h, [&] {
        if (level < 0 || level >= h->nlev || !f) throw Fail{VLBM_ERR_ARG, "bad level or f"};
        Level& L = h->lev[level];
        if (ld < L.nx) throw Fail{VLBM_ERR_ARG, "ld < nx"};
        if (!to_ext) settle_after_audit(h);
        const size_t n = (size_t)16 * ld * L.ny;
        double* ext = f;
        if (!on_device) {
            h->stage.ensure(h->mem, n);
            ext = h->stage.p;
            if (!to_ext) VCK(cudaMemcpyAsync(ext, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        }
        VCK(launch_copy_pop(lvdev(h, level), ext, ld, to_ext, h->stream));
        h->klaunch += 1;
        if (!on_device && to_ext) VCK(cudaMemcpyAsync(f, ext, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        VCK(cudaStreamSynchronize(h->stream));
    });
}

vlbm_status vlbm_set_populations(vlbm_hier* h, int32_t level, const double* f, int64_t ld, int32_t on_device) {
    return pop_copy(h, level, const_cast<double*>(f), ld, on_device, 0);
}

vlbm_status vlbm_get_populations(vlbm_hier* h, int32_t level, double* f, int64_t ld, int32_t on_device) {
    return pop_copy(h, level, f, ld, on_device, 1);
}

// Queues the copy of `rows` per-step totals (8 doubles each) from the
// device block `src` into the hierarchy's pinned history ring.
static void record_rows(vlbm_hier* h, const double* src, long long rows) {
    long long done = 0;
    while (done < rows) {
        const long long at = (h->hist_n + done) % h->hist_cap;
        const long long n = std::min(rows - done, h->hist_cap - at);
        VCK(cudaMemcpyAsync(h->hist + at * 8, src + done * 8, (size_t)n * 8 * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
        done += n;
    }
    h->hist_n += rows;
}

vlbm_status vlbm_advance(vlbm_hier* h, int64_t coarse_steps) {
    return run(h, [&] {
        if (coarse_steps < 0) throw Fail{VLBM_ERR_ARG, "negative step count"};
        if (h->engine) throw Fail{VLBM_ERR_ARG, "hierarchy is resident in an engine"};
        if (h->step_audit) settle_after_audit(h);
        if (!h->step_audit) {
            // on the device lists: nothing here waits for the GPU
            long long left = coarse_steps;
            while (left > 0) {
                const int sched = dev_schedule_mode(h);
                long long n = left;
                if (h->tune.schedule == 2 && sched == 0) n = std::min(left, h->tune.persist_after - h->layout_steps);
                dev_advance(h, n, sched);
                h->steps += n;
                h->layout_steps += n;
                left -= n;
            }
            return;
        }
        long long left = coarse_steps;
        while (left > 0) {
            const int sched = effective_schedule(h);
            // under auto, per-phase launches only up to the switch point
            long long n = left;
            if (h->tune.schedule == 2 && sched == 0) n = std::min(left, h->tune.persist_after - h->layout_steps);
            ensure_own_batch(h, sched);
            Batch& b = *h->own;
            if (!b.audit) {
                b.advance(n, h->stream);
            } else {
                long long m = n;
                if (m >= b.G) {
                    cudaGraphExec_t ex = b.exec_for(1, h->stream);
                    for (; m >= b.G; m -= b.G) {
                        VCK(cudaGraphLaunch(ex, h->stream));
                        b.count(ex);
                        record_rows(h, h->tl[1].aout.p, b.G);
                    }
                }
                if (m > 0) {
                    cudaGraphExec_t ex = b.exec_for(0, h->stream);
                    for (; m > 0; m--) {
                        VCK(cudaGraphLaunch(ex, h->stream));
                        b.count(ex);
                        record_rows(h, h->tl[0].aout.p, 1);
                    }
                }
            }
            h->steps += n;
            h->layout_steps += n;
            left -= n;
        }
        count_lups(h, coarse_steps);
        h->klaunch += 1;
    });
}

// ---- checkpoint / resume ---------------------------------------------------

namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, nlev, nx0, ny0, bc[4];
    double gamma, c, beta;
    int64_t steps;
    int32_t par0, pad;
};

size_t ckpt_bytes(const vlbm_hier* h) {
    size_t b = sizeof(CkptHeader);
    for (int l = 0; l < h->nlev; l++) {
        const Level& L = h->lev[l];
        b += 2 * (size_t)L.bx * L.by;                        // block maps
        b += (size_t)L.plane * sizeof(uint16_t);             // flags
        b += (size_t)16 * L.plane * sizeof(double);          // state buffer
    }
    return b;
}
}  // namespace

vlbm_status vlbm_checkpoint_size(vlbm_hier* h, size_t* bytes) {
    return run(h, [&] {
        if (!bytes) throw Fail{VLBM_ERR_ARG, "null size"};
        *bytes = ckpt_bytes(h);
    });
}

vlbm_status vlbm_checkpoint_save(vlbm_hier* h, void* blob, size_t bytes) {
    return run(h, [&] {
        if (!blob || bytes < ckpt_bytes(h)) throw Fail{VLBM_ERR_ARG, "blob too small"};
        VCK(cudaStreamSynchronize(h->stream));
        check_status(h);
        ensure_host(h);
        int par0 = 0;
        VCK(cudaMemcpy(&par0, h->words, sizeof(int), cudaMemcpyDeviceToHost));
        CkptHeader H{};
        std::memcpy(H.magic, "VLBMCKP1", 8);
        H.version = 1;
        H.nlev = h->nlev;
        H.nx0 = h->cfg.nx0;
        H.ny0 = h->cfg.ny0;
        for (int i = 0; i < 4; i++) H.bc[i] = h->cfg.bc[i];
        H.gamma = h->cfg.gamma;
        H.c = h->cfg.c;
        H.beta = h->cfg.beta;
        H.steps = h->steps;
        H.par0 = par0;
        char* p = (char*)blob;
        std::memcpy(p, &H, sizeof H);
        p += sizeof H;
        for (int l = 0; l < h->nlev; l++) {
            const Level& L = h->lev[l];
            std::memcpy(p, L.bin.data(), L.bin.size());
            p += L.bin.size();
            std::memcpy(p, L.bcov.data(), L.bcov.size());
            p += L.bcov.size();
            VCK(cudaMemcpy(p, L.flags, (size_t)L.plane * sizeof(uint16_t), cudaMemcpyDeviceToHost));
            p += (size_t)L.plane * sizeof(uint16_t);
            const double* st = L.buf[l == 0 ? par0 : 0];
            VCK(cudaMemcpy(p, st, (size_t)16 * L.plane * sizeof(double), cudaMemcpyDeviceToHost));
            p += (size_t)16 * L.plane * sizeof(double);
        }
    });
}

vlbm_status vlbm_checkpoint_load(vlbm_hier* h, const void* blob, size_t bytes) {
    return run(h, [&] {
        if (!blob || bytes < sizeof(CkptHeader)) throw Fail{VLBM_ERR_ARG, "blob too small"};
        if (h->engine) throw Fail{VLBM_ERR_ARG, "hierarchy is resident in an engine"};
        CkptHeader H;
        std::memcpy(&H, blob, sizeof H);
        if (std::memcmp(H.magic, "VLBMCKP1", 8) != 0 || H.version != 1) throw Fail{VLBM_ERR_ARG, "not a checkpoint"};
        bool same = H.nlev == h->nlev && H.nx0 == h->cfg.nx0 && H.ny0 == h->cfg.ny0 && H.gamma == h->cfg.gamma &&
                    H.c == h->cfg.c && H.beta == h->cfg.beta;
        for (int i = 0; i < 4; i++) same = same && H.bc[i] == h->cfg.bc[i];
        if (!same) throw Fail{VLBM_ERR_ARG, "checkpoint made under another configuration"};
        if (bytes < ckpt_bytes(h)) throw Fail{VLBM_ERR_ARG, "blob too small"};
        settle_after_audit(h);
        VCK(cudaStreamSynchronize(h->stream));
        const char* p = (const char*)blob + sizeof H;
        std::vector<uint8_t> bin[VLBM_MAX_LEVELS], bcov[VLBM_MAX_LEVELS];
        const char* q = p;
        for (int l = 0; l < h->nlev; l++) {
            const Level& L = h->lev[l];
            const size_t nb = (size_t)L.bx * L.by;
            bin[l].assign((const uint8_t*)q, (const uint8_t*)q + nb);
            bcov[l].assign((const uint8_t*)q + nb, (const uint8_t*)q + 2 * nb);
            q += 2 * nb + (size_t)L.plane * sizeof(uint16_t) + (size_t)16 * L.plane * sizeof(double);
        }
        std::string why;
        if (!nested(h, bin, bcov, why)) throw Fail{VLBM_ERR_ARG, "checkpoint layout: " + why};
        install_layout(h, bin, bcov);  // tables and lists; flags are overwritten below
        const int par0 = H.par0 & 1;
        VCK(cudaMemcpy(h->words, &par0, sizeof(int), cudaMemcpyHostToDevice));
        for (int l = 0; l < h->nlev; l++) {
            Level& L = h->lev[l];
            p += 2 * (size_t)L.bx * L.by;
            VCK(cudaMemcpy(L.flags, p, (size_t)L.plane * sizeof(uint16_t), cudaMemcpyHostToDevice));
            p += (size_t)L.plane * sizeof(uint16_t);
            VCK(cudaMemcpy(L.buf[l == 0 ? par0 : 0], p, (size_t)16 * L.plane * sizeof(double), cudaMemcpyHostToDevice));
            p += (size_t)16 * L.plane * sizeof(double);
        }
        h->steps = H.steps;
        invalidate(h);
        VCK(cudaDeviceSynchronize());
    });
}

vlbm_status vlbm_set_step_totals(vlbm_hier* h, int32_t on) {
    return run(h, [&] {
        if (on && h->tune.schedule == 0) throw Fail{VLBM_ERR_ARG, "per-step totals need the persistent schedule"};
        if (on && h->sensor_on) throw Fail{VLBM_ERR_ARG, "per-step totals and the relaxation sensor exclude each other"};
        if (on && !h->hist) h->hist = (double*)pin_alloc((size_t)h->hist_cap * 8 * sizeof(double));
        VCK(cudaStreamSynchronize(h->stream));
        if (on) ensure_host(h);
        h->step_audit = on != 0;
        h->hist_n = h->hist_read = 0;
        if (h->own) h->own->valid = false;
    });
}

vlbm_status vlbm_get_step_totals(vlbm_hier* h, double* out, int64_t cap, int64_t* n) {
    return run(h, [&] {
        if (!n || cap < 0 || (cap > 0 && !out)) throw Fail{VLBM_ERR_ARG, "bad arguments"};
        VCK(cudaStreamSynchronize(h->stream));
        check_status(h);
        long long avail = h->hist_n - h->hist_read;
        if (avail > h->hist_cap) avail = h->hist_cap;  // older rows were overwritten
        const long long take = std::min<long long>(avail, cap);
        const long long first = h->hist_n - take;  // the most recent `take` rows, oldest first
        for (long long r = 0; r < take; r++) std::memcpy(out + r * 8, h->hist + ((first + r) % h->hist_cap) * 8,
                                                         8 * sizeof(double));
        *n = take;
        h->hist_read = h->hist_n;
    });
}

vlbm_status vlbm_sync(vlbm_hier* h) {
    return run(h, [&] {
        VCK(cudaStreamSynchronize(h->stream));
        check_status(h);
    });
}

// Exact totals over the active cells of every level (two passes of
// 192-bit fixed-point sums); one 64-byte read-back.
static void audit_impl(vlbm_hier* h, double* totals, double* abs_totals) {
    if (!h->hout) h->hout = (double*)pin_alloc(8 * sizeof(double));
    VCK(launch_audit(h->atab.p, h->ditems, (int)std::min<size_t>(h->ditems_cap, 1u << 30), h->partial.p, h->tot.p,
                     h->aticket.p, h->stream, h->dcount));
    h->klaunch += 1;
    VCK(cudaMemcpyAsync(h->hout, h->tot.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    VCK(cudaStreamSynchronize(h->stream));
    if (totals) std::memcpy(totals, h->hout, 4 * sizeof(double));
    if (abs_totals) std::memcpy(abs_totals, h->hout + 4, 4 * sizeof(double));
}

vlbm_status vlbm_audit(vlbm_hier* h, double totals[4], double abs_totals[4]) {
    return run(h, [&] {
        audit_impl(h, totals, abs_totals);
        check_status(h);
    });
}

vlbm_status vlbm_get_conserved(vlbm_hier* h, int32_t level, double* W, int64_t ld, uint8_t* valid, double totals[4],
                               double abs_totals[4]) {
    return run(h, [&] {
        if (level < 0 || level >= h->nlev) throw Fail{VLBM_ERR_ARG, "bad level"};
        Level& L = h->lev[level];
        check_status(h);
        if (W || valid) {
            const long long ldd = W ? ld : L.nx;
            if (W && ld < L.nx) throw Fail{VLBM_ERR_ARG, "ld < nx"};
            const size_t n = (size_t)4 * ldd * L.ny;
            h->stage.ensure(h->mem, n);
            h->stage8.ensure(h->mem, (size_t)L.nx * L.ny);
            VCK(launch_gather_W(lvdev(h, level), h->stage.p, ldd, valid ? h->stage8.p : nullptr, h->stream));
            h->klaunch += 1;
            if (W) VCK(cudaMemcpyAsync(W, h->stage.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            if (valid)
                VCK(cudaMemcpyAsync(valid, h->stage8.p, (size_t)L.nx * L.ny, cudaMemcpyDeviceToHost, h->stream));
            VCK(cudaStreamSynchronize(h->stream));
        }
        if (totals || abs_totals) audit_impl(h, totals, abs_totals);
    });
}

vlbm_status vlbm_get_layout(vlbm_hier* h, int32_t level, uint8_t* in, uint8_t* ref) {
    return run(h, [&] {
        if (level < 0 || level >= h->nlev) throw Fail{VLBM_ERR_ARG, "bad level"};
        ensure_host(h);
        Level& L = h->lev[level];
        for (int y = 0; y < L.ny; y++)
            for (int x = 0; x < L.nx; x++) {
                const size_t b = (size_t)(y / TILE) * L.bx + x / TILE;
                if (in) in[(size_t)y * L.nx + x] = L.bin[b];
                if (ref) ref[(size_t)y * L.nx + x] = L.bin[b] && L.bcov[b];
            }
    });
}

vlbm_status vlbm_regrid_masks(vlbm_hier* h, const uint8_t* const* ref) {
    return run(h, [&] {
        check_status(h);
        settle_after_audit(h);
        std::vector<uint8_t> bcov[VLBM_MAX_LEVELS];
        masks_to_maps(h, ref, bcov);
        regrid_to(h, bcov, false);
        invalidate(h);
    });
}

vlbm_status vlbm_regrid(vlbm_hier* h, const vlbm_box* boxes, int32_t nboxes) {
    return run(h, [&] {
        auto t0 = std::chrono::steady_clock::now();
        settle_after_audit(h);
        if (boxes || nboxes > 0) {
            std::vector<uint8_t> bcov[VLBM_MAX_LEVELS];
            check_status(h);
            if (nboxes < 0 || !boxes) throw Fail{VLBM_ERR_ARG, "bad boxes"};
            boxes_to_maps(h, boxes, nboxes, bcov);
            h->times[VLBM_T_LAYOUT] += ms_since(t0);
            t0 = std::chrono::steady_clock::now();
            regrid_to(h, bcov, false);
            h->times[VLBM_T_REGRID] += ms_since(t0);
        } else if (!h->engine) {
            // on the device alone: queued, nothing waits
            device_regrid(h);
            h->times[VLBM_T_REGRID] += ms_since(t0);
        } else {
            tag_begin(h);
            t0 = std::chrono::steady_clock::now();
            VCK(cudaEventSynchronize(h->rg_ev));
            h->times[VLBM_T_TAG] += ms_since(t0);
            tag_finish(h);
        }
        h->times[VLBM_T_NREGRIDS] += 1;
        invalidate(h);
    });
}

vlbm_status vlbm_set_sensor(vlbm_hier* h, int32_t on, double beta_min, double c_sensor, double eps) {
    return run(h, [&] {
        if (h->engine) throw Fail{VLBM_ERR_ARG, "hierarchy is resident in an engine"};
        if (on && !(beta_min >= 0.0 && beta_min <= h->cfg.beta && c_sensor >= 0.0 && eps >= 0.0))
            throw Fail{VLBM_ERR_ARG, "bad sensor parameters"};
        if (on && h->step_audit) throw Fail{VLBM_ERR_ARG, "per-step totals and the relaxation sensor exclude each other"};
        ensure_host(h);
        cudaStream_t s = h->stream;
        if (on) {
            // the flux maxima over the active cells of every level, now
            h->qmax.ensure(h->mem, 4);
            VCK(cudaMemsetAsync(h->qmax.p, 0, 4 * sizeof(unsigned long long), s));
            for (int l = 0; l < h->nlev; l++) {
                h->listbuf.upload(h->mem, h->lev[l].act, s);
                VCK(launch_qmax(lvdev(h, l), h->listbuf.p, (int)h->listbuf.n, h->qmax.p, s));
            }
            unsigned long long q[4];
            VCK(cudaMemcpyAsync(q, h->qmax.p, sizeof q, cudaMemcpyDeviceToHost, s));
            VCK(cudaStreamSynchronize(s));
            for (int k = 0; k < 4; k++) {
                double m;
                std::memcpy(&m, &q[k], sizeof m);
                h->s_iq[k] = m > 0.0 ? 1.0 / (2.0 * m) : 0.0;
            }
            for (int l = 0; l < h->nlev; l++)
                if (!h->sens[l]) {
                    const size_t b = (size_t)SENS_PLANES * h->lev[l].plane * sizeof(double);
                    h->sens[l] = (double*)h->mem.get(b);
                    VCK(cudaMemsetAsync(h->sens[l], 0, b, s));
                }
            h->s_beta_min = beta_min;
            h->s_csens = c_sensor;
            h->s_eps = eps;
        }
        h->sensor_on = on != 0;
        refresh_atab(h);
        invalidate(h);
    });
}

vlbm_status vlbm_host_times(const vlbm_hier* h, double out[VLBM_T_COUNT]) {
    if (!h || !out) return VLBM_ERR_ARG;
    for (int i = 0; i < VLBM_T_COUNT; i++) out[i] = h->times[i];
    return VLBM_OK;
}

vlbm_status vlbm_get_info(const vlbm_hier* hc, vlbm_info* info) {
    if (!hc || !info) return VLBM_ERR_ARG;
    vlbm_hier* h = const_cast<vlbm_hier*>(hc);
    if (!h->host_ok) {  // the active cell counts of a layout made on the device
        const vlbm_status st = run(h, [&] { ensure_host(h); });
        if (st != VLBM_OK) return st;
    }
    std::memset(info, 0, sizeof *info);
    info->nlev = h->nlev;
    long long lups = 0;
    for (int l = 0; l < h->nlev; l++) {
        info->nx[l] = h->lev[l].nx;
        info->ny[l] = h->lev[l].ny;
        info->active_cells[l] = h->lev[l].active_cells;
        lups += h->lev[l].active_cells << l;
    }
    info->lups_per_step = lups;
    info->device_bytes = (int64_t)h->mem.bytes;
    info->steps = h->steps;
    info->c = h->cfg.c;
    info->beta = h->cfg.beta;
    info->gamma = h->cfg.gamma;
    info->dx0 = h->cfg.dx0;
    return VLBM_OK;
}

vlbm_status vlbm_selftest_layout(uint64_t seed, int32_t cases, int64_t* mismatches, int64_t* second_pass,
                                 char* first_bad, int32_t cap) {
    if (cases < 0 || !mismatches) return VLBM_ERR_ARG;
    *mismatches = 0;
    if (second_pass) *second_pass = 0;
    if (first_bad && cap > 0) first_bad[0] = 0;
    uint64_t st = seed;
    auto rnd = [&]() {  // SplitMix64
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto bad = [&](const std::string& why) {
        if (*mismatches == 0 && first_bad && cap > 0) std::snprintf(first_bad, (size_t)cap, "%s", why.c_str());
        (*mismatches)++;
    };
    for (int cs = 0; cs < cases; cs++) {
        vlbm_config cfg{};
        cfg.max_levels = 2 + (int)(rnd() % 3);
        cfg.nx0 = 4 + (int)(rnd() % 37);
        cfg.ny0 = 4 + (int)(rnd() % 37);
        cfg.dx0 = 1.0;
        const int bx = (rnd() & 1) ? VLBM_BC_PERIODIC : VLBM_BC_OUTFLOW, by = (rnd() & 1) ? VLBM_BC_PERIODIC : VLBM_BC_OUTFLOW;
        cfg.bc[0] = cfg.bc[1] = bx;
        cfg.bc[2] = cfg.bc[3] = by;
        cfg.gamma = 1.4;
        cfg.c = 5.0;
        cfg.beta = 0.9;
        vlbm_hier* h = nullptr;
        vlbm_status e = vlbm_create_hierarchy(&cfg, nullptr, nullptr, &h);
        if (e != VLBM_OK) return e;
        const vlbm_status r = run(h, [&] {
            const int nl = h->nlev;
            for (int round = 0; round < 3; round++) {
                // random block flags on every refinable level, some in clusters
                std::vector<uint8_t> bflag[VLBM_MAX_LEVELS], all;
                const int dens = 2 + (int)(rnd() % 40);  // percent
                for (int l = 0; l <= nl - 2; l++) {
                    const Level& L = h->lev[l];
                    bflag[l].assign((size_t)L.bx * L.by, 0);
                    for (auto& b : bflag[l]) b = (int)(rnd() % 100) < dens ? 1 : 0;
                    all.insert(all.end(), bflag[l].begin(), bflag[l].end());
                }
                std::vector<uint8_t> hcov[VLBM_MAX_LEVELS], hin[VLBM_MAX_LEVELS];
                layout_rule(h, bflag, hcov);
                derive_in(h, hin, hcov);
                std::string why;
                if (!nested(h, hin, hcov, why)) {
                    bad("host layout not nested: " + why);
                    return;
                }
                if (all.empty()) all.push_back(0);
                h->bflag.ensure(h->mem, all.size());
                VCK(cudaMemcpyAsync(h->bflag.p, all.data(), all.size(), cudaMemcpyHostToDevice, h->stream));
                device_apply_flags(h, h->bflag.p);
                h->host_ok = false;
                layout_changed(h);
                const int k = 1 + (int)(rnd() % 3);
                dev_plan(h, k, false);
                dev_plan(h, 1, true);
                VCK(cudaStreamSynchronize(h->stream));
                int stw[2];
                VCK(cudaMemcpy(stw, h->words, sizeof stw, cudaMemcpyDeviceToHost));
                if (stw[1]) bad("status word " + std::to_string(stw[1]));
                // maps and lists
                std::vector<TileLists> tl(nl);
                std::vector<TaskLevel> lv(nl);
                const bool px = bx == VLBM_BC_PERIODIC, py = by == VLBM_BC_PERIODIC;
                for (int l = 0; l < nl; l++) {
                    const Level& L = h->lev[l];
                    const LayoutDev& DL = L.dl;
                    const size_t nb = (size_t)L.bx * L.by;
                    std::vector<uint8_t> din(nb), dcov(nb), drec(nb);
                    VCK(cudaMemcpy(din.data(), DL.bin, nb, cudaMemcpyDeviceToHost));
                    VCK(cudaMemcpy(dcov.data(), DL.bcov, nb, cudaMemcpyDeviceToHost));
                    VCK(cudaMemcpy(drec.data(), DL.recon, nb, cudaMemcpyDeviceToHost));
                    if (din != hin[l]) bad("level " + std::to_string(l) + ": on-level map");
                    if (dcov != hcov[l]) bad("level " + std::to_string(l) + ": covered map");
                    tile_lists(l, L.nx, L.ny, L.bx, L.by, px, py, hin[l].data(), hcov[l].data(), tl[l]);
                    if (drec != tl[l].recon) bad("level " + std::to_string(l) + ": recon map");
                    int cnt[NLST];
                    VCK(cudaMemcpy(cnt, DL.cnt, sizeof cnt, cudaMemcpyDeviceToHost));
                    const std::vector<Item>* want[4] = {&tl[l].act, &tl[l].ring, &tl[l].cov, &tl[l].in};
                    for (int q = 0; q < 4; q++) {
                        std::vector<Item> got((size_t)cnt[q]);
                        if (cnt[q]) VCK(cudaMemcpy(got.data(), DL.list[q], got.size() * sizeof(Item), cudaMemcpyDeviceToHost));
                        bool same = got.size() == want[q]->size();
                        for (size_t i = 0; same && i < got.size(); i++)
                            same = got[i].tx == (*want[q])[i].tx && got[i].ty == (*want[q])[i].ty && got[i].lid == l;
                        if (!same) bad("level " + std::to_string(l) + ": list " + std::to_string(q));
                    }
                    unsigned long long cells = 0;
                    VCK(cudaMemcpy(&cells, DL.cells, sizeof cells, cudaMemcpyDeviceToHost));
                    if ((long long)cells != tl[l].active_cells) bad("level " + std::to_string(l) + ": active cells");
                    lv[l].nx = L.nx;
                    lv[l].ny = L.ny;
                    lv[l].bx = L.bx;
                    lv[l].by = L.by;
                    lv[l].px = px;
                    lv[l].py = py;
                    lv[l].act = &tl[l].act;
                    lv[l].ring = &tl[l].ring;
                    lv[l].recon = &tl[l].recon;
                }
                // task lists: the host builder against the device's
                auto compare_list = [&](const vlbm_hier::DevPlan& D, const std::vector<Task>& wt,
                                        const std::vector<int>& wd, int step_shift, const char* what) {
                    int need[5];
                    VCK(cudaMemcpy(need, D.need.p, sizeof need, cudaMemcpyDeviceToHost));
                    if (second_pass) *second_pass += need[4];
                    if (need[0] != (int)wt.size()) {
                        bad(std::string(what) + ": task count " + std::to_string(need[0]) + " vs " +
                            std::to_string(wt.size()));
                        return;
                    }
                    std::vector<Task> gt(wt.size());
                    if (!gt.empty())
                        VCK(cudaMemcpy(gt.data(), D.tasks.p, gt.size() * sizeof(Task), cudaMemcpyDeviceToHost));
                    // the dependency array as far as any task's slot reaches
                    long long reach = 0;
                    for (const Task& T : gt) reach = std::max(reach, (long long)T.dep0 + T.ndep);
                    std::vector<int> gd((size_t)reach);
                    if (reach) VCK(cudaMemcpy(gd.data(), D.deps.p, (size_t)reach * sizeof(int), cudaMemcpyDeviceToHost));
                    for (size_t i = 0; i < gt.size(); i++) {
                        const Task &x = gt[i], &y = wt[i];
                        const int ya = y.kind == 0 ? -1 : y.aslot;  // no audit slots on the device lists
                        bool same = x.lid == y.lid && x.tx == y.tx && x.ty == y.ty && x.kind == y.kind && x.kk == y.kk &&
                                    x.kkp == y.kkp && x.step + step_shift == y.step && x.ndep == y.ndep && x.aslot == ya;
                        for (int q = 0; same && q < x.ndep; q++) same = gd[x.dep0 + q] == wd[y.dep0 + q];
                        if (!same) {
                            bad(std::string(what) + ": task " + std::to_string(i) + " of " + std::to_string(gt.size()) +
                                " (kind " + std::to_string(y.kind) + ", level " + std::to_string(y.lid) + ", ndep " +
                                std::to_string(x.ndep) + " vs " + std::to_string(y.ndep) + ")");
                            break;
                        }
                    }
                };
                TaskLists want;
                build_tasks(lv, k, want);
                compare_list(h->dp[1], want.t, want.d, 0, "k-step list");
                // the cyclic one-step list is the second step of a two-step
                // list from a synchronised state: dependencies into its first
                // step become ~index, those within it lose the step's offset
                TaskLists two;
                build_tasks(lv, 2, two);
                const int m = (int)two.t.size() / 2;
                std::vector<Task> ct(two.t.begin() + m, two.t.end());
                std::vector<int> cd;
                for (Task& T : ct) {
                    std::vector<int> v(two.d.begin() + T.dep0, two.d.begin() + T.dep0 + T.ndep);
                    for (int& d : v) d = d >= m ? d - m : ~d;
                    std::sort(v.begin(), v.end());
                    T.dep0 = (int)cd.size();
                    cd.insert(cd.end(), v.begin(), v.end());
                }
                compare_list(h->dp[0], ct, cd, 1, "cyclic list");
            }
        });
        vlbm_destroy(h);
        if (r != VLBM_OK) return r;
    }
    return VLBM_OK;
}

vlbm_status vlbm_kernels_launched(const vlbm_hier* h, int64_t* n) {
    if (!h || !n) return VLBM_ERR_ARG;
    *n = h->klaunch;
    return VLBM_OK;
}

vlbm_status vlbm_lups_mark(vlbm_hier* h, int64_t* dst) {
    return run(h, [&] {
        if (!dst) throw Fail{VLBM_ERR_ARG, "null destination"};
        VCK(cudaMemcpyAsync(dst, h->lupc, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    });
}

vlbm_status vlbm_set_regrid_audit(vlbm_hier* h, int32_t on) {
    return run(h, [&] {
        if (on && !h->raud) {
            h->raud = (double*)h->mem.get((size_t)vlbm_hier::RA_CAP * 16 * sizeof(double));
            VCK(cudaMemsetAsync(h->raud, 0, (size_t)vlbm_hier::RA_CAP * 16 * sizeof(double), h->stream));
        }
        h->regrid_audit = on != 0;
        h->ra_n = h->ra_read = 0;
        h->after_pending = -1;  // its row is dropped with the others
    });
}

vlbm_status vlbm_get_regrid_audits(vlbm_hier* h, double* out, int64_t cap, int64_t* n) {
    return run(h, [&] {
        if (!n || cap < 0 || (cap > 0 && !out)) throw Fail{VLBM_ERR_ARG, "bad arguments"};
        settle_after_audit(h);
        VCK(cudaStreamSynchronize(h->stream));
        check_status(h);
        long long avail = h->ra_n - h->ra_read;
        if (avail > vlbm_hier::RA_CAP) avail = vlbm_hier::RA_CAP;  // older rows were overwritten
        const long long take = std::min<long long>(avail, cap);
        const long long first = h->ra_n - take;  // the most recent `take` rows, oldest first
        for (long long r = 0; r < take; r++)
            VCK(cudaMemcpy(out + r * 16, h->raud + ((first + r) % vlbm_hier::RA_CAP) * 16, 16 * sizeof(double),
                           cudaMemcpyDeviceToHost));
        *n = take;
        h->ra_read = h->ra_n;
    });
}

vlbm_status vlbm_lups_done(vlbm_hier* h, int64_t* lups) {
    return run(h, [&] {
        if (!lups) throw Fail{VLBM_ERR_ARG, "null output"};
        unsigned long long v = 0;
        VCK(cudaMemcpyAsync(&v, h->lupc, sizeof v, cudaMemcpyDeviceToHost, h->stream));
        VCK(cudaStreamSynchronize(h->stream));
        check_status(h);
        *lups = (int64_t)v;
    });
}

int32_t vlbm_num_variants(void) { return sweep_variants(); }

vlbm_status vlbm_set_tuning(vlbm_hier* h, const vlbm_tuning* t) {
    return run(h, [&] {
        if (!t || t->variant < 0 || t->variant >= sweep_variants() || t->max_ctas < 0 || t->graph_steps < 1 ||
            t->graph_steps > 64 || t->schedule < 0 || t->schedule > 2 || t->persist_after < 0)
            throw Fail{VLBM_ERR_ARG, "bad tuning"};
        if (h->step_audit && t->schedule == 0) throw Fail{VLBM_ERR_ARG, "per-step totals need the persistent schedule"};
        h->tune = *t;
        h->tl[0].steps = h->tl[1].steps = -1;
        if (h->own) h->own->valid = false;
    });
}

vlbm_status vlbm_get_tuning(const vlbm_hier* h, vlbm_tuning* t) {
    if (!h || !t) return VLBM_ERR_ARG;
    *t = h->tune;
    return VLBM_OK;
}

vlbm_status vlbm_profile(vlbm_hier* h, int64_t coarse_steps, vlbm_kernel_time* out, int32_t cap, int32_t* n) {
    return run(h, [&] {
        if (coarse_steps < 0 || !out || !n) throw Fail{VLBM_ERR_ARG, "bad profile arguments"};
        if (h->engine) throw Fail{VLBM_ERR_ARG, "hierarchy is resident in an engine"};
        settle_after_audit(h);
        ensure_own_batch(h, effective_schedule(h));  // profile() launches phase by phase
        count_lups(h, coarse_steps);
        long long cells[VLBM_MAX_LEVELS] = {};
        for (int l = 0; l < h->nlev; l++) cells[l] = h->lev[l].active_cells;
        std::vector<Batch::Rec> recs;
        h->own->profile(coarse_steps, cells, recs, h->stream);
        for (const auto& r : recs) h->klaunch += r.launches;
        h->steps += coarse_steps;
        h->layout_steps += coarse_steps;
        if ((int)recs.size() > cap) throw Fail{VLBM_ERR_ARG, "record capacity too small"};
        for (size_t i = 0; i < recs.size(); i++) {
            out[i].kind = recs[i].kind;
            out[i].level = recs[i].level;
            out[i].launches = recs[i].launches;
            out[i].cells = recs[i].cells;
            out[i].ms = recs[i].ms;
        }
        *n = (int32_t)recs.size();
    });
}

// ---- engine ------------------------------------------------------------------

vlbm_status vlbm_engine_create(size_t mem_budget, const vlbm_allocator* alloc, void* stream, vlbm_engine** out) {
    if (!out) return VLBM_ERR_ARG;
    *out = nullptr;
    if (alloc && (!alloc->alloc || !alloc->free)) return VLBM_ERR_ARG;
    vlbm_engine* e = new (std::nothrow) vlbm_engine();
    if (!e) return VLBM_ERR_OOM;
    e->budget = mem_budget;
    if (alloc) {
        e->mem.a = *alloc;
        e->mem.has = true;
    }
    if (stream) {
        e->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete e;
            return VLBM_ERR_CUDA;
        }
        e->own_stream = true;
    }
    e->mem.s = e->stream;
    e->batch.mem = &e->mem;
    e->batch.schedule_mode = 0;
    e->batch.variant = 1;  // three CTAs per SM (the single-hierarchy default)
    *out = e;
    return VLBM_OK;
}

vlbm_status vlbm_engine_set_schedule(vlbm_engine* e, int32_t schedule) {
    if (!e || (schedule != 0 && schedule != 1)) return VLBM_ERR_ARG;
    e->schedule = schedule;
    return VLBM_OK;
}

vlbm_status vlbm_engine_slot_stats(const vlbm_engine* e, int32_t slot, int64_t* steps_done, int64_t* lups_done) {
    if (!e || slot < 0 || slot >= (int)e->res.size() || !e->res[slot].live) return VLBM_ERR_ARG;
    if (steps_done) *steps_done = e->res[slot].done;
    if (lups_done) *lups_done = e->res[slot].lups;
    return VLBM_OK;
}

vlbm_status vlbm_engine_host_times(const vlbm_engine* e, double out[VLBM_ET_COUNT]) {
    if (!e || !out) return VLBM_ERR_ARG;
    for (int i = 0; i < VLBM_ET_COUNT; i++) out[i] = e->times[i];
    return VLBM_OK;
}

vlbm_status vlbm_engine_usage(const vlbm_engine* e, int32_t* residents, int64_t* bytes) {
    if (!e) return VLBM_ERR_ARG;
    int n = 0;
    long long b = 0;
    for (const auto& r : e->res)
        if (r.live) {
            n++;
            b += (long long)r.h->device_bytes();
        }
    if (residents) *residents = n;
    if (bytes) *bytes = b;
    return VLBM_OK;
}

vlbm_status vlbm_engine_admit(vlbm_engine* e, vlbm_hier* h, int64_t coarse_steps, int32_t regrid_every, int32_t* slot) {
    if (!e || !h || coarse_steps < 0 || regrid_every < 0) return VLBM_ERR_ARG;
    if (h->poisoned) return VLBM_ERR_STATE;
    if (h->engine) return VLBM_ERR_ARG;
    long long used = 0;
    for (const auto& r : e->res)
        if (r.live) used += (long long)r.h->device_bytes();
    if (e->budget && (size_t)(used + (long long)h->device_bytes()) > e->budget) return VLBM_ERR_OOM;
    // the hierarchy's own queue must be drained before it joins the engine,
    // with its layout on the host (and the totals after its last regrid)
    if (run(h, [&] { settle_after_audit(h); }) != VLBM_OK) return VLBM_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return VLBM_ERR_CUDA;
    if (run(h, [&] { ensure_host(h); }) != VLBM_OK) return VLBM_ERR_CUDA;
    int s = -1;
    for (size_t i = 0; i < e->res.size(); i++)
        if (!e->res[i].live) { s = (int)i; break; }
    if (s < 0) {
        s = (int)e->res.size();
        e->res.emplace_back();
    }
    if (coarse_steps == 0) {
        // nothing to do: reported finished by the next call, once this event
        // (recorded before the slot is published) has completed
        auto& r = e->res[s];
        if (!r.ev && cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess) return VLBM_ERR_CUDA;
        if (cudaEventRecord(r.ev, e->stream) != cudaSuccess) return VLBM_ERR_CUDA;
    }
    e->res[s].h = h;
    e->res[s].target = coarse_steps;
    e->res[s].done = 0;
    e->res[s].paused = false;
    e->res[s].tagging = false;
    e->res[s].finishing = false;
    e->res[s].reported = false;
    e->res[s].regridded_at = -1;
    e->admitted = true;
    e->res[s].regrid_every = regrid_every;
    e->res[s].lups = 0;
    e->res[s].live = true;
    h->engine = e;
    e->dirty = true;
    if (coarse_steps == 0) e->res[s].finishing = true;
    // completion marks the hierarchy's own launches left could pass for the
    // engine's epochs: they restart with the engine
    if (h->dp[0].done.p &&
        cudaMemsetAsync(h->dp[0].done.p, 0, h->dp[0].done.cap * sizeof(unsigned), e->stream) != cudaSuccess)
        return VLBM_ERR_CUDA;
    if (slot) *slot = s;
    return VLBM_OK;
}

vlbm_status vlbm_engine_release(vlbm_engine* e, int32_t slot) {
    if (!e || slot < 0 || slot >= (int)e->res.size() || !e->res[slot].live) return VLBM_ERR_ARG;
    // a resident reported finished has no work left in flight; any other
    // may still be in a queued launch
    if (!e->res[slot].reported) cudaStreamSynchronize(e->stream);
    if (e->res[slot].tagging) {
        // a regrid left half done: its copies land before the slot is free
        cudaEventSynchronize(e->res[slot].h->rg_ev);
        e->res[slot].tagging = false;
    }
    e->res[slot].h->engine = nullptr;
    e->res[slot].live = false;
    e->res[slot].h = nullptr;
    e->dirty = true;
    e->admitted = true;
    return VLBM_OK;
}

vlbm_status vlbm_engine_advance(vlbm_engine* e, int32_t max_steps, int32_t* finished, int32_t* nfinished,
                                int32_t* steps) {
    if (!e || max_steps < 1) return VLBM_ERR_ARG;
    if (nfinished) *nfinished = 0;
    if (steps) *steps = 0;
    try {
        // 0. second halves of the regrids whose block flags have arrived (all
        //    of them, waiting, when no other resident can step); the
        //    resident's steps resume after its regrid's kernels
        auto t0 = std::chrono::steady_clock::now();
        e->times[VLBM_ET_CALLS] += 1;
        auto can_step = [&] {
            for (const auto& r : e->res)
                if (r.live && !r.paused && r.done < r.target) return true;
            return false;
        };
        bool runnable = can_step();
        for (auto& r : e->res) {
            if (!r.live || !r.tagging) continue;
            vlbm_hier* h = r.h;
            const cudaError_t q = runnable ? cudaEventQuery(h->rg_ev) : cudaEventSynchronize(h->rg_ev);
            if (q == cudaErrorNotReady) continue;
            VCK(q);
            on_stream(h, e->hi, [&] { tag_finish(h); });
            VCK(cudaEventRecord(r.ev, e->hi));
            VCK(cudaStreamWaitEvent(e->stream, r.ev, 0));
            h->times[VLBM_T_NREGRIDS] += 1;
            if (h->own) h->own->valid = false;
            r.tagging = false;
            r.paused = false;
            r.regridded_at = r.done;
            e->dirty = true;
            e->regridded = true;
        }
        e->times[VLBM_ET_REGRID_FINISH] += ms_since(t0);
        // residents whose last step has completed on the GPU are reported
        // finished (waiting for them when no other resident can step), after
        // a look at their status words
        t0 = std::chrono::steady_clock::now();
        runnable = can_step();
        int nf = 0;
        for (size_t i = 0; i < e->res.size(); i++) {
            auto& r = e->res[i];
            if (!r.live || !r.finishing) continue;
            const cudaError_t q = runnable ? cudaEventQuery(r.ev) : cudaEventSynchronize(r.ev);
            if (q == cudaErrorNotReady) continue;
            VCK(q);
            int st[2];
            VCK(cudaMemcpy(st, r.h->words, sizeof st, cudaMemcpyDeviceToHost));
            if (st[1]) {
                r.h->poisoned = true;
                r.h->err = (st[1] & ST_NONPHYS)  ? "non-physical state"
                           : (st[1] & ST_TIMEOUT) ? "a bounded device wait timed out"
                           : (st[1] & ST_TASKCAP) ? "task list or footprint capacity exceeded"
                                                  : "device status " + std::to_string(st[1]);
            }
            r.finishing = false;
            r.reported = true;
            if (finished) finished[nf] = (int)i;
            nf++;
        }
        e->times[VLBM_ET_FINISH] += ms_since(t0);
        // 1. adaptive residents due for a regrid leave the batches; an event
        //    marks the end of their last step on the engine's stream
        std::vector<size_t> due;
        for (size_t i = 0; i < e->res.size(); i++) {
            auto& r = e->res[i];
            if (!r.live || !r.adaptive() || r.paused) continue;
            if (r.done > 0 && r.done % r.regrid_every == 0 && r.done < r.target && r.regridded_at != r.done) {
                if (!r.ev) VCK(cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming));
                VCK(cudaEventRecord(r.ev, e->stream));
                r.paused = true;
                due.push_back(i);
                e->dirty = true;
            }
        }
        t0 = std::chrono::steady_clock::now();
        if (e->dirty) {
            // rebuild the launch tables when the members changed or one of
            // them regridded (an admission or release since the last rebuild
            // always counts as a change: a new hierarchy may sit at a released
            // one's address)
            std::vector<vlbm_hier*> ms;
            for (auto& r : e->res)
                if (r.live && !r.paused && r.done < r.target) ms.push_back(r.h);
            if (e->admitted || e->regridded || ms != e->batch.members || !e->batch.valid) {
                e->batch.members = ms;
                if (!ms.empty()) e->batch.build(e->stream);
            }
            e->admitted = e->regridded = false;
            e->dirty = false;
        }
        e->times[VLBM_ET_REBUILD] += ms_since(t0);
        // 2. as many steps of the other residents as none of them finishes or
        //    regrids in between
        long long k = max_steps;
        bool any = false;
        for (const auto& r : e->res) {
            if (!r.live || r.paused || r.done >= r.target) continue;
            any = true;
            k = std::min(k, r.target - r.done);
            if (r.adaptive()) k = std::min<long long>(k, r.regrid_every - r.done % r.regrid_every);
        }
        if (!any) k = 0;
        // the per-phase launches are issued directly: the batch changes at
        // nearly every call (admissions, finishes, regrids), so capturing and
        // instantiating a graph each time would cost more than the launches
        if (k > 0) {
            t0 = std::chrono::steady_clock::now();
            // the persistent launch takes at most 64 steps, and its tickets
            // (tasks of one step of every resident x steps) must fit an int
            long long cap = 0;
            for (vlbm_hier* h : e->batch.members) cap += h->dp[0].task_cap > 0 ? h->dp[0].task_cap : 1LL << 20;
            if (e->schedule == 1 && !e->batch.sensor && k <= 64 && cap * k < (1LL << 31) - 1)
                e->batch.device_steps(k, e->stream);
            else
                for (long long i = 0; i < k; i++) e->batch.one_step(e->stream);
            e->times[VLBM_ET_LAUNCH] += ms_since(t0);
            t0 = std::chrono::steady_clock::now();
            int& c = e->lead_i;
            if (!e->lead[c]) VCK(cudaEventCreateWithFlags(&e->lead[c], cudaEventDisableTiming));
            if (e->lead_set[c]) VCK(cudaEventSynchronize(e->lead[c]));  // the steps of LEAD calls ago
            VCK(cudaEventRecord(e->lead[c], e->stream));
            e->lead_set[c] = true;
            c = (c + 1) % vlbm_engine::LEAD;
            e->times[VLBM_ET_LEAD] += ms_since(t0);
            e->times[VLBM_ET_STEPS] += (double)k;
        }
        for (size_t i = 0; i < e->res.size(); i++) {
            auto& r = e->res[i];
            if (!r.live || r.paused || r.done >= r.target || k == 0) continue;
            r.done += k;
            r.h->steps += k;
            r.h->layout_steps += k;
            long long per = 0;
            for (int l = 0; l < r.h->nlev; l++) per += r.h->lev[l].active_cells << l;
            r.lups += per * k;
            if (r.done == r.target) {
                // reported by a later call, once this event has completed
                if (!r.ev) VCK(cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming));
                VCK(cudaEventRecord(r.ev, e->stream));
                r.finishing = true;
                e->dirty = true;
            }
        }
        // 3. the first halves of the due residents' regrids, after their
        //    events, on the engine's high-priority stream (its small kernels
        //    are scheduled at the next launch boundary instead of queueing
        //    behind every step already queued); nothing waits for them here:
        //    a later call finishes each regrid once its block flags are on
        //    the host, while the other residents keep stepping
        if (!due.empty() && !e->hi) {
            int lo = 0, hi = 0;
            VCK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            VCK(cudaStreamCreateWithPriority(&e->hi, cudaStreamNonBlocking, hi));
        }
        t0 = std::chrono::steady_clock::now();
        for (size_t i : due) {
            auto& r = e->res[i];
            vlbm_hier* h = r.h;
            VCK(cudaStreamWaitEvent(e->hi, r.ev, 0));
            on_stream(h, e->hi, [&] { tag_begin(h); });
            r.tagging = true;
        }
        e->times[VLBM_ET_REGRID_BEGIN] += ms_since(t0);
        if (nfinished) *nfinished = nf;
        if (steps) *steps = (int32_t)k;
        return VLBM_OK;
    } catch (const Fail& f) {
        e->err = f.msg;
        return f.st;
    }
}

vlbm_status vlbm_engine_step(vlbm_engine* e, int32_t* finished, int32_t* nfinished) {
    return vlbm_engine_advance(e, 1, finished, nfinished, nullptr);
}

void vlbm_engine_destroy(vlbm_engine* e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    if (e->hi) cudaStreamSynchronize(e->hi);
    for (cudaEvent_t& ev : e->lead)
        if (ev) cudaEventDestroy(ev), ev = nullptr;
    for (auto& r : e->res) {
        if (r.live && r.h) r.h->engine = nullptr;
        if (r.ev) cudaEventDestroy(r.ev);
        r.ev = nullptr;
    }
    e->batch.release();
    cudaStreamSynchronize(e->stream);
    if (e->hi) cudaStreamDestroy(e->hi);
    if (e->own_stream) cudaStreamDestroy(e->stream);
    delete e;
}

}  // extern "C"
