// Task lists of the persistent schedule (host code; no CUDA).
//
// One coarse step of a hierarchy is the recursive phase sequence of the
// sub-cycle (Sec. 3.2, Fig. 1): the sweep of level l, then for every level
// l + 1 two sub-steps of the same sequence, then the reflux close of level l
// (Sec. 3.3, Eq. 24).  A task is one 8 x 8 tile of one phase.  Its
// dependencies are the tasks it must wait for, derived per resource -- each
// tile of each level's two population buffers and of its flag plane:
//   * a read waits for the writers of the last phase that wrote the resource
//     (read-after-write);
//   * a write waits for the writers of the last phase that wrote it and for
//     every task that read it since (write-after-write, write-after-read);
//   * tasks of one phase never wait for one another: a phase's writers write
//     disjoint cells, and no phase reads what it writes.
// What each phase touches:
//   sweep of level l, tile T   reads src(l) at T; writes dst(l) at T and its
//                              four face neighbours (push streaming); on a
//                              tile next to coarser land also reads both
//                              buffers and the flags of the parent's tiles
//                              under its footprint (Eqs. 20-23)
//   close of level l, tile T   reads both buffers of the child's tiles under
//                              T; writes dst(l) and the flags at T
//
// Two builders produce the same order.  build_tasks_tracked replays the
// phases in order and keeps, per resource, its last writers and the readers
// since -- the plain definition, kept as the reference.  build_tasks derives
// each task's dependencies on its own: the phase sequence is known, and which
// tasks of a phase touch a given tile follows from the tile maps, so every
// task is independent (and the work can be split across host threads).  It also
// leaves out the write-after-write edges that a write-after-read edge
// already implies (a reader waits for every writer it read from), so its
// lists have the same transitive closure with fewer edges.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <thread>
#include <vector>

#include "vlbm_dev.cuh"

namespace vlbm {

constexpr int TASK_MAX_LEVELS = 4;  // the phase recursion always walks 4 levels

// Tile lists of one level from its block maps.
struct TileLists {
    std::vector<Item> act;       // on the level and not covered (swept)
    std::vector<Item> ring;      // active with a covered face neighbour (closed)
    std::vector<Item> cov;       // covered by the next level
    std::vector<Item> in;        // on the level
    std::vector<uint8_t> recon;  // per tile: active with a face neighbour off the level
    long long active_cells = 0;
};

inline void tile_lists(int level, int nx, int ny, int bx, int by, bool px, bool py, const uint8_t* bin,
                       const uint8_t* bcov, TileLists& o) {
    o.act.clear();
    o.ring.clear();
    o.cov.clear();
    o.in.clear();
    o.recon.assign((size_t)bx * by, 0);
    o.active_cells = 0;
    const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
    for (int jb = 0; jb < by; jb++)
        for (int ib = 0; ib < bx; ib++) {
            const size_t b = (size_t)jb * bx + ib;
            if (!bin[b]) continue;
            const Item it{level, (unsigned short)ib, (unsigned short)jb};
            o.in.push_back(it);
            if (bcov[b]) {
                o.cov.push_back(it);
                continue;
            }
            o.act.push_back(it);
            o.active_cells += (long long)(std::min(nx, ib * TILE + TILE) - ib * TILE) *
                              (std::min(ny, jb * TILE + TILE) - jb * TILE);
            bool ring = false, rec = false;
            for (int d = 0; d < 4; d++) {
                int i2 = ib + di[d], j2 = jb + dj[d];
                if (i2 < 0 || i2 >= bx) {
                    if (!px) continue;
                    i2 = (i2 + bx) % bx;
                }
                if (j2 < 0 || j2 >= by) {
                    if (!py) continue;
                    j2 = (j2 + by) % by;
                }
                const size_t b2 = (size_t)j2 * bx + i2;
                ring = ring || (bin[b2] && bcov[b2]);
                rec = rec || !bin[b2];
            }
            if (ring) o.ring.push_back(it);
            o.recon[b] = rec;
        }
}

// One level of one hierarchy as the task builders see it.
struct TaskLevel {
    int nx = 0, ny = 0, bx = 0, by = 0;  // cells, tiles
    bool px = false, py = false;         // periodic
    const std::vector<Item>* act = nullptr;
    const std::vector<Item>* ring = nullptr;
    const std::vector<uint8_t>* recon = nullptr;
};

struct TaskLists {
    std::vector<Task> t;
    std::vector<int> d;
};

namespace taskdetail {

// relative buffer ids: level 0 at coarse step s reads (s & 1) and writes the
// other; level >= 1 at sub-step 1 reads 0 and writes 1, at sub-step 2 the
// reverse
inline int src_of(int level, int kk, int step) { return level == 0 ? (step & 1) : (kk == 1 ? 0 : 1); }

inline int wrap(int v, int n, bool per, bool& ok) {
    if (v < 0 || v >= n) {
        if (!per) {
            ok = false;
            return 0;
        }
        v = (v % n + n) % n;
    }
    return v;
}

// the five tiles a sweep of tile (tx, ty) writes (push streaming)
const int SDI[5] = {0, 1, -1, 0, 0}, SDJ[5] = {0, 0, 0, 1, -1};

// Parent tiles read by the reconstruction of fine tile (tx, ty): the coarse
// tiles under the coarse cells [4 t - 1, 4 t + 4] in each direction.
inline int footprint(const TaskLevel& P, int tx, int ty, int* keys) {
    int ns = 0;
    const int c0x = tx * TILE / 2 - 1, c1x = tx * TILE / 2 + TILE / 2;
    const int c0y = ty * TILE / 2 - 1, c1y = ty * TILE / 2 + TILE / 2;
    for (int cy2 = c0y; cy2 <= c1y; cy2++)
        for (int cx2 = c0x; cx2 <= c1x; cx2++) {
            bool ok = true;
            const int xx = wrap(cx2, P.nx, P.px, ok), yy = wrap(cy2, P.ny, P.py, ok);
            if (!ok) continue;
            const int key = (yy / TILE) * P.bx + xx / TILE;
            bool dup = false;
            for (int q = 0; q < ns; q++) dup = dup || keys[q] == key;
            if (dup || ns == 16) continue;
            keys[ns++] = key;
        }
    return ns;
}

struct Phase {
    int kind;  // 0 sweep, 1 close
    int l, kk, kkp, step;
    bool first;
    int offset, count;  // task range
};

// The phase sequence of nsteps coarse steps (identical for both builders).
inline void phases(int nlev, int nsteps, const std::vector<TaskLevel>& lev, std::vector<Phase>& out) {
    out.clear();
    int off = 0;
    struct Rec {
        static void run(int nlev, const std::vector<TaskLevel>& lev, int l, int kk, int kkp, int step, bool first,
                        std::vector<Phase>& out, int& off) {
            const int ns = l < nlev ? (int)lev[l].act->size() : 0;
            out.push_back(Phase{0, l, kk, kkp, step, first, off, ns});
            off += ns;
            if (l + 1 < TASK_MAX_LEVELS) {
                run(nlev, lev, l + 1, 1, kk, step, first, out, off);
                run(nlev, lev, l + 1, 2, kk, step, false, out, off);
                const int nc = l + 1 < nlev ? (int)lev[l].ring->size() : 0;
                out.push_back(Phase{1, l, kk, 0, step, false, off, nc});
                off += nc;
            }
        }
    };
    for (int st = 0; st < nsteps; st++) Rec::run(nlev, lev, 0, 0, 0, st, true, out, off);
}

inline Task make_task(const Phase& ph, const Item& it) {
    Task T{};
    T.lid = ph.l;
    T.tx = it.tx;
    T.ty = it.ty;
    T.kind = (signed char)ph.kind;
    T.kk = (signed char)ph.kk;
    T.kkp = (signed char)(ph.kind == 0 ? ph.kkp : 0);
    T.step = (signed char)ph.step;
    T.aslot = (ph.kind == 0 && ph.first) ? -2 : -1;  // -2: audited sweep (slot assigned by the caller)
    return T;
}

}  // namespace taskdetail

// ---- reference builder: replay with per-resource state ---------------------

inline void build_tasks_tracked(const std::vector<TaskLevel>& lev, int nsteps, TaskLists& out) {
    using namespace taskdetail;
    const int nlev = (int)lev.size();
    struct Res {
        int phase = -1;
        std::vector<int> writers, readers, prior;
    };
    std::vector<std::vector<Res>> r(nlev);
    for (int l = 0; l < nlev; l++) r[l].assign((size_t)3 * lev[l].bx * lev[l].by, Res{});
    auto at = [&](int l, int kind, int tx, int ty) -> Res& {
        return r[l][((size_t)kind * lev[l].by + ty) * lev[l].bx + tx];
    };
    std::vector<int> cur;
    auto add = [&](const std::vector<int>& v, int task) {
        for (int q : v)
            if (q != task) cur.push_back(q);
    };
    auto read = [&](int l, int kind, int tx, int ty, int task) {
        Res& x = at(l, kind, tx, ty);
        add(x.writers, task);
        if (x.readers.empty() || x.readers.back() != task) x.readers.push_back(task);
    };
    auto write = [&](int l, int kind, int tx, int ty, int task, int phase) {
        Res& x = at(l, kind, tx, ty);
        if (x.phase != phase) {
            x.prior.swap(x.writers);
            x.prior.insert(x.prior.end(), x.readers.begin(), x.readers.end());
            x.writers.clear();
            x.readers.clear();
            x.phase = phase;
        }
        add(x.prior, task);
        if (x.writers.empty() || x.writers.back() != task) x.writers.push_back(task);
    };
    std::vector<Phase> ph;
    phases(nlev, nsteps, lev, ph);
    out.t.clear();
    out.d.clear();
    for (int p = 0; p < (int)ph.size(); p++) {
        const Phase& P = ph[p];
        if (!P.count) continue;
        const int l = P.l;
        const TaskLevel& L = lev[l];
        const std::vector<Item>& tiles = P.kind == 0 ? *L.act : *L.ring;
        for (const Item& it : tiles) {
            const int t = (int)out.t.size();
            cur.clear();
            if (P.kind == 0) {
                const int bs = src_of(l, P.kk, P.step), bd = bs ^ 1;
                read(l, bs, it.tx, it.ty, t);
                for (int d = 0; d < 5; d++) {
                    bool ok = true;
                    const int tx = wrap(it.tx + SDI[d], L.bx, L.px, ok);
                    const int ty = wrap(it.ty + SDJ[d], L.by, L.py, ok);
                    if (ok) write(l, bd, tx, ty, t, p);
                }
                if (l > 0 && (*L.recon)[(size_t)it.ty * L.bx + it.tx]) {
                    const TaskLevel& Pl = lev[l - 1];
                    const int pbs = src_of(l - 1, P.kkp, P.step), pbd = pbs ^ 1;
                    int keys[16];
                    const int nk = footprint(Pl, it.tx, it.ty, keys);
                    for (int q = 0; q < nk; q++) {
                        const int cx = keys[q] % Pl.bx, cy = keys[q] / Pl.bx;
                        read(l - 1, pbs, cx, cy, t);
                        read(l - 1, pbd, cx, cy, t);
                        read(l - 1, 2, cx, cy, t);
                    }
                }
            } else {
                const int bd = src_of(l, P.kk, P.step) ^ 1;
                const TaskLevel& C = lev[l + 1];
                for (int b = 0; b < 2; b++)
                    for (int a = 0; a < 2; a++) {
                        const int fx = 2 * it.tx + a, fy = 2 * it.ty + b;
                        if (fx >= C.bx || fy >= C.by) continue;
                        read(l + 1, 0, fx, fy, t);
                        read(l + 1, 1, fx, fy, t);
                    }
                write(l, bd, it.tx, it.ty, t, p);
                write(l, 2, it.tx, it.ty, t, p);
            }
            std::sort(cur.begin(), cur.end());
            cur.erase(std::unique(cur.begin(), cur.end()), cur.end());
            Task T = make_task(P, it);
            T.dep0 = (int)out.d.size();
            T.ndep = (int)cur.size();
            out.d.insert(out.d.end(), cur.begin(), cur.end());
            out.t.push_back(T);
        }
    }
}

// ---- fast builder: every task's dependencies on their own ------------------

namespace taskdetail {

// An access of one phase to one resource class (level, kind: 0/1 buffer,
// 2 flags): who in the phase touches a given tile of it.
enum Pattern { OWN, STENCIL, FOOT, CHILD4, OWNRING };
struct Access {
    int phase;
    bool write;
    Pattern pat;
};

struct FastCtx {
    const std::vector<TaskLevel>* lev;
    std::vector<Phase> ph;
    std::vector<std::vector<int>> act_idx, ring_idx;  // per level: tile -> index or -1
    // per level l: the reconstructing tiles of level l + 1 (their indices in
    // its active list) whose footprint holds tile c of level l, as
    // foot_idx[l][foot_off[l][c] .. foot_off[l][c + 1])
    std::vector<std::vector<int>> foot_off, foot_idx;
    // per level and tile: bit 0 = some sweep pushes into it, bit 1 = a close
    // writes it (ring tile).  A read of a tile no phase ever writes has no
    // dependency, and its backward scan is skipped.
    std::vector<std::vector<uint8_t>> wmask;
    std::vector<Access> acc[TASK_MAX_LEVELS][3];      // per (level, kind), in phase order
    std::vector<int> acc_pos[TASK_MAX_LEVELS][3];     // per (level, kind): phase -> first entry at or after it

    // tasks of access a that touch tile (tx, ty) of its resource
    template <class F>
    void touching(const Access& a, int l, int tx, int ty, F&& emit) const {
        const std::vector<TaskLevel>& L = *lev;
        const Phase& P = ph[a.phase];
        switch (a.pat) {
            case OWN: {  // a sweep of level l reads its own tile
                const int i = act_idx[l][(size_t)ty * L[l].bx + tx];
                if (i >= 0) emit(P.offset + i);
                break;
            }
            case STENCIL: {  // sweeps of level l whose pushes land in the tile
                const TaskLevel& V = L[l];
                for (int d = 0; d < 5; d++) {
                    bool ok = true;
                    const int sx = wrap(tx - SDI[d], V.bx, V.px, ok);
                    const int sy = wrap(ty - SDJ[d], V.by, V.py, ok);
                    if (!ok) continue;
                    bool ok2 = true;  // the push from (sx, sy) in direction d must land here
                    const int rx = wrap(sx + SDI[d], V.bx, V.px, ok2), ry = wrap(sy + SDJ[d], V.by, V.py, ok2);
                    if (!ok2 || rx != tx || ry != ty) continue;
                    const int i = act_idx[l][(size_t)sy * V.bx + sx];
                    if (i >= 0) emit(P.offset + i);
                }
                break;
            }
            case FOOT: {  // reconstructing sweeps of level l + 1 over parent tile (tx, ty)
                const size_t c = (size_t)ty * L[l].bx + tx;
                for (int k = foot_off[l][c]; k < foot_off[l][c + 1]; k++) emit(P.offset + foot_idx[l][k]);
                break;
            }
            case CHILD4: {  // the close of level l - 1 over child tile (tx, ty)
                const int i = ring_idx[l - 1][(size_t)(ty / 2) * L[l - 1].bx + tx / 2];
                if (i >= 0) emit(P.offset + i);
                break;
            }
            case OWNRING: {  // the close of level l writes its own tile
                const int i = ring_idx[l][(size_t)ty * L[l].bx + tx];
                if (i >= 0) emit(P.offset + i);
                break;
            }
        }
    }

    // dependencies of an access of phase p to tile (tx, ty) of (l, kind)
    template <class F>
    void deps_of(int p, bool write, int l, int kind, int tx, int ty, F&& emit) const {
        if (!write) {
            const uint8_t m = wmask[l][(size_t)ty * (*lev)[l].bx + tx];
            if (kind == 2 ? !(m & 2) : !m) return;
        }
        const std::vector<Access>& A = acc[l][kind];
        bool readers = false;
        for (int e = acc_pos[l][kind][p] - 1; e >= 0; e--) {
            const Access& a = A[e];
            if (a.write) {
                // the last phase that wrote the tile.  A write that waits for
                // a reader since then needs no edge to these writers: every
                // such reader already waits for all of them.
                bool any = false;
                touching(a, l, tx, ty, [&](int q) {
                    any = true;
                    if (!readers) emit(q);
                });
                if (any) return;
            } else if (write) {
                touching(a, l, tx, ty, [&](int q) {  // readers since that phase
                    readers = true;
                    emit(q);
                });
            }
        }
    }
};

}  // namespace taskdetail

// Host threads the builder may use: the CPUs this process may actually use
// -- the smaller of the visible cores and a cgroup CPU quota (cgroup v2
// cpu.max or v1 cfs quota), at most 8.  The library itself builds on one
// thread (build_tasks' default): on hosts where threads are expensive (a
// sandboxed container measured 42 ms on one thread and 165 ms on two for
// the same list) more threads only cost; callers that know better pass a
// count.
inline int builder_threads() {
    static int cached = 0;
    if (cached) return cached;
    int n = (int)std::thread::hardware_concurrency();
    if (n <= 0) n = 1;
    double quota = -1.0;
    if (FILE* f = std::fopen("/sys/fs/cgroup/cpu.max", "r")) {
        char q[32] = {0};
        double period = 0.0;
        if (std::fscanf(f, "%31s %lf", q, &period) == 2 && q[0] != 'm' && period > 0) quota = std::atof(q) / period;
        std::fclose(f);
    } else if (FILE* f1 = std::fopen("/sys/fs/cgroup/cpu/cpu.cfs_quota_us", "r")) {
        double qv = -1.0, period = 0.0;
        if (std::fscanf(f1, "%lf", &qv) != 1) qv = -1.0;
        std::fclose(f1);
        if (FILE* f2 = std::fopen("/sys/fs/cgroup/cpu/cpu.cfs_period_us", "r")) {
            if (std::fscanf(f2, "%lf", &period) == 1 && qv > 0 && period > 0) quota = qv / period;
            std::fclose(f2);
        }
    }
    if (quota > 0) n = std::min(n, std::max(1, (int)quota));
    cached = std::max(1, std::min(n, 8));
    return cached;
}

inline void build_tasks(const std::vector<TaskLevel>& lev, int nsteps, TaskLists& out, int threads = 1) {
    using namespace taskdetail;
    const int nlev = (int)lev.size();
    FastCtx X;
    X.lev = &lev;
    phases(nlev, nsteps, lev, X.ph);
    X.act_idx.resize(nlev);
    X.ring_idx.resize(nlev);
    for (int l = 0; l < nlev; l++) {
        X.act_idx[l].assign((size_t)lev[l].bx * lev[l].by, -1);
        X.ring_idx[l].assign((size_t)lev[l].bx * lev[l].by, -1);
        for (size_t i = 0; i < lev[l].act->size(); i++) {
            const Item& it = (*lev[l].act)[i];
            X.act_idx[l][(size_t)it.ty * lev[l].bx + it.tx] = (int)i;
        }
        for (size_t i = 0; i < lev[l].ring->size(); i++) {
            const Item& it = (*lev[l].ring)[i];
            X.ring_idx[l][(size_t)it.ty * lev[l].bx + it.tx] = (int)i;
        }
    }
    X.wmask.assign(nlev, {});
    for (int l = 0; l < nlev; l++) {
        const TaskLevel& V = lev[l];
        X.wmask[l].assign((size_t)V.bx * V.by, 0);
        for (const Item& it : *V.act)
            for (int d = 0; d < 5; d++) {
                bool ok = true;
                const int tx = wrap(it.tx + SDI[d], V.bx, V.px, ok), ty = wrap(it.ty + SDJ[d], V.by, V.py, ok);
                if (ok) X.wmask[l][(size_t)ty * V.bx + tx] |= 1;
            }
        if (l + 1 < nlev)
            for (const Item& it : *V.ring) X.wmask[l][(size_t)it.ty * V.bx + it.tx] |= 2;
    }
    // reverse footprints
    X.foot_off.assign(nlev, {});
    X.foot_idx.assign(nlev, {});
    for (int l = 0; l + 1 < nlev; l++) {
        const TaskLevel& Pl = lev[l];
        const TaskLevel& C = lev[l + 1];
        std::vector<int>& off = X.foot_off[l];
        std::vector<int>& idx = X.foot_idx[l];
        off.assign((size_t)Pl.bx * Pl.by + 1, 0);
        std::vector<std::pair<int, int>> pairs;  // (parent tile, child active index)
        int keys[16];
        for (size_t i = 0; i < C.act->size(); i++) {
            const Item& it = (*C.act)[i];
            if (!(*C.recon)[(size_t)it.ty * C.bx + it.tx]) continue;
            const int nk = footprint(Pl, it.tx, it.ty, keys);
            for (int q = 0; q < nk; q++) pairs.emplace_back(keys[q], (int)i);
        }
        for (const auto& pr : pairs) off[pr.first + 1]++;
        for (size_t c = 0; c + 1 < off.size(); c++) off[c + 1] += off[c];
        idx.assign(pairs.size(), 0);
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (const auto& pr : pairs) idx[fill[pr.first]++] = pr.second;
    }
    // the accesses of every non-empty phase, per resource class
    const int np = (int)X.ph.size();
    for (int p = 0; p < np; p++) {
        const Phase& P = X.ph[p];
        if (!P.count) continue;
        const int l = P.l;
        if (P.kind == 0) {
            const int bs = src_of(l, P.kk, P.step);
            X.acc[l][bs].push_back({p, false, OWN});
            X.acc[l][bs ^ 1].push_back({p, true, STENCIL});
            if (l > 0) {
                const int pbs = src_of(l - 1, P.kkp, P.step);
                X.acc[l - 1][pbs].push_back({p, false, FOOT});
                X.acc[l - 1][pbs ^ 1].push_back({p, false, FOOT});
                X.acc[l - 1][2].push_back({p, false, FOOT});
            }
        } else {
            const int bd = src_of(l, P.kk, P.step) ^ 1;
            X.acc[l + 1][0].push_back({p, false, CHILD4});
            X.acc[l + 1][1].push_back({p, false, CHILD4});
            X.acc[l][bd].push_back({p, true, OWNRING});
            X.acc[l][2].push_back({p, true, OWNRING});
        }
    }
    for (int l = 0; l < nlev; l++)
        for (int k = 0; k < 3; k++) {
            std::vector<int>& pos = X.acc_pos[l][k];
            pos.assign(np + 1, 0);
            int e = 0;
            for (int p = 0; p <= np; p++) {
                while (e < (int)X.acc[l][k].size() && X.acc[l][k][e].phase < p) e++;
                pos[p] = e;
            }
        }
    const int ntask = X.ph.empty() ? 0 : X.ph.back().offset + X.ph.back().count;
    out.t.assign(ntask, Task{});
    // task -> phase
    std::vector<int> tph(ntask);
    for (int p = 0; p < np; p++)
        for (int i = 0; i < X.ph[p].count; i++) tph[X.ph[p].offset + i] = p;
    int nth = threads > 0 ? threads : builder_threads();
    nth = std::max(1, std::min(nth, std::max(1, ntask / 2048)));
    std::vector<std::vector<int>> dpart(nth);
    auto work = [&](int w) {
        const int a = (int)((long long)ntask * w / nth), b = (int)((long long)ntask * (w + 1) / nth);
        std::vector<int>& D = dpart[w];
        std::vector<int> cur;
        for (int t = a; t < b; t++) {
            const int p = tph[t];
            const Phase& P = X.ph[p];
            const int l = P.l;
            const TaskLevel& L = lev[l];
            const Item& it = P.kind == 0 ? (*L.act)[t - P.offset] : (*L.ring)[t - P.offset];
            cur.clear();
            auto emit = [&](int q) { cur.push_back(q); };
            if (P.kind == 0) {
                const int bs = src_of(l, P.kk, P.step), bd = bs ^ 1;
                X.deps_of(p, false, l, bs, it.tx, it.ty, emit);
                for (int d = 0; d < 5; d++) {
                    bool ok = true;
                    const int tx = wrap(it.tx + SDI[d], L.bx, L.px, ok);
                    const int ty = wrap(it.ty + SDJ[d], L.by, L.py, ok);
                    if (ok) X.deps_of(p, true, l, bd, tx, ty, emit);
                }
                if (l > 0 && (*L.recon)[(size_t)it.ty * L.bx + it.tx]) {
                    const TaskLevel& Pl = lev[l - 1];
                    const int pbs = src_of(l - 1, P.kkp, P.step), pbd = pbs ^ 1;
                    int keys[16];
                    const int nk = footprint(Pl, it.tx, it.ty, keys);
                    for (int q = 0; q < nk; q++) {
                        const int cx = keys[q] % Pl.bx, cy = keys[q] / Pl.bx;
                        X.deps_of(p, false, l - 1, pbs, cx, cy, emit);
                        X.deps_of(p, false, l - 1, pbd, cx, cy, emit);
                        X.deps_of(p, false, l - 1, 2, cx, cy, emit);
                    }
                }
            } else {
                const int bd = src_of(l, P.kk, P.step) ^ 1;
                const TaskLevel& C = lev[l + 1];
                for (int b2 = 0; b2 < 2; b2++)
                    for (int a2 = 0; a2 < 2; a2++) {
                        const int fx = 2 * it.tx + a2, fy = 2 * it.ty + b2;
                        if (fx >= C.bx || fy >= C.by) continue;
                        X.deps_of(p, false, l + 1, 0, fx, fy, emit);
                        X.deps_of(p, false, l + 1, 1, fx, fy, emit);
                    }
                X.deps_of(p, true, l, bd, it.tx, it.ty, emit);
                X.deps_of(p, true, l, 2, it.tx, it.ty, emit);
            }
            std::sort(cur.begin(), cur.end());
            cur.erase(std::unique(cur.begin(), cur.end()), cur.end());
            Task T = make_task(P, it);
            T.dep0 = (int)D.size();  // local; rebased below
            T.ndep = (int)cur.size();
            D.insert(D.end(), cur.begin(), cur.end());
            out.t[t] = T;
        }
    };
    if (nth == 1) {
        work(0);
    } else {
        std::vector<std::thread> pool;
        for (int w = 0; w < nth; w++) pool.emplace_back(work, w);
        for (auto& th : pool) th.join();
    }
    size_t total = 0;
    for (int w = 0; w < nth; w++) total += dpart[w].size();
    out.d.clear();
    out.d.reserve(total);
    for (int w = 0; w < nth; w++) {
        const int a = (int)((long long)ntask * w / nth), b = (int)((long long)ntask * (w + 1) / nth);
        const int base = (int)out.d.size();
        for (int t = a; t < b; t++) out.t[t].dep0 += base;
        out.d.insert(out.d.end(), dpart[w].begin(), dpart[w].end());
    }
}

// Exact per-step conservation audit (Sec. 4.1.2, 4.1.3, 4.2) on a built task list.
// With block_slots > 0: every first sweep of a tile in a step (aslot == -2)
// gets an audit slot, numbered step by step in list order; scale[j] is the
// weight exponent of slot j (4^-level: -2 level); the slots of each step are
// cut into reduction blocks rng[b] = [first, last) of at most block_slots
// slots, never across steps, and bseg[st] .. bseg[st + 1] are the blocks of
// step st.  Each block gets four reduction tasks (kind 2, one per field kk,
// aslot = the block), each depending on the sweeps that write the block's
// slots and inserted `lag` tasks after the last of them (at the end of the
// list at the latest): tasks are claimed in list order by every resident
// thread group at once, so with a lag of about twice the number of resident
// groups the writers are complete when a reduction is claimed and its group
// does not wait; the reductions run between later sweeps.  The other tasks
// keep their order and their (remapped) dependencies, which all point to
// earlier tasks.  With block_slots == 0 nothing is audited (aslot = -1
// everywhere).  Returns the number of slots.
inline int assign_audit(std::vector<Task>& t, std::vector<int>& d, int nsteps, int block_slots,
                        std::vector<int>& scale, std::vector<int2>& rng, std::vector<int>& bseg, int lag = 0) {
    scale.clear();
    rng.clear();
    bseg.assign(1, 0);
    if (block_slots <= 0) {
        for (Task& T : t)
            if (T.kind == 0) T.aslot = -1;
        return 0;
    }
    std::vector<int> seg(nsteps + 1, 0);
    for (const Task& T : t)
        if (T.kind == 0 && T.aslot == -2) seg[T.step + 1]++;
    for (int i = 0; i < nsteps; i++) seg[i + 1] += seg[i];
    const int nslots = seg.back();
    std::vector<int> fill(nsteps, 0), writer(nslots, -1);
    scale.assign(std::max(1, nslots), 0);
    const int n = (int)t.size();
    for (int i = 0; i < n; i++) {
        Task& T = t[i];
        if (T.kind != 0) continue;
        T.aslot = T.aslot == -2 ? seg[T.step] + fill[T.step]++ : -1;
        if (T.aslot >= 0) {
            scale[T.aslot] = -2 * T.lid;
            writer[T.aslot] = i;
        }
    }
    for (int st = 0; st < nsteps; st++) {
        for (int j = seg[st]; j < seg[st + 1]; j += block_slots) {
            int2 r;
            r.x = j;
            r.y = std::min(j + block_slots, seg[st + 1]);
            rng.push_back(r);
        }
        bseg.push_back((int)rng.size());
    }
    std::vector<int> blk_step(rng.size(), 0);
    for (int st = 0; st < nsteps; st++)
        for (int b = bseg[st]; b < bseg[st + 1]; b++) blk_step[b] = st;
    // the blocks whose last writer is task i
    std::vector<std::vector<int>> after(n);
    for (int b = 0; b < (int)rng.size(); b++) {
        int last = -1;
        for (int j = rng[b].x; j < rng[b].y; j++) last = std::max(last, writer[j]);
        after[std::min(n - 1, last + std::max(0, lag))].push_back(b);
    }
    std::vector<Task> nt;
    std::vector<int> nd, remap(n);
    nt.reserve(n + 4 * rng.size());
    nd.reserve(d.size() + 4 * (size_t)nslots);
    for (int i = 0; i < n; i++) {
        Task T = t[i];
        const int d0 = (int)nd.size();
        for (int j = 0; j < T.ndep; j++) nd.push_back(remap[d[T.dep0 + j]]);  // earlier tasks: remapped already
        T.dep0 = d0;
        remap[i] = (int)nt.size();
        nt.push_back(T);
        for (int b : after[i])
            for (int k = 0; k < 4; k++) {
                Task A{};
                A.lid = T.lid;
                A.kind = 2;
                A.kk = (signed char)k;
                A.step = (signed char)blk_step[b];
                A.dep0 = (int)nd.size();
                A.ndep = rng[b].y - rng[b].x;
                A.aslot = b;
                for (int j = rng[b].x; j < rng[b].y; j++) nd.push_back(remap[writer[j]]);
                nt.push_back(A);
            }
    }
    t.swap(nt);
    d.swap(nd);
    return nslots;
}

}  // namespace vlbm
