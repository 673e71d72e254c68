// Host-only check of the persistent schedule's task builder: on seeded
// random layouts (1-4 levels, ragged sizes, periodic or not in each
// direction, 1-3 coarse steps) the fast builder and the reference replay
// must produce the same tasks, the fast builder's edges must be reference
// edges pointing backwards, and both lists must order the tasks the same
// way (equal transitive closures); the fast builder must give the same
// lists on 1 and 4 threads, and the audit's slots, blocks and reduction
// tasks must be placed as assign_audit states.  With --time it reports the build time of both
// on a large three-level layout.
//
//   task_builder_check [--layouts N] [--seed S] [--time [--threads T]]
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "vlbm_tasks.h"

using namespace vlbm;

struct Layout {
    int nlev, nx0, ny0;
    bool px, py;
    std::vector<std::vector<uint8_t>> bin, bcov;
    std::vector<TileLists> tl;
    std::vector<TaskLevel> lev;
};

static int ceil8(int n) { return (n + TILE - 1) / TILE; }

// covered blocks: a few random rectangles of in-blocks per level; the next
// level holds the children of the covered blocks
static void make_layout(Layout& L, std::mt19937_64& rng, int nlev, int nx0, int ny0, bool px, bool py, int rects) {
    L.nlev = nlev;
    L.nx0 = nx0;
    L.ny0 = ny0;
    L.px = px;
    L.py = py;
    L.bin.assign(nlev, {});
    L.bcov.assign(nlev, {});
    for (int l = 0; l < nlev; l++) {
        const int bx = ceil8(nx0 << l), by = ceil8(ny0 << l);
        L.bin[l].assign((size_t)bx * by, l == 0 ? 1 : 0);
        L.bcov[l].assign((size_t)bx * by, 0);
        if (l > 0) {
            const int pbx = ceil8(nx0 << (l - 1)), pby = ceil8(ny0 << (l - 1));
            for (int j = 0; j < pby; j++)
                for (int i = 0; i < pbx; i++)
                    if (L.bcov[l - 1][(size_t)j * pbx + i])
                        for (int b = 0; b < 2; b++)
                            for (int a = 0; a < 2; a++) {
                                const int ci = 2 * i + a, cj = 2 * j + b;
                                if (ci < bx && cj < by) L.bin[l][(size_t)cj * bx + ci] = 1;
                            }
        }
        if (l + 1 < nlev)
            for (int r = 0; r < rects; r++) {
                const int w = 1 + (int)(rng() % std::max(1, bx / 2)), h = 1 + (int)(rng() % std::max(1, by / 2));
                const int i0 = (int)(rng() % bx), j0 = (int)(rng() % by);
                for (int j = j0; j < j0 + h; j++)
                    for (int i = i0; i < i0 + w; i++) {
                        int ii = i, jj = j;
                        if (ii >= bx) {
                            if (!px) continue;
                            ii -= bx;
                        }
                        if (jj >= by) {
                            if (!py) continue;
                            jj -= by;
                        }
                        const size_t b = (size_t)jj * bx + ii;
                        if (L.bin[l][b]) L.bcov[l][b] = 1;
                    }
            }
    }
    L.tl.assign(nlev, {});
    L.lev.assign(nlev, {});
    for (int l = 0; l < nlev; l++) {
        const int nx = nx0 << l, ny = ny0 << l, bx = ceil8(nx), by = ceil8(ny);
        tile_lists(l, nx, ny, bx, by, px, py, L.bin[l].data(), L.bcov[l].data(), L.tl[l]);
        TaskLevel& t = L.lev[l];
        t.nx = nx;
        t.ny = ny;
        t.bx = bx;
        t.by = by;
        t.px = px;
        t.py = py;
        t.act = &L.tl[l].act;
        t.ring = &L.tl[l].ring;
        t.recon = &L.tl[l].recon;
    }
}

static bool same(const TaskLists& a, const TaskLists& b, char* why) {
    if (a.t.size() != b.t.size()) {
        sprintf(why, "task count %zu vs %zu", a.t.size(), b.t.size());
        return false;
    }
    for (size_t i = 0; i < a.t.size(); i++) {
        const Task &x = a.t[i], &y = b.t[i];
        if (x.lid != y.lid || x.tx != y.tx || x.ty != y.ty || x.kind != y.kind || x.kk != y.kk || x.kkp != y.kkp ||
            x.step != y.step || x.aslot != y.aslot || x.ndep != y.ndep) {
            sprintf(why, "task %zu differs (ndep %d vs %d, kind %d lid %d tile %d,%d)", i, x.ndep, y.ndep, x.kind,
                    x.lid, x.tx, x.ty);
            return false;
        }
        for (int k = 0; k < x.ndep; k++)
            if (a.d[x.dep0 + k] != b.d[y.dep0 + k]) {
                sprintf(why, "task %zu dependency %d differs (%d vs %d)", i, k, a.d[x.dep0 + k], b.d[y.dep0 + k]);
                return false;
            }
    }
    return true;
}

// Same tasks, fast edges a subset of the reference edges, and the same
// transitive closure (checked on lists of at most `cap` tasks).
static bool same_order(const TaskLists& ref, const TaskLists& f, char* why, size_t cap = 6000) {
    if (ref.t.size() != f.t.size()) {
        sprintf(why, "task count %zu vs %zu", ref.t.size(), f.t.size());
        return false;
    }
    const size_t n = ref.t.size();
    for (size_t i = 0; i < n; i++) {
        const Task &x = ref.t[i], &y = f.t[i];
        if (x.lid != y.lid || x.tx != y.tx || x.ty != y.ty || x.kind != y.kind || x.kk != y.kk || x.kkp != y.kkp ||
            x.step != y.step || x.aslot != y.aslot) {
            sprintf(why, "task %zu differs", i);
            return false;
        }
        for (int k = 0; k < y.ndep; k++) {
            const int q = f.d[y.dep0 + k];
            if (!std::binary_search(ref.d.begin() + x.dep0, ref.d.begin() + x.dep0 + x.ndep, q)) {
                sprintf(why, "task %zu: edge to %d not in the reference", i, q);
                return false;
            }
            if (q >= (int)i) {
                sprintf(why, "task %zu: edge to a later task %d", i, q);
                return false;
            }
        }
    }
    if (n > cap) return true;
    const size_t W = (n + 63) / 64;
    std::vector<uint64_t> A(n * W, 0), B(n * W, 0);
    auto closure = [&](const TaskLists& L, std::vector<uint64_t>& C) {
        for (size_t i = 0; i < n; i++)
            for (int k = 0; k < L.t[i].ndep; k++) {
                const int q = L.d[L.t[i].dep0 + k];
                C[i * W + q / 64] |= 1ull << (q % 64);
                for (size_t w = 0; w < W; w++) C[i * W + w] |= C[q * W + w];
            }
    };
    closure(ref, A);
    closure(f, B);
    for (size_t i = 0; i < n; i++)
        for (size_t w = 0; w < W; w++)
            if (A[i * W + w] != B[i * W + w]) {
                sprintf(why, "task %zu: ancestors differ", i);
                return false;
            }
    return true;
}

// assign_audit on a copy of list `a`: the sweeps and closes keep their
// order, fields and (remapped) dependencies; every first sweep of a step
// owns one slot of its step, with weight exponent -2 level; the blocks tile
// each step's slots in at most `bs` slots; every block has exactly one
// reduction task per field, after all of the block's writers, depending on
// exactly those writers; every edge points backwards.
static bool audit_ok(const TaskLists& a, int nsteps, int bs, int lag, char* why) {
    std::vector<Task> t = a.t;
    std::vector<int> d = a.d, scale, bseg;
    std::vector<int2> rng;
    const int nslots = assign_audit(t, d, nsteps, bs, scale, rng, bseg, lag);
    std::vector<int> first(nsteps, 0);
    for (const Task& T : a.t)
        if (T.kind == 0 && T.aslot == -2) first[T.step]++;
    int expect = 0;
    for (int v : first) expect += v;
    if (nslots != expect) return sprintf(why, "audit: %d slots, %d first sweeps", nslots, expect), false;
    if ((int)bseg.size() != nsteps + 1 || bseg.back() != (int)rng.size())
        return sprintf(why, "audit: step segmentation of the blocks"), false;
    std::vector<int> pos(a.t.size(), -1), writer(nslots, -1), slot_step(nslots, -1);
    std::vector<std::vector<int>> red(rng.size());
    std::vector<int> red_k(rng.size(), -1), writer_k(nslots, -1);  // original tasks before it
    size_t k = 0;
    for (size_t i = 0; i < t.size(); i++) {
        const Task& T = t[i];
        for (int j = 0; j < T.ndep; j++)
            if (d[T.dep0 + j] >= (int)i) return sprintf(why, "audit: task %zu has a forward edge", i), false;
        if (T.kind == 2) {
            if (T.aslot < 0 || T.aslot >= (int)rng.size()) return sprintf(why, "audit: block index"), false;
            red[T.aslot].push_back((int)i);
            if (red_k[T.aslot] >= 0 && red_k[T.aslot] != (int)k)
                return sprintf(why, "audit: tasks of block %d apart", T.aslot), false;
            red_k[T.aslot] = (int)k;
            continue;
        }
        if (k >= a.t.size()) return sprintf(why, "audit: extra task"), false;
        const Task& O = a.t[k];
        if (O.lid != T.lid || O.tx != T.tx || O.ty != T.ty || O.kind != T.kind || O.kk != T.kk || O.kkp != T.kkp ||
            O.step != T.step || O.ndep != T.ndep)
            return sprintf(why, "audit: task %zu changed", k), false;
        for (int j = 0; j < T.ndep; j++)
            if (d[T.dep0 + j] != pos[a.d[O.dep0 + j]]) return sprintf(why, "audit: task %zu edge changed", k), false;
        const bool owns = O.kind == 0 && O.aslot == -2;
        if (owns != (T.aslot >= 0)) return sprintf(why, "audit: slot owner %zu", k), false;
        if (T.aslot >= 0) {
            if (T.aslot >= nslots || writer[T.aslot] >= 0) return sprintf(why, "audit: slot %d", T.aslot), false;
            writer[T.aslot] = (int)i;
            writer_k[T.aslot] = (int)k;
            slot_step[T.aslot] = T.step;
            if (scale[T.aslot] != -2 * T.lid) return sprintf(why, "audit: weight of slot %d", T.aslot), false;
        }
        pos[k++] = (int)i;
    }
    if (k != a.t.size()) return sprintf(why, "audit: lost tasks"), false;
    int next = 0;
    for (int st = 0; st < nsteps; st++)
        for (int b = bseg[st]; b < bseg[st + 1]; b++) {
            const int2 r = rng[b];
            if (r.x != next || r.y <= r.x || r.y - r.x > bs) return sprintf(why, "audit: block %d range", b), false;
            next = r.y;
            for (int j = r.x; j < r.y; j++)
                if (slot_step[j] != st) return sprintf(why, "audit: block %d crosses steps", b), false;
            if (red[b].size() != 4) return sprintf(why, "audit: block %d has %zu tasks", b, red[b].size()), false;
            int last = -1;
            for (int j = r.x; j < r.y; j++) last = std::max(last, writer_k[j]);
            if (red_k[b] != std::min((int)a.t.size() - 1, last + lag) + 1)
                return sprintf(why, "audit: block %d placed after %d original tasks, not %d + lag %d", b, red_k[b],
                               last, lag), false;
            for (int q = 0; q < 4; q++) {
                const Task& A = t[red[b][q]];
                if (A.kk != q || A.step != st || A.ndep != r.y - r.x) return sprintf(why, "audit: task of block %d", b), false;
                for (int j = 0; j < A.ndep; j++)
                    if (d[A.dep0 + j] != writer[r.x + j]) return sprintf(why, "audit: block %d edge", b), false;
            }
        }
    if (next != nslots) return sprintf(why, "audit: blocks cover %d of %d slots", next, nslots), false;
    return true;
}

static double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int main(int argc, char** argv) {
    int layouts = 300;
    unsigned long long seed = 7;
    bool timing = false;
    int threads = 0;  // builder threads in the timing run (0: the builder's own choice)
    for (int i = 1; i < argc; i++) {
        if (!strcmp(argv[i], "--layouts") && i + 1 < argc) layouts = atoi(argv[++i]);
        else if (!strcmp(argv[i], "--seed") && i + 1 < argc) seed = strtoull(argv[++i], nullptr, 10);
        else if (!strcmp(argv[i], "--time")) timing = true;
        else if (!strcmp(argv[i], "--threads") && i + 1 < argc) threads = atoi(argv[++i]);
    }
    std::mt19937_64 rng(seed);
    long long ntasks = 0, ndeps = 0, nfast = 0;
    for (int n = 0; n < layouts; n++) {
        Layout L;
        const int nlev = 1 + (int)(rng() % 4);
        const int nx0 = 8 + (int)(rng() % 57), ny0 = 8 + (int)(rng() % 57);  // ragged sizes included
        const bool px = rng() & 1, py = rng() & 1;
        make_layout(L, rng, nlev, nx0, ny0, px, py, 1 + (int)(rng() % 4));
        const int nsteps = 1 + (int)(rng() % 3);
        TaskLists ref, fast1, fast4;
        build_tasks_tracked(L.lev, nsteps, ref);
        build_tasks(L.lev, nsteps, fast1, 1);
        build_tasks(L.lev, nsteps, fast4, 4);
        char why[256];
        const int bs = 1 + (int)(rng() % 40);
        if (!same_order(ref, fast1, why) || !same(fast1, fast4, why) || !audit_ok(fast1, nsteps, bs, (int)(rng() % 3) * (int)(rng() % 200), why)) {
            printf("MISMATCH layout %d (nlev %d, %dx%d, periodic %d%d, steps %d): %s\n", n, nlev, nx0, ny0, px, py,
                   nsteps, why);
            return 1;
        }
        ntasks += (long long)ref.t.size();
        ndeps += (long long)ref.d.size();
        nfast += (long long)fast1.d.size();
    }
    printf("OK %d layouts, %lld tasks, %lld reference edges, %lld fast edges\n", layouts, ntasks, ndeps, nfast);
    if (timing) {
        // a 2048 x 1024 coarse grid with two finer levels over bands
        Layout L;
        std::mt19937_64 r2(11);
        make_layout(L, r2, 3, 2048, 1024, false, true, 6);
        for (int nsteps : {1, 8}) {
            TaskLists a, b;
            auto t0 = std::chrono::steady_clock::now();
            build_tasks_tracked(L.lev, nsteps, a);
            const double ta = ms_since(t0);
            t0 = std::chrono::steady_clock::now();
            build_tasks(L.lev, nsteps, b, 1);
            const double tb = ms_since(t0);
            t0 = std::chrono::steady_clock::now();
            build_tasks(L.lev, nsteps, b, threads);
            const double tc = ms_since(t0);
            char why[256];
            const bool ok = same_order(a, b, why);
            printf("TIME steps %d tasks %zu edges %zu/%zu tracked_ms %.1f fast1_ms %.1f fastN_ms %.1f threads %d %s\n",
                   nsteps, a.t.size(), a.d.size(), b.d.size(), ta, tb, tc,
                   threads > 0 ? threads : builder_threads(), ok ? "same order" : why);
            if (!ok) return 1;
        }
    }
    return 0;
}
