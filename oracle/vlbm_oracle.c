/*
 * ORACLE -- test infrastructure, not product code.
 *
 * A plain, slow, FP64 CPU rendering of the conservative locally refined
 * vectorial lattice Boltzmann method (VLBM) of Hosseini, Strassle & Karlin,
 * "Conservative local grid refinement for the vectorial lattice Boltzmann
 * method".  Only tests/, __graft_entry__.smoke() and the cpu_baseline leg of
 * bench.py may load or run it.  It shares no code with the CUDA path.
 *
 * Layout: every level l owns dense arrays over its whole index space
 * (nx0*r^l by ny0*r^l cells).  Per cell:  in_l  (the cell belongs to level l)
 * and ref_l (the cell is covered by level l+1).  A cell is ACTIVE on level l
 * when in_l && !ref_l.  Populations are f[q*n + cell] with q = 4*i + k,
 * direction i in {+x,-x,+y,-y}, field k in {rho, rho*u, rho*v, rho*E}.
 * The state at sync times is the pre-collision f of every active cell.
 *
 * One coarse step is step(0, 1).  step(l, k) follows the five-step cycle of
 * Sec. 3.2 (Fig. 1), applied per edge in 2-D as in Sec. 3.3:
 *   1. BGK collision of every active cell of level l       (Sec. 2.2, Eq. 6)
 *   2. fine side (l >= 1): the post-collision population leaving towards
 *      coarser territory is kept in the reflux register of its face, indexed
 *      by this sub-step k and the cell's tangential index j  (Eq. 24)
 *   3. coarse side (l has a finer level): every interface face captures
 *      cur = f*_d(L0), and the tangential minmod slope sigma      (Eq. 22)
 *   4. exact shift streaming on level l                    (Sec. 2.2, Eq. 5)
 *      - upwind cell active on l        : ordinary pull
 *      - upwind cell covered by l+1     : left pending (filled in 6.)
 *      - upwind cell in coarser land    : mean-preserving reconstruction
 *                                         (Eq. 23, with Eq. 20 in time)
 *      - upwind cell outside the domain : boundary condition
 *   5. r sub-steps step(l+1, 1..r)                       (Sec. 3.2, Eq. 15)
 *   6. reflux: the pending population of every coarse ring cell is the
 *      plain average of its r*r register values (Eq. 24); prev <- cur.
 *
 * Canonical arithmetic.  Expressions are evaluated exactly as written here,
 * with fma() only where it is spelled out and no other contraction (build
 * with -ffp-contract=off).  The CUDA path evaluates the same expressions in
 * the same order, so both produce the same bits.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *  - the r register values averaged in Eq. 24 are the post-collision values
 *    of the r fine sub-steps executed inside the coarse cycle;
 *  - the reconstructed value with index k is the one streamed into R0 at the
 *    end of fine sub-step k;
 *  - a face seen for the first time has no previous sample: prev := cur;
 *  - sigma uses L0-1 and L0+1 only when both are active cells of the same
 *    level (else sigma = 0);  j grows with the tangential coordinate;
 *  - split slopes use active values, or the average of the children for a
 *    neighbour that stays covered; at a non-periodic edge the slope is 0;
 *  - boundaries: periodic, zero-gradient outflow, fixed-state inflow
 *    (ghost in equilibrium at W_b) and reflective walls.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_MAXLEV 6
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW = 2, BC_REFLECT = 3 };

static const int CX[4] = {1, -1, 0, 0};
static const int CY[4] = {0, 0, 1, -1};
#define QI(i, k) ((i) * 4 + (k))

typedef struct {
    int nx, ny;
    size_t n;
    uint8_t *in, *ref;
    double *f, *fs;
    /* interface faces seen from this level (coarse side) */
    int32_t *fidx; /* [4][n] face id of (cell, d) or -1 */
    int nface;
    int32_t *fcell;
    int8_t *fdir;
    uint8_t *fresh;
    double *cur, *prev, *sig; /* [nface][4] */
    double *slot;             /* [nface][r][r][4] */
} OLevel;

typedef struct {
    int nlev, r, nx0, ny0;
    int bc[4]; /* sides W, E, S, N */
    double wb[4][4];
    double feqb[4][16];
    double gamma, c, beta;
    double om, hb, bcs, gm1, hc;
    /* sensor-driven relaxation (off unless ora_set_sensor) */
    int sensor;
    double beta_min, csens, eps, iq[4], ninth;
    OLevel lev[ORA_MAXLEV];
} OHier;

/* ------------------------------------------------------------------ */
/* Single-cell operators                                               */
/* ------------------------------------------------------------------ */

/* Target flux Q(W) of the 2-D Euler system with the ideal-gas closure
 * p = (gamma-1)(rho E - |rho u|^2 / (2 rho))  (Sec. 2.1, Eq. 1). */
static void euler_flux(double gm1, const double W[4], double Qx[4], double Qy[4]) {
    double inv = 1.0 / W[0];
    double u = W[1] * inv;
    double v = W[2] * inv;
    double ruu = W[1] * u;
    double rvv = W[2] * v;
    double p = gm1 * fma(-0.5, ruu + rvv, W[3]);
    double H = W[3] + p;
    Qx[0] = W[1];
    Qx[1] = ruu + p;
    Qx[2] = W[2] * u;
    Qx[3] = H * u;
    Qy[0] = W[2];
    Qy[1] = W[1] * v;
    Qy[2] = rvv + p;
    Qy[3] = H * v;
}

/* Zeroth moment W = sum_i f_i, summed as (f_+x + f_-x) + (f_+y + f_-y). */
static void moments(const double f[16], double W[4]) {
    for (int k = 0; k < 4; k++)
        W[k] = (f[QI(0, k)] + f[QI(1, k)]) + (f[QI(2, k)] + f[QI(3, k)]);
}

/* Vector equilibrium of Eq. 4 with D = 2:
 * f^eq_{+-alpha} = W/4 +- Q_alpha/(2c). */
void ora_feq(double gamma, double c, const double W[4], double feq[16]) {
    double Qx[4], Qy[4];
    euler_flux(gamma - 1.0, W, Qx, Qy);
    double hc = 0.5 / c;
    for (int k = 0; k < 4; k++) {
        double qw = 0.25 * W[k];
        feq[QI(0, k)] = fma(hc, Qx[k], qw);
        feq[QI(1, k)] = fma(-hc, Qx[k], qw);
        feq[QI(2, k)] = fma(hc, Qy[k], qw);
        feq[QI(3, k)] = fma(-hc, Qy[k], qw);
    }
}

/* BGK relaxation of Eq. 6: f* = 2 beta f^eq(W) + (1 - 2 beta) f with
 * W = sum_i f_i.  With 2 beta f^eq_{+-alpha} = (beta/2) W +- (beta/c) Q_alpha,
 * f* = fma(+-beta/c, Q_alpha, fma(1-2beta, f, (beta/2) W)). */
static void collide_with(double gm1, double om, double hb, double bcs, const double f[16], double fs[16]) {
    double W[4], Qx[4], Qy[4];
    moments(f, W);
    euler_flux(gm1, W, Qx, Qy);
    for (int k = 0; k < 4; k++) {
        double A = hb * W[k];
        fs[QI(0, k)] = fma(bcs, Qx[k], fma(om, f[QI(0, k)], A));
        fs[QI(1, k)] = fma(-bcs, Qx[k], fma(om, f[QI(1, k)], A));
        fs[QI(2, k)] = fma(bcs, Qy[k], fma(om, f[QI(2, k)], A));
        fs[QI(3, k)] = fma(-bcs, Qy[k], fma(om, f[QI(3, k)], A));
    }
}

static void collide_cell(const OHier* H, const double f[16], double fs[16]) {
    collide_with(H->gm1, H->om, H->hb, H->bcs, f, fs);
}

void ora_collide(double gamma, double c, double beta, const double f[16], double fs[16]) {
    OHier H;
    memset(&H, 0, sizeof H);
    H.gm1 = gamma - 1.0;
    H.om = 1.0 - 2.0 * beta;
    H.hb = 0.5 * beta;
    H.bcs = beta / c;
    collide_cell(&H, f, fs);
}

/* minmod(a, b) = sign(a) min(|a|, |b|) when a and b agree in sign, else 0
 * (Eqs. 22 and 26). */
double ora_minmod(double a, double b) {
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* Eq. 23: value handed to fine cell R_{0,j} at fine sub-step k (1..r):
 * a + (a - a_prev)(2k-r-1)/(2r) + sigma (2j-r+1)/(2r). */
double ora_recon(double a, double a_prev, double sigma, int r, int k, int j) {
    double wk = (double)(2 * k - r - 1) / (double)(2 * r);
    double wj = (double)(2 * j - r + 1) / (double)(2 * r);
    return fma(sigma, wj, fma(a - a_prev, wk, a));
}

/* Eq. 25 for r = 2: plain average of the four children, paired as
 * (c00 + c11) + (c10 + c01) so that the result is symmetric under x<->y;
 * other r: rows summed in x, then rows summed in y, times 1/r^2. */
static double merge_vals(const double* ch, int r) {
    if (r == 2) return ((ch[0] + ch[3]) + (ch[1] + ch[2])) * 0.25;
    double tot = 0.0;
    for (int b = 0; b < r; b++) {
        double row = ch[b * r];
        for (int a = 1; a < r; a++) row += ch[b * r + a];
        tot = (b == 0) ? row : tot + row;
    }
    return tot * (1.0 / (double)(r * r));
}

double ora_merge4(double c00, double c10, double c01, double c11) {
    double ch[4] = {c00, c10, c01, c11};
    return merge_vals(ch, 2);
}

/* Eqs. 26-27: child (a, b) of a split cell with value fc and minmod slopes
 * sx, sy:  fc + (sx xi_a + sy xi_b),  xi = (2a - r + 1)/(2r). */
double ora_split_child(double fc, double sx, double sy, int r, int a, int b) {
    double xa = (double)(2 * a - r + 1) / (double)(2 * r);
    double xb = (double)(2 * b - r + 1) / (double)(2 * r);
    return fc + (sx * xa + sy * xb);
}

/* ------------------------------------------------------------------ */
/* Hierarchy helpers                                                   */
/* ------------------------------------------------------------------ */

static inline size_t cidx(const OLevel* L, int x, int y) { return (size_t)y * (size_t)L->nx + (size_t)x; }

/* Resolves (x, y) on level l against the domain.  Returns 0 when the cell is
 * inside (coordinates wrapped across periodic sides) or 1 + side when it lies
 * beyond a non-periodic side (0 W, 1 E, 2 S, 3 N). */
static int resolve(const OHier* H, const OLevel* L, int* px, int* py) {
    int x = *px, y = *py;
    if (x < 0) {
        if (H->bc[0] != BC_PERIODIC) return 1;
        x += L->nx;
    } else if (x >= L->nx) {
        if (H->bc[1] != BC_PERIODIC) return 2;
        x -= L->nx;
    }
    if (y < 0) {
        if (H->bc[2] != BC_PERIODIC) return 3;
        y += L->ny;
    } else if (y >= L->ny) {
        if (H->bc[3] != BC_PERIODIC) return 4;
        y -= L->ny;
    }
    *px = x;
    *py = y;
    return 0;
}

static inline int is_active(const OLevel* L, size_t c) { return L->in[c] && !L->ref[c]; }

static void free_faces(OLevel* L) {
    free(L->fcell); free(L->fdir); free(L->fresh);
    free(L->cur); free(L->prev); free(L->sig); free(L->slot);
    L->fcell = NULL; L->fdir = NULL; L->fresh = NULL;
    L->cur = L->prev = L->sig = L->slot = NULL;
    L->nface = 0;
}

/* Builds the interface faces (L0 active on l, L0 + c_d covered on l).
 * Faces that already existed keep prev and their fresh flag; new faces are
 * fresh (no previous sample yet). */
static void build_faces(OHier* H, int l) {
    OLevel* L = &H->lev[l];
    int r = H->r;
    int32_t* oldidx = L->fidx;
    int oldn = L->nface;
    double* oldprev = L->prev;
    uint8_t* oldfresh = L->fresh;
    L->prev = NULL; L->fresh = NULL;
    double* oldcur = L->cur; L->cur = NULL;
    free(L->fcell); free(L->fdir); free(L->sig); free(L->slot);
    L->fcell = NULL; L->fdir = NULL; L->sig = NULL; L->slot = NULL;
    L->nface = 0;
    if (l >= H->nlev - 1) {
        free(oldidx); free(oldprev); free(oldfresh); free(oldcur);
        L->fidx = NULL;
        return;
    }
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * 4 * L->n);
    for (size_t t = 0; t < 4 * L->n; t++) idx[t] = -1;
    int cap = 0;
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c0 = cidx(L, x, y);
            if (!is_active(L, c0)) continue;
            for (int d = 0; d < 4; d++) {
                int xx = x + CX[d], yy = y + CY[d];
                if (resolve(H, L, &xx, &yy)) continue;
                size_t c1 = cidx(L, xx, yy);
                if (L->in[c1] && L->ref[c1]) cap++;
            }
        }
    L->fcell = (int32_t*)malloc(sizeof(int32_t) * (cap + 1));
    L->fdir = (int8_t*)malloc(cap + 1);
    L->fresh = (uint8_t*)malloc(cap + 1);
    L->cur = (double*)calloc((size_t)(cap + 1) * 4, sizeof(double));
    L->prev = (double*)calloc((size_t)(cap + 1) * 4, sizeof(double));
    L->sig = (double*)calloc((size_t)(cap + 1) * 4, sizeof(double));
    L->slot = (double*)calloc((size_t)(cap + 1) * r * r * 4, sizeof(double));
    int nf = 0;
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c0 = cidx(L, x, y);
            if (!is_active(L, c0)) continue;
            for (int d = 0; d < 4; d++) {
                int xx = x + CX[d], yy = y + CY[d];
                if (resolve(H, L, &xx, &yy)) continue;
                size_t c1 = cidx(L, xx, yy);
                if (!(L->in[c1] && L->ref[c1])) continue;
                L->fcell[nf] = (int32_t)c0;
                L->fdir[nf] = (int8_t)d;
                int of = oldidx ? oldidx[(size_t)d * L->n + c0] : -1;
                if (of >= 0 && of < oldn) {
                    L->fresh[nf] = oldfresh[of];
                    for (int k = 0; k < 4; k++) L->prev[nf * 4 + k] = oldprev[of * 4 + k];
                } else {
                    L->fresh[nf] = 1;
                }
                idx[(size_t)d * L->n + c0] = nf;
                nf++;
            }
        }
    L->nface = nf;
    free(oldidx); free(oldprev); free(oldfresh); free(oldcur);
    L->fidx = idx;
}

/* ------------------------------------------------------------------ */
/* Life cycle                                                          */
/* ------------------------------------------------------------------ */

void* ora_create(int nx0, int ny0, int nlev, int r, const int* bc, const double* wb,
                 double gamma, double c, double beta) {
    if (nlev < 1 || nlev > ORA_MAXLEV || r < 1 || nx0 < 1 || ny0 < 1) return NULL;
    for (int a = 0; a < 2; a++)
        if ((bc[2 * a] == BC_PERIODIC) != (bc[2 * a + 1] == BC_PERIODIC)) return NULL;
    OHier* H = (OHier*)calloc(1, sizeof(OHier));
    H->nlev = nlev; H->r = r; H->nx0 = nx0; H->ny0 = ny0;
    H->gamma = gamma; H->c = c; H->beta = beta;
    H->gm1 = gamma - 1.0;
    H->om = 1.0 - 2.0 * beta;
    H->hb = 0.5 * beta;
    H->bcs = beta / c;
    H->hc = 0.5 / c;
    for (int s = 0; s < 4; s++) {
        H->bc[s] = bc[s];
        for (int k = 0; k < 4; k++) H->wb[s][k] = wb ? wb[s * 4 + k] : 0.0;
        if (bc[s] == BC_INFLOW) ora_feq(gamma, c, H->wb[s], H->feqb[s]);
    }
    long sx = nx0, sy = ny0;
    for (int l = 0; l < nlev; l++) {
        OLevel* L = &H->lev[l];
        L->nx = (int)sx; L->ny = (int)sy;
        L->n = (size_t)sx * (size_t)sy;
        L->in = (uint8_t*)calloc(L->n, 1);
        L->ref = (uint8_t*)calloc(L->n, 1);
        L->f = (double*)calloc(16 * L->n, sizeof(double));
        L->fs = (double*)calloc(16 * L->n, sizeof(double));
        if (l == 0) memset(L->in, 1, L->n);
        sx *= r; sy *= r;
    }
    return H;
}

void ora_destroy(void* h) {
    OHier* H = (OHier*)h;
    if (!H) return;
    for (int l = 0; l < H->nlev; l++) {
        OLevel* L = &H->lev[l];
        free(L->in); free(L->ref); free(L->f); free(L->fs); free(L->fidx);
        free_faces(L);
    }
    free(H);
}

/* Nesting: every cell covered on level l >= 1 has its four face neighbours
 * (inside the domain) on level l, so that a level-(l+1) cell only ever
 * borders level-l cells.  Returns 0 when nested. */
static int check_nesting(const OHier* H, uint8_t* const* in, uint8_t* const* ref) {
    for (int l = 0; l < H->nlev; l++) {
        const OLevel* L = &H->lev[l];
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                size_t c = cidx(L, x, y);
                if (!ref[l][c]) continue;
                if (!in[l][c] || l == H->nlev - 1) return 1;
                if (l == 0) continue;
                for (int d = 0; d < 4; d++) {
                    int xx = x + CX[d], yy = y + CY[d];
                    if (resolve(H, L, &xx, &yy)) continue;
                    if (!in[l][cidx(L, xx, yy)]) return 2;
                }
            }
    }
    return 0;
}

/* in_{l+1} = children of cells covered on level l. */
static void derive_in(const OHier* H, uint8_t** in, uint8_t* const* ref) {
    int r = H->r;
    for (int l = 1; l < H->nlev; l++) {
        const OLevel* L = &H->lev[l];
        const OLevel* P = &H->lev[l - 1];
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                size_t pc = cidx(P, x / r, y / r);
                in[l][cidx(L, x, y)] = (uint8_t)(in[l - 1][pc] && ref[l - 1][pc]);
            }
    }
}

/* Installs a refinement layout without moving data (used before set_state).
 * ref[l] is a per-cell mask on level l (l < nlev-1).  Returns 0 or an error. */
int ora_set_layout(void* h, uint8_t* const* ref_in) {
    OHier* H = (OHier*)h;
    uint8_t* in[ORA_MAXLEV];
    uint8_t* ref[ORA_MAXLEV];
    for (int l = 0; l < H->nlev; l++) {
        OLevel* L = &H->lev[l];
        in[l] = (uint8_t*)calloc(L->n, 1);
        ref[l] = (uint8_t*)calloc(L->n, 1);
        if (l == 0) memset(in[0], 1, L->n);
        if (l < H->nlev - 1 && ref_in[l])
            for (size_t c = 0; c < L->n; c++) ref[l][c] = ref_in[l][c] ? 1 : 0;
    }
    derive_in(H, in, ref);
    int err = check_nesting(H, in, ref);
    if (!err) {
        for (int l = 0; l < H->nlev; l++) {
            OLevel* L = &H->lev[l];
            memcpy(L->in, in[l], L->n);
            memcpy(L->ref, ref[l], L->n);
            free(L->fidx); L->fidx = NULL;
            free_faces(L);
        }
        for (int l = 0; l < H->nlev; l++) build_faces(H, l);
    }
    for (int l = 0; l < H->nlev; l++) { free(in[l]); free(ref[l]); }
    return err;
}

/* f = f^eq(W) on every cell of level l (W is [4][ny][nx]). */
void ora_set_state(void* h, int l, const double* W) {
    OHier* H = (OHier*)h;
    OLevel* L = &H->lev[l];
    for (size_t c = 0; c < L->n; c++) {
        if (!L->in[c]) continue;
        double w[4], fe[16];
        for (int k = 0; k < 4; k++) w[k] = W[k * L->n + c];
        ora_feq(H->gamma, H->c, w, fe);
        for (int q = 0; q < 16; q++) L->f[q * L->n + c] = fe[q];
    }
}

void ora_set_f(void* h, int l, const double* f) {
    OHier* H = (OHier*)h;
    memcpy(H->lev[l].f, f, sizeof(double) * 16 * H->lev[l].n);
}

void ora_get_f(void* h, int l, double* f) {
    OHier* H = (OHier*)h;
    memcpy(f, H->lev[l].f, sizeof(double) * 16 * H->lev[l].n);
}

/* W = sum_i f_i on every cell of level l; flags: bit0 in_l, bit1 covered. */
void ora_get_W(void* h, int l, double* W, uint8_t* flags) {
    OHier* H = (OHier*)h;
    OLevel* L = &H->lev[l];
    for (size_t c = 0; c < L->n; c++) {
        double f[16], w[4];
        for (int q = 0; q < 16; q++) f[q] = L->f[q * L->n + c];
        moments(f, w);
        for (int k = 0; k < 4; k++) W[k * L->n + c] = L->in[c] ? w[k] : 0.0;
        if (flags) flags[c] = (uint8_t)(L->in[c] | (L->ref[c] << 1));
    }
}

void ora_get_layout(void* h, int l, uint8_t* in, uint8_t* ref) {
    OHier* H = (OHier*)h;
    memcpy(in, H->lev[l].in, H->lev[l].n);
    memcpy(ref, H->lev[l].ref, H->lev[l].n);
}

/* ------------------------------------------------------------------ */
/* Time stepping                                                       */
/* ------------------------------------------------------------------ */

static void gather(const OLevel* L, const double* a, size_t c, double v[16]) {
    for (int q = 0; q < 16; q++) v[q] = a[q * L->n + c];
}

/* ---- sensor-driven relaxation (Sec. 2.2, Eq. sensor-B) -------------
 * Per level step, on the pre-collision state of the level's active cells:
 *   s_k   = dx (div Q)_k / max_{x,alpha} |Q_{alpha,k}|, central differences,
 *           so s_k = g_k / (2 qmax_k) with g_k = (Qx_k(E) - Qx_k(W)) +
 *           (Qy_k(N) - Qy_k(S)); qmax_k fixed when the sensor is switched on
 *   s     = ((1/(D+2)) sum_k s_k^2)^(1/2), D = 2 (summed as
 *           (s_0^2 + s_3^2) + (s_1^2 + s_2^2))
 *   theta = dil^2 / (dil^2 + vort^2 + eps) where dil < 0, else 0 (Ducros-
 *           type), dil = (u(E) - u(W)) + (v(N) - v(S)),
 *           vort = (v(E) - v(W)) - (u(N) - u(S))  (undivided differences)
 *   s_bar, theta_bar = 3 x 3 box filters (box9)
 *   beta  = beta_max - (beta_max - beta_min) clip(C s_bar theta_bar, 0, 1)
 * A neighbour that is not an active cell of the level (covered, off the
 * level, beyond a non-periodic side) takes the centre cell's value. */
static double nbv(const OHier* H, const OLevel* L, const double* a, int x, int y, int dx, int dy) {
    int xx = x + dx, yy = y + dy;
    if (!resolve(H, L, &xx, &yy)) {
        size_t cn = cidx(L, xx, yy);
        if (is_active(L, cn)) return a[cn];
    }
    return a[cidx(L, x, y)];
}

/* Sum of a 3 x 3 neighbourhood, grouped so that swapping x and y gives
 * the same rounding: centre + ((E + W) + (N + S)) + ((NE + SW) + (NW + SE)). */
static double box9(const OHier* H, const OLevel* L, const double* a, int x, int y) {
    double edges = (nbv(H, L, a, x, y, 1, 0) + nbv(H, L, a, x, y, -1, 0)) +
                   (nbv(H, L, a, x, y, 0, 1) + nbv(H, L, a, x, y, 0, -1));
    double corners = (nbv(H, L, a, x, y, 1, 1) + nbv(H, L, a, x, y, -1, -1)) +
                     (nbv(H, L, a, x, y, -1, 1) + nbv(H, L, a, x, y, 1, -1));
    return (a[cidx(L, x, y)] + edges) + corners;
}

/* beta[c] for every active cell of level l (other cells untouched). */
static void sensor_beta(const OHier* H, const OLevel* L, double* beta) {
    const size_t n = L->n;
    double* pr = (double*)calloc(10 * n, sizeof(double));  /* Qx[4], Qy[4], u, v */
    double* st = (double*)calloc(2 * n, sizeof(double));   /* s, theta */
    for (size_t c = 0; c < n; c++) {
        if (!is_active(L, c)) continue;
        double f[16], W[4], Qx[4], Qy[4];
        gather(L, L->f, c, f);
        moments(f, W);
        euler_flux(H->gm1, W, Qx, Qy);
        double inv = 1.0 / W[0];
        for (int k = 0; k < 4; k++) {
            pr[k * n + c] = Qx[k];
            pr[(4 + k) * n + c] = Qy[k];
        }
        pr[8 * n + c] = W[1] * inv;
        pr[9 * n + c] = W[2] * inv;
    }
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = cidx(L, x, y);
            if (!is_active(L, c)) continue;
            double sh[4];
            for (int k = 0; k < 4; k++) {
                const double* qx = pr + k * n;
                const double* qy = pr + (4 + k) * n;
                double g = (nbv(H, L, qx, x, y, 1, 0) - nbv(H, L, qx, x, y, -1, 0)) +
                           (nbv(H, L, qy, x, y, 0, 1) - nbv(H, L, qy, x, y, 0, -1));
                sh[k] = g * H->iq[k];
            }
            /* fields paired (rho, rho E), (rho u, rho v): the grouping is
             * the same after swapping x and y */
            st[c] = sqrt(0.25 * ((sh[0] * sh[0] + sh[3] * sh[3]) + (sh[1] * sh[1] + sh[2] * sh[2])));
            const double* u = pr + 8 * n;
            const double* v = pr + 9 * n;
            double dil = (nbv(H, L, u, x, y, 1, 0) - nbv(H, L, u, x, y, -1, 0)) +
                         (nbv(H, L, v, x, y, 0, 1) - nbv(H, L, v, x, y, 0, -1));
            double vort = (nbv(H, L, v, x, y, 1, 0) - nbv(H, L, v, x, y, -1, 0)) -
                          (nbv(H, L, u, x, y, 0, 1) - nbv(H, L, u, x, y, 0, -1));
            double d2 = dil * dil;
            st[n + c] = dil < 0.0 ? d2 / ((d2 + vort * vort) + H->eps) : 0.0;
        }
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = cidx(L, x, y);
            if (!is_active(L, c)) continue;
            double as = box9(H, L, st, x, y), at = box9(H, L, st + n, x, y);
            double z = (H->csens * (H->ninth * as)) * (H->ninth * at);
            if (z < 0.0) z = 0.0;
            if (z > 1.0) z = 1.0;
            beta[c] = H->beta - (H->beta - H->beta_min) * z;
        }
    free(pr);
    free(st);
}

static void step(OHier* H, int l, int k) {
    OLevel* L = &H->lev[l];
    const int r = H->r;
    const size_t n = L->n;

    /* 1. collision on every active cell of level l (relaxation parameter
     *    per cell from the sensor when it is on) */
    double* beta = NULL;
    if (H->sensor) {
        beta = (double*)calloc(n, sizeof(double));
        sensor_beta(H, L, beta);
    }
    for (size_t c = 0; c < n; c++) {
        if (!is_active(L, c)) continue;
        double f[16], fs[16];
        gather(L, L->f, c, f);
        if (beta) {
            double b = beta[c];
            collide_with(H->gm1, 1.0 - 2.0 * b, 0.5 * b, b / H->c, f, fs);
        } else {
            collide_cell(H, f, fs);
        }
        for (int q = 0; q < 16; q++) L->fs[q * n + c] = fs[q];
    }
    free(beta);

    /* 2. fine side: post-collision populations leaving towards coarser
     *    territory go to the register of their face, slot (k, j). */
    if (l >= 1) {
        OLevel* P = &H->lev[l - 1];
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                size_t c = cidx(L, x, y);
                if (!is_active(L, c)) continue;
                for (int i = 0; i < 4; i++) {
                    int xx = x + CX[i], yy = y + CY[i];
                    if (resolve(H, L, &xx, &yy)) continue;
                    if (L->in[cidx(L, xx, yy)]) continue;
                    int d = i ^ 1; /* from the coarse cell L0 towards this cell */
                    size_t l0 = cidx(P, xx / r, yy / r);
                    int F = P->fidx[(size_t)d * P->n + l0];
                    int j = (d < 2) ? (y % r) : (x % r);
                    for (int kf = 0; kf < 4; kf++)
                        P->slot[(((size_t)F * r + (k - 1)) * r + j) * 4 + kf] = L->fs[QI(i, kf) * n + c];
                }
            }
    }

    /* 3. coarse side: capture cur and the tangential slope of every face */
    if (l < H->nlev - 1) {
        for (int F = 0; F < L->nface; F++) {
            size_t c0 = (size_t)L->fcell[F];
            int d = L->fdir[F];
            int x = (int)(c0 % (size_t)L->nx), y = (int)(c0 / (size_t)L->nx);
            int tx = (d < 2) ? 0 : 1, ty = (d < 2) ? 1 : 0;
            int xm = x - tx, ym = y - ty, xp = x + tx, yp = y + ty;
            int okm = !resolve(H, L, &xm, &ym) && is_active(L, cidx(L, xm, ym));
            int okp = !resolve(H, L, &xp, &yp) && is_active(L, cidx(L, xp, yp));
            for (int kf = 0; kf < 4; kf++) {
                double a = L->fs[QI(d, kf) * n + c0];
                L->cur[F * 4 + kf] = a;
                double s = 0.0;
                if (okm && okp) {
                    double am = L->fs[QI(d, kf) * n + cidx(L, xm, ym)];
                    double ap = L->fs[QI(d, kf) * n + cidx(L, xp, yp)];
                    s = ora_minmod(a - am, ap - a);
                }
                L->sig[F * 4 + kf] = s;
                if (L->fresh[F]) L->prev[F * 4 + kf] = a;
            }
            L->fresh[F] = 0;
        }
    }

    /* 4. streaming */
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = cidx(L, x, y);
            if (!is_active(L, c)) continue;
            for (int i = 0; i < 4; i++) {
                int ux = x - CX[i], uy = y - CY[i];
                int side = resolve(H, L, &ux, &uy);
                for (int kf = 0; kf < 4; kf++) {
                    size_t dst = QI(i, kf) * n + c;
                    if (side) {
                        int s = side - 1;
                        int bc = H->bc[s];
                        if (bc == BC_OUTFLOW) {
                            L->f[dst] = L->fs[QI(i, kf) * n + c];
                        } else if (bc == BC_INFLOW) {
                            L->f[dst] = H->feqb[s][QI(i, kf)];
                        } else { /* reflective wall: mirror state, normal momentum flipped */
                            int normal = (s < 2) ? 1 : 2;
                            double v = L->fs[QI(i ^ 1, kf) * n + c];
                            L->f[dst] = (kf == normal) ? -v : v;
                        }
                        continue;
                    }
                    size_t u = cidx(L, ux, uy);
                    if (is_active(L, u)) {
                        L->f[dst] = L->fs[QI(i, kf) * n + u];
                    } else if (L->in[u]) {
                        /* covered: pending, filled by the reflux of level l+1 */
                    } else {
                        OLevel* P = &H->lev[l - 1];
                        size_t l0 = cidx(P, ux / r, uy / r);
                        int F = P->fidx[(size_t)i * P->n + l0];
                        int j = (i < 2) ? (y % r) : (x % r);
                        L->f[dst] = ora_recon(P->cur[F * 4 + kf], P->prev[F * 4 + kf], P->sig[F * 4 + kf], r, k, j);
                    }
                }
            }
        }

    /* 5. sub-cycle the finer level, 6. reflux */
    if (l < H->nlev - 1) {
        for (int kk = 1; kk <= r; kk++) step(H, l + 1, kk);
        double w = 1.0 / (double)(r * r);
        for (int F = 0; F < L->nface; F++) {
            size_t c0 = (size_t)L->fcell[F];
            int d = L->fdir[F];
            for (int kf = 0; kf < 4; kf++) {
                double tot = 0.0;
                for (int kk = 0; kk < r; kk++) {
                    double row = L->slot[(((size_t)F * r + kk) * r + 0) * 4 + kf];
                    for (int j = 1; j < r; j++) row += L->slot[(((size_t)F * r + kk) * r + j) * 4 + kf];
                    tot = (kk == 0) ? row : tot + row;
                }
                L->f[QI(d ^ 1, kf) * n + c0] = tot * w;
                L->prev[F * 4 + kf] = L->cur[F * 4 + kf];
            }
        }
    }
}

void ora_advance(void* h, int nsteps) {
    OHier* H = (OHier*)h;
    for (int s = 0; s < nsteps; s++) step(H, 0, 1);
}

/* ------------------------------------------------------------------ */
/* Adaptive refinement: average-down, tagging, layout, merge, split     */
/* ------------------------------------------------------------------ */

/* comp[l] = f on level l, with every covered cell replaced by the merge of
 * its children (finest level first), Eq. 25. */
static double** composite(const OHier* H) {
    int r = H->r;
    double** comp = (double**)calloc(H->nlev, sizeof(double*));
    for (int l = H->nlev - 1; l >= 0; l--) {
        const OLevel* L = &H->lev[l];
        comp[l] = (double*)malloc(sizeof(double) * 16 * L->n);
        memcpy(comp[l], L->f, sizeof(double) * 16 * L->n);
        if (l == H->nlev - 1) continue;
        const OLevel* C = &H->lev[l + 1];
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                size_t c = cidx(L, x, y);
                if (!(L->in[c] && L->ref[c])) continue;
                for (int q = 0; q < 16; q++) {
                    double ch[64];
                    for (int b = 0; b < r; b++)
                        for (int a = 0; a < r; a++)
                            ch[b * r + a] = comp[l + 1][q * C->n + cidx(C, x * r + a, y * r + b)];
                    comp[l][q * L->n + c] = merge_vals(ch, r);
                }
            }
    }
    return comp;
}

static void free_comp(const OHier* H, double** comp) {
    for (int l = 0; l < H->nlev; l++) free(comp[l]);
    free(comp);
}

static double rho_of(const OLevel* L, const double* a, size_t c) {
    double f[16], W[4];
    gather(L, a, c, f);
    moments(f, W);
    return W[0];
}

/* Normalised density-gradient indicator on level l: a cell is tagged when
 * (rho_E - rho_W)^2 + (rho_N - rho_S)^2 > tol^2 (2 rho_C)^2.  Neighbours that
 * are not on level l, or lie beyond a non-periodic side, take rho_C. */
static void tag_level(const OHier* H, int l, double* const* comp, double tol2, uint8_t* tag) {
    const OLevel* L = &H->lev[l];
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = cidx(L, x, y);
            tag[c] = 0;
            if (!L->in[c]) continue;
            double rc = rho_of(L, comp[l], c);
            double rn[4];
            for (int d = 0; d < 4; d++) {
                int xx = x + CX[d], yy = y + CY[d];
                if (!resolve(H, L, &xx, &yy) && L->in[cidx(L, xx, yy)])
                    rn[d] = rho_of(L, comp[l], cidx(L, xx, yy));
                else
                    rn[d] = rc;
            }
            double d1 = rn[0] - rn[1];
            double d2 = rn[2] - rn[3];
            double num = d1 * d1 + d2 * d2;
            double t = 2.0 * rc;
            tag[c] = (uint8_t)(num > tol2 * (t * t));
        }
}

/* Flux-jump sensor of Sec. 3.4, Eq. amr-sigma: per field k the jump
 * estimate s_k = dx (div Q)_k / max_{x,alpha} |Q_{alpha,k}|, combined with a
 * max norm, s = max_k |s_k|; a cell is tagged when s > tol.  With central
 * differences (div Q)_k = ((Qx_k(E) - Qx_k(W)) + (Qy_k(N) - Qy_k(S))) / (2 dx),
 * so dx cancels and s_k > tol reads |g_k| > (2 tol) qmax_k with
 * g_k = (Qx_k(E) - Qx_k(W)) + (Qy_k(N) - Qy_k(S)) (no division; a field
 * whose flux vanishes everywhere never tags).  Q is the Euler flux of the
 * composite state; qmax_k runs over every cell of every level (covered
 * cells holding the average of their children); neighbours off the level or
 * beyond a non-periodic side take the cell's own flux. */
static void comp_flux(const OHier* H, const OLevel* L, const double* a, size_t c, double Qx[4], double Qy[4]) {
    double f[16], W[4];
    gather(L, a, c, f);
    moments(f, W);
    euler_flux(H->gamma - 1.0, W, Qx, Qy);
}

static void flux_max(const OHier* H, double* const* comp, double qmax[4]) {
    for (int k = 0; k < 4; k++) qmax[k] = 0.0;
    for (int l = 0; l < H->nlev; l++) {
        const OLevel* L = &H->lev[l];
        for (size_t c = 0; c < L->n; c++) {
            if (!L->in[c]) continue;
            double Qx[4], Qy[4];
            comp_flux(H, L, comp[l], c, Qx, Qy);
            for (int k = 0; k < 4; k++) {
                if (fabs(Qx[k]) > qmax[k]) qmax[k] = fabs(Qx[k]);
                if (fabs(Qy[k]) > qmax[k]) qmax[k] = fabs(Qy[k]);
            }
        }
    }
}

static void tag_level_flux(const OHier* H, int l, double* const* comp, const double qmax[4], double tol,
                           uint8_t* tag) {
    const OLevel* L = &H->lev[l];
    for (int y = 0; y < L->ny; y++)
        for (int x = 0; x < L->nx; x++) {
            size_t c = cidx(L, x, y);
            tag[c] = 0;
            if (!L->in[c]) continue;
            double Qx[4][4], Qy[4][4], Qcx[4], Qcy[4];
            comp_flux(H, L, comp[l], c, Qcx, Qcy);
            for (int d = 0; d < 4; d++) {
                int xx = x + CX[d], yy = y + CY[d];
                if (!resolve(H, L, &xx, &yy) && L->in[cidx(L, xx, yy)]) {
                    comp_flux(H, L, comp[l], cidx(L, xx, yy), Qx[d], Qy[d]);
                } else {
                    for (int k = 0; k < 4; k++) {
                        Qx[d][k] = Qcx[k];
                        Qy[d][k] = Qcy[k];
                    }
                }
            }
            int t = 0;
            for (int k = 0; k < 4; k++) {
                double g = (Qx[0][k] - Qx[1][k]) + (Qy[2][k] - Qy[3][k]);
                if (fabs(g) > (2.0 * tol) * qmax[k]) t = 1;
            }
            tag[c] = (uint8_t)t;
        }
}

/* The tags of every refinable level: sensor 0 = normalised density
 * gradient, 1 = flux jump (max norm). */
static void tag_all(const OHier* H, double* const* comp, int sensor, double tol, uint8_t* const* tags) {
    double qmax[4];
    if (sensor == 1) flux_max(H, comp, qmax);
    for (int l = 0; l <= H->nlev - 2; l++) {
        if (sensor == 1) tag_level_flux(H, l, comp, qmax, tol, tags[l]);
        else tag_level(H, l, comp, tol * tol, tags[l]);
    }
}

/* Regrid layout.  tags[l] (l <= nlev-2) are per-cell tags on level l.  From
 * the finest refinable level down: dilate the tags by `buffer` cells (square
 * neighbourhood), add the parents of the 8-neighbourhood of the next finer
 * refined set (proper nesting), and round up to aligned `block` x `block`
 * blocks of level-l cells.  Writes newref[l] (per cell, level l). */
static void layout_from_tags(const OHier* H, uint8_t* const* tags, int buffer, int block, uint8_t** newref) {
    int r = H->r;
    for (int l = H->nlev - 1; l >= 0; l--) {
        const OLevel* L = &H->lev[l];
        memset(newref[l], 0, L->n);
        if (l == H->nlev - 1) continue;
        uint8_t* D = (uint8_t*)calloc(L->n, 1);
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                if (!tags[l][cidx(L, x, y)]) continue;
                for (int dy = -buffer; dy <= buffer; dy++)
                    for (int dx = -buffer; dx <= buffer; dx++) {
                        int xx = x + dx, yy = y + dy;
                        if (resolve(H, L, &xx, &yy)) continue;
                        D[cidx(L, xx, yy)] = 1;
                    }
            }
        if (l + 1 <= H->nlev - 2) {
            const OLevel* C = &H->lev[l + 1];
            for (int y = 0; y < C->ny; y++)
                for (int x = 0; x < C->nx; x++) {
                    if (!newref[l + 1][cidx(C, x, y)]) continue;
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            int xx = x + dx, yy = y + dy;
                            if (resolve(H, C, &xx, &yy)) continue;
                            D[cidx(L, xx / r, yy / r)] = 1;
                        }
                }
        }
        int bx = (L->nx + block - 1) / block, by = (L->ny + block - 1) / block;
        for (int jb = 0; jb < by; jb++)
            for (int ib = 0; ib < bx; ib++) {
                int any = 0;
                for (int y = jb * block; y < (jb + 1) * block && y < L->ny && !any; y++)
                    for (int x = ib * block; x < (ib + 1) * block && x < L->nx; x++)
                        if (D[cidx(L, x, y)]) { any = 1; break; }
                if (!any) continue;
                for (int y = jb * block; y < (jb + 1) * block && y < L->ny; y++)
                    for (int x = ib * block; x < (ib + 1) * block && x < L->nx; x++) newref[l][cidx(L, x, y)] = 1;
            }
        free(D);
    }
}

/* Conservative regrid to the layout newref (Sec. 3.4, Fig. 2): cells leaving
 * refinement take the merge of their children (finest level first, Eq. 25);
 * cells entering refinement are split with minmod slopes (coarsest level
 * first, Eqs. 26-27).  Faces that persist keep their previous sample. */
static int regrid_to(OHier* H, uint8_t* const* newref_in, double** comp) {
    int r = H->r;
    uint8_t* in[ORA_MAXLEV];
    uint8_t* ref[ORA_MAXLEV];
    for (int l = 0; l < H->nlev; l++) {
        OLevel* L = &H->lev[l];
        in[l] = (uint8_t*)calloc(L->n, 1);
        ref[l] = (uint8_t*)calloc(L->n, 1);
        if (l == 0) memset(in[0], 1, L->n);
        if (l < H->nlev - 1)
            for (size_t c = 0; c < L->n; c++) ref[l][c] = newref_in[l][c] ? 1 : 0;
    }
    derive_in(H, in, ref);
    int err = check_nesting(H, in, ref);
    if (err) {
        for (int l = 0; l < H->nlev; l++) { free(in[l]); free(ref[l]); }
        return err;
    }
    /* merge: every cell covered before and not covered now */
    for (int l = H->nlev - 2; l >= 0; l--) {
        OLevel* L = &H->lev[l];
        for (size_t c = 0; c < L->n; c++) {
            int oldcov = L->in[c] && L->ref[c];
            int newcov = in[l][c] && ref[l][c];
            if (oldcov && !newcov)
                for (int q = 0; q < 16; q++) L->f[q * L->n + c] = comp[l][q * L->n + c];
        }
    }
    /* split: every cell covered now and not before, coarsest first */
    for (int l = 0; l <= H->nlev - 2; l++) {
        OLevel* L = &H->lev[l];
        OLevel* C = &H->lev[l + 1];
        for (int y = 0; y < L->ny; y++)
            for (int x = 0; x < L->nx; x++) {
                size_t c = cidx(L, x, y);
                int oldcov = L->in[c] && L->ref[c];
                int newcov = in[l][c] && ref[l][c];
                if (!newcov || oldcov) continue;
                int nb[4];
                int ok[4];
                for (int d = 0; d < 4; d++) {
                    int xx = x + CX[d], yy = y + CY[d];
                    ok[d] = !resolve(H, L, &xx, &yy);
                    nb[d] = ok[d] ? (int)cidx(L, xx, yy) : -1;
                }
                for (int q = 0; q < 16; q++) {
                    double fc = L->f[q * L->n + c];
                    double v[4];
                    for (int d = 0; d < 4; d++) {
                        if (!ok[d]) { v[d] = fc; continue; }
                        size_t cn = (size_t)nb[d];
                        int ncov = L->in[cn] && L->ref[cn]; /* covered before: use its children */
                        v[d] = ncov ? comp[l][q * L->n + cn] : L->f[q * L->n + cn];
                    }
                    double sx = (ok[0] && ok[1]) ? ora_minmod(fc - v[1], v[0] - fc) : 0.0;
                    double sy = (ok[2] && ok[3]) ? ora_minmod(fc - v[3], v[2] - fc) : 0.0;
                    for (int b = 0; b < r; b++)
                        for (int a = 0; a < r; a++)
                            C->f[q * C->n + cidx(C, x * r + a, y * r + b)] = ora_split_child(fc, sx, sy, r, a, b);
                }
            }
    }
    for (int l = 0; l < H->nlev; l++) {
        OLevel* L = &H->lev[l];
        memcpy(L->in, in[l], L->n);
        memcpy(L->ref, ref[l], L->n);
    }
    for (int l = 0; l < H->nlev; l++) build_faces(H, l);
    for (int l = 0; l < H->nlev; l++) { free(in[l]); free(ref[l]); }
    return 0;
}

/* Regrid to a given layout (per-cell masks newref[l], l <= nlev-2). */
int ora_regrid(void* h, uint8_t* const* newref) {
    OHier* H = (OHier*)h;
    double** comp = composite(H);
    int err = regrid_to(H, newref, comp);
    free_comp(H, comp);
    return err;
}

/* Tag-driven regrid: indicator, dilation, block rounding, nesting, then the
 * conservative merge/split.  Writes the chosen layout to newref_out when it
 * is not NULL.  Returns 0 or an error. */
int ora_regrid_tagged(void* h, int sensor, double tol, int buffer, int block, uint8_t** newref_out) {
    OHier* H = (OHier*)h;
    double** comp = composite(H);
    uint8_t* tags[ORA_MAXLEV];
    uint8_t* newref[ORA_MAXLEV];
    for (int l = 0; l < H->nlev; l++) {
        tags[l] = (uint8_t*)calloc(H->lev[l].n, 1);
        newref[l] = (uint8_t*)calloc(H->lev[l].n, 1);
    }
    tag_all(H, comp, sensor, tol, tags);
    layout_from_tags(H, tags, buffer, block, newref);
    int err = regrid_to(H, newref, comp);
    if (newref_out)
        for (int l = 0; l < H->nlev - 1; l++) memcpy(newref_out[l], newref[l], H->lev[l].n);
    for (int l = 0; l < H->nlev; l++) { free(tags[l]); free(newref[l]); }
    free_comp(H, comp);
    return err;
}

/* Exposes the layout rule alone (tags given per level) for tests. */
void ora_layout_from_tags(void* h, uint8_t* const* tags, int buffer, int block, uint8_t** newref) {
    layout_from_tags((OHier*)h, tags, buffer, block, newref);
}

/* Exposes the indicator alone on the current composite state. */
void ora_tags(void* h, int sensor, double tol, uint8_t** tags) {
    OHier* H = (OHier*)h;
    double** comp = composite(H);
    tag_all(H, comp, sensor, tol, tags);
    free_comp(H, comp);
}

/* The flux maxima qmax_k of the flux-jump sensor on the composite state. */
void ora_flux_max(void* h, double qmax[4]) {
    OHier* H = (OHier*)h;
    double** comp = composite(H);
    flux_max(H, comp, qmax);
    free_comp(H, comp);
}

/* Sensor-driven relaxation: on = 1 switches it on with beta_max = the
 * hierarchy's beta, the given beta_min, C_sensor and eps, and fixes
 * qmax_k = max |Q_{alpha,k}| over the active cells of every level of the
 * current state; on = 0 returns to the constant beta. */
void ora_set_sensor(void* h, int on, double beta_min, double csens, double eps) {
    OHier* H = (OHier*)h;
    H->sensor = on;
    H->beta_min = beta_min;
    H->csens = csens;
    H->eps = eps;
    H->ninth = 1.0 / 9.0;
    double qmax[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < H->nlev; l++) {
        const OLevel* L = &H->lev[l];
        for (size_t c = 0; c < L->n; c++) {
            if (!is_active(L, c)) continue;
            double f[16], W[4], Qx[4], Qy[4];
            gather(L, L->f, c, f);
            moments(f, W);
            euler_flux(H->gm1, W, Qx, Qy);
            for (int k = 0; k < 4; k++) {
                if (fabs(Qx[k]) > qmax[k]) qmax[k] = fabs(Qx[k]);
                if (fabs(Qy[k]) > qmax[k]) qmax[k] = fabs(Qy[k]);
            }
        }
    }
    for (int k = 0; k < 4; k++) H->iq[k] = qmax[k] > 0.0 ? 1.0 / (2.0 * qmax[k]) : 0.0;
}

/* The relaxation parameter the next step of level l would use on each
 * active cell (constant beta when the sensor is off; 0 elsewhere). */
void ora_sensor_beta(void* h, int l, double* out) {
    OHier* H = (OHier*)h;
    const OLevel* L = &H->lev[l];
    for (size_t c = 0; c < L->n; c++) out[c] = is_active(L, c) ? H->beta : 0.0;
    if (H->sensor) {
        double* b = (double*)calloc(L->n, sizeof(double));
        sensor_beta(H, L, b);
        for (size_t c = 0; c < L->n; c++)
            if (is_active(L, c)) out[c] = b[c];
        free(b);
    }
}
