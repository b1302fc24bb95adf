/*
 * DMTz CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the method of "Preserving Discrete
 * Morse-Smale Complexes in Error-Bounded Lossy Compression" (Li, Xia, Liang, Wang, Guo):
 * the iterative edit loop that corrects a decompressed scalar field g until its discrete
 * Morse-Smale complex (critical cells and separatrices) equals that of the original f,
 * while |f - g| <= xi holds at every vertex.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg load this
 * library.  It shares no code, table or header with the CUDA path: every structure below
 * is derived at run time from the definitions, with generic set operations.
 *
 *  - Complex: the Freudenthal (Kuhn) triangulation of the regular grid (Sec. 4.8.1, six
 *    tetrahedra per cube; Sec. 5, "regular grid-based triangulation").  A cell is a set of
 *    pairwise adjacent vertices whose offsets from its smallest-index vertex are 0/1 axis
 *    vectors forming a chain under inclusion.  Two vertices are adjacent when their
 *    coordinate difference is +-(a non-zero 0/1 vector).
 *  - Vertex order: simulation of simplicity (Sec. 4.1, "Degeneracy handling"):
 *    a < b  <=>  f[a] < f[b], or f[a] == f[b] and a < b (IEEE comparison, -0 == +0).
 *  - Discrete gradient: the closed-form pairing rules of Sec. 4.2 (gradient_rules), pinned
 *    against a brute-force evaluation of the function extension of Eq. 1 together with the
 *    lowest-cofacet rule of Sec. 3.1 (gradient_brute).
 *  - Fix loop: C-passes (Sec. 4.3), S-passes (Sec. 4.4), quantised edits (Eq. 2, Sec. 4.7),
 *    alternation until convergence (Sec. 4.5), tiers (Sec. 4.1 / 4.6).
 *
 * Readings taken where the paper is silent (each is listed in the design notes):
 *  - FN targets choose, among the paper's allowed vertices, the one lowest in f; when the
 *    cell's vertex order already matches f, the f-pairing of the facet is repaired instead.
 *  - The clamp bounds are rounded outward-safe: lb = f - xi rounded up, ub = f + xi rounded
 *    down, so |f - g| <= xi holds exactly.
 *  - A case whose target vertex can no longer move (floor or exact) is "stuck"; with the
 *    exact fallback, every vertex of the closed 1-rings of the case cell's vertices is
 *    restored to f exactly.  Stuck cases arise only from float ties of f - xi.
 *  - T3 compares per-path terminals of descending and ascending separatrices (saddle-to-
 *    extremum connectivity); T4 compares every pair along every separatrix, including
 *    saddle-saddle connectors in 3D.
 *
 * Threads: the per-cell loops (pairing within one dimension, the C-pass, the separatrices of
 * the S-pass) run as OpenMP loops over cells or paths.  Within a dimension each cell's pairing
 * reads only pairings of the dimension below, and the target sets are sets, so every result
 * is the same for any number of threads (a CPU test checks 1 thread against several); a
 * pass that records its case list or walk (test exports) runs on one thread.
 *
 * Parity unpinned: exact iteration counts and edit sequences have no printed worked loop;
 * they are pinned only through the invariants (monotone edits, bound, termination, final
 * MSC equality) that the tests check.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_NOT_CONVERGED 4
#define ORC_ERR_STALLED 6
#define ORC_ERR_INTERNAL 9

/* vertex states during the loop */
#define ST_FLOOR 0xF0   /* g == lb, stored losslessly (Eq. 2, "otherwise" branch) */
#define ST_EXACT 0xF1   /* g == f,  stored losslessly (stuck-case fallback)       */

/* ------------------------------------------------------------------------- */
/* grid and implicit cells                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int nx, ny, nz, dim;
    i64 n;
    int K;                    /* number of cell shapes per anchor vertex            */
    int shape_mask[32];       /* bit (A-1) set <=> anchor + e_A is a vertex of cell */
    int shape_dim[32];
    int mask_to_shape[128];
} grid_t;

static int grid_init(grid_t *g, int nx, int ny, int nz)
{
    if (nx < 2 || ny < 2 || nz < 1) return -1;
    g->nx = nx; g->ny = ny; g->nz = nz;
    g->dim = nz >= 2 ? 3 : 2;
    g->n = (i64)nx * ny * nz;
    int axes = g->dim == 3 ? 7 : 3;
    g->K = 0;
    for (int m = 0; m < 128; m++) g->mask_to_shape[m] = -1;
    for (int m = 0; m < 128; m++) {
        int ok = 1, cnt = 0;
        for (int A = 1; A <= 7; A++) {
            if (!((m >> (A - 1)) & 1)) continue;
            cnt++;
            if (A & ~axes) ok = 0;
            for (int B = 1; B <= 7; B++) {
                if (B == A || !((m >> (B - 1)) & 1)) continue;
                if ((A & B) != A && (A & B) != B) ok = 0;   /* not a chain */
            }
        }
        if (!ok) continue;
        g->shape_mask[g->K] = m;
        g->shape_dim[g->K] = cnt;
        g->mask_to_shape[m] = g->K;
        g->K++;
    }
    return 0;
}

static void vcoord(const grid_t *g, i64 v, int *x, int *y, int *z)
{
    if (g->n <= (i64)UINT32_MAX) {        /* the same quotients in 32-bit arithmetic */
        uint32_t u = (uint32_t)v, t = u / (uint32_t)g->nx;
        *x = (int)(u - t * (uint32_t)g->nx);
        *y = (int)(t % (uint32_t)g->ny);
        *z = (int)(t / (uint32_t)g->ny);
        return;
    }
    *x = (int)(v % g->nx);
    *y = (int)((v / g->nx) % g->ny);
    *z = (int)(v / ((i64)g->nx * g->ny));
}

static i64 vindex(const grid_t *g, int x, int y, int z)
{
    if (x < 0 || y < 0 || z < 0 || x >= g->nx || y >= g->ny || z >= g->nz) return -1;
    return (i64)x + (i64)g->nx * ((i64)y + (i64)g->ny * z);
}

/* u ~ v  <=>  v - u = +-(non-zero 0/1 vector) */
static int adjacent(const grid_t *g, i64 u, i64 v)
{
    if (u == v) return 0;
    int ux, uy, uz, vx, vy, vz;
    vcoord(g, u, &ux, &uy, &uz);
    vcoord(g, v, &vx, &vy, &vz);
    int dx = vx - ux, dy = vy - uy, dz = vz - uz;
    int pos = dx >= 0 && dy >= 0 && dz >= 0 && dx <= 1 && dy <= 1 && dz <= 1;
    int neg = dx <= 0 && dy <= 0 && dz <= 0 && dx >= -1 && dy >= -1 && dz >= -1;
    return pos || neg;
}

/* the same test as adjacent(), on the coordinate difference itself */
static int adjacent_offset(int dx, int dy, int dz)
{
    if (dx == 0 && dy == 0 && dz == 0) return 0;
    int pos = dx >= 0 && dy >= 0 && dz >= 0;
    int neg = dx <= 0 && dy <= 0 && dz <= 0;
    return pos || neg;
}

static int neighbours(const grid_t *g, i64 v, i64 out[26])
{
    int x, y, z, n = 0;
    vcoord(g, v, &x, &y, &z);
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                if (!adjacent_offset(dx, dy, dz)) continue;
                i64 w = vindex(g, x + dx, y + dy, z + dz);
                if (w >= 0) out[n++] = w;
            }
    return n;
}

static void sort_ids(i64 *v, int n)
{
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && v[j - 1] > v[j]; j--) { i64 t = v[j]; v[j] = v[j - 1]; v[j - 1] = t; }
}

/* vertices (ascending index) of cell id; returns the vertex count, 0 if no such cell */
static int cell_verts(const grid_t *g, i64 id, i64 v[4])
{
    i64 p = id / g->K;
    int k = (int)(id % g->K), x, y, z, nv = 0;
    vcoord(g, p, &x, &y, &z);
    v[nv++] = p;
    for (int A = 1; A <= 7; A++) {
        if (!((g->shape_mask[k] >> (A - 1)) & 1)) continue;
        i64 w = vindex(g, x + (A & 1), y + ((A >> 1) & 1), z + ((A >> 2) & 1));
        if (w < 0) return 0;
        v[nv++] = w;
    }
    sort_ids(v, nv);
    return nv;
}

static int cell_dim(const grid_t *g, i64 id) { return g->shape_dim[id % g->K]; }

/* id of the cell with the given vertex set, -1 if the set is not a cell */
static i64 cell_id(const grid_t *g, const i64 *vin, int nv)
{
    i64 v[4];
    if (nv < 1 || nv > 4) return -1;
    for (int i = 0; i < nv; i++) v[i] = vin[i];
    sort_ids(v, nv);
    int px, py, pz, mask = 0;
    vcoord(g, v[0], &px, &py, &pz);
    for (int i = 1; i < nv; i++) {
        int x, y, z;
        if (v[i] == v[i - 1]) return -1;
        vcoord(g, v[i], &x, &y, &z);
        int dx = x - px, dy = y - py, dz = z - pz;
        if (dx < 0 || dy < 0 || dz < 0 || dx > 1 || dy > 1 || dz > 1) return -1;
        int A = dx | (dy << 1) | (dz << 2);
        if (A == 0) return -1;
        mask |= 1 << (A - 1);
    }
    int k = g->mask_to_shape[mask];
    if (k < 0 || g->shape_dim[k] != nv - 1) return -1;
    return v[0] * g->K + k;
}

static int cell_exists(const grid_t *g, i64 id) { i64 v[4]; return cell_verts(g, id, v) > 0; }

/* cofacets: cells with one more vertex */
static int cofacets(const grid_t *g, i64 id, i64 out[16])
{
    i64 v[5], nb[26];
    int nv = cell_verts(g, id, v), n = 0;
    int nn = neighbours(g, v[0], nb);
    for (int i = 0; i < nn; i++) {
        int ok = 1;
        for (int j = 0; j < nv; j++)
            if (nb[i] == v[j] || !adjacent(g, nb[i], v[j])) ok = 0;
        if (!ok) continue;
        v[nv] = nb[i];
        i64 c = cell_id(g, v, nv + 1);
        if (c >= 0) out[n++] = c;
    }
    return n;
}

/* facets: cells with one vertex removed */
static int facets(const grid_t *g, i64 id, i64 out[4])
{
    i64 v[4], w[4];
    int nv = cell_verts(g, id, v), n = 0;
    if (nv < 2) return 0;
    for (int drop = 0; drop < nv; drop++) {
        int m = 0;
        for (int j = 0; j < nv; j++) if (j != drop) w[m++] = v[j];
        out[n++] = cell_id(g, w, m);
    }
    return n;
}

/* the vertex of U that is not in L (L a facet of U) */
static i64 extra_vertex(const grid_t *g, i64 U, i64 L)
{
    i64 u[4], l[4];
    int nu = cell_verts(g, U, u), nl = cell_verts(g, L, l);
    for (int i = 0; i < nu; i++) {
        int in = 0;
        for (int j = 0; j < nl; j++) if (u[i] == l[j]) in = 1;
        if (!in) return u[i];
    }
    return -1;
}

/* ------------------------------------------------------------------------- */
/* simulation of simplicity (Sec. 4.1)                                        */
/* ------------------------------------------------------------------------- */

static int sos_lt(const float *f, i64 a, i64 b)
{
    return f[a] < f[b] || (f[a] == f[b] && a < b);
}

static i64 lowest_vertex(const grid_t *g, i64 id, const float *f)
{
    i64 v[4];
    int nv = cell_verts(g, id, v);
    i64 lo = v[0];
    for (int i = 1; i < nv; i++) if (sos_lt(f, v[i], lo)) lo = v[i];
    return lo;
}

/* ------------------------------------------------------------------------- */
/* discrete gradient                                                          */
/* ------------------------------------------------------------------------- */
/* pr[id] = partner cell, -1 = critical (unpaired), -2 = no such cell */

static void pairing_init(const grid_t *g, i64 *pr)
{
    i64 ncell = g->n * g->K;
#pragma omp parallel for schedule(static)
    for (i64 id = 0; id < ncell; id++) pr[id] = cell_exists(g, id) ? -1 : -2;
}

/* Sec. 4.2, the three pairing rules: a vertex pairs with the edge to its lowest lower
 * neighbour; a cell not paired by a facet pairs with the cofacet whose extra vertex lies
 * below every vertex of the cell, taking the lowest such extra vertex.  Dimensions are
 * processed in ascending order, so "not paired by a facet" is known when a cell is seen. */
static void gradient_rules(const grid_t *g, const float *f, i64 *pr)
{
    pairing_init(g, pr);
    for (int d = 0; d < g->dim; d++) {
        /* cells of dimension d decide independently: each reads pr of its own (set by the
         * pass of dimension d - 1) and writes pr of itself and of one cofacet, which no other
         * cell of dimension d takes (the pairs form a matching) */
#pragma omp parallel for schedule(dynamic, 4096)
        for (i64 id = 0; id < g->n * g->K; id++) {
            if (cell_dim(g, id) != d || pr[id] != -1) continue;
            i64 v[5], nb[26];
            int nv = cell_verts(g, id, v);
            i64 lo = lowest_vertex(g, id, f), best = -1;
            int nn = neighbours(g, v[0], nb);
            for (int i = 0; i < nn; i++) {
                i64 w = nb[i];
                int ok = sos_lt(f, w, lo);
                for (int j = 0; j < nv && ok; j++) if (w == v[j] || !adjacent(g, w, v[j])) ok = 0;
                if (!ok) continue;
                v[nv] = w;
                if (cell_id(g, v, nv + 1) < 0) continue;
                if (best < 0 || sos_lt(f, w, best)) best = w;
            }
            if (best >= 0) {
                v[nv] = best;
                i64 c = cell_id(g, v, nv + 1);
                pr[id] = c;
                pr[c] = id;
            }
        }
    }
}

/* Eq. 1 read lexicographically: F(cell) is the list of its vertices sorted descending in
 * SoS order; cells of equal dimension compare by that list, first difference decides. */
static void sorted_desc(const grid_t *g, const float *f, i64 id, i64 v[4], int *nv)
{
    *nv = cell_verts(g, id, v);
    for (int i = 1; i < *nv; i++)
        for (int j = i; j > 0 && sos_lt(f, v[j - 1], v[j]); j--) { i64 t = v[j]; v[j] = v[j - 1]; v[j - 1] = t; }
}

static int cmp_ext(const grid_t *g, const float *f, i64 a, i64 b)
{
    i64 va[4], vb[4];
    int na, nb;
    sorted_desc(g, f, a, va, &na);
    sorted_desc(g, f, b, vb, &nb);
    for (int i = 0; i < na; i++)
        if (va[i] != vb[i]) return sos_lt(f, va[i], vb[i]) ? -1 : 1;
    return 0;
}

static i64 highest_facet(const grid_t *g, const float *f, i64 beta)
{
    i64 fc[4];
    int n = facets(g, beta, fc);
    i64 best = fc[0];
    for (int i = 1; i < n; i++) if (cmp_ext(g, f, fc[i], best) > 0) best = fc[i];
    return best;
}

/* Sec. 3.1: P_alpha = cofacets beta whose highest facet under F is alpha; alpha pairs with
 * the member of P_alpha of smallest F, unless alpha was already paired with a facet. */
static void gradient_brute(const grid_t *g, const float *f, i64 *pr)
{
    pairing_init(g, pr);
    for (int d = 0; d < g->dim; d++) {
        for (i64 id = 0; id < g->n * g->K; id++) {
            if (cell_dim(g, id) != d || pr[id] != -1) continue;
            i64 cf[16], best = -1;
            int n = cofacets(g, id, cf);
            for (int i = 0; i < n; i++) {
                if (highest_facet(g, f, cf[i]) != id) continue;
                if (best < 0 || cmp_ext(g, f, cf[i], best) < 0) best = cf[i];
            }
            if (best >= 0) { pr[id] = best; pr[best] = id; }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* separatrix traces (Sec. 3.1 gradient paths, Sec. 4.4)                      */
/* ------------------------------------------------------------------------- */

typedef struct { i64 *L, *U; i64 n, cap; } pathbuf;

static int pb_push(pathbuf *b, i64 L, i64 U)
{
    if (b->n == b->cap) {
        i64 nc = b->cap ? 2 * b->cap : 64;
        i64 *nl = realloc(b->L, nc * sizeof(i64)), *nu;
        if (!nl) return -1;
        b->L = nl;
        nu = realloc(b->U, nc * sizeof(i64));
        if (!nu) return -1;
        b->U = nu;
        b->cap = nc;
    }
    b->L[b->n] = L; b->U[b->n] = U; b->n++;
    return 0;
}

/* descending V-path from vertex u: u -> partner edge -> its other vertex -> ... until a
 * critical vertex (minimum).  Returns the terminal vertex's cell id, -3 on a cycle. */
static i64 trace_desc(const grid_t *g, const i64 *pr, i64 u, pathbuf *out)
{
    for (i64 step = 0; step <= g->n; step++) {
        i64 vc = u * g->K, e = pr[vc];
        if (e == -1) return vc;
        if (out && pb_push(out, vc, e)) return -4;
        i64 ev[4];
        cell_verts(g, e, ev);
        u = ev[0] == u ? ev[1] : ev[0];
    }
    return -3;
}

/* ascending V-path from (D-1)-saddle s through its top-dimensional cofacet beta: at a top
 * cell that is critical the path ends (maximum); otherwise the top cell is paired with a
 * facet alpha, and the path crosses alpha into alpha's other top cofacet.  A facet with a
 * single cofacet ends the path on the domain boundary (terminal = that facet). */
static i64 trace_asc(const grid_t *g, const i64 *pr, i64 beta, pathbuf *out)
{
    for (i64 step = 0; step <= g->n * g->K; step++) {
        i64 a = pr[beta];
        if (a == -1) return beta;
        if (out && pb_push(out, a, beta)) return -4;
        i64 cf[16], next = -1;
        int n = cofacets(g, a, cf);
        for (int i = 0; i < n; i++) if (cf[i] != beta) next = cf[i];
        if (next < 0) return a;
        beta = next;
    }
    return -3;
}

/* ------------------------------------------------------------------------- */
/* fix-loop state                                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    const grid_t *g;
    const float *f, *fhat;
    float *gv;
    uint8_t *state;
    i64 *prf, *prg;
    uint8_t *markT, *markX;
    int exact_fallback;
    i64 ncase, nlive;
    /* optional record of (target, case cell) for the case tests */
    i64 *rec; i64 rec_cap, rec_n;
    /* optional record of the saddle-saddle walk, rows (2-saddle, kind, edge, other):
     * kind 0 = 1-saddle edge reached, 1 = pair (edge, other triangle) crossed,
     * 2 = dead-end edge paired down with vertex other */
    i64 *walk; i64 walk_cap, walk_n;
} loopctx;

static void walk_note(loopctx *c, i64 t0, i64 kind, i64 e, i64 other)
{
    if (!c->walk) return;
    if (c->walk_n < c->walk_cap) {
        i64 *r = c->walk + 4 * c->walk_n;
        r[0] = t0; r[1] = kind; r[2] = e; r[3] = other;
    }
    c->walk_n++;
}

static int stuck(const loopctx *c, i64 t) { return c->state[t] == ST_FLOOR || c->state[t] == ST_EXACT; }

/* one false case: lower vertex t (set semantics, Sec. 4.8.3 read as "each vertex edited at
 * most once per iteration"); a stuck case restores the closed 1-rings of its cell to f. */
static void set_mark(uint8_t *m, i64 i)
{
#pragma omp atomic write
    m[i] = 1;
}

static void add_case(loopctx *c, i64 t, i64 case_cell)
{
    set_mark(c->markT, t);
#pragma omp atomic
    c->ncase++;
    if (c->rec && c->rec_n < c->rec_cap) {
        c->rec[2 * c->rec_n] = t;
        c->rec[2 * c->rec_n + 1] = case_cell;
        c->rec_n++;
    }
    if (!stuck(c, t)) {
#pragma omp atomic
        c->nlive++;
        return;
    }
    if (!c->exact_fallback) return;
    i64 v[4], nb[26];
    int nv = cell_verts(c->g, case_cell, v);
    for (int i = 0; i < nv; i++) {
        set_mark(c->markX, v[i]);
        int nn = neighbours(c->g, v[i], nb);
        for (int j = 0; j < nn; j++) set_mark(c->markX, nb[j]);
    }
}

/* Sec. 4.3: every cell whose criticality differs between V_f and V_g is a false case.
 * False positive (paired in f as (L,U), critical in g): lower U \ L, the extra vertex of
 * the f-partner (FPmin: j; FP1saddle: j or l; FP2saddle: k or l; FPmax: j or l).
 * False negative (critical in f, paired in g): lower the cell's lowest vertex in f
 * (FNmin: i; FN1saddle: i or j; FN2saddle: i, j or k; FNmax: i, j or k); when the cell is
 * paired down in g with its g-highest facet L and its f-lowest vertex is already the
 * g-lowest, the f-pairing of L is repaired instead.  Tier 1 looks at extrema only. */
static void c_targets(loopctx *c, int tier)
{
    const grid_t *g = c->g;
#pragma omp parallel for schedule(dynamic, 4096) if (!c->rec)
    for (i64 id = 0; id < g->n * g->K; id++) {
        if (c->prf[id] == -2) continue;
        int d = cell_dim(g, id);
        if (tier == 1 && d != 0 && d != g->dim) continue;
        int cf = c->prf[id] == -1, cg = c->prg[id] == -1;
        if (cf == cg) continue;
        i64 t;
        if (!cf) {
            i64 P = c->prf[id];
            t = cell_dim(g, P) > d ? extra_vertex(g, P, id) : extra_vertex(g, id, P);
        } else {
            i64 P = c->prg[id];
            if (cell_dim(g, P) > d) {
                t = lowest_vertex(g, id, c->f);
            } else {
                i64 y = extra_vertex(g, id, P), yf = lowest_vertex(g, id, c->f);
                if (y != yf) {
                    t = yf;
                } else {
                    i64 Q = c->prf[P];
                    if (Q == -1) t = lowest_vertex(g, P, c->f);
                    else if (cell_dim(g, Q) > cell_dim(g, P)) t = extra_vertex(g, Q, P);
                    else t = extra_vertex(g, P, Q);
                }
            }
        }
        add_case(c, t, id);
    }
}

/* one separatrix of f checked against V_g (Sec. 4.4).  T4: the first pair (L,U) of the
 * f-path that is not a pair of V_g is the troublemaker; lower U \ L.  T3: only when the
 * g-trace from the same start ends elsewhere than the f-trace. */
static int check_path(loopctx *c, int tier, const pathbuf *p, i64 fterm, i64 gterm)
{
    if (tier == 3 && fterm == gterm) return 0;
    for (i64 k = 0; k < p->n; k++) {
        if (c->prg[p->L[k]] != p->U[k]) {
            add_case(c, extra_vertex(c->g, p->U[k], p->L[k]), p->U[k]);
            return 1;
        }
    }
    return 0;
}

/* Saddle-saddle connectors (3D): from 2-saddle t0, walk the f-gradient over triangles
 * through their facet edges.  An examined edge is a 1-saddle (end), paired down in f (dead
 * end), or paired up with a triangle t' (continue into t').  Only pairs also present in
 * V_g are crossed; the first disagreeing pairs reached are the troublemakers.  A dead-end
 * edge that V_g pairs upward is repaired through its f-pair (v, e).  Returns the number of
 * troublemakers found. */
typedef struct { i64 *v; i64 cap; } i64queue;

/* make room for entries [0, need) of a growable queue; -1 when out of memory */
static int q_reserve(i64queue *q, i64 need)
{
    if (need <= q->cap) return 0;
    i64 nc = q->cap ? q->cap : 1024;
    while (nc < need) nc *= 2;
    i64 *nv = realloc(q->v, nc * sizeof(i64));
    if (!nv) return -1;
    q->v = nv;
    q->cap = nc;
    return 0;
}

static i64 saddle_saddle(loopctx *c, i64 t0, i64 *stamp, i64 stampval, i64queue *Q)
{
    const grid_t *g = c->g;
    i64 qh = 0, qt = 0, found = 0;
    if (q_reserve(Q, 2)) return -1;
    Q->v[qt] = t0; Q->v[qt + 1] = -1; qt += 2;
    stamp[t0] = stampval;
    while (qh < qt) {
        i64 t = Q->v[qh], entry = Q->v[qh + 1];
        qh += 2;
        i64 fc[4];
        int n = facets(g, t, fc);
        for (int i = 0; i < n; i++) {
            i64 e = fc[i];
            if (e == entry) continue;
            i64 pe = c->prf[e];
            if (pe == -1) { walk_note(c, t0, 0, e, -1); continue; }
            if (cell_dim(g, pe) == 0) {
                walk_note(c, t0, 2, e, pe);
                i64 q = c->prg[e];
                if (q == -1 || cell_dim(g, q) != 0) {
                    add_case(c, extra_vertex(g, e, pe), e);
                    found++;
                }
                continue;
            }
            if (pe == t) continue;
            walk_note(c, t0, 1, e, pe);
            if (c->prg[e] != pe) {
                add_case(c, extra_vertex(g, pe, e), pe);
                found++;
                continue;
            }
            if (stamp[pe] != stampval) {
                stamp[pe] = stampval;
                if (q_reserve(Q, qt + 2)) return -1;
                Q->v[qt] = pe; Q->v[qt + 1] = e; qt += 2;
            }
        }
    }
    return found;
}

static void report_add(i64 *report, int k, i64 v)
{
    if (!report || !v) return;
#pragma omp atomic
    report[k] += v;
}

static int s_targets(loopctx *c, int tier, i64 *report)
{
    const grid_t *g = c->g;
    i64 ncell = g->n * g->K;
    int err = ORC_OK;
    const int serial = c->rec != NULL;   /* the recorded case list keeps the serial order */
    /* descending separatrices of every 1-saddle edge, one per endpoint */
#pragma omp parallel if (!serial)
    {
        pathbuf pb = {0};
#pragma omp for schedule(dynamic, 256)
        for (i64 id = 0; id < ncell; id++) {
            if (cell_dim(g, id) != 1 || c->prf[id] != -1) continue;
            i64 v[4];
            cell_verts(g, id, v);
            for (int s = 0; s < 2; s++) {
                pb.n = 0;
                i64 ft = trace_desc(g, c->prf, v[s], &pb);
                i64 gt = trace_desc(g, c->prg, v[s], NULL);
                if (ft < -1 || gt < -1) {
#pragma omp atomic write
                    err = ORC_ERR_INTERNAL;
                    continue;
                }
                int bad = check_path(c, tier, &pb, ft, gt);
                report_add(report, 0, bad);
                report_add(report, 3, ft != gt);
            }
        }
        /* ascending separatrices of every (D-1)-saddle, one per top-dimensional cofacet */
#pragma omp for schedule(dynamic, 256)
        for (i64 id = 0; id < ncell; id++) {
            if (cell_dim(g, id) != g->dim - 1 || c->prf[id] != -1) continue;
            i64 cf[16];
            int n = cofacets(g, id, cf);
            for (int i = 0; i < n; i++) {
                pb.n = 0;
                i64 ft = trace_asc(g, c->prf, cf[i], &pb);
                i64 gt = trace_asc(g, c->prg, cf[i], NULL);
                if (ft < -1 || gt < -1) {
#pragma omp atomic write
                    err = ORC_ERR_INTERNAL;
                    continue;
                }
                int bad = check_path(c, tier, &pb, ft, gt);
                report_add(report, 1, bad);
                report_add(report, 4, ft != gt);
            }
        }
        free(pb.L); free(pb.U);
    }
    if (err) return err;
    if (g->dim == 3 && tier >= 4) {
        /* each 2-saddle walks with its own visited marks: one stamp array per thread,
         * stamped with the 2-saddle's id */
#pragma omp parallel if (!serial && !c->walk)
        {
            i64 *stamp = malloc(ncell * sizeof(i64));
            i64queue q = {0};
            if (!stamp) {
#pragma omp atomic write
                err = ORC_ERR_OOM;
            } else {
                for (i64 i = 0; i < ncell; i++) stamp[i] = -1;
            }
#pragma omp for schedule(dynamic, 64)
            for (i64 id = 0; id < ncell; id++) {
                if (!stamp || cell_dim(g, id) != 2 || c->prf[id] != -1) continue;
                i64 found = saddle_saddle(c, id, stamp, id, &q);
                if (found < 0) {
#pragma omp atomic write
                    err = ORC_ERR_OOM;
                    continue;
                }
                report_add(report, 2, found > 0);
            }
            free(stamp); free(q.v);
        }
    }
    return err;
}

/* ------------------------------------------------------------------------- */
/* edit arithmetic (Eq. 2)                                                    */
/* ------------------------------------------------------------------------- */

/* a - b rounded toward +inf, from the round-to-nearest difference and its exact error
 * (Knuth's TwoSum); used so that lb = f - xi never lies below the exact f - xi. */
static float sub_round_up(float a, float b)
{
    volatile float s = a - b;
    volatile float bb = s - a;
    volatile float e1 = s - bb;
    volatile float e2 = a - e1;
    volatile float e3 = -b - bb;
    float err = e2 + e3;
    if (err > 0.0f) return nextafterf(s, INFINITY);
    return s;
}

/* a + b rounded toward -inf (same construction) */
static float add_round_down(float a, float b)
{
    volatile float s = a + b;
    volatile float bb = s - a;
    volatile float e1 = s - bb;
    volatile float e2 = a - e1;
    volatile float e3 = b - bb;
    float err = e2 + e3;
    if (err < 0.0f) return nextafterf(s, -INFINITY);
    /* an exact zero sum is -0 under rounding toward -inf unless both operands are +0 */
    if (s == 0.0f && !(a == 0.0f && b == 0.0f && !signbit(a) && !signbit(b))) return -0.0f;
    return s;
}

static float lower_bound(float f, float xi) { return sub_round_up(f, xi); }
static float upper_bound(float f, float xi) { return add_round_down(f, xi); }

/* the base compressor's value re-clamped into [lb, ub] */
static float clamped_base(float f, float fhat, float xi)
{
    float lb = lower_bound(f, xi), ub = upper_bound(f, xi);
    return fhat < lb ? lb : (fhat > ub ? ub : fhat);
}

/* quantised value after q steps of xi / 2^qmax (Sec. 4.7: delta = q * xi / 2^qmax),
 * evaluated as one subtraction from the clamped base so it can be rebuilt exactly */
static float quant_value(float fc, int q, float step)
{
    volatile float t = (float)q * step;
    volatile float r = fc - t;
    return r;
}

/* Eq. 2: one more quantised step while q < qmax and the result stays >= f - xi,
 * otherwise snap to the floor f - xi.  Floating edits (Sec. 4.7, the form the paper
 * compares against): every edit is stored as a float, so the count q needs no bound; the
 * same steps continue until the next one would pass f - xi (qcap = QCAP_FLOAT, more steps
 * than fit between f + xi and f - xi). */
#define QCAP_FLOAT 0xEF

static int apply_edits(loopctx *c, float xi, int qmax, int qcap)
{
    const grid_t *g = c->g;
    float step = xi / (float)(1 << qmax);
    int changed = 0;
    for (i64 v = 0; v < g->n; v++) {
        if (c->markX[v]) {
            if (c->state[v] != ST_EXACT) { c->gv[v] = c->f[v]; c->state[v] = ST_EXACT; changed++; }
            continue;
        }
        if (!c->markT[v] || c->state[v] > qcap) continue;
        int q = c->state[v];
        float lb = lower_bound(c->f[v], xi);
        float fc = clamped_base(c->f[v], c->fhat[v], xi);
        if (q < qcap) {
            float cand = quant_value(fc, q + 1, step);
            if (cand >= lb) { c->gv[v] = cand; c->state[v] = (uint8_t)(q + 1); changed++; continue; }
        }
        c->gv[v] = lb;
        c->state[v] = ST_FLOOR;
        changed++;
    }
    return changed;
}

/* ------------------------------------------------------------------------- */
/* exported entry points                                                      */
/* ------------------------------------------------------------------------- */

static int valid_field(const float *a, i64 n)
{
    for (i64 i = 0; i < n; i++) if (!isfinite(a[i])) return 0;
    return 1;
}

static void write_cell(const grid_t *g, i64 id, int64_t *out)
{
    i64 v[4];
    int nv = cell_verts(g, id, v);
    for (int i = 0; i < 4; i++) out[i] = i < nv ? v[i] : -1;
}

/* all pairs (L, U) of the discrete gradient of a field, rows of 8 vertex ids
 * (L ascending, -1 padded; then U).  brute != 0 uses the Eq. 1 evaluation. */
int orc_gradient_pairs(const float *field, int nx, int ny, int nz, int brute,
                       int64_t *out, int64_t cap, int64_t *n_out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz) || !valid_field(field, (i64)nx * ny * nz)) return ORC_ERR_ARG;
    i64 ncell = g.n * g.K, n = 0;
    i64 *pr = malloc(ncell * sizeof(i64));
    if (!pr) return ORC_ERR_OOM;
    if (brute) gradient_brute(&g, field, pr); else gradient_rules(&g, field, pr);
    for (i64 id = 0; id < ncell; id++) {
        if (pr[id] < 0 || cell_dim(&g, pr[id]) < cell_dim(&g, id)) continue;
        if (n < cap) { write_cell(&g, id, out + 8 * n); write_cell(&g, pr[id], out + 8 * n + 4); }
        n++;
    }
    free(pr);
    *n_out = n;
    return ORC_OK;
}

/* critical cells: rows of 4 vertex ids (-1 padded), dimension in out_dim */
int orc_critical_cells(const float *field, int nx, int ny, int nz,
                       int64_t *out, int32_t *out_dim, int64_t cap, int64_t *n_out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz) || !valid_field(field, (i64)nx * ny * nz)) return ORC_ERR_ARG;
    i64 ncell = g.n * g.K, n = 0;
    i64 *pr = malloc(ncell * sizeof(i64));
    if (!pr) return ORC_ERR_OOM;
    gradient_rules(&g, field, pr);
    for (i64 id = 0; id < ncell; id++) {
        if (pr[id] != -1) continue;
        if (n < cap) { write_cell(&g, id, out + 4 * n); out_dim[n] = cell_dim(&g, id); }
        n++;
    }
    free(pr);
    *n_out = n;
    return ORC_OK;
}

/* all cells of the complex (rows of 4 ids) -- used to pin the cell enumeration */
int orc_cells(int nx, int ny, int nz, int64_t *out, int64_t cap, int64_t *n_out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz)) return ORC_ERR_ARG;
    i64 n = 0;
    for (i64 id = 0; id < g.n * g.K; id++) {
        if (!cell_exists(&g, id)) continue;
        if (n < cap) write_cell(&g, id, out + 4 * n);
        n++;
    }
    *n_out = n;
    return ORC_OK;
}

/* separatrices of a field: kind 0 = descending (from 1-saddles, one row per endpoint),
 * kind 1 = ascending (from (D-1)-saddles, one row per top cofacet).  Row layout (14):
 * saddle cell (4 ids), start cell (4 ids), path length, terminal cell (4 ids), terminal dim. */
int orc_separatrices(const float *field, int nx, int ny, int nz, int kind,
                     int64_t *out, int64_t cap, int64_t *n_out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz) || !valid_field(field, (i64)nx * ny * nz)) return ORC_ERR_ARG;
    i64 ncell = g.n * g.K, n = 0;
    i64 *pr = malloc(ncell * sizeof(i64));
    if (!pr) return ORC_ERR_OOM;
    gradient_rules(&g, field, pr);
    pathbuf pb = {0};
    for (i64 id = 0; id < ncell; id++) {
        if (pr[id] != -1) continue;
        int d = cell_dim(&g, id);
        i64 starts[16];
        int ns = 0;
        if (kind == 0 && d == 1) {
            i64 v[4];
            cell_verts(&g, id, v);
            starts[0] = v[0] * g.K; starts[1] = v[1] * g.K; ns = 2;
        } else if (kind == 1 && d == g.dim - 1) {
            ns = cofacets(&g, id, starts);
        }
        for (int s = 0; s < ns; s++) {
            pb.n = 0;
            i64 term = kind == 0 ? trace_desc(&g, pr, starts[s] / g.K, &pb) : trace_asc(&g, pr, starts[s], &pb);
            if (term < 0) { free(pr); free(pb.L); free(pb.U); return ORC_ERR_INTERNAL; }
            if (n < cap) {
                int64_t *r = out + 14 * n;
                write_cell(&g, id, r);
                write_cell(&g, starts[s], r + 4);
                r[8] = pb.n;
                write_cell(&g, term, r + 9);
                r[13] = cell_dim(&g, term);
            }
            n++;
        }
    }
    free(pr); free(pb.L); free(pb.U);
    *n_out = n;
    return ORC_OK;
}

/* The saddle-saddle walk of a 3D field's own gradient (Sec. 3.1, Sec. 4.4), as the S-pass
 * runs it with V_g = V_f: one row of 13 per item examined from each 2-saddle,
 * (2-saddle 4 ids, kind, edge 4 ids, other 4 ids) with kind 0 = 1-saddle edge reached
 * (other -1), 1 = pair (edge, other triangle) crossed, 2 = dead-end edge paired down with
 * vertex other.  Items reached along several routes appear once per route examined. */
int orc_saddle_connectors(const float *field, int nx, int ny, int nz, int64_t *out, int64_t cap, int64_t *n_out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz) || g.dim != 3 || !valid_field(field, (i64)nx * ny * nz)) return ORC_ERR_ARG;
    i64 ncell = g.n * g.K;
    loopctx c = {0};
    c.g = &g; c.f = field; c.gv = (float *)field;
    c.prf = malloc(ncell * sizeof(i64));
    c.markT = calloc(g.n, 1);
    c.markX = calloc(g.n, 1);
    c.state = calloc(g.n, 1);
    c.walk = malloc(4 * (cap > 0 ? cap : 1) * sizeof(i64));
    c.walk_cap = cap;
    i64 *stamp = malloc(ncell * sizeof(i64));
    i64queue q = {0};
    int rc = ORC_OK;
    if (!c.prf || !c.markT || !c.markX || !c.state || !c.walk || !stamp) { rc = ORC_ERR_OOM; goto done; }
    gradient_rules(&g, field, c.prf);
    c.prg = c.prf;
    for (i64 i = 0; i < ncell; i++) stamp[i] = -1;
    for (i64 id = 0; id < ncell; id++) {
        if (cell_dim(&g, id) != 2 || c.prf[id] != -1) continue;
        if (saddle_saddle(&c, id, stamp, id, &q) != 0) { rc = ORC_ERR_INTERNAL; goto done; }
    }
    for (i64 i = 0; i < c.walk_n && i < cap; i++) {
        const i64 *r = c.walk + 4 * i;
        int64_t *o = out + 13 * i;
        write_cell(&g, r[0], o);
        o[4] = r[1];
        write_cell(&g, r[2], o + 5);
        if (r[3] >= 0) write_cell(&g, r[3], o + 9);
        else for (int k = 0; k < 4; k++) o[9 + k] = -1;
    }
    *n_out = c.walk_n;
done:
    free(c.prf); free(c.markT); free(c.markX); free(c.state); free(c.walk); free(stamp); free(q.v);
    return rc;
}

/* One targeting pass on (f, g, state): pass 0 = C-pass, 1 = S-pass.  Writes the case list
 * as rows (target vertex, case cell 4 ids) and returns the counts; used by the tests that
 * pin each false-case rule on a hand-built field. */
int orc_targets(const float *f, const float *gfield, const uint8_t *state_in,
                int nx, int ny, int nz, int pass, int tier, int exact_fallback,
                int64_t *out, int64_t cap, int64_t *n_out, uint8_t *markX_out)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz)) return ORC_ERR_ARG;
    i64 ncell = g.n * g.K;
    loopctx c = {0};
    c.g = &g; c.f = f; c.gv = (float *)gfield;
    c.state = (uint8_t *)state_in;
    c.exact_fallback = exact_fallback;
    c.prf = malloc(ncell * sizeof(i64));
    c.prg = malloc(ncell * sizeof(i64));
    c.markT = calloc(g.n, 1);
    c.markX = calloc(g.n, 1);
    c.rec = malloc(2 * (cap > 0 ? cap : 1) * sizeof(i64));
    c.rec_cap = cap;
    int rc = ORC_OK;
    if (!c.prf || !c.prg || !c.markT || !c.markX || !c.rec) { rc = ORC_ERR_OOM; goto done; }
    gradient_rules(&g, f, c.prf);
    gradient_rules(&g, gfield, c.prg);
    if (pass == 0) c_targets(&c, tier);
    else rc = s_targets(&c, tier, NULL);
    for (i64 i = 0; i < c.rec_n; i++) {
        out[5 * i] = c.rec[2 * i];
        write_cell(&g, c.rec[2 * i + 1], out + 5 * i + 1);
    }
    *n_out = c.ncase;
    if (markX_out) memcpy(markX_out, c.markX, g.n);
done:
    free(c.prf); free(c.prg); free(c.markT); free(c.markX); free(c.rec);
    return rc;
}

/* The whole fix loop (Sec. 4.2-4.7).  edit_mode 0: quantised edits (Eq. 2); 1: floating
 * edits (no cap on the step count, Sec. 4.7).  Outputs: g, per-vertex state (the step count
 * q, 0xF0 floor, 0xF1 exact), counts, and one trace row per iteration:
 * (kind 0=C/1=S, |T|, |X|, sum of T ids, sum of X ids, number of cases). */
int orc_fix(const float *f, const float *fhat, int nx, int ny, int nz, float xi,
            int tier, int qmax, int max_iters, int exact_fallback, int edit_mode,
            float *g_out, uint8_t *state_out, int32_t *counts /* n_c, n_s, n_exact_iters */,
            int64_t *trace, int64_t trace_cap, int64_t *n_trace)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz)) return ORC_ERR_ARG;
    if (!(xi > 0.0f) || !isfinite(xi) || qmax < 1 || qmax > 7 || tier < 1 || tier > 4) return ORC_ERR_ARG;
    if (edit_mode < 0 || edit_mode > 1 || (edit_mode == 1 && qmax > 6)) return ORC_ERR_ARG;
    const int qcap = edit_mode == 1 ? QCAP_FLOAT : qmax;
    if (!valid_field(f, g.n) || !valid_field(fhat, g.n)) return ORC_ERR_ARG;
    i64 ncell = g.n * g.K;
    loopctx c = {0};
    c.g = &g; c.f = f; c.fhat = fhat; c.gv = g_out; c.state = state_out;
    c.exact_fallback = exact_fallback;
    c.prf = malloc(ncell * sizeof(i64));
    c.prg = malloc(ncell * sizeof(i64));
    c.markT = malloc(g.n);
    c.markX = malloc(g.n);
    int rc = ORC_OK;
    if (!c.prf || !c.prg || !c.markT || !c.markX) { rc = ORC_ERR_OOM; goto done; }

    /* initial field: the decompressed values re-clamped into the error bound */
    for (i64 v = 0; v < g.n; v++) { g_out[v] = clamped_base(f[v], fhat[v], xi); state_out[v] = 0; }
    gradient_rules(&g, f, c.prf);
    counts[0] = counts[1] = counts[2] = 0;
    *n_trace = 0;

    for (;;) {
        gradient_rules(&g, g_out, c.prg);
        memset(c.markT, 0, g.n);
        memset(c.markX, 0, g.n);
        c.ncase = c.nlive = 0;
        int kind = 0;
        c_targets(&c, tier);
        if (c.ncase == 0) {
            if (tier < 3) break;
            kind = 1;
            rc = s_targets(&c, tier, NULL);
            if (rc) goto done;
            if (c.ncase == 0) break;
        }
        if (!exact_fallback && c.nlive == 0) { rc = ORC_ERR_STALLED; goto done; }
        if (counts[0] + counts[1] >= max_iters) { rc = ORC_ERR_NOT_CONVERGED; goto done; }
        i64 nT = 0, nX = 0, sT = 0, sX = 0;
        for (i64 v = 0; v < g.n; v++) {
            if (c.markT[v]) { nT++; sT += v; }
            if (c.markX[v]) { nX++; sX += v; }
        }
        apply_edits(&c, xi, qmax, qcap);
        counts[kind]++;
        if (nX) counts[2]++;
        if (*n_trace < trace_cap) {
            int64_t *r = trace + 6 * *n_trace;
            r[0] = kind; r[1] = nT; r[2] = nX; r[3] = sT; r[4] = sX; r[5] = c.ncase;
        }
        (*n_trace)++;
    }
done:
    free(c.prf); free(c.prg); free(c.markT); free(c.markX);
    return rc;
}

/* Compare the MSC of g with that of f (Sec. 5.1 metrics).  report[13]:
 * [0..3] false positives by dimension, [4..7] false negatives by dimension,
 * [8] descending separatrices with a pair missing from V_g, [9] ascending ditto,
 * [10] 2-saddles whose saddle-saddle connectors differ,
 * [11] descending terminal mismatches, [12] ascending terminal mismatches.
 * Separatrix entries are computed only when the critical cells agree. */
int orc_verify(const float *f, const float *gfield, int nx, int ny, int nz,
               int64_t *report, double *max_abs_err)
{
    grid_t g;
    if (grid_init(&g, nx, ny, nz)) return ORC_ERR_ARG;
    if (!valid_field(f, g.n) || !valid_field(gfield, g.n)) return ORC_ERR_ARG;
    i64 ncell = g.n * g.K;
    loopctx c = {0};
    c.g = &g; c.f = f; c.gv = (float *)gfield;
    c.prf = malloc(ncell * sizeof(i64));
    c.prg = malloc(ncell * sizeof(i64));
    c.markT = calloc(g.n, 1);
    c.markX = calloc(g.n, 1);
    c.state = calloc(g.n, 1);
    int rc = ORC_OK;
    if (!c.prf || !c.prg || !c.markT || !c.markX || !c.state) { rc = ORC_ERR_OOM; goto done; }
    gradient_rules(&g, f, c.prf);
    gradient_rules(&g, gfield, c.prg);
    for (int i = 0; i < 13; i++) report[i] = 0;
    i64 crit_bad = 0;
    for (i64 id = 0; id < ncell; id++) {
        if (c.prf[id] == -2) continue;
        int d = cell_dim(&g, id);
        int cf = c.prf[id] == -1, cg = c.prg[id] == -1;
        if (cg && !cf) { report[d]++; crit_bad++; }
        if (cf && !cg) { report[4 + d]++; crit_bad++; }
    }
    if (crit_bad == 0) {
        i64 sep[5] = {0, 0, 0, 0, 0};
        rc = s_targets(&c, 4, sep);
        report[8] = sep[0]; report[9] = sep[1]; report[10] = sep[2];
        report[11] = sep[3]; report[12] = sep[4];
    }
    double m = 0.0;
    for (i64 v = 0; v < g.n; v++) {
        double e = fabs((double)gfield[v] - (double)f[v]);
        if (e > m) m = e;
    }
    *max_abs_err = m;
done:
    free(c.prf); free(c.prg); free(c.markT); free(c.markX); free(c.state);
    return rc;
}

/* edit arithmetic exposed for the closed-form pins: lb, ub, clamped base and the value
 * after q quantised steps, for each input */
int orc_edit_values(const float *f, const float *fhat, int64_t n, float xi, int qmax, int nq,
                    float *lb, float *ub, float *fc, float *qvals /* n x nq: q = 0 .. nq-1 */)
{
    if (!(xi > 0.0f) || qmax < 1 || qmax > 7 || nq < 1 || nq > 256) return ORC_ERR_ARG;
    float step = xi / (float)(1 << qmax);
    for (i64 i = 0; i < n; i++) {
        lb[i] = lower_bound(f[i], xi);
        ub[i] = upper_bound(f[i], xi);
        fc[i] = clamped_base(f[i], fhat[i], xi);
        for (int q = 0; q < nq; q++) qvals[i * nq + q] = quant_value(fc[i], q, step);
    }
    return ORC_OK;
}

/* decompression side (Sec. 3.2 / 4.7): g = fhat - q * xi / 2^qmax for quantised vertices,
 * the stored value for lossless ones (q_map == 0xFF) */
int orc_apply_edits(const float *fhat, int64_t n, float xi, int qmax, const uint8_t *q_map,
                    const int64_t *lossless_idx, const float *lossless_val, int64_t n_lossless,
                    float *g_out)
{
    if (!(xi > 0.0f) || qmax < 1 || qmax > 7) return ORC_ERR_ARG;
    float step = xi / (float)(1 << qmax);
    for (i64 i = 0; i < n; i++) g_out[i] = q_map[i] == 0xFF ? fhat[i] : quant_value(fhat[i], q_map[i], step);
    for (i64 k = 0; k < n_lossless; k++) g_out[lossless_idx[k]] = lossless_val[k];
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* packed edit record (Sec. 4.7: quantised counts as a fixed-bit bitstream)    */
/* ------------------------------------------------------------------------- */
/* Layout, little-endian:
 *   32-byte header: "MSCE", version 1, q_max, b (bits per vertex), 0, n_vertices (u64),
 *                   n_lossless (u64), 0 (u64);
 *   the q-map, b bits per vertex, in groups of 8 vertices stored as b bytes each: vertex 8k+j
 *   of group k is the bit field [j*b, j*b + b) of that group's little-endian integer;
 *   a quantised count is stored as itself (0..q_max), a lossless vertex as 2^b - 1;
 *   b is the least number of bits that holds q_max + 2 distinct values;
 *   the lossless values (float32), one per lossless vertex, in increasing vertex order. */
static int pack_bits(int qmax)
{
    int b = 1;
    while ((1 << b) < qmax + 2) b++;
    return b;
}

int64_t orc_packed_bytes(int64_t n, int64_t n_lossless, int qmax)
{
    return 32 + ((n + 7) / 8) * pack_bits(qmax) + 4 * n_lossless;
}

static void put_u64(uint8_t *p, uint64_t v)
{
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}

static uint64_t get_u64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

int orc_pack_edits(const uint8_t *q_map, int64_t n, int qmax, const float *lossless_val, int64_t n_lossless,
                   uint8_t *out, int64_t cap, int64_t *n_out)
{
    if (qmax < 1 || qmax > 7 || n < 0 || n_lossless < 0) return ORC_ERR_ARG;
    int b = pack_bits(qmax);
    int64_t size = orc_packed_bytes(n, n_lossless, qmax);
    *n_out = size;
    if (cap < size) return ORC_ERR_ARG;
    memset(out, 0, (size_t)size);
    out[0] = 'M'; out[1] = 'S'; out[2] = 'C'; out[3] = 'E';
    out[4] = 1; out[5] = (uint8_t)qmax; out[6] = (uint8_t)b; out[7] = 0;
    put_u64(out + 8, (uint64_t)n);
    put_u64(out + 16, (uint64_t)n_lossless);
    uint8_t *bits = out + 32;
    int64_t seen = 0;
    for (int64_t v = 0; v < n; v++) {
        unsigned code;
        if (q_map[v] == 0xFF) { code = (1u << b) - 1; seen++; }
        else if (q_map[v] <= qmax) code = q_map[v];
        else return ORC_ERR_ARG;
        int64_t bit = (v / 8) * 8 * b + (v % 8) * b;     /* group k starts at bit 8*b*k */
        for (int i = 0; i < b; i++)
            if ((code >> i) & 1u) bits[(bit + i) / 8] |= (uint8_t)(1u << ((bit + i) % 8));
    }
    if (seen != n_lossless) return ORC_ERR_ARG;
    memcpy(bits + ((n + 7) / 8) * b, lossless_val, (size_t)n_lossless * 4);
    return ORC_OK;
}

/* header fields of a packed record; returns ORC_ERR_ARG if it is not one */
int orc_packed_header(const uint8_t *buf, int64_t size, int64_t *n, int64_t *n_lossless, int *qmax)
{
    if (size < 32 || memcmp(buf, "MSCE", 4) != 0 || buf[4] != 1) return ORC_ERR_ARG;
    *qmax = buf[5];
    *n = (int64_t)get_u64(buf + 8);
    *n_lossless = (int64_t)get_u64(buf + 16);
    if (*qmax < 1 || *qmax > 7 || buf[6] != pack_bits(*qmax)) return ORC_ERR_ARG;
    if (orc_packed_bytes(*n, *n_lossless, *qmax) != size) return ORC_ERR_ARG;
    return ORC_OK;
}

int orc_unpack_edits(const uint8_t *buf, int64_t size, uint8_t *q_map, int64_t *lossless_idx, float *lossless_val)
{
    int64_t n, nl;
    int qmax;
    if (orc_packed_header(buf, size, &n, &nl, &qmax) != ORC_OK) return ORC_ERR_ARG;
    int b = pack_bits(qmax);
    const uint8_t *bits = buf + 32;
    int64_t k = 0;
    for (int64_t v = 0; v < n; v++) {
        int64_t bit = (v / 8) * 8 * b + (v % 8) * b;
        unsigned code = 0;
        for (int i = 0; i < b; i++) code |= (unsigned)((bits[(bit + i) / 8] >> ((bit + i) % 8)) & 1u) << i;
        if (code == (1u << b) - 1) {
            if (k >= nl) return ORC_ERR_ARG;
            q_map[v] = 0xFF;
            lossless_idx[k++] = v;
        } else if ((int)code <= qmax) {
            q_map[v] = (uint8_t)code;
        } else {
            return ORC_ERR_ARG;
        }
    }
    if (k != nl) return ORC_ERR_ARG;
    memcpy(lossless_val, bits + ((n + 7) / 8) * b, (size_t)nl * 4);
    return ORC_OK;
}

/* threads used by the oracle's parallel loops: set (n >= 1) and query */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
