/*
 * oracle/sandwich.c -- the oracle of the sandwich's own steps, for the
 * variants whose result has no plainer definition.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  It
 * shares no code, header, table or helper with the CUDA path of the package.
 *
 * pairsimplices.c gives the diagrams by their plain definition, the standard
 * reduction.  Two variants depend on the method's own steps instead:
 *  - no virtual maximum on the outer boundary (Sec. 5.2, "Domains with
 *    boundary"; App. A): the D2 step no longer matches the standard
 *    reduction, and the 2-saddles it leaves unpaired change the D1 step;
 *  - persistent 1-cycle generators (Sec. 8): the cycle held by Boundary(sigma_j)
 *    when the homologous propagation of Alg. 3 stops at an unpaired edge.
 * So this file runs the steps themselves, one after the other, in the
 * paper's order, with nothing blocked, fused or reordered:
 *  1. Discrete gradient (Alg. 2, first step): every vertex lower star is
 *     expanded with ProcessLowerStars (Robins et al.; the paper cites it
 *     without pseudo-code).  G is the lexicographic key, so "smallest G" is
 *     the earliest filtration position; both priority queues are sets; a
 *     cell taken from a queue after it was classified is skipped; faces
 *     outside the lower star never count as unclassified.
 *  2. Zero-persistence skip (Alg. 2): a simplex in a gradient pair is paired
 *     with its partner; the others are critical, in lexicographic order.
 *  3. D0 (Sec. 5.1): for every critical edge in increasing order, the two
 *     descending v-paths from its vertices end at minima; union-find with
 *     the elder rule (a component is named by its lowest minimum; an edge
 *     joining two components kills the younger).
 *  4. D2 (Sec. 5.2): for every critical triangle in decreasing order, the
 *     ascending v-path on each side ends at a maximum, or leaves the domain
 *     through a boundary triangle.  With the virtual maximum, leaving the
 *     domain ends at one extra node older than every maximum.  Without it,
 *     a triangle with a side that leaves the domain merges nothing and is
 *     left to step 5 (the rest of the step unchanged, which is what the
 *     paper calls the option).  Union-find with the elder rule.
 *  5. D1 (Alg. 3, PairCriticalSimplices) over the critical triangles that
 *     step 4 left, in increasing order: Boundary starts as the three edges
 *     of the triangle; while it is not empty, its highest edge tau is
 *     taken; an unpaired critical tau ends the propagation and is paired
 *     with the triangle; otherwise the Boundary of tau's partner is added
 *     mod 2 (the three edges of a gradient partner; the stored final
 *     Boundary of a triangle paired before).  The final Boundary is the
 *     generator of the pair (Sec. 8).
 *  6. Infinite classes (Sec. 6): every critical simplex left unpaired.
 *
 * With the virtual maximum the result must equal oracle_pairsimplices: the
 * sandwich returns the diagrams of the standard reduction (Sec. 4.1 (c),
 * Sec. 5).  The tests check that equality, which pins steps 1-6.
 *
 * Result rows are 8 int64 each, as in pairsimplices.c:
 *   dim, birth_id, death_id (-1 if infinite), birth_vertex, death_vertex
 *   (-1 if infinite), infinite flag, birth_pos, death_pos (positions in the
 *   lexicographic filtration; -1 if infinite).
 * Generator records are flat int64: birth edge id, death triangle id, the
 * number k of edges, then the k edge ids in increasing filtration order.
 */
#include "complex.h"

#define OR_ERR_INTERNAL 4

/* ------------------------------------------------------------ the complex */

typedef struct {
    grid_t g;
    int64_t n, m;          /* vertices, simplices */
    simp_t *s;             /* every simplex, in lexicographic order */
    int64_t *pos[4];       /* simplex id -> position in s */
    int64_t *vert_of_rank;
    int64_t *facet;        /* 4 per position: positions of the facets */
    int64_t *side;         /* 2 per triangle position: its tets, -1 if none */
    int64_t *grad;         /* position -> gradient partner, -1 if critical */
} sw_t;

static void sw_free(sw_t *w)
{
    free(w->s);
    for (int d = 0; d < 4; d++) free(w->pos[d]);
    free(w->vert_of_rank); free(w->facet); free(w->side); free(w->grad);
}

static int sw_init(sw_t *w, int64_t nx, int64_t ny, int64_t nz, int dtype, const void *values)
{
    memset(w, 0, sizeof(*w));
    w->g.nx = nx; w->g.ny = ny; w->g.nz = nz;
    w->n = nx * ny * nz;
    int64_t n = w->n;
    int64_t *rank = malloc(sizeof(int64_t) * (size_t)n);
    if (!rank) return OR_ERR_MEM;
    int st = vertex_ranks(dtype, values, n, rank);
    if (!st) st = build_filtration(&w->g, rank, &w->s, &w->m);
    if (st) { free(rank); return st; }
    int64_t m = w->m;
    w->vert_of_rank = malloc(sizeof(int64_t) * (size_t)n);
    w->facet = malloc(sizeof(int64_t) * 4 * (size_t)m);
    w->side = malloc(sizeof(int64_t) * 2 * (size_t)m);
    w->grad = malloc(sizeof(int64_t) * (size_t)m);
    for (int d = 0; d < 4; d++) w->pos[d] = malloc(sizeof(int64_t) * (size_t)(n * ID_MULT[d]));
    if (!w->vert_of_rank || !w->facet || !w->side || !w->grad || !w->pos[0] || !w->pos[1] ||
        !w->pos[2] || !w->pos[3]) {
        free(rank);
        return OR_ERR_MEM;
    }
    for (int64_t v = 0; v < n; v++) w->vert_of_rank[rank[v]] = v;
    free(rank);
    for (int d = 0; d < 4; d++)
        for (int64_t i = 0; i < n * ID_MULT[d]; i++) w->pos[d][i] = -1;
    for (int64_t p = 0; p < m; p++) w->pos[w->s[p].dim][w->s[p].id] = p;
    for (int64_t p = 0; p < m; p++) {
        int dim = w->s[p].dim;
        int64_t vs[4], fv[3];
        w->side[2 * p] = w->side[2 * p + 1] = -1;
        w->grad[p] = -1;
        for (int i = 0; i < 4; i++) w->facet[4 * p + i] = -1;
        if (dim == 0) continue;
        simplex_vertices(&w->g, dim, w->s[p].id, vs);
        for (int drop = 0; drop <= dim; drop++) {
            int c = 0;
            for (int i = 0; i <= dim; i++) if (i != drop) fv[c++] = vs[i];
            w->facet[4 * p + drop] = w->pos[dim - 1][simplex_id(&w->g, dim - 1, fv)];
        }
    }
    for (int64_t p = 0; p < m; p++) {
        if (w->s[p].dim != 3) continue;
        for (int i = 0; i < 4; i++) {
            int64_t f = w->facet[4 * p + i];
            if (w->side[2 * f] < 0) w->side[2 * f] = p; else w->side[2 * f + 1] = p;
        }
    }
    return OR_OK;
}

/* --------------------------------------- step 1: ProcessLowerStars (Alg. 2) */

/* Number of facets of p inside the lower star [lo, hi) still unclassified;
 * *which receives one of them. */
static int unclassified_faces(const sw_t *w, const char *done, int64_t p, int64_t lo,
                              int64_t hi, int64_t *which)
{
    int k = 0;
    for (int i = 0; i <= w->s[p].dim && w->s[p].dim > 0; i++) {
        int64_t f = w->facet[4 * p + i];
        if (f >= lo && f < hi && !done[f]) { k++; *which = f; }
    }
    return k;
}

static int is_facet(const sw_t *w, int64_t f, int64_t p)
{
    for (int i = 0; i <= w->s[p].dim && w->s[p].dim > 0; i++)
        if (w->facet[4 * p + i] == f) return 1;
    return 0;
}

/* Adds to PQone the cofacets of c in [lo, hi) with exactly one unclassified
 * facet.  Queues are membership flags indexed by position - lo. */
static void push_cofacets(const sw_t *w, const char *done, char *pqone, int64_t c,
                          int64_t lo, int64_t hi)
{
    int64_t f;
    for (int64_t q = lo; q < hi; q++)
        if (!done[q] && w->s[q].dim == w->s[c].dim + 1 && is_facet(w, c, q) &&
            unclassified_faces(w, done, q, lo, hi, &f) == 1)
            pqone[q - lo] = 1;
}

static int64_t pop_min(char *pq, int64_t lo, int64_t hi)
{
    for (int64_t q = lo; q < hi; q++)
        if (pq[q - lo]) { pq[q - lo] = 0; return q; }
    return -1;
}

static void pair_cells(sw_t *w, char *done, int64_t a, int64_t b)
{
    w->grad[a] = b; w->grad[b] = a;
    done[a] = done[b] = 1;
}

/* The lower star of the vertex at position lo is the block [lo, hi) of
 * simplices whose highest vertex it is (contiguous in lexicographic order). */
static int process_lower_star(sw_t *w, char *done, int64_t lo, int64_t hi)
{
    char pqzero[80], pqone[80];
    if (hi - lo > 80 || w->s[lo].dim != 0) return OR_ERR_INTERNAL;
    memset(pqzero, 0, sizeof pqzero);
    memset(pqone, 0, sizeof pqone);
    if (hi - lo == 1) { done[lo] = 1; return OR_OK; }   /* a minimum */
    int64_t delta = -1, f;
    for (int64_t q = lo + 1; q < hi && delta < 0; q++) if (w->s[q].dim == 1) delta = q;
    if (delta < 0) return OR_ERR_INTERNAL;
    pair_cells(w, done, lo, delta);
    for (int64_t q = lo + 1; q < hi; q++) if (w->s[q].dim == 1 && q != delta) pqzero[q - lo] = 1;
    push_cofacets(w, done, pqone, delta, lo, hi);
    for (;;) {
        int64_t a;
        while ((a = pop_min(pqone, lo, hi)) >= 0) {
            if (done[a]) continue;
            if (unclassified_faces(w, done, a, lo, hi, &f) == 0) { pqzero[a - lo] = 1; continue; }
            pair_cells(w, done, f, a);
            pqzero[f - lo] = 0;
            push_cofacets(w, done, pqone, a, lo, hi);
            push_cofacets(w, done, pqone, f, lo, hi);
        }
        int64_t c = pop_min(pqzero, lo, hi);
        if (c < 0) break;
        if (done[c]) continue;
        done[c] = 1;                                  /* critical */
        push_cofacets(w, done, pqone, c, lo, hi);
    }
    for (int64_t q = lo; q < hi; q++) if (!done[q]) return OR_ERR_INTERNAL;
    return OR_OK;
}

static int discrete_gradient(sw_t *w)
{
    char *done = calloc((size_t)w->m, 1);
    if (!done) return OR_ERR_MEM;
    int st = OR_OK;
    for (int64_t lo = 0; lo < w->m && !st;) {
        int64_t hi = lo + 1;
        while (hi < w->m && w->s[hi].r[0] == w->s[lo].r[0]) hi++;
        st = process_lower_star(w, done, lo, hi);
        lo = hi;
    }
    free(done);
    return st;
}

/* ------------------------------------------------------------ v-paths */

/* Descending v-path from a vertex: through its gradient edge to the edge's
 * other vertex, until a critical vertex (a minimum). */
static int64_t descend(const sw_t *w, int64_t p)
{
    for (int64_t guard = 0; guard <= w->m; guard++) {
        int64_t e = w->grad[p];
        if (e < 0) return p;
        p = w->facet[4 * e] == p ? w->facet[4 * e + 1] : w->facet[4 * e];
    }
    return -1;
}

/* Ascending v-path from tet q: through its gradient triangle to the
 * triangle's other tet, until a critical tet (a maximum), or `outside`
 * when the triangle lies on the boundary. */
static int64_t ascend(const sw_t *w, int64_t q, int64_t outside)
{
    for (int64_t guard = 0; guard <= w->m; guard++) {
        int64_t t = w->grad[q];
        if (t < 0) return q;
        int64_t a = w->side[2 * t], b = w->side[2 * t + 1];
        q = a == q ? b : a;
        if (q < 0) return outside;
    }
    return -1;
}

/* ------------------------------------------------------------- the steps */

typedef struct {
    result_t rows;
    int64_t *gen; int64_t gen_n, gen_cap;
} out_t;

static int push_gen(out_t *o, int64_t v)
{
    if (o->gen_n == o->gen_cap) {
        int64_t nc = o->gen_cap ? 2 * o->gen_cap : 256;
        int64_t *ng = realloc(o->gen, sizeof(int64_t) * (size_t)nc);
        if (!ng) return OR_ERR_MEM;
        o->gen = ng; o->gen_cap = nc;
    }
    o->gen[o->gen_n++] = v;
    return OR_OK;
}

static int push_pair(const sw_t *w, out_t *o, int dim, int64_t b, int64_t d)
{
    int64_t row[8] = {dim, w->s[b].id, w->s[d].id, w->vert_of_rank[w->s[b].r[0]],
                      w->vert_of_rank[w->s[d].r[0]], 0, b, d};
    return push_row(&o->rows, row);
}

static int run(sw_t *w, int virtual_max, out_t *o)
{
    int64_t m = w->m;
    int st = discrete_gradient(w);
    if (st) return st;
    int64_t *partner = malloc(sizeof(int64_t) * (size_t)m);   /* persistence pair */
    int64_t *parent = malloc(sizeof(int64_t) * (size_t)(m + 1));
    col_t *cache = calloc((size_t)m, sizeof(col_t));
    col_t B = {0};
    int64_t *tmp = NULL, tmpcap = 0;
    if (!partner || !parent || !cache) { st = OR_ERR_MEM; goto done; }
    for (int64_t p = 0; p < m; p++) partner[p] = -1;

    /* step 3: D0 */
    for (int64_t p = 0; p <= m; p++) parent[p] = p;
    for (int64_t e = 0; e < m && !st; e++) {
        if (w->s[e].dim != 1 || w->grad[e] >= 0) continue;
        int64_t a = descend(w, w->facet[4 * e]), b = descend(w, w->facet[4 * e + 1]);
        if (a < 0 || b < 0) { st = OR_ERR_INTERNAL; break; }
        a = uf_find(parent, a); b = uf_find(parent, b);
        if (a == b) continue;
        int64_t young = a > b ? a : b, old = a > b ? b : a;
        parent[young] = old;
        partner[young] = e; partner[e] = young;
        st = push_pair(w, o, 0, young, e);
    }

    /* step 4: D2 (node m is the virtual maximum, older than every tet) */
    for (int64_t p = 0; p <= m; p++) parent[p] = p;
    for (int64_t t = m - 1; t >= 0 && !st; t--) {
        if (w->s[t].dim != 2 || w->grad[t] >= 0) continue;
        int64_t end[2];
        for (int i = 0; i < 2; i++) {
            int64_t q = w->side[2 * t + i];
            end[i] = q < 0 ? m : ascend(w, q, m);
        }
        if (end[0] < 0 || end[1] < 0) { st = OR_ERR_INTERNAL; break; }
        if (!virtual_max && (end[0] == m || end[1] == m)) continue;
        int64_t a = uf_find(parent, end[0]), b = uf_find(parent, end[1]);
        if (a == b) continue;
        int64_t young = a < b ? a : b, old = a < b ? b : a;
        parent[young] = old;
        partner[young] = t; partner[t] = young;
        st = push_pair(w, o, 2, t, young);
    }

    /* step 5: D1, Alg. 3 with homologous propagation */
    for (int64_t t = 0; t < m && !st; t++) {
        if (w->s[t].dim != 2 || w->grad[t] >= 0 || partner[t] >= 0) continue;
        int64_t edges[3] = {w->facet[4 * t], w->facet[4 * t + 1], w->facet[4 * t + 2]};
        qsort(edges, 3, sizeof(int64_t), cmp_i64);
        col_t F = {edges, 3, 3};
        B.n = 0;
        if ((st = col_xor(&B, &F, &tmp, &tmpcap))) break;
        int64_t tau = -1;
        for (int64_t guard = 0; B.n > 0; guard++) {
            if (guard > 64 * m + 1000000) { st = OR_ERR_INTERNAL; break; }
            tau = B.e[B.n - 1];
            if (w->grad[tau] < 0) {                       /* critical edge */
                int64_t q = partner[tau];
                if (q < 0) break;                         /* unpaired: a new cycle */
                if (w->s[q].dim != 2) { st = OR_ERR_INTERNAL; break; }
                st = col_xor(&B, &cache[q], &tmp, &tmpcap);
            } else {                                      /* gradient partner */
                int64_t q = w->grad[tau];
                if (w->s[q].dim != 2) { st = OR_ERR_INTERNAL; break; }
                int64_t fs[3] = {w->facet[4 * q], w->facet[4 * q + 1], w->facet[4 * q + 2]};
                qsort(fs, 3, sizeof(int64_t), cmp_i64);
                col_t G = {fs, 3, 3};
                st = col_xor(&B, &G, &tmp, &tmpcap);
            }
            if (st) break;
        }
        if (st || B.n == 0) continue;
        partner[tau] = t; partner[t] = tau;
        cache[t] = B;                                     /* keeps the storage */
        B = (col_t){0};
        if ((st = push_pair(w, o, 1, tau, t))) break;
        st = push_gen(o, w->s[tau].id);
        if (!st) st = push_gen(o, w->s[t].id);
        if (!st) st = push_gen(o, cache[t].n);
        for (int64_t i = 0; i < cache[t].n && !st; i++) st = push_gen(o, w->s[cache[t].e[i]].id);
    }

    /* step 6: infinite classes */
    for (int64_t p = 0; p < m && !st; p++) {
        if (w->grad[p] >= 0 || partner[p] >= 0) continue;
        int64_t row[8] = {w->s[p].dim, w->s[p].id, -1, w->vert_of_rank[w->s[p].r[0]], -1, 1,
                          p, -1};
        st = push_row(&o->rows, row);
    }

done:
    if (cache) for (int64_t p = 0; p < m; p++) free(cache[p].e);
    free(cache); free(B.e); free(tmp); free(partner); free(parent);
    return st;
}

/* The diagrams by the sandwich's steps.  virtual_max selects the option of
 * Sec. 5.2; *out_gen receives the generator records of the D1 pairs. */
int oracle_sandwich(int64_t nx, int64_t ny, int64_t nz, int dtype, const void *values,
                    int virtual_max, int64_t **out_rows, int64_t *out_n, int64_t **out_gen,
                    int64_t *out_gen_n)
{
    if (!grid_ok(nx, ny, nz) || !values || !out_rows || !out_n || !out_gen || !out_gen_n)
        return OR_ERR_ARG;
    sw_t w;
    out_t o = {{0}, NULL, 0, 0};
    int st = sw_init(&w, nx, ny, nz, dtype, values);
    if (!st) st = run(&w, virtual_max, &o);
    sw_free(&w);
    if (st) { free(o.rows.rows); free(o.gen); return st; }
    *out_rows = o.rows.rows; *out_n = o.rows.n;
    *out_gen = o.gen; *out_gen_n = o.gen_n;
    return OR_OK;
}

/* The discrete gradient of step 1, one row of 4 int64 per simplex:
 * dim, id, partner dim, partner id (-1, -1 for a critical simplex). */
int oracle_gradient(int64_t nx, int64_t ny, int64_t nz, int dtype, const void *values,
                    int64_t **out_rows, int64_t *out_n)
{
    if (!grid_ok(nx, ny, nz) || !values || !out_rows || !out_n) return OR_ERR_ARG;
    sw_t w;
    int st = sw_init(&w, nx, ny, nz, dtype, values);
    if (!st) st = discrete_gradient(&w);
    int64_t *rows = st ? NULL : malloc(sizeof(int64_t) * 4 * (size_t)(w.m ? w.m : 1));
    if (!st && !rows) st = OR_ERR_MEM;
    for (int64_t p = 0; p < w.m && !st; p++) {
        int64_t q = w.grad[p];
        rows[4 * p] = w.s[p].dim; rows[4 * p + 1] = w.s[p].id;
        rows[4 * p + 2] = q < 0 ? -1 : w.s[q].dim;
        rows[4 * p + 3] = q < 0 ? -1 : w.s[q].id;
    }
    int64_t m = w.m;
    sw_free(&w);
    if (st) { free(rows); return st; }
    *out_rows = rows; *out_n = m;
    return OR_OK;
}
