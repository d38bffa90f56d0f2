/*
 * oracle/pairsimplices.c -- the oracle: plain, slow, CPU-only persistence
 * pairing of a scalar field on a 3D regular grid (Freudenthal triangulation).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  It
 * shares no code, header, table or helper with the CUDA path of the package.
 *
 * What it computes (definitions restated from the paper):
 *  - Sec. 2.1: a PL field on the vertices, made injective by symbolic
 *    perturbation: vertices are ordered by (value, vertex id).
 *  - Sec. 2.2: the lexicographic filtration: a simplex is keyed by its vertex
 *    values sorted in decreasing order; two keys compare lexicographically;
 *    a proper prefix (a face) comes first.
 *  - Sec. 2.4 / Alg. 1 (PairSimplices), which Sec. 2.5 identifies with the
 *    standard boundary-matrix reduction: for every column j in filtration
 *    order, while the lowest non-zero row of column j is owned by an earlier
 *    column k, add column k to column j (mod 2); a non-empty column pairs
 *    (low(j), j).
 *  - Sec. 4.1 (c) / Sec. 6: pairs whose two simplices share their maximum
 *    vertex have zero persistence and are not reported; unpaired simplices
 *    are infinite-persistence classes.
 *
 * Two textbook special cases are provided as independent checks:
 *  - oracle_kruskal_d0: D0 by union-find over all edges in increasing
 *    lexicographic order, elder rule (the sub-level-set connectivity method
 *    the paper attributes to Edelsbrunner et al., Sec. 1.1).
 *  - oracle_kruskal_d2: D2 by union-find over the dual graph (tets as nodes,
 *    triangles as arcs, one virtual maximum for the outer boundary) in
 *    decreasing lexicographic order (Sec. 5.2, duality and "Domains with
 *    boundary").
 *
 * Simplex ids (a convention of this project; the paper fixes none): with
 * v = x + nx*(y + ny*z) and an offset bitmask o (bit0 +x, bit1 +y, bit2 +z),
 * every Freudenthal simplex is a chain of offsets anchored at its min corner
 * v:  edge (v, v+o)                    id = 7v + (o-1),  o in 1..7
 *     triangle (v, v+a, v+b), a < b    id = 12v + k, k over the (b,a) list
 *        (3,1)(3,2)(5,1)(5,4)(6,2)(6,4)(7,1)(7,2)(7,3)(7,4)(7,5)(7,6)
 *     tet (v, v+a, v+b, v+7)           id = 6v + k, k over the (a,b) list
 *        (1,3)(1,5)(2,3)(2,6)(4,5)(4,6)
 *
 * Result rows are 8 int64 each:
 *   dim, birth_id, death_id (-1 if essential), birth_vertex, death_vertex
 *   (-1 if essential), essential flag, birth_pos, death_pos (positions in
 *   the lexicographic filtration; -1 if essential).
 */
#include "complex.h"

/* Standard reduction over all simplices.  keep_zero != 0 also reports the
 * zero-persistence pairs (used by tests of the pairing itself). */
int oracle_pairsimplices(int64_t nx, int64_t ny, int64_t nz, int dtype,
                         const void *values, int keep_zero, int64_t **out_rows,
                         int64_t *out_n)
{
    if (!grid_ok(nx, ny, nz) || !values || !out_rows || !out_n) return OR_ERR_ARG;
    grid_t g = {nx, ny, nz};
    int64_t n = nx * ny * nz, m = 0;
    int st;
    int64_t *rank = malloc(sizeof(int64_t) * (size_t)n);
    if (!rank) return OR_ERR_MEM;
    if ((st = vertex_ranks(dtype, values, n, rank))) { free(rank); return st; }
    int64_t *vert_of_rank = malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; v++) vert_of_rank[rank[v]] = v;

    simp_t *s = NULL;
    if ((st = build_filtration(&g, rank, &s, &m))) { free(rank); free(vert_of_rank); return st; }

    /* position of every simplex id in the filtration */
    int64_t *pos[4];
    for (int d = 0; d < 4; d++) {
        pos[d] = malloc(sizeof(int64_t) * (size_t)(n * ID_MULT[d]));
        for (int64_t i = 0; i < n * ID_MULT[d]; i++) pos[d][i] = -1;
    }
    for (int64_t i = 0; i < m; i++) pos[s[i].dim][s[i].id] = i;

    col_t *R = calloc((size_t)m, sizeof(col_t));
    int64_t *owner = malloc(sizeof(int64_t) * (size_t)m);  /* low -> column */
    int64_t *partner = malloc(sizeof(int64_t) * (size_t)m);
    int64_t *tmp = NULL, tmpcap = 0;
    for (int64_t i = 0; i < m; i++) { owner[i] = -1; partner[i] = -1; }

    for (int64_t j = 0; j < m && !st; j++) {
        int dim = s[j].dim;
        if (dim == 0) continue;
        /* boundary: the dim+1 facets */
        int64_t vs[4], fv[3];
        simplex_vertices(&g, dim, s[j].id, vs);
        R[j].e = malloc(sizeof(int64_t) * (size_t)(dim + 1));
        R[j].cap = dim + 1;
        for (int drop = 0; drop <= dim; drop++) {
            int c = 0;
            for (int i = 0; i <= dim; i++) if (i != drop) fv[c++] = vs[i];
            R[j].e[R[j].n++] = pos[dim - 1][simplex_id(&g, dim - 1, fv)];
        }
        qsort(R[j].e, (size_t)R[j].n, sizeof(int64_t), cmp_i64);
        /* reduce: add earlier columns while the low is already owned */
        while (R[j].n > 0) {
            int64_t low = R[j].e[R[j].n - 1];
            if (owner[low] < 0) break;
            if ((st = col_xor(&R[j], &R[owner[low]], &tmp, &tmpcap))) break;
        }
        if (R[j].n > 0) {
            int64_t low = R[j].e[R[j].n - 1];
            owner[low] = j;
            partner[low] = j;
            partner[j] = low;
        }
    }

    result_t res = {0};
    for (int64_t i = 0; i < m && !st; i++) {
        int64_t row[8];
        int64_t bmax = vert_of_rank[s[i].r[0]];
        if (partner[i] < 0) {          /* unpaired: infinite persistence */
            row[0] = s[i].dim; row[1] = s[i].id; row[2] = -1; row[3] = bmax;
            row[4] = -1; row[5] = 1; row[6] = i; row[7] = -1;
            st = push_row(&res, row);
        } else if (partner[i] > i) {   /* i is the birth of a pair */
            int64_t j = partner[i];
            int64_t dmax = vert_of_rank[s[j].r[0]];
            if (dmax == bmax && !keep_zero) continue;
            row[0] = s[i].dim; row[1] = s[i].id; row[2] = s[j].id; row[3] = bmax;
            row[4] = dmax; row[5] = 0; row[6] = i; row[7] = j;
            st = push_row(&res, row);
        }
    }

    for (int64_t j = 0; j < m; j++) free(R[j].e);
    free(R); free(owner); free(partner); free(tmp); free(s);
    for (int d = 0; d < 4; d++) free(pos[d]);
    free(rank); free(vert_of_rank);
    if (st) { free(res.rows); return st; }
    *out_rows = res.rows;
    *out_n = res.n;
    return OR_OK;
}

/* ------------------------------------------- textbook union-find checkers */

/* D0 by union-find over all edges in increasing lexicographic order.
 * Each component is represented by its oldest (lowest) vertex; an edge that
 * joins two components kills the younger one (elder rule). */
int oracle_kruskal_d0(int64_t nx, int64_t ny, int64_t nz, int dtype,
                      const void *values, int64_t **out_rows, int64_t *out_n)
{
    if (!grid_ok(nx, ny, nz) || !values || !out_rows || !out_n) return OR_ERR_ARG;
    grid_t g = {nx, ny, nz};
    int64_t n = nx * ny * nz;
    int st;
    int64_t *rank = malloc(sizeof(int64_t) * (size_t)n);
    if ((st = vertex_ranks(dtype, values, n, rank))) { free(rank); return st; }
    int64_t *vert_of_rank = malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; v++) vert_of_rank[rank[v]] = v;
    /* edges keyed by (rank of upper vertex, rank of lower vertex) */
    int64_t ne = 0;
    simp_t *e = malloc(sizeof(simp_t) * (size_t)(7 * n));
    for (int64_t id = 0; id < 7 * n; id++) {
        int64_t vs[4];
        if (!simplex_vertices(&g, 1, id, vs)) continue;
        simp_t *t = &e[ne++];
        t->dim = 1; t->id = id;
        t->r[0] = rank[vs[0]]; t->r[1] = rank[vs[1]]; t->r[2] = t->r[3] = -1;
        sort_desc(t->r, 2);
    }
    qsort(e, (size_t)ne, sizeof(simp_t), cmp_lex);
    int64_t *parent = malloc(sizeof(int64_t) * (size_t)n);   /* over ranks */
    for (int64_t r = 0; r < n; r++) parent[r] = r;
    result_t res = {0};
    for (int64_t i = 0; i < ne && !st; i++) {
        int64_t a = uf_find(parent, e[i].r[0]), b = uf_find(parent, e[i].r[1]);
        if (a == b) continue;
        int64_t young = a > b ? a : b, old = a > b ? b : a;
        parent[young] = old;
        int64_t bv = vert_of_rank[young], dv = vert_of_rank[e[i].r[0]];
        if (bv == dv) continue;       /* zero persistence */
        int64_t row[8] = {0, bv, e[i].id, bv, dv, 0, -1, -1};
        st = push_row(&res, row);
    }
    if (!st && n > 0) {
        int64_t gmin = vert_of_rank[0];
        int64_t row[8] = {0, gmin, -1, gmin, -1, 1, -1, -1};
        st = push_row(&res, row);
    }
    free(parent); free(e); free(rank); free(vert_of_rank);
    if (st) { free(res.rows); return st; }
    *out_rows = res.rows;
    *out_n = res.n;
    return OR_OK;
}

/* D2 by union-find on the dual graph: nodes are the tets plus one virtual
 * maximum for the outside, arcs are the triangles (a boundary triangle links
 * its tet to the virtual maximum), processed in decreasing lexicographic
 * order.  Each component is represented by its oldest (highest) tet; the
 * virtual maximum is older than every tet.  A triangle joining two
 * components kills the younger one. */
int oracle_kruskal_d2(int64_t nx, int64_t ny, int64_t nz, int dtype,
                      const void *values, int64_t **out_rows, int64_t *out_n)
{
    if (!grid_ok(nx, ny, nz) || !values || !out_rows || !out_n) return OR_ERR_ARG;
    grid_t g = {nx, ny, nz};
    int64_t n = nx * ny * nz;
    int st;
    int64_t *rank = malloc(sizeof(int64_t) * (size_t)n);
    if ((st = vertex_ranks(dtype, values, n, rank))) { free(rank); return st; }
    int64_t *vert_of_rank = malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; v++) vert_of_rank[rank[v]] = v;

    /* tets in lexicographic order; node index = order position */
    int64_t nt = 0, ntri = 0;
    simp_t *T = malloc(sizeof(simp_t) * (size_t)(6 * n));
    for (int64_t id = 0; id < 6 * n; id++) {
        int64_t vs[4];
        if (!simplex_vertices(&g, 3, id, vs)) continue;
        simp_t *t = &T[nt++];
        t->dim = 3; t->id = id;
        for (int i = 0; i < 4; i++) t->r[i] = rank[vs[i]];
        sort_desc(t->r, 4);
    }
    qsort(T, (size_t)nt, sizeof(simp_t), cmp_lex);
    int64_t *tetpos = malloc(sizeof(int64_t) * (size_t)(6 * n));
    for (int64_t i = 0; i < 6 * n; i++) tetpos[i] = -1;
    for (int64_t i = 0; i < nt; i++) tetpos[T[i].id] = i;

    /* triangles with their (up to two) cofacet tets */
    simp_t *F = malloc(sizeof(simp_t) * (size_t)(12 * n));
    int64_t *cof = malloc(sizeof(int64_t) * 2 * (size_t)(12 * n));
    for (int64_t id = 0; id < 12 * n; id++) {
        int64_t vs[4];
        if (!simplex_vertices(&g, 2, id, vs)) continue;
        simp_t *t = &F[ntri];
        t->dim = 2; t->id = id;
        for (int i = 0; i < 3; i++) t->r[i] = rank[vs[i]];
        t->r[3] = -1;
        sort_desc(t->r, 3);
        ntri++;
    }
    qsort(F, (size_t)ntri, sizeof(simp_t), cmp_lex);
    /* cofacets: tets whose vertex set contains the triangle's */
    for (int64_t i = 0; i < ntri; i++) { cof[2 * i] = cof[2 * i + 1] = nt; }
    int64_t *tripos = malloc(sizeof(int64_t) * (size_t)(12 * n));
    for (int64_t i = 0; i < 12 * n; i++) tripos[i] = -1;
    for (int64_t i = 0; i < ntri; i++) tripos[F[i].id] = i;
    for (int64_t i = 0; i < nt; i++) {
        int64_t vs[4], fv[3];
        simplex_vertices(&g, 3, T[i].id, vs);
        for (int drop = 0; drop < 4; drop++) {
            int c = 0;
            for (int k = 0; k < 4; k++) if (k != drop) fv[c++] = vs[k];
            int64_t f = tripos[simplex_id(&g, 2, fv)];
            if (cof[2 * f] == nt) cof[2 * f] = i; else cof[2 * f + 1] = i;
        }
    }
    /* node nt is the virtual maximum */
    int64_t *parent = malloc(sizeof(int64_t) * (size_t)(nt + 1));
    for (int64_t i = 0; i <= nt; i++) parent[i] = i;
    result_t res = {0};
    for (int64_t i = ntri - 1; i >= 0 && !st; i--) {
        int64_t a = uf_find(parent, cof[2 * i]), b = uf_find(parent, cof[2 * i + 1]);
        if (a == b) continue;
        int64_t young = a < b ? a : b, old = a < b ? b : a;
        parent[young] = old;
        int64_t bv = vert_of_rank[F[i].r[0]], dv = vert_of_rank[T[young].r[0]];
        if (bv == dv) continue;       /* zero persistence */
        int64_t row[8] = {2, F[i].id, T[young].id, bv, dv, 0, -1, -1};
        st = push_row(&res, row);
    }
    free(parent); free(tripos); free(cof); free(F); free(tetpos); free(T);
    free(rank); free(vert_of_rank);
    if (st) { free(res.rows); return st; }
    *out_rows = res.rows;
    *out_n = res.n;
    return OR_OK;
}

/* Number of valid simplices of each dimension (by enumeration). */
int oracle_simplex_counts(int64_t nx, int64_t ny, int64_t nz, int64_t *counts)
{
    if (!grid_ok(nx, ny, nz) || !counts) return OR_ERR_ARG;
    grid_t g = {nx, ny, nz};
    int64_t n = nx * ny * nz;
    for (int d = 0; d < 4; d++) {
        counts[d] = 0;
        for (int64_t id = 0; id < n * ID_MULT[d]; id++) {
            int64_t vs[4];
            counts[d] += simplex_vertices(&g, d, id, vs);
        }
    }
    return OR_OK;
}

/* Vertices of a simplex id (for tests); returns 1 if valid. */
int oracle_simplex_vertices(int64_t nx, int64_t ny, int64_t nz, int dim, int64_t id,
                            int64_t *vs)
{
    grid_t g = {nx, ny, nz};
    if (!grid_ok(nx, ny, nz) || dim < 0 || dim > 3 || id < 0 ||
        id >= nx * ny * nz * ID_MULT[dim])
        return 0;
    return simplex_vertices(&g, dim, id, vs);
}

void oracle_free(void *p) { free(p); }
