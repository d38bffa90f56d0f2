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
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NAN 2
#define OR_ERR_MEM 3

/* ---------------------------------------------------------------- values */

/* Maps a value to an unsigned key whose order is the numeric order.
 * -0.0 and +0.0 compare equal; NaN is rejected. */
static int value_key(int dtype, const void *values, int64_t v, uint64_t *key)
{
    if (dtype == 0) {
        *key = ((const uint16_t *)values)[v];
        return OR_OK;
    }
    if (dtype == 1) {
        float f = ((const float *)values)[v];
        if (f != f) return OR_ERR_NAN;
        if (f == 0.0f) f = 0.0f;
        uint32_t u;
        memcpy(&u, &f, 4);
        u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        *key = u;
        return OR_OK;
    }
    if (dtype == 2) {
        double d = ((const double *)values)[v];
        if (d != d) return OR_ERR_NAN;
        if (d == 0.0) d = 0.0;
        uint64_t u;
        memcpy(&u, &d, 8);
        u = (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
        *key = u;
        return OR_OK;
    }
    return OR_ERR_ARG;
}

typedef struct { uint64_t key; int64_t id; } vkey_t;

static int cmp_vkey(const void *a, const void *b)
{
    const vkey_t *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* rank[v] = position of v in the order by (value, id). */
static int vertex_ranks(int dtype, const void *values, int64_t n, int64_t *rank)
{
    vkey_t *k = malloc(sizeof(vkey_t) * (size_t)(n ? n : 1));
    if (!k) return OR_ERR_MEM;
    for (int64_t v = 0; v < n; v++) {
        int st = value_key(dtype, values, v, &k[v].key);
        if (st) { free(k); return st; }
        k[v].id = v;
    }
    qsort(k, (size_t)n, sizeof(vkey_t), cmp_vkey);
    for (int64_t r = 0; r < n; r++) rank[k[r].id] = r;
    free(k);
    return OR_OK;
}

/* ------------------------------------------------------------- simplices */

/* Triangle chains (b, a) in id order, and tet chains (a, b). */
static const int TRI_B[12] = {3, 3, 5, 5, 6, 6, 7, 7, 7, 7, 7, 7};
static const int TRI_A[12] = {1, 2, 1, 4, 2, 4, 1, 2, 3, 4, 5, 6};
static const int TET_A[6] = {1, 1, 2, 2, 4, 4};
static const int TET_B[6] = {3, 5, 3, 6, 5, 6};

typedef struct { int64_t nx, ny, nz; } grid_t;

static int64_t vid(const grid_t *g, int64_t x, int64_t y, int64_t z)
{
    return x + g->nx * (y + g->ny * z);
}

static int64_t add_offset(const grid_t *g, int64_t v, int o, int *ok)
{
    int64_t x = v % g->nx, y = (v / g->nx) % g->ny, z = v / (g->nx * g->ny);
    x += o & 1; y += (o >> 1) & 1; z += (o >> 2) & 1;
    *ok = (x < g->nx && y < g->ny && z < g->nz);
    return vid(g, x, y, z);
}

/* Vertices of simplex (dim, id); returns 0 if the id is not a valid simplex. */
static int simplex_vertices(const grid_t *g, int dim, int64_t id, int64_t *vs)
{
    int ok = 1, o1 = 1, o2 = 1, o3 = 1;
    if (dim == 0) { vs[0] = id; return 1; }
    if (dim == 1) {
        int64_t v = id / 7; int o = (int)(id % 7) + 1;
        vs[0] = v; vs[1] = add_offset(g, v, o, &ok);
        return ok;
    }
    if (dim == 2) {
        int64_t v = id / 12; int k = (int)(id % 12);
        vs[0] = v;
        vs[1] = add_offset(g, v, TRI_A[k], &o1);
        vs[2] = add_offset(g, v, TRI_B[k], &o2);
        return o1 && o2;
    }
    if (dim == 3) {
        int64_t v = id / 6; int k = (int)(id % 6);
        vs[0] = v;
        vs[1] = add_offset(g, v, TET_A[k], &o1);
        vs[2] = add_offset(g, v, TET_B[k], &o2);
        vs[3] = add_offset(g, v, 7, &o3);
        return o1 && o2 && o3;
    }
    return 0;
}

/* Id of the simplex spanned by vs[0..dim] (any order): the anchor is the
 * componentwise-minimum corner; the others are offset bitmasks from it. */
static int64_t simplex_id(const grid_t *g, int dim, const int64_t *vs)
{
    int64_t cx[4], cy[4], cz[4], mx = -1, my = -1, mz = -1;
    for (int i = 0; i <= dim; i++) {
        cx[i] = vs[i] % g->nx; cy[i] = (vs[i] / g->nx) % g->ny;
        cz[i] = vs[i] / (g->nx * g->ny);
        if (mx < 0 || cx[i] < mx) mx = cx[i];
        if (my < 0 || cy[i] < my) my = cy[i];
        if (mz < 0 || cz[i] < mz) mz = cz[i];
    }
    int64_t anchor = vid(g, mx, my, mz);
    int offs[4], n = 0;
    for (int i = 0; i <= dim; i++) {
        int o = (int)((cx[i] - mx) | ((cy[i] - my) << 1) | ((cz[i] - mz) << 2));
        if (o) offs[n++] = o;
    }
    if (dim == 0) return vs[0];
    if (dim == 1) return 7 * anchor + (offs[0] - 1);
    if (dim == 2) {
        int a = offs[0], b = offs[1];
        if ((a & b) != a) { int t = a; a = b; b = t; }
        for (int k = 0; k < 12; k++)
            if (TRI_A[k] == a && TRI_B[k] == b) return 12 * anchor + k;
        return -1;
    }
    if (dim == 3) {
        int a = 0, b = 0;
        for (int i = 0; i < 3; i++) {
            int c = __builtin_popcount(offs[i]);
            if (c == 1) a = offs[i];
            if (c == 2) b = offs[i];
        }
        for (int k = 0; k < 6; k++)
            if (TET_A[k] == a && TET_B[k] == b) return 6 * anchor + k;
        return -1;
    }
    return -1;
}

static const int ID_MULT[4] = {1, 7, 12, 6};

/* A simplex of the filtration: vertex ranks sorted decreasingly. */
typedef struct {
    int64_t r[4];   /* ranks, decreasing; unused entries -1 */
    int64_t id;
    int32_t dim;
} simp_t;

static int cmp_lex(const void *a, const void *b)
{
    const simp_t *x = a, *y = b;
    int n = (x->dim < y->dim ? x->dim : y->dim) + 1;
    for (int i = 0; i < n; i++)
        if (x->r[i] != y->r[i]) return x->r[i] < y->r[i] ? -1 : 1;
    /* a proper prefix (a face) comes first */
    if (x->dim != y->dim) return x->dim < y->dim ? -1 : 1;
    return 0;
}

static void sort_desc(int64_t *r, int n)
{
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && r[j - 1] < r[j]; j--) {
            int64_t t = r[j]; r[j] = r[j - 1]; r[j - 1] = t;
        }
}

/* Every valid simplex, keyed, in lexicographic filtration order. */
static int build_filtration(const grid_t *g, const int64_t *rank, simp_t **out,
                            int64_t *count)
{
    int64_t n = g->nx * g->ny * g->nz, total = 0, cap = 26 * n;
    simp_t *s = malloc(sizeof(simp_t) * (size_t)(cap ? cap : 1));
    if (!s) return OR_ERR_MEM;
    for (int dim = 0; dim <= 3; dim++) {
        for (int64_t id = 0; id < n * ID_MULT[dim]; id++) {
            int64_t vs[4];
            if (!simplex_vertices(g, dim, id, vs)) continue;
            simp_t *t = &s[total++];
            t->dim = dim; t->id = id;
            for (int i = 0; i < 4; i++) t->r[i] = i <= dim ? rank[vs[i]] : -1;
            sort_desc(t->r, dim + 1);
        }
    }
    qsort(s, (size_t)total, sizeof(simp_t), cmp_lex);
    *out = s;
    *count = total;
    return OR_OK;
}

/* ------------------------------------------------------------ the result */

typedef struct { int64_t *rows; int64_t n, cap; } result_t;

static int push_row(result_t *res, const int64_t *row)
{
    if (res->n == res->cap) {
        int64_t nc = res->cap ? 2 * res->cap : 64;
        int64_t *nr = realloc(res->rows, sizeof(int64_t) * 8 * (size_t)nc);
        if (!nr) return OR_ERR_MEM;
        res->rows = nr; res->cap = nc;
    }
    memcpy(res->rows + 8 * res->n, row, 8 * sizeof(int64_t));
    res->n++;
    return OR_OK;
}

static int grid_ok(int64_t nx, int64_t ny, int64_t nz)
{
    return nx >= 1 && ny >= 1 && nz >= 1 && nx <= (1 << 20) && ny <= (1 << 20) &&
           nz <= (1 << 20) && nx * ny * nz <= ((int64_t)1 << 31);
}

/* ------------------------------------------------ Alg. 1: standard reduction */

typedef struct { int64_t *e; int64_t n, cap; } col_t;   /* sorted ascending */

static int col_xor(col_t *dst, const col_t *src, int64_t **tmp, int64_t *tmpcap)
{
    int64_t need = dst->n + src->n;
    if (need > *tmpcap) {
        int64_t *nt = realloc(*tmp, sizeof(int64_t) * (size_t)need);
        if (!nt) return OR_ERR_MEM;
        *tmp = nt; *tmpcap = need;
    }
    int64_t i = 0, j = 0, k = 0, *t = *tmp;
    while (i < dst->n || j < src->n) {
        if (j >= src->n || (i < dst->n && dst->e[i] < src->e[j])) t[k++] = dst->e[i++];
        else if (i >= dst->n || src->e[j] < dst->e[i]) t[k++] = src->e[j++];
        else { i++; j++; }          /* 1 + 1 = 0 (mod 2) */
    }
    if (k > dst->cap) {
        int64_t *ne = realloc(dst->e, sizeof(int64_t) * (size_t)k);
        if (!ne && k) return OR_ERR_MEM;
        dst->e = ne; dst->cap = k;
    }
    memcpy(dst->e, t, sizeof(int64_t) * (size_t)k);
    dst->n = k;
    return OR_OK;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : x > y;
}

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

static int64_t uf_find(int64_t *parent, int64_t a)
{
    while (parent[a] != a) { parent[a] = parent[parent[a]]; a = parent[a]; }
    return a;
}

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
