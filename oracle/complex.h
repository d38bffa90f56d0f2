/*
 * oracle/complex.h -- shared parts of the oracle: vertex order, the
 * Freudenthal simplices of a 3D grid and their ids, the lexicographic
 * filtration, Z/2 columns and result rows.
 *
 * TEST INFRASTRUCTURE ONLY (see pairsimplices.c).  Included by the oracle's
 * C files and by nothing else.
 */
#ifndef ORACLE_COMPLEX_H
#define ORACLE_COMPLEX_H
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
static inline int value_key(int dtype, const void *values, int64_t v, uint64_t *key)
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

static inline int cmp_vkey(const void *a, const void *b)
{
    const vkey_t *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* rank[v] = position of v in the order by (value, id). */
static inline int vertex_ranks(int dtype, const void *values, int64_t n, int64_t *rank)
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

static inline int64_t vid(const grid_t *g, int64_t x, int64_t y, int64_t z)
{
    return x + g->nx * (y + g->ny * z);
}

static inline int64_t add_offset(const grid_t *g, int64_t v, int o, int *ok)
{
    int64_t x = v % g->nx, y = (v / g->nx) % g->ny, z = v / (g->nx * g->ny);
    x += o & 1; y += (o >> 1) & 1; z += (o >> 2) & 1;
    *ok = (x < g->nx && y < g->ny && z < g->nz);
    return vid(g, x, y, z);
}

/* Vertices of simplex (dim, id); returns 0 if the id is not a valid simplex. */
static inline int simplex_vertices(const grid_t *g, int dim, int64_t id, int64_t *vs)
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
static inline int64_t simplex_id(const grid_t *g, int dim, const int64_t *vs)
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

static inline int cmp_lex(const void *a, const void *b)
{
    const simp_t *x = a, *y = b;
    int n = (x->dim < y->dim ? x->dim : y->dim) + 1;
    for (int i = 0; i < n; i++)
        if (x->r[i] != y->r[i]) return x->r[i] < y->r[i] ? -1 : 1;
    /* a proper prefix (a face) comes first */
    if (x->dim != y->dim) return x->dim < y->dim ? -1 : 1;
    return 0;
}

static inline void sort_desc(int64_t *r, int n)
{
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && r[j - 1] < r[j]; j--) {
            int64_t t = r[j]; r[j] = r[j - 1]; r[j - 1] = t;
        }
}

/* Every valid simplex, keyed, in lexicographic filtration order. */
static inline int build_filtration(const grid_t *g, const int64_t *rank, simp_t **out,
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

static inline int push_row(result_t *res, const int64_t *row)
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

static inline int grid_ok(int64_t nx, int64_t ny, int64_t nz)
{
    return nx >= 1 && ny >= 1 && nz >= 1 && nx <= (1 << 20) && ny <= (1 << 20) &&
           nz <= (1 << 20) && nx * ny * nz <= ((int64_t)1 << 31);
}

/* ------------------------------------------------------ Z/2 columns (sets) */

/* A mod-2 chain: the filtration positions of its simplices, sorted ascending. */
typedef struct { int64_t *e; int64_t n, cap; } col_t;

static inline int col_xor(col_t *dst, const col_t *src, int64_t **tmp, int64_t *tmpcap)
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

static inline int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : x > y;
}

/* ------------------------------------------------------------- union-find */

static inline int64_t uf_find(int64_t *parent, int64_t a)
{
    while (parent[a] != a) { parent[a] = parent[parent[a]]; a = parent[a]; }
    return a;
}

#endif
