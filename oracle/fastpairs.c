/*
 * oracle/fastpairs.c -- the oracle's standard reduction in "fast mode":
 * the same persistence pairing as oracle_pairsimplices (pairsimplices.c),
 * computed with result-preserving shortcuts so that it reaches grids of
 * 128^3 vertices and more on one CPU core.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this code.  It
 * shares no code, header, table or helper with the CUDA path of the package.
 *
 * What is computed is unchanged (Sec. 2.2, Sec. 2.4-2.5, Alg. 1): the
 * standard reduction of the boundary matrix of the lexicographic filtration
 * of every simplex -- for each column j in filtration order, while the
 * lowest non-zero row of column j is the pivot of an earlier column k, add
 * column k to column j (mod 2) -- keeping the pairs whose two simplices have
 * different maximum vertices (Sec. 4.1 (c)) and the unpaired simplices as
 * infinite classes (Sec. 6).  The shortcuts, each of which leaves every
 * pivot of the reduction unchanged:
 *
 *  1. Dimension separability.  A column of dimension d only ever receives
 *     columns of dimension d (a column is added only to a column with the
 *     same lowest row, and rows of a d-column are (d-1)-simplices), so the
 *     reduction runs one dimension at a time, each in filtration order.
 *  2. Clearing (the twist; Sec. 4, observation (a)).  Dimensions are reduced
 *     from 3 down to 1.  A d-simplex that is the pivot of a (d+1)-column is
 *     a birth, so its own column reduces to zero: it is skipped.
 *  3. Apparent pairs.  A column that needs no addition keeps its boundary as
 *     its reduced form; it is not stored, and is regenerated from the
 *     simplex id whenever a later column adds it.
 *  4. Implicit boundaries and streamed filtration.  No global list of
 *     simplices is built or sorted.  The key of a simplex (its vertex ranks
 *     in decreasing order, Sec. 2.2) is computed from its id; the d-simplices
 *     of the filtration are visited vertex by vertex in increasing rank,
 *     and within the lower star of a vertex in increasing key.  Every
 *     simplex lies in the lower star of its maximum vertex, and the key of a
 *     simplex starts with the rank of that vertex, so this is exactly the
 *     filtration order restricted to dimension d.
 *  5. The column under reduction is kept as a max-heap of keys in which a
 *     key may occur several times (its value: the keys of odd
 *     multiplicity).  Adding a column pushes its keys, and the lowest row is
 *     read off the top after equal keys there cancel in pairs; this is the
 *     same sum mod 2 without merging whole columns at every addition.
 *
 * Result rows as pairsimplices.c (8 int64: dim, birth_id, death_id,
 * birth_vertex, death_vertex, essential, birth_pos, death_pos), except that
 * the two filtration positions are -1 (no global list is formed).
 */
#include "complex.h"

/* A filtration key: the vertex ranks r0 > r1 > r2 > r3 of a simplex, missing
 * ranks as -1, packed so that unsigned (hi, lo) order is the lexicographic
 * order with a face (a prefix) before its cofaces. */
typedef struct { uint64_t hi, lo; } fkey_t;

static inline int key_lt(fkey_t a, fkey_t b)
{
    return a.hi != b.hi ? a.hi < b.hi : a.lo < b.lo;
}

static inline int key_eq(fkey_t a, fkey_t b) { return a.hi == b.hi && a.lo == b.lo; }

typedef struct {
    grid_t g;
    int64_t n;
    int64_t *rank;          /* rank of each vertex in the (value, id) order */
    int64_t *vert_of_rank;
} fctx_t;

static fkey_t key_of_vertices(const fctx_t *c, int dim, const int64_t *vs)
{
    int64_t r[4] = {-1, -1, -1, -1};
    for (int i = 0; i <= dim; i++) r[i] = c->rank[vs[i]];
    sort_desc(r, dim + 1);
    fkey_t k;
    k.hi = ((uint64_t)(r[0] + 1) << 32) | (uint64_t)(r[1] + 1);
    k.lo = ((uint64_t)(r[2] + 1) << 32) | (uint64_t)(r[3] + 1);
    return k;
}

/* The simplex of dimension dim with key k (its vertices are the vertices of
 * the ranks in k). */
static int64_t id_of_key(const fctx_t *c, int dim, fkey_t k)
{
    int64_t r[4] = {(int64_t)(k.hi >> 32) - 1, (int64_t)(k.hi & 0xffffffffu) - 1,
                    (int64_t)(k.lo >> 32) - 1, (int64_t)(k.lo & 0xffffffffu) - 1};
    int64_t vs[4];
    for (int i = 0; i <= dim; i++) vs[i] = c->vert_of_rank[r[i]];
    return simplex_id(&c->g, dim, vs);
}

static int64_t max_vertex_of_key(const fctx_t *c, fkey_t k)
{
    return c->vert_of_rank[(int64_t)(k.hi >> 32) - 1];
}

/* The boundary of (dim, id): keys of its dim+1 facets, in increasing order. */
static int boundary_keys(const fctx_t *c, int dim, int64_t id, fkey_t *out)
{
    int64_t vs[4], fv[3];
    simplex_vertices(&c->g, dim, id, vs);
    for (int drop = 0; drop <= dim; drop++) {
        int m = 0;
        for (int i = 0; i <= dim; i++) if (i != drop) fv[m++] = vs[i];
        out[drop] = key_of_vertices(c, dim - 1, fv);
    }
    for (int i = 1; i <= dim; i++)
        for (int j = i; j > 0 && key_lt(out[j], out[j - 1]); j--) {
            fkey_t t = out[j]; out[j] = out[j - 1]; out[j - 1] = t;
        }
    return dim + 1;
}

/* The d-simplices of the lower star of v (those containing v whose other
 * vertices all have lower rank), with their keys, in increasing key order.
 * A simplex containing v is anchored at v - o for an offset o of its chain. */
static int lower_star(const fctx_t *c, int64_t v, int dim, int64_t *ids, fkey_t *keys)
{
    static const int EDGE_CHAIN[7][2] = {{0, 1}, {0, 2}, {0, 3}, {0, 4}, {0, 5}, {0, 6}, {0, 7}};
    const grid_t *g = &c->g;
    int64_t x = v % g->nx, y = (v / g->nx) % g->ny, z = v / (g->nx * g->ny);
    int cnt = 0;
    for (int o = 0; o < 8; o++) {
        int64_t ax = x - (o & 1), ay = y - ((o >> 1) & 1), az = z - ((o >> 2) & 1);
        if (ax < 0 || ay < 0 || az < 0) continue;
        int64_t a = vid(g, ax, ay, az);
        int nk = ID_MULT[dim];
        for (int k = 0; k < nk; k++) {
            int chain[4], m = 0;
            if (dim == 1) { chain[m++] = EDGE_CHAIN[k][0]; chain[m++] = EDGE_CHAIN[k][1]; }
            else if (dim == 2) { chain[m++] = 0; chain[m++] = TRI_A[k]; chain[m++] = TRI_B[k]; }
            else { chain[m++] = 0; chain[m++] = TET_A[k]; chain[m++] = TET_B[k]; chain[m++] = 7; }
            int has = 0;
            for (int i = 0; i < m; i++) has |= chain[i] == o;
            if (!has) continue;
            int64_t id = ID_MULT[dim] * a + k, vs[4];
            if (!simplex_vertices(g, dim, id, vs)) continue;
            int lower = 1;
            for (int i = 0; i <= dim; i++)
                if (vs[i] != v && c->rank[vs[i]] > c->rank[v]) lower = 0;
            if (!lower) continue;
            ids[cnt] = id;
            keys[cnt] = key_of_vertices(c, dim, vs);
            cnt++;
        }
    }
    for (int i = 1; i < cnt; i++)
        for (int j = i; j > 0 && key_lt(keys[j], keys[j - 1]); j--) {
            fkey_t tk = keys[j]; keys[j] = keys[j - 1]; keys[j - 1] = tk;
            int64_t ti = ids[j]; ids[j] = ids[j - 1]; ids[j - 1] = ti;
        }
    return cnt;
}

/* Reduced columns kept in an append-only arena (standard reduction: a
 * column is final once processed), made of chunks of fixed size so that it
 * grows without copying.  A column lies within one chunk; its place is
 * (chunk << 40) | offset. */
#define ARENA_CHUNK ((int64_t)1 << 24)
typedef struct {
    fkey_t **chunk;
    int64_t nchunk, capchunk, used;    /* used: entries in the last chunk */
    int64_t lastcap;                   /* entries the last chunk holds */
} arena_t;

static int arena_push(arena_t *a, const fkey_t *src, int64_t len, int64_t *start)
{
    if (a->nchunk == 0 || a->used + len > a->lastcap) {
        if (a->nchunk == a->capchunk) {
            int64_t nc = a->capchunk ? 2 * a->capchunk : 64;
            fkey_t **nch = realloc(a->chunk, sizeof(fkey_t *) * (size_t)nc);
            if (!nch) return OR_ERR_MEM;
            a->chunk = nch; a->capchunk = nc;
        }
        int64_t cap = len > ARENA_CHUNK ? len : ARENA_CHUNK;
        fkey_t *c = malloc(sizeof(fkey_t) * (size_t)cap);
        if (!c) return OR_ERR_MEM;
        a->chunk[a->nchunk++] = c;
        a->used = 0;
        a->lastcap = cap;
    }
    memcpy(a->chunk[a->nchunk - 1] + a->used, src, sizeof(fkey_t) * (size_t)len);
    *start = ((a->nchunk - 1) << 40) | a->used;
    a->used += len;
    return OR_OK;
}

static const fkey_t *arena_at(const arena_t *a, int64_t start)
{
    return a->chunk[start >> 40] + (start & (((int64_t)1 << 40) - 1));
}

static void arena_free(arena_t *a)
{
    for (int64_t i = 0; i < a->nchunk; i++) free(a->chunk[i]);
    free(a->chunk);
}

/* The column under reduction as a max-heap of keys in which a key may occur
 * several times: its value is the set of keys of odd multiplicity (a sum
 * mod 2).  Adding a column pushes its keys; equal keys cancel in pairs when
 * they reach the top, so the lowest row (the largest key of odd
 * multiplicity) is found without merging whole columns. */
typedef struct { fkey_t *h; int64_t n, cap; } kheap_t;

static int kheap_push(kheap_t *q, fkey_t k)
{
    if (q->n == q->cap) {
        int64_t nc = q->cap ? 2 * q->cap : 64;
        fkey_t *nh = realloc(q->h, sizeof(fkey_t) * (size_t)nc);
        if (!nh) return OR_ERR_MEM;
        q->h = nh; q->cap = nc;
    }
    int64_t i = q->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!key_lt(q->h[p], k)) break;
        q->h[i] = q->h[p];
        i = p;
    }
    q->h[i] = k;
    return OR_OK;
}

static fkey_t kheap_pop(kheap_t *q)
{
    fkey_t top = q->h[0], last = q->h[--q->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, m = l;
        if (l >= q->n) break;
        if (l + 1 < q->n && key_lt(q->h[l], q->h[l + 1])) m = l + 1;
        if (!key_lt(last, q->h[m])) break;
        q->h[i] = q->h[m];
        i = m;
    }
    if (q->n > 0) q->h[i] = last;
    return top;
}

/* The keys of odd multiplicity, in decreasing order, into out (which holds
 * q->n entries); the heap is emptied.  Returns their number. */
static int64_t kheap_drain(kheap_t *q, fkey_t *out)
{
    int64_t m = 0;
    while (q->n > 0) {
        fkey_t t = kheap_pop(q);
        int odd = 1;
        while (q->n > 0 && key_eq(q->h[0], t)) { kheap_pop(q); odd ^= 1; }
        if (odd) out[m++] = t;
    }
    return m;
}

/* The lowest row of the column: equal keys at the top cancel in pairs; 0
 * when the column is zero. */
static int kheap_pivot(kheap_t *q, fkey_t *top)
{
    while (q->n > 0) {
        fkey_t t = kheap_pop(q);
        if (q->n > 0 && key_eq(q->h[0], t)) { kheap_pop(q); continue; }
        *top = t;
        return kheap_push(q, t) == OR_OK ? 1 : -1;
    }
    return 0;
}

/* Reduction of the columns of dimension dim (1..3).
 *   cleared: (dim)-simplex ids to skip (pivots of dimension dim+1), or NULL.
 *   owner:   out, per (dim-1)-simplex id: the dim-simplex whose reduced
 *            column has it as pivot, or -1.
 *   zero:    out, per dim-simplex id: 1 when its column reduced to zero (or
 *            was cleared), else 0.
 * Simplex ids fit in int32 (checked by the caller). */
static int reduce_dim(const fctx_t *c, int dim, const int32_t *cleared, int32_t *owner,
                      uint8_t *zero, int64_t *additions)
{
    const int64_t n = c->n, nrow = n * ID_MULT[dim - 1], ncol = n * ID_MULT[dim];
    for (int64_t i = 0; i < nrow; i++) owner[i] = -1;
    for (int64_t i = 0; i < ncol; i++) zero[i] = 1;
    /* stored (non-apparent) columns: colidx[tau] indexes cstart/clen, -1 for
     * a column kept implicit */
    int32_t *colidx = calloc((size_t)ncol + 1, sizeof(int32_t));
    int64_t *cstart = NULL, ncols = 0, capcols = 0;
    int64_t *clen = NULL;
    if (!colidx) return OR_ERR_MEM;
    for (int64_t i = 0; i < ncol; i++) colidx[i] = -1;
    arena_t arena = {0};
    kheap_t q = {0};
    fkey_t *col = NULL, bnd[4];
    int64_t ccap = 0, live = 0;
    int64_t ids[36];
    fkey_t keys[36];
    int st = OR_OK;
    for (int64_t r = 0; r < n && !st; r++) {
        int64_t v = c->vert_of_rank[r];
        int cnt = lower_star(c, v, dim, ids, keys);
        for (int s = 0; s < cnt && !st; s++) {
            int64_t tau = ids[s];
            if (cleared && cleared[tau] >= 0) continue;    /* a birth: its column is zero */
            int nb = boundary_keys(c, dim, tau, bnd);
            q.n = 0;
            for (int e = 0; e < nb && !st; e++) st = kheap_push(&q, bnd[e]);
            live = nb;
            int added = 0;
            fkey_t top;
            int has = 0;
            while (!st && (has = kheap_pivot(&q, &top)) == 1) {
                int64_t low = id_of_key(c, dim - 1, top);
                int64_t k = owner[low];
                if (k < 0) break;
                int32_t ki = colidx[k];
                if (ki >= 0) {
                    const fkey_t *src = arena_at(&arena, cstart[ki]);
                    for (int64_t e = 0; e < clen[ki] && !st; e++) st = kheap_push(&q, src[e]);
                } else {
                    fkey_t kb[4];
                    int kn = boundary_keys(c, dim, k, kb);
                    for (int e = 0; e < kn && !st; e++) st = kheap_push(&q, kb[e]);
                }
                added = 1;
                (*additions)++;
                if (!st && q.n > 2 * live + 64) {
                    /* cancel the pairs below the top too: a decreasing list
                     * is itself a valid max-heap */
                    if (q.n > ccap) {
                        fkey_t *nc2 = realloc(col, sizeof(fkey_t) * (size_t)q.n);
                        if (!nc2) { st = OR_ERR_MEM; break; }
                        col = nc2; ccap = q.n;
                    }
                    int64_t m = kheap_drain(&q, col);
                    memcpy(q.h, col, sizeof(fkey_t) * (size_t)m);
                    q.n = m;
                    live = m;
                }
            }
            if (has < 0) st = OR_ERR_MEM;
            if (st || has == 0) continue;                   /* a zero column */
            int64_t low = id_of_key(c, dim - 1, top);
            owner[low] = (int32_t)tau;
            zero[tau] = 0;
            if (added) {
                /* the reduced column, stored increasingly */
                if (q.n > ccap) {
                    fkey_t *nc2 = realloc(col, sizeof(fkey_t) * (size_t)q.n);
                    if (!nc2) { st = OR_ERR_MEM; break; }
                    col = nc2; ccap = q.n;
                }
                int64_t cn = kheap_drain(&q, col);
                for (int64_t i = 0, j = cn - 1; i < j; i++, j--) {
                    fkey_t t = col[i]; col[i] = col[j]; col[j] = t;
                }
                if (ncols == capcols) {
                    int64_t nc = capcols ? 2 * capcols : 1 << 16;
                    int64_t *ns = realloc(cstart, sizeof(int64_t) * (size_t)nc);
                    if (!ns) { st = OR_ERR_MEM; break; }
                    cstart = ns;
                    int64_t *nl = realloc(clen, sizeof(int64_t) * (size_t)nc);
                    if (!nl) { st = OR_ERR_MEM; break; }
                    clen = nl;
                    capcols = nc;
                }
                if (ncols >= INT32_MAX) { st = OR_ERR_MEM; break; }
                st = arena_push(&arena, col, cn, &cstart[ncols]);
                clen[ncols] = cn;
                colidx[tau] = (int32_t)ncols++;
            }
        }
    }
    free(q.h);
    free(col); arena_free(&arena); free(cstart); free(clen); free(colidx);
    return st;
}

static int emit_pairs(const fctx_t *c, int dim, const int32_t *owner, int keep_zero,
                      result_t *res)
{
    /* owner indexes (dim-1)-simplices; each pivot gives the pair
     * (birth = that (dim-1)-simplex, death = its owner). */
    const int64_t nrow = c->n * ID_MULT[dim - 1];
    for (int64_t b = 0; b < nrow; b++) {
        int64_t d = owner[b];
        if (d < 0) continue;
        int64_t vb[4], vd[4];
        simplex_vertices(&c->g, dim - 1, b, vb);
        simplex_vertices(&c->g, dim, d, vd);
        int64_t bmax = max_vertex_of_key(c, key_of_vertices(c, dim - 1, vb));
        int64_t dmax = max_vertex_of_key(c, key_of_vertices(c, dim, vd));
        if (bmax == dmax && !keep_zero) continue;
        int64_t row[8] = {dim - 1, b, d, bmax, dmax, 0, -1, -1};
        int st = push_row(res, row);
        if (st) return st;
    }
    return OR_OK;
}

int oracle_fastpairs(int64_t nx, int64_t ny, int64_t nz, int dtype, const void *values,
                     int keep_zero, int64_t **out_rows, int64_t *out_n, int64_t *additions)
{
    if (!grid_ok(nx, ny, nz) || !values || !out_rows || !out_n) return OR_ERR_ARG;
    if (12 * nx * ny * nz >= ((int64_t)1 << 31)) return OR_ERR_ARG;   /* int32 simplex ids */
    fctx_t c = {{nx, ny, nz}, nx * ny * nz, NULL, NULL};
    const int64_t n = c.n;
    int st;
    int64_t adds = 0;
    c.rank = malloc(sizeof(int64_t) * (size_t)n);
    c.vert_of_rank = malloc(sizeof(int64_t) * (size_t)n);
    if (!c.rank || !c.vert_of_rank) { free(c.rank); free(c.vert_of_rank); return OR_ERR_MEM; }
    if ((st = vertex_ranks(dtype, values, n, c.rank))) {
        free(c.rank); free(c.vert_of_rank); return st;
    }
    for (int64_t v = 0; v < n; v++) c.vert_of_rank[c.rank[v]] = v;

    /* owner[d]: per (d-1)-simplex, the d-simplex whose column it is the
     * pivot of; zero[d]: per d-simplex, column reduced to zero */
    int32_t *owner[4] = {NULL, NULL, NULL, NULL};
    uint8_t *zero[4] = {NULL, NULL, NULL, NULL};
    for (int d = 1; d <= 3 && !st; d++) {
        owner[d] = malloc(sizeof(int32_t) * (size_t)(n * ID_MULT[d - 1]));
        zero[d] = malloc((size_t)(n * ID_MULT[d]));
        if (!owner[d] || !zero[d]) st = OR_ERR_MEM;
    }
    /* tets first, then triangles cleared by the tets' pivots, then edges
     * cleared by the triangles' pivots */
    for (int d = 3; d >= 1 && !st; d--)
        st = reduce_dim(&c, d, d < 3 ? owner[d + 1] : NULL, owner[d], zero[d], &adds);

    result_t res = {0};
    for (int d = 1; d <= 3 && !st; d++) st = emit_pairs(&c, d, owner[d], keep_zero, &res);
    /* infinite classes: simplices that are neither a pivot of the next
     * dimension nor the owner of a pivot */
    for (int dim = 0; dim <= 3 && !st; dim++) {
        for (int64_t id = 0; id < n * ID_MULT[dim] && !st; id++) {
            int birth = dim < 3 && owner[dim + 1][id] >= 0;
            int death = dim > 0 && !zero[dim][id];
            int64_t vs[4];
            if (birth || death || !simplex_vertices(&c.g, dim, id, vs)) continue;
            int64_t v = max_vertex_of_key(&c, key_of_vertices(&c, dim, vs));
            int64_t row[8] = {dim, id, -1, v, -1, 1, -1, -1};
            st = push_row(&res, row);
        }
    }
    for (int d = 1; d <= 3; d++) { free(owner[d]); free(zero[d]); }
    free(c.rank); free(c.vert_of_rank);
    if (st) { free(res.rows); return st; }
    *out_rows = res.rows;
    *out_n = res.n;
    if (additions) *additions = adds;
    return OR_OK;
}
