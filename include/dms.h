/*
 * dms.h -- C ABI of libdms: persistence diagrams D0, D1, D2 of a piecewise
 * linear scalar field on a 3D regular grid by the Discrete Morse Sandwich
 * (Guillou, Vidal, Tierny, arXiv 2206.13932), computed on one NVIDIA GPU.
 *
 * The paper's definitions this library follows:
 *   Sec. 2.1  input: a PL field on the vertices of a 3D grid triangulated by
 *             Freudenthal (6 tetrahedra per cube, 14 neighbours per vertex),
 *             made injective by symbolic perturbation: vertices are ordered
 *             by (value, vertex id).
 *   Sec. 2.2  the lexicographic filtration of all simplices.
 *   Sec. 2.4  persistence pairs (birth p-simplex, death (p+1)-simplex);
 *             the value of a simplex is the value of its maximum vertex.
 *   Sec. 4    Alg. 2 (zero-persistence skip through the discrete gradient of
 *             Robins et al.'s ProcessLowerStars) and Alg. 3
 *             (PairCriticalSimplices).
 *   Sec. 5    D0 from the unstable sets of 1-saddles, D2 from the stable sets
 *             of 2-saddles with a virtual maximum on the outer boundary.
 *   Sec. 6    infinite-persistence classes, reported at (f(sigma), f*),
 *             f* = the maximum value.
 *
 * The result equals, simplex id for simplex id, the pairs of the standard
 * reduction of the lexicographic filtration whose two simplices have
 * different maximum vertices, plus the infinite-persistence classes.
 *
 * Threading: one handle per stream; calls on one handle are not reentrant.
 * Errors: every entry point returns a dms_status; no exception crosses the
 * ABI.  After a failed dms_compute_diagram the handle holds no result
 * (dms_get_counts and dms_fetch_pairs return DMS_ERR_STATE) until the next
 * successful compute.
 */
#ifndef DMS_H
#define DMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DMS_OK = 0,
    DMS_ERR_INVALID_ARG = 1,   /* bad size, dtype, pointer or dimension      */
    DMS_ERR_NAN = 2,           /* the field holds a NaN                      */
    DMS_ERR_OOM = 3,           /* device or host allocation failed           */
    DMS_ERR_CUDA = 4,          /* a CUDA runtime call failed                 */
    DMS_ERR_ITER_LIMIT = 5,    /* a bounded device loop hit its limit        */
    DMS_ERR_STATE = 6,         /* no result available / inconsistent result  */
    DMS_ERR_CAPACITY = 7       /* a scratch or index limit was exceeded      */
} dms_status;

typedef enum { DMS_U16 = 0, DMS_F32 = 1, DMS_F64 = 2 } dms_dtype;

typedef struct {
    int virtual_max;      /* 1: the outer boundary is one virtual maximum,
                             older than every tet (Sec. 5.2, "Domains with
                             boundary"); D2 then equals the standard
                             reduction of the cube.  0: no virtual maximum
                             (App. A): a 2-saddle whose ascending path
                             leaves the domain on either side merges nothing
                             in D2 and goes to D1; maxima left unpaired are
                             infinite classes of dimension 3, and 2-saddles
                             whose D1 column reduces to zero infinite classes
                             of dimension 2.                                 */
    int64_t max_iters;    /* cap on device loops and path lengths; 0 = default */
    int d1_mode;          /* D1 reduction: 0 = by density (3 when there are
                             fewer 2-saddle columns than 1 per 32 vertices,
                             else 1), 1 = reduce the
                             2-saddle columns (Alg. 3 order), 2 = reduce their
                             anti-transpose (persistent cohomology), 3 = lazy
                             columns: each 2-saddle's Morse boundary is
                             expanded only as far as its current pivot,
                             between rounds of the reduction (Alg. 3's
                             interleaving); all modes give the same pairs    */
    int generators;       /* 1: also compute a persistent 1-cycle generator
                             of every D1 pair (Sec. 8; dms_fetch_generators).
                             Single grids of fewer than 2^31 / 7 vertices,
                             with d1_mode 0 or 1 (the traced reduction runs
                             in rounds); 0: not computed (the default)       */
} dms_options;

/* One persistence pair (or infinite class) of the result.
 * Simplex ids (a convention of this library; the paper fixes none).  With
 * v = x + nx*(y + ny*z) and offsets o (bit0 +x, bit1 +y, bit2 +z), each
 * simplex is a chain of offsets anchored at its componentwise-min corner v:
 *   vertex   v                                  id = v
 *   edge     (v, v+o), o in 1..7                id = 7v + (o-1)
 *   triangle (v, v+a, v+b), a subset of b       id = 12v + k, k indexing (b,a)
 *            (3,1)(3,2)(5,1)(5,4)(6,2)(6,4)(7,1)(7,2)(7,3)(7,4)(7,5)(7,6)
 *   tet      (v, v+a, v+b, v+7)                 id = 6v + k, k indexing (a,b)
 *            (1,3)(1,5)(2,3)(2,6)(4,5)(4,6)
 * birth_vertex / death_vertex are the maximum vertices of the two simplices;
 * birth_bits / death_bits are the raw bits of their values (zero-extended
 * uint16, float or double bits).  An infinite class has death_simplex = -1,
 * death_vertex = -1 and death_bits = the bits of the maximum value f*.  */
typedef struct {
    int64_t birth_simplex, death_simplex;
    int64_t birth_vertex, death_vertex;
    uint64_t birth_bits, death_bits;
    uint8_t dim, essential, pad[6];
} dms_pair;

typedef struct dms_grid_s *dms_grid;

/* Creates a handle for an nx*ny*nz grid (each >= 1, product < 2^31) of the
 * given dtype.  opts may be NULL (defaults).  Allocates the grid-sized device
 * buffers on the current device.  *out is set only on success. */
dms_status dms_grid_create(int64_t nx, int64_t ny, int64_t nz, dms_dtype dtype,
                           const dms_options *opts, dms_grid *out);

/* Creates a handle for a batch of nfields grids (1 <= nfields <= 65535) of
 * their own shapes: shapes[3f..3f+2] = nx, ny, nz of field f (each >= 1,
 * total vertex count < 2^31), one dtype.  The batch is computed in one pass
 * of the pipeline -- one launch of each kernel for all fields -- over the
 * disjoint union of the grids, whose persistence diagrams are those of the
 * fields (a union of disjoint complexes has block-diagonal boundary
 * matrices; the shared virtual maximum is older than every other node, so
 * no field's merges change).
 *   dms_compute_diagram: values = the fields one after another, each x
 *     fastest (field f starts at element sum of the sizes of fields < f).
 *   dms_fetch_pairs: the pairs of all fields grouped by field (field 0
 *     first), each field's pairs in the order of a single-grid compute, with
 *     simplex and vertex ids relative to the field; dms_batch_offsets gives
 *     the ranges.  An infinite class dies at the maximum of its own field.
 *   dms_get_counts: totals over the batch.
 *   dms_backward_pairs: grad_field in the layout of values.
 *   dms_grid_reshape: not available (DMS_ERR_INVALID_ARG). */
dms_status dms_batch_create(int64_t nfields, const int64_t *shapes, dms_dtype dtype,
                            const dms_options *opts, dms_grid *out);

/* Re-targets a batch handle to another batch (same dtype and options): new
 * field count and shapes as in dms_batch_create.  Device buffers are kept and
 * grow only when needed, so one handle serves a stream of batches.  Drops the
 * last result.  DMS_ERR_INVALID_ARG for a single-grid handle. */
dms_status dms_batch_reshape(dms_grid grid, int64_t nfields, const int64_t *shapes);

/* offsets[f] .. offsets[f+1] (nfields + 1 host int64) = the positions of
 * field f's pairs of dimension dim in dms_fetch_pairs order, for the last
 * successful compute of a batch (DMS_ERR_STATE for a single grid or without
 * a result). */
dms_status dms_batch_offsets(dms_grid grid, int dim, int64_t *offsets);

/* Changes the grid dimensions of a handle (same dtype and options), keeping
 * its device buffers and growing them only when the new grid is larger, so
 * that one handle serves fields of many shapes.  Drops the last result. */
dms_status dms_grid_reshape(dms_grid grid, int64_t nx, int64_t ny, int64_t nz);

/* Computes D0, D1, D2 and the infinite classes of the field `values`
 * (nx*ny*nz elements, x fastest).  values_on_host = 0: a device pointer that
 * must stay valid until `stream` (a cudaStream_t, NULL = legacy default)
 * reaches the end of the call; = 1: a host pointer, copied in on `stream`.
 * The call returns after the result is resident on the device (it
 * synchronises `stream`).  NaN in the field -> DMS_ERR_NAN.  Critical
 * simplices are indexed in int32: a field (or batch) with more than
 * (2^31 - 1) / 12 = 178956970 PL-critical vertices -> DMS_ERR_CAPACITY (a
 * lower star holds at most 12 critical cells). */
dms_status dms_compute_diagram(dms_grid grid, const void *values, int values_on_host,
                               void *stream);

/* Number of finite pairs per dimension and of infinite classes per dimension
 * of the last successful compute. */
dms_status dms_get_counts(dms_grid grid, int64_t pairs[3], int64_t essential[4]);

/* Copies the pairs of dimension dim (0..2) -- the finite pairs in increasing
 * lexicographic order of the critical simplex that indexes them (the death
 * edge for D0, the death triangle for D1, the birth triangle for D2), then the
 * infinite classes of that dimension; for dim 2, last, the infinite classes
 * of dimension 3 (dim field 3; only with virtual_max = 0) -- into
 * out[0..cap): pairs[dim] + essential[dim] rows (+ essential[3] for dim 2).  *written = number copied; if cap is smaller
 * than the count, DMS_ERR_CAPACITY is returned and nothing is copied.
 * out_is_device = 1: out is a device pointer (a synchronous device-to-device
 * copy; the result is already complete when dms_compute_diagram returns). */
dms_status dms_fetch_pairs(dms_grid grid, int dim, dms_pair *out, int64_t cap,
                           int64_t *written, int out_is_device);

/* Persistent 1-cycle generators of the D1 pairs of the last compute (Sec. 8),
 * for a handle created with dms_options.generators = 1 (DMS_ERR_STATE
 * otherwise, or without a result).  out[0..cap) receives int64 records, one
 * per D1 pair in the order of dms_fetch_pairs(1): the birth edge id, the
 * death triangle id, k, then the ids of the k edges of the cycle.  The cycle
 * has the birth edge as its highest edge and differs from the boundary of
 * the death triangle by a sum of boundaries of triangles before it: it is
 * the Boundary of Alg. 3 for that pair up to the order of propagation (the
 * reduction here expands every regular edge of a column, Alg. 3 only those
 * that become its highest), so a valid generator, not necessarily the same
 * edges.  *written = the number of int64 words of all records; if cap is
 * smaller, DMS_ERR_CAPACITY is returned and nothing is copied. */
dms_status dms_fetch_generators(dms_grid grid, int64_t *out, int64_t cap, int64_t *written);

/* Identifier of the last successful compute of the handle: every
 * successful dms_compute_diagram gives a new value (a counter of the
 * handle).  DMS_ERR_STATE without a result. */
dms_status dms_get_result_id(dms_grid grid, uint64_t *result_id);

/* Backward pass of a loss of the diagram (differentiation).  The value of a
 * pair is the value of its maximum vertices (Sec. 2.4: persistence =
 * f(max vertex of death) - f(max vertex of birth)), so the gradient of a
 * loss with respect to the field is the sum, at each vertex, of the
 * gradients of the births and deaths whose maximum vertex it is.
 * result_id: the dms_get_result_id of the compute whose pairs the gradients
 * belong to; if the handle has computed another field since (or holds no
 * result), the call returns DMS_ERR_STATE and launches nothing, since the
 * gradient arrays would not match the current pairs.
 * grad_birth / grad_death: device arrays of doubles, one per pair of
 * dimension dim in dms_fetch_pairs order (either may be NULL; the death
 * gradient of an infinite class is ignored).  grad_field: device array of
 * nx*ny*nz doubles that the call adds into (atomically; the caller zeroes
 * it first).  Runs on `stream`, asynchronously. */
dms_status dms_backward_pairs(dms_grid grid, int dim, uint64_t result_id,
                              const double *grad_birth, const double *grad_death,
                              double *grad_field, void *stream);

/* Per-stage device milliseconds of the last compute (CUDA events):
 * [0] gradient (classification + ProcessLowerStars + compaction),
 * [1] sorting critical simplices, [2] D0 (D2's ascending walks run beside
 * it on a second stream of the handle, as the paper runs D0 and D2 as
 * parallel tasks), [3] D2 (its elder rule, once those walks are done),
 * [4] D1, [5] output, [6] total, [7] host-to-device copy (values_on_host =
 * 1 only). */
dms_status dms_get_stage_ms(dms_grid grid, float ms[8]);

/* Statistics of the last compute: [0] critical vertices, [1..4] critical
 * simplices of dimension 0..3, [5] kernel launches, [6] D0 halving levels,
 * [7] D2 halving levels (both over the spanning forest's arcs), [8] D1 reduction rounds, [9] D1 columns, [10] D1
 * columns whose boundary outgrew the first scratch pass (lazy mode: column
 * advances that did), [11] D1 column additions, [12] D1 column-pool entries
 * used (4 B each; lazy mode 16 B), [13] D1 pool regrowths, [14] bytes read
 * by D1 column additions, [15] bytes written by D1 column additions. */
dms_status dms_get_stats(dms_grid grid, int64_t stats[16]);

/* Work counts of the last compute that rooflines are computed from: [0]
 * edges toggled by the D1 boundary trace (each reads the gradient record,
 * flag byte, value and row word of the edge's vertex: the walks of the
 * descending paths of Sec. 5.3), [1] regular edges it expanded, [2] the
 * longest chain of dependent column additions one reduction kernel made
 * (a column adding the owners of its pivots one after another; the rounds'
 * and the asynchronous tail's chains), [3] 0 (reserved).  The lazy D1 mode
 * (d1_mode 3) reports 0 in [0] and [1]. */
dms_status dms_get_work(dms_grid grid, int64_t work[4]);

/* Device memory the handle holds now, in bytes: the sum of its device
 * arenas (grid-sized state, critical lists, union-find tables, D1 pools and
 * output), which only grow and are kept across computes and reshapes.  Host
 * pinned memory and the library's fixed tables are not counted. */
dms_status dms_get_device_bytes(dms_grid grid, int64_t *bytes);

/* Device milliseconds of the last compute per kernel family, from CUDA event
 * pairs recorded on the compute stream around the launches (host round trips
 * between launches of one family are included): [0] classify (the per-vertex
 * stencil), [1] compaction, [2] radix sort, [3] ProcessLowerStars, [4] emit
 * of the critical simplices, [5] D0 arcs, [6] D0 elder rule (spanning
 * forest and halving levels), [7] D2 arcs (timed on the second stream,
 * beside [5]-[6]), [8] D2 elder rule, [9] D1 boundary tracing, [10] D1
 * reduction (lazy mode: [9] is 0, [10] covers both), [11] output.  [6] and
 * [8] include the host's round trips between Borůvka rounds. */
dms_status dms_get_kernel_ms(dms_grid grid, float ms[12]);

/* Lower-link classification of every vertex and the id-ordered list of the
 * PL-critical vertices (the first step of the gradient), computed without
 * allocating any memory.  The paper has no counterpart: this entry point
 * exists for callers that cannot let a library call cudaMalloc -- for
 * example a process whose device memory is all handed to its own pool
 * allocator at start-up, a service running under a fixed per-request memory
 * budget, or a latency-critical pipeline where an allocation (which may
 * synchronise the device) would stall its other streams.
 *
 * Its scratch is one fixed array in the library's device memory, sized for
 * at most 2^28 vertices (about 1 MB); every GPU that loads the library holds
 * it until the process exits.  Grids with more vertices are rejected with
 * DMS_ERR_INVALID_ARG.  All calls share that array: calls that overlap on
 * the GPU (from several streams or threads) race and must be serialised by
 * the caller.  The first call on a device (with that device current) looks
 * up the array's address and uploads the star tables.
 *
 * values:       device pointer, nx*ny*nz elements of dtype, x fastest.
 * flags_out:    device pointer, nx*ny*nz bytes: low nibble = link index of
 *               the lowest lower neighbour (0xF: a minimum), bit 4 set for
 *               a PL-critical vertex (other bits 0).
 * critical_out: device pointer with room for cap int32: the ids of the
 *               PL-critical vertices in increasing order.
 * n_critical:   host pointer: their number (also set when cap is too small,
 *               in which case DMS_ERR_CAPACITY is returned and critical_out
 *               is not written).
 * stream:       cudaStream_t (NULL = legacy default); the call synchronises
 *               it.  NaN in the field -> DMS_ERR_NAN. */
dms_status dms_classify_static(const void *values, dms_dtype dtype, int64_t nx, int64_t ny,
                               int64_t nz, uint8_t *flags_out, int32_t *critical_out,
                               int64_t cap, int64_t *n_critical, void *stream);

/* Launch shapes and capacities of a handle, for an autotuner (values[k] in
 * this order; none changes a result, only its speed):
 *   DMS_TUNE_PLS_BLOCK        threads per block of ProcessLowerStars
 *                             (32..512, a multiple of 32; default 128)
 *   DMS_TUNE_TRACE_BLOCK      threads per block of the first D1 trace pass
 *                             (32..256, a multiple of 32; default 128)
 *   DMS_TUNE_TRACE_PER_SM     first-pass trace threads per SM (a multiple of
 *                             the block, <= 8192; default 2048)
 *   DMS_TUNE_TRACE_HEAP       first-pass trace heap entries per thread
 *                             (8..1024; default 48; larger traces retry with
 *                             16x more)
 *   DMS_TUNE_RED_BLOCK_BELOW  active columns below which a whole block
 *                             performs a column's additions (>= 0; -1, the
 *                             default: the larger of 4096 and one column
 *                             in 1600)
 *   DMS_TUNE_LAZY_HEAP        first-pass heap entries of a lazy advance
 *                             (8..1024; default 48)
 *   DMS_TUNE_LAZY_DENSITY     d1_mode 0 reduces lazily when there are fewer
 *                             2-saddle columns than vertices / this (1..4096;
 *                             default 32)
 *   DMS_TUNE_RED_ASYNC        1: below DMS_TUNE_RED_BLOCK_BELOW active columns
 *                             the traced reduction finishes in one
 *                             asynchronous pass (compare-and-swap ownership
 *                             and a device work queue); 0: in rounds
 *                             (default 1)
 *   DMS_TUNE_PLS_SORT         ProcessLowerStars in two passes with the stars
 *                             sorted by shape (lower-link mask) in between:
 *                             0 never, 1 when more than a quarter of the
 *                             vertices are critical (default), 2 always
 *   DMS_TUNE_D2_BESIDE_D0     1: D2's ascending walks run on a second stream of
 *                             the handle beside D0 (the paper's D0 || D2
 *                             tasks); 0: after D0 on the compute stream
 *                             (default 1)
 * dms_set_tuning checks every value and changes nothing when one is out of
 * range (DMS_ERR_INVALID_ARG); count must be DMS_TUNING_COUNT. */
enum {
    DMS_TUNE_PLS_BLOCK = 0, DMS_TUNE_TRACE_BLOCK, DMS_TUNE_TRACE_PER_SM, DMS_TUNE_TRACE_HEAP,
    DMS_TUNE_RED_BLOCK_BELOW, DMS_TUNE_LAZY_HEAP, DMS_TUNE_LAZY_DENSITY, DMS_TUNE_RED_ASYNC,
    DMS_TUNE_PLS_SORT, DMS_TUNE_D2_BESIDE_D0, DMS_TUNING_COUNT
};
dms_status dms_set_tuning(dms_grid grid, const int32_t *values, int count);
dms_status dms_get_tuning(dms_grid grid, int32_t *values, int count);

/* Frees every device and host resource of the handle. */
dms_status dms_grid_destroy(dms_grid grid);

/* Static description of a status code. */
const char *dms_status_string(dms_status status);

/* Test hook, host only (no GPU involved): copies the tables of the 14-vertex
 * Freudenthal star that the kernels use (link offsets, the star's triangles
 * and tetrahedra and their incidences; the layout of StarTables in
 * csrc/dms_common.cuh) into `out` when `bytes` is at least their size.
 * Returns that size, or -1 if the tables cannot be built.  Lets tests run the
 * lower-star code on the host against the oracle. */
int64_t dms_star_tables(void *out, int64_t bytes);

/* Test hook, host only (no GPU involved): copies the classification's table
 * of PL-regular lower links (bit m of word m / 32 set: a vertex whose lower
 * link vertices form mask m, in the link order of dms_star_tables, has no
 * critical cell) into `out` when `words` is at least its length (2^14 / 32).
 * Returns that length, or -1 if the tables cannot be built. */
int64_t dms_regular_table(uint32_t *out, int64_t words);

#ifdef __cplusplus
}
#endif

#endif /* DMS_H */
