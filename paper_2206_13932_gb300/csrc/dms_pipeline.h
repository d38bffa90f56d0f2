// dms_pipeline.h -- host-side pipeline of libdms (one grid, one stream).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dms.h"

namespace dms {

// A growable device allocation owned by the pipeline.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool ensure(size_t need);          // grows (never shrinks); false on OOM
    void release();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// Per-thread scratch of the lazy D1 advances: nt threads, each with a heap of
// hcap entries, a hash of hashcap entries and a generation word.
struct LazyScratch {
    DevBuf buf;
    int hcap = 0, hashcap = 0;
    int64_t nt = 0;
};

struct Pipeline {
    int64_t nx = 0, ny = 0, nz = 0, n = 0;
    dms_dtype dtype = DMS_F32;
    int64_t max_iters = 0;
    int virtual_max = 1;    // 1: the outer boundary is one virtual maximum (Sec. 5.2);
                            // 0: no virtual maximum (App. A)
    int generators = 0;     // 1: a 1-cycle generator per D1 pair (Sec. 8)
    DevBuf gen_out;         // the generator records of the last compute (int64)
    int64_t gen_words = 0;
    int d1_mode = 0;        // 0: by column density, 1: reduce columns (homology),
                            // 2: anti-transpose (cohomology), 3: lazy columns
                            // (propagation interleaved with the reduction)
    int d1_mode_used = 1;   // the mode the last compute ran
    int device = 0;

    // grid-sized state
    DevBuf values_dev;      // copy of host values (values_on_host = 1)
    DevBuf flags;           // u8 per vertex: descent link | critical flag
    DevBuf vrank;           // i32 per vertex: position among sorted critical vertices
    DevBuf grad;            // 48 B per vertex: memoised lower-star pairing
    DevBuf tile_cnt, tile_off;
    // critical-count-sized state
    DevBuf vc, vc_tmp, keys, keys_tmp, recs;
    DevBuf cnt[4], base[4];
    DevBuf c_vert[4], c_loc[4];
    DevBuf arc_a, arc_b, young, died, rowcol, flag_a, flag_b;
    DevBuf dc_keys, dc_par, dc_lab;   // elder-rule halving levels
    DevBuf bv_node, bv_msf, bv_arcs;  // elder rule: spanning-forest nodes, flags, arcs
    DevBuf d1_act, d1_next, d1_re, d1_stamp, d1_work;   // D1 reduction work lists
    DevBuf d1_row, d1_rowpaired;               // D1 result per column / row
    DevBuf d1_rowpos, d1_rowmap, d1_cocnt, d1_costart, d1_cofill;   // transpose
    DevBuf d1_colmap, d1_start, d1_len, d1_owner, d1_ovf, d1_pool, d1_scratch, d1_todo;
    DevBuf d1_rowcol;                          // D1: owner of each row with its list
    DevBuf d1_info, d1_queue, d1_aq;           // D1: asynchronous tail (lists, queue)
    DevBuf ord_k[4], ord_v[4], ord_h[2];       // vertex-id orders of walks (two slots); slot 0
                                               // also sorts stars for ProcessLowerStars
    DevBuf pls_ranks;                          // u64 per sorted star: its link ranks
    DevBuf d1_astamp;                          // lazy D1: last advance per column
    LazyScratch lz_small, lz_big;              // lazy D1: advance scratch
    DevBuf bx_buf[2];                          // lazy D1: block expansion scratch
    DevBuf out_pairs[3];
    // a batch: nf fields laid out one after another (field f at ids
    // field_off[f] ..), computed in one pass
    bool batch = false;
    int64_t nf = 1;
    std::vector<int64_t> shapes;      // nx, ny, nz per field
    std::vector<int64_t> field_off;   // nf + 1 offsets
    DevBuf fields_dev, field_of, field_off_dev, fmax_field;
    DevBuf out_field[3], bt_k[2], bt_v[2], bt_h[2], bt_cnt, out_tmp, batch_pofs[3];
    std::vector<int64_t> batch_off[3];   // per dimension: nf + 1 pair offsets
    DevBuf scan_tmp, scan_tmp2;   // scan partials: compute stream, second stream
    DevBuf arc2_a, arc2_b;        // D2 arcs (computed beside D0 on the second stream)
    DevBuf vcrit;                 // D1 trace: a word per critical vertex (rows among its edges)
    bool dense_grad = false;      // every gradient record was computed before the walks
    void *s2 = nullptr;           // cudaStream_t: D2's ascending walks run there beside D0
    void *ev_fork = nullptr, *ev_join = nullptr;   // cudaEvent_t between the two streams
    DevBuf dstat;           // device status words
    void *hstat = nullptr;  // pinned host mirror

    // launch shapes and capacities (dms_set_tuning; order of DMS_TUNE_*)
    int32_t tune[DMS_TUNING_COUNT] = {128, 128, 2048, 48, -1, 48, 32, 1, 1, 1};

    int64_t n_crit = 0, n_c[4] = {0, 0, 0, 0};
    int64_t n_pairs[3] = {0, 0, 0}, n_ess[4] = {0, 0, 0, 0};
    int64_t launches = 0, rounds_d0 = 0, rounds_d2 = 0, rounds_d1 = 0  /* D0/D2: halving levels */, d1_cols = 0;
    int64_t d1_overflow = 0, d1_additions = 0, d1_pool_used = 0, d1_pool_grows = 0;
    int64_t d1_io_read = 0, d1_io_written = 0;
    int64_t trace_toggles = 0, trace_expansions = 0, d1_longest_chain = 0;
    float stage_ms[8] = {0};
    float kernel_ms[12] = {0};
    void *kev[24] = {nullptr};   // cudaEvent_t pairs per kernel family
    void *sev[8] = {nullptr};    // cudaEvent_t stage boundaries
    bool has_result = false;
    uint64_t result_id = 0;   // bumped by every successful compute

    dms_status init(int64_t nx, int64_t ny, int64_t nz, dms_dtype dt, const dms_options *o);
    dms_status init_batch(int64_t nf, const int64_t *shapes, dms_dtype dt, const dms_options *o);
    dms_status init_common(const dms_options *o);
    dms_status set_batch(int64_t nf, const int64_t *shapes);
    dms_status compute(const void *values, int on_host, void *stream);
    dms_status reshape(int64_t nx, int64_t ny, int64_t nz);
    dms_status fetch(int dim, dms_pair *out, int64_t cap, int64_t *written, int out_is_device);
    dms_status fetch_generators(int64_t *out, int64_t cap, int64_t *written);
    // rows of output list dim: its finite pairs and infinite classes (the D2
    // list also holds the infinite classes of dimension 3)
    int64_t list_rows(int dim) const {
        return n_pairs[dim] + n_ess[dim] + (dim == 2 ? n_ess[3] : 0);
    }
    dms_status backward(int dim, uint64_t rid, const double *gbirth, const double *gdeath,
                        double *grad, void *stream);
    void destroy();
    std::vector<DevBuf *> buffers();   // every device buffer of the handle
    int64_t device_bytes();            // bytes they hold now
};

}  // namespace dms
