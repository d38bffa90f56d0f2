// dms_capi.cu -- the extern "C" entry points of libdms (declared in
// include/dms.h).  Argument checking and handle management only; the work is
// in dms_pipeline.cu.
#include <new>

#include "dms_pipeline.h"

struct dms_grid_s {
    dms::Pipeline p;
};

extern "C" {

dms_status dms_grid_create(int64_t nx, int64_t ny, int64_t nz, dms_dtype dtype,
                           const dms_options *opts, dms_grid *out) {
    if (!out) return DMS_ERR_INVALID_ARG;
    dms_grid g = new (std::nothrow) dms_grid_s;
    if (!g) return DMS_ERR_OOM;
    dms_status s = g->p.init(nx, ny, nz, dtype, opts);
    if (s != DMS_OK) {
        g->p.destroy();
        delete g;
        return s;
    }
    *out = g;
    return DMS_OK;
}

dms_status dms_batch_create(int64_t nfields, const int64_t *shapes, dms_dtype dtype,
                            const dms_options *opts, dms_grid *out) {
    if (!out || !shapes) return DMS_ERR_INVALID_ARG;
    dms_grid g = new (std::nothrow) dms_grid_s;
    if (!g) return DMS_ERR_OOM;
    dms_status s = g->p.init_batch(nfields, shapes, dtype, opts);
    if (s != DMS_OK) {
        g->p.destroy();
        delete g;
        return s;
    }
    *out = g;
    return DMS_OK;
}

dms_status dms_batch_reshape(dms_grid grid, int64_t nfields, const int64_t *shapes) {
    if (!grid || !shapes) return DMS_ERR_INVALID_ARG;
    return grid->p.set_batch(nfields, shapes);
}

dms_status dms_batch_offsets(dms_grid grid, int dim, int64_t *offsets) {
    if (!grid || !offsets || dim < 0 || dim > 2) return DMS_ERR_INVALID_ARG;
    const dms::Pipeline &p = grid->p;
    if (!p.batch || !p.has_result) return DMS_ERR_STATE;
    for (int64_t f = 0; f <= p.nf; f++) offsets[f] = p.batch_off[dim][f];
    return DMS_OK;
}

dms_status dms_grid_reshape(dms_grid grid, int64_t nx, int64_t ny, int64_t nz) {
    if (!grid) return DMS_ERR_INVALID_ARG;
    return grid->p.reshape(nx, ny, nz);
}

dms_status dms_compute_diagram(dms_grid grid, const void *values, int values_on_host,
                               void *stream) {
    if (!grid) return DMS_ERR_INVALID_ARG;
    return grid->p.compute(values, values_on_host, stream);
}

dms_status dms_get_counts(dms_grid grid, int64_t pairs[3], int64_t essential[4]) {
    if (!grid || !pairs || !essential) return DMS_ERR_INVALID_ARG;
    if (!grid->p.has_result) return DMS_ERR_STATE;
    for (int d = 0; d < 3; d++) pairs[d] = grid->p.n_pairs[d];
    for (int d = 0; d < 4; d++) essential[d] = grid->p.n_ess[d];
    return DMS_OK;
}

dms_status dms_fetch_pairs(dms_grid grid, int dim, dms_pair *out, int64_t cap, int64_t *written,
                           int out_is_device) {
    if (!grid) return DMS_ERR_INVALID_ARG;
    return grid->p.fetch(dim, out, cap, written, out_is_device);
}

dms_status dms_fetch_generators(dms_grid grid, int64_t *out, int64_t cap, int64_t *written) {
    if (!grid) return DMS_ERR_INVALID_ARG;
    return grid->p.fetch_generators(out, cap, written);
}

dms_status dms_get_result_id(dms_grid grid, uint64_t *result_id) {
    if (!grid || !result_id) return DMS_ERR_INVALID_ARG;
    if (!grid->p.has_result) return DMS_ERR_STATE;
    *result_id = grid->p.result_id;
    return DMS_OK;
}

dms_status dms_backward_pairs(dms_grid grid, int dim, uint64_t result_id,
                              const double *grad_birth, const double *grad_death,
                              double *grad_field, void *stream) {
    if (!grid) return DMS_ERR_INVALID_ARG;
    return grid->p.backward(dim, result_id, grad_birth, grad_death, grad_field, stream);
}

dms_status dms_get_stage_ms(dms_grid grid, float ms[8]) {
    if (!grid || !ms) return DMS_ERR_INVALID_ARG;
    if (!grid->p.has_result) return DMS_ERR_STATE;
    for (int k = 0; k < 8; k++) ms[k] = grid->p.stage_ms[k];
    return DMS_OK;
}

dms_status dms_get_stats(dms_grid grid, int64_t stats[16]) {
    if (!grid || !stats) return DMS_ERR_INVALID_ARG;
    if (!grid->p.has_result) return DMS_ERR_STATE;
    const dms::Pipeline &p = grid->p;
    stats[0] = p.n_crit;
    for (int d = 0; d < 4; d++) stats[1 + d] = p.n_c[d];
    stats[5] = p.launches;
    stats[6] = p.rounds_d0;
    stats[7] = p.rounds_d2;
    stats[8] = p.rounds_d1;
    stats[9] = p.d1_cols;
    stats[10] = p.d1_overflow;
    stats[11] = p.d1_additions;
    stats[12] = p.d1_pool_used;
    stats[13] = p.d1_pool_grows;
    stats[14] = p.d1_io_read;
    stats[15] = p.d1_io_written;
    return DMS_OK;
}

dms_status dms_get_work(dms_grid grid, int64_t work[4]) {
    if (!grid || !work) return DMS_ERR_INVALID_ARG;
    if (!grid->p.has_result) return DMS_ERR_STATE;
    work[0] = grid->p.trace_toggles;
    work[1] = grid->p.trace_expansions;
    work[2] = grid->p.d1_longest_chain;
    work[3] = 0;
    return DMS_OK;
}

dms_status dms_get_device_bytes(dms_grid grid, int64_t *bytes) {
    if (!grid || !bytes) return DMS_ERR_INVALID_ARG;
    *bytes = grid->p.device_bytes();
    return DMS_OK;
}

dms_status dms_get_kernel_ms(dms_grid grid, float ms[12]) {
    if (!grid || !ms) return DMS_ERR_INVALID_ARG;
    if (!grid->p.has_result) return DMS_ERR_STATE;
    for (int k = 0; k < 12; k++) ms[k] = grid->p.kernel_ms[k];
    return DMS_OK;
}

dms_status dms_set_tuning(dms_grid grid, const int32_t *v, int count) {
    if (!grid || !v || count != DMS_TUNING_COUNT) return DMS_ERR_INVALID_ARG;
    // the trace kernel is compiled for at most 256 threads per block
    auto block_ok = [](int32_t b, int32_t most) { return b >= 32 && b <= most && b % 32 == 0; };
    if (!block_ok(v[DMS_TUNE_PLS_BLOCK], 512) || !block_ok(v[DMS_TUNE_TRACE_BLOCK], 256))
        return DMS_ERR_INVALID_ARG;
    if (v[DMS_TUNE_PLS_SORT] < 0 || v[DMS_TUNE_PLS_SORT] > 2) return DMS_ERR_INVALID_ARG;
    const int32_t per_sm = v[DMS_TUNE_TRACE_PER_SM];
    if (per_sm < v[DMS_TUNE_TRACE_BLOCK] || per_sm > 8192 || per_sm % v[DMS_TUNE_TRACE_BLOCK])
        return DMS_ERR_INVALID_ARG;
    if (v[DMS_TUNE_TRACE_HEAP] < 8 || v[DMS_TUNE_TRACE_HEAP] > 1024) return DMS_ERR_INVALID_ARG;
    if (v[DMS_TUNE_RED_BLOCK_BELOW] < -1) return DMS_ERR_INVALID_ARG;
    if (v[DMS_TUNE_LAZY_HEAP] < 8 || v[DMS_TUNE_LAZY_HEAP] > 1024) return DMS_ERR_INVALID_ARG;
    if (v[DMS_TUNE_LAZY_DENSITY] < 1 || v[DMS_TUNE_LAZY_DENSITY] > 4096) return DMS_ERR_INVALID_ARG;
    if (v[DMS_TUNE_RED_ASYNC] != 0 && v[DMS_TUNE_RED_ASYNC] != 1) return DMS_ERR_INVALID_ARG;
    if (v[DMS_TUNE_D2_BESIDE_D0] != 0 && v[DMS_TUNE_D2_BESIDE_D0] != 1) return DMS_ERR_INVALID_ARG;
    for (int k = 0; k < DMS_TUNING_COUNT; k++) grid->p.tune[k] = v[k];
    return DMS_OK;
}

dms_status dms_get_tuning(dms_grid grid, int32_t *v, int count) {
    if (!grid || !v || count != DMS_TUNING_COUNT) return DMS_ERR_INVALID_ARG;
    for (int k = 0; k < DMS_TUNING_COUNT; k++) v[k] = grid->p.tune[k];
    return DMS_OK;
}

dms_status dms_grid_destroy(dms_grid grid) {
    if (!grid) return DMS_ERR_INVALID_ARG;
    grid->p.destroy();
    delete grid;
    return DMS_OK;
}

const char *dms_status_string(dms_status status) {
    switch (status) {
        case DMS_OK: return "ok";
        case DMS_ERR_INVALID_ARG: return "invalid argument";
        case DMS_ERR_NAN: return "the field holds a NaN";
        case DMS_ERR_OOM: return "out of memory";
        case DMS_ERR_CUDA: return "CUDA runtime error";
        case DMS_ERR_ITER_LIMIT: return "a bounded device loop reached its limit";
        case DMS_ERR_STATE: return "no result available or inconsistent state";
        case DMS_ERR_CAPACITY: return "capacity exceeded";
    }
    return "unknown status";
}

}  // extern "C"
