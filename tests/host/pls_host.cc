// pls_host.cc -- the library's ProcessLowerStars source (csrc/dms_common.cuh)
// compiled for the host, so that tests compare it with the oracle's gradient
// without a GPU.  The CUDA bit intrinsics it calls get their host meaning
// here; everything else is the header as the kernels include it.
#include <cstdint>
#include <cstring>

static inline int __ffs(unsigned int x) { return __builtin_ffs((int)x); }
static inline int __ffsll(unsigned long long x) { return __builtin_ffsll((long long)x); }
static inline int __popc(unsigned int x) { return __builtin_popcount(x); }
static inline int __popcll(unsigned long long x) { return __builtin_popcountll(x); }
static inline unsigned int __float_as_uint(float f) {
    unsigned int u;
    memcpy(&u, &f, sizeof u);
    return u;
}
static inline long long __double_as_longlong(double d) {
    long long u;
    memcpy(&u, &d, sizeof u);
    return u;
}

#include "dms_common.cuh"   // -I the kernels' csrc/ (or a copy of it)

extern "C" int64_t harness_tables_size() { return (int64_t)sizeof(dms::StarTables); }

// ProcessLowerStars of one lower star: lower link mask L, rank[n] = position
// of lower link vertex n among the lower ones (0 = lowest).  out[0..3] =
// critical edges, triangles, tets, is-minimum; out[4..9] = the packed
// pairing (GradRec words).
extern "C" void harness_pls(const void *tables, uint32_t L, const uint8_t *rank, int64_t *out) {
    dms::StarTables S;
    memcpy(&S, tables, sizeof S);
    dms::PLSResult R;
    dms::GradRec G;
    dms::pls(S, (uint16_t)L, rank, R, &G);
    out[0] = R.crit_e;
    out[1] = (int64_t)R.crit_t;
    out[2] = R.crit_h;
    out[3] = R.is_min;
    for (int k = 0; k < 6; k++) out[4 + k] = (int64_t)G.w[k];
}

// The star layout: out[0..41] link offsets (dx, dy, dz per link vertex),
// out[42..113] the two link vertices of each star triangle, out[114..185]
// the three link vertices of each star tet.
extern "C" void harness_layout(const void *tables, int64_t *out) {
    dms::StarTables S;
    memcpy(&S, tables, sizeof S);
    int k = 0;
    for (int n = 0; n < dms::kLinks; n++) {
        out[k++] = S.dx[n]; out[k++] = S.dy[n]; out[k++] = S.dz[n];
    }
    for (int s = 0; s < dms::kTris; s++) { out[k++] = S.tri_v[s][0]; out[k++] = S.tri_v[s][1]; }
    for (int h = 0; h < dms::kTets; h++)
        for (int i = 0; i < 3; i++) out[k++] = S.tet_v[h][i];
}

// The star view the gradient kernels load for vertex v of an nx*ny*nz grid
// (load_star): out[0] present links, out[1] lower links, out[2] the descent
// link, out[3..16] the rank of each lower link.  dtype 0 uint16, 1 float32,
// 2 float64.  The grid's linear link offsets come from the star's offsets.
extern "C" void harness_load_star(const void *tables, int dtype, const void *values, int nx,
                                  int ny, int nz, int64_t v, int64_t *out) {
    dms::StarTables S;
    memcpy(&S, tables, sizeof S);
    dms::GridParams g;
    memset(&g, 0, sizeof g);
    g.nx = nx; g.ny = ny; g.nz = nz; g.n = (int64_t)nx * ny * nz; g.off = 0;
    for (int n = 0; n < dms::kLinks; n++) g.dlin[n] = S.dx[n] + nx * (S.dy[n] + ny * S.dz[n]);
    dms::StarView sv;
    if (dtype == 0) dms::load_star(S, g, (const uint16_t *)values, v, sv);
    else if (dtype == 1) dms::load_star(S, g, (const float *)values, v, sv);
    else dms::load_star(S, g, (const double *)values, v, sv);
    out[0] = sv.present;
    out[1] = sv.lower;
    out[2] = sv.descent;
    for (int n = 0; n < dms::kLinks; n++) out[3 + n] = sv.rank[n];
}

// The order keys (Key<T>::of) and NaN tests of the vertex values.
extern "C" uint64_t harness_key_f32(float f) { return dms::Key<float>::of(f); }
extern "C" uint64_t harness_key_f64(double d) { return dms::Key<double>::of(d); }
extern "C" int harness_nan_f32(float f) { return dms::Key<float>::nan(f); }
extern "C" int harness_nan_f64(double d) { return dms::Key<double>::nan(d); }
