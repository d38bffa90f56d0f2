// dms_pipeline.cu -- the device pipeline of libdms.
//
// Stages (the paper's order, Sec. 7.1):
//   gradient   classify every vertex by its lower link (HBM-bound stencil),
//              compact the PL-critical vertices in id order, sort them by
//              value, run ProcessLowerStars on each (Alg. 2: the critical
//              simplices C0..C3, already in lexicographic order);
//   D0         descend from both ends of each critical edge along the
//              vertex->edge vectors to two minima (Sec. 5.1 (a)-(b)) and pair
//              the arcs of that graph by the elder rule (Sec. 5.1 (c)-(d));
//   D2         ascend from each critical triangle through tet->triangle
//              vectors to critical tets or the virtual maximum (Sec. 5.2) and
//              pair in decreasing order;
//   D1         trace the Morse boundary of each 2-saddle not paired in D2 over
//              the 1-saddles not paired in D0 and reduce those columns
//              (Alg. 3 restricted, Sec. 4.2 (b), Sec. 6);
//   output     pairs and infinite classes (Sec. 6).
#include <algorithm>
#include <chrono>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dms_common.cuh"
#include "dms_pipeline.h"

namespace dms {

__device__ StarTables g_star;
__device__ uint32_t g_regular[(1 << kLinks) / 32];   // bit m: lower mask m is PL-regular

enum : uint32_t { kErrNan = 1, kErrIter = 2, kErrCap = 4, kErrState = 8 };
constexpr int32_t kNoOwner = 0x7F7F7F7F;   // memset(0x7F) fill of the pivot owners

struct DevStatus {
    uint32_t err;
    uint32_t pad;
    unsigned long long maxkey;     // largest vertex key
    long long total[4];            // scan totals
    long long parts[8];            // output part sizes
    long long red_io[2];           // D1 additions: bytes read, bytes written
    int changed;                   // D1: columns changed this round
    unsigned long long pool_top;   // D1 column pool bump pointer
    long long misc[4];
    long long bx[4];               // block expansions: nodes, levels (discovery, order), columns
    unsigned long long trace_next; // D1 trace: next column to take
    unsigned long long red_work;   // D1 reduction round: columns that add this round
    unsigned long long trace_work[2];   // D1 trace: edges toggled, edges expanded
};

// Record of a critical vertex after ProcessLowerStars.
struct CritRec {
    uint64_t crit_t;      // critical star triangles
    uint64_t ranks;       // 4-bit rank of each lower link vertex (0xF: not lower)
    uint32_t crit_h;      // critical star tets
    uint16_t crit_e;      // critical star edges
    uint8_t is_min, pad;
};

struct HeapEnt { unsigned long long hi, lo; };
struct HashEnt {
    unsigned long long key;
    int32_t gen;
    uint32_t info;   // row (bits 0-23... see kRowBits), pair (6 bits), kind (2), parity (1)
};
// info packing: bits 0-22 unused when kind = reg; a row index needs up to 31
// bits, so rows are kept apart in the per-thread row list and info holds the
// position in that list
__device__ __forceinline__ uint32_t hinfo(uint32_t aux, int pair, int kind, int parity) {
    return (aux & 0x7FFFFF) | ((uint32_t)pair << 23) | ((uint32_t)kind << 29) | ((uint32_t)parity << 31);
}
__device__ __forceinline__ uint32_t hinfo_aux(uint32_t i) { return i & 0x7FFFFF; }
__device__ __forceinline__ int hinfo_pair(uint32_t i) { return (i >> 23) & 63; }
__device__ __forceinline__ int hinfo_kind(uint32_t i) { return (i >> 29) & 3; }
__device__ __forceinline__ int hinfo_parity(uint32_t i) { return (i >> 31) & 1; }
enum { kKindRow = 1, kKindReg = 2 };

// ------------------------------------------------------------ host tables

static bool build_star_tables(StarTables &S) {
    memset(&S, 0, sizeof S);
    int d[kLinks][3];
    for (int n = 0; n < kLinks; n++) {
        int o = n % 7 + 1, sg = n < 7 ? 1 : -1;
        d[n][0] = sg * (o & 1); d[n][1] = sg * ((o >> 1) & 1); d[n][2] = sg * ((o >> 2) & 1);
        S.dx[n] = (int8_t)d[n][0]; S.dy[n] = (int8_t)d[n][1]; S.dz[n] = (int8_t)d[n][2];
        S.edge_anchor[n] = (int8_t)(n < 7 ? -1 : n);
        S.edge_type[n] = (int8_t)(o - 1);
        for (int a = 0; a < 3; a++) {
            if (d[n][a] < 0) S.neg[a] |= (uint16_t)(1u << n);
            if (d[n][a] > 0) S.pos[a] |= (uint16_t)(1u << n);
        }
    }
    for (int i = 0; i < 27; i++) S.link_of_dc[i] = -1;
    for (int n = 0; n < kLinks; n++)
        S.link_of_dc[(d[n][0] + 1) + 3 * (d[n][1] + 1) + 9 * (d[n][2] + 1)] = (int8_t)n;
    for (int a = 0; a < kLinks; a++)
        for (int b = 0; b < kLinks; b++) S.tri_of_pair[a][b] = -1;

    static const int TRI_B[12] = {3, 3, 5, 5, 6, 6, 7, 7, 7, 7, 7, 7};
    static const int TRI_A[12] = {1, 2, 1, 4, 2, 4, 1, 2, 3, 4, 5, 6};
    static const int TET_A[6] = {1, 1, 2, 2, 4, 4};
    static const int TET_B[6] = {3, 5, 3, 6, 5, 6};

    // points: index -1 = the centre (0,0,0), otherwise a link vertex
    auto pt = [&](int l, int k) { return l < 0 ? 0 : d[l][k]; };
    // is {centre} + links a chain of the componentwise order within one cube?
    // returns the anchor (min point) and the offset masks of the others.
    auto chain = [&](const int *ls, int cnt, int *anchor, int *offs) -> bool {
        int pts[4] = {-1, ls[0], cnt > 1 ? ls[1] : -1, cnt > 2 ? ls[2] : -1};
        int m = cnt + 1;
        // sort by coordinate sum
        for (int i = 1; i < m; i++)
            for (int j = i; j > 0; j--) {
                int sa = pt(pts[j - 1], 0) + pt(pts[j - 1], 1) + pt(pts[j - 1], 2);
                int sb = pt(pts[j], 0) + pt(pts[j], 1) + pt(pts[j], 2);
                if (sa > sb) std::swap(pts[j - 1], pts[j]);
            }
        for (int i = 0; i + 1 < m; i++)
            for (int k = 0; k < 3; k++)
                if (pt(pts[i], k) > pt(pts[i + 1], k)) return false;
        for (int k = 0; k < 3; k++) {
            int e = pt(pts[m - 1], k) - pt(pts[0], k);
            if (e < 0 || e > 1) return false;
        }
        *anchor = pts[0];
        for (int i = 1; i < m; i++) {
            int o = 0;
            for (int k = 0; k < 3; k++) o |= (pt(pts[i], k) - pt(pts[0], k)) << k;
            offs[i - 1] = o;
        }
        return true;
    };
    int nt = 0, nh = 0;
    for (int a = 0; a < kLinks; a++)
        for (int b = a + 1; b < kLinks; b++) {
            int ls[2] = {a, b}, anc, offs[2];
            if (!chain(ls, 2, &anc, offs)) continue;
            if (nt >= kTris) return false;
            S.tri_v[nt][0] = (uint8_t)a; S.tri_v[nt][1] = (uint8_t)b;
            S.tri_mask[nt] = (uint16_t)((1u << a) | (1u << b));
            S.tri_of_pair[a][b] = S.tri_of_pair[b][a] = (int8_t)nt;
            S.tri_anchor[nt] = (int8_t)anc;
            int lo = offs[0], hi = offs[1];
            if (__builtin_popcount(lo) > __builtin_popcount(hi)) std::swap(lo, hi);
            S.tri_type[nt] = -1;
            for (int k = 0; k < 12; k++)
                if (TRI_A[k] == lo && TRI_B[k] == hi) S.tri_type[nt] = (int8_t)k;
            if (S.tri_type[nt] < 0) return false;
            S.tris_of_link[a] |= 1ull << nt;
            S.tris_of_link[b] |= 1ull << nt;
            nt++;
        }
    for (int a = 0; a < kLinks; a++)
        for (int b = a + 1; b < kLinks; b++)
            for (int c = b + 1; c < kLinks; c++) {
                int ls[3] = {a, b, c}, anc, offs[3];
                if (!chain(ls, 3, &anc, offs)) continue;
                if (nh >= kTets) return false;
                S.tet_v[nh][0] = (uint8_t)a; S.tet_v[nh][1] = (uint8_t)b; S.tet_v[nh][2] = (uint8_t)c;
                S.tet_mask[nh] = (uint16_t)((1u << a) | (1u << b) | (1u << c));
                S.tet_f[nh][0] = (uint8_t)S.tri_of_pair[a][b];
                S.tet_f[nh][1] = (uint8_t)S.tri_of_pair[a][c];
                S.tet_f[nh][2] = (uint8_t)S.tri_of_pair[b][c];
                S.tet_anchor[nh] = (int8_t)anc;
                int one = 0, two = 0;
                for (int i = 0; i < 3; i++) {
                    if (__builtin_popcount(offs[i]) == 1) one = offs[i];
                    if (__builtin_popcount(offs[i]) == 2) two = offs[i];
                }
                S.tet_type[nh] = -1;
                for (int k = 0; k < 6; k++)
                    if (TET_A[k] == one && TET_B[k] == two) S.tet_type[nh] = (int8_t)k;
                if (S.tet_type[nh] < 0) return false;
                for (int i = 0; i < 3; i++) {
                    S.tets_of_link[S.tet_v[nh][i]] |= 1u << nh;
                    S.tets_of_tri[S.tet_f[nh][i]] |= 1u << nh;
                }
                nh++;
            }
    return nt == kTris && nh == kTets;
}

// Lower mask m is PL-regular iff the subcomplex of the link induced by m is
// non-empty and acyclic (reduced Betti numbers all zero).  Robins et al.'s
// gradient puts critical cells exactly where the lower link has homology.
static void build_regular_lut(const StarTables &S, std::vector<uint32_t> &lut) {
    lut.assign((1 << kLinks) / 32, 0);
    for (int m = 0; m < (1 << kLinks); m++) {
        int parent[kLinks];
        for (int i = 0; i < kLinks; i++) parent[i] = i;
        auto find = [&](int a) { while (parent[a] != a) a = parent[a] = parent[parent[a]]; return a; };
        int V = __builtin_popcount(m), E = 0, F = 0;
        for (int s = 0; s < kTris; s++)
            if ((S.tri_mask[s] & m) == S.tri_mask[s]) {
                E++;
                int a = find(S.tri_v[s][0]), b = find(S.tri_v[s][1]);
                if (a != b) parent[a] = b;
            }
        for (int h = 0; h < kTets; h++)
            if ((S.tet_mask[h] & m) == S.tet_mask[h]) F++;
        int b0 = 0;
        for (int i = 0; i < kLinks; i++)
            if ((m >> i & 1) && find(i) == i) b0++;
        int b2 = m == kAllLinks ? 1 : 0;
        int chi = V - E + F;
        int b1 = b0 - chi + b2;
        bool regular = V > 0 && b0 == 1 && b1 == 0 && b2 == 0;
        if (regular) lut[m >> 5] |= 1u << (m & 31);
    }
}

// ------------------------------------------------------------- utilities

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Local index of critical cell `loc` of dimension `dim` among the critical
// cells of that dimension of the same vertex, in lexicographic (G) order.
__device__ __forceinline__ int local_index(const StarTables &S, const CritRec &rec, int dim,
                                           int loc) {
    uint8_t r[kLinks];
    unpack_ranks(rec.ranks, r);
    int k = 0;
    if (dim == 1) {
        uint16_t c = code_edge(r, loc);
        for (uint16_t m = rec.crit_e; m; m &= m - 1) k += code_edge(r, __ffs(m) - 1) < c;
    } else if (dim == 2) {
        uint16_t c = code_tri(S, r, loc);
        for (uint64_t m = rec.crit_t; m; m &= m - 1) k += code_tri(S, r, __ffsll(m) - 1) < c;
    } else {
        uint16_t c = code_tet(S, r, loc);
        for (uint32_t m = rec.crit_h; m; m &= m - 1) k += code_tet(S, r, __ffs(m) - 1) < c;
    }
    return k;
}

__device__ __forceinline__ int64_t edge_id(const StarTables &S, const GridParams &g, int64_t x,
                                           int n) {
    int64_t anchor = S.edge_anchor[n] < 0 ? x : x + g.dlin[S.edge_anchor[n]];
    return 7 * anchor + S.edge_type[n];
}
__device__ __forceinline__ int64_t tri_id(const StarTables &S, const GridParams &g, int64_t x,
                                          int s) {
    int64_t anchor = S.tri_anchor[s] < 0 ? x : x + g.dlin[S.tri_anchor[s]];
    return 12 * anchor + S.tri_type[s];
}
__device__ __forceinline__ int64_t tet_id(const StarTables &S, const GridParams &g, int64_t x,
                                          int h) {
    int64_t anchor = S.tet_anchor[h] < 0 ? x : x + g.dlin[S.tet_anchor[h]];
    return 6 * anchor + S.tet_type[h];
}

// ------------------------------------------------------------------ scan

constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
    __shared__ int ws[kScanThreads / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int pre = 0, tot = 0;
    for (int i = 0; i < kScanThreads / 32; i++) {
        if (i < w) pre += ws[i];
        tot += ws[i];
    }
    __syncthreads();
    *total = tot;
    return pre + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partial(const int32_t *__restrict__ in,
                                                               int64_t n, int32_t *partial) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    int tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int32_t *__restrict__ in,
                                                             int32_t *out, int64_t n,
                                                             const int32_t *__restrict__ off,
                                                             long long *total) {
    __shared__ int tile[kScanTile];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        tile[k * kScanThreads + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    int loc[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; k++) { loc[k] = tile[threadIdx.x * kScanItems + k]; s += loc[k]; }
    int tot;
    int pre = block_exclusive_scan(s, &tot) + (off ? off[blockIdx.x] : 0);
    for (int k = 0; k < kScanItems; k++) { tile[threadIdx.x * kScanItems + k] = pre; pre += loc[k]; }
    __syncthreads();
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = tile[k * kScanThreads + threadIdx.x];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1)
        *total = (long long)pre;
}

// --------------------------------------------------- stage 1: classification

constexpr int kClsThreads = 256, kClsItems = 8, kClsTile = kClsThreads * kClsItems;

// ---- the tier-1 stencil, register-tiled
//
// A thread classifies a run of K = 16/sizeof(T) consecutive vertices of one
// row (x fastest).  Interior runs (all 14 neighbours present, 16-byte
// aligned rows) load the 7 rows they need as 16-byte vectors plus the two
// edge values and index every neighbour statically; other runs use the
// per-vertex path.  A block covers R whole consecutive rows, i.e. a
// contiguous id range (a tile of R*nx vertices), so that the ordered
// compaction can follow.  Link id order (used for ties): -7..-1, +1..+7.

// per-vertex path (boundary runs)
template <typename T>
__device__ __forceinline__ uint8_t classify_vertex(const StarTables &S, const GridParams &g,
                                                   const uint32_t *lut, const T *__restrict__ values,
                                                   int64_t v, int cx, int cy, int cz,
                                                   typename Key<T>::K &kv) {
    using K = typename Key<T>::K;
    uint16_t pres = present_links(S, g, cx, cy, cz);
    kv = Key<T>::of(values[v]);
    uint16_t lower = 0;
    K best = 0;
    int bn = -1;
#pragma unroll
    for (int n = 0; n < kLinks; n++) {
        if (pres >> n & 1) {
            K kn = Key<T>::of(values[v + g.dlin[n]]);
            bool lo = kn < kv || (kn == kv && n >= 7);
            if (lo) {
                lower |= (uint16_t)(1u << n);
                if (bn < 0 || kn < best || (kn == best && g.dlin[n] < g.dlin[bn])) {
                    best = kn;
                    bn = n;
                }
            }
        }
    }
    bool crit = !((lut[lower >> 5] >> (lower & 31)) & 1);
    return (uint8_t)((bn < 0 ? kNoDescent : bn) | (crit ? kFlagCritical : 0));
}

template <typename T> struct VecOf;
template <> struct VecOf<uint16_t> { static constexpr int K = 8; };
template <> struct VecOf<float> { static constexpr int K = 4; };
template <> struct VecOf<double> { static constexpr int K = 2; };

template <typename T>
__global__ void __launch_bounds__(kClsThreads)
    k_classify2(const T *__restrict__ values, GridParams g, int rows_per_block, int runs_per_row,
                int aligned, uint8_t *__restrict__ flags, int32_t *__restrict__ tile_cnt,
                DevStatus *st) {
    using Kt = typename Key<T>::K;
    constexpr int K = VecOf<T>::K;
    __shared__ uint32_t lut[(1 << kLinks) / 32];
    __shared__ int scnt[kClsThreads / 32];
    __shared__ unsigned long long smax[kClsThreads / 32];
    for (int i = threadIdx.x; i < (1 << kLinks) / 32; i += kClsThreads) lut[i] = g_regular[i];
    __syncthreads();
    const StarTables &S = g_star;
    const int64_t nrows = (int64_t)g.ny * g.nz;
    const int64_t row0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t plane = (int64_t)g.nx * g.ny;
    int cnt = 0;
    Kt kmax = 0;
    bool bad = false;
    for (int s = threadIdx.x; s < rows_per_block * runs_per_row; s += kClsThreads) {
        const int64_t row = row0 + s / runs_per_row;
        if (row >= nrows) break;
        const int x0 = (s % runs_per_row) * K;
        const int cy = (int)(row % g.ny), cz = (int)(row / g.ny);
        const int64_t base = row * g.nx + x0;
        // y/z-interior rows take the fast path (uniform across a warp, which
        // covers one row); x-edge vertices are masked inside it
        const bool interior = aligned && cy >= 1 && cy <= g.ny - 2 && cz >= 1 && cz <= g.nz - 2;
        const bool xlo = x0 == 0, xhi = x0 + K >= g.nx;
        uint8_t f[K];
        if (interior) {
            // rows: 0 (0,0) 1 (+y) 2 (-y) 3 (+z) 4 (-z) 5 (+y+z) 6 (-y-z); values x0-1 .. x0+K
            Kt r[7][K + 2];
            const int64_t roff[7] = {0, g.nx, -(int64_t)g.nx, plane, -plane, g.nx + plane,
                                     -(int64_t)g.nx - plane};
#pragma unroll
            for (int q = 0; q < 7; q++) {
                const T *p = values + base + roff[q];
                union { uint4 u; T t[K]; } vec;
                vec.u = __ldg((const uint4 *)p);
                r[q][0] = xlo ? Kt(0) : Key<T>::of(__ldg(p - 1));
#pragma unroll
                for (int i = 0; i < K; i++) {
                    r[q][i + 1] = Key<T>::of(vec.t[i]);
                    if (q == 0) bad |= Key<T>::nan(vec.t[i]);
                }
                r[q][K + 1] = xhi ? Kt(0) : Key<T>::of(__ldg(p + K));
            }
#pragma unroll
            for (int i = 0; i < K; i++) {
                const Kt kv = r[0][i + 1];
                // neighbours in id order -7 -6 -5 -4 -3 -2 -1 +1 .. +7 with their link
                // index (o-1 for +o, o+6 for -o)
                const Kt nb[14] = {r[6][i], r[6][i + 1], r[4][i], r[4][i + 1], r[2][i], r[2][i + 1],
                                   r[0][i], r[0][i + 2], r[1][i + 1], r[1][i + 2], r[3][i + 1],
                                   r[3][i + 2], r[5][i + 1], r[5][i + 2]};
                constexpr int link[14] = {13, 12, 11, 10, 9, 8, 7, 0, 1, 2, 3, 4, 5, 6};
                uint32_t lower = 0;
                int bn = kNoDescent;
                // absent x neighbours: -x links (q 0 2 4 6) at x = 0, +x links
                // (q 7 9 11 13) at x = nx-1
                const bool nox_lo = xlo && i == 0, nox_hi = xhi && x0 + i == g.nx - 1;
                if constexpr (sizeof(Kt) == 4 && sizeof(T) == 2) {
                    // 16-bit values: key = value << 4 | position in id order (-7..-1 at
                    // 0..6, +1..+7 at 8..14), centre = value << 4 | 7.  A neighbour is
                    // lower iff its key is smaller (ties resolved by id), and the lowest
                    // lower neighbour is the smallest key.
                    const uint32_t c = (kv << 4) | 7u;
                    uint32_t mn = 0xFFFFFFFFu;
#pragma unroll
                    for (int q = 0; q < 14; q++) {
                        const bool absent = ((q == 0 || q == 2 || q == 4 || q == 6) && nox_lo) ||
                                            ((q == 7 || q == 9 || q == 11 || q == 13) && nox_hi);
                        const uint32_t key = absent ? 0xFFFFFFFFu
                                                    : (((uint32_t)nb[q] << 4) | (uint32_t)(q < 7 ? q : q + 1));
                        lower |= (uint32_t)(key < c) << link[q];
                        mn = key < mn ? key : mn;
                    }
                    if (mn < c) {
                        const uint32_t pos = mn & 15u;
                        // position -> link index: 0..6 -> 13..7, 8..14 -> 0..6
                        bn = pos < 7 ? 13 - (int)pos : (int)pos - 8;
                    }
                } else {
                    Kt best = kv;
#pragma unroll
                    for (int q = 0; q < 14; q++) {
                        const bool absent = ((q == 0 || q == 2 || q == 4 || q == 6) && nox_lo) ||
                                            ((q == 7 || q == 9 || q == 11 || q == 13) && nox_hi);
                        const bool lo = !absent && (q < 7 ? nb[q] <= kv : nb[q] < kv);
                        lower |= (uint32_t)lo << link[q];
                        // in id order, strict-less keeps the smallest id among equal values
                        const bool take = lo && (bn == kNoDescent || nb[q] < best);
                        best = take ? nb[q] : best;
                        bn = take ? link[q] : bn;
                    }
                }
                const bool crit = !((lut[lower >> 5] >> (lower & 31)) & 1);
                f[i] = (uint8_t)(bn | (crit ? kFlagCritical : 0));
                cnt += crit;
                kmax = kv > kmax ? kv : kmax;
            }
            if constexpr (K == 8) {
                *(uint2 *)(flags + base) = make_uint2(
                    f[0] | (f[1] << 8) | (f[2] << 16) | ((uint32_t)f[3] << 24),
                    f[4] | (f[5] << 8) | (f[6] << 16) | ((uint32_t)f[7] << 24));
            } else if constexpr (K == 4) {
                *(uint32_t *)(flags + base) =
                    f[0] | (f[1] << 8) | (f[2] << 16) | ((uint32_t)f[3] << 24);
            } else {
                *(uint16_t *)(flags + base) = (uint16_t)(f[0] | (f[1] << 8));
            }
        } else {
            for (int i = 0; i < K && x0 + i < g.nx; i++) {
                Kt kv;
                const uint8_t fl = classify_vertex<T>(S, g, lut, values, base + i, x0 + i, cy, cz, kv);
                bad |= Key<T>::nan(values[base + i]);
                flags[base + i] = fl;
                cnt += (fl & kFlagCritical) != 0;
                kmax = kv > kmax ? kv : kmax;
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long km = kmax;
    for (int o = 16; o; o >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        unsigned long long y = __shfl_down_sync(0xffffffffu, km, o);
        km = y > km ? y : km;
    }
    if (lane == 0) { scnt[w] = cnt; smax[w] = km; }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&st->err, kErrNan);
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        unsigned long long m = 0;
        for (int i = 0; i < kClsThreads / 32; i++) { c += scnt[i]; m = smax[i] > m ? smax[i] : m; }
        tile_cnt[blockIdx.x] = c;
        atomicMax(&st->maxkey, m);
    }
}

// Critical vertex ids of a tile of `tile` consecutive ids, in increasing id
// order, at the tile's offset.
__global__ void __launch_bounds__(kClsThreads)
    k_compact2(const uint8_t *__restrict__ flags, int64_t n, int64_t tile,
               const int32_t *__restrict__ tile_off, int32_t *__restrict__ vc) {
    __shared__ int ws[kClsThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * tile;
    const int64_t end = base + tile < n ? base + tile : n;
    int off = tile_off[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t v0 = base; v0 < end; v0 += kClsThreads) {
        const int64_t v = v0 + threadIdx.x;
        const bool c = v < end && (flags[v] & kFlagCritical);
        const unsigned b = __ballot_sync(0xffffffffu, c);
        if (lane == 0) ws[w] = __popc(b);
        __syncthreads();
        int pre = 0, tot = 0;
        for (int i = 0; i < kClsThreads / 32; i++) { if (i < w) pre += ws[i]; tot += ws[i]; }
        if (c) vc[off + pre + __popc(b & lanemask_lt())] = (int32_t)v;
        off += tot;
        __syncthreads();
    }
}

// The tier-1 classification of a batch: blocks of kClsTile consecutive ids
// (the tiles of k_compact2) over all fields, each vertex with the grid of
// its field; also the largest key of each field (its infinite classes die
// there).
template <typename T>
__global__ void __launch_bounds__(kClsThreads)
    k_classify_batch(const T *__restrict__ values, Geo<true> geo, int64_t n,
                     uint8_t *__restrict__ flags, int32_t *__restrict__ tile_cnt,
                     unsigned long long *fmax_field, DevStatus *st) {
    __shared__ uint32_t lut[(1 << kLinks) / 32];
    __shared__ int scnt[kClsThreads / 32];
    for (int i = threadIdx.x; i < (1 << kLinks) / 32; i += kClsThreads) lut[i] = g_regular[i];
    __syncthreads();
    const StarTables &S = g_star;
    const int64_t base = (int64_t)blockIdx.x * kClsTile;
    int cnt = 0, cur = -1;
    unsigned long long cmax = 0;
    bool bad = false;
    for (int k = 0; k < kClsItems; k++) {
        const int64_t v = base + (int64_t)k * kClsThreads + threadIdx.x;
        if (v >= n) break;
        const int f = geo.field(v);
        const GridParams &g = geo.fields[f];
        int cx, cy, cz;
        coords(g, v, cx, cy, cz);
        typename Key<T>::K kv;
        const uint8_t fl = classify_vertex<T>(S, g, lut, values, v, cx, cy, cz, kv);
        bad |= Key<T>::nan(values[v]);
        flags[v] = fl;
        cnt += (fl & kFlagCritical) != 0;
        if (f != cur) {
            if (cur >= 0) atomicMax(&fmax_field[cur], cmax);
            cur = f;
            cmax = 0;
        }
        cmax = (unsigned long long)kv > cmax ? (unsigned long long)kv : cmax;
    }
    if (cur >= 0) atomicMax(&fmax_field[cur], cmax);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0) scnt[w] = cnt;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&st->err, kErrNan);
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int i = 0; i < kClsThreads / 32; i++) c += scnt[i];
        tile_cnt[blockIdx.x] = c;
    }
}

// field index of every vertex of a batch (offsets: nf + 1 ascending ids)
__global__ void k_field_of(const int64_t *__restrict__ offsets, int nf, int64_t n,
                           uint16_t *field_of) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int lo = 0, hi = nf - 1;
    while (lo < hi) {            // the last field whose offset is <= v
        const int mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    field_of[v] = (uint16_t)lo;
}

// pairs per field (batch output)
__global__ void k_field_count(const int32_t *__restrict__ ofield, int64_t n, int32_t *cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[ofield[i]], 1);
}

// out[i] = in[perm[i]]
__global__ void k_gather_pairs(const dms_pair *__restrict__ in, const int32_t *__restrict__ perm,
                               int64_t n, dms_pair *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[perm[i]];
}

// ----------------------------------- stage 2: stable LSD radix sort by key

constexpr int kRsThreads = 256, kRsWarps = kRsThreads / 32, kRsPerWarp = 512,
              kRsTile = kRsWarps * kRsPerWarp;

template <typename T>
__global__ void k_gather_keys(const T *__restrict__ values, const int32_t *__restrict__ vc,
                              int64_t nc, typename Key<T>::K *keys) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) keys[i] = Key<T>::of(values[vc[i]]);
}

// keys[i] = vertex of item i (vert[idx[i]], or vert[i]), vals[i] = i: the
// input of a radix sort that puts items in vertex-id order
__global__ void k_gather_vid(const int32_t *__restrict__ vert, const int32_t *__restrict__ idx,
                             int64_t n, uint32_t *keys, int32_t *vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = (uint32_t)vert[idx ? idx[i] : i];
    vals[i] = (int32_t)i;
}

template <typename K>
__global__ void __launch_bounds__(kRsThreads)
    k_rs_hist(const K *__restrict__ keys, int64_t n, int shift, int32_t *hist, int ntiles) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int k = threadIdx.x; k < kRsTile; k += kRsThreads) {
        int64_t i = base + k;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// One stable LSD pass: the items of a tile of kRsTile go to their digit's
// run, after the runs of the earlier tiles (hoff: the scanned histograms).
// Staged (32-bit keys only): the tile is first ordered by digit in shared
// memory, so that the writes of a warp go to a few consecutive runs instead
// of 32 scattered positions.  It takes 43 KB of shared memory a block, which
// is why the sorts that run beside latency-bound walks on another stream
// use the unstaged form (their L1 would shrink).
template <typename K, bool kStaged = false>
__global__ void __launch_bounds__(kRsThreads)
    k_rs_scatter(const K *__restrict__ kin, const int32_t *__restrict__ vin, K *kout,
                 int32_t *vout, int64_t n, int shift, const int32_t *__restrict__ hoff,
                 int ntiles) {
    static_assert(!kStaged || sizeof(K) == 4, "staged scatter: 32-bit keys");
    __shared__ int wc[kRsWarps][256];
    __shared__ int wb[kStaged ? 1 : kRsWarps][256];
    __shared__ int dstart[256], gbase[256], wsum[kRsWarps];
    __shared__ K skey[kStaged ? kRsTile : 1];
    __shared__ int32_t sval[kStaged ? kRsTile : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * kRsTile;
    const int64_t wbase = tbase + (int64_t)w * kRsPerWarp;
    for (int it = 0; it < kRsPerWarp / 32; it++) {
        int64_t i = wbase + it * 32 + lane;
        bool ok = i < n;
        int d = ok ? (int)((kin[i] >> shift) & 255) : 256 + lane;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (ok && lane == __ffs(peers) - 1) wc[w][d] += __popc(peers);
    }
    __syncthreads();
    if constexpr (kStaged) {
        // thread t: digit t's run in the tile (a block scan of the digit
        // totals), each warp's place in it, and the run's global start
        const int t = threadIdx.x;
        int tot = 0;
        for (int q = 0; q < kRsWarps; q++) tot += wc[q][t];
        int x = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        int pre = 0;
        for (int q = 0; q < w; q++) pre += wsum[q];
        const int excl = pre + x - tot;
        dstart[t] = excl;
        int run = excl;
        for (int q = 0; q < kRsWarps; q++) { const int c = wc[q][t]; wc[q][t] = run; run += c; }
        gbase[t] = hoff[(int64_t)t * ntiles + blockIdx.x];
        __syncthreads();
        for (int it = 0; it < kRsPerWarp / 32; it++) {
            int64_t i = wbase + it * 32 + lane;
            bool ok = i < n;
            K kv = ok ? kin[i] : 0;
            int d = ok ? (int)((kv >> shift) & 255) : 256 + lane;
            unsigned peers = __match_any_sync(0xffffffffu, d);
            if (ok) {
                const int li = wc[w][d] + __popc(peers & lanemask_lt());
                skey[li] = kv;
                sval[li] = vin[i];
            }
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) wc[w][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        const int cnt = (int)(n - tbase < kRsTile ? n - tbase : kRsTile);
        for (int li = threadIdx.x; li < cnt; li += kRsThreads) {
            const K kv = skey[li];
            const int d = (int)((kv >> shift) & 255);
            const int pos = gbase[d] + (li - dstart[d]);
            kout[pos] = kv;
            vout[pos] = sval[li];
        }
    } else {
        {
            int d = threadIdx.x;
            int run = hoff[(int64_t)d * ntiles + blockIdx.x];
            for (int q = 0; q < kRsWarps; q++) { wb[q][d] = run; run += wc[q][d]; }
        }
        __syncthreads();
        for (int it = 0; it < kRsPerWarp / 32; it++) {
            int64_t i = wbase + it * 32 + lane;
            bool ok = i < n;
            K kv = ok ? kin[i] : 0;
            int d = ok ? (int)((kv >> shift) & 255) : 256 + lane;
            unsigned peers = __match_any_sync(0xffffffffu, d);
            if (ok) {
                int pos = wb[w][d] + __popc(peers & lanemask_lt());
                kout[pos] = kv;
                vout[pos] = vin[i];
            }
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) wb[w][d] += __popc(peers);
            __syncwarp();
        }
    }
}

// -------------------------------- stage 3: ProcessLowerStars

// ProcessLowerStars of the vertices of an id-ordered list (or of every vertex
// if list is null): the packed pairing of each lower star.
template <typename T, bool B>
__global__ void k_pls(const T *__restrict__ values, Geo<B> geo, const int32_t *__restrict__ list,
                      int64_t count, uint8_t *flags, GradRec *grad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const StarTables &S = g_star;
    int64_t x = list ? list[i] : i;
    const GridParams &g = geo.at(x);
    StarView sv;
    load_star(S, g, values, x, sv);
    PLSResult R;
    GradRec G;
    pls(S, sv.lower, sv.rank, R, &G);
    grad[x] = G;
    flags[x] = (uint8_t)(flags[x] | kFlagGradient);
}

// The same in two passes, for fields whose stars vary widely (noise): the
// work of a lower star depends on its shape (which links are lower) and
// grows with its size.  The first pass loads each star in id order
// (coalesced stencils) and keeps its lower mask as a sort key, its position
// and its link ranks (4 bits a link); the stars are then sorted by mask over
// the whole grid, and the second pass runs ProcessLowerStars in that order,
// so the 32 threads of a warp share one shape and only the order of the
// lower links differs between them.  Each warp and block finishes on its
// own: no barrier ties a fast star to a slow one.
template <typename T, bool B>
__global__ void __launch_bounds__(256)
    k_pls_keys(const T *__restrict__ values, Geo<B> geo, const int32_t *__restrict__ list,
               int64_t count, uint32_t *__restrict__ key, int32_t *__restrict__ pos,
               unsigned long long *__restrict__ ranks, uint8_t *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t x = list ? list[i] : i;
    StarView sv;
    load_star(g_star, geo.at(x), values, x, sv);
    unsigned long long rk = 0;
    for (int n = 0; n < kLinks; n++) rk |= (unsigned long long)(sv.rank[n] & 15) << (4 * n);
    ranks[i] = rk;
    key[i] = sv.lower;
    pos[i] = (int32_t)i;
    // the second pass fills the record before any later kernel reads it
    flags[x] = (uint8_t)(flags[x] | kFlagGradient);
}

__global__ void k_pls_run(const int32_t *__restrict__ list, const uint32_t *__restrict__ key,
                          const int32_t *__restrict__ pos,
                          const unsigned long long *__restrict__ ranks, int64_t count,
                          GradRec *grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int32_t j = pos[i];
    const int64_t x = list ? list[j] : j;
    const unsigned long long rk = ranks[j];
    uint8_t rank[kLinks];
    for (int n = 0; n < kLinks; n++) rank[n] = (uint8_t)((rk >> (4 * n)) & 15);
    PLSResult R;
    GradRec G;
    pls(g_star, (uint16_t)(key[i] & kAllLinks), rank, R, &G);
    grad[x] = G;
}

// The critical cells of the lower star of each sorted critical vertex, read
// off its packed pairing: the critical edges and tets are the lower ones left
// unpaired, the critical triangles those paired with neither an edge nor a
// tet, a vertex without lower edge is a minimum.
__global__ void k_critrec(const int32_t *__restrict__ vc, int64_t nc,
                          const GradRec *__restrict__ grad, CritRec *recs, int32_t *cnt0,
                          int32_t *cnt1, int32_t *cnt2, int32_t *cnt3, int32_t *vrank) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const StarTables &S = g_star;
    int64_t x = vc[i];
    GradRec G = grad[x];
    uint16_t L = 0;
    for (int n = 0; n < kLinks; n++) L |= (uint16_t)((grad_rank(G, n) != 0xF) << n);
    uint64_t LT = kAllTris;
    uint32_t LH = kAllTets;
    for (uint16_t out = (uint16_t)(~L & kAllLinks); out; out &= out - 1) {
        int n = __ffs(out) - 1;
        LT &= ~S.tris_of_link[n];
        LH &= ~S.tets_of_link[n];
    }
    uint16_t ce = 0;
    uint64_t paired_t = 0;
    uint32_t ch = 0;
    for (uint16_t m = L; m; m &= m - 1) {
        int n = __ffs(m) - 1;
        int p = grad_edge_pair(G, n);
        if (p == kNone) ce |= (uint16_t)(1u << n);
        else if (p < kTris) paired_t |= 1ull << p;
    }
    for (uint32_t m = LH; m; m &= m - 1) {
        int h = __ffs(m) - 1;
        int p = grad_tet_pair(G, h);
        if (p == kNone) ch |= 1u << h;
        else paired_t |= 1ull << p;
    }
    CritRec rec;
    rec.crit_t = LT & ~paired_t;
    rec.ranks = G.w[5];
    rec.crit_h = ch;
    rec.crit_e = ce;
    rec.is_min = L == 0;
    rec.pad = 0;
    recs[i] = rec;
    cnt0[i] = rec.is_min;
    cnt1[i] = __popc(ce);
    cnt2[i] = __popcll(rec.crit_t);
    cnt3[i] = __popc(ch);
    vrank[x] = (int32_t)i;
}

// Critical simplices of each dimension in lexicographic order: by vertex (the
// critical vertices are sorted) then by G inside the lower star.
__global__ void k_emit(const int32_t *__restrict__ vc, int64_t nc, const CritRec *__restrict__ recs,
                       const int32_t *b0, const int32_t *b1, const int32_t *b2, const int32_t *b3,
                       int32_t *v0, int32_t *v1, uint8_t *l1, int32_t *v2, uint8_t *l2,
                       int32_t *v3, uint8_t *l3) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const StarTables &S = g_star;
    CritRec rec = recs[i];
    int32_t x = vc[i];
    uint8_t r[kLinks];
    unpack_ranks(rec.ranks, r);
    if (rec.is_min) v0[b0[i]] = x;
    int k = b1[i];
    for (uint16_t m = rec.crit_e; m;) {
        int bi = -1; uint16_t bc = 0xFFFF;
        for (uint16_t q = m; q; q &= q - 1) {
            int n = __ffs(q) - 1; uint16_t c = code_edge(r, n);
            if (c < bc) { bc = c; bi = n; }
        }
        v1[k] = x; l1[k] = (uint8_t)bi; k++;
        m &= (uint16_t)~(1u << bi);
    }
    k = b2[i];
    for (uint64_t m = rec.crit_t; m;) {
        int bi = -1; uint16_t bc = 0xFFFF;
        for (uint64_t q = m; q; q &= q - 1) {
            int s = __ffsll(q) - 1; uint16_t c = code_tri(S, r, s);
            if (c < bc) { bc = c; bi = s; }
        }
        v2[k] = x; l2[k] = (uint8_t)bi; k++;
        m &= ~(1ull << bi);
    }
    k = b3[i];
    for (uint32_t m = rec.crit_h; m;) {
        int bi = -1; uint16_t bc = 0xFFFF;
        for (uint32_t q = m; q; q &= q - 1) {
            int h = __ffs(q) - 1; uint16_t c = code_tet(S, r, h);
            if (c < bc) { bc = c; bi = h; }
        }
        v3[k] = x; l3[k] = (uint8_t)bi; k++;
        m &= ~(1u << bi);
    }
}

// ------------------------------------------------------ stage 4: D0 arcs

// The minimum reached by following descent links from w, or -1 (and the
// iteration-limit error) if max_steps is exceeded.
__device__ __forceinline__ int64_t descend(const GridParams &g, const uint8_t *__restrict__ flags,
                                           int64_t w, int64_t max_steps, DevStatus *st) {
    for (int64_t s = 0; s < max_steps; s++) {
        int d = flags[w] & 0xF;
        if (d == kNoDescent) return w;
        w += g.dlin[d];
    }
    atomicOr(&st->err, kErrIter);
    return -1;
}

// Each critical edge links the two minima that its two descending v-paths
// (vertex -> edge vectors: each regular vertex is paired with the edge to its
// lowest neighbour) reach (Sec. 5.1 (a)-(b)).
template <bool Bt>
__global__ void k_d0_arcs(Geo<Bt> geo, const uint8_t *__restrict__ flags,
                          const int32_t *__restrict__ vrank, const int32_t *__restrict__ base0,
                          const int32_t *__restrict__ v1,
                          const uint8_t *__restrict__ l1, int64_t n1, int32_t *A, int32_t *B,
                          int32_t *young, int64_t max_steps, DevStatus *st) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n1) return;
    int64_t x = v1[j];
    const GridParams &g = geo.at(x);
    int64_t u = x + g.dlin[l1[j]];
    int64_t ma = descend(g, flags, x, max_steps, st), mb = descend(g, flags, u, max_steps, st);
    // nodes are the minima by their index in C0 (the lexicographic order, so a
    // smaller index is an older minimum); on failure both ends go to node 0: a
    // self-loop, harmless until the host reports the error
    A[j] = ma < 0 || mb < 0 ? 0 : base0[vrank[ma]];
    B[j] = ma < 0 || mb < 0 ? 0 : base0[vrank[mb]];
    young[j] = -1;
}

// ------------------------------------- elder rule by divide and conquer
//
// The elder rule (Sec. 5.1 (c)-(d)) processes arcs in (in/de)creasing order
// with a union-find: an arc joining two components kills the younger
// component's extremum; an arc inside one component closes a cycle and stays
// unpaired.  Its outcome depends only on the two components at the arc's
// turn.  Those are computed for every arc at once by halving the arc order:
// for a segment of arcs whose endpoint labels name the components at the
// segment's start (each component is named by its oldest node), the light
// half keeps those labels and the heavy half is relabelled by the connected
// components of the light half (named by their oldest label).  After
// ceil(log2 E) levels every arc's labels name the components at its own turn.
// Each level runs a lock-free union-find keyed by (segment, label) in a hash
// table, since one label may name different components in different
// segments.

__device__ __forceinline__ uint32_t hash_key(unsigned long long k) {
    k ^= k >> 31; k *= 0x7fb5d329728ea185ull; k ^= k >> 27; k *= 0x81dadef4bc2dd44dull;
    k ^= k >> 33;
    return (uint32_t)k;
}

// One slot of the (segment, label) table: the key, the union-find parent (a
// slot index) and the label the slot stands for, in one 16-byte line so that
// a probe, a find step and a label read touch one sector.
struct DcSlot {
    unsigned long long key;   // ~0: empty
    int32_t par, lab;
};

__device__ __forceinline__ int64_t dc_time(int64_t j, int64_t narcs, int descending) {
    return descending ? narcs - 1 - j : j;
}

// Keys of level `shift` carry, above the label, the segment's first turn
// with bit shift-1 set: (seg << shift) | 1 << (shift - 1).  The lowest set
// bit names the level, so the table is cleared once per call: a slot left by
// an earlier (higher) level reads as free.  Within a level keys are only
// added, so a lookup that meets a free slot has passed every slot its key
// could occupy.
__device__ __forceinline__ unsigned long long dc_key(int64_t seg, int shift, int32_t label) {
    const unsigned long long code = ((unsigned long long)seg << shift) | (1ull << (shift - 1));
    return (code << 32) | (uint32_t)label;
}

__device__ __forceinline__ bool dc_free(unsigned long long k, int shift) {
    const uint32_t low = (uint32_t)(k >> 32) & ((1u << shift) - 1);
    return k == ~0ull || low != (1u << (shift - 1));
}

// slot of key (inserting it if absent); -1 if the table is full
__device__ __forceinline__ int32_t dc_insert(DcSlot *tab, uint32_t mask, unsigned long long key,
                                             int shift, bool *fresh) {
    uint32_t h = hash_key(key) & mask;
    for (uint32_t p = 0; p <= mask; p++) {
        uint32_t s = (h + p) & mask;
        unsigned long long k = tab[s].key;
        if (k == key) { *fresh = false; return (int32_t)s; }
        if (dc_free(k, shift)) {
            unsigned long long old = atomicCAS(&tab[s].key, k, key);
            if (old == k) { *fresh = true; return (int32_t)s; }
            if (old == key) { *fresh = false; return (int32_t)s; }
        }
    }
    return -1;
}

__device__ __forceinline__ int32_t dc_lookup(const DcSlot *tab, uint32_t mask,
                                             unsigned long long key, int shift) {
    uint32_t h = hash_key(key) & mask;
    for (uint32_t p = 0; p <= mask; p++) {
        uint32_t s = (h + p) & mask;
        unsigned long long k = tab[s].key;
        if (k == key) return (int32_t)s;
        if (dc_free(k, shift)) return -1;
    }
    return -1;
}

__device__ __forceinline__ int32_t dc_find(DcSlot *tab, int32_t a) {
    while (true) {
        int32_t p = tab[a].par;
        if (p == a) return a;
        int32_t gp = tab[p].par;
        if (gp != p) tab[a].par = gp;
        a = gp;
    }
}

// light arcs of each segment: register both endpoint labels.  An arc whose
// two ends already carry the same label joins nothing: its label is left out
// (a heavy arc looking it up keeps it, as its component in the light half
// is then itself or is registered by another arc).
__global__ void k_dc_insert(int64_t narcs, int shift, int descending, const int32_t *A,
                            const int32_t *B, DcSlot *tab, uint32_t mask, DevStatus *st) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= narcs) return;
    int64_t t = dc_time(j, narcs, descending);
    int64_t seg = t >> shift;
    if ((t >> (shift - 1)) & 1) return;                  // heavy half
    int32_t ab[2] = {A[j], B[j]};
    if (ab[0] == ab[1]) return;
    for (int e = 0; e < 2; e++) {
        const unsigned long long key = dc_key(seg, shift, ab[e]);
        bool fresh;
        int32_t s = dc_insert(tab, mask, key, shift, &fresh);
        if (s < 0) { atomicOr(&st->err, kErrCap); return; }
        if (fresh) { tab[s].par = s; tab[s].lab = ab[e]; }
    }
}

// light arcs: union their endpoints; a root is hooked under the root holding
// the older label (smaller for D0, larger for D2)
__global__ void k_dc_union(int64_t narcs, int shift, int descending, int older_is_larger,
                           const int32_t *A, const int32_t *B, DcSlot *tab, uint32_t mask,
                           DevStatus *st) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= narcs) return;
    int64_t t = dc_time(j, narcs, descending);
    int64_t seg = t >> shift;
    if ((t >> (shift - 1)) & 1) return;
    int32_t a = A[j], b = B[j];
    if (a == b) return;
    int32_t sa = dc_lookup(tab, mask, dc_key(seg, shift, a), shift);
    int32_t sb = dc_lookup(tab, mask, dc_key(seg, shift, b), shift);
    if (sa < 0 || sb < 0) { atomicOr(&st->err, kErrState); return; }
    for (int it = 0; it < (1 << 20); it++) {
        int32_t ra = dc_find(tab, sa), rb = dc_find(tab, sb);
        if (ra == rb) return;
        const int32_t la = tab[ra].lab, lb = tab[rb].lab;
        bool a_older = older_is_larger ? la > lb : la < lb;
        int32_t young = a_older ? rb : ra, old = a_older ? ra : rb;
        if (atomicCAS(&tab[young].par, young, old) == young) return;
    }
    atomicOr(&st->err, kErrIter);
}

// heavy arcs: relabel endpoints by the light half's components
__global__ void k_dc_relabel(int64_t narcs, int shift, int descending, int32_t *A, int32_t *B,
                             DcSlot *tab, uint32_t mask) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= narcs) return;
    int64_t t = dc_time(j, narcs, descending);
    int64_t seg = t >> shift;
    if (!((t >> (shift - 1)) & 1)) return;               // light half
    int32_t *ends[2] = {&A[j], &B[j]};
    for (int e = 0; e < 2; e++) {
        int32_t s = dc_lookup(tab, mask, dc_key(seg, shift, *ends[e]), shift);
        if (s >= 0) *ends[e] = tab[dc_find(tab, s)].lab;
    }
}

// The last levels at once: segments of 2^kDcSegBits consecutive turns, each
// taken through its arcs in turn order by one warp, with a union-find over
// the segment's labels in shared memory (the lanes register the labels, then
// lane 0 walks the arcs).  Within a segment this is what the remaining
// halving levels compute: every arc gets the components at its own turn,
// each named by its oldest label.
constexpr int kDcSegBits = 8, kDcSeg = 1 << kDcSegBits, kDcSegSlots = 4 * kDcSeg;
__global__ void __launch_bounds__(32)
    k_dc_segment(int64_t narcs, int descending, int older_is_larger, int32_t *A, int32_t *B,
                 DevStatus *st) {
    __shared__ int32_t lab[kDcSegSlots];    // label of each slot (-1: free)
    __shared__ int16_t par[kDcSegSlots];    // union-find parent (a slot)
    __shared__ int16_t ends[2 * kDcSeg];    // each arc's two slots, in turn order
    const int lane = threadIdx.x;
    const int64_t t0 = (int64_t)blockIdx.x * kDcSeg;
    const int cnt = (int)(narcs - t0 < kDcSeg ? narcs - t0 : kDcSeg);
    for (int i = lane; i < kDcSegSlots; i += 32) lab[i] = -1;
    __syncwarp();
    for (int k = lane; k < cnt; k += 32) {
        const int64_t j = dc_time(t0 + k, narcs, descending);   // the arc of turn t0 + k
        for (int e = 0; e < 2; e++) {
            const int32_t v = e ? B[j] : A[j];
            const uint32_t h = hash_key((unsigned long long)(uint32_t)v) & (kDcSegSlots - 1);
            int sl = -1;
            for (int p = 0; p < kDcSegSlots; p++) {   // at most 2 * kDcSeg labels: never full
                const int q = (int)((h + p) & (kDcSegSlots - 1));
                const int32_t old = atomicCAS(&lab[q], -1, v);
                if (old == -1 || old == v) { sl = q; break; }
            }
            if (sl < 0) { atomicOr(&st->err, kErrCap); sl = 0; }
            par[sl] = (int16_t)sl;
            ends[2 * k + e] = (int16_t)sl;
        }
    }
    __syncwarp();
    if (lane != 0) return;
    for (int k = 0; k < cnt; k++) {
        int ra = ends[2 * k], rb = ends[2 * k + 1];
        while (par[ra] != ra) { par[ra] = par[par[ra]]; ra = par[ra]; }
        while (par[rb] != rb) { par[rb] = par[par[rb]]; rb = par[rb]; }
        const int64_t j = dc_time(t0 + k, narcs, descending);
        const int32_t la = lab[ra], lb = lab[rb];
        A[j] = la;
        B[j] = lb;
        if (ra != rb) {
            const bool a_older = older_is_larger ? la > lb : la < lb;
            if (a_older) par[rb] = (int16_t)ra;
            else par[ra] = (int16_t)rb;
        }
    }
}

// ------------------------------- minimum spanning forest of an arc graph
//
// Only the arcs of the minimum spanning forest (weight = the arc's turn,
// distinct for all arcs) can join two components at their turn: Kruskal's
// order takes exactly those.  The others close cycles and pair nothing, so
// the elder rule's halving levels run over the forest's arcs only.  The
// forest is found by Borůvka's rounds: every component takes its lightest
// arc to another component; a component is named by a root node, and nodes
// point (comp) to their root after every round.
__global__ void k_bv_best(const int32_t *__restrict__ act, int64_t nact, int64_t narcs,
                          int descending, const int32_t *__restrict__ A,
                          const int32_t *__restrict__ B, const int32_t *__restrict__ comp,
                          uint32_t *best, int32_t *open) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nact) return;
    const int64_t j = act ? act[k] : k;
    const int32_t ca = comp[A[j]], cb = comp[B[j]];
    open[k] = ca != cb;
    if (ca == cb) return;
    const uint32_t w = (uint32_t)dc_time(j, narcs, descending);
    atomicMin(&best[ca], w);
    atomicMin(&best[cb], w);
}

// each root that found an arc: the root at its other end (comp is not
// written in this kernel), and the arc joins the forest
__global__ void k_bv_pick(int64_t nnodes, int64_t narcs, int descending,
                          const int32_t *__restrict__ A, const int32_t *__restrict__ B,
                          const int32_t *__restrict__ comp, const uint32_t *__restrict__ best,
                          int32_t *tgt, uint8_t *msf) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nnodes) return;
    tgt[r] = -1;
    if (comp[r] != r || best[r] == 0xFFFFFFFFu) return;
    const int64_t w = best[r];
    const int64_t j = descending ? narcs - 1 - w : w;
    const int32_t ca = comp[A[j]], cb = comp[B[j]];
    tgt[r] = ca == r ? cb : ca;
    msf[j] = 1;
}

// hook every such root under the other end's root; when two roots took the
// same arc, the smaller one stays a root (no other cycle can form: weights
// are distinct)
__global__ void k_bv_hook(int64_t nnodes, const int32_t *__restrict__ tgt, int32_t *comp,
                          unsigned long long *hooks) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nnodes) return;
    const int32_t t = tgt[r];
    if (t < 0) return;
    if (tgt[t] == r && r < t) return;
    comp[r] = t;
    atomicAdd(hooks, 1ull);
}

// every node to its root (concurrent writes only shorten paths to one root)
__global__ void k_bv_jump(int64_t nnodes, int32_t *comp, DevStatus *st) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nnodes) return;
    int32_t x = comp[v];
    for (int64_t it = 0; it <= nnodes; it++) {
        const int32_t p = comp[x];
        if (p == x) { comp[v] = x; return; }
        x = p;
    }
    atomicOr(&st->err, kErrIter);
}

// the forest's arcs in their order: positions (scan of msf) -> packed arrays
__global__ void k_bv_gather(int64_t narcs, const uint8_t *__restrict__ msf,
                            const int32_t *__restrict__ pos, const int32_t *__restrict__ A,
                            const int32_t *__restrict__ B, int32_t *A2, int32_t *B2,
                            int32_t *idx) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= narcs || !msf[j]) return;
    const int32_t k = pos[j];
    A2[k] = A[j]; B2[k] = B[j]; idx[k] = (int32_t)j;
}

// every arc now sees the components at its turn: the elder rule
__global__ void k_dc_decide(int64_t narcs, int older_is_larger, const int32_t *A,
                            const int32_t *B, const int32_t *__restrict__ idx, int32_t *young,
                            uint8_t *died) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= narcs) return;
    const int64_t j = idx ? idx[k] : k;
    int32_t a = A[k], b = B[k];
    if (a == b) { young[j] = -1; return; }
    int32_t y = older_is_larger ? (a < b ? a : b) : (a > b ? a : b);
    young[j] = y;
    died[y] = 1;
}

// ------------------------------------------- the gradient, memoised lazily
//
// The pairing of a lower star is computed once per vertex and per compute:
// by k_pls for the critical vertices, on first use for the others.  Two
// threads may fill the same record; they write identical bytes.  The record
// is stored before the flag bit is set (with a fence) and read through L2,
// so a reader that sees the bit sees the record.
template <typename T>
__device__ __noinline__ GradRec grad_fill(const StarTables &S, const GridParams &g,
                                          const T *__restrict__ values, uint8_t *flags,
                                          GradRec *grad, int64_t y);

// dense: every record was computed before the walks (nothing writes flags or
// records meanwhile), so the record is read through L1 without its flag.
template <typename T>
__device__ __forceinline__ GradRec grad_get(const StarTables &S, const GridParams &g,
                                            const T *__restrict__ values, uint8_t *flags,
                                            GradRec *grad, int64_t y, bool dense = false) {
    if (dense) {
        GradRec G;
        const ulonglong2 *src = (const ulonglong2 *)&grad[y];
        for (int k = 0; k < 3; k++) {
            const ulonglong2 v = __ldg(src + k);
            G.w[2 * k] = v.x;
            G.w[2 * k + 1] = v.y;
        }
        return G;
    }
    if (((volatile const uint8_t *)flags)[y] & kFlagGradient) {
        GradRec G;
        const ulonglong2 *src = (const ulonglong2 *)&grad[y];
        for (int k = 0; k < 3; k++) {
            ulonglong2 v = __ldcg(src + k);
            G.w[2 * k] = v.x;
            G.w[2 * k + 1] = v.y;
        }
        return G;
    }
    return grad_fill(S, g, values, flags, grad, y);
}

// Computes and stores the record of vertex y (out of line: one copy of
// ProcessLowerStars per kernel instead of one per call site).
template <typename T>
__device__ __noinline__ GradRec grad_fill(const StarTables &S, const GridParams &g,
                                          const T *__restrict__ values, uint8_t *flags,
                                          GradRec *grad, int64_t y) {
    GradRec G;
    StarView sv;
    load_star(S, g, values, y, sv);
    PLSResult R;
    pls(S, sv.lower, sv.rank, R, &G);
    ulonglong2 *dst = (ulonglong2 *)&grad[y];
    for (int k = 0; k < 3; k++) __stcg(dst + k, make_ulonglong2(G.w[2 * k], G.w[2 * k + 1]));
    __threadfence();
    volatile uint8_t *f = (volatile uint8_t *)flags;
    f[y] = (uint8_t)(f[y] | kFlagGradient);
    return G;
}

// ------------------------------------------------------ stage 5: D2 arcs

// Per critical vertex: its critical star tets (bits 32-55) and the C3 index
// of the first (bits 0-31), so that an ascending walk tests a tet with the
// loads of its step instead of two more dependent ones.
__global__ void k_tet_words(const int32_t *__restrict__ vc, int64_t nc,
                            const CritRec *__restrict__ recs, const int32_t *__restrict__ base3,
                            unsigned long long *tw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    tw[vc[i]] = ((unsigned long long)recs[i].crit_h << 32) | (uint32_t)base3[i];
}

// The critical tet (node index) or the virtual maximum reached from tet h of
// the star of y by the ascending walk of the dual gradient (Sec. 5.2): a
// regular tet is the head of a triangle->tet vector; cross that triangle to
// its other tet; the outer boundary is the virtual maximum.
template <typename T>
__device__ int32_t ascend(const StarTables &S, const GridParams &g, const T *__restrict__ values,
                          uint8_t *flags, GradRec *grad, const unsigned long long *__restrict__ tw,
                          int64_t y, int h, int32_t vmax, int64_t max_steps, bool dense,
                          DevStatus *st) {
    using K = typename Key<T>::K;
    int cx, cy, cz;     // coordinates of y, followed as the walk moves
    coords(g, y, cx, cy, cz);
    K ky = Key<T>::of(values[y]);
    int wn = -1;        // after a crossing: the link of the tet's one new vertex
    for (int64_t step = 0; step < max_steps; step++) {
        // the maximum vertex of the tet: any of its vertices for the first
        // tet; after crossing a face of the lower star of y, y or the new one
        K kb = ky;
        int64_t best = y;
        int bl = -1;
        for (int k = 0; k < 3; k++) {
            const int l = wn >= 0 ? wn : S.tet_v[h][k];
            const int64_t v = y + g.dlin[l];
            const K kv = Key<T>::of(values[v]);
            if (kv > kb || (kv == kb && v > best)) { kb = kv; best = v; bl = l; }
            if (wn >= 0) break;
        }
        ky = kb;
        if (bl >= 0) {   // re-express the tet in the star of its maximum vertex
            int ox = -S.dx[bl], oy = -S.dy[bl], oz = -S.dz[bl];
            int ly = S.link_of_dc[(ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)];
            if (ly < 0) { atomicOr(&st->err, kErrState); return vmax; }
            int lks[2], nk = 0;
            for (int k = 0; k < 3; k++) {
                int l = S.tet_v[h][k];
                if (l == bl) continue;
                int ex = S.dx[l] + ox, ey = S.dy[l] + oy, ez = S.dz[l] + oz;
                if (ex < -1 || ex > 1 || ey < -1 || ey > 1 || ez < -1 || ez > 1 || nk >= 2) {
                    atomicOr(&st->err, kErrState);
                    return vmax;
                }
                int lk = S.link_of_dc[(ex + 1) + 3 * (ey + 1) + 9 * (ez + 1)];
                if (lk < 0) { atomicOr(&st->err, kErrState); return vmax; }
                lks[nk++] = lk;
            }
            if (nk != 2) { atomicOr(&st->err, kErrState); return vmax; }
            // the star tet on links (ly, lks[0], lks[1]): one of the (at most
            // two) star tets on the star triangle (lks[0], lks[1])
            const int sf = S.tri_of_pair[lks[0]][lks[1]];
            if (sf < 0) { atomicOr(&st->err, kErrState); return vmax; }
            int hn = -1;
            for (uint32_t cm = S.tets_of_tri[sf]; cm; cm &= cm - 1) {
                const int q = __ffs(cm) - 1;
                if (S.tet_mask[q] >> ly & 1) hn = q;
            }
            if (hn < 0) { atomicOr(&st->err, kErrState); return vmax; }
            y = best;
            cx += S.dx[bl]; cy += S.dy[bl]; cz += S.dz[bl];
            h = hn;
        }
        // the vertex's flag, tet word and record, read together
        const uint8_t fy = dense ? __ldg(flags + y) : ((volatile const uint8_t *)flags)[y];
        const unsigned long long twy = tw[y];
        GradRec G = grad_get(S, g, values, flags, grad, y, dense);
        if ((fy & kFlagCritical) && (twy >> (32 + h) & 1)) {
            // a critical tet: the vertex's first C3 index plus its critical
            // tets of lower G (the ranks are the record's)
            uint8_t r[kLinks];
            unpack_ranks(G.w[5], r);
            const uint16_t ch = code_tet(S, r, h);
            int k = 0;
            for (uint32_t m = (uint32_t)(twy >> 32); m; m &= m - 1)
                k += code_tet(S, r, __ffs(m) - 1) < ch;
            return (int32_t)(uint32_t)twy + k;
        }
        int s2 = grad_tet_pair(G, h);
        if (s2 >= kTris) { atomicOr(&st->err, kErrState); return vmax; }
        uint32_t other = S.tets_of_tri[s2] & ~(1u << h);
        if (!other) { atomicOr(&st->err, kErrState); return vmax; }
        int h2 = __ffs(other) - 1;
        int w = __ffs(S.tet_mask[h2] & ~S.tri_mask[s2]) - 1;
        if (!(present_links(S, g, cx, cy, cz) >> w & 1)) return vmax;   // the outer boundary
        h = h2;
        wn = w;
    }
    atomicOr(&st->err, kErrIter);
    return vmax;
}

template <typename T, bool Bt>
__global__ void k_d2_arcs(const T *__restrict__ values, Geo<Bt> geo, uint8_t *flags,
                          GradRec *grad, const unsigned long long *__restrict__ tw,
                          const int32_t *__restrict__ v2, const uint8_t *__restrict__ l2,
                          int64_t n2, const int32_t *__restrict__ order, int32_t vmax,
                          int vmax_on, int32_t *A, int32_t *B, int32_t *young, int64_t max_steps,
                          int dense, DevStatus *st) {
    // arcs in vertex-id order (`order`), so that the walks of a warp start
    // close together and share the records they read.  Without the virtual
    // maximum (App. A) a 2-saddle whose ascent leaves the domain on either
    // side merges nothing: its arc becomes a loop at the outside node.
    const int64_t jj = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (jj >= n2) return;
    const int64_t j = order ? order[jj] : jj;
    const StarTables &S = g_star;
    int64_t x = v2[j];
    const GridParams &g = geo.at(x);
    int s = l2[j];
    int cx, cy, cz;
    coords(g, x, cx, cy, cz);
    uint16_t pres = present_links(S, g, cx, cy, cz);
    int32_t ends[2];
    uint32_t m = S.tets_of_tri[s];
    for (int e = 0; e < 2; e++) {
        int h = __ffs(m) - 1;
        m &= m - 1;
        int w = __ffs(S.tet_mask[h] & ~S.tri_mask[s]) - 1;
        ends[e] = (pres >> w & 1) ? ascend(S, g, values, flags, grad, tw, x, h,
                                           vmax, max_steps, dense != 0, st)
                                  : vmax;
    }
    if (!vmax_on && (ends[0] == vmax || ends[1] == vmax)) ends[0] = ends[1] = vmax;
    A[j] = ends[0];
    B[j] = ends[1];
    young[j] = -1;
}

// ------------------------------------------ stage 6: D1 boundary tracing

struct TraceCtx {
    HeapEnt *heap;
    HashEnt *hash;
    int32_t *rows;     // C1 index of each row met (in order of first contact)
    int32_t *rslot;    // its hash slot
    int hcap, hashmask, rcap;
    int hn, rn, used;
    int32_t gen;
    bool overflow;
    bool dense;        // every record was computed before the walks: nothing
                       // writes flags or records meanwhile, so they may be
                       // cached in L1
    bool gens;         // generator mode: compressed edges kept as passive entries
};

__device__ __forceinline__ uint32_t hash64(unsigned long long k) {
    k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}

__device__ __forceinline__ bool heap_less(const HeapEnt &a, const HeapEnt &b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

__device__ void heap_push(TraceCtx &c, HeapEnt e) {
    if (c.hn >= c.hcap) { c.overflow = true; return; }
    int i = c.hn++;
    while (i > 0) {
        int p = (i - 1) >> 1;
        if (!heap_less(c.heap[p], e)) break;
        c.heap[i] = c.heap[p];
        i = p;
    }
    c.heap[i] = e;
}

__device__ HeapEnt heap_pop(TraceCtx &c) {
    HeapEnt top = c.heap[0];
    HeapEnt last = c.heap[--c.hn];
    int i = 0;
    while (true) {
        int l = 2 * i + 1;
        if (l >= c.hn) break;
        int r = l + 1;
        int m = (r < c.hn && heap_less(c.heap[l], c.heap[r])) ? r : l;
        if (!heap_less(last, c.heap[m])) break;
        c.heap[i] = c.heap[m];
        i = m;
    }
    if (c.hn > 0) c.heap[i] = last;
    return top;
}

// Toggles (mod 2) edge (y, link m) of the expanding boundary.  Edges that are
// heads of vertex->edge vectors and critical edges already paired in D0 are
// dropped (they never carry the pivot; compression of Sec. 1.1 / 5).  A
// regular edge is pushed on the max-heap keyed by (vertex order of its
// maximum vertex y, classification order inside the lower star of y), which is
// a topological order of the gradient paths, so that every regular edge is
// expanded at most once; the two edges its expansion yields are precomputed
// (the spec in the hash entry), so the expansion reads no record.  The
// vertex's flag, value and record are loaded together up front.
template <typename T>
__device__ void trace_toggle(TraceCtx &c, const StarTables &S, const GridParams &g,
                             const T *__restrict__ values, uint8_t *flags, GradRec *grad,
                             const unsigned long long *__restrict__ vcrit, int64_t y, int m,
                             DevStatus *st) {
    if (m < 0 || m >= kLinks) { atomicOr(&st->err, kErrState); c.overflow = true; return; }
    const uint8_t fy = c.dense ? __ldg(flags + y) : ((volatile const uint8_t *)flags)[y];
    const T vy = values[y];
    const unsigned long long cw = vcrit[y];   // read beside the others; used if y is critical
    GradRec G;
    {
        const ulonglong2 *src = (const ulonglong2 *)&grad[y];
        for (int k = 0; k < 3; k++) {
            const ulonglong2 v = c.dense ? __ldg(src + k) : __ldcg(src + k);
            G.w[2 * k] = v.x;
            G.w[2 * k + 1] = v.y;
        }
    }
    // the head of y's vertex->edge vector: compressed away (Sec. 1.1 / 5), or
    // a passive entry in the generator mode
    const bool head = (fy & 0xF) == m;
    if (head && !c.gens) return;
    unsigned long long key = (((unsigned long long)y << 4) | (unsigned)m) + 1;
    uint32_t hpos = hash64(key) & c.hashmask;
    HashEnt *slot = nullptr;
    for (int p = 0; p <= c.hashmask; p++) {
        HashEnt *e = &c.hash[(hpos + p) & c.hashmask];
        if (e->gen != c.gen) { slot = e; break; }
        if (e->key == key) { e->info ^= 1u << 31; return; }
    }
    if (!slot || c.used * 4 >= (c.hashmask + 1) * 3) { c.overflow = true; return; }
    uint32_t info;
    const bool crit = (fy & kFlagCritical) && (cw >> (32 + m) & 1);
    if (head || (crit && !(cw >> (48 + m) & 1))) {
        // a head, or a critical edge paired in D0 (dropped unless generator mode
        // -- heads returned above then): a passive entry -(edge id + 1)
        if (!c.gens) return;
        if (c.rn >= c.rcap) { c.overflow = true; return; }
        c.rows[c.rn] = (int32_t)(-1 - edge_id(S, g, y, m));
        c.rslot[c.rn] = (int32_t)(slot - c.hash);
        c.rn++;
        slot->key = key;
        slot->gen = c.gen;
        slot->info = hinfo((uint32_t)(c.rn - 1), 0, kKindRow, 1);
        c.used++;
        return;
    }
    if (crit) {                                            // a row
        {
            // its C1 index: the vertex's first, plus its critical edges of lower
            // rank (the G order of edges of one lower star)
            const int rm = grad_rank(G, m);
            int32_t j1 = (int32_t)(uint32_t)cw;
            for (uint32_t q = (uint32_t)(cw >> 32) & kAllLinks; q; q &= q - 1)
                j1 += grad_rank(G, __ffs(q) - 1) < rm;
            if (c.rn >= c.rcap) { c.overflow = true; return; }
            c.rows[c.rn] = j1;
            c.rslot[c.rn] = (int32_t)(slot - c.hash);
            info = hinfo((uint32_t)c.rn, 0, kKindRow, 1);
            c.rn++;
            slot->key = key;
            slot->gen = c.gen;
            slot->info = info;
            c.used++;
            return;
        }
    }
    if (!(fy & kFlagGradient)) G = grad_fill(S, g, values, flags, grad, y);
    int sp = grad_edge_pair(G, m);
    if (sp >= kTris) { atomicOr(&st->err, kErrState); return; }
    // the expansion through triangle sp: the other star edge of y, and the
    // edge between the triangle's link vertices in the star of the higher one
    const int ta = S.tri_v[sp][0], tb = S.tri_v[sp][1];
    const bool aup = grad_rank(G, ta) > grad_rank(G, tb);
    const int hi = aup ? ta : tb, lo = aup ? tb : ta;
    const int l = S.link_of_dc[(S.dx[lo] - S.dx[hi] + 1) + 3 * (S.dy[lo] - S.dy[hi] + 1) +
                               9 * (S.dz[lo] - S.dz[hi] + 1)];
    if (l < 0) { atomicOr(&st->err, kErrState); c.overflow = true; return; }
    const uint32_t spec = (uint32_t)(ta == m ? tb : ta) | ((uint32_t)hi << 4) | ((uint32_t)l << 8);
    HeapEnt he;
    he.hi = (unsigned long long)Key<T>::of(vy);
    he.lo = ((unsigned long long)y << 12) | ((unsigned long long)grad_edge_order(G, m) << 4) |
            (unsigned)m;
    heap_push(c, he);
    if (c.overflow) return;
    slot->key = key;
    slot->gen = c.gen;
    slot->info = hinfo(spec, sp, kKindReg, 1);
    c.used++;
}

__device__ __forceinline__ HashEnt *trace_find(TraceCtx &c, int64_t y, int m) {
    unsigned long long key = (((unsigned long long)y << 4) | (unsigned)m) + 1;
    uint32_t hpos = hash64(key) & c.hashmask;
    for (int p = 0; p <= c.hashmask; p++) {
        HashEnt *e = &c.hash[(hpos + p) & c.hashmask];
        if (e->gen != c.gen) return nullptr;
        if (e->key == key) return e;
    }
    return nullptr;
}

// One thread per column: the Morse boundary of a critical triangle restricted
// to the rows (1-saddles not paired in D0), as a descending list of C1
// indices appended to the column pool.  The walks differ widely in length,
// so the loop is flat: in every iteration each lane takes one step of its
// current column -- one toggle of an edge its start or an expansion queued,
// or the column's write-out -- and lanes that finish fetch the next column at
// once (one atomic per warp), instead of the warp waiting for its longest
// walk before the next batch of columns.
template <typename T, bool B>
__global__ void __launch_bounds__(256, 4)
    k_d1_trace(const T *__restrict__ values, Geo<B> geo, uint8_t *flags, GradRec *grad,
               const unsigned long long *__restrict__ vcrit, const int32_t *__restrict__ v2, const uint8_t *__restrict__ l2,
               const int32_t *__restrict__ colmap, const int32_t *__restrict__ todo,
               int64_t ntodo, HeapEnt *heap_all, HashEnt *hash_all, int32_t *rows_all, int hcap,
               int hashcap, int rcap, int32_t gen_base, int32_t *pool, int64_t pool_cap,
               int64_t *col_start, int32_t *col_len, uint8_t *overflow,
               unsigned long long *next_col, int dense, int gens, DevStatus *st) {
    const StarTables &S = g_star;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    TraceCtx c;
    c.dense = dense != 0;
    c.gens = gens != 0;
    c.heap = heap_all + tid * hcap;
    c.hash = hash_all + tid * hashcap;
    c.rows = rows_all + tid * 2 * rcap;
    c.rslot = c.rows + rcap;
    c.hcap = hcap; c.hashmask = hashcap - 1; c.rcap = rcap;
    int32_t cj = -1;
    bool done = false;
    const GridParams *gp = nullptr;
    // every iteration runs the same two warp collectives on all lanes (the
    // ballot and the vote); the per-lane work after them has none.  A column
    // takes at most 2 * hashcap + 4 iterations (its start, a pop and two
    // toggles per pushed edge, its write-out), which bounds the loop.
    const int64_t max_iter = ntodo * (int64_t)(2 * hashcap + 8) + 64;
    // Pending toggles of this lane: the three edges of a column's start or the
    // two of an expansion.  One is done per iteration, so the lanes of a warp
    // run the toggle -- its loads, hash probe and heap push -- together,
    // whatever step their columns are at.
    int np = 0;
    int64_t y0 = 0, y1 = 0, y2 = 0;
    int m0 = 0, m1 = 0, m2 = 0;
    unsigned long long ntog = 0, nexp = 0;
    for (int64_t iter = 0;; iter++) {
        // lanes without a column take the next ones
        const bool need = cj < 0 && !done;
        const unsigned want = __ballot_sync(0xffffffffu, need);
        unsigned long long base = 0;
        if (want) {
            const int leader = __ffs(want) - 1;
            if (lane == leader) base = atomicAdd(next_col, (unsigned long long)__popc(want));
            base = __shfl_sync(0xffffffffu, base, leader);
        }
        bool started = false;
        if (need) {
            const int64_t q = (int64_t)base + __popc(want & lanemask_lt());
            if (q >= ntodo) done = true;
            else { cj = todo ? todo[q] : (int32_t)q; started = true; }
        }
        if (__all_sync(0xffffffffu, done)) break;
        if (iter >= max_iter) {                  // cannot happen: every step makes progress
            atomicOr(&st->err, kErrIter);
            break;
        }
        if (cj < 0) continue;
        if (np == 0) {
            if (started) {
                const int32_t j2 = colmap[cj];
                const int64_t x = v2[j2];
                gp = &geo.at(x);
                const int s = l2[j2];
                c.hn = 0; c.rn = 0; c.used = 0; c.overflow = false;
                c.gen = gen_base + cj;
                // boundary: (x,a), (x,b) and the edge between x+a and x+b, in the
                // star of the higher of the two
                const GradRec Gx = grad_get(S, *gp, values, flags, grad, x, c.dense);
                const int ta = S.tri_v[s][0], tb = S.tri_v[s][1];
                const bool aup = grad_rank(Gx, ta) > grad_rank(Gx, tb);
                const int hi = aup ? ta : tb, lo = aup ? tb : ta;
                y0 = x; m0 = ta;
                y1 = x; m1 = tb;
                y2 = x + gp->dlin[hi];
                m2 = S.link_of_dc[(S.dx[lo] - S.dx[hi] + 1) + 3 * (S.dy[lo] - S.dy[hi] + 1) +
                                  9 * (S.dz[lo] - S.dz[hi] + 1)];
                np = 3;
            } else if (c.hn > 0 && !c.overflow) {
                // one expansion, if the popped edge's parity is odd
                const HeapEnt top = heap_pop(c);
                const int64_t y = (int64_t)(top.lo >> 12);
                const int m = (int)(top.lo & 0xF);
                HashEnt *e = trace_find(c, y, m);
                if (e && hinfo_parity(e->info)) {
                    e->info &= ~(1u << 31);
                    const uint32_t spec = hinfo_aux(e->info);
                    y0 = y; m0 = (int)(spec & 15);
                    y1 = y + gp->dlin[(spec >> 4) & 15]; m1 = (int)((spec >> 8) & 15);
                    np = 2;
                    nexp++;
                }
            }
        }
        if (c.overflow) np = 0;                  // the column is dropped: no more toggles
        if (np > 0) {
            const int64_t ty = np == 3 ? y2 : np == 2 ? y1 : y0;
            const int tm = np == 3 ? m2 : np == 2 ? m1 : m0;
            np--;
            ntog++;
            trace_toggle<T>(c, S, *gp, values, flags, grad, vcrit, ty, tm, st);
            continue;
        }
        if (c.hn > 0 && !c.overflow) continue;
        // the column is complete (or outgrew the scratch): write it out
        const int32_t col = cj;
        cj = -1;
        if (c.overflow) {
            overflow[col] = 1;
            col_len[col] = 0;
            continue;
        }
        // the rows with odd multiplicity, sorted decreasingly
        int len = 0;
        for (int k = 0; k < c.rn; k++)
            if (hinfo_parity(c.hash[c.rslot[k]].info)) c.rows[len++] = c.rows[k];
        for (int k = 1; k < len; k++) {
            const int32_t v = c.rows[k];
            int p = k;
            while (p > 0 && c.rows[p - 1] < v) { c.rows[p] = c.rows[p - 1]; p--; }
            c.rows[p] = v;
        }
        overflow[col] = 0;
        if (len == 0) { col_len[col] = 0; col_start[col] = 0; continue; }
        const unsigned long long pos = atomicAdd(&st->pool_top, (unsigned long long)len);
        if ((int64_t)(pos + len) > pool_cap) {
            atomicOr(&st->err, kErrCap);
            col_len[col] = 0;
            continue;
        }
        for (int k = 0; k < len; k++) pool[pos + k] = c.rows[k];
        col_start[col] = (int64_t)pos;
        col_len[col] = len;
    }
    // the loop ends on warp-uniform conditions: all lanes are here
    for (int o = 16; o > 0; o >>= 1) {
        ntog += __shfl_down_sync(0xffffffffu, ntog, o);
        nexp += __shfl_down_sync(0xffffffffu, nexp, o);
    }
    if (lane == 0) {
        atomicAdd(&st->trace_work[0], ntog);
        atomicAdd(&st->trace_work[1], nexp);
    }
}

// --------------------------------------------- stage 7: D1 column reduction
//
// Standard reduction of the columns (increasing lexicographic order) with the
// pivot = the largest row (Alg. 3 = reduction restricted to critical columns,
// Sec. 4.2 (b)), run in rounds: every non-zero column claims its pivot with
// an atomic minimum over column indices; a column that lost its pivot to an
// earlier column adds that column's current boundary (mod 2).  The owner of a
// pivot never changes in a round, so the boundary it adds is stable; the
// owner of a row is always a column whose pivot is that row (the CAS
// "temporary pairs" of Sec. 7.2, made round-synchronous).

// Column lists are decreasing int32.  Rows (C1 indices) are >= 0; in the
// generator mode a column also carries passive entries, -(edge id + 1), for
// the edges the Morse boundary compresses away (heads of vertex->edge vectors
// and critical edges paired in D0): they sort after every row, are added mod
// 2 like rows and are never a pivot.  A column has a pivot iff its first
// entry is a row.  kListEnd is below every entry.
constexpr int32_t kListEnd = INT32_MIN;

// Appends v to list[*count] with one atomic per warp (all active lanes call).
__device__ __forceinline__ void warp_append(bool take, int32_t v, int32_t *list,
                                            unsigned long long *count) {
    unsigned m = __ballot_sync(__activemask(), take);
    if (!m) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(__activemask(), base, leader);
    if (take) list[base + __popc(m & lanemask_lt())] = v;
}

// Active columns (new pivots since the previous round) claim their pivots;
// a claim that displaces a later owner queues that owner for a recheck.
__global__ void k_red_claim(const int32_t *__restrict__ active, int64_t nactive,
                            const int64_t *__restrict__ start, const int32_t *__restrict__ len,
                            const int32_t *__restrict__ pool, int32_t *owner, int32_t *recheck,
                            DevStatus *st) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool take = false;
    int32_t old = 0;
    if (q < nactive) {
        int32_t cj = active[q];
        const int32_t piv = len[cj] > 0 ? pool[start[cj]] : -1;
        if (piv >= 0) {
            old = atomicMin(&owner[piv], cj);
            take = old != kNoOwner && old > cj;
        }
    }
    warp_append(take, old, recheck, (unsigned long long *)&st->misc[0]);
}

// The owner of each row with the owner's current list, published after the
// claims of a round so that an addition finds the column to add in one load
// (the owner's list is stable until the owner loses the row).
struct RowCol {
    long long start;
    int32_t len;
    int32_t col;     // kNoOwner: unclaimed (the whole record is memset 0x7F)
};

// Listed columns that won their pivot publish it.
__global__ void k_red_publish(const int32_t *__restrict__ active, int64_t nactive,
                              const int64_t *__restrict__ start, const int32_t *__restrict__ len,
                              const int32_t *__restrict__ pool, const int32_t *__restrict__ owner,
                              RowCol *rowcol) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nactive) return;
    const int32_t cj = active[q];
    const int l = len[cj];
    if (l <= 0) return;
    const long long s0 = start[cj];
    const int32_t r = pool[s0];
    if (r >= 0 && owner[r] == cj) rowcol[r] = RowCol{s0, l, cj};
}

// Every non-zero column that owns its pivot publishes it (after the pool moved).
__global__ void k_red_publish_all(int64_t ncol, const int64_t *__restrict__ start,
                                  const int32_t *__restrict__ len,
                                  const int32_t *__restrict__ pool,
                                  const int32_t *__restrict__ owner, RowCol *rowcol) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol || len[c] <= 0) return;
    const long long s0 = start[c];
    const int32_t r = pool[s0];
    if (r >= 0 && owner[r] == (int32_t)c) rowcol[r] = RowCol{s0, len[c], (int32_t)c};
}

// Merge path split of two decreasing lists: how many of the first d
// elements of their merge (ties: A first) come from A.  A tie that would
// straddle the split is moved to the earlier side, so that equal entries of A
// and B always meet in the same segment.
__device__ __forceinline__ void merge_split(const int32_t *A, int la, const int32_t *B, int lb,
                                            int d, int &i, int &j) {
    int lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (A[mid] >= B[d - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    i = lo;
    j = d - lo;
    if (i > 0 && j < lb && A[i - 1] == B[j]) j++;
}

// out = A + B (mod 2) for decreasing lists, by one warp; returns the length.
__device__ int warp_symdiff(const int32_t *A, int la, const int32_t *B, int lb, int32_t *out) {
    const int lane = threadIdx.x & 31;
    const int L = la + lb, per = (L + 31) >> 5;
    int i0, j0, i1, j1;
    merge_split(A, la, B, lb, min(lane * per, L), i0, j0);
    merge_split(A, la, B, lb, min(lane * per + per, L), i1, j1);
    int cnt = 0;
    {
        int i = i0, j = j0;
        while (i < i1 || j < j1) {
            int32_t x = i < i1 ? A[i] : kListEnd, y = j < j1 ? B[j] : kListEnd;
            if (x > y) { cnt++; i++; }
            else if (y > x) { cnt++; j++; }
            else { i++; j++; }
        }
    }
    int inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    int total = __shfl_sync(0xffffffffu, inc, 31);
    int o = inc - cnt;
    int i = i0, j = j0;
    while (i < i1 || j < j1) {
        int32_t x = i < i1 ? A[i] : kListEnd, y = j < j1 ? B[j] : kListEnd;
        if (x > y) { out[o++] = x; i++; }
        else if (y > x) { out[o++] = y; j++; }
        else { i++; j++; }                      // 1 + 1 = 0 (mod 2)
    }
    return total;
}

// The listed columns (active, then displaced owners) that add something in
// this round: their pivot is owned by an earlier column.  One thread per
// entry, so the common case -- a column that owns its pivot, or whose pivot
// is free or owned by a later column -- costs one thread's loads instead of
// a warp's turn; each column is taken once per round (stamp).  Owners do not
// change until the next claims, so the list is exactly the columns that
// k_red_add changes.
__global__ void k_red_need(const int32_t *__restrict__ active, int64_t nactive,
                           const int32_t *__restrict__ recheck,
                           const int64_t *__restrict__ start, const int32_t *__restrict__ len,
                           const int32_t *__restrict__ pool, const RowCol *__restrict__ rowcol,
                           int32_t *stamp, int32_t round, int32_t *work, DevStatus *st) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nre = *(volatile long long *)&st->misc[0];
    bool take = false;
    int32_t cj = 0;
    if (q < nactive + nre) {
        cj = q < nactive ? active[q] : recheck[q - nactive];
        if (atomicExch(&stamp[cj], round) != round && len[cj] > 0) {
            const int32_t head = pool[start[cj]];
            if (head >= 0) {
                const int32_t k = rowcol[head].col;
                take = k != kNoOwner && k < cj;
            }
        }
    }
    warp_append(take, cj, work, &st->red_work);
}

// One warp per column of the round's work list (k_red_need): while its pivot
// is owned by an earlier column, add that column (mod 2).  Owners never
// change inside this kernel (a column owns a row only while the row is its
// pivot, and claims happen in k_red_claim), so every column added is stable.
// Stops at its own pivot, an unclaimed pivot or one claimed by a later
// column (those claim it in the next round).
// Short columns stay in the warp's shared memory through their chain (the
// merge-path searches then probe shared memory, not the pool), and the
// added column is staged there too; the result is written to the pool once.
constexpr int kWarpAcc = 256;
__global__ void __launch_bounds__(256)
    k_red_add(const int32_t *__restrict__ work, int64_t *start, int32_t *len, int32_t *pool,
              const RowCol *__restrict__ rowcol, int32_t *next, int64_t pool_cap,
              DevStatus *st) {
    __shared__ int32_t wsm[8][3 * kWarpAcc];
    const int lane = threadIdx.x & 31;
    int32_t *acc[2] = {wsm[threadIdx.x >> 5], wsm[threadIdx.x >> 5] + kWarpAcc};
    int32_t *stg = wsm[threadIdx.x >> 5] + 2 * kWarpAcc;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nwork = (int64_t)*(volatile unsigned long long *)&st->red_work;
    unsigned adds = 0, longest = 0;
    unsigned long long io_r = 0, io_w = 0;
    for (int64_t q = warp; q < nwork; q += nwarps) {
        const int32_t cj = work[q];
        int la = len[cj];
        int64_t sa = start[cj];
        bool resident = la <= kWarpAcc;
        int cur = 0;
        if (resident) {
            for (int k = lane; k < la; k += 32) acc[0][k] = pool[sa + k];
            __syncwarp();
        }
        bool changed = false;
        unsigned chain = 0;
        for (int it = 0; la > 0 && it < (1 << 24); it++) {
            const int32_t head = resident ? acc[cur][0] : pool[sa];
            if (head < 0) break;                 // no row left: no pivot
            const RowCol rc = rowcol[head];
            const int32_t k = rc.col;
            if (k == cj || k == kNoOwner || k > cj) break;
            const int lb = rc.len;
            const int32_t *B = pool + rc.start;
            if (lb <= kWarpAcc) {
                for (int t = lane; t < lb; t += 32) stg[t] = B[t];
                __syncwarp();
                B = stg;
            }
            io_r += (unsigned long long)(la + lb);
            if (resident && la + lb <= kWarpAcc) {
                la = warp_symdiff(acc[cur], la, B, lb, acc[cur ^ 1]);
                cur ^= 1;
            } else {
                unsigned long long pos = 0;
                if (lane == 0) pos = atomicAdd(&st->pool_top, (unsigned long long)(la + lb));
                pos = __shfl_sync(0xffffffffu, pos, 0);
                if ((int64_t)(pos + la + lb) > pool_cap) {
                    if (lane == 0) atomicOr(&st->err, kErrCap);
                    break;
                }
                la = warp_symdiff(resident ? acc[cur] : pool + sa, la, B, lb, pool + pos);
                sa = (int64_t)pos;
                resident = false;
            }
            __syncwarp();
            io_w += (unsigned long long)la;
            changed = true;
            chain++;
        }
        if (changed && resident) {
            // the chain ended in shared memory: one write to the pool
            unsigned long long pos = 0;
            if (lane == 0 && la > 0) pos = atomicAdd(&st->pool_top, (unsigned long long)la);
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (la > 0 && (int64_t)(pos + la) > pool_cap) {
                if (lane == 0) atomicOr(&st->err, kErrCap);
                changed = false;                 // the column keeps its previous state
            } else {
                for (int t = lane; t < la; t += 32) pool[pos + t] = acc[cur][t];
                sa = (int64_t)pos;
            }
        }
        adds += chain;
        longest = max(longest, chain);
        __syncwarp();
        if (changed && lane == 0) {
            start[cj] = sa;
            len[cj] = la;
            if (la > 0 && pool[sa] >= 0) next[atomicAdd((unsigned long long *)&st->misc[1], 1ull)] = cj;
        }
        __syncwarp();
    }
    if (lane == 0 && adds) {
        atomicAdd((unsigned long long *)&st->misc[2], (unsigned long long)adds);
        atomicMax((unsigned long long *)&st->misc[3], (unsigned long long)longest);
        atomicAdd((unsigned long long *)&st->red_io[0], io_r * 4ull);
        atomicAdd((unsigned long long *)&st->red_io[1], io_w * 4ull);
    }
}

// out = A + B (mod 2) by a block of NT threads; both lists are staged in
// shared memory when they fit (cap entries each).  Returns the length.
template <int NT>
__device__ int block_symdiff(const int32_t *A, int la, const int32_t *B, int lb, int32_t *out,
                             int32_t *sA, int32_t *sB, int cap, int *sscan) {
    const int t = threadIdx.x;
    if (sA && la <= cap && lb <= cap) {
        for (int k = t; k < la; k += NT) sA[k] = A[k];
        for (int k = t; k < lb; k += NT) sB[k] = B[k];
        __syncthreads();
        A = sA;
        B = sB;
    }
    const int L = la + lb, per = (L + NT - 1) / NT;
    int i0, j0, i1, j1;
    merge_split(A, la, B, lb, min(t * per, L), i0, j0);
    merge_split(A, la, B, lb, min(t * per + per, L), i1, j1);
    int cnt = 0;
    {
        int i = i0, j = j0;
        while (i < i1 || j < j1) {
            int32_t x = i < i1 ? A[i] : kListEnd, y = j < j1 ? B[j] : kListEnd;
            if (x > y) { cnt++; i++; }
            else if (y > x) { cnt++; j++; }
            else { i++; j++; }
        }
    }
    // block exclusive scan of cnt
    const int lane = t & 31, w = t >> 5;
    int inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) sscan[w] = inc;
    __syncthreads();
    int pre = 0, total = 0;
    for (int q = 0; q < NT / 32; q++) { if (q < w) pre += sscan[q]; total += sscan[q]; }
    int o = pre + inc - cnt;
    int i = i0, j = j0;
    while (i < i1 || j < j1) {
        int32_t x = i < i1 ? A[i] : kListEnd, y = j < j1 ? B[j] : kListEnd;
        if (x > y) { out[o++] = x; i++; }
        else if (y > x) { out[o++] = y; j++; }
        else { i++; j++; }
    }
    __syncthreads();   // smem reused by the next addition
    return total;
}

// The same as k_red_add with one block per listed column, for the last rounds
// where few columns remain and their chains of additions are long.  The
// column being reduced stays in shared memory (two buffers) while it fits:
// an addition reads only the added column from global memory; the result is
// written back once at the end.  A column that outgrows the buffers continues
// with merges through the global pool.
constexpr int kRedBlock = 512, kRedAcc = 24576, kRedStage = 4096;
constexpr size_t kRedSmem = sizeof(int32_t) * (2 * kRedAcc + kRedStage);
constexpr int kAsyncBlock = 256, kAsyncAcc = 12288, kAsyncStage = 2048;
constexpr size_t kAsyncSmem = sizeof(int32_t) * (2 * kAsyncAcc + kAsyncStage);
__global__ void __launch_bounds__(kRedBlock)
    k_red_add_block(const int32_t *__restrict__ active, int64_t nactive,
                    const int32_t *__restrict__ recheck, int64_t *start, int32_t *len,
                    int32_t *pool, const RowCol *__restrict__ rowcol, int32_t *stamp,
                    int32_t round, int32_t *next, int64_t pool_cap, DevStatus *st) {
    extern __shared__ int32_t smem[];
    int32_t *acc[2] = {smem, smem + kRedAcc};
    int32_t *sB = smem + 2 * kRedAcc;
    __shared__ int sscan[kRedBlock / 32];
    __shared__ int32_t s_cj, s_fresh;
    __shared__ RowCol s_rc;
    __shared__ unsigned long long s_pos;
    const int64_t nre = *(volatile long long *)&st->misc[0];
    const int64_t q = blockIdx.x;
    if (q >= nactive + nre) return;
    if (threadIdx.x == 0) {
        s_cj = q < nactive ? active[q] : recheck[q - nactive];
        s_fresh = atomicExch(&stamp[s_cj], round) != round;
    }
    __syncthreads();
    if (!s_fresh) return;
    const int32_t cj = s_cj;
    int la = len[cj];
    int64_t sa = start[cj];
    // resident: the column lives in acc[cur]; otherwise at pool[sa]
    bool resident = la <= kRedAcc;
    int cur = 0;
    if (resident) {
        for (int k = threadIdx.x; k < la; k += kRedBlock) acc[0][k] = pool[sa + k];
        __syncthreads();
    }
    bool changed = false, failed = false;
    unsigned chain = 0;
    unsigned long long io_r = 0, io_w = 0;
    // thread 0 keeps the owner record of the next pivot; it is loaded for the
    // predicted pivot before each merge, so its latency overlaps the merge
    RowCol pre{0, 0, kNoOwner};
    if (threadIdx.x == 0 && la > 0) {
        const int32_t head = resident ? acc[0][0] : pool[sa];
        if (head >= 0) pre = rowcol[head];
    }
    for (int it = 0; la > 0 && it < (1 << 24); it++) {
        if (threadIdx.x == 0) s_rc = pre;
        __syncthreads();
        const int32_t k = s_rc.col;
        if (k == cj || k == kNoOwner || k > cj) break;
        const int64_t sb = s_rc.start;
        const int lb = s_rc.len;
        const int32_t *B = pool + sb;
        if (lb <= kRedStage) {
            for (int t = threadIdx.x; t < lb; t += kRedBlock) sB[t] = B[t];
            B = sB;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            // the pivot after this addition: the first entry past the two
            // cancelling tops that the lists do not share
            const int32_t *A = resident ? acc[cur] : pool + sa;
            int i = 1, j = 1;
            int32_t nt = kListEnd;
            while (i < la || j < lb) {
                const int32_t x = i < la ? A[i] : kListEnd, y = j < lb ? B[j] : kListEnd;
                if (x != y) { nt = x > y ? x : y; break; }
                i++; j++;
            }
            pre = nt >= 0 ? rowcol[nt] : RowCol{0, 0, kNoOwner};
        }
        io_r += (unsigned long long)(la + lb);
        if (resident && la + lb <= kRedAcc) {
            __syncthreads();
            la = block_symdiff<kRedBlock>(acc[cur], la, B, lb, acc[cur ^ 1], nullptr, nullptr, 0,
                                          sscan);
            cur ^= 1;
        } else {
            if (threadIdx.x == 0) s_pos = atomicAdd(&st->pool_top, (unsigned long long)(la + lb));
            __syncthreads();
            const unsigned long long pos = s_pos;
            if ((int64_t)(pos + la + lb) > pool_cap) {
                if (threadIdx.x == 0) atomicOr(&st->err, kErrCap);
                failed = true;
                break;
            }
            la = block_symdiff<kRedBlock>(resident ? acc[cur] : pool + sa, la, B, lb, pool + pos,
                                          nullptr, nullptr, 0, sscan);
            sa = (int64_t)pos;
            resident = false;
        }
        io_w += (unsigned long long)la;
        changed = true;
        chain++;
    }
    if (changed && resident && !failed) {
        // write the reduced column back to the pool
        if (threadIdx.x == 0) s_pos = la ? atomicAdd(&st->pool_top, (unsigned long long)la) : 0;
        __syncthreads();
        const unsigned long long pos = s_pos;
        if ((int64_t)(pos + la) > pool_cap) {
            if (threadIdx.x == 0) atomicOr(&st->err, kErrCap);
            changed = false;    // the column keeps its previous state
        } else {
            for (int t = threadIdx.x; t < la; t += kRedBlock) pool[pos + t] = acc[cur][t];
            sa = (int64_t)pos;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (changed) {
            start[cj] = sa;
            len[cj] = la;
            if (la > 0 && pool[sa] >= 0) next[atomicAdd((unsigned long long *)&st->misc[1], 1ull)] = cj;
        }
        if (chain) {
            atomicAdd((unsigned long long *)&st->misc[2], (unsigned long long)chain);
            atomicMax((unsigned long long *)&st->misc[3], (unsigned long long)chain);
            atomicAdd((unsigned long long *)&st->red_io[0], io_r * 4ull);
            atomicAdd((unsigned long long *)&st->red_io[1], io_w * 4ull);
        }
    }
}

// ---- the tail of the reduction, asynchronous
//
// Once few columns remain active, the rounds are dominated by their longest
// chain of additions while displaced columns wait for the round to end.  This
// persistent kernel runs the same reduction without rounds (the lock-free
// form of Sec. 7.2's temporary pairs): blocks take columns from a device
// queue; a column adds the current list of the owner of its pivot while that
// owner is an earlier column, and takes the pivot by compare-and-swap when it
// is unowned or owned by a later column, which then goes back to the queue.
// Any list a column o has held is a sum of columns <= o whose top is o's
// pivot at that time, so adding a snapshot of an earlier column's list is a
// valid step of the reduction even if that column is being displaced
// meanwhile; the pivots reached are those of the standard reduction.  A
// column's list is published (start << 32 | length, one 64-bit word) before
// the compare-and-swap that makes it an owner.
struct AsyncQ {
    unsigned int head, tail;
    int pending;       // columns queued or in progress
    int abort;         // the pool or the queue filled up: stop taking columns
};

// A list written by another block in this kernel is read from L2 (ld.cg): an
// L1 line cached while reading a neighbouring list could hold stale entries.
template <bool G>
__device__ __forceinline__ int32_t ld_list(const int32_t *p) {
    if constexpr (G) return __ldcg(p);
    else return *p;
}

template <bool AG, bool BG>
__device__ __forceinline__ void merge_split_g(const int32_t *A, int la, const int32_t *B, int lb,
                                              int d, int &i, int &j) {
    int lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (ld_list<AG>(A + mid) >= ld_list<BG>(B + d - 1 - mid)) lo = mid + 1;
        else hi = mid;
    }
    i = lo;
    j = d - lo;
    if (i > 0 && j < lb && ld_list<AG>(A + i - 1) == ld_list<BG>(B + j)) j++;
}

// block_symdiff with global operands read from L2 (AG / BG: A / B in global memory)
template <int NT, bool AG, bool BG>
__device__ int block_symdiff_g(const int32_t *A, int la, const int32_t *B, int lb, int32_t *out,
                               int *sscan) {
    const int t = threadIdx.x;
    const int L = la + lb, per = (L + NT - 1) / NT;
    int i0, j0, i1, j1;
    merge_split_g<AG, BG>(A, la, B, lb, min(t * per, L), i0, j0);
    merge_split_g<AG, BG>(A, la, B, lb, min(t * per + per, L), i1, j1);
    int cnt = 0;
    {
        int i = i0, j = j0;
        while (i < i1 || j < j1) {
            int32_t x = i < i1 ? ld_list<AG>(A + i) : kListEnd, y = j < j1 ? ld_list<BG>(B + j) : kListEnd;
            if (x > y) { cnt++; i++; }
            else if (y > x) { cnt++; j++; }
            else { i++; j++; }
        }
    }
    const int lane = t & 31, w = t >> 5;
    int inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) sscan[w] = inc;
    __syncthreads();
    int pre = 0, total = 0;
    for (int q = 0; q < NT / 32; q++) { if (q < w) pre += sscan[q]; total += sscan[q]; }
    int o = pre + inc - cnt;
    int i = i0, j = j0;
    while (i < i1 || j < j1) {
        int32_t x = i < i1 ? ld_list<AG>(A + i) : kListEnd, y = j < j1 ? ld_list<BG>(B + j) : kListEnd;
        if (x > y) { out[o++] = x; i++; }
        else if (y > x) { out[o++] = y; j++; }
        else { i++; j++; }
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ unsigned long long pack_list(int64_t start, int32_t len) {
    return ((unsigned long long)start << 32) | (uint32_t)len;
}

__device__ __forceinline__ void aq_push(AsyncQ *q, int32_t *queue, unsigned int qcap, int32_t c,
                                        bool count, DevStatus *st) {
    if (count) atomicAdd(&q->pending, 1);
    const unsigned int i = atomicAdd(&q->tail, 1u);
    if (i >= qcap) {                     // cannot happen with the capacity reserved
        atomicOr(&st->err, kErrCap);
        atomicExch(&q->abort, 1);
        return;
    }
    ((volatile int32_t *)queue)[i] = c;
    __threadfence();
}

template <int NT, int ACC, int STAGE>
__global__ void __launch_bounds__(NT)
    k_red_async(AsyncQ *q, int32_t *queue, unsigned int qcap, int32_t *owner,
                unsigned long long *info, int64_t *start, int32_t *len, int32_t *pool,
                int64_t pool_cap, DevStatus *st) {
    extern __shared__ int32_t smem[];
    int32_t *acc[2] = {smem, smem + ACC};
    int32_t *sB = smem + 2 * ACC;
    __shared__ int sscan[NT / 32];
    __shared__ int32_t s_cj, s_o, s_state;
    __shared__ unsigned long long s_rec, s_pos;
    const int t = threadIdx.x;
    unsigned adds = 0;
    unsigned long long io_r = 0, io_w = 0;
    for (;;) {
        // take a column (thread 0), or leave once nothing is queued or in progress
        if (t == 0) {
            s_cj = -1;
            for (int spin = 0; spin < (1 << 22); spin++) {
                if (*(volatile int *)&q->abort) break;
                const unsigned int h = *(volatile unsigned int *)&q->head;
                const unsigned int tl = *(volatile unsigned int *)&q->tail;
                if (h < tl && h < qcap) {
                    if (atomicCAS(&q->head, h, h + 1) != h) continue;
                    int32_t c = -1;
                    for (int w = 0; w < (1 << 20) && c < 0; w++) {
                        c = ((volatile int32_t *)queue)[h];
                        if (c < 0) __nanosleep(64);
                    }
                    if (c < 0) { atomicOr(&st->err, kErrIter); atomicExch(&q->abort, 1); }
                    s_cj = c;
                    break;
                }
                if (*(volatile int *)&q->pending == 0) break;
                __nanosleep(256);
                if (spin == (1 << 22) - 1) { atomicOr(&st->err, kErrIter); atomicExch(&q->abort, 1); }
            }
        }
        __syncthreads();
        const int32_t cj = s_cj;
        if (cj < 0) break;
        if (t == 0) s_rec = *(volatile unsigned long long *)&info[cj];
        __syncthreads();
        int la = (int)(uint32_t)(s_rec & 0xffffffffull);
        int64_t sa = (int64_t)(s_rec >> 32);
        bool resident = la <= ACC;
        int cur = 0;
        if (resident) {
            for (int k = t; k < la; k += NT) acc[0][k] = __ldcg(pool + sa + k);
            __syncthreads();
        }
        // state: 0 working, 1 done, 2 stopped (pool full: requeued)
        int state = 0;
        for (int it = 0; state == 0 && it < (1 << 24); it++) {
            if (la == 0) {
                if (t == 0) {
                    *(volatile unsigned long long *)&info[cj] = pack_list(0, 0);
                    start[cj] = 0;
                    len[cj] = 0;
                }
                state = 1;
                break;
            }
            if (t == 0) s_o = *(volatile int32_t *)&owner[resident ? acc[cur][0] : __ldcg(pool + sa)];
            __syncthreads();
            const int32_t o = s_o;
            if (o == cj) { state = 1; break; }             // already the owner
            if (o != kNoOwner && o < cj) {
                // add the earlier owner's current list
                if (t == 0) s_rec = *(volatile unsigned long long *)&info[o];
                __syncthreads();
                const int lb = (int)(uint32_t)(s_rec & 0xffffffffull);
                const int32_t *B = pool + (int64_t)(s_rec >> 32);
                const bool staged = lb <= STAGE;
                if (staged) {
                    for (int k = t; k < lb; k += NT) sB[k] = __ldcg(B + k);
                    B = sB;
                }
                io_r += (unsigned long long)(la + lb);
                if (resident && la + lb <= ACC) {
                    __syncthreads();
                    la = staged ? block_symdiff_g<NT, false, false>(acc[cur], la, B, lb,
                                                                           acc[cur ^ 1], sscan)
                                : block_symdiff_g<NT, false, true>(acc[cur], la, B, lb,
                                                                          acc[cur ^ 1], sscan);
                    cur ^= 1;
                } else {
                    if (t == 0) s_pos = atomicAdd(&st->pool_top, (unsigned long long)(la + lb));
                    __syncthreads();
                    const unsigned long long pos = s_pos;
                    if ((int64_t)(pos + la + lb) > pool_cap) {
                        if (t == 0) { atomicOr(&st->err, kErrCap); atomicExch(&q->abort, 1); }
                        state = 2;
                        break;
                    }
                    __syncthreads();
                    if (resident)
                        la = staged ? block_symdiff_g<NT, false, false>(acc[cur], la, B, lb,
                                                                               pool + pos, sscan)
                                    : block_symdiff_g<NT, false, true>(acc[cur], la, B, lb,
                                                                              pool + pos, sscan);
                    else
                        la = staged ? block_symdiff_g<NT, true, false>(pool + sa, la, B, lb,
                                                                              pool + pos, sscan)
                                    : block_symdiff_g<NT, true, true>(pool + sa, la, B, lb,
                                                                             pool + pos, sscan);
                    sa = (int64_t)pos;
                    resident = false;
                }
                io_w += (unsigned long long)la;
                adds++;
                continue;
            }
            // unowned, or owned by a later column: publish the list and take the pivot
            __threadfence();
            __syncthreads();
            if (resident) {
                if (t == 0) s_pos = atomicAdd(&st->pool_top, (unsigned long long)la);
                __syncthreads();
                const unsigned long long pos = s_pos;
                if ((int64_t)(pos + la) > pool_cap) {
                    if (t == 0) { atomicOr(&st->err, kErrCap); atomicExch(&q->abort, 1); }
                    state = 2;
                    break;
                }
                for (int k = t; k < la; k += NT) pool[pos + k] = acc[cur][k];
                sa = (int64_t)pos;
                resident = false;
                __threadfence();
                __syncthreads();
            }
            if (t == 0) {
                start[cj] = sa;
                len[cj] = la;
                *(volatile unsigned long long *)&info[cj] = pack_list(sa, la);
                __threadfence();
                const int32_t prev = atomicCAS(&owner[__ldcg(pool + sa)], o, cj);
                s_state = prev == o ? 1 : 0;
                if (prev == o && o != kNoOwner) aq_push(q, queue, qcap, o, true, st);
            }
            __syncthreads();
            state = s_state;
            // on a lost race the owner is read again; the list stays in the pool
            if (state == 0) {
                resident = la <= ACC;
                if (resident) {
                    cur = 0;
                    for (int k = t; k < la; k += NT) acc[0][k] = __ldcg(pool + sa + k);
                    __syncthreads();
                }
            }
        }
        __syncthreads();
        if (state == 0 && t == 0) {        // the chain bound ran out
            atomicOr(&st->err, kErrIter);
            atomicExch(&q->abort, 1);
        }
        if (t == 0) {
            if (state == 2) {
                // the column keeps its last published list; it goes back to the queue
                aq_push(q, queue, qcap, cj, false, st);
            } else {
                atomicSub(&q->pending, 1);
            }
        }
        __syncthreads();
    }
    if (t == 0 && adds) {
        atomicAdd((unsigned long long *)&st->misc[2], (unsigned long long)adds);
        atomicAdd((unsigned long long *)&st->red_io[0], io_r * 4ull);
        atomicAdd((unsigned long long *)&st->red_io[1], io_w * 4ull);
    }
}

// info[c] = start << 32 | length of every column
__global__ void k_pack_info(int64_t ncol, const int64_t *__restrict__ start,
                            const int32_t *__restrict__ len, unsigned long long *info) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncol) info[c] = pack_list(start[c], len[c]);
}

__global__ void k_iota32(int32_t *p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

// ---- the anti-transpose of the column set (persistent cohomology): the
// rows, in decreasing order, become columns whose entries are the original
// columns, also reversed (entry kappa = ncols-1-c), so that the pivot (the
// largest entry) is the oldest column.  Reducing it yields the same pairs.

// rho(r) = nrows-1-rowpos[r] for the rows (critical edges not paired in D0)
__global__ void k_co_count(int64_t ncols, const int64_t *__restrict__ start,
                           const int32_t *__restrict__ len, const int32_t *__restrict__ pool,
                           const int32_t *__restrict__ rowpos, int64_t nrows, int32_t *cnt) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    int64_t s0 = start[c];
    for (int k = 0; k < len[c]; k++) atomicAdd(&cnt[nrows - 1 - rowpos[pool[s0 + k]]], 1);
}

__global__ void k_co_scatter(int64_t ncols, const int64_t *__restrict__ start,
                             const int32_t *__restrict__ len, const int32_t *__restrict__ pool,
                             const int32_t *__restrict__ rowpos, int64_t nrows,
                             const int32_t *__restrict__ costart, int32_t *fill, int32_t *copool) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    int64_t s0 = start[c];
    int32_t kappa = (int32_t)(ncols - 1 - c);
    for (int k = 0; k < len[c]; k++) {
        int64_t rho = nrows - 1 - rowpos[pool[s0 + k]];
        int32_t at = atomicAdd(&fill[rho], 1);
        copool[costart[rho] + at] = kappa;
    }
}

// sorts each cocolumn decreasingly (heap sort in place)
__global__ void k_co_sort(int64_t nrows, const int32_t *__restrict__ costart,
                          const int32_t *__restrict__ cnt, int32_t *copool, int64_t *start) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int32_t *a = copool + costart[r];
    int n = cnt[r];
    start[r] = costart[r];
    if (n <= 16) {
        for (int i = 1; i < n; i++) {
            int32_t v = a[i];
            int p = i;
            while (p > 0 && a[p - 1] < v) { a[p] = a[p - 1]; p--; }
            a[p] = v;
        }
        return;
    }
    // min-heap sort gives decreasing order
    auto sift = [&](int i, int m) {
        while (true) {
            int l = 2 * i + 1, b = i;
            if (l < m && a[l] < a[b]) b = l;
            if (l + 1 < m && a[l + 1] < a[b]) b = l + 1;
            if (b == i) return;
            int32_t t = a[i]; a[i] = a[b]; a[b] = t;
            i = b;
        }
    };
    for (int i = n / 2 - 1; i >= 0; i--) sift(i, n);
    for (int m = n - 1; m > 0; m--) {
        int32_t t = a[0]; a[0] = a[m]; a[m] = t;
        sift(0, m);
    }
}

// per-column D1 partner row (-1: the column stays unpaired) and row flags
__global__ void k_d1_result_homology(int64_t ncols, const int64_t *__restrict__ start,
                                     const int32_t *__restrict__ len,
                                     const int32_t *__restrict__ pool, int32_t *d1_row,
                                     uint8_t *row_paired) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    int32_t r = len[c] > 0 ? pool[start[c]] : -1;
    if (r < 0) r = -1;                  // no row: no pivot (passive entries only)
    d1_row[c] = r;
    if (r >= 0) row_paired[r] = 1;
}

__global__ void k_d1_result_cohomology(int64_t nrows, int64_t ncols,
                                       const int64_t *__restrict__ start,
                                       const int32_t *__restrict__ len,
                                       const int32_t *__restrict__ pool,
                                       const int32_t *__restrict__ rowmap, int32_t *d1_row,
                                       uint8_t *row_paired) {
    int64_t rho = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (rho >= nrows || len[rho] == 0) return;
    int32_t kappa = pool[start[rho]];
    int32_t r = rowmap[nrows - 1 - rho];
    d1_row[ncols - 1 - kappa] = r;
    row_paired[r] = 1;
}

// copies the live columns into a fresh pool (after an overflow)
__global__ void k_pool_compact(int64_t ncol, int64_t *start, const int32_t *__restrict__ len,
                               const int32_t *__restrict__ off, const int32_t *__restrict__ src,
                               int32_t *dst) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    int64_t s0 = start[c];
    int32_t o = off[c];
    for (int k = 0; k < len[c]; k++) dst[o + k] = src[s0 + k];
    start[c] = o;
}


// ------------------------------ D1, lazy: propagation interleaved with the reduction
//
// Alg. 3 as the paper states it: a column keeps its boundary only partially
// expanded (the cached Boundary), and expands it only as far as the pivot.
// Here a column is a set of star edges E with Morse boundary Phi(E), Phi
// linear mod 2: a critical row maps to itself, a regular edge to the image of
// the other two edges of its paired triangle, a vertex->edge head and a
// critical edge paired in D0 to nothing.  E is kept sorted by decreasing
// priority (the vertex order of the edge's maximum vertex y, then the edge's
// classification order inside the lower star of y).  Expanding a regular
// edge only yields edges of lower priority (the other edge of the triangle
// was classified earlier in the same lower star, the third edge lies in the
// lower star of a lower vertex), and the critical edges of one lower star are
// classified in increasing lexicographic order.  So when the highest-priority
// edge of E with odd multiplicity is critical, it is the largest row of
// Phi(E): the pivot.  Advancing a column expands its top until that holds.
// The reduction rounds are those of the eager path (claims by atomic minimum,
// additions of stable owners), with E + E' (mod 2) in place of the sum of
// the expanded boundaries; a column whose top turns regular is advanced at
// the start of the next round.
//
// Entry: hi = key of the value at y; lo = y << 15 | order << 11 | m << 7 |
// pair << 1 | critical (pair: the star triangle of y a regular edge is paired
// with; 0 for a critical edge).  (hi, lo) orders by (key, y, order).
struct Ent {
    unsigned long long hi, lo;
};
__device__ __forceinline__ bool ent_gt(const Ent &a, const Ent &b) {
    return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ bool ent_eq(const Ent &a, const Ent &b) {
    return a.hi == b.hi && a.lo == b.lo;
}
__device__ __forceinline__ int64_t ent_y(const Ent &e) { return (int64_t)(e.lo >> 15); }
__device__ __forceinline__ int ent_m(const Ent &e) { return (int)((e.lo >> 7) & 15); }
__device__ __forceinline__ int ent_pair(const Ent &e) { return (int)((e.lo >> 1) & 63); }
__device__ __forceinline__ bool ent_crit(const Ent &e) { return e.lo & 1; }

// C1 index of the critical edge (y, link m)
__device__ __forceinline__ int32_t crit_edge_row(const StarTables &S,
                                                 const int32_t *__restrict__ vrank,
                                                 const CritRec *__restrict__ recs,
                                                 const int32_t *__restrict__ base1, int64_t y,
                                                 int m) {
    const int32_t i = vrank[y];
    const CritRec rec = recs[i];
    return base1[i] + local_index(S, rec, 1, m);
}

// Per-thread scratch of an advance: a max-heap of the edges produced by
// expansions and a hash of their parities (the list's own entries are merged
// in order, not hashed).
struct LazyCtx {
    HeapEnt *heap;
    HashEnt *hash;
    int hcap, hashmask, hn, used;
    int32_t gen;
    bool overflow;
    bool dense;        // every record was computed before the walks: nothing
                       // writes flags or records meanwhile, so they may be
                       // cached in L1
    bool gens;         // generator mode: compressed edges kept as passive entries
};

__device__ __forceinline__ HashEnt *lz_find(LazyCtx &c, unsigned long long key) {
    const uint32_t hpos = hash64(key) & c.hashmask;
    for (int p = 0; p <= c.hashmask; p++) {
        HashEnt *e = &c.hash[(hpos + p) & c.hashmask];
        if (e->gen != c.gen) return nullptr;
        if (e->key == key) return e;
    }
    return nullptr;
}
__device__ __forceinline__ unsigned long long lz_key(int64_t y, int m) {
    return (((unsigned long long)y << 4) | (unsigned)m) + 1;
}

// Toggles edge (y, m) among the products; drops heads of vertex->edge vectors
// and critical edges paired in D0.  A new edge is pushed with its entry.
template <typename T>
__device__ void lz_toggle(LazyCtx &c, const StarTables &S, const GridParams &g,
                          const T *__restrict__ values, uint8_t *flags, GradRec *grad,
                          const int32_t *__restrict__ vrank, const CritRec *__restrict__ recs,
                          const int32_t *__restrict__ base1, const uint8_t *__restrict__ is_row,
                          int64_t y, int m, DevStatus *st) {
    if (m < 0 || m >= kLinks) { atomicOr(&st->err, kErrState); c.overflow = true; return; }
    const uint8_t fy = flags[y];
    if ((fy & 0xF) == m) return;
    bool crit = false;
    if (fy & kFlagCritical) {
        const int32_t i = vrank[y];
        const CritRec rec = recs[i];
        if (rec.crit_e >> m & 1) {
            if (!is_row[base1[i] + local_index(S, rec, 1, m)]) return;   // paired in D0
            crit = true;
        }
    }
    const unsigned long long key = lz_key(y, m);
    const uint32_t hpos = hash64(key) & c.hashmask;
    HashEnt *slot = nullptr;
    for (int p = 0; p <= c.hashmask; p++) {
        HashEnt *e = &c.hash[(hpos + p) & c.hashmask];
        if (e->gen != c.gen) { slot = e; break; }
        if (e->key == key) { e->info ^= 1u; return; }
    }
    if (!slot || c.used * 4 >= (c.hashmask + 1) * 3 || c.hn >= c.hcap) {
        c.overflow = true;
        return;
    }
    const GradRec G = grad_get(S, g, values, flags, grad, y);
    int pair = 0;
    if (!crit) {
        pair = grad_edge_pair(G, m);
        if (pair >= kTris) { atomicOr(&st->err, kErrState); c.overflow = true; return; }
    }
    HeapEnt he;
    he.hi = (unsigned long long)Key<T>::of(values[y]);
    he.lo = ((unsigned long long)y << 15) | ((unsigned long long)grad_edge_order(G, m) << 11) |
            ((unsigned long long)m << 7) | ((unsigned long long)pair << 1) |
            (crit ? 1ull : 0ull);
    int i = c.hn++;
    while (i > 0) {
        const int p = (i - 1) >> 1;
        if (!heap_less(c.heap[p], he)) break;
        c.heap[i] = c.heap[p];
        i = p;
    }
    c.heap[i] = he;
    slot->key = key;
    slot->gen = c.gen;
    slot->info = 1u;
    c.used++;
}

__device__ __forceinline__ HeapEnt lz_pop(LazyCtx &c) {
    const HeapEnt top = c.heap[0];
    const HeapEnt last = c.heap[--c.hn];
    int i = 0;
    while (true) {
        const int l = 2 * i + 1;
        if (l >= c.hn) break;
        const int r = l + 1;
        const int m = (r < c.hn && heap_less(c.heap[l], c.heap[r])) ? r : l;
        if (!heap_less(last, c.heap[m])) break;
        c.heap[i] = c.heap[m];
        i = m;
    }
    if (c.hn > 0) c.heap[i] = last;
    return top;
}

// Expansion of regular edge (y, m) through its paired star triangle s: the
// other star edge of s and the edge between its two link vertices, in the
// star of the higher one.
template <typename T>
__device__ __forceinline__ void lz_expand(LazyCtx &c, const StarTables &S, const GridParams &g,
                                          const T *__restrict__ values, uint8_t *flags,
                                          GradRec *grad, const int32_t *__restrict__ vrank,
                                          const CritRec *__restrict__ recs,
                                          const int32_t *__restrict__ base1,
                                          const uint8_t *__restrict__ is_row, int64_t y, int s,
                                          int m, DevStatus *st) {
    const int ta = S.tri_v[s][0], tb = S.tri_v[s][1];
    if (m >= 0) lz_toggle<T>(c, S, g, values, flags, grad, vrank, recs, base1, is_row, y,
                             ta == m ? tb : ta, st);
    const GradRec G = grad_get(S, g, values, flags, grad, y);
    const bool aup = grad_rank(G, ta) > grad_rank(G, tb);
    const int hi = aup ? ta : tb, lo = aup ? tb : ta;
    const int l = S.link_of_dc[(S.dx[lo] - S.dx[hi] + 1) + 3 * (S.dy[lo] - S.dy[hi] + 1) +
                               9 * (S.dz[lo] - S.dz[hi] + 1)];
    lz_toggle<T>(c, S, g, values, flags, grad, vrank, recs, base1, is_row, y + g.dlin[hi], l, st);
}

// Advances column cj (list at sa, la entries; la < 0: no list yet, start
// from the boundary of the critical triangle) until its top is a critical
// row or it is zero, and writes it back as a new list.  Returns 0 when done
// (col_start/col_len updated), 1 when the products outgrow the scratch, 2
// when the pool is full; the column is unchanged then.
template <typename T>
__device__ int lz_advance_col(LazyCtx &c, const StarTables &S, const T *__restrict__ values,
                              const GridParams &g, uint8_t *flags, GradRec *grad,
                              const int32_t *__restrict__ vrank, const CritRec *__restrict__ recs,
                              const int32_t *__restrict__ base1,
                              const uint8_t *__restrict__ is_row, const int32_t *__restrict__ v2,
                              const uint8_t *__restrict__ l2, const int32_t *__restrict__ colmap,
                              int32_t cj, int la, int64_t sa, Ent *pool, int64_t pool_cap,
                              int64_t *col_start, int32_t *col_len, DevStatus *st) {
    c.hn = 0; c.used = 0; c.overflow = false;
    const Ent *L = pool + sa;
    int li = 0;
    const int ln = la > 0 ? la : 0;
    if (la < 0) {
        // the boundary of the critical triangle: (x,a), (x,b), edge(x+a, x+b)
        const int32_t j2 = colmap[cj];
        const int64_t x = v2[j2];
        const int s = l2[j2];
        lz_toggle<T>(c, S, g, values, flags, grad, vrank, recs, base1, is_row, x, S.tri_v[s][0],
                     st);
        lz_expand<T>(c, S, g, values, flags, grad, vrank, recs, base1, is_row, x, s,
                     S.tri_v[s][0], st);
    }
    Ent stop{0, 0};
    bool have = false;
    while (!c.overflow) {
        const bool hl = li < ln;
        if (!hl && c.hn == 0) break;
        Ent e;
        int par;
        if (c.hn > 0 && (!hl || !ent_gt(L[li], Ent{c.heap[0].hi, c.heap[0].lo}))) {
            const HeapEnt h = lz_pop(c);
            e = Ent{h.hi, h.lo};
            HashEnt *slot = lz_find(c, lz_key(ent_y(e), ent_m(e)));
            par = slot ? (int)(slot->info & 1u) : 0;
            if (hl && ent_eq(L[li], e)) { par ^= 1; li++; }
        } else {
            e = L[li++];
            par = 1;
        }
        if (!par) continue;
        if (ent_crit(e)) { stop = e; have = true; break; }
        lz_expand<T>(c, S, g, values, flags, grad, vrank, recs, base1, is_row, ent_y(e),
                     ent_pair(e), ent_m(e), st);
    }
    if (c.overflow) return 1;
    // write back: the stop row, then the rest of the list merged with the
    // remaining products of odd parity
    const int64_t room = (have ? 1 : 0) + (ln - li) + c.hn;
    if (room == 0) { col_start[cj] = 0; col_len[cj] = 0; return 0; }
    const unsigned long long pos = atomicAdd(&st->pool_top, (unsigned long long)room);
    if ((int64_t)(pos + room) > pool_cap) { atomicOr(&st->err, kErrCap); return 2; }
    Ent *out = pool + pos;
    int o = 0;
    if (have) out[o++] = stop;
    while (li < ln || c.hn > 0) {
        if (c.hn > 0 && (li >= ln || !ent_gt(L[li], Ent{c.heap[0].hi, c.heap[0].lo}))) {
            const HeapEnt h = lz_pop(c);
            const Ent e{h.hi, h.lo};
            HashEnt *slot = lz_find(c, lz_key(ent_y(e), ent_m(e)));
            int par = slot ? (int)(slot->info & 1u) : 0;
            if (li < ln && ent_eq(L[li], e)) { par ^= 1; li++; }
            if (par) out[o++] = e;
        } else {
            out[o++] = L[li++];
        }
    }
    col_start[cj] = (int64_t)pos;
    col_len[cj] = o;
    return 0;
}

// The inputs every advance reads.
template <typename T, bool B> struct LzArgs {
    const T *values;
    Geo<B> geo;
    uint8_t *flags;
    GradRec *grad;
    const int32_t *vrank;
    const CritRec *recs;
    const int32_t *base1;
    const uint8_t *is_row;
    const int32_t *v2;
    const uint8_t *l2;
    const int32_t *colmap;
    HeapEnt *heap_all;
    HashEnt *hash_all;
    int32_t *tgen;
    int hcap, hashcap;
};

template <typename T, bool B>
__device__ __forceinline__ LazyCtx lz_ctx(const LzArgs<T, B> &a, int64_t slot) {
    LazyCtx c;
    c.heap = a.heap_all + slot * a.hcap;
    c.hash = a.hash_all + slot * a.hashcap;
    c.hcap = a.hcap;
    c.hashmask = a.hashcap - 1;
    c.hn = 0; c.used = 0; c.gen = 0; c.overflow = false;
    return c;
}

// Advances the listed columns (one thread each) whose top is regular or that
// have no list yet.  A column that outgrows the scratch, or finds the pool
// full, is left as it was and queued on `retry`.
template <typename T, bool B>
__global__ void __launch_bounds__(128)
    k_lz_advance(LzArgs<T, B> a, const int32_t *__restrict__ todo, int64_t ntodo, int32_t *astamp,
                 int32_t launch, Ent *pool, int64_t pool_cap, int64_t *col_start,
                 int32_t *col_len, int32_t *retry, DevStatus *st) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    LazyCtx c = lz_ctx(a, tid);
    int32_t gen = a.tgen[tid];
    for (int64_t q = tid; q < ntodo; q += nth) {
        const int32_t cj = todo[q];
        const int la = col_len[cj];
        const int64_t sa = col_start[cj];
        if (la == 0) continue;                                   // zero column
        if (la > 0 && (pool[sa].lo & 1)) continue;               // critical top
        if (atomicExch(&astamp[cj], launch) == launch) continue; // listed twice
        c.gen = ++gen;
        const GridParams &g = a.geo.at(a.v2[a.colmap[cj]]);
        const int r = lz_advance_col<T>(c, g_star, a.values, g, a.flags, a.grad, a.vrank,
                                        a.recs, a.base1, a.is_row, a.v2, a.l2, a.colmap, cj, la,
                                        sa, pool, pool_cap, col_start, col_len, st);
        if (r) retry[atomicAdd((unsigned long long *)&st->misc[3], 1ull)] = cj;
    }
    a.tgen[tid] = gen;
}

// ---- whole-column expansion by a block (columns with a large wall)
//
// A column whose advance outgrows the per-thread scratch usually sits on a
// large descending wall, and a serial walk through it is long.  Here a block
// expands such a column completely, in parallel, in two passes over the DAG
// of the gradient flow restricted to the column (an edge -> the two edges its
// expansion yields; acyclic since priorities strictly decrease):
//   1. discovery, level by level from the column's entries: each new regular
//      edge is expanded once, its products are inserted into a hash (one
//      slot per edge) and their in-degrees counted;
//   2. Kahn's order: an edge whose predecessors are all done adds its parity
//      (mod 2) into its products; the multiplicity of a critical row is
//      final when its in-degree is exhausted.
// The column becomes the sorted list of its critical rows of odd
// multiplicity: its Morse boundary, the limit of the advances.  A column
// that does not fit the block's hash or lists is left unchanged and retried
// by the serial advance in global memory.
// Per block: a hash of the column's edges in three arrays (keys, states,
// data), cleared before each column.
struct BxData {
    unsigned long long hi, lo;   // the edge's entry
    int32_t p0, p1;              // product slots (-1: none)
    int32_t spec;                // products of a regular edge: other star edge of its
                                 // triangle | link of the higher triangle vertex << 4 |
                                 // edge there << 8 (bit 12: invalid)
    int32_t pad;
};
// state: bits 0-7 count the parity-1 contributions (mod 2 is the
// multiplicity), bits 8-15 the in-edges not yet done
constexpr uint32_t kBxIn = 256;
constexpr int kBxThreads = 256;
// block scratch sizes: hash slots (log2), frontier capacity, sink capacity,
// blocks in flight
struct BxLevel {
    int hbits, fcap, scap, blocks;
};
constexpr BxLevel kBxLevels[2] = {{17, 65536, 16384, 152}, {21, 1 << 20, 1 << 16, 16}};
constexpr size_t kBxSlotBytes = 8 + 4 + sizeof(BxData);

struct BxCtx {
    unsigned long long *keys;
    uint32_t *state;
    BxData *data;
    uint32_t hmask;
    int32_t *next;        // frontier being filled
    int *nnext, fcap;
    int32_t *sink;        // slots of critical rows
    int *nsink, scap;
    int *used, *fail;
};

// Inserts edge (y, m) (dropping heads of vertex->edge vectors and critical
// edges paired in D0) or finds it; returns its slot or -1.  `initial`: an
// entry of the column (parity 1, not counted as an in-edge); otherwise a
// product (one more in-edge).  A new regular edge joins the next frontier
// with its two products precomputed; a new critical row joins the sinks.
// The vertex's flag, value and gradient record are loaded together up front.
template <typename T>
__device__ __noinline__ int32_t bx_insert(BxCtx &c, const StarTables &S, const GridParams &g,
                                          const T *__restrict__ values, uint8_t *flags,
                                          GradRec *grad, const int32_t *__restrict__ vrank,
                                          const CritRec *__restrict__ recs,
                                          const int32_t *__restrict__ base1,
                                          const uint8_t *__restrict__ is_row, int64_t y, int m,
                                          bool initial, DevStatus *st) {
    if (m < 0 || m >= kLinks) { atomicOr(&st->err, kErrState); *c.fail = 1; return -1; }
    const uint8_t fy = ((volatile const uint8_t *)flags)[y];
    const T vy = values[y];
    GradRec G;
    {
        const ulonglong2 *src = (const ulonglong2 *)&grad[y];
        for (int k = 0; k < 3; k++) {
            const ulonglong2 v = __ldcg(src + k);
            G.w[2 * k] = v.x;
            G.w[2 * k + 1] = v.y;
        }
    }
    if ((fy & 0xF) == m) return -1;
    bool crit = false;
    if (fy & kFlagCritical) {
        const int32_t i = vrank[y];
        const CritRec rec = recs[i];
        if (rec.crit_e >> m & 1) {
            if (!is_row[base1[i] + local_index(S, rec, 1, m)]) return -1;
            crit = true;
        }
    }
    const unsigned long long key = lz_key(y, m);
    uint32_t pos = hash64(key) & c.hmask;
    int32_t slot = -1;
    bool fresh = false;
    for (uint32_t p = 0; p <= c.hmask; p++, pos = (pos + 1) & c.hmask) {
        const unsigned long long prev = atomicCAS(&c.keys[pos], 0ull, key);
        if (prev == 0ull) { slot = (int32_t)pos; fresh = true; break; }
        if (prev == key) { slot = (int32_t)pos; break; }
    }
    if (slot < 0) { *c.fail = 1; return -1; }
    if (fresh) {
        if (atomicAdd(c.used, 1) * 4 >= (int)(c.hmask + 1) * 3) *c.fail = 1;
        if (!(fy & kFlagGradient)) G = grad_fill(S, g, values, flags, grad, y);
        int pair = 0, spec = 0;
        if (!crit) {
            pair = grad_edge_pair(G, m);
            if (pair >= kTris) {                 // not a valid pairing: never expanded
                atomicOr(&st->err, kErrState);
                *c.fail = 1;
                crit = true;
                pair = 0;
            } else {
                const int ta = S.tri_v[pair][0], tb = S.tri_v[pair][1];
                const bool aup = grad_rank(G, ta) > grad_rank(G, tb);
                const int hi = aup ? ta : tb, lo = aup ? tb : ta;
                const int l = S.link_of_dc[(S.dx[lo] - S.dx[hi] + 1) +
                                           3 * (S.dy[lo] - S.dy[hi] + 1) +
                                           9 * (S.dz[lo] - S.dz[hi] + 1)];
                spec = (ta == m ? tb : ta) | (hi << 4) | ((l & 15) << 8) | (l < 0 ? 1 << 12 : 0);
            }
        }
        BxData &d = c.data[slot];
        d.hi = (unsigned long long)Key<T>::of(vy);
        d.lo = ((unsigned long long)y << 15) | ((unsigned long long)grad_edge_order(G, m) << 11) |
               ((unsigned long long)m << 7) | ((unsigned long long)(pair & 63) << 1) |
               (crit ? 1ull : 0ull);
        d.p0 = -1;
        d.p1 = -1;
        d.spec = spec;
        if (crit) {
            const int k = atomicAdd(c.nsink, 1);
            if (k < c.scap) c.sink[k] = slot; else *c.fail = 1;
        } else {
            const int k = atomicAdd(c.nnext, 1);
            if (k < c.fcap) c.next[k] = slot; else *c.fail = 1;
        }
    }
    atomicAdd(&c.state[slot], initial ? 1u : kBxIn);
    return slot;
}

// descending order of (hi, lo) for a power-of-two count, by the block
__device__ void bx_sort_desc(Ent *a, int n) {
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool desc = (i & k) == 0;
                    const Ent x = a[i], y = a[l];
                    if (desc ? ent_gt(y, x) : ent_gt(x, y)) { a[i] = y; a[l] = x; }
                }
            }
            __syncthreads();
        }
}

template <typename T, bool B>
__global__ void __launch_bounds__(kBxThreads)
    k_lz_expand_block(LzArgs<T, B> a, const int32_t *__restrict__ todo, int64_t ntodo,
                      int32_t *astamp, int32_t launch, Ent *pool, int64_t pool_cap,
                      int64_t *col_start, int32_t *col_len, int32_t *retry, char *hash_all,
                      int hbits, int32_t *list_all, int fcap, int32_t *sink_all, Ent *sort_all,
                      int scap, DevStatus *st) {
    // frontier counts rotate through three words so that a level needs one
    // barrier: level i reads cnt[i%3], fills cnt[(i+1)%3] and clears
    // cnt[(i+2)%3], which every thread finished reading before the last barrier
    __shared__ int s_cnt[3];
    __shared__ int s_take, s_nil, s_nsink, s_used, s_fail, s_nout;
    __shared__ long long s_pos;
    const StarTables &S = g_star;
    const int t = threadIdx.x;
    const size_t hn = (size_t)1 << hbits;
    BxCtx c;
    {
        char *h = hash_all + (size_t)blockIdx.x * hn * kBxSlotBytes;
        c.keys = (unsigned long long *)h;
        c.data = (BxData *)(h + hn * 8);
        c.state = (uint32_t *)(h + hn * (8 + sizeof(BxData)));
    }
    c.hmask = (uint32_t)hn - 1;
    int32_t *F[2];
    F[0] = list_all + (size_t)blockIdx.x * 3 * fcap;
    F[1] = F[0] + fcap;
    int32_t *IL = F[1] + fcap;
    c.sink = sink_all + (size_t)blockIdx.x * scap;
    Ent *SR = sort_all + (size_t)blockIdx.x * 2 * scap;
    c.fcap = fcap; c.nsink = &s_nsink; c.scap = scap;
    c.used = &s_used; c.fail = &s_fail;
    for (int64_t q = blockIdx.x; q < ntodo; q += gridDim.x) {
        const int32_t cj = todo[q];
        const int la = col_len[cj];
        const int64_t sa = col_start[cj];
        if (la == 0) continue;
        if (la > 0 && (pool[sa].lo & 1)) continue;
        if (t == 0) s_take = atomicExch(&astamp[cj], launch) != launch;
        __syncthreads();
        if (!s_take) continue;
        // clear the keys and states of the hash
        {
            uint4 *k4 = (uint4 *)c.keys;
            for (size_t i = t; i < hn / 2; i += kBxThreads) k4[i] = make_uint4(0, 0, 0, 0);
            uint4 *s4 = (uint4 *)c.state;
            for (size_t i = t; i < hn / 4; i += kBxThreads) s4[i] = make_uint4(0, 0, 0, 0);
        }
        const int64_t x = a.v2[a.colmap[cj]];
        const GridParams &g = a.geo.at(x);
        if (t == 0) {
            s_cnt[0] = 0; s_cnt[1] = 0; s_cnt[2] = 0;
            s_nsink = 0; s_used = 0; s_fail = 0; s_nil = 0;
        }
        __syncthreads();
        // the column's entries (parity 1 each), listed in IL; the regular ones
        // form the first frontier
        c.next = F[0];
        c.nnext = &s_cnt[0];
        if (la < 0) {
            if (t == 0) {
                const int s = a.l2[a.colmap[cj]];
                const int ta = S.tri_v[s][0], tb = S.tri_v[s][1];
                const GradRec Gx = grad_get(S, g, a.values, a.flags, a.grad, x);
                const bool aup = grad_rank(Gx, ta) > grad_rank(Gx, tb);
                const int hi = aup ? ta : tb, lo = aup ? tb : ta;
                const int l = S.link_of_dc[(S.dx[lo] - S.dx[hi] + 1) + 3 * (S.dy[lo] - S.dy[hi] + 1) +
                                           9 * (S.dz[lo] - S.dz[hi] + 1)];
                IL[0] = bx_insert<T>(c, S, g, a.values, a.flags, a.grad, a.vrank, a.recs, a.base1,
                                     a.is_row, x, ta, true, st);
                IL[1] = bx_insert<T>(c, S, g, a.values, a.flags, a.grad, a.vrank, a.recs, a.base1,
                                     a.is_row, x, tb, true, st);
                IL[2] = bx_insert<T>(c, S, g, a.values, a.flags, a.grad, a.vrank, a.recs, a.base1,
                                     a.is_row, x + g.dlin[hi], l, true, st);
                s_nil = 3;
            }
        } else if (la > fcap) {
            if (t == 0) s_fail = 1;
        } else {
            for (int k = t; k < la; k += kBxThreads) {
                const Ent e = pool[sa + k];
                IL[k] = bx_insert<T>(c, S, g, a.values, a.flags, a.grad, a.vrank, a.recs,
                                     a.base1, a.is_row, ent_y(e), ent_m(e), true, st);
            }
            if (t == 0) s_nil = la;
        }
        __syncthreads();
        // 1. discovery, level by level: expand each new regular edge once (a
        //    thread per product), counting the in-edges of the products
        int lv1 = 0;
        for (int lv = 0;; lv++) {
            const int ncur = s_cnt[lv % 3];
            lv1 = lv;
            if (ncur == 0 || s_fail) break;
            if (t == 0) s_cnt[(lv + 2) % 3] = 0;
            const int32_t *cur = F[lv & 1];
            c.next = F[(lv + 1) & 1];
            c.nnext = &s_cnt[(lv + 1) % 3];
            for (int k = t; k < 2 * ncur; k += kBxThreads) {
                const int32_t u = cur[k >> 1];
                BxData &du = c.data[u];
                const int64_t y = (int64_t)(du.lo >> 15);
                const int spec = du.spec;
                if (spec >> 12) { atomicOr(&st->err, kErrState); s_fail = 1; continue; }
                if (k & 1)
                    du.p1 = bx_insert<T>(c, S, g, a.values, a.flags, a.grad, a.vrank, a.recs,
                                         a.base1, a.is_row, y + g.dlin[(spec >> 4) & 15],
                                         (spec >> 8) & 15, false, st);
                else
                    du.p0 = bx_insert<T>(c, S, g, a.values, a.flags, a.grad, a.vrank, a.recs,
                                         a.base1, a.is_row, y, spec & 15, false, st);
            }
            __syncthreads();
        }
        if (s_fail) {
            if (t == 0) retry[atomicAdd((unsigned long long *)&st->misc[3], 1ull)] = cj;
            __syncthreads();
            continue;
        }
        // 2. Kahn's order from the entries without in-edges: an edge whose
        //    in-edges are all done adds its parity into its products (a thread
        //    per product)
        if (t == 0) { s_cnt[0] = 0; s_cnt[1] = 0; s_cnt[2] = 0; }
        __syncthreads();
        const int nil = s_nil;
        for (int k = t; k < nil; k += kBxThreads) {
            const int32_t u = IL[k];
            if (u >= 0 && (c.state[u] >> 8) == 0) F[0][atomicAdd(&s_cnt[0], 1)] = u;
        }
        __syncthreads();
        int lv2 = 0;
        for (int lv = 0;; lv++) {
            const int ncur = s_cnt[lv % 3];
            lv2 = lv;
            if (ncur == 0 || s_fail) break;
            if (t == 0) s_cnt[(lv + 2) % 3] = 0;
            const int32_t *cur = F[lv & 1];
            int32_t *nxt = F[(lv + 1) & 1];
            int *nn = &s_cnt[(lv + 1) % 3];
            for (int k = t; k < 2 * ncur; k += kBxThreads) {
                const int32_t u = cur[k >> 1];
                const BxData &du = c.data[u];
                if (du.lo & 1) continue;                      // a critical row: a sink
                const int32_t pr = (k & 1) ? du.p1 : du.p0;
                if (pr < 0) continue;
                const uint32_t par = c.state[u] & 1u;
                const uint32_t old = atomicAdd(&c.state[pr], par - kBxIn);
                if ((old >> 8) == 1) {
                    const int w = atomicAdd(nn, 1);
                    if (w < fcap) nxt[w] = pr; else s_fail = 1;
                }
            }
            __syncthreads();
        }
        if (s_fail) {
            if (t == 0) retry[atomicAdd((unsigned long long *)&st->misc[3], 1ull)] = cj;
            __syncthreads();
            continue;
        }
        if (t == 0) {
            atomicAdd((unsigned long long *)&st->bx[0], (unsigned long long)s_used);
            atomicAdd((unsigned long long *)&st->bx[1], (unsigned long long)lv1);
            atomicAdd((unsigned long long *)&st->bx[2], (unsigned long long)lv2);
            atomicAdd((unsigned long long *)&st->bx[3], 1ull);
            s_nout = 0;
        }
        __syncthreads();
        // the critical rows of odd multiplicity, sorted by decreasing priority
        const int ns = s_nsink;
        for (int k = t; k < ns; k += kBxThreads) {
            const int32_t sk = c.sink[k];
            if (c.state[sk] & 1u) SR[atomicAdd(&s_nout, 1)] = Ent{c.data[sk].hi, c.data[sk].lo};
        }
        __syncthreads();
        const int nout = s_nout;
        int np2 = 1;
        while (np2 < nout) np2 <<= 1;
        for (int k = nout + t; k < np2; k += kBxThreads) SR[k] = Ent{0, 0};
        __syncthreads();
        if (nout > 1) bx_sort_desc(SR, np2);
        if (nout == 0) {
            if (t == 0) { col_start[cj] = 0; col_len[cj] = 0; }
            __syncthreads();
            continue;
        }
        if (t == 0) {
            const unsigned long long pos = atomicAdd(&st->pool_top, (unsigned long long)nout);
            if ((int64_t)(pos + nout) > pool_cap) {
                atomicOr(&st->err, kErrCap);
                retry[atomicAdd((unsigned long long *)&st->misc[3], 1ull)] = cj;
                s_take = -1;
            } else {
                s_take = 1;
                s_pos = (long long)pos;
                col_start[cj] = (int64_t)pos;
                col_len[cj] = nout;
            }
        }
        __syncthreads();
        if (s_take == 1)
            for (int k = t; k < nout; k += kBxThreads) pool[s_pos + k] = SR[k];
        __syncthreads();
    }
}

// Listed columns with a critical top claim it (atomic minimum of the column
// index); a claim that displaces a later owner queues it on `recheck`.
__global__ void k_lz_claim(const int32_t *__restrict__ active, int64_t nactive,
                           const int64_t *__restrict__ start, const int32_t *__restrict__ len,
                           const Ent *__restrict__ pool, const int32_t *__restrict__ vrank,
                           const CritRec *__restrict__ recs, const int32_t *__restrict__ base1,
                           int32_t *owner, int32_t *recheck, DevStatus *st) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool take = false;
    int32_t old = 0;
    if (q < nactive) {
        const int32_t cj = active[q];
        if (len[cj] > 0) {
            const Ent top = pool[start[cj]];
            if (ent_crit(top)) {
                const int32_t row =
                    crit_edge_row(g_star, vrank, recs, base1, ent_y(top), ent_m(top));
                old = atomicMin(&owner[row], cj);
                take = old != kNoOwner && old > cj;
            }
        }
    }
    warp_append(take, old, recheck, (unsigned long long *)&st->misc[0]);
}

// Merge path split of two decreasing entry lists (ties: A first; an equal
// pair never straddles the split).
__device__ __forceinline__ void ent_split(const Ent *A, int la, const Ent *B, int lb, int d,
                                          int &i, int &j) {
    int lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (!ent_gt(B[d - 1 - mid], A[mid])) lo = mid + 1;
        else hi = mid;
    }
    i = lo;
    j = d - lo;
    if (i > 0 && j < lb && ent_eq(A[i - 1], B[j])) j++;
}

// out = A + B (mod 2) for decreasing entry lists, by one warp; returns the length
__device__ int ent_warp_symdiff(const Ent *A, int la, const Ent *B, int lb, Ent *out) {
    const int lane = threadIdx.x & 31;
    const int L = la + lb, per = (L + 31) >> 5;
    int i0, j0, i1, j1;
    ent_split(A, la, B, lb, min(lane * per, L), i0, j0);
    ent_split(A, la, B, lb, min(lane * per + per, L), i1, j1);
    int cnt = 0;
    {
        int i = i0, j = j0;
        while (i < i1 || j < j1) {
            if (j >= j1 || (i < i1 && ent_gt(A[i], B[j]))) { cnt++; i++; }
            else if (i >= i1 || ent_gt(B[j], A[i])) { cnt++; j++; }
            else { i++; j++; }
        }
    }
    int inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    int o = inc - cnt;
    int i = i0, j = j0;
    while (i < i1 || j < j1) {
        if (j >= j1 || (i < i1 && ent_gt(A[i], B[j]))) out[o++] = A[i++];
        else if (i >= i1 || ent_gt(B[j], A[i])) out[o++] = B[j++];
        else { i++; j++; }                         // the same edge twice: 1 + 1 = 0
    }
    return total;
}

// One warp per listed column: while its top is a critical row owned by an
// earlier (stable) column, add that column's list; when an addition leaves a
// regular top, lane 0 advances the column in place (with the warp's slot of
// the scratch) and the additions go on, so a column's whole chain runs in one
// round.  A changed column is listed for the next round (for its claim, or
// for an advance with larger scratch when the inline one did not fit).
template <typename T, bool B>
__global__ void k_lz_add(LzArgs<T, B> a, const int32_t *__restrict__ active, int64_t nactive,
                         const int32_t *__restrict__ recheck, int64_t *start, int32_t *len,
                         Ent *pool, const int32_t *__restrict__ owner, int32_t *stamp,
                         int32_t round, int32_t *next, int64_t pool_cap, DevStatus *st) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nre = *(volatile long long *)&st->misc[0];
    LazyCtx c = lz_ctx(a, warp);
    int32_t gen = lane == 0 ? a.tgen[warp] : 0;
    unsigned adds = 0;
    unsigned long long io_r = 0, io_w = 0;
    for (int64_t q = warp; q < nactive + nre; q += nwarps) {
        const int32_t cj = q < nactive ? active[q] : recheck[q - nactive];
        int fresh = 0;
        if (lane == 0) fresh = atomicExch(&stamp[cj], round) != round;
        if (!__shfl_sync(0xffffffffu, fresh, 0)) continue;
        int la = len[cj];
        int64_t sa = start[cj];
        bool changed = false;
        for (int it = 0; la > 0 && it < (1 << 24); it++) {
            const Ent top = pool[sa];
            if (!ent_crit(top)) {
                if (!changed) break;     // not advanced yet: the next round's advance
                int r = 0, la2 = 0;
                long long sa2 = 0;
                if (lane == 0) {
                    c.gen = ++gen;
                    const GridParams &g = a.geo.at(a.v2[a.colmap[cj]]);
                    r = lz_advance_col<T>(c, g_star, a.values, g, a.flags, a.grad, a.vrank,
                                          a.recs, a.base1, a.is_row, a.v2, a.l2, a.colmap, cj,
                                          la, sa, pool, pool_cap, start, len, st);
                    if (r == 0) { la2 = len[cj]; sa2 = start[cj]; }
                }
                r = __shfl_sync(0xffffffffu, r, 0);
                if (r) break;
                la = __shfl_sync(0xffffffffu, la2, 0);
                sa = __shfl_sync(0xffffffffu, sa2, 0);
                continue;
            }
            const int32_t row = crit_edge_row(g_star, a.vrank, a.recs, a.base1, ent_y(top),
                                              ent_m(top));
            const int32_t k = owner[row];
            if (k == cj || k == kNoOwner || k > cj) break;
            const int64_t sb = start[k];
            const int lb = len[k];
            unsigned long long pos = 0;
            if (lane == 0) pos = atomicAdd(&st->pool_top, (unsigned long long)(la + lb));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if ((int64_t)(pos + la + lb) > pool_cap) {
                if (lane == 0) atomicOr(&st->err, kErrCap);
                break;
            }
            io_r += (unsigned long long)(la + lb);
            la = ent_warp_symdiff(pool + sa, la, pool + sb, lb, pool + pos);
            io_w += (unsigned long long)la;
            sa = (int64_t)pos;
            changed = true;
            adds++;
        }
        if (changed && lane == 0) {
            start[cj] = sa;
            len[cj] = la;
            if (la > 0) next[atomicAdd((unsigned long long *)&st->misc[1], 1ull)] = cj;
        }
    }
    if (lane == 0) {
        a.tgen[warp] = gen;
        if (adds) {
            atomicAdd((unsigned long long *)&st->misc[2], (unsigned long long)adds);
            atomicAdd((unsigned long long *)&st->red_io[0], io_r * sizeof(Ent));
            atomicAdd((unsigned long long *)&st->red_io[1], io_w * sizeof(Ent));
        }
    }
}

// per-column D1 partner (the owned top row) once no column changes
__global__ void k_lz_result(int64_t ncols, const int64_t *__restrict__ start,
                            const int32_t *__restrict__ len, const Ent *__restrict__ pool,
                            const int32_t *__restrict__ vrank, const CritRec *__restrict__ recs,
                            const int32_t *__restrict__ base1, int32_t *d1_row,
                            uint8_t *row_paired, DevStatus *st) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    if (len[c] <= 0) { if (len[c] < 0) atomicOr(&st->err, kErrState); d1_row[c] = -1; return; }
    const Ent top = pool[start[c]];
    if (!ent_crit(top)) { atomicOr(&st->err, kErrState); d1_row[c] = -1; return; }
    const int32_t r = crit_edge_row(g_star, vrank, recs, base1, ent_y(top), ent_m(top));
    d1_row[c] = r;
    row_paired[r] = 1;
}

// live lengths (a column not yet listed, len < 0, holds nothing)
__global__ void k_lz_live(int64_t ncol, const int32_t *__restrict__ len, int32_t *out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncol) out[c] = len[c] > 0 ? len[c] : 0;
}

// copies the live entry lists into a fresh pool (after the pool filled up)
__global__ void k_lz_compact(int64_t ncol, int64_t *start, const int32_t *__restrict__ len,
                             const int32_t *__restrict__ off, const Ent *__restrict__ src,
                             Ent *dst) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncol || len[c] <= 0) return;
    const int64_t s0 = start[c];
    const int32_t o = off[c];
    for (int k = 0; k < len[c]; k++) dst[o + k] = src[s0 + k];
    start[c] = o;
}


// ------------------------------------------------------ stage 8: output

__device__ __forceinline__ uint64_t key_to_bits32(uint32_t k) {   // f32 keys
    return (k & 0x80000000u) ? (uint64_t)(k ^ 0x80000000u) : (uint64_t)(~k);
}

template <typename T> __device__ __forceinline__ uint64_t fmax_bits(unsigned long long key);
template <> __device__ __forceinline__ uint64_t fmax_bits<uint16_t>(unsigned long long key) {
    return key;
}
template <> __device__ __forceinline__ uint64_t fmax_bits<float>(unsigned long long key) {
    return key_to_bits32((uint32_t)key) & 0xffffffffull;
}
template <> __device__ __forceinline__ uint64_t fmax_bits<double>(unsigned long long key) {
    return (key & 0x8000000000000000ull) ? (key ^ 0x8000000000000000ull) : ~key;
}

struct OutArgs {
    const int32_t *vc;
    const int32_t *v0;
    const int32_t *v1; const uint8_t *l1;
    const int32_t *v2; const uint8_t *l2;
    const int32_t *v3; const uint8_t *l3;
    const int32_t *young0, *young2;
    const uint8_t *died0, *died3;
    const int32_t *colmap;
    const int32_t *d1_row;          // per column: paired row (C1 index) or -1
    const uint8_t *row_paired;      // per C1 index: paired in D1
    const uint8_t *is_row, *is_col;
};

// flag kernels for the ordered output: one per (dimension, kind)
__global__ void k_flag(int kind, OutArgs a, int64_t n, int32_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int f = 0;
    switch (kind) {
        case 0: f = a.young0[i] >= 0; break;                          // D0 finite (C1)
        case 2: f = a.d1_row[i] >= 0; break;                          // D1 finite (cols)
        case 3: f = a.is_row[i] && !a.row_paired[i]; break;           // D1 infinite (C1)
        case 4: f = a.young2[i] >= 0; break;                          // D2 finite (C2)
        case 5: f = a.d1_row[i] < 0; break;                           // D2 infinite (cols)
        case 6: f = !a.died3[i]; break;                               // D3 infinite (C3)
    }
    flag[i] = f;
}

// D0 infinite: minima never killed (D0 nodes are the minima's indices in C0).
__global__ void k_flag_min(int64_t n0, const uint8_t *died0, int32_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n0) flag[i] = !died0[i];
}

// In a batch the ids are written relative to the pair's field (a simplex id
// of dimension d is a multiple of the field offset: 1, 7, 12, 6 ids per
// vertex), the field index goes to `ofield`, and an infinite class dies at
// the maximum of its own field.
template <typename T, bool B>
__global__ void k_write(int kind, OutArgs a, const T *__restrict__ values, Geo<B> geo,
                        int64_t n, const int32_t *__restrict__ flag,
                        const int32_t *__restrict__ pos, int64_t offset, const int32_t *vrank,
                        unsigned long long fmax_key,
                        const unsigned long long *__restrict__ fmax_field, int32_t *ofield,
                        dms_pair *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    const StarTables &S = g_star;
    dms_pair p;
    memset(&p, 0, sizeof p);
    int64_t bs = -1, ds = -1, bv = -1, dv = -1;
    int dim = 0, ess = 0;
    switch (kind) {
        case 0: {   // D0: (minimum, critical edge)
            bv = a.v0[a.young0[i]]; bs = bv;
            dv = a.v1[i]; ds = edge_id(S, geo.at(dv), dv, a.l1[i]);
            dim = 0; break;
        }
        case 1: {   // D0 infinite
            bv = a.v0[i]; bs = bv; dim = 0; ess = 1; break;
        }
        case 2: {   // D1: (critical edge = pivot row, critical triangle)
            int32_t row = a.d1_row[i];
            bv = a.v1[row]; bs = edge_id(S, geo.at(bv), bv, a.l1[row]);
            int32_t j2 = a.colmap[i];
            dv = a.v2[j2]; ds = tri_id(S, geo.at(dv), dv, a.l2[j2]);
            dim = 1; break;
        }
        case 3: {
            bv = a.v1[i]; bs = edge_id(S, geo.at(bv), bv, a.l1[i]); dim = 1; ess = 1; break;
        }
        case 4: {   // D2: (critical triangle, critical tet)
            bv = a.v2[i]; bs = tri_id(S, geo.at(bv), bv, a.l2[i]);
            int32_t t = a.young2[i];
            dv = a.v3[t]; ds = tet_id(S, geo.at(dv), dv, a.l3[t]);
            dim = 2; break;
        }
        case 5: {
            int32_t j2 = a.colmap[i];
            bv = a.v2[j2]; bs = tri_id(S, geo.at(bv), bv, a.l2[j2]); dim = 2; ess = 1; break;
        }
        case 6: {
            bv = a.v3[i]; bs = tet_id(S, geo.at(bv), bv, a.l3[i]); dim = 3; ess = 1; break;
        }
    }
    p.birth_bits = Key<T>::bits(values[bv]);
    unsigned long long fkey = fmax_key;
    if constexpr (B) {
        const int f = geo.field(bv);
        const int64_t off = geo.fields[f].off;
        const int64_t per[4] = {1, 7, 12, 6};
        bs -= per[dim] * off;
        if (ds >= 0) ds -= per[dim + 1 > 3 ? 3 : dim + 1] * off;
        fkey = fmax_field[f];
        p.death_bits = dv >= 0 ? Key<T>::bits(values[dv]) : fmax_bits<T>(fkey);
        bv -= off;
        if (dv >= 0) dv -= off;
        ofield[offset + pos[i]] = f;
    } else {
        p.death_bits = dv >= 0 ? Key<T>::bits(values[dv]) : fmax_bits<T>(fkey);
    }
    p.birth_simplex = bs; p.death_simplex = ds; p.birth_vertex = bv; p.death_vertex = dv;
    p.dim = (uint8_t)dim; p.essential = (uint8_t)ess;
    out[offset + pos[i]] = p;
}

// ------------------------------------------------------ small helper kernels

__global__ void k_unpaired(const int32_t *young, int64_t n, uint8_t *flag, int32_t *flag32) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { uint8_t f = young[i] < 0; flag[i] = f; if (flag32) flag32[i] = f; }
}
__global__ void k_u8_to_i32(const uint8_t *in, int64_t n, int32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}
__global__ void k_compact_idx(const uint8_t *flag, const int32_t *pos, int64_t n, int32_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = (int32_t)i;
}
// flag32[k] = flag[list[k]] (list null: flag[k])
__global__ void k_flags_of(const int32_t *list, int64_t m, const uint8_t *flag, int32_t *flag32) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) flag32[k] = flag[list ? list[k] : k];
}
// out[pos[k]] = list[k] (list null: k) for the flagged entries
__global__ void k_compact_list(const int32_t *list, const int32_t *flag32, const int32_t *pos,
                               int64_t m, int32_t *out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m && flag32[k]) out[pos[k]] = list ? list[k] : (int32_t)k;
}

// The word of each critical vertex that the D1 trace reads beside its flags
// and record: bits 0-31 the C1 index of its first critical edge, bits 32-45
// its critical edges (star links), bits 48-61 those that are rows (1-saddles
// not paired in D0).  One load in place of the chain vrank -> record ->
// base -> row flag.
__global__ void k_row_words(const int32_t *__restrict__ vc, int64_t nc,
                            const CritRec *__restrict__ recs, const int32_t *__restrict__ base1,
                            const uint8_t *__restrict__ is_row, unsigned long long *vcrit) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const StarTables &S = g_star;
    const CritRec rec = recs[i];
    const int32_t b1 = base1[i];
    uint32_t rows = 0;
    for (uint16_t m = rec.crit_e; m; m &= m - 1) {
        const int n = __ffs(m) - 1;
        if (is_row[b1 + local_index(S, rec, 1, n)]) rows |= 1u << n;
    }
    vcrit[vc[i]] = (unsigned long long)(uint32_t)b1 | ((unsigned long long)rec.crit_e << 32) |
                   ((unsigned long long)rows << 48);
}

// ------------------------------------------------ backward (differentiation)
//
// For a loss of the diagram, the value of a pair is the value of its maximum
// vertices (Sec. 2.4: persistence = f(max vertex of the death simplex) -
// f(max vertex of the birth simplex)), so d loss / d f(v) collects the
// gradients of the births and deaths whose maximum vertex is v.  FP64
// atomics accumulate them (a vertex is the maximum vertex of a few pairs at
// most); the caller casts.
// In a batch (pofs non-null) pair i belongs to the field f with
// pofs[f] <= i < pofs[f+1], and its vertex ids are relative to vofs[f].
__global__ void k_scatter_pair_grads(const dms_pair *__restrict__ pairs, int64_t n,
                                     const double *__restrict__ gbirth,
                                     const double *__restrict__ gdeath, double *grad,
                                     const int64_t *__restrict__ pofs,
                                     const int64_t *__restrict__ vofs, int nf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dms_pair p = pairs[i];
    int64_t base = 0;
    if (pofs) {
        int lo = 0, hi = nf - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pofs[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        base = vofs[lo];
    }
    if (gbirth && gbirth[i] != 0.0) atomicAdd(&grad[base + p.birth_vertex], gbirth[i]);
    if (gdeath && !p.essential && gdeath[i] != 0.0)
        atomicAdd(&grad[base + p.death_vertex], gdeath[i]);
}

// ------------------------------------------------------------- host side

bool DevBuf::ensure(size_t need) {
    if (need <= bytes && p) return true;
    if (p) { cudaFree(p); p = nullptr; bytes = 0; }
    size_t b = need < 256 ? 256 : need;
    if (cudaMalloc(&p, b) != cudaSuccess) { p = nullptr; cudaGetLastError(); return false; }
    bytes = b;
    return true;
}
void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Grids up to this many vertices get every gradient record computed densely
// (cheap at this size; the D1 walls of smooth fields then never wait on a
// single-threaded lazy ProcessLowerStars).
constexpr int64_t kDenseGradientBelow = (int64_t)1 << 25;

// The smallest power of two holding `heap` entries at most 3/4 full.
inline int hash_cap_for(int heap) {
    int h = 16;
    while (h * 3 < heap * 4) h *= 2;
    return h;
}

// Host-side NVTX ranges named after the stages ("dms/gradient", ..., one at
// a time), so that a profiler can pick out one stage's kernels, e.g.
// ncu --nvtx --nvtx-include "dms/d1/".  With no tool attached the calls do
// nothing.
struct StageRanges {
    bool open = false;
    void next(const char *name) {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~StageRanges() {
        if (open) nvtxRangePop();
    }
};

// Most PL-critical vertices of one compute: 12 critical cells at most per
// lower star must keep every critical-simplex index below 2^31.
constexpr int64_t kMaxCriticalVertices = (((int64_t)1 << 31) - 1) / 12;

// Tiling of the tier-1 stencil: R whole rows per block, at least 2048
// vertices per tile.
struct ClsTiling {
    int rows_per_block, runs_per_row, aligned;
    int64_t tile, ntiles;
};
template <typename T> ClsTiling cls_tiling(const GridParams &g, const void *values) {
    constexpr int K = VecOf<T>::K;
    ClsTiling t;
    t.runs_per_row = (g.nx + K - 1) / K;
    t.rows_per_block = std::max(1, (2048 + g.nx - 1) / g.nx);
    t.tile = (int64_t)t.rows_per_block * g.nx;
    const int64_t rows = (int64_t)g.ny * g.nz;
    t.ntiles = (rows + t.rows_per_block - 1) / t.rows_per_block;
    t.aligned = ((uintptr_t)values % 16 == 0) && ((int64_t)g.nx * sizeof(T)) % 16 == 0;
    return t;
}

struct Ctx {
    Pipeline &P;
    cudaStream_t s;
    GridParams g;
    Geo<true> bgeo{};                        // a batch: per-field grids
    DevStatus *st;
    DevStatus *hst;
    cudaEvent_t *ev;    // stage boundaries
    cudaEvent_t *kev;   // kernel family start/end pairs
    int64_t launches = 0;
    StageRanges nv;     // NVTX range of the current stage
    DevBuf *scan_buf = nullptr;   // scan partials of this stream (null: P.scan_tmp)
};
#define KEV(i) cudaEventRecord(c.kev[i], c.s)

template <bool B> Geo<B> geo_of(const Ctx &c);
template <> Geo<false> geo_of<false>(const Ctx &c) {
    Geo<false> g;
    g.g0 = c.g;
    return g;
}
template <> Geo<true> geo_of<true>(const Ctx &c) { return c.bgeo; }

// Devices whose constant tables are uploaded, guarded by g_tables_mutex: handles are
// created from several host threads (one per serving slot), and the upload must
// happen once per device, before any kernel there reads the tables.
std::mutex g_tables_mutex;
std::vector<char> g_tables_ready;   // indexed by device id

#define DMS_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            fprintf(stderr, "libdms: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
            return DMS_ERR_CUDA;                                                       \
        }                                                                              \
    } while (0)
#define DMS_TRY(x)                      \
    do {                                \
        dms_status s_ = (x);            \
        if (s_ != DMS_OK) return s_;    \
    } while (0)
#define DMS_ALLOC(buf, nbytes)                               \
    do {                                                     \
        if (!(buf).ensure((size_t)(nbytes))) return DMS_ERR_OOM; \
    } while (0)
// launches a kernel over `count` items unless there are none
#define DMS_LAUNCH(count, threads, kernel, ...)                                          \
    do {                                                                                 \
        if ((count) > 0) {                                                               \
            kernel<<<blocks_for((count), (threads)), (threads), 0, c.s>>>(__VA_ARGS__);  \
            c.launches++;                                                                \
            cudaError_t e_ = cudaGetLastError();                                         \
            if (e_ != cudaSuccess) {                                                     \
                fprintf(stderr, "libdms: launch of %s failed: %s\n", #kernel,            \
                        cudaGetErrorString(e_));                                         \
                return DMS_ERR_CUDA;                                                     \
            }                                                                            \
        }                                                                                \
    } while (0)

dms_status ensure_tables(int device) {
    if (device < 0) return DMS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tables_mutex);
    if ((size_t)device < g_tables_ready.size() && g_tables_ready[device]) return DMS_OK;
    StarTables S;
    if (!build_star_tables(S)) return DMS_ERR_STATE;
    std::vector<uint32_t> lut;
    build_regular_lut(S, lut);
    DMS_CUDA(cudaMemcpyToSymbol(g_star, &S, sizeof S));
    DMS_CUDA(cudaMemcpyToSymbol(g_regular, lut.data(), lut.size() * sizeof(uint32_t)));
    DMS_CUDA(cudaFuncSetAttribute(k_red_async<kAsyncBlock, kAsyncAcc, kAsyncStage>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAsyncSmem));
    DMS_CUDA(cudaFuncSetAttribute(k_red_add_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kRedSmem));
    if ((size_t)device >= g_tables_ready.size()) g_tables_ready.resize(device + 1, 0);
    g_tables_ready[device] = 1;
    return DMS_OK;
}

// Exclusive scan of n int32 values into out; the total goes to *total.
dms_status scan(Ctx &c, const int32_t *in, int32_t *out, int64_t n, long long *total) {
    if (n == 0) {
        DMS_CUDA(cudaMemsetAsync(total, 0, sizeof(long long), c.s));
        return DMS_OK;
    }
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 1) {
        k_scan_apply<<<1, kScanThreads, 0, c.s>>>(in, out, n, nullptr, total);
        c.launches++;
        return cudaGetLastError() == cudaSuccess ? DMS_OK : DMS_ERR_CUDA;
    }
    std::vector<int64_t> sizes;   // partial counts per level, all > 1
    for (int64_t m = ntiles; m > 1; m = (m + kScanTile - 1) / kScanTile) sizes.push_back(m);
    size_t need = 0;
    for (int64_t m : sizes) need += 2 * (size_t)m;
    DevBuf &tmp = c.scan_buf ? *c.scan_buf : c.P.scan_tmp;
    if (!tmp.ensure(4 * need + 1024)) return DMS_ERR_OOM;
    int32_t *base = tmp.as<int32_t>();
    std::vector<const int32_t *> lin;
    std::vector<int32_t *> loff;
    const int32_t *cur = in;
    int64_t curn = n;
    size_t at = 0;
    for (int64_t m : sizes) {
        int32_t *part = base + at; at += m;
        int32_t *off = base + at; at += m;
        k_scan_partial<<<(unsigned)m, kScanThreads, 0, c.s>>>(cur, curn, part);
        c.launches++;
        lin.push_back(cur);
        loff.push_back(off);
        cur = part;
        curn = m;
    }
    k_scan_apply<<<1, kScanThreads, 0, c.s>>>(cur, loff.back(), curn, nullptr, nullptr);
    c.launches++;
    for (int lv = (int)sizes.size() - 1; lv >= 0; lv--) {
        int64_t lvn = lv == 0 ? n : sizes[lv - 1];
        int32_t *lvout = lv == 0 ? out : loff[lv - 1];
        k_scan_apply<<<(unsigned)sizes[lv], kScanThreads, 0, c.s>>>(lin[lv], lvout, lvn, loff[lv],
                                                                    lv == 0 ? total : nullptr);
        c.launches++;
    }
    return cudaGetLastError() == cudaSuccess ? DMS_OK : DMS_ERR_CUDA;
}

dms_status sync_status(Ctx &c) {
    DMS_CUDA(cudaMemcpyAsync(c.hst, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.s));
    DMS_CUDA(cudaStreamSynchronize(c.s));
    if (c.hst->err & kErrNan) return DMS_ERR_NAN;
    if (c.hst->err & kErrIter) return DMS_ERR_ITER_LIMIT;
    if (c.hst->err & kErrCap) return DMS_ERR_CAPACITY;
    if (c.hst->err & kErrState) return DMS_ERR_STATE;
    return DMS_OK;
}

// Elder-rule pairing of one arc graph over nodes 0..nnodes-1 (D0: the
// minima, increasing order, older = smaller node; D2: the maxima and the
// outside node, decreasing order, older = larger node).  The minimum
// spanning forest's arcs are found first (Borůvka); the halving levels then
// run over them alone.  Returns the number of halving levels.
dms_status elder_rule(Ctx &c, int32_t *A, int32_t *B, int64_t narcs, int64_t nnodes,
                      int descending, int older_is_larger, int32_t *young, uint8_t *died,
                      int64_t *levels_out) {
    Pipeline &P = c.P;
    *levels_out = 0;
    if (narcs == 0 || nnodes == 0) return DMS_OK;
    // ---- Borůvka: comp (nodes), best (nodes), tgt (nodes); the open arcs
    // (two lists), their flags and scan; the forest flag per arc
    DMS_ALLOC(P.bv_node, 12 * nnodes + 16);
    int32_t *comp = P.bv_node.as<int32_t>(), *tgt = comp + nnodes;
    uint32_t *best = (uint32_t *)(tgt + nnodes);
    DMS_ALLOC(P.dc_par, 8 * narcs + 8);
    DMS_ALLOC(P.dc_lab, 8 * narcs + 8);
    DMS_ALLOC(P.bv_msf, narcs + 8);
    int32_t *act = P.dc_par.as<int32_t>(), *act2 = act + narcs;
    int32_t *open = P.dc_lab.as<int32_t>(), *pos = open + narcs;
    uint8_t *msf = P.bv_msf.as<uint8_t>();
    DMS_LAUNCH(nnodes, 256, k_iota32, comp, nnodes);
    DMS_CUDA(cudaMemsetAsync(msf, 0, narcs, c.s));
    const int32_t *list = nullptr;      // all arcs in the first round
    int64_t nact = narcs;
    for (int round = 0; nact > 0; round++) {
        if (round > 64) return DMS_ERR_ITER_LIMIT;   // each round at least halves the roots
        DMS_CUDA(cudaMemsetAsync(best, 0xFF, 4 * nnodes, c.s));
        DMS_CUDA(cudaMemsetAsync(&c.st->misc[0], 0, sizeof(long long), c.s));
        DMS_LAUNCH(nact, 256, k_bv_best, list, nact, narcs, descending, A, B, comp, best, open);
        DMS_LAUNCH(nnodes, 256, k_bv_pick, nnodes, narcs, descending, A, B, comp, best, tgt, msf);
        DMS_LAUNCH(nnodes, 256, k_bv_hook, nnodes, tgt, comp,
                   (unsigned long long *)&c.st->misc[0]);
        DMS_LAUNCH(nnodes, 256, k_bv_jump, nnodes, comp, c.st);
        // the arcs still open at the round's start that may join components
        DMS_TRY(scan(c, open, pos, nact, &c.st->total[3]));
        DMS_TRY(sync_status(c));
        const int64_t nnext = c.hst->total[3];
        if (c.hst->misc[0] == 0) break;              // no component took an arc: done
        DMS_LAUNCH(nact, 256, k_compact_list, list, open, pos, nact, act2);
        std::swap(act, act2);
        list = act;
        nact = nnext;
    }
    // ---- the forest's arcs, in their order
    DMS_LAUNCH(narcs, 256, k_u8_to_i32, msf, narcs, open);
    DMS_TRY(scan(c, open, pos, narcs, &c.st->total[3]));
    DMS_TRY(sync_status(c));
    const int64_t m = c.hst->total[3];
    if (m == 0) return DMS_OK;
    DMS_ALLOC(P.bv_arcs, 12 * m + 16);
    int32_t *A2 = P.bv_arcs.as<int32_t>(), *B2 = A2 + m, *idx = B2 + m;
    DMS_LAUNCH(narcs, 256, k_bv_gather, narcs, msf, pos, A, B, A2, B2, idx);
    // ---- halving levels over the forest's arcs
    int L = 0;
    while (((int64_t)1 << L) < m) L++;
    // at most one key per light-arc endpoint per level: a table at most 2/3 full
    uint32_t cap = 1024;
    while ((int64_t)cap * 2 < 3 * m + 2) cap <<= 1;
    DMS_ALLOC(P.dc_keys, sizeof(DcSlot) * (size_t)cap);
    DcSlot *tab = P.dc_keys.as<DcSlot>();
    // cleared once: the keys of each level tell its slots from earlier levels
    DMS_CUDA(cudaMemsetAsync(tab, 0xFF, sizeof(DcSlot) * (size_t)cap, c.s));
    for (int shift = L; shift > kDcSegBits; shift--) {
        DMS_LAUNCH(m, 256, k_dc_insert, m, shift, descending, A2, B2, tab, cap - 1, c.st);
        DMS_LAUNCH(m, 256, k_dc_union, m, shift, descending, older_is_larger, A2, B2, tab,
                   cap - 1, c.st);
        DMS_LAUNCH(m, 256, k_dc_relabel, m, shift, descending, A2, B2, tab, cap - 1);
    }
    // levels kDcSegBits .. 1: each segment of 2^kDcSegBits turns in one warp
    k_dc_segment<<<(unsigned)((m + kDcSeg - 1) / kDcSeg), 32, 0, c.s>>>(
        m, descending, older_is_larger, A2, B2, c.st);
    c.launches++;
    DMS_CUDA(cudaGetLastError());
    DMS_LAUNCH(m, 256, k_dc_decide, m, older_is_larger, A2, B2, idx, young, died);
    *levels_out = L;
    return DMS_OK;
}

// Reduces a set of columns (entries sorted decreasingly, pivot first) stored
// in P.d1_pool at P.d1_start/P.d1_len, claiming pivots in owner[0..nent).
// Rounds continue until no column changes; on a pool overflow the live
// columns are compacted into a larger pool and the round is repeated.
// Initial capacity (entries) of the lazy D1 column pool: `dflt`, unless the
// environment sets DMS_D1_POOL_ENTRIES (a smaller pool exercises the
// compaction and regrowth path).
int64_t d1_pool_entries(int64_t dflt) {
    const char *e = getenv("DMS_D1_POOL_ENTRIES");
    if (!e) return dflt;
    const long long v = atoll(e);
    return v >= 64 ? (int64_t)v : dflt;
}


// Compacts the live columns (int32 entries) into a fresh pool at least twice
// as large (and 4x the live entries), clears the status error and resets the
// bump pointer.  The host status mirror keeps the other words of the last sync.
dms_status grow_pool(Ctx &c, int64_t ncol, int64_t *pool_cap) {
    Pipeline &P = c.P;
    DMS_ALLOC(P.flag_a, 4 * ncol + 4);
    DMS_ALLOC(P.flag_b, 4 * ncol + 4);
    DMS_CUDA(cudaMemcpyAsync(P.flag_a.p, P.d1_len.p, 4 * ncol, cudaMemcpyDeviceToDevice, c.s));
    DMS_TRY(scan(c, P.flag_a.as<int32_t>(), P.flag_b.as<int32_t>(), ncol, &c.st->total[3]));
    DMS_CUDA(cudaMemcpyAsync(c.hst, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.s));
    DMS_CUDA(cudaStreamSynchronize(c.s));
    const int64_t live = c.hst->total[3];
    const int64_t cap2 = std::max<int64_t>(2 * *pool_cap, 4 * live + (1 << 20));
    if (cap2 >= ((int64_t)1 << 31)) return DMS_ERR_CAPACITY;
    DevBuf fresh;
    if (!fresh.ensure(4 * (size_t)cap2)) return DMS_ERR_OOM;
    DMS_LAUNCH(ncol, 256, k_pool_compact, ncol, P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(),
               P.flag_b.as<int32_t>(), P.d1_pool.as<int32_t>(), fresh.as<int32_t>());
    DMS_CUDA(cudaStreamSynchronize(c.s));
    P.d1_pool.release();
    P.d1_pool = fresh;
    *pool_cap = cap2;
    c.hst->err = 0;
    c.hst->pool_top = (unsigned long long)live;
    DMS_CUDA(cudaMemcpyAsync(c.st, c.hst, sizeof(DevStatus), cudaMemcpyHostToDevice, c.s));
    P.d1_pool_grows++;
    return DMS_OK;
}

// The tail of the reduction in one asynchronous pass (k_red_async) over the
// `nactive` columns listed in P.d1_act.  Returns DMS_OK when every column is
// reduced, or DMS_ERR_CAPACITY with the unfinished columns back in P.d1_act
// (*nactive) when the pool filled up.
dms_status reduce_tail_async(Ctx &c, int64_t ncol, int64_t *nactive, int64_t pool_cap) {
    Pipeline &P = c.P;
    const int64_t n0 = *nactive;
    const int64_t qcap = std::max<int64_t>(4 * ncol, n0 + (1 << 20));
    if (qcap >= ((int64_t)1 << 31)) return DMS_ERR_CAPACITY;
    DMS_ALLOC(P.d1_info, 8 * ncol + 8);
    DMS_ALLOC(P.d1_queue, 4 * qcap);
    DMS_ALLOC(P.d1_aq, sizeof(AsyncQ));
    DMS_LAUNCH(ncol, 256, k_pack_info, ncol, P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(),
               P.d1_info.as<unsigned long long>());
    DMS_CUDA(cudaMemsetAsync(P.d1_queue.p, 0xFF, 4 * qcap, c.s));
    DMS_CUDA(cudaMemcpyAsync(P.d1_queue.p, P.d1_act.p, 4 * n0, cudaMemcpyDeviceToDevice, c.s));
    AsyncQ q0{0u, (unsigned int)n0, (int)n0, 0};
    DMS_CUDA(cudaMemcpyAsync(P.d1_aq.p, &q0, sizeof q0, cudaMemcpyHostToDevice, c.s));
    // 2 blocks of 256 threads per SM, each holding up to 12 K-entry columns in
    // shared memory (larger ones merge through the pool)
    k_red_async<kAsyncBlock, kAsyncAcc, kAsyncStage><<<2 * 152, kAsyncBlock, kAsyncSmem, c.s>>>(
        P.d1_aq.as<AsyncQ>(), P.d1_queue.as<int32_t>(), (unsigned int)qcap,
        P.d1_owner.as<int32_t>(), P.d1_info.as<unsigned long long>(), P.d1_start.as<int64_t>(),
        P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(), pool_cap, c.st);
    c.launches++;
    DMS_CUDA(cudaGetLastError());
    AsyncQ q1;
    DMS_CUDA(cudaMemcpyAsync(&q1, P.d1_aq.p, sizeof q1, cudaMemcpyDeviceToHost, c.s));
    dms_status s = sync_status(c);
    if (s != DMS_OK && s != DMS_ERR_CAPACITY) return s;
    if (s == DMS_OK && !q1.abort && q1.pending == 0) return DMS_OK;
    if (s == DMS_OK) return DMS_ERR_STATE;
    // the pool filled up: the queued columns go back to the rounds
    const int64_t h = q1.head, tl = std::min<int64_t>(q1.tail, qcap);
    if (tl < h || tl - h > 4 * ncol) return DMS_ERR_STATE;
    DMS_CUDA(cudaMemcpyAsync(P.d1_act.p, P.d1_queue.as<int32_t>() + h, 4 * (tl - h),
                             cudaMemcpyDeviceToDevice, c.s));
    *nactive = tl - h;
    return DMS_ERR_CAPACITY;
}

dms_status reduce_columns(Ctx &c, int64_t ncol, int64_t nent, int64_t pool_used) {
    Pipeline &P = c.P;
    DMS_ALLOC(P.d1_owner, 4 * nent + 4);
    DMS_ALLOC(P.d1_rowcol, sizeof(RowCol) * (nent + 1));
    RowCol *rowcol = P.d1_rowcol.as<RowCol>();
    DMS_ALLOC(P.d1_act, 4 * 3 * ncol + 4);
    DMS_ALLOC(P.d1_next, 4 * 3 * ncol + 4);
    DMS_ALLOC(P.d1_re, 4 * ncol + 4);
    DMS_ALLOC(P.d1_stamp, 4 * ncol + 4);
    DMS_ALLOC(P.d1_work, 4 * 2 * ncol + 4);
    DMS_CUDA(cudaMemsetAsync(P.d1_owner.p, 0x7F, 4 * nent + 4, c.s));
    DMS_CUDA(cudaMemsetAsync(rowcol, 0x7F, sizeof(RowCol) * (nent + 1), c.s));
    DMS_CUDA(cudaMemsetAsync(P.d1_stamp.p, 0xFF, 4 * ncol + 4, c.s));
    DMS_LAUNCH(ncol, 256, k_iota32, P.d1_act.as<int32_t>(), ncol);
    DMS_CUDA(cudaMemsetAsync(&c.st->misc[2], 0, 2 * sizeof(long long), c.s));
    c.hst->pool_top = (unsigned long long)pool_used;
    DMS_CUDA(cudaMemcpyAsync(&c.st->pool_top, &c.hst->pool_top, sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, c.s));
    int64_t pool_cap = (int64_t)(P.d1_pool.bytes / 4);
    int64_t nactive = ncol, stamp = 0;
    const int64_t limit = P.max_iters > 0 ? P.max_iters : ((int64_t)1 << 22);
    // rounds end below this many active columns (-1: the larger of 4096 and
    // one column in 1600; measured on GB300: 4096 best for 3.3 M columns at
    // 256^3, 16384 for 26 M at 512^3)
    const int64_t below = P.tune[DMS_TUNE_RED_BLOCK_BELOW] >= 0
                              ? (int64_t)P.tune[DMS_TUNE_RED_BLOCK_BELOW]
                              : std::max<int64_t>(4096, ncol / 1600);
    for (int64_t r = 0; r < limit; r++, stamp++) {
        if (nactive <= below && P.tune[DMS_TUNE_RED_ASYNC] && !P.generators) {
            // the tail: one asynchronous pass instead of rounds
            dms_status s = reduce_tail_async(c, ncol, &nactive, pool_cap);
            P.rounds_d1 = r + 1;
            if (s == DMS_OK) {
                P.d1_io_read = c.hst->red_io[0];
                P.d1_io_written = c.hst->red_io[1];
                P.d1_additions = c.hst->misc[2];
                P.d1_longest_chain = c.hst->misc[3];
                P.d1_pool_used = (int64_t)c.hst->pool_top;
                return DMS_OK;
            }
            if (s != DMS_ERR_CAPACITY) return s;
            // compact into a larger pool, publish the owners again, go on in rounds
            DMS_TRY(grow_pool(c, ncol, &pool_cap));
            DMS_LAUNCH(ncol, 256, k_red_publish_all, ncol, P.d1_start.as<int64_t>(),
                       P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(),
                       P.d1_owner.as<int32_t>(), rowcol);
            continue;
        }
        DMS_CUDA(cudaMemsetAsync(&c.st->misc[0], 0, 2 * sizeof(long long), c.s));
        DMS_LAUNCH(nactive, 256, k_red_claim, P.d1_act.as<int32_t>(), nactive,
                   P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(),
                   P.d1_owner.as<int32_t>(), P.d1_re.as<int32_t>(), c.st);
        DMS_LAUNCH(nactive, 256, k_red_publish, P.d1_act.as<int32_t>(), nactive,
                   P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(),
                   P.d1_owner.as<int32_t>(), rowcol);
        if (nactive > below) {
            // the columns that add something (displaced owners included: at
            // most one per claim), then a warp for each of them
            DMS_CUDA(cudaMemsetAsync(&c.st->red_work, 0, sizeof(unsigned long long), c.s));
            DMS_LAUNCH(2 * nactive, 256, k_red_need, P.d1_act.as<int32_t>(), nactive,
                       P.d1_re.as<int32_t>(), P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(),
                       P.d1_pool.as<int32_t>(), rowcol, P.d1_stamp.as<int32_t>(), (int32_t)stamp,
                       P.d1_work.as<int32_t>(), c.st);
            DMS_LAUNCH(std::min<int64_t>(64 * nactive, (int64_t)152 * 64 * 256), 256, k_red_add,
                       P.d1_work.as<int32_t>(), P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(),
                       P.d1_pool.as<int32_t>(), rowcol, P.d1_next.as<int32_t>(), pool_cap, c.st);
        } else {
            // one block per column (grid covers active + displaced, <= 2x active)
            k_red_add_block<<<(unsigned)(2 * nactive), kRedBlock, kRedSmem, c.s>>>(
                P.d1_act.as<int32_t>(), nactive, P.d1_re.as<int32_t>(), P.d1_start.as<int64_t>(),
                P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(), rowcol,
                P.d1_stamp.as<int32_t>(), (int32_t)stamp, P.d1_next.as<int32_t>(), pool_cap, c.st);
            c.launches++;
            DMS_CUDA(cudaGetLastError());
        }
        dms_status s = sync_status(c);
        P.rounds_d1 = r + 1;
        if (getenv("DMS_DEBUG")) {
            static std::chrono::steady_clock::time_point t_last;
            auto now = std::chrono::steady_clock::now();
            double ms = r ? std::chrono::duration<double, std::milli>(now - t_last).count() : 0.0;
            t_last = now;
            fprintf(stderr, "d1 round %lld: active %lld rechecked %lld next %lld adds %lld "
                    "max-chain %lld pool %llu (%.3f ms)\n", (long long)r, (long long)nactive,
                    c.hst->misc[0], c.hst->misc[1], c.hst->misc[2], c.hst->misc[3],
                    c.hst->pool_top, ms);
        }
        if (s == DMS_ERR_CAPACITY) {
            // compact the live columns into a pool twice as large, then sweep all columns
            DMS_TRY(grow_pool(c, ncol, &pool_cap));
            // the owners' lists moved: publish them again
            DMS_LAUNCH(ncol, 256, k_red_publish_all, ncol, P.d1_start.as<int64_t>(),
                       P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(),
                       P.d1_owner.as<int32_t>(), rowcol);
            // every column the interrupted round listed or changed is listed again
            const int64_t nre = c.hst->misc[0], nnext = c.hst->misc[1];
            DMS_CUDA(cudaMemcpyAsync(P.d1_act.as<int32_t>() + nactive, P.d1_re.p, 4 * nre,
                                     cudaMemcpyDeviceToDevice, c.s));
            DMS_CUDA(cudaMemcpyAsync(P.d1_act.as<int32_t>() + nactive + nre, P.d1_next.p,
                                     4 * nnext, cudaMemcpyDeviceToDevice, c.s));
            nactive += nre + nnext;
            continue;
        }
        if (s != DMS_OK) return s;
        nactive = c.hst->misc[1];
        std::swap(P.d1_act, P.d1_next);
        if (nactive == 0) {
            P.d1_io_read = c.hst->red_io[0];
            P.d1_io_written = c.hst->red_io[1];
            P.d1_additions = c.hst->misc[2];
            P.d1_longest_chain = c.hst->misc[3];
            P.d1_pool_used = (int64_t)c.hst->pool_top;
            return DMS_OK;
        }
    }
    return DMS_ERR_ITER_LIMIT;
}

// D1 from the traced columns: reduce them directly (homology) or reduce
// their anti-transpose (cohomology); both give the pairs of Alg. 3.
dms_status reduce_d1(Ctx &c, int64_t ncols, int64_t n1, const uint8_t *is_row) {
    Pipeline &P = c.P;
    DMS_CUDA(cudaMemcpyAsync(c.hst, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.s));
    DMS_CUDA(cudaStreamSynchronize(c.s));
    const int64_t traced = (int64_t)c.hst->pool_top;
    if (P.d1_mode_used == 1) {
        DMS_TRY(reduce_columns(c, ncols, n1, traced));
        DMS_LAUNCH(ncols, 256, k_d1_result_homology, ncols, P.d1_start.as<int64_t>(),
                   P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(), P.d1_row.as<int32_t>(),
                   P.d1_rowpaired.as<uint8_t>());
        return DMS_OK;
    }
    // rows: their positions among the rows (scan of the row flags)
    DMS_ALLOC(P.flag_a, 4 * (n1 + 4));
    DMS_ALLOC(P.d1_rowpos, 4 * (n1 + 4));
    DMS_LAUNCH(n1, 256, k_u8_to_i32, is_row, n1, P.flag_a.as<int32_t>());
    DMS_TRY(scan(c, P.flag_a.as<int32_t>(), P.d1_rowpos.as<int32_t>(), n1, &c.st->total[3]));
    DMS_CUDA(cudaMemcpyAsync(c.hst, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.s));
    DMS_CUDA(cudaStreamSynchronize(c.s));
    const int64_t nrows = c.hst->total[3];
    DMS_ALLOC(P.d1_rowmap, 4 * (nrows + 4));
    DMS_LAUNCH(n1, 256, k_compact_idx, is_row, P.d1_rowpos.as<int32_t>(), n1,
               P.d1_rowmap.as<int32_t>());
    // transpose: count, scan, scatter, sort
    DMS_ALLOC(P.d1_cocnt, 4 * (nrows + 4));
    DMS_ALLOC(P.d1_costart, 4 * (nrows + 4));
    DMS_ALLOC(P.d1_cofill, 4 * (nrows + 4));
    DMS_CUDA(cudaMemsetAsync(P.d1_cocnt.p, 0, 4 * (nrows + 4), c.s));
    DMS_CUDA(cudaMemsetAsync(P.d1_cofill.p, 0, 4 * (nrows + 4), c.s));
    DMS_LAUNCH(ncols, 256, k_co_count, ncols, P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(),
               P.d1_pool.as<int32_t>(), P.d1_rowpos.as<int32_t>(), nrows, P.d1_cocnt.as<int32_t>());
    DMS_TRY(scan(c, P.d1_cocnt.as<int32_t>(), P.d1_costart.as<int32_t>(), nrows, &c.st->total[3]));
    int64_t cap = std::max<int64_t>(1 << 22, 8 * traced + 1024);
    DevBuf copool;
    if (!copool.ensure(4 * (size_t)cap)) return DMS_ERR_OOM;
    DMS_LAUNCH(ncols, 256, k_co_scatter, ncols, P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(),
               P.d1_pool.as<int32_t>(), P.d1_rowpos.as<int32_t>(), nrows,
               P.d1_costart.as<int32_t>(), P.d1_cofill.as<int32_t>(), copool.as<int32_t>());
    // the cocolumns replace the columns in the reduction buffers
    DMS_CUDA(cudaStreamSynchronize(c.s));
    DMS_ALLOC(P.d1_start, 8 * (nrows + 4));
    DMS_ALLOC(P.d1_len, 4 * (nrows + 4));
    DMS_CUDA(cudaMemcpyAsync(P.d1_len.p, P.d1_cocnt.p, 4 * nrows, cudaMemcpyDeviceToDevice, c.s));
    DMS_LAUNCH(nrows, 128, k_co_sort, nrows, P.d1_costart.as<int32_t>(), P.d1_cocnt.as<int32_t>(),
               copool.as<int32_t>(), P.d1_start.as<int64_t>());
    DMS_CUDA(cudaStreamSynchronize(c.s));
    P.d1_pool.release();
    P.d1_pool = copool;
    DMS_TRY(reduce_columns(c, nrows, ncols, traced));
    DMS_LAUNCH(nrows, 256, k_d1_result_cohomology, nrows, ncols, P.d1_start.as<int64_t>(),
               P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(), P.d1_rowmap.as<int32_t>(),
               P.d1_row.as<int32_t>(), P.d1_rowpaired.as<uint8_t>());
    return DMS_OK;
}

// D1 by the lazy reduction (d1_mode 3): no separate tracing; columns are
// advanced only as far as their pivots, between rounds of claims and
// additions of partially expanded columns.
HeapEnt *lz_heap(LazyScratch &s) { return s.buf.as<HeapEnt>(); }
HashEnt *lz_hash(LazyScratch &s) { return (HashEnt *)(lz_heap(s) + (size_t)s.hcap * s.nt); }
int32_t *lz_tgen(LazyScratch &s) { return (int32_t *)(lz_hash(s) + (size_t)s.hashcap * s.nt); }

dms_status lazy_scratch(Ctx &c, LazyScratch &s, int hcap, int hashcap, int64_t nt) {
    if (s.buf.p && s.hcap == hcap && s.hashcap == hashcap && s.nt >= nt) return DMS_OK;
    const size_t per = (size_t)hcap * sizeof(HeapEnt) + (size_t)hashcap * sizeof(HashEnt) + 4;
    s.buf.release();
    if (!s.buf.ensure(per * (size_t)nt + 16)) return DMS_ERR_OOM;
    s.hcap = hcap; s.hashcap = hashcap; s.nt = nt;
    DMS_CUDA(cudaMemsetAsync(lz_hash(s), 0xFF, (size_t)hashcap * nt * sizeof(HashEnt), c.s));
    DMS_CUDA(cudaMemsetAsync(lz_tgen(s), 0, 4 * (size_t)nt, c.s));
    return DMS_OK;
}

dms_status order_by_vertex(Ctx &c, const int32_t *vert, const int32_t *idx, int64_t n, int slot,
                           const int32_t **perm);

template <typename T, bool B>
dms_status reduce_lazy(Ctx &c, const T *values, int64_t ncols, int64_t n1, const uint8_t *is_row) {
    Pipeline &P = c.P;
    DMS_ALLOC(P.d1_owner, 4 * n1 + 4);
    DMS_ALLOC(P.d1_act, 4 * 4 * ncols + 4);
    DMS_ALLOC(P.d1_next, 4 * 4 * ncols + 4);
    DMS_ALLOC(P.d1_re, 4 * ncols + 4);
    DMS_ALLOC(P.d1_todo, 4 * ncols + 4);
    DMS_ALLOC(P.d1_stamp, 4 * ncols + 4);
    DMS_ALLOC(P.d1_astamp, 4 * ncols + 4);
    DMS_CUDA(cudaMemsetAsync(P.d1_owner.p, 0x7F, 4 * n1 + 4, c.s));
    DMS_CUDA(cudaMemsetAsync(P.d1_stamp.p, 0xFF, 4 * ncols + 4, c.s));
    DMS_CUDA(cudaMemsetAsync(P.d1_astamp.p, 0xFF, 4 * ncols + 4, c.s));
    DMS_CUDA(cudaMemsetAsync(P.d1_len.p, 0xFF, 4 * ncols + 4, c.s));   // -1: not yet listed
    {
        // the first advances in vertex-id order (nearby walks share their records)
        const int32_t *corder = nullptr;
        DMS_TRY(order_by_vertex(c, P.c_vert[2].as<int32_t>(), P.d1_colmap.as<int32_t>(), ncols, 1,
                                &corder));
        DMS_CUDA(cudaMemcpyAsync(P.d1_act.p, corder, 4 * ncols, cudaMemcpyDeviceToDevice, c.s));
    }
    DMS_CUDA(cudaMemsetAsync(&c.st->misc[0], 0, 4 * sizeof(long long), c.s));
    DMS_CUDA(cudaMemsetAsync(&c.st->red_io[0], 0, 2 * sizeof(long long), c.s));
    DMS_CUDA(cudaMemsetAsync(&c.st->pool_top, 0, sizeof(unsigned long long), c.s));
    int64_t pool_cap = d1_pool_entries(std::max<int64_t>(1 << 18, 24 * ncols + 1024));
    DMS_ALLOC(P.d1_pool, sizeof(Ent) * pool_cap);
    Ent *pool = P.d1_pool.as<Ent>();

    // scratch: the first pass small (stays in L2), retries 16x larger per level
    const int64_t nt_small = std::min<int64_t>(152 * 16 * 128, (ncols + 127) / 128 * 128);
    const int heap0 = P.tune[DMS_TUNE_LAZY_HEAP];
    DMS_TRY(lazy_scratch(c, P.lz_small, heap0, hash_cap_for(heap0), nt_small));
    int big_hash = 1 << 22;   // the serial walks in global memory, after the block levels
    int32_t launch = 0;

    auto args = [&](LazyScratch &s) {
        LzArgs<T, B> a;
        a.values = values; a.geo = geo_of<B>(c); a.flags = P.flags.as<uint8_t>();
        a.grad = P.grad.as<GradRec>(); a.vrank = P.vrank.as<int32_t>();
        a.recs = P.recs.as<CritRec>(); a.base1 = P.base[1].as<int32_t>(); a.is_row = is_row;
        a.v2 = P.c_vert[2].as<int32_t>(); a.l2 = P.c_loc[2].as<uint8_t>();
        a.colmap = P.d1_colmap.as<int32_t>();
        a.heap_all = lz_heap(s); a.hash_all = lz_hash(s); a.tgen = lz_tgen(s);
        a.hcap = s.hcap; a.hashcap = s.hashcap;
        return a;
    };
    // one thread per listed column, at most the scratch's threads (a
    // multiple of 32), in blocks that divide that count exactly
    auto advance = [&](LazyScratch &s, const int32_t *todo, int64_t ntodo, int32_t *retry) {
        if (ntodo == 0) return cudaSuccess;
        const int64_t nt = std::min<int64_t>(s.nt, (ntodo + 31) / 32 * 32);
        const int threads = nt % 128 == 0 ? 128 : 32;
        k_lz_advance<T, B><<<(unsigned)(nt / threads), threads, 0, c.s>>>(
            args(s), todo, ntodo, P.d1_astamp.as<int32_t>(), launch++, pool, pool_cap,
            P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(), retry, c.st);
        c.launches++;
        return cudaGetLastError();
    };

    int64_t nactive = ncols, stamp = 0, overflowed = 0;
    const int64_t list_cap = 4 * ncols;
    const int64_t limit = P.max_iters > 0 ? P.max_iters : ((int64_t)1 << 22);
    DMS_CUDA(cudaMemsetAsync(&c.st->misc[2], 0, sizeof(long long), c.s));
    KEV(18);
    KEV(19);
    KEV(20);
    const bool debug = getenv("DMS_DEBUG") != nullptr;
    struct Events {
        cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Events() { for (auto x : e) if (x) cudaEventDestroy(x); }
    } dbg;
    cudaEvent_t *dev = dbg.e;
    if (debug)
        for (int i = 0; i < 4; i++) cudaEventCreate(&dev[i]);
    for (int64_t r = 0; r < limit; r++, stamp++) {
        DMS_CUDA(cudaMemsetAsync(&c.st->misc[0], 0, 2 * sizeof(long long), c.s));
        DMS_CUDA(cudaMemsetAsync(&c.st->misc[3], 0, sizeof(long long), c.s));
        if (debug) cudaEventRecord(dev[0], c.s);
        if (advance(P.lz_small, P.d1_act.as<int32_t>(), nactive, P.d1_todo.as<int32_t>()) !=
            cudaSuccess)
            return DMS_ERR_CUDA;
        if (debug) cudaEventRecord(dev[1], c.s);
        DMS_LAUNCH(nactive, 256, k_lz_claim, P.d1_act.as<int32_t>(), nactive,
                   P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(), pool,
                   P.vrank.as<int32_t>(), P.recs.as<CritRec>(), P.base[1].as<int32_t>(),
                   P.d1_owner.as<int32_t>(), P.d1_re.as<int32_t>(), c.st);
        if (debug) cudaEventRecord(dev[2], c.s);
        {
            // one warp per listed column, at most one per thread slot of the
            // small scratch (a large wall fails fast here and is expanded by a
            // block between rounds)
            const int64_t want = std::min<int64_t>(64 * nactive, (int64_t)152 * 64 * 256);
            LazyScratch &sc = P.lz_small;
            const int64_t th = std::min<int64_t>(want, 32 * sc.nt);
            k_lz_add<T, B><<<(unsigned)((th + 255) / 256), 256, 0, c.s>>>(
                args(sc), P.d1_act.as<int32_t>(), nactive, P.d1_re.as<int32_t>(),
                P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(), pool, P.d1_owner.as<int32_t>(),
                P.d1_stamp.as<int32_t>(), (int32_t)stamp, P.d1_next.as<int32_t>(), pool_cap, c.st);
            c.launches++;
            DMS_CUDA(cudaGetLastError());
        }
        if (debug) cudaEventRecord(dev[3], c.s);
        dms_status s = sync_status(c);
        P.rounds_d1 = r + 1;
        const int64_t nre = c.hst->misc[0], nnext = c.hst->misc[1];
        int64_t nretry = c.hst->misc[3];
        if (debug) {
            float ta = 0, tc = 0, td = 0;
            cudaEventElapsedTime(&ta, dev[0], dev[1]);
            cudaEventElapsedTime(&tc, dev[1], dev[2]);
            cudaEventElapsedTime(&td, dev[2], dev[3]);
            fprintf(stderr, "d1 lazy round %lld: listed %lld retry %lld rechecked %lld next %lld "
                    "adds %lld pool %llu | advance %.3f claim %.3f add %.3f ms\n", (long long)r,
                    (long long)nactive, (long long)nretry, (long long)nre, (long long)nnext,
                    c.hst->misc[2], c.hst->pool_top, ta, tc, td);
        }
        if (s != DMS_OK && s != DMS_ERR_CAPACITY) return s;
        bool full = s == DMS_ERR_CAPACITY;
        // the next round's list: the columns changed by additions, then those
        // that were not advanced (or, after the pool filled up, every column
        // this round listed)
        int32_t *nx = P.d1_next.as<int32_t>();
        int64_t nlist = nnext;
        if (full) {
            if (nlist + nactive + nre <= list_cap) {
                DMS_CUDA(cudaMemcpyAsync(nx + nlist, P.d1_act.p, 4 * nactive,
                                         cudaMemcpyDeviceToDevice, c.s));
                DMS_CUDA(cudaMemcpyAsync(nx + nlist + nactive, P.d1_re.p, 4 * nre,
                                         cudaMemcpyDeviceToDevice, c.s));
                nlist += nactive + nre;
            } else {
                DMS_LAUNCH(ncols, 256, k_iota32, nx, ncols);   // listing every column is safe
                nlist = ncols;
            }
        } else if (nretry > 0) {
            // columns that outgrew the small scratch: advance them now with
            // larger scratch (16x per level), then list them for their claims
            overflowed += nretry;
            int32_t *todo = P.d1_todo.as<int32_t>(), *retry = P.d1_re.as<int32_t>();
            DMS_CUDA(cudaMemcpyAsync(nx + nlist, todo, 4 * nretry, cudaMemcpyDeviceToDevice,
                                     c.s));
            nlist += nretry;
            // first expanded whole by blocks (two sizes of block scratch), then
            // walked serially with per-thread scratch in global memory; the
            // environment may set the first level (DMS_D1_LAZY_LEVEL = 0, 1, 2),
            // which exercises the later ones
            int level = 0;
            if (const char *e = getenv("DMS_D1_LAZY_LEVEL")) level = std::min(2, std::max(0, atoi(e)));
            while (nretry > 0 && !full) {
                DMS_CUDA(cudaMemsetAsync(&c.st->misc[3], 0, sizeof(long long), c.s));
                if (level < 2) {
                    const BxLevel &L = kBxLevels[level];
                    const size_t hash_b = (size_t)L.blocks * ((size_t)1 << L.hbits) * kBxSlotBytes;
                    const size_t list_b = (size_t)L.blocks * 3 * L.fcap * 4;
                    const size_t sink_b = (size_t)L.blocks * L.scap * 4;
                    const size_t sort_b = (size_t)L.blocks * 2 * L.scap * sizeof(Ent);
                    DevBuf &bx = P.bx_buf[level];
                    DMS_ALLOC(bx, hash_b + list_b + sink_b + sort_b);
                    char *base = bx.as<char>();
                    k_lz_expand_block<T, B>
                        <<<(unsigned)std::min<int64_t>(nretry, L.blocks), kBxThreads, 0, c.s>>>(
                            args(P.lz_small), todo, nretry, P.d1_astamp.as<int32_t>(), launch++,
                            pool, pool_cap, P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(),
                            retry, base, L.hbits, (int32_t *)(base + hash_b), L.fcap,
                            (int32_t *)(base + hash_b + list_b),
                            (Ent *)(base + hash_b + list_b + sink_b), L.scap, c.st);
                    c.launches++;
                    DMS_CUDA(cudaGetLastError());
                } else {
                    if (!P.lz_big.buf.p || P.lz_big.hashcap < big_hash) {
                        const int bh = big_hash * 3 / 4;
                        const size_t per = (size_t)bh * sizeof(HeapEnt) +
                                           (size_t)big_hash * sizeof(HashEnt) + 4;
                        int64_t nt = std::max<int64_t>(
                            32, std::min<int64_t>(ncols, ((int64_t)4 << 30) / (int64_t)per));
                        DMS_TRY(lazy_scratch(c, P.lz_big, bh, big_hash, (nt + 31) / 32 * 32));
                    }
                    if (advance(P.lz_big, todo, nretry, retry) != cudaSuccess)
                        return DMS_ERR_CUDA;
                }
                const auto t_retry = std::chrono::steady_clock::now();
                s = sync_status(c);
                if (debug)
                    fprintf(stderr, "  retry %lld columns at level %d: %.3f ms (host); block "
                            "expansions so far: %lld columns, %lld edges, %lld + %lld levels\n",
                            (long long)nretry, level,
                            std::chrono::duration<double, std::milli>(
                                std::chrono::steady_clock::now() - t_retry).count(),
                            c.hst->bx[3], c.hst->bx[0], c.hst->bx[1], c.hst->bx[2]);
                if (s != DMS_OK && s != DMS_ERR_CAPACITY) return s;
                full = s == DMS_ERR_CAPACITY;
                const int64_t again = c.hst->misc[3];
                if (again > 0 && !full) {
                    if (level >= 2) big_hash *= 16;     // still too large: 16x more
                    level++;
                    if (big_hash > (1 << 24)) return DMS_ERR_CAPACITY;
                }
                std::swap(todo, retry);
                nretry = again;
            }
        }
        if (full) {
            // compact the live lists into a pool twice as large
            DMS_ALLOC(P.flag_a, 4 * ncols + 4);
            DMS_ALLOC(P.flag_b, 4 * ncols + 4);
            DMS_LAUNCH(ncols, 256, k_lz_live, ncols, P.d1_len.as<int32_t>(),
                       P.flag_a.as<int32_t>());
            DMS_TRY(scan(c, P.flag_a.as<int32_t>(), P.flag_b.as<int32_t>(), ncols,
                         &c.st->total[3]));
            DMS_CUDA(cudaMemcpyAsync(c.hst, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.s));
            DMS_CUDA(cudaStreamSynchronize(c.s));
            const int64_t live = c.hst->total[3];
            // at least 3x the live entries stay free after the compaction
            const int64_t cap2 = std::max<int64_t>(pool_cap, 4 * live + (1 << 20));
            if (cap2 >= ((int64_t)1 << 31)) return DMS_ERR_CAPACITY;
            DevBuf fresh;
            if (!fresh.ensure(sizeof(Ent) * (size_t)cap2)) return DMS_ERR_OOM;
            DMS_LAUNCH(ncols, 256, k_lz_compact, ncols, P.d1_start.as<int64_t>(),
                       P.d1_len.as<int32_t>(), P.flag_b.as<int32_t>(), pool, fresh.as<Ent>());
            DMS_CUDA(cudaStreamSynchronize(c.s));
            P.d1_pool.release();
            P.d1_pool = fresh;
            pool = P.d1_pool.as<Ent>();
            pool_cap = cap2;
            c.hst->err = 0;
            c.hst->pool_top = (unsigned long long)live;
            DMS_CUDA(cudaMemcpyAsync(c.st, c.hst, sizeof(DevStatus), cudaMemcpyHostToDevice, c.s));
            P.d1_pool_grows++;
        }
        nactive = nlist;
        std::swap(P.d1_act, P.d1_next);
        if (nactive == 0) {
            P.d1_overflow = overflowed;
            P.d1_io_read = c.hst->red_io[0];
            P.d1_io_written = c.hst->red_io[1];
            P.d1_additions = c.hst->misc[2];
            P.d1_pool_used = (int64_t)c.hst->pool_top;
            DMS_LAUNCH(ncols, 256, k_lz_result, ncols, P.d1_start.as<int64_t>(),
                       P.d1_len.as<int32_t>(), pool, P.vrank.as<int32_t>(),
                       P.recs.as<CritRec>(), P.base[1].as<int32_t>(), P.d1_row.as<int32_t>(),
                       P.d1_rowpaired.as<uint8_t>(), c.st);
            KEV(21);
            return DMS_OK;
        }
    }
    return DMS_ERR_ITER_LIMIT;
}

// Batch output: the pairs of dimension d (all fields, in the order of the
// single-grid output) regrouped field by field with a stable LSD radix sort
// on the field index, so that each field's pairs keep their order; the
// per-field ranges go to P.batch_off[d].
dms_status group_by_field(Ctx &c, int d, int64_t rows) {
    Pipeline &P = c.P;
    const int nf = (int)P.nf;
    P.batch_off[d].assign(nf + 1, 0);
    if (rows == 0) {
        DMS_ALLOC(P.batch_pofs[d], 8 * (nf + 1));
        DMS_CUDA(cudaMemsetAsync(P.batch_pofs[d].p, 0, 8 * (nf + 1), c.s));
        return DMS_OK;
    }
    for (int k = 0; k < 2; k++) {
        DMS_ALLOC(P.bt_k[k], 4 * rows + 4);
        DMS_ALLOC(P.bt_v[k], 4 * rows + 4);
    }
    const int rtiles = (int)((rows + kRsTile - 1) / kRsTile);
    DMS_ALLOC(P.bt_h[0], 4 * (size_t)256 * rtiles);
    DMS_ALLOC(P.bt_h[1], 4 * (size_t)256 * rtiles);
    DMS_ALLOC(P.bt_cnt, 4 * (nf + 1));
    DMS_ALLOC(P.out_tmp, sizeof(dms_pair) * (rows + 1));
    DMS_CUDA(cudaMemcpyAsync(P.bt_k[0].p, P.out_field[d].p, 4 * rows, cudaMemcpyDeviceToDevice,
                             c.s));
    DMS_LAUNCH(rows, 256, k_iota32, P.bt_v[0].as<int32_t>(), rows);
    uint32_t *kin = P.bt_k[0].as<uint32_t>(), *kout = P.bt_k[1].as<uint32_t>();
    int32_t *vin = P.bt_v[0].as<int32_t>(), *vout = P.bt_v[1].as<int32_t>();
    for (int shift = 0; shift < 16 && (shift == 0 || nf > (1 << shift)); shift += 8) {
        k_rs_hist<uint32_t><<<rtiles, kRsThreads, 0, c.s>>>(kin, rows, shift,
                                                           P.bt_h[0].as<int32_t>(), rtiles);
        c.launches++;
        DMS_TRY(scan(c, P.bt_h[0].as<int32_t>(), P.bt_h[1].as<int32_t>(), (int64_t)256 * rtiles,
                     &c.st->total[1]));
        k_rs_scatter<uint32_t><<<rtiles, kRsThreads, 0, c.s>>>(kin, vin, kout, vout, rows, shift,
                                                              P.bt_h[1].as<int32_t>(), rtiles);
        c.launches++;
        DMS_CUDA(cudaGetLastError());
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    DMS_LAUNCH(rows, 256, k_gather_pairs, P.out_pairs[d].as<dms_pair>(), vin, rows,
               P.out_tmp.as<dms_pair>());
    std::swap(P.out_pairs[d], P.out_tmp);
    DMS_CUDA(cudaMemsetAsync(P.bt_cnt.p, 0, 4 * (nf + 1), c.s));
    DMS_LAUNCH(rows, 256, k_field_count, P.out_field[d].as<int32_t>(), rows,
               P.bt_cnt.as<int32_t>());
    std::vector<int32_t> cnt(nf);
    DMS_CUDA(cudaMemcpyAsync(cnt.data(), P.bt_cnt.p, 4 * nf, cudaMemcpyDeviceToHost, c.s));
    DMS_CUDA(cudaStreamSynchronize(c.s));
    for (int f = 0; f < nf; f++) P.batch_off[d][f + 1] = P.batch_off[d][f] + cnt[f];
    DMS_ALLOC(P.batch_pofs[d], 8 * (nf + 1));
    DMS_CUDA(cudaMemcpyAsync(P.batch_pofs[d].p, P.batch_off[d].data(), 8 * (nf + 1),
                             cudaMemcpyHostToDevice, c.s));
    DMS_CUDA(cudaStreamSynchronize(c.s));
    return DMS_OK;
}

// Stable LSD radix sort of n (32-bit key, int32 value) pairs on the low
// `bits` bits of the keys, 8 bits a pass, with P.ord_h as histograms; the
// sorted pairs end in (kin, vin) (the pointers swap with each pass).
dms_status radix_u32(Ctx &c, uint32_t *&kin, int32_t *&vin, uint32_t *&kout, int32_t *&vout,
                     int64_t n, int bits, int rtiles, bool staged = false) {
    Pipeline &P = c.P;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<uint32_t><<<rtiles, kRsThreads, 0, c.s>>>(kin, n, shift, P.ord_h[0].as<int32_t>(),
                                                           rtiles);
        c.launches++;
        DMS_TRY(scan(c, P.ord_h[0].as<int32_t>(), P.ord_h[1].as<int32_t>(), (int64_t)256 * rtiles,
                     &c.st->total[1]));
        if (staged)
            k_rs_scatter<uint32_t, true><<<rtiles, kRsThreads, 0, c.s>>>(
                kin, vin, kout, vout, n, shift, P.ord_h[1].as<int32_t>(), rtiles);
        else
            k_rs_scatter<uint32_t><<<rtiles, kRsThreads, 0, c.s>>>(
                kin, vin, kout, vout, n, shift, P.ord_h[1].as<int32_t>(), rtiles);
        c.launches++;
        DMS_CUDA(cudaGetLastError());
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return DMS_OK;
}

// A permutation of n items (item i at vertex vert[idx[i]], or vert[i]) into
// vertex-id order, by a stable LSD radix sort; *perm points into scratch
// buffer `slot` (0 or 1) and stays valid until the next call with that slot.
dms_status order_by_vertex(Ctx &c, const int32_t *vert, const int32_t *idx, int64_t n, int slot,
                           const int32_t **perm) {
    Pipeline &P = c.P;
    *perm = nullptr;
    if (n <= 0) return DMS_OK;
    DevBuf *kb = &P.ord_k[2 * slot], *vb = &P.ord_v[2 * slot];
    for (int k = 0; k < 2; k++) {
        DMS_ALLOC(kb[k], 4 * n + 4);
        DMS_ALLOC(vb[k], 4 * n + 4);
    }
    const int rtiles = (int)((n + kRsTile - 1) / kRsTile);
    DMS_ALLOC(P.ord_h[0], 4 * (size_t)256 * rtiles);
    DMS_ALLOC(P.ord_h[1], 4 * (size_t)256 * rtiles);
    uint32_t *kin = kb[0].as<uint32_t>(), *kout = kb[1].as<uint32_t>();
    int32_t *vin = vb[0].as<int32_t>(), *vout = vb[1].as<int32_t>();
    DMS_LAUNCH(n, 256, k_gather_vid, vert, idx, n, kin, vin);
    int bits = 0;
    while (bits < 32 && (((int64_t)1 << bits) < P.n)) bits++;
    DMS_TRY(radix_u32(c, kin, vin, kout, vout, n, bits, rtiles));
    *perm = vin;
    return DMS_OK;
}

// ProcessLowerStars with the tuned block size: in id order, or, when
// `sorted`, in two passes with the stars sorted by shape in between.
template <typename T, bool B>
dms_status launch_pls(Ctx &c, const T *values, const Geo<B> &geo, const int32_t *list,
                      int64_t count, bool sorted) {
    Pipeline &P = c.P;
    if (count <= 0) return DMS_OK;
    uint8_t *fl = P.flags.as<uint8_t>();
    GradRec *gr = P.grad.as<GradRec>();
    const int nt = P.tune[DMS_TUNE_PLS_BLOCK];
    if (!sorted) {
        k_pls<T, B><<<blocks_for(count, nt), nt, 0, c.s>>>(values, geo, list, count, fl, gr);
        c.launches++;
        DMS_CUDA(cudaGetLastError());
        return DMS_OK;
    }
    // the vertex-order scratch is free here: the walks that use it come later
    for (int k = 0; k < 2; k++) {
        DMS_ALLOC(P.ord_k[k], 4 * count + 4);
        DMS_ALLOC(P.ord_v[k], 4 * count + 4);
    }
    DMS_ALLOC(P.pls_ranks, 8 * count + 8);
    const int rtiles = (int)((count + kRsTile - 1) / kRsTile);
    DMS_ALLOC(P.ord_h[0], 4 * (size_t)256 * rtiles);
    DMS_ALLOC(P.ord_h[1], 4 * (size_t)256 * rtiles);
    uint32_t *kin = P.ord_k[0].as<uint32_t>(), *kout = P.ord_k[1].as<uint32_t>();
    int32_t *vin = P.ord_v[0].as<int32_t>(), *vout = P.ord_v[1].as<int32_t>();
    unsigned long long *rk = P.pls_ranks.as<unsigned long long>();
    k_pls_keys<T, B><<<blocks_for(count, 256), 256, 0, c.s>>>(values, geo, list, count, kin, vin,
                                                              rk, fl);
    c.launches++;
    DMS_CUDA(cudaGetLastError());
    DMS_TRY(radix_u32(c, kin, vin, kout, vout, count, kLinks, rtiles, true));
    k_pls_run<<<blocks_for(count, nt), nt, 0, c.s>>>(list, kin, vin, rk, count, gr);
    c.launches++;
    DMS_CUDA(cudaGetLastError());
    return DMS_OK;
}

// ------------------------------------------ generators of the D1 pairs
//
// In the generator mode each traced column also carries, as passive entries,
// the edges the Morse boundary compresses away, so its list is the full
// simplicial boundary of the 2-chain it swept: the 2-saddle and the
// triangles of its descending paths.  Additions keep that (a sum of such
// boundaries), so when the reduction ends the list of a paired column is a
// 1-cycle homologous to the boundary of its 2-saddle among the simplices
// before it (every swept triangle and every column added is earlier), with
// no triangle-paired edge left, and its highest edge is its pivot: the
// highest edge of a 1-cycle is a positive edge, and the rows are the
// positive edges left (Sec. 8's generator, Boundary(sigma_j)).
//
// Records per D1 pair, in column order (the order of the D1 pairs): birth
// edge id, death triangle id, k, then the k edge ids of the cycle.
__global__ void k_gen_count(int64_t ncols, const int32_t *__restrict__ d1_row,
                            const int32_t *__restrict__ len, int32_t *cnt) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncols) cnt[c] = d1_row[c] >= 0 ? 3 + len[c] : 0;
}

__global__ void k_gen_write(int64_t ncols, const int32_t *__restrict__ d1_row,
                            const int64_t *__restrict__ start, const int32_t *__restrict__ len,
                            const int32_t *__restrict__ pool, const int32_t *__restrict__ pos,
                            const int32_t *__restrict__ colmap, const int32_t *__restrict__ v1,
                            const uint8_t *__restrict__ l1, const int32_t *__restrict__ v2,
                            const uint8_t *__restrict__ l2, GridParams g, int64_t *out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols || d1_row[c] < 0) return;
    const StarTables &S = g_star;
    int64_t o = pos[c];
    const int32_t r = d1_row[c], j2 = colmap[c];
    out[o++] = edge_id(S, g, v1[r], l1[r]);
    out[o++] = tri_id(S, g, v2[j2], l2[j2]);
    const int L = len[c];
    out[o++] = L;
    const int32_t *e = pool + start[c];
    for (int k = 0; k < L; k++) {
        const int32_t x = e[k];
        out[o++] = x >= 0 ? edge_id(S, g, v1[x], l1[x]) : -1 - (int64_t)x;
    }
}

dms_status generator_records(Ctx &c, int64_t ncols) {
    Pipeline &P = c.P;
    DMS_ALLOC(P.flag_a, 4 * ncols + 4);
    DMS_ALLOC(P.flag_b, 4 * ncols + 4);
    int32_t *cnt = P.flag_a.as<int32_t>(), *pos = P.flag_b.as<int32_t>();
    DMS_LAUNCH(ncols, 256, k_gen_count, ncols, P.d1_row.as<int32_t>(), P.d1_len.as<int32_t>(),
               cnt);
    DMS_TRY(scan(c, cnt, pos, ncols, &c.st->total[3]));
    DMS_TRY(sync_status(c));
    const int64_t words = c.hst->total[3];
    if (words >= ((int64_t)1 << 31)) return DMS_ERR_CAPACITY;
    DMS_ALLOC(P.gen_out, 8 * words + 8);
    DMS_LAUNCH(ncols, 128, k_gen_write, ncols, P.d1_row.as<int32_t>(), P.d1_start.as<int64_t>(),
               P.d1_len.as<int32_t>(), P.d1_pool.as<int32_t>(), pos, P.d1_colmap.as<int32_t>(),
               P.c_vert[1].as<int32_t>(), P.c_loc[1].as<uint8_t>(), P.c_vert[2].as<int32_t>(),
               P.c_loc[2].as<uint8_t>(), c.g, P.gen_out.as<int64_t>());
    P.gen_words = words;
    return DMS_OK;
}

// D2's ascending walks (Sec. 5.2) on the stream of c: every critical triangle
// ascends on both sides to the maxima (or the outside node) it links; the
// arcs go to P.arc2_a / P.arc2_b.  The walks of a warp start at nearby
// vertices (vertex-id order), so they share the records they read.
template <typename T, bool B>
dms_status d2_walks(Ctx &c, const T *values, const Geo<B> &geo, int64_t n2, int32_t vmax,
                    int64_t max_steps, int32_t *young2) {
    Pipeline &P = c.P;
    KEV(14);
    const int32_t *order2 = nullptr;
    DMS_TRY(order_by_vertex(c, P.c_vert[2].as<int32_t>(), nullptr, n2, 0, &order2));
    // the tet words share the buffer of the D1 trace's row words (written later)
    DMS_ALLOC(P.vcrit, 8 * P.n + 8);
    DMS_LAUNCH(P.n_crit, 256, k_tet_words, P.vc.as<int32_t>(), P.n_crit, P.recs.as<CritRec>(),
               P.base[3].as<int32_t>(), P.vcrit.as<unsigned long long>());
    DMS_LAUNCH(n2, 128, (k_d2_arcs<T, B>), values, geo, P.flags.as<uint8_t>(),
               P.grad.as<GradRec>(), P.vcrit.as<unsigned long long>(),
               P.c_vert[2].as<int32_t>(), P.c_loc[2].as<uint8_t>(), n2,
               order2, vmax, P.virtual_max, P.arc2_a.as<int32_t>(), P.arc2_b.as<int32_t>(),
               young2, max_steps, P.dense_grad ? 1 : 0, c.st);
    KEV(15);
    return DMS_OK;
}

template <typename T, bool B> dms_status run(Ctx &c, const T *values) {
    using K = typename Key<T>::K;
    Pipeline &P = c.P;
    const Geo<B> geo = geo_of<B>(c);
    cudaEvent_t *ev = c.ev;
    const int64_t n = P.n;
    const int64_t max_steps = P.max_iters > 0 ? P.max_iters : n + 1;
    P.dense_grad = false;
    DMS_CUDA(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), c.s));

    // ---- gradient: classification, compaction, sort, ProcessLowerStars
    ClsTiling ct;
    if constexpr (B) {
        ct.tile = kClsTile;
        ct.ntiles = (n + kClsTile - 1) / kClsTile;
    } else {
        ct = cls_tiling<T>(c.g, values);
    }
    const int64_t ntiles = ct.ntiles;
    DMS_ALLOC(P.tile_cnt, 4 * ntiles + 4);
    DMS_ALLOC(P.tile_off, 4 * ntiles + 4);
    for (int i = 0; i < 24; i++) KEV(i);   // families that do not run read 0 ms
    KEV(0);
    if constexpr (B) {
        DMS_CUDA(cudaMemsetAsync(P.fmax_field.p, 0, 8 * P.nf, c.s));
        k_classify_batch<T><<<(unsigned)ntiles, kClsThreads, 0, c.s>>>(
            values, geo, n, P.flags.as<uint8_t>(), P.tile_cnt.as<int32_t>(),
            P.fmax_field.as<unsigned long long>(), c.st);
    } else {
        k_classify2<T><<<(unsigned)ntiles, kClsThreads, 0, c.s>>>(
            values, c.g, ct.rows_per_block, ct.runs_per_row, ct.aligned, P.flags.as<uint8_t>(),
            P.tile_cnt.as<int32_t>(), c.st);
    }
    c.launches++;
    DMS_CUDA(cudaGetLastError());
    KEV(1);
    DMS_TRY(scan(c, P.tile_cnt.as<int32_t>(), P.tile_off.as<int32_t>(), ntiles, &c.st->total[0]));
    DMS_TRY(sync_status(c));
    const int64_t nc = c.hst->total[0];
    P.n_crit = nc;
    // Critical simplices are indexed and scanned in int32.  A lower star
    // holds at most 1 + 5 + 5 + 1 critical cells (the largest reduced Betti
    // numbers of a lower link), so up to (2^31 - 1) / 12 PL-critical
    // vertices every index, per dimension and over all of them, fits.
    if (nc > kMaxCriticalVertices) return DMS_ERR_CAPACITY;
    DMS_ALLOC(P.vc, 4 * nc + 4);
    DMS_ALLOC(P.vc_tmp, 4 * nc + 4);
    DMS_ALLOC(P.keys, sizeof(K) * nc + 8);
    DMS_ALLOC(P.keys_tmp, sizeof(K) * nc + 8);
    DMS_ALLOC(P.recs, sizeof(CritRec) * nc + 8);
    for (int d = 0; d < 4; d++) {
        DMS_ALLOC(P.cnt[d], 4 * nc + 4);
        DMS_ALLOC(P.base[d], 4 * nc + 4);
    }
    KEV(2);
    k_compact2<<<(unsigned)ntiles, kClsThreads, 0, c.s>>>(P.flags.as<uint8_t>(), n, ct.tile,
                                                         P.tile_off.as<int32_t>(),
                                                         P.vc.as<int32_t>());
    c.launches++;
    DMS_CUDA(cudaGetLastError());
    KEV(3);
    if (nc > 0) {
        // ProcessLowerStars in id order (coalesced stencils): on every vertex
        // when critical vertices are dense (the walks of D2 and D1 then visit
        // most vertices), otherwise on the critical ones, the rest on demand
        KEV(6);
        const int ps = P.tune[DMS_TUNE_PLS_SORT];
        const bool sort_stars = ps == 2 || (ps == 1 && nc * 4 > n);
        P.dense_grad = nc * 4 > n || n <= kDenseGradientBelow;
        if (P.dense_grad)
            DMS_TRY((launch_pls<T, B>(c, values, geo, nullptr, n, sort_stars)));
        else
            DMS_TRY((launch_pls<T, B>(c, values, geo, P.vc.as<int32_t>(), nc, sort_stars)));
        KEV(7);
        // stable LSD radix sort of the critical vertices (in id order) by value
        KEV(4);
        DMS_LAUNCH(nc, 256, k_gather_keys<T>, values, P.vc.as<int32_t>(), nc, P.keys.as<K>());
        const int rtiles = (int)((nc + kRsTile - 1) / kRsTile);
        DMS_ALLOC(P.flag_a, 4 * (size_t)256 * rtiles);
        DMS_ALLOC(P.flag_b, 4 * (size_t)256 * rtiles);
        K *kin = P.keys.as<K>(), *kout = P.keys_tmp.as<K>();
        int32_t *vin = P.vc.as<int32_t>(), *vout = P.vc_tmp.as<int32_t>();
        for (int shift = 0; shift < (int)(8 * sizeof(T)); shift += 8) {
            k_rs_hist<K><<<rtiles, kRsThreads, 0, c.s>>>(kin, nc, shift, P.flag_a.as<int32_t>(),
                                                        rtiles);
            c.launches++;
            DMS_TRY(scan(c, P.flag_a.as<int32_t>(), P.flag_b.as<int32_t>(), (int64_t)256 * rtiles,
                         &c.st->total[1]));
            k_rs_scatter<K, sizeof(K) == 4><<<rtiles, kRsThreads, 0, c.s>>>(kin, vin, kout, vout, nc, shift,
                                                           P.flag_b.as<int32_t>(), rtiles);
            c.launches++;
            DMS_CUDA(cudaGetLastError());
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        if (vin != P.vc.as<int32_t>()) {
            std::swap(P.vc, P.vc_tmp);
            std::swap(P.keys, P.keys_tmp);
        }
        KEV(5);
        DMS_LAUNCH(nc, 256, k_critrec, P.vc.as<int32_t>(), nc, P.grad.as<GradRec>(),
                   P.recs.as<CritRec>(), P.cnt[0].as<int32_t>(), P.cnt[1].as<int32_t>(),
                   P.cnt[2].as<int32_t>(), P.cnt[3].as<int32_t>(), P.vrank.as<int32_t>());
    }
    cudaEventRecord(ev[2], c.s);
    c.nv.next("dms/sort");

    // ---- critical simplices C0..C3 in lexicographic order
    for (int d = 0; d < 4; d++)
        DMS_TRY(scan(c, P.cnt[d].as<int32_t>(), P.base[d].as<int32_t>(), nc, &c.st->total[d]));
    DMS_TRY(sync_status(c));
    for (int d = 0; d < 4; d++) P.n_c[d] = c.hst->total[d];
    const int64_t n0 = P.n_c[0], n1 = P.n_c[1], n2 = P.n_c[2], n3 = P.n_c[3];
    for (int d = 0; d < 4; d++) {
        DMS_ALLOC(P.c_vert[d], 4 * P.n_c[d] + 4);
        DMS_ALLOC(P.c_loc[d], P.n_c[d] + 4);
    }
    KEV(8);
    DMS_LAUNCH(nc, 128, k_emit, P.vc.as<int32_t>(), nc, P.recs.as<CritRec>(),
               P.base[0].as<int32_t>(), P.base[1].as<int32_t>(), P.base[2].as<int32_t>(),
               P.base[3].as<int32_t>(), P.c_vert[0].as<int32_t>(), P.c_vert[1].as<int32_t>(),
               P.c_loc[1].as<uint8_t>(), P.c_vert[2].as<int32_t>(), P.c_loc[2].as<uint8_t>(),
               P.c_vert[3].as<int32_t>(), P.c_loc[3].as<uint8_t>());
    KEV(9);
    cudaEventRecord(ev[3], c.s);
    c.nv.next("dms/d0");

    // union-find state shared by D0 and D2; results kept for the output
    DMS_ALLOC(P.arc_a, 4 * n1 + 4);
    DMS_ALLOC(P.arc_b, 4 * n1 + 4);
    DMS_ALLOC(P.arc2_a, 4 * n2 + 4);
    DMS_ALLOC(P.arc2_b, 4 * n2 + 4);
    DMS_ALLOC(P.young, 4 * (n1 + n2) + 8);
    DMS_ALLOC(P.died, nc + n3 + 16);
    int32_t *young0 = P.young.as<int32_t>(), *young2 = young0 + n1;
    uint8_t *died0 = P.died.as<uint8_t>(), *died3 = died0 + nc;
    DMS_CUDA(cudaMemsetAsync(died0, 0, nc + n3 + 1, c.s));

    // ---- D2's ascending walks on the second stream, beside D0 (the paper runs
    // D0 and D2 as parallel tasks, Sec. 7.2); they read only the gradient and
    // the critical lists, and write their own arcs
    const int32_t vmax = (int32_t)n3;
    const bool beside = P.tune[DMS_TUNE_D2_BESIDE_D0] != 0;
    if (beside) {
        DMS_CUDA(cudaEventRecord((cudaEvent_t)P.ev_fork, c.s));
        DMS_CUDA(cudaStreamWaitEvent((cudaStream_t)P.s2, (cudaEvent_t)P.ev_fork, 0));
        Ctx c2 = c;
        c2.s = (cudaStream_t)P.s2;
        c2.scan_buf = &P.scan_tmp2;
        c2.launches = 0;
        c2.nv.open = false;
        DMS_TRY((d2_walks<T, B>(c2, values, geo, n2, vmax, max_steps, young2)));
        c.launches += c2.launches;
        DMS_CUDA(cudaEventRecord((cudaEvent_t)P.ev_join, c2.s));
    }

    // ---- D0: arcs between minima, elder rule in increasing order
    KEV(10);
    DMS_LAUNCH(n1, 256, k_d0_arcs<B>, geo, P.flags.as<uint8_t>(), P.vrank.as<int32_t>(),
               P.base[0].as<int32_t>(),
               P.c_vert[1].as<int32_t>(), P.c_loc[1].as<uint8_t>(), n1, P.arc_a.as<int32_t>(),
               P.arc_b.as<int32_t>(), young0, max_steps, c.st);
    KEV(11);
    KEV(12);
    DMS_TRY(elder_rule(c, P.arc_a.as<int32_t>(), P.arc_b.as<int32_t>(), n1, n0, 0, 0, young0,
                       died0, &P.rounds_d0));
    KEV(13);
    cudaEventRecord(ev[4], c.s);
    c.nv.next("dms/d2");

    // ---- D2: arcs between maxima (node n3 = the virtual maximum), decreasing,
    // once the walks on the second stream are done
    if (beside) DMS_CUDA(cudaStreamWaitEvent(c.s, (cudaEvent_t)P.ev_join, 0));
    else DMS_TRY((d2_walks<T, B>(c, values, geo, n2, vmax, max_steps, young2)));
    KEV(16);
    DMS_TRY(elder_rule(c, P.arc2_a.as<int32_t>(), P.arc2_b.as<int32_t>(), n2, n3 + 1, 1, 1,
                       young2, died3, &P.rounds_d2));
    KEV(17);
    DMS_TRY(sync_status(c));
    cudaEventRecord(ev[5], c.s);
    c.nv.next("dms/d1");

    // ---- D1: rows = C1 not paired in D0, columns = C2 not paired in D2
    DMS_ALLOC(P.rowcol, n1 + n2 + 16);
    uint8_t *is_row = P.rowcol.as<uint8_t>(), *is_col = is_row + n1;
    DMS_ALLOC(P.flag_a, 4 * (n2 + 4));
    DMS_ALLOC(P.flag_b, 4 * (n2 + 4));
    DMS_LAUNCH(n1, 256, k_unpaired, young0, n1, is_row, (int32_t *)nullptr);
    DMS_LAUNCH(n2, 256, k_unpaired, young2, n2, is_col, P.flag_a.as<int32_t>());
    DMS_TRY(scan(c, P.flag_a.as<int32_t>(), P.flag_b.as<int32_t>(), n2, &c.st->total[2]));
    DMS_TRY(sync_status(c));
    const int64_t ncols = c.hst->total[2];
    P.d1_cols = ncols;
    DMS_ALLOC(P.d1_colmap, 4 * ncols + 4);
    DMS_ALLOC(P.d1_start, 8 * ncols + 8);
    DMS_ALLOC(P.d1_len, 4 * ncols + 4);
    DMS_ALLOC(P.d1_ovf, ncols + 4);
    DMS_LAUNCH(n2, 256, k_compact_idx, is_col, P.flag_b.as<int32_t>(), n2, P.d1_colmap.as<int32_t>());
    DMS_CUDA(cudaMemsetAsync(P.d1_len.p, 0, 4 * ncols + 4, c.s));
    P.rounds_d1 = 0;
    DMS_ALLOC(P.d1_row, 4 * ncols + 4);
    DMS_ALLOC(P.d1_rowpaired, n1 + 4);
    DMS_CUDA(cudaMemsetAsync(P.d1_rowpaired.p, 0, n1 + 4, c.s));
    DMS_CUDA(cudaMemsetAsync(P.d1_row.p, 0xFF, 4 * ncols + 4, c.s));
    // mode 0 picks by the density of the columns: sparse 2-saddles (smooth
    // fields) have long descending walls that the lazy columns expand only
    // as far as their pivots; dense ones (noisy fields) have short traces and
    // long chains of additions that the traced 4-byte columns serve better
    const int mode = P.generators ? 1
                     : P.d1_mode != 0 ? P.d1_mode
                                      : (ncols * P.tune[DMS_TUNE_LAZY_DENSITY] < n ? 3 : 1);
    P.d1_mode_used = mode;
    P.trace_toggles = P.trace_expansions = P.d1_longest_chain = 0;
    if (ncols > 0 && mode == 3) {
        DMS_TRY((reduce_lazy<T, B>(c, values, ncols, n1, is_row)));
    } else if (ncols > 0) {
        DMS_ALLOC(P.vcrit, 8 * n + 8);
        DMS_LAUNCH(nc, 256, k_row_words, P.vc.as<int32_t>(), nc, P.recs.as<CritRec>(),
                   P.base[1].as<int32_t>(), is_row, P.vcrit.as<unsigned long long>());
        int64_t pool_cap = std::max<int64_t>(1 << 24, 128 * ncols + 1024);
        DMS_ALLOC(P.d1_pool, 4 * pool_cap);
        uint8_t *ovf = P.d1_ovf.as<uint8_t>();
        DMS_CUDA(cudaMemsetAsync(ovf, 0, ncols, c.s));
        DMS_CUDA(cudaMemsetAsync(&c.st->pool_top, 0, sizeof(unsigned long long), c.s));
        // first pass: small per-thread scratch that stays in L2
        int hcap = P.tune[DMS_TUNE_TRACE_HEAP], hashcap = hash_cap_for(hcap), rcap = hcap;
        const int tb = P.tune[DMS_TUNE_TRACE_BLOCK];
        int64_t nthreads = (int64_t)152 * P.tune[DMS_TUNE_TRACE_PER_SM];
        if (ncols < nthreads) nthreads = (ncols + tb - 1) / tb * tb;
        size_t per = (size_t)hcap * sizeof(HeapEnt) + (size_t)hashcap * sizeof(HashEnt) +
                     (size_t)rcap * 8;
        DMS_ALLOC(P.d1_scratch, per * nthreads);
        HeapEnt *heap = P.d1_scratch.as<HeapEnt>();
        HashEnt *hash = (HashEnt *)(heap + (size_t)hcap * nthreads);
        int32_t *rows = (int32_t *)(hash + (size_t)hashcap * nthreads);
        DMS_CUDA(cudaMemsetAsync(hash, 0xFF, (size_t)hashcap * nthreads * sizeof(HashEnt), c.s));
        KEV(18);
        auto dbg_p1 = std::chrono::steady_clock::now();
        // columns in vertex-id order: the walks of a warp share the records they read
        const int32_t *corder = nullptr;
        DMS_TRY(order_by_vertex(c, P.c_vert[2].as<int32_t>(), P.d1_colmap.as<int32_t>(), ncols, 1,
                                &corder));
        DMS_CUDA(cudaMemsetAsync(&c.st->trace_next, 0, sizeof(unsigned long long), c.s));
        k_d1_trace<T, B><<<(unsigned)(nthreads / tb), tb, 0, c.s>>>(
            values, geo, P.flags.as<uint8_t>(), P.grad.as<GradRec>(),
            P.vcrit.as<unsigned long long>(), P.c_vert[2].as<int32_t>(), P.c_loc[2].as<uint8_t>(),
            P.d1_colmap.as<int32_t>(), corder, ncols, heap, hash, rows, hcap, hashcap, rcap, 0,
            P.d1_pool.as<int32_t>(), pool_cap, P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(),
            ovf, &c.st->trace_next, P.dense_grad ? 1 : 0, P.generators, c.st);
        c.launches++;
        DMS_CUDA(cudaGetLastError());
        // columns whose trace outgrew the scratch run again with 16x more; the
        // list of them is compacted on the device (flag, scan, scatter), the
        // host reads only its length
        DMS_ALLOC(P.flag_a, 4 * ncols + 4);
        DMS_ALLOC(P.flag_b, 4 * ncols + 4);
        int32_t *f32 = P.flag_a.as<int32_t>(), *fpos = P.flag_b.as<int32_t>();
        DMS_LAUNCH(ncols, 256, k_flags_of, (const int32_t *)nullptr, ncols, ovf, f32);
        DMS_TRY(scan(c, f32, fpos, ncols, &c.st->total[3]));
        DMS_TRY(sync_status(c));
        int64_t ntodo = c.hst->total[3];
        P.d1_overflow = ntodo;
        DMS_ALLOC(P.d1_todo, 8 * ntodo + 8);   // two lists: this pass's and the next's
        int32_t *todo = P.d1_todo.as<int32_t>(), *todo_next = todo + ntodo;
        DMS_LAUNCH(ncols, 256, k_compact_list, (const int32_t *)nullptr, f32, fpos, ncols, todo);
        auto dbg_t0 = std::chrono::steady_clock::now();
        if (getenv("DMS_DEBUG")) {
            fprintf(stderr, "d1 trace pass 1: %lld columns, %lld overflow, pool %llu, %.3f ms\n",
                    (long long)ncols, (long long)ntodo, c.hst->pool_top,
                    std::chrono::duration<double, std::milli>(dbg_t0 - dbg_p1).count());
        }
        int32_t gen = (int32_t)ncols;
        while (ntodo > 0) {
            hcap *= 16; hashcap *= 16; rcap *= 16;
            if (hashcap > (1 << 24)) return DMS_ERR_CAPACITY;
            per = (size_t)hcap * sizeof(HeapEnt) + (size_t)hashcap * sizeof(HashEnt) +
                  (size_t)rcap * 8;
            int64_t nt = std::min<int64_t>(ntodo,
                                           std::max<int64_t>(32, ((int64_t)4 << 30) / (int64_t)per));
            nt = (nt + 31) / 32 * 32;
            DMS_ALLOC(P.d1_scratch, per * nt);
            heap = P.d1_scratch.as<HeapEnt>();
            hash = (HashEnt *)(heap + (size_t)hcap * nt);
            rows = (int32_t *)(hash + (size_t)hashcap * nt);
            DMS_CUDA(cudaMemsetAsync(hash, 0xFF, (size_t)hashcap * nt * sizeof(HashEnt), c.s));
            DMS_CUDA(cudaMemsetAsync(&c.st->trace_next, 0, sizeof(unsigned long long), c.s));
            k_d1_trace<T, B><<<(unsigned)(nt / 32), 32, 0, c.s>>>(
                values, geo, P.flags.as<uint8_t>(), P.grad.as<GradRec>(),
                P.vcrit.as<unsigned long long>(), P.c_vert[2].as<int32_t>(), P.c_loc[2].as<uint8_t>(), P.d1_colmap.as<int32_t>(), todo, ntodo, heap, hash,
                rows, hcap, hashcap, rcap, gen, P.d1_pool.as<int32_t>(), pool_cap,
                P.d1_start.as<int64_t>(), P.d1_len.as<int32_t>(), ovf, &c.st->trace_next,
                P.dense_grad ? 1 : 0, P.generators, c.st);
            c.launches++;
            DMS_CUDA(cudaGetLastError());
            gen += (int32_t)ncols;
            DMS_LAUNCH(ntodo, 256, k_flags_of, todo, ntodo, ovf, f32);
            DMS_TRY(scan(c, f32, fpos, ntodo, &c.st->total[3]));
            DMS_TRY(sync_status(c));
            const int64_t nnext = c.hst->total[3];
            DMS_LAUNCH(ntodo, 256, k_compact_list, todo, f32, fpos, ntodo, todo_next);
            std::swap(todo, todo_next);
            ntodo = nnext;
        }
        if (getenv("DMS_DEBUG"))
            fprintf(stderr, "d1 trace retries: %.3f ms\n",
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                              dbg_t0).count());
        P.trace_toggles = (int64_t)c.hst->trace_work[0];   // read by the last status sync
        P.trace_expansions = (int64_t)c.hst->trace_work[1];
        KEV(19);
        KEV(20);
        DMS_TRY(reduce_d1(c, ncols, n1, is_row));
        if constexpr (!B) {
            if (P.generators) DMS_TRY(generator_records(c, ncols));
        }
        KEV(21);
    }
    cudaEventRecord(ev[6], c.s);
    c.nv.next("dms/output");
    KEV(22);

    // ---- output: per dimension, finite pairs (ordered by the simplex that
    // indexes them) then the infinite classes
    OutArgs a;
    a.vc = P.vc.as<int32_t>();
    a.v0 = P.c_vert[0].as<int32_t>();
    a.v1 = P.c_vert[1].as<int32_t>(); a.l1 = P.c_loc[1].as<uint8_t>();
    a.v2 = P.c_vert[2].as<int32_t>(); a.l2 = P.c_loc[2].as<uint8_t>();
    a.v3 = P.c_vert[3].as<int32_t>(); a.l3 = P.c_loc[3].as<uint8_t>();
    a.young0 = young0; a.young2 = young2; a.died0 = died0; a.died3 = died3;
    a.colmap = P.d1_colmap.as<int32_t>();
    a.d1_row = P.d1_row.as<int32_t>(); a.row_paired = P.d1_rowpaired.as<uint8_t>();
    a.is_row = is_row; a.is_col = is_col;
    // parts: 0 D0 finite (over C1), 1 D0 infinite (C0), 2 D1 finite (columns),
    // 3 D1 infinite (C1), 4 D2 finite (C2), 5 D2 infinite (columns), 6 D3 infinite (C3)
    const int64_t part_n[7] = {n1, n0, ncols, n1, n2, ncols, n3};
    const int part_dim[7] = {0, 0, 1, 1, 2, 2, 3};
    int64_t foff[8] = {0};
    for (int q = 0; q < 7; q++) foff[q + 1] = foff[q] + part_n[q] + 1;
    DMS_ALLOC(P.flag_a, 4 * foff[7] + 4);
    DMS_ALLOC(P.flag_b, 4 * foff[7] + 4);
    int32_t *fl = P.flag_a.as<int32_t>(), *ps = P.flag_b.as<int32_t>();
    for (int q = 0; q < 7; q++) {
        if (q == 1)
            DMS_LAUNCH(part_n[q], 256, k_flag_min, part_n[q], died0, fl + foff[q]);
        else
            DMS_LAUNCH(part_n[q], 256, k_flag, q, a, part_n[q], fl + foff[q]);
        DMS_TRY(scan(c, fl + foff[q], ps + foff[q], part_n[q], &c.st->parts[q]));
    }
    DMS_TRY(sync_status(c));
    int64_t cntp[7];
    for (int q = 0; q < 7; q++) cntp[q] = c.hst->parts[q];
    // rows per output list: the D2 list ends with the infinite classes of
    // dimension 3 (maxima left unpaired, only without the virtual maximum)
    const int64_t list_rows[3] = {cntp[0] + cntp[1], cntp[2] + cntp[3],
                                  cntp[4] + cntp[5] + cntp[6]};
    for (int d = 0; d < 3; d++) DMS_ALLOC(P.out_pairs[d], sizeof(dms_pair) * (list_rows[d] + 1));
    if constexpr (B) {
        for (int d = 0; d < 3; d++) DMS_ALLOC(P.out_field[d], 4 * (list_rows[d] + 1));
    }
    for (int q = 0; q < 7; q++) {
        const int d = part_dim[q] < 3 ? part_dim[q] : 2;
        const int64_t off = q == 6 ? cntp[4] + cntp[5] : (q & 1) ? cntp[q - 1] : 0;
        DMS_LAUNCH(part_n[q], 128, (k_write<T, B>), q, a, values, geo, part_n[q], fl + foff[q],
                   ps + foff[q], off, P.vrank.as<int32_t>(), c.hst->maxkey,
                   P.fmax_field.as<unsigned long long>(), P.out_field[d].as<int32_t>(),
                   P.out_pairs[d].as<dms_pair>());
    }
    if constexpr (B) {
        // group each dimension's pairs by field, keeping their order inside a field
        for (int d = 0; d < 3; d++) DMS_TRY(group_by_field(c, d, list_rows[d]));
    }
    P.n_pairs[0] = cntp[0]; P.n_pairs[1] = cntp[2]; P.n_pairs[2] = cntp[4];
    P.n_ess[0] = cntp[1]; P.n_ess[1] = cntp[3]; P.n_ess[2] = cntp[5]; P.n_ess[3] = cntp[6];
    KEV(23);
    cudaEventRecord(ev[7], c.s);
    DMS_TRY(sync_status(c));
    return DMS_OK;
}

}  // namespace

// ------------------------------------------------------------------------
// Classification without allocation (dms_classify_static).
//
// Its scratch is a file-scope device array of fixed size, sized for grids of
// up to kStaticMaxVertices vertices: the per-tile counts and offsets of the
// ordered compaction, the partial sums of their scan and a status block.
// Every device that loads this library holds the array until the process
// exits.  Host code cannot use the array's name as a device address, so its
// address is looked up once per device with cudaGetSymbolAddress and passed
// to the kernels.
constexpr int64_t kStaticMaxVertices = (int64_t)1 << 28;
constexpr int64_t kStaticTiles = kStaticMaxVertices / kClsTile;           // 131072
constexpr int64_t kStaticParts = (kStaticTiles + kScanTile - 1) / kScanTile;  // 64
struct StaticScratch {
    int32_t tile_cnt[kStaticTiles];
    int32_t tile_off[kStaticTiles];
    int32_t part[kStaticParts];
    int32_t part_off[kStaticParts];
    DevStatus status;
};
static __device__ __align__(256) StaticScratch g_static_scratch;

namespace {
std::mutex g_static_mutex;
StaticScratch *g_static_ptr[64] = {nullptr};   // per device, from cudaGetSymbolAddress

// Set-up on first use on a device (that device current): the star tables and
// the address of the scratch array.
dms_status static_setup(int device, StaticScratch **out) {
    if (device < 0 || device >= 64) return DMS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[device]) {
        dms_status s = ensure_tables(device);
        if (s != DMS_OK) return s;
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            fprintf(stderr, "libdms: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
            return DMS_ERR_CUDA;
        }
        g_static_ptr[device] = (StaticScratch *)ptr;
    }
    *out = g_static_ptr[device];
    return DMS_OK;
}

template <typename T>
dms_status classify_static(const T *values, GridParams g, uint8_t *flags, int32_t *critical,
                           int64_t cap, int64_t *n_critical, cudaStream_t s, StaticScratch *scr) {
    const ClsTiling ct = cls_tiling<T>(g, values);
    const int64_t ntiles = ct.ntiles;
    if (ntiles > kStaticTiles) return DMS_ERR_INVALID_ARG;
    DevStatus *st = &scr->status;
    DMS_CUDA(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));   // starts at zero every call
    k_classify2<T><<<(unsigned)ntiles, kClsThreads, 0, s>>>(values, g, ct.rows_per_block,
                                                           ct.runs_per_row, ct.aligned, flags,
                                                           scr->tile_cnt, st);
    DMS_CUDA(cudaGetLastError());
    if (ntiles <= kScanTile) {
        k_scan_apply<<<1, kScanThreads, 0, s>>>(scr->tile_cnt, scr->tile_off, ntiles, nullptr,
                                                &st->total[0]);
    } else {
        const int64_t m = (ntiles + kScanTile - 1) / kScanTile;
        k_scan_partial<<<(unsigned)m, kScanThreads, 0, s>>>(scr->tile_cnt, ntiles, scr->part);
        k_scan_apply<<<1, kScanThreads, 0, s>>>(scr->part, scr->part_off, m, nullptr, nullptr);
        k_scan_apply<<<(unsigned)m, kScanThreads, 0, s>>>(scr->tile_cnt, scr->tile_off, ntiles,
                                                          scr->part_off, &st->total[0]);
    }
    DMS_CUDA(cudaGetLastError());
    long long total = 0;
    uint32_t err = 0;
    DMS_CUDA(cudaMemcpyAsync(&total, &st->total[0], sizeof total, cudaMemcpyDeviceToHost, s));
    DMS_CUDA(cudaMemcpyAsync(&err, &st->err, sizeof err, cudaMemcpyDeviceToHost, s));
    DMS_CUDA(cudaStreamSynchronize(s));
    if (err & kErrNan) return DMS_ERR_NAN;
    *n_critical = total;
    if (total > cap) return DMS_ERR_CAPACITY;
    k_compact2<<<(unsigned)ntiles, kClsThreads, 0, s>>>(flags, g.n, ct.tile, scr->tile_off,
                                                       critical);
    DMS_CUDA(cudaGetLastError());
    DMS_CUDA(cudaStreamSynchronize(s));
    return DMS_OK;
}
}  // namespace

dms_status Pipeline::init(int64_t nx_, int64_t ny_, int64_t nz_, dms_dtype dt,
                          const dms_options *o) {
    if (nx_ < 1 || ny_ < 1 || nz_ < 1 || nx_ > (1 << 30) || ny_ > (1 << 30) || nz_ > (1 << 30))
        return DMS_ERR_INVALID_ARG;
    if (nx_ * ny_ >= ((int64_t)1 << 31) || nx_ * ny_ * nz_ >= ((int64_t)1 << 31))
        return DMS_ERR_INVALID_ARG;
    if (dt != DMS_U16 && dt != DMS_F32 && dt != DMS_F64) return DMS_ERR_INVALID_ARG;
    if (o && o->virtual_max != 0 && o->virtual_max != 1) return DMS_ERR_INVALID_ARG;
    if (o && o->max_iters < 0) return DMS_ERR_INVALID_ARG;
    if (o && (o->generators != 0 && o->generators != 1)) return DMS_ERR_INVALID_ARG;
    // generators: the traced reduction (mode 0 or 1); passive entries hold
    // edge ids in int32
    if (o && o->generators &&
        (o->d1_mode > 1 || 7 * nx_ * ny_ * nz_ >= ((int64_t)1 << 31)))
        return DMS_ERR_INVALID_ARG;
    if (o && (o->d1_mode < 0 || o->d1_mode > 3)) return DMS_ERR_INVALID_ARG;
    nx = nx_; ny = ny_; nz = nz_; n = nx * ny * nz; dtype = dt;
    return init_common(o);
}

// The grid of one field of a batch (or of the single grid) at offset `off`.
static GridParams grid_params(int64_t nx, int64_t ny, int64_t nz, int64_t off) {
    GridParams g;
    g.nx = (int32_t)nx; g.ny = (int32_t)ny; g.nz = (int32_t)nz; g.n = nx * ny * nz; g.off = off;
    for (int l = 0; l < kLinks; l++) {
        const int o = l % 7 + 1, sg = l < 7 ? 1 : -1;
        g.dlin[l] = sg * ((o & 1) + (int32_t)nx * (((o >> 1) & 1) + (int32_t)ny * ((o >> 2) & 1)));
    }
    return g;
}

// The shapes of a batch are valid: 1..65535 fields (the field index is 16
// bits), each 1 <= n <= 2^30 per axis, every count below 2^31.
static bool batch_shapes_ok(int64_t nf_, const int64_t *shp) {
    if (nf_ < 1 || nf_ > 65535 || !shp) return false;
    int64_t total = 0;
    for (int64_t f = 0; f < nf_; f++) {
        const int64_t a = shp[3 * f], b = shp[3 * f + 1], c = shp[3 * f + 2];
        if (a < 1 || b < 1 || c < 1 || a > (1 << 30) || b > (1 << 30) || c > (1 << 30) ||
            a * b >= ((int64_t)1 << 31) || a * b * c >= ((int64_t)1 << 31))
            return false;
        total += a * b * c;
        if (total >= ((int64_t)1 << 31)) return false;
    }
    return true;
}

dms_status Pipeline::init_batch(int64_t nf_, const int64_t *shp, dms_dtype dt,
                                const dms_options *o) {
    if (dt != DMS_U16 && dt != DMS_F32 && dt != DMS_F64) return DMS_ERR_INVALID_ARG;
    if (!batch_shapes_ok(nf_, shp)) return DMS_ERR_INVALID_ARG;   // before any CUDA call
    if (o && ((o->virtual_max != 0 && o->virtual_max != 1) || o->max_iters < 0 ||
              o->d1_mode < 0 || o->d1_mode > 3 || o->generators != 0))
        return DMS_ERR_INVALID_ARG;   // generators: single grids only
    batch = true;
    dtype = dt;
    dms_status s = init_common(o);
    if (s != DMS_OK) return s;
    return set_batch(nf_, shp);
}

// The layout of a batch: per-field grids and offsets, the field of every id.
// Device buffers only grow, so a handle can be re-targeted to other batches.
dms_status Pipeline::set_batch(int64_t nf_, const int64_t *shp) {
    if (!batch) return DMS_ERR_INVALID_ARG;
    if (!batch_shapes_ok(nf_, shp)) return DMS_ERR_INVALID_ARG;
    std::vector<int64_t> off(nf_ + 1, 0);
    std::vector<GridParams> gp(nf_);
    for (int64_t f = 0; f < nf_; f++) {
        const int64_t a = shp[3 * f], b = shp[3 * f + 1], c = shp[3 * f + 2];
        if (a < 1 || b < 1 || c < 1 || a > (1 << 30) || b > (1 << 30) || c > (1 << 30) ||
            a * b >= ((int64_t)1 << 31) || a * b * c >= ((int64_t)1 << 31))
            return DMS_ERR_INVALID_ARG;
        gp[f] = grid_params(a, b, c, off[f]);
        off[f + 1] = off[f] + a * b * c;
        if (off[f + 1] >= ((int64_t)1 << 31)) return DMS_ERR_INVALID_ARG;
    }
    const int64_t n2 = off[nf_];
    const int64_t ntiles = (n2 + kClsTile - 1) / kClsTile;
    if (!flags.ensure(n2) || !vrank.ensure(4 * n2) || !grad.ensure(sizeof(GradRec) * n2) ||
        !tile_cnt.ensure(4 * ntiles) || !tile_off.ensure(4 * ntiles) ||
        !fields_dev.ensure(sizeof(GridParams) * nf_) || !field_of.ensure(2 * n2 + 2) ||
        !field_off_dev.ensure(8 * (nf_ + 1)) || !fmax_field.ensure(8 * nf_))
        return DMS_ERR_OOM;
    has_result = false;
    nf = nf_;
    shapes.assign(shp, shp + 3 * nf_);
    field_off = off;
    n = n2;
    nx = n; ny = 1; nz = 1;   // the id space (the geometry comes from the fields)
    if (cudaMemcpy(fields_dev.p, gp.data(), sizeof(GridParams) * nf_, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(field_off_dev.p, field_off.data(), 8 * (nf_ + 1), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return DMS_ERR_CUDA;
    k_field_of<<<blocks_for(n, 256), 256>>>(field_off_dev.as<int64_t>(), (int)nf_, n,
                                            field_of.as<uint16_t>());
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return DMS_ERR_CUDA;
    return DMS_OK;
}

dms_status Pipeline::init_common(const dms_options *o) {
    virtual_max = o ? o->virtual_max : 1;
    generators = o ? o->generators : 0;
    max_iters = o ? o->max_iters : 0;
    d1_mode = o ? o->d1_mode : 0;
    if (cudaGetDevice(&device) != cudaSuccess) return DMS_ERR_CUDA;
    dms_status s = ensure_tables(device);
    if (s != DMS_OK) return s;
    const int64_t ntiles = (n + kClsTile - 1) / kClsTile;
    if (!flags.ensure(n) || !vrank.ensure(4 * n) || !grad.ensure(sizeof(GradRec) * n) || !tile_cnt.ensure(4 * ntiles) ||
        !tile_off.ensure(4 * ntiles) || !dstat.ensure(sizeof(DevStatus)))
        return DMS_ERR_OOM;
    if (cudaMallocHost(&hstat, sizeof(DevStatus)) != cudaSuccess) {
        hstat = nullptr;
        return DMS_ERR_OOM;
    }
    for (int i = 0; i < 24; i++)
        if (cudaEventCreate((cudaEvent_t *)&kev[i]) != cudaSuccess) return DMS_ERR_CUDA;
    for (int i = 0; i < 8; i++)
        if (cudaEventCreate((cudaEvent_t *)&sev[i]) != cudaSuccess) return DMS_ERR_CUDA;
    if (cudaStreamCreateWithFlags((cudaStream_t *)&s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags((cudaEvent_t *)&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags((cudaEvent_t *)&ev_join, cudaEventDisableTiming) != cudaSuccess)
        return DMS_ERR_CUDA;
    return DMS_OK;
}

dms_status Pipeline::reshape(int64_t nx_, int64_t ny_, int64_t nz_) {
    if (batch) return DMS_ERR_INVALID_ARG;
    if (nx_ < 1 || ny_ < 1 || nz_ < 1 || nx_ > (1 << 30) || ny_ > (1 << 30) || nz_ > (1 << 30))
        return DMS_ERR_INVALID_ARG;
    if (nx_ * ny_ >= ((int64_t)1 << 31) || nx_ * ny_ * nz_ >= ((int64_t)1 << 31))
        return DMS_ERR_INVALID_ARG;
    const int64_t n2 = nx_ * ny_ * nz_;
    if (generators && 7 * n2 >= ((int64_t)1 << 31)) return DMS_ERR_INVALID_ARG;
    if (!flags.ensure(n2) || !vrank.ensure(4 * n2) || !grad.ensure(sizeof(GradRec) * n2))
        return DMS_ERR_OOM;
    nx = nx_; ny = ny_; nz = nz_; n = n2;
    has_result = false;
    return DMS_OK;
}

// Every device buffer of the handle.
std::vector<DevBuf *> Pipeline::buffers() {
    std::vector<DevBuf *> all = {&d1_row, &d1_rowpaired, &d1_rowpos, &d1_rowmap, &d1_cocnt, &d1_costart,
                     &d1_cofill, &d1_act, &d1_next, &d1_re, &d1_stamp, &d1_work, &grad, &values_dev, &flags,    &vrank,     &tile_cnt,  &tile_off,   &vc,
                     &vc_tmp,     &keys,     &keys_tmp,  &recs,      &arc_a,      &arc_b,
                     &dc_keys,    &dc_par,   &dc_lab,    &bv_node,   &bv_msf,    &bv_arcs,
                     &young,     &died,       &rowcol,
                     &flag_a,     &flag_b,   &d1_colmap, &d1_start,  &d1_len,     &d1_owner,
                     &d1_ovf,     &d1_pool,  &d1_scratch, &d1_todo,  &scan_tmp,   &scan_tmp2, &arc2_a, &arc2_b, &vcrit, &gen_out, &dstat,
                     &d1_astamp, &lz_small.buf, &lz_big.buf, &d1_rowcol,
                     &fields_dev, &field_of, &field_off_dev, &fmax_field, &bt_k[0], &bt_k[1],
                     &bt_v[0], &bt_v[1], &bt_h[0], &bt_h[1], &bt_cnt, &out_tmp, &bx_buf[0],
                     &bx_buf[1], &d1_info, &d1_queue, &d1_aq, &ord_k[0], &ord_k[1], &ord_k[2],
                     &ord_k[3], &ord_v[0], &ord_v[1], &ord_v[2], &ord_v[3], &ord_h[0], &ord_h[1],
                     &pls_ranks};
    for (int d = 0; d < 4; d++)
        for (DevBuf *b : {&cnt[d], &base[d], &c_vert[d], &c_loc[d]}) all.push_back(b);
    for (int d = 0; d < 3; d++)
        for (DevBuf *b : {&out_pairs[d], &out_field[d], &batch_pofs[d]}) all.push_back(b);
    return all;
}

int64_t Pipeline::device_bytes() {
    int64_t total = 0;
    for (DevBuf *b : buffers()) total += (int64_t)b->bytes;
    return total;
}

void Pipeline::destroy() {
    for (DevBuf *b : buffers()) b->release();
    if (hstat) cudaFreeHost(hstat);
    hstat = nullptr;
    for (int i = 0; i < 24; i++) if (kev[i]) cudaEventDestroy((cudaEvent_t)kev[i]);
    for (int i = 0; i < 8; i++) if (sev[i]) cudaEventDestroy((cudaEvent_t)sev[i]);
    for (int i = 0; i < 24; i++) kev[i] = nullptr;
    for (int i = 0; i < 8; i++) sev[i] = nullptr;
    if (ev_fork) cudaEventDestroy((cudaEvent_t)ev_fork);
    if (ev_join) cudaEventDestroy((cudaEvent_t)ev_join);
    if (s2) cudaStreamDestroy((cudaStream_t)s2);
    ev_fork = ev_join = s2 = nullptr;
}

dms_status Pipeline::compute(const void *values, int on_host, void *stream) {
    has_result = false;
    gen_words = 0;
    if (!values || (on_host != 0 && on_host != 1)) return DMS_ERR_INVALID_ARG;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return DMS_ERR_CUDA;
    if (cur != device && cudaSetDevice(device) != cudaSuccess) return DMS_ERR_CUDA;
    cudaEvent_t *ev = (cudaEvent_t *)sev, *kv = (cudaEvent_t *)kev;
    Ctx c{*this, (cudaStream_t)stream};
    c.kev = kv;
    c.st = dstat.as<DevStatus>();
    c.hst = (DevStatus *)hstat;
    c.ev = ev;
    c.g = grid_params(nx, ny, nz, 0);
    if (batch) {
        c.bgeo.fields = fields_dev.as<GridParams>();
        c.bgeo.field_of = field_of.as<uint16_t>();
    }
    const size_t esz = dtype == DMS_U16 ? 2 : dtype == DMS_F32 ? 4 : 8;
    dms_status s = DMS_OK;
    cudaEventRecord(ev[0], c.s);
    c.nv.next("dms/h2d");
    const void *dv = values;
    if (on_host) {
        if (!values_dev.ensure(n * esz)) s = DMS_ERR_OOM;
        else if (cudaMemcpyAsync(values_dev.p, values, n * esz, cudaMemcpyHostToDevice, c.s) !=
                 cudaSuccess)
            s = DMS_ERR_CUDA;
        dv = values_dev.p;
    }
    cudaEventRecord(ev[1], c.s);
    c.nv.next("dms/gradient");
    if (s == DMS_OK) {
        if (batch) {
            if (dtype == DMS_U16) s = run<uint16_t, true>(c, (const uint16_t *)dv);
            else if (dtype == DMS_F32) s = run<float, true>(c, (const float *)dv);
            else s = run<double, true>(c, (const double *)dv);
        } else {
            if (dtype == DMS_U16) s = run<uint16_t, false>(c, (const uint16_t *)dv);
            else if (dtype == DMS_F32) s = run<float, false>(c, (const float *)dv);
            else s = run<double, false>(c, (const double *)dv);
        }
    }
    launches = c.launches;
    if (s == DMS_OK) {
        cudaEventSynchronize(ev[7]);
        float t = 0;
        // 0 start, 1 after H2D, 2 gradient, 3 sort, 4 D0, 5 D2, 6 D1, 7 output
        const int from[8] = {1, 2, 3, 4, 5, 6, 1, 0}, to[8] = {2, 3, 4, 5, 6, 7, 7, 1};
        for (int k = 0; k < 8; k++) {
            cudaEventElapsedTime(&t, ev[from[k]], ev[to[k]]);
            stage_ms[k] = t;
        }
        if (!on_host) stage_ms[7] = 0.f;
        for (int k = 0; k < 12; k++) {
            cudaEventElapsedTime(&t, kv[2 * k], kv[2 * k + 1]);
            kernel_ms[k] = t;
        }
        has_result = true;
        result_id++;
    } else {
        cudaStreamSynchronize(c.s);
        if (s2) cudaStreamSynchronize((cudaStream_t)s2);
        cudaGetLastError();
    }
    return s;
}

dms_status Pipeline::backward(int dim, uint64_t rid, const double *gbirth, const double *gdeath,
                              double *grad, void *stream) {
    if (!has_result || rid != result_id) return DMS_ERR_STATE;   // not the caller's pairing
    if (dim < 0 || dim > 2 || !grad) return DMS_ERR_INVALID_ARG;
    const int64_t total = list_rows(dim);
    if (total == 0) return DMS_OK;
    const int64_t *pofs = nullptr, *vofs = nullptr;
    if (batch) {   // per-field pair ranges of this dimension and field offsets
        pofs = batch_pofs[dim].as<int64_t>();
        vofs = field_off_dev.as<int64_t>();
    }
    k_scatter_pair_grads<<<blocks_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
        out_pairs[dim].as<dms_pair>(), total, gbirth, gdeath, grad, pofs, vofs, (int)nf);
    return cudaGetLastError() == cudaSuccess ? DMS_OK : DMS_ERR_CUDA;
}

dms_status Pipeline::fetch_generators(int64_t *out, int64_t cap, int64_t *written) {
    if (!written) return DMS_ERR_INVALID_ARG;
    *written = 0;
    if (!has_result || !generators) return DMS_ERR_STATE;
    *written = gen_words;
    if (gen_words > cap) return DMS_ERR_CAPACITY;
    if (gen_words == 0) return DMS_OK;
    if (!out) return DMS_ERR_INVALID_ARG;
    if (cudaMemcpy(out, gen_out.p, 8 * gen_words, cudaMemcpyDeviceToHost) != cudaSuccess)
        return DMS_ERR_CUDA;
    return DMS_OK;
}

dms_status Pipeline::fetch(int dim, dms_pair *out, int64_t cap, int64_t *written,
                           int out_is_device) {
    if (!written) return DMS_ERR_INVALID_ARG;
    *written = 0;
    if (!has_result) return DMS_ERR_STATE;
    if (dim < 0 || dim > 2) return DMS_ERR_INVALID_ARG;
    const int64_t total = list_rows(dim);
    if (total > cap) return DMS_ERR_CAPACITY;
    if (total == 0) return DMS_OK;
    if (!out) return DMS_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(out, out_pairs[dim].p, sizeof(dms_pair) * total,
                               out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return DMS_ERR_CUDA;
    *written = total;
    return DMS_OK;
}

}  // namespace dms

extern "C" dms_status dms_classify_static(const void *values, dms_dtype dtype, int64_t nx,
                                          int64_t ny, int64_t nz, uint8_t *flags_out,
                                          int32_t *critical_out, int64_t cap,
                                          int64_t *n_critical, void *stream) {
    using namespace dms;
    if (!values || !flags_out || !n_critical || cap < 0 || (cap > 0 && !critical_out))
        return DMS_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || nx > kStaticMaxVertices || ny > kStaticMaxVertices ||
        nz > kStaticMaxVertices || nx * ny > kStaticMaxVertices ||
        nx * ny * nz > kStaticMaxVertices)
        return DMS_ERR_INVALID_ARG;   // beyond the fixed scratch
    if (dtype != DMS_U16 && dtype != DMS_F32 && dtype != DMS_F64) return DMS_ERR_INVALID_ARG;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return DMS_ERR_CUDA;
    StaticScratch *scr = nullptr;
    dms_status st = static_setup(device, &scr);
    if (st != DMS_OK) return st;
    const GridParams g = grid_params(nx, ny, nz, 0);
    *n_critical = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == DMS_U16)
        return classify_static<uint16_t>((const uint16_t *)values, g, flags_out, critical_out, cap,
                                         n_critical, s, scr);
    if (dtype == DMS_F32)
        return classify_static<float>((const float *)values, g, flags_out, critical_out, cap,
                                      n_critical, s, scr);
    return classify_static<double>((const double *)values, g, flags_out, critical_out, cap,
                                   n_critical, s, scr);
}


// The star tables of the kernels, copied to the host (no GPU involved), for
// tests that run the lower-star code on the host.
extern "C" int64_t dms_star_tables(void *out, int64_t bytes) {
    dms::StarTables S;
    if (!dms::build_star_tables(S)) return -1;
    if (out && bytes >= (int64_t)sizeof S) memcpy(out, &S, sizeof S);
    return (int64_t)sizeof S;
}

// The regular-vertex table of the classification (bit m set: lower link mask
// m is PL-regular), copied to the host (no GPU involved), for tests.
extern "C" int64_t dms_regular_table(uint32_t *out, int64_t words) {
    dms::StarTables S;
    if (!dms::build_star_tables(S)) return -1;
    std::vector<uint32_t> lut;
    dms::build_regular_lut(S, lut);
    if (out && words >= (int64_t)lut.size()) memcpy(out, lut.data(), 4 * lut.size());
    return (int64_t)lut.size();
}
