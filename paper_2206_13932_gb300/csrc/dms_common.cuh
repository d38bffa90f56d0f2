// dms_common.cuh -- shared device definitions of libdms: the star of a vertex
// in the Freudenthal triangulation, the vertex order and ProcessLowerStars.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace dms {

// ---------------------------------------------------------------------------
// The star of a vertex x (Sec. 2.1: Freudenthal, 14-vertex neighbourhood).
//
// Link vertex n in [0,14): n < 7 is x + o, n >= 7 is x - o, with offset
// bitmask o = (n % 7) + 1 (bit0 x, bit1 y, bit2 z).  A set of grid points is
// a Freudenthal simplex iff it is a chain of the componentwise order whose
// extent fits in one unit cube; the star holds 14 edges (one per link
// vertex), 36 triangles (link edges) and 24 tetrahedra (link triangles).
// ---------------------------------------------------------------------------
constexpr int kLinks = 14, kTris = 36, kTets = 24;
constexpr uint16_t kAllLinks = 0x3FFF;
constexpr uint64_t kAllTris = (1ull << kTris) - 1;
constexpr uint32_t kAllTets = (1u << kTets) - 1;
constexpr uint8_t kNoDescent = 0xF;   // flags low nibble of a minimum
constexpr uint8_t kFlagCritical = 0x10;
constexpr uint8_t kFlagGradient = 0x20;   // the vertex's GradRec is filled

struct StarTables {
    int8_t dx[kLinks], dy[kLinks], dz[kLinks];
    uint8_t tri_v[kTris][2];          // the two link vertices of a star triangle
    uint8_t tet_v[kTets][3];          // the three link vertices of a star tet
    uint8_t tet_f[kTets][3];          // its three star triangles (faces in the star)
    uint16_t tri_mask[kTris];         // link-vertex mask of a star triangle
    uint16_t tet_mask[kTets];         // link-vertex mask of a star tet
    uint64_t tris_of_link[kLinks];    // star triangles containing link vertex n
    uint32_t tets_of_link[kLinks];    // star tets containing link vertex n
    uint32_t tets_of_tri[kTris];      // star tets containing star triangle s
    int8_t tri_of_pair[kLinks][kLinks];
    int8_t link_of_dc[27];            // (dx+1)+3(dy+1)+9(dz+1) -> link or -1
    int8_t edge_anchor[kLinks], edge_type[kLinks];   // anchor: -1 = x itself
    int8_t tri_anchor[kTris], tri_type[kTris];
    int8_t tet_anchor[kTets], tet_type[kTets];
    uint16_t neg[3], pos[3];          // links with d = -1 / +1 along each axis
};

// Grid constants passed by value to kernels.  A batch lays several grids
// (fields) out one after another in one id space; `off` is the id of a
// field's vertex (0,0,0) (0 for a single grid).
struct GridParams {
    int32_t nx, ny, nz;
    int64_t n;                        // nx*ny*nz (< 2^31)
    int32_t dlin[kLinks];             // linear id offset of each link vertex
    int64_t off;
};

// The grid of a vertex: the only one (B = false), or the field of a batch
// that holds the vertex (B = true: a field index per vertex).
template <bool B> struct Geo;
template <> struct Geo<false> {
    GridParams g0;
    __device__ __forceinline__ const GridParams &at(int64_t) const { return g0; }
};
template <> struct Geo<true> {
    const GridParams *fields;
    const uint16_t *field_of;
    __device__ __forceinline__ int field(int64_t v) const { return field_of[v]; }
    __device__ __forceinline__ const GridParams &at(int64_t v) const {
        return fields[field_of[v]];
    }
};

// ---------------------------------------------------------------------------
// Vertex order (Sec. 2.1): values mapped to unsigned keys that order like the
// numbers (-0.0 = +0.0), ties broken by vertex id.
// ---------------------------------------------------------------------------
template <typename T> struct Key;
template <> struct Key<uint16_t> {
    using K = uint32_t;
    __device__ __forceinline__ static K of(uint16_t v) { return v; }
    __device__ __forceinline__ static bool nan(uint16_t) { return false; }
    __device__ __forceinline__ static uint64_t bits(uint16_t v) { return v; }
};
template <> struct Key<float> {
    using K = uint32_t;
    __device__ __forceinline__ static K of(float f) {
        uint32_t u = __float_as_uint(f);
        if (u == 0x80000000u) u = 0;
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
    __device__ __forceinline__ static bool nan(float f) {
        return (__float_as_uint(f) & 0x7fffffffu) > 0x7f800000u;
    }
    __device__ __forceinline__ static uint64_t bits(float f) { return __float_as_uint(f); }
};
template <> struct Key<double> {
    using K = uint64_t;
    __device__ __forceinline__ static K of(double d) {
        uint64_t u = (uint64_t)__double_as_longlong(d);
        if (u == 0x8000000000000000ull) u = 0;
        return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
    }
    __device__ __forceinline__ static bool nan(double d) {
        return ((uint64_t)__double_as_longlong(d) & 0x7fffffffffffffffull) >
               0x7ff0000000000000ull;
    }
    __device__ __forceinline__ static uint64_t bits(double d) {
        return (uint64_t)__double_as_longlong(d);
    }
};

// Present link vertices of vertex (cx, cy, cz) (those inside the grid).
__device__ __forceinline__ uint16_t present_links(const StarTables &S, const GridParams &g,
                                                  int cx, int cy, int cz) {
    uint16_t m = kAllLinks;
    if (cx == 0) m &= ~S.neg[0];
    if (cx == g.nx - 1) m &= ~S.pos[0];
    if (cy == 0) m &= ~S.neg[1];
    if (cy == g.ny - 1) m &= ~S.pos[1];
    if (cz == 0) m &= ~S.neg[2];
    if (cz == g.nz - 1) m &= ~S.pos[2];
    return m;
}

__device__ __forceinline__ void coords(const GridParams &g, int64_t v, int &cx, int &cy,
                                       int &cz) {
    int32_t vi = (int32_t)(v - g.off);
    int32_t row = vi / g.nx;
    cx = vi - row * g.nx;
    cz = row / g.ny;
    cy = row - cz * g.ny;
}

// The star of vertex v with the vertex order: lower mask (the link vertices
// below v) and the rank of each lower link vertex among them (0 = lowest).
struct StarView {
    uint16_t present, lower;
    uint8_t rank[kLinks];   // valid for lower links
    uint8_t descent;        // lowest lower link or kNoDescent
};

template <typename T>
__device__ __forceinline__ void load_star(const StarTables &S, const GridParams &g,
                                          const T *__restrict__ values, int64_t v,
                                          StarView &sv) {
    using K = typename Key<T>::K;
    int cx, cy, cz;
    coords(g, v, cx, cy, cz);
    sv.present = present_links(S, g, cx, cy, cz);
    const K kv = Key<T>::of(values[v]);
    K kn[kLinks];
    uint16_t lower = 0;
#pragma unroll
    for (int n = 0; n < kLinks; n++) {
        kn[n] = 0;
        if (sv.present >> n & 1) {
            kn[n] = Key<T>::of(values[v + g.dlin[n]]);
            // a neighbour is lower if its value is smaller, or equal with a
            // smaller id (a negative offset)
            bool lo = kn[n] < kv || (kn[n] == kv && n >= 7);
            lower |= (uint16_t)lo << n;
        }
    }
    sv.lower = lower;
    sv.descent = kNoDescent;
    if constexpr (sizeof(K) <= 4) {
        // Ties are broken by vertex id, and among the links that are present
        // the id order is fixed: the negative offsets -7..-1 (links 13..7),
        // then +1..+7 (links 0..6).  So (key, position in that order) packs
        // into one integer, and one comparison per pair of links fills the
        // masks below[n] of the links ordered before link n.
        using P = typename std::conditional<sizeof(T) <= 2, uint32_t, unsigned long long>::type;
        P pk[kLinks];
#pragma unroll
        for (int n = 0; n < kLinks; n++)
            pk[n] = ((P)kn[n] << 4) | (P)(n < 7 ? 7 + n : 13 - n);
        uint16_t below[kLinks];
#pragma unroll
        for (int n = 0; n < kLinks; n++) below[n] = 0;
#pragma unroll
        for (int n = 1; n < kLinks; n++)
#pragma unroll
            for (int m = 0; m < n; m++) {
                const bool mb = pk[m] < pk[n];
                below[n] |= (uint16_t)mb << m;
                below[m] |= (uint16_t)!mb << n;
            }
#pragma unroll
        for (int n = 0; n < kLinks; n++) {
            const uint8_t r = (uint8_t)__popc(below[n] & lower);
            if ((lower >> n & 1) && r == 0) sv.descent = (uint8_t)n;
            sv.rank[n] = (lower >> n & 1) ? r : 0;
        }
    } else {
#pragma unroll
        for (int n = 0; n < kLinks; n++) {
            uint8_t r = 0;
            if (lower >> n & 1) {
#pragma unroll
                for (int m = 0; m < kLinks; m++)
                    if ((lower >> m & 1) && m != n &&
                        (kn[m] < kn[n] || (kn[m] == kn[n] && g.dlin[m] < g.dlin[n])))
                        r++;
                if (r == 0) sv.descent = (uint8_t)n;
            }
            sv.rank[n] = r;
        }
    }
}

// ---------------------------------------------------------------------------
// ProcessLowerStars (the expansion gradient of Robins et al., which Alg. 2
// applies; the paper cites it without pseudo-code).  Inside the lower star
// of a vertex x every cell is keyed by G = the ranks of its other vertices in
// decreasing order (the lexicographic key restricted to one lower star); a
// face precedes its cofaces.
//   - no lower edge: x is a minimum;
//   - else x is paired with its lowest edge; the other edges wait in PQzero;
//     cofaces with exactly one unclassified face in the lower star go to
//     PQone;
//   - PQone is drained by smallest G: a cell with no unclassified face moves
//     to PQzero, otherwise it is paired with its unique unclassified face;
//     then the smallest cell of PQzero becomes critical.
// Faces outside the lower star never count as unclassified; a cell popped
// after it was classified is skipped.
// ---------------------------------------------------------------------------
struct PLSResult {
    uint16_t crit_e;       // critical star edges
    uint32_t crit_h;       // critical star tets
    uint64_t crit_t;       // critical star triangles
    bool is_min;
};

// The gradient of one lower star, packed (40 bytes):
//   tet h of the lower star  -> the star triangle it is paired with (6 bits,
//                               kNone if critical or not in the lower star)
//   edge n of the lower star -> the star triangle it is paired with, kHead
//                               if it is paired with the vertex, kNone if
//                               critical or not lower; plus the order (4 bits)
//                               in which the lower star's edges were
//                               classified.
// Layout: w[0] tets 0-9, w[1] tets 10-19, w[2] tets 20-23 (bits 0-23) and
// edge pairs 0-5 (bits 24-59), w[3] edge pairs 6-13, w[4] edge orders 0-13,
// w[5] the 4-bit rank of each lower link vertex (0xF: not lower).
constexpr int kNone = 63, kHead = 62;
struct __align__(16) GradRec {
    uint64_t w[6];
};
__device__ __forceinline__ int grad_rank(const GradRec &g, int n) {
    return (int)((g.w[5] >> (4 * n)) & 15);
}

__device__ __forceinline__ int grad_tet_pair(const GradRec &g, int h) {
    int word = h < 10 ? 0 : h < 20 ? 1 : 2;
    int bit = 6 * (h - 10 * word);
    return (int)((g.w[word] >> bit) & 63);
}
__device__ __forceinline__ int grad_edge_pair(const GradRec &g, int n) {
    if (n < 6) return (int)((g.w[2] >> (24 + 6 * n)) & 63);
    return (int)((g.w[3] >> (6 * (n - 6))) & 63);
}
__device__ __forceinline__ int grad_edge_order(const GradRec &g, int n) {
    return (int)((g.w[4] >> (4 * n)) & 15);
}

__device__ __forceinline__ uint16_t code_edge(const uint8_t *r, int n) {
    return (uint16_t)((r[n] + 1) << 8);
}
__device__ __forceinline__ uint16_t code_tri(const StarTables &S, const uint8_t *r, int s) {
    int a = r[S.tri_v[s][0]], b = r[S.tri_v[s][1]];
    int hi = a > b ? a : b, lo = a > b ? b : a;
    return (uint16_t)(((hi + 1) << 8) | ((lo + 1) << 4));
}
__device__ __forceinline__ uint16_t code_tet(const StarTables &S, const uint8_t *r, int h) {
    int a = r[S.tet_v[h][0]], b = r[S.tet_v[h][1]], c = r[S.tet_v[h][2]];
    int t;
    if (a < b) { t = a; a = b; b = t; }
    if (b < c) { t = b; b = c; c = t; }
    if (a < b) { t = a; a = b; b = t; }
    return (uint16_t)(((a + 1) << 8) | ((b + 1) << 4) | (c + 1));
}

// With G non-null the whole pairing of the lower star is packed into *G.
__device__ inline void pls(const StarTables &S, uint16_t L, const uint8_t *rank, PLSResult &R,
                           GradRec *G) {
    R.crit_e = 0; R.crit_h = 0; R.crit_t = 0; R.is_min = false;
    uint8_t tpair[kTets], epair[kLinks], eord[kLinks];
    if (G) {
        for (int h = 0; h < kTets; h++) tpair[h] = kNone;
        for (int n = 0; n < kLinks; n++) { epair[n] = kNone; eord[n] = 0; }
    }
    auto pack = [&]() {
        if (!G) return;
        uint64_t w[5] = {0, 0, 0, 0, 0};
        for (int h = 0; h < kTets; h++) {
            int word = h < 10 ? 0 : h < 20 ? 1 : 2;
            w[word] |= (uint64_t)tpair[h] << (6 * (h - 10 * word));
        }
        for (int n = 0; n < kLinks; n++) {
            if (n < 6) w[2] |= (uint64_t)epair[n] << (24 + 6 * n);
            else w[3] |= (uint64_t)epair[n] << (6 * (n - 6));
            w[4] |= (uint64_t)(eord[n] & 15) << (4 * n);
        }
        uint64_t rk = 0;
        for (int n = 0; n < kLinks; n++)
            rk |= (uint64_t)((L >> n & 1) ? rank[n] : 0xF) << (4 * n);
        for (int k = 0; k < 5; k++) G->w[k] = w[k];
        G->w[5] = rk;
    };
    if (L == 0) { R.is_min = true; pack(); return; }

    // lower star cells
    uint64_t LT = kAllTris;
    uint32_t LH = kAllTets;
    for (uint16_t out = (uint16_t)(~L & kAllLinks); out; out &= out - 1) {
        int n = __ffs(out) - 1;
        LT &= ~S.tris_of_link[n];
        LH &= ~S.tets_of_link[n];
    }
    // the link of each rank (nibble r of lrw) and the rank of each lower link
    unsigned long long lrw = 0, rkw = 0;
    int p = 0;
    for (uint16_t m = L; m; m &= m - 1) {
        const int n = __ffs(m) - 1;
        lrw |= (unsigned long long)n << (4 * rank[n]);
        rkw |= (unsigned long long)rank[n] << (4 * n);
        p++;
    }
    // The lower triangles and tets in G order, each given its position in it:
    // a cell's G is its link ranks in decreasing order, so for each highest
    // rank hi, each triangle (hi, lo) for lo increasing, followed by its tets
    // (hi, lo, t) for t increasing.  The priority queues are then bit sets
    // over positions, and a pop is a find-first-set.
    int8_t posT[kTris], posH[kTets];
    uint8_t cell_at[kTris + kTets], hi_at[kTris + kTets];   // tet h: 0x40 | h
    int np = 0;
    for (int hi = 1; hi < p; hi++) {
        const int a = (int)((lrw >> (4 * hi)) & 15);
        for (int lo = 0; lo < hi; lo++) {
            const int b = (int)((lrw >> (4 * lo)) & 15);
            const int s = S.tri_of_pair[a][b];
            if (s < 0) continue;
            posT[s] = (int8_t)np; cell_at[np] = (uint8_t)s; hi_at[np] = (uint8_t)hi; np++;
            for (int t = 0; t < lo; t++) {
                const int c = (int)((lrw >> (4 * t)) & 15);
                for (uint32_t m = S.tets_of_tri[s]; m; m &= m - 1) {
                    const int q = __ffs(m) - 1;
                    if (S.tet_mask[q] >> c & 1) {
                        posH[q] = (int8_t)np; cell_at[np] = (uint8_t)(0x40 | q);
                        hi_at[np] = (uint8_t)hi; np++;
                    }
                }
            }
        }
    }

    uint16_t cE = 0;  uint64_t cT = 0;  uint32_t cH = 0;   // classified
    uint64_t pq = 0;                                       // PQone, by position
    uint32_t zr = 0;  uint64_t pz = 0;                     // PQzero: edges by rank, cells by position
    int eorder = 0;

    auto unpaired_tri = [&](int s) -> uint16_t {   // unclassified edges of s
        return (uint16_t)(((1u << S.tri_v[s][0]) | (1u << S.tri_v[s][1])) & ~cE);
    };
    auto unpaired_tet = [&](int h) -> uint64_t {   // unclassified faces of h
        return ((1ull << S.tet_f[h][0]) | (1ull << S.tet_f[h][1]) | (1ull << S.tet_f[h][2])) & ~cT;
    };
    auto push_cof_edge = [&](int n) {
        for (uint64_t m = S.tris_of_link[n] & LT & ~cT; m; m &= m - 1) {
            int s = __ffsll(m) - 1;
            if (__popc(unpaired_tri(s)) == 1) pq |= 1ull << posT[s];
        }
    };
    auto push_cof_tri = [&](int s) {
        for (uint32_t m = S.tets_of_tri[s] & LH & ~cH; m; m &= m - 1) {
            int h = __ffs(m) - 1;
            if (__popcll(unpaired_tet(h)) == 1) pq |= 1ull << posH[h];
        }
    };

    // the vertex is paired with its lowest edge
    const int n0 = (int)(lrw & 15);
    cE = (uint16_t)(1u << n0);
    if (G) { epair[n0] = kHead; eord[n0] = (uint8_t)eorder; }
    eorder++;
    zr = ((1u << p) - 1) & ~1u;
    push_cof_edge(n0);

    for (int guard = 0; guard < 4 * (kLinks + kTris + kTets); guard++) {
        while (pq) {
            // pop the smallest G among PQone
            const int ps = __ffsll(pq) - 1;
            pq &= pq - 1;
            const int cell = cell_at[ps];
            if (!(cell & 0x40)) {
                int s = cell;
                if (cT >> s & 1) continue;
                uint16_t u = unpaired_tri(s);
                if (u == 0) { pz |= 1ull << ps; continue; }
                int n = __ffs(u) - 1;                  // the unique unclassified edge
                cE |= (uint16_t)(1u << n); cT |= 1ull << s;
                zr &= ~(1u << ((rkw >> (4 * n)) & 15));
                if (G) { epair[n] = (uint8_t)s; eord[n] = (uint8_t)eorder; }
                eorder++;
                push_cof_tri(s);
                push_cof_edge(n);
            } else {
                int h = cell & 63;
                if (cH >> h & 1) continue;
                uint64_t u = unpaired_tet(h);
                if (u == 0) { pz |= 1ull << ps; continue; }
                int s = __ffsll(u) - 1;                // the unique unclassified face
                cT |= 1ull << s; cH |= 1u << h; pz &= ~(1ull << posT[s]);
                if (G) tpair[h] = (uint8_t)s;
                push_cof_tri(s);
            }
        }
        if (!(zr | pz)) break;
        // the smallest G among PQzero is critical: an edge of rank r comes
        // before every cell whose highest rank is r or more
        const int re = zr ? __ffs(zr) - 1 : kLinks;
        const int pc = pz ? __ffsll(pz) - 1 : -1;
        if (pc < 0 || re <= hi_at[pc]) {
            const int bi = (int)((lrw >> (4 * re)) & 15);
            zr &= ~(1u << re); cE |= (uint16_t)(1u << bi); R.crit_e |= (uint16_t)(1u << bi);
            if (G) eord[bi] = (uint8_t)eorder;
            eorder++;
            push_cof_edge(bi);
        } else {
            pz &= ~(1ull << pc);
            const int cell = cell_at[pc];
            if (!(cell & 0x40)) {
                cT |= 1ull << cell; R.crit_t |= 1ull << cell;
                push_cof_tri(cell);
            } else {
                cH |= 1u << (cell & 63); R.crit_h |= 1u << (cell & 63);
            }
        }
    }
    pack();
}

// Code of a critical cell of a lower star from packed 4-bit ranks.
__device__ __forceinline__ void unpack_ranks(uint64_t packed, uint8_t *r) {
#pragma unroll
    for (int n = 0; n < kLinks; n++) r[n] = (uint8_t)((packed >> (4 * n)) & 0xF);
}

}  // namespace dms
