// hmap.cuh -- the launch plan and the block-space maps of arXiv 2208.11617.
//
// Everything here is integer-only and shared by the kernels (device) and by the
// host-side map evaluation (simplex_map_block), so the host tests exercise the
// exact code the GPU runs.
//
// Frames.  Tiles have side rho cells; the block lattice has N tiles per axis,
// N a power of two with N*rho >= n + 1.  Block coordinates X = (X_1..X_m)
// with the orthogonal corner at the origin and X_m the fastest (memory) axis.
// Every tile holding a simplex cell satisfies X_1 + ... + X_m <= N - 1; the
// maps below cover that block simplex exactly once (tiles of it past the
// domain, rho * sum(X) > n, exit in the kernels).
//
// Map summary (one linear CUDA block index v per launch):
//   m = 2  H2 (Sec. 4.1, Thm. 1, Eq. map2d) on the N/2 x (N-1) grid covers the
//          blocks with sum <= N-2; a row of N blocks covers the diagonal
//          sum = N-1 (the diagonal gets its own threads, Sec. 4.1).
//          Trapezoid form (Sec. 4.2, concurrent trapezoids, in one launch):
//          the block triangle of side Ne (any multiple of the band height h)
//          is cut into bands of h tile rows; band k is a trapezoid made of a
//          rectangle h x (Ne - (k+1) h) (identity map) and a triangle of side
//          h mapped by H2 + diagonal.  Bands run in order, so the blocks in
//          flight stream whole memory rows.
//   m = 3  beta = 2: H3 (Sec. 4.3): the big cube (N/2)^3 at the corner, a layer
//          of height N/4 holding the smaller cubes laid out by the 2-D levels
//          b, q of Thm. 1, and the hinge that reflects each cube's overhang
//          onto the third corner; the plane sum = N-1 is a 2-simplex of blocks
//          mapped by H2 plus its diagonal.  Fully efficient form (h3_exact):
//          the same cubes, one index range per stack level, no packing waste.
//          beta = 3: the generic construction below.
//   m >= 3 generic, r = 1/2, beta = m (Sec. 6, Eq. generic-m): level k holds
//          m^(k-1) cubes of side b = N / 2^k; a cube is named by k-1 base-m
//          digits, each digit choosing the corner axis of one recursion step;
//          blocks of a cube's overhang (local sum > 2b-2) exit.  The plane
//          sum = N-1 is the (m-1)-dimensional cover of the same kind.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define SX_HD __host__ __device__ __forceinline__
#else
#define SX_HD inline
#endif

namespace sx {

constexpr int kMaxM = 4;
constexpr int kMaxLevels = 16;  // log2 N <= 15 keeps every count well inside 64 bits

// kMapBBThread: the bounding box with only a per-thread filter (the paper's
// baseline): blocks wholly outside the domain run too, their threads find no
// cell.  kMapBB exits such blocks as a whole.
enum MapKind : int { kMapH = 0, kMapBB = 1, kMapBBThread = 2 };

SX_HD bool is_bb(int kind) { return kind != kMapH; }

// Launch plan, passed by value to every kernel.
struct Plan {
    int32_t m;
    int32_t rho, log_rho;
    int32_t N, logN;
    int32_t beta;
    int64_t n;
    int64_t side;
    // m = 2 trapezoid form: band height h (power of two) and triangle side Ne
    // (a multiple of h, >= ceil((n+1)/rho)); band = 0 selects the single H2
    // grid on the power-of-two side N
    int32_t band, log_band;
    int32_t Ne, nbands;
    // automaton launch form: 0 = one CTA per block of the map (the paper's
    // execution model), 1 = persistent CTAs streaming runs of tiles along the
    // fastest axis (m = 3, see xrun_decode; seg_len = tiles per run), 2 =
    // persistent CTAs streaming bricks along the slowest axis (m = 3, see
    // plane_unit_decode)
    int32_t persistent, seg_len;
    // m = 3, beta = 2: 0 = the single packed grid of Sec. 4.3 (the layer of
    // height N/4 with per-level exits), 1 = one block range per stack level
    // (the fully efficient form of Sec. 4.3: no waste)
    int32_t h3_exact;
    // scale factor of the map: rinv = 1/r, 2 (every map above) or 3 (m = 2,
    // beta = 3: h2_r3 on the lattice of N3 = 3^L3 tiles per axis; the bounding
    // box keeps the power-of-two lattice N)
    int32_t rinv;
    int32_t N3, L3;
    uint64_t h_blocks;   // CUDA blocks of one H launch
    uint64_t bb_blocks;  // N^m
    // H3 (beta = 2): region sizes
    uint64_t h3_cube, h3_layer;
    // generic cubes of dimension d (3..kMaxM): level_end[d-3][k] = number of
    // blocks in levels 1..k; cube_total[d-3] = level_end[d-3][logN]
    uint64_t level_end[kMaxM - 2][kMaxLevels + 1];
    uint64_t cube_total[kMaxM - 2];
};

// floor(log2 x) for x >= 1 from the count of leading zeros (Sec. 4.1: the
// paper's "bits - clz" read with bits = 31 for a 32-bit word).
SX_HD int ilog2_u32(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return 31 - __clz(x);
#else
    return 31 - __builtin_clz(x);
#endif
}

// Eq. map2d of Thm. 1.  (wx, wy) in [0, N/2) x [0, N-1) -> the paper's
// (H_x, H_y) = (wx + q b, wy + 2 q b + 1) with b = 2^floor(log2(wy + 1)),
// q = floor(wx / b); H_x < H_y.  Returned in the corner frame:
// X1 = N - 1 - H_y, X2 = H_x, so X1 + X2 <= N - 2.  b and q are returned too.
SX_HD void h2_map(int32_t wx, int32_t wy, int32_t N, int32_t &X1, int32_t &X2, int32_t &b,
                  int32_t &q)
{
    const int lb = ilog2_u32((uint32_t)wy + 1u);
    b = 1 << lb;
    q = wx >> lb;
    const int32_t hx = wx + q * b;
    const int32_t hy = wy + 2 * q * b + 1;
    X1 = N - 1 - hy;
    X2 = hx;
}

// Blocks of the 2-simplex sum <= N-1: H2 grid, then the diagonal row.
SX_HD uint64_t h2_cover_blocks(int32_t N) { return (uint64_t)(N >> 1) * (uint64_t)(N - 1) + (uint64_t)N; }

SX_HD bool h2_cover(uint64_t v, int32_t N, int32_t logN, int32_t *X)
{
    const uint64_t grid = (uint64_t)(N >> 1) * (uint64_t)(N - 1);
    if (v < grid) {
        const int32_t wx = (int32_t)(v & (uint64_t)((N >> 1) - 1));
        const int32_t wy = (int32_t)(v >> (logN - 1));
        int32_t b, q;
        h2_map(wx, wy, N, X[0], X[1], b, q);
        return true;
    }
    const int32_t d = (int32_t)(v - grid);
    X[0] = d;
    X[1] = N - 1 - d;
    return true;
}

// m = 2 with r = 1/3, beta = 3 (Sec. 6 with 1/r = 3): the block triangle
// X1 + X2 <= N3 - 1 of side N3 = 3s is three squares of side s -- at (0, 0),
// (s, 0) and (0, s) -- and three triangles of side s at (2s, 0), (0, 2s) and
// (s, s), each split the same way; the triangles of side 1 are the blocks of
// the diagonal X1 + X2 = N3 - 1.  Level k (1 ... L3) holds 3^k squares of
// side b = N3 / 3^k, numbered triangle by triangle (the triangle's index in
// base 3, least significant digit = the last split, picks its corner at each
// split) and square by square; the N3 diagonal blocks follow.  The squares
// and the diagonal cover the triangle exactly once: N3 (N3 + 1) / 2 blocks.
// Integer arithmetic only (divisions by powers of three, no roots).
SX_HD bool h2_r3(int32_t N3, int32_t L3, uint64_t v, int32_t *X)
{
    uint64_t tris = 1;  // triangles the level's squares lie in: 3^(k-1)
    int64_t b = N3;
    for (int k = 1; k <= L3; ++k) {
        b /= 3;  // side of this level's squares
        const uint64_t bb = (uint64_t)b * (uint64_t)b, level = 3 * tris * bb;
        if (v < level) {
            const uint64_t sq = v / bb, loc = v - sq * bb;
            uint64_t t = sq / 3;
            const int q = (int)(sq - 3 * t);
            int64_t o1 = q == 1 ? b : 0, o2 = q == 2 ? b : 0;
            for (int64_t s = 3 * b, i = 1; i < k; ++i, s *= 3) {  // the triangle's corners, last split first
                const uint64_t d = t % 3;
                t /= 3;
                o1 += d == 0 ? 2 * s : (d == 2 ? s : 0);
                o2 += d == 1 ? 2 * s : (d == 2 ? s : 0);
            }
            X[0] = (int32_t)(o1 + (int64_t)(loc / (uint64_t)b));
            X[1] = (int32_t)(o2 + (int64_t)(loc % (uint64_t)b));
            return true;
        }
        v -= level;
        tris *= 3;
    }
    if (v >= (uint64_t)N3) return false;
    int64_t o1 = 0, o2 = 0;
    uint64_t t = v;
    for (int64_t s = 1, i = 0; i < L3; ++i, s *= 3) {
        const uint64_t d = t % 3;
        t /= 3;
        o1 += d == 0 ? 2 * s : (d == 2 ? s : 0);
        o2 += d == 1 ? 2 * s : (d == 2 ? s : 0);
    }
    X[0] = (int32_t)o1;
    X[1] = (int32_t)o2;
    return true;
}

// The plan with the single Eq. map2d grid (plus its diagonal row) on the
// power-of-two side N for m = 2, whatever its band: the kernels without a
// stencil (write, MAP, EDM) have no halo to keep in L2, so they take the
// paper's map and its clz-only decode instead of the trapezoid form's search.
// (An r = 1/3 plan has no band and keeps its own map.)
SX_HD Plan single_grid(const Plan &p)
{
    Plan q = p;
    if (q.m == 2 && q.band && q.rinv != 3) {
        q.band = 0;
        q.log_band = 0;
        q.h_blocks = h2_cover_blocks(q.N);
    }
    return q;
}

// x-stream form (m = 3).  Work unit w names a run of at most seg_len tiles
// along the fastest axis X3 in one tile column (X1, X2): the column comes from
// H2 plus its diagonal over the triangle X1 + X2 <= N - 1 (kMapH, the 2-D map
// of Thm. 1 applied to the columns) or from the N x N square of columns
// (kMapBB); run s of a column holds X3 = s * seg_len ... up to the last tile
// with a simplex cell, rho * (X1 + X2 + X3) <= n.
struct XRun {
    int32_t X1, X2, a, b;  // tiles X3 = a ... b
};

SX_HD uint64_t xrun_units(const Plan &p, int kind)
{
    const uint64_t cols = is_bb(kind) ? (uint64_t)p.N * (uint64_t)p.N : h2_cover_blocks(p.N);
    return cols * (uint64_t)(p.N / p.seg_len);
}

SX_HD bool xrun_decode(const Plan &p, int kind, uint64_t w, XRun &r)
{
    const uint32_t segs = (uint32_t)(p.N / p.seg_len);
    const uint64_t col = w / segs;
    const int32_t s = (int32_t)(w - col * segs);
    int32_t Y[2];
    if (is_bb(kind)) {
        Y[0] = (int32_t)(col >> p.logN);
        Y[1] = (int32_t)(col & (uint64_t)(p.N - 1));
    } else {
        h2_cover(col, p.N, p.logN, Y);
    }
    const int64_t last = (p.n >> p.log_rho) - Y[0] - Y[1];
    r.X1 = Y[0];
    r.X2 = Y[1];
    r.a = s * p.seg_len;
    r.b = (int32_t)(last < (int64_t)(r.a + p.seg_len - 1) ? last : (int64_t)(r.a + p.seg_len - 1));
    return last >= (int64_t)r.a;
}

// Plane-stream form (m = 3, launch 3).  The tetrahedron is cut into slabs of
// consecutive planes x1 (segments) and each slab's cross-section, the
// triangle x2 + x3 <= n - x1, into bricks of kPlaneTY rows x2 by kPlaneTX
// cells x3.  A work unit is one brick of one segment: the CTA streams the
// brick's planes along x1 (see k_ca3p.cu).  Units are numbered segment by
// segment (the whole cross-section of one slab before the next, so the
// bricks processed at the same time are neighbours and their halos meet in
// L2); within a segment the row band Y (x2 = 32 Y ...) comes before Y + 1,
// and inside a band the bricks X = 0, 1, ... (a compact numbering: every
// unit index names a brick that holds cells of the segment's first plane,
// found from prefix counts instead of a map with padding).  The bounding box
// numbers every brick of the (n+1) x (n+1) square in every segment; bricks
// past the domain exit (kMapBB) or run with every store masked
// (kMapBBThread).  Segments shrink towards the apex so that the last units
// of a launch are short: a segment starting at plane b has
// clamp(2^floor(log2((n + 1 - b) / 64)), 4, 64) planes (16 at the base of
// the n = 1023 tetrahedron; twice and four times as long were 2 % and 16 %
// slower).
constexpr int kPlaneTY = 32, kPlaneTX = 128;
constexpr int kPlaneMaxSegs = 320;

struct PlaneSched {
    int32_t nseg;        // segments
    int32_t nty, ntx;    // bricks per axis of the square: ceil((n+1)/TY), ceil((n+1)/TX)
    int32_t kind;        // map kind the units were counted for
    int64_t n;
    uint64_t units;      // work units of one step
    int32_t seg_b[kPlaneMaxSegs + 1];   // first plane of segment s; seg_b[nseg] = n + 1
    uint32_t seg_u[kPlaneMaxSegs + 1];  // first unit of segment s; seg_u[nseg] = units
};

// Planes of the segment that starts at plane b.
SX_HD int32_t plane_seg_len(int64_t n, int64_t b)
{
    const int64_t q = (n + 1 - b) / 64;
    int32_t s = 4;
    while (s < 64 && (int64_t)(2 * s) <= q) s *= 2;
    return s;
}

// Bricks of the cross-section x2 + x3 <= K that hold a cell (K >= 0):
// column X has floor((K - TX X) / TY) + 1 rows.
SX_HD uint64_t plane_tri_bricks(int64_t K)
{
    uint64_t c = 0;
    for (int64_t x0 = 0; x0 <= K; x0 += kPlaneTX) c += (uint64_t)((K - x0) / kPlaneTY + 1);
    return c;
}

// Fills s for a map of side n; false if n needs more than kPlaneMaxSegs
// segments or more than 2^32 units.  fixed_len > 0: every segment has that
// many planes (the batched engine's small instances, where the length of the
// whole batch's queue, not of one instance, decides the tail).
inline bool plane_sched_build(int64_t n, int kind, PlaneSched *s, int32_t fixed_len = 0)
{
    s->n = n;
    s->kind = kind;
    s->nty = (int32_t)((n + kPlaneTY) / kPlaneTY);
    s->ntx = (int32_t)((n + kPlaneTX) / kPlaneTX);
    uint64_t u = 0;
    int32_t k = 0;
    for (int64_t b = 0; b <= n; b += fixed_len > 0 ? fixed_len : plane_seg_len(n, b)) {
        if (k >= kPlaneMaxSegs) return false;
        s->seg_b[k] = (int32_t)b;
        s->seg_u[k] = (uint32_t)u;
        u += is_bb(kind) ? (uint64_t)s->nty * (uint64_t)s->ntx : plane_tri_bricks(n - b);
        if (u >= (1ull << 32)) return false;
        ++k;
    }
    s->nseg = k;
    s->seg_b[k] = (int32_t)(n + 1);
    s->seg_u[k] = (uint32_t)u;
    s->units = u;
    return true;
}

// One work unit: brick rows y0 ... y0 + TY - 1, cells x0 ... x0 + TX - 1,
// output planes b ... e (inclusive).
struct PlaneUnit {
    int32_t y0, x0, b, e;
};

// Unit w -> its brick and planes.  False when the brick has no cell in the
// segment (bounding box only; kMapBBThread keeps such bricks, with e the
// segment's last plane, and their stores are all masked).
// seg_b / seg_u: the schedule's segment tables (s.seg_b, s.seg_u, or a copy
// of them in device memory, where the kernel reads them through L1).
SX_HD bool plane_unit_decode(const PlaneSched &s, const int32_t *seg_b, const uint32_t *seg_u, uint64_t w,
                             PlaneUnit &u)
{
    // segment: the last s with seg_u[s] <= w
    int32_t lo = 0, hi = s.nseg - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if ((uint64_t)seg_u[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const int64_t b = seg_b[lo], e = (int64_t)seg_b[lo + 1] - 1;
    uint64_t r = w - (uint64_t)seg_u[lo];
    int64_t Y, X;
    if (is_bb(s.kind)) {
        Y = (int64_t)(r / (uint64_t)s.ntx);
        X = (int64_t)(r - (uint64_t)Y * (uint64_t)s.ntx);
    } else {
        // row band Y holds the bricks X with TX X <= K - TY Y
        const int64_t K = s.n - b;
        Y = 0;
        for (;;) {
            const uint64_t cols = (uint64_t)((K - Y * kPlaneTY) / kPlaneTX + 1);
            if (r < cols) break;
            r -= cols;
            ++Y;
        }
        X = (int64_t)r;
    }
    u.y0 = (int32_t)(Y * kPlaneTY);
    u.x0 = (int32_t)(X * kPlaneTX);
    u.b = (int32_t)b;
    const int64_t last = s.n - Y * kPlaneTY - X * kPlaneTX;  // last plane with a cell of the brick
    if (s.kind == kMapBBThread) {
        u.e = (int32_t)e;
        return true;
    }
    u.e = (int32_t)(last < e ? last : e);
    return last >= b;
}

SX_HD bool plane_unit_decode(const PlaneSched &s, uint64_t w, PlaneUnit &u)
{
    return plane_unit_decode(s, s.seg_b, s.seg_u, w, u);
}

// Device copy of a schedule's segment tables: seg_b[kPlaneSegTable] then
// seg_u[kPlaneSegTable] (int32 / uint32), kPlaneSegWords words per mode.
constexpr int kPlaneSegTable = kPlaneMaxSegs + 1;
constexpr int kPlaneSegWords = 2 * kPlaneSegTable;

// Blocks before band k of the trapezoid form: sum over j < k of
// h (Ne - (j+1) h) + h (h+1) / 2 = k h (2 Ne - k h + 1) / 2.
SX_HD uint64_t trapezoid_prefix(int64_t k, int64_t h, int64_t Ne) { return (uint64_t)(k * h * (2 * Ne - k * h + 1) / 2); }

SX_HD bool h2_trapezoids(const Plan &p, uint64_t v, int32_t *X)
{
    const int64_t h = p.band, Ne = p.Ne;
    // band k: the largest k with prefix(k) <= v (binary search, uniform per block)
    int32_t lo = 0, hi = p.nbands - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (trapezoid_prefix(mid, h, Ne) <= v) lo = mid; else hi = mid - 1;
    }
    const int32_t k = lo;
    uint64_t u = v - trapezoid_prefix(k, h, Ne);
    const int32_t W = (int32_t)(Ne - (int64_t)(k + 1) * h);  // rectangle width
    const uint64_t rect = (uint64_t)h * (uint64_t)W;
    if (u < rect) {
        const uint32_t i = (uint32_t)u / (uint32_t)W;  // rectangle row-major
        X[0] = (int32_t)(k * h) + (int32_t)i;
        X[1] = (int32_t)((uint32_t)u - i * (uint32_t)W);
        return true;
    }
    int32_t Y[2];
    h2_cover(u - rect, (int32_t)h, p.log_band, Y);  // triangle of side h
    X[0] = (int32_t)(k * h) + Y[0];
    X[1] = W + Y[1];
    return true;
}

// Hinge of Sec. 4.3: a cube of side b with corner (c1, c2, 0) and local
// offset l; if l falls past the tetrahedron (l1 + l2 + l3 >= 2b - 1), it is
// reflected in x, y and complemented in z onto the cube's third corner
// (c1, c2, b) + ... which that overhang fills exactly.
SX_HD void h3_place(int32_t c1, int32_t c2, int32_t b, int32_t l1, int32_t l2, int32_t l3, int32_t *X)
{
    if (l1 + l2 + l3 >= 2 * b - 1) {
        X[0] = c1 + b - 1 - l1;
        X[1] = c2 + b - 1 - l2;
        X[2] = 2 * b - 1 - l3;
    } else {
        X[0] = c1 + l1;
        X[1] = c2 + l2;
        X[2] = l3;
    }
}

SX_HD bool h3_cover(const Plan &p, uint64_t v, int32_t *X)
{
    const int32_t N = p.N, logN = p.logN, half = N >> 1;
    if (v < p.h3_cube) {
        // the big cube (N/2)^3 at the orthogonal corner
        const int lh = logN - 1;
        const int32_t l3 = (int32_t)(v & (uint64_t)(half - 1));
        const int32_t l2 = (int32_t)((v >> lh) & (uint64_t)(half - 1));
        const int32_t l1 = (int32_t)(v >> (2 * lh));
        h3_place(0, 0, half, l1, l2, l3, X);
        return true;
    }
    v -= p.h3_cube;
    if (v < p.h3_layer) {
        // layer of height N/4: cubes of side b <= N/4 stacked by the 2-D levels
        const int32_t wx = (int32_t)(v & (uint64_t)(half - 1));
        const uint64_t t = v >> (logN - 1);
        const int32_t lz = (int32_t)(t & (uint64_t)((N >> 2) - 1));
        const int32_t wy = (int32_t)(t >> (logN - 2));
        int32_t X1, X2, b, q;
        h2_map(wx, wy, N, X1, X2, b, q);
        if (lz >= b) return false;  // packing waste of the layer (Lemma 4)
        const int32_t c1 = N - 2 * b - 2 * q * b, c2 = 2 * q * b;
        h3_place(c1, c2, b, X1 - c1, X2 - c2, lz, X);
        return true;
    }
    v -= p.h3_layer;
    // diagonal plane X1 + X2 + X3 = N - 1 (Sec. 4.3 leaves it aside): a
    // 2-simplex of blocks mapped by H2 plus its diagonal
    int32_t Y[2];
    h2_cover(v, N, logN, Y);
    X[0] = Y[0];
    X[1] = Y[1];
    X[2] = N - 1 - Y[0] - Y[1];
    return true;
}

// Fully efficient H3 (Sec. 4.3, closing paragraph): instead of packing the
// cubes of side b <= N/4 into one layer of height N/4 (blocks with lz >= b
// exit), each stack level k = 2 ... log2 N (b = N >> k) gets its own range of
// block indices, N/(2b) cubes of b^3 blocks each, one after the other in a
// single launch.  Blocks before level k: sum over j < k of N (N >> j)^2 / 2
// = (N^3 - N^3 / 4^(k-2)) / 24.  Together with the big cube (N/2)^3 this is
// exactly (N^3 - N) / 6, the blocks below the plane sum = N - 1.
SX_HD uint64_t h3_level_prefix(int32_t N, int k)
{
    const uint64_t c = (uint64_t)N * (uint64_t)N * (uint64_t)N;
    return (c - (c >> (2 * k - 4))) / 24;
}

SX_HD bool h3_exact(const Plan &p, uint64_t v, int32_t *X)
{
    const int32_t N = p.N, logN = p.logN, half = N >> 1;
    if (v < p.h3_cube) {
        const int lh = logN - 1;
        const int32_t l3 = (int32_t)(v & (uint64_t)(half - 1));
        const int32_t l2 = (int32_t)((v >> lh) & (uint64_t)(half - 1));
        const int32_t l1 = (int32_t)(v >> (2 * lh));
        h3_place(0, 0, half, l1, l2, l3, X);
        return true;
    }
    v -= p.h3_cube;
    if (v < p.h3_layer) {
        // level k holds N (N >> k)^2 / 2 = N^3 / 2^(2k+1) blocks
        const uint64_t c = (uint64_t)N * (uint64_t)N * (uint64_t)N;
        uint64_t u = v;
        int k = 2;
        for (; k < logN; ++k) {
            const uint64_t sz = c >> (2 * k + 1);
            if (u < sz) break;
            u -= sz;
        }
        const int lb = logN - k;
        const int32_t b = 1 << lb;
        const int32_t q = (int32_t)(u >> (3 * lb));
        const uint32_t l = (uint32_t)(u & ((1ull << (3 * lb)) - 1ull));
        const int32_t l3 = (int32_t)(l & (uint32_t)(b - 1));
        const int32_t l2 = (int32_t)((l >> lb) & (uint32_t)(b - 1));
        const int32_t l1 = (int32_t)(l >> (2 * lb));
        h3_place(N - 2 * b - 2 * q * b, 2 * q * b, b, l1, l2, l3, X);
        return true;
    }
    v -= p.h3_layer;
    int32_t Y[2];
    h2_cover(v, N, logN, Y);
    X[0] = Y[0];
    X[1] = Y[1];
    X[2] = N - 1 - Y[0] - Y[1];
    return true;
}

// Generic self-similar cubes of dimension D (r = 1/2, beta = D), covering the
// blocks with sum <= N - 2.
template <int D>
SX_HD bool cubes_generic(const Plan &p, uint64_t v, int32_t *X)
{
    const int32_t N = p.N, logN = p.logN;
    int k = 1;
    while (k < logN && v >= p.level_end[D - 3][k]) ++k;
    const int lb = logN - k;
    const int32_t b = 1 << lb;
    const uint64_t local = v - p.level_end[D - 3][k - 1];
    uint64_t c = local >> (D * lb);
    const uint64_t l = local & ((1ull << (D * lb)) - 1ull);
    int32_t corner[D];
#pragma unroll
    for (int i = 0; i < D; ++i) corner[i] = 0;
    for (int j = k - 1; j >= 1; --j) {
        const int dig = (int)(c % (uint64_t)D);
        c /= (uint64_t)D;
#pragma unroll
        for (int i = 0; i < D; ++i)
            if (i == dig) corner[i] += N >> j;
    }
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const int32_t li = (int32_t)((l >> ((D - 1 - i) * lb)) & (uint64_t)(b - 1));
        X[i] = corner[i] + li;
        s += li;
    }
    return s <= 2 * b - 2;  // blocks of the cube's overhang exit
}

// Cover of {X in [0,N)^D : sum X <= N - 1}: the cubes, then the plane
// sum = N - 1 as a (D-1)-dimensional cover.
template <int D>
struct Cover {
    static SX_HD bool run(const Plan &p, uint64_t v, int32_t *X)
    {
        if (v < p.cube_total[D - 3]) return cubes_generic<D>(p, v, X);
        v -= p.cube_total[D - 3];
        const bool ok = Cover<D - 1>::run(p, v, X);
        int32_t s = 0;
#pragma unroll
        for (int i = 0; i < D - 1; ++i) s += X[i];
        X[D - 1] = p.N - 1 - s;
        return ok;
    }
};

template <>
struct Cover<2> {
    static SX_HD bool run(const Plan &p, uint64_t v, int32_t *X) { return h2_cover(v, p.N, p.logN, X); }
};

// The map of one launch: linear CUDA block index v -> tile X.  Returns false
// when the block has no tile (packing waste or overhang).
template <int M>
SX_HD bool decode(const Plan &p, int kind, uint64_t v, int32_t *X)
{
    if (is_bb(kind)) {
        // bounding box, f(x) = x (Eq. 3), on the N^m lattice linearised to 1-D
#pragma unroll
        for (int i = 0; i < M; ++i)
            X[M - 1 - i] = (int32_t)((v >> (i * p.logN)) & (uint64_t)(p.N - 1));
        return true;
    }
    if (M == 2) {
        if (p.rinv == 3) return h2_r3(p.N3, p.L3, v, X);
        return p.band ? h2_trapezoids(p, v, X) : h2_cover(v, p.N, p.logN, X);
    }
    if (M == 3 && p.beta == 2) return p.h3_exact ? h3_exact(p, v, X) : h3_cover(p, v, X);
    return Cover<M>::run(p, v, X);
}

// rho * sum(X): first cell-coordinate sum of the tile.
template <int M>
SX_HD int64_t tile_base_sum(const Plan &p, const int32_t *X)
{
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) s += X[i];
    return s * p.rho;
}

}  // namespace sx
