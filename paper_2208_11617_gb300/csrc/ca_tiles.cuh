// ca_tiles.cuh -- the per-tile bodies of the automaton step, shared by the
// single-instance kernels (k_ca2.cu, k_ca3.cu) and the batched engine
// (k_batch.cu).  Each reads one tile plus its one-cell halo from a staged
// shared-memory box, writes the tile's next state to global memory with
// 16-byte stores (masked on tiles crossing x_1 + ... + x_m = n) and returns
// the number of live cells the calling thread wrote.
#pragma once

#include "common.cuh"

namespace sx {

// m = 2: the box is (RHO + 32) x (RHO + 2) bytes (16-byte halo columns, one
// halo row each side).  Thread (tx, ty) owns the 16-byte column chunk tx and
// walks the R output rows ty*R .. ty*R + R - 1, keeping the horizontal 3-sums
// of three rows in registers.
template <int RHO, int R, bool ORK>
__device__ __forceinline__ uint32_t ca2_tile(const uint8_t *tile, int64_t n, int64_t side, const Rule &rule,
                                             uint8_t *__restrict__ out, int64_t x0, int64_t y0, bool partial,
                                             int tx, int ty)
{
    constexpr int BW = RHO + 32;
    const uint8_t *col = tile + 16 + 16 * tx;
    const int r0 = ty * R;                  // first output row of this thread
    const int64_t xc = x0 + 16 * tx;        // first cell of the chunk
    uint32_t hp[4], hc[4], ac[4], tmp[4], lacc = 0;
    hsum_row(col + r0 * BW, hp, tmp);
    hsum_row(col + (r0 + 1) * BW, hc, ac);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        uint32_t hn[4], an[4], s[4], nw[4];
        hsum_row(col + (r0 + i + 2) * BW, hn, an);
#pragma unroll
        for (int w = 0; w < 4; ++w) s[w] = hp[w] + hc[w] + hn[w];
        next_state4<ORK>(s, ac, rule, nw);
        const int64_t y = y0 + r0 + i;
        bool store = true;
        if (partial) {
            const int64_t c64 = n - y - xc + 1;  // domain cells in this chunk
            const int c = (int)(c64 < 0 ? 0 : (c64 > 16 ? 16 : c64));
#pragma unroll
            for (int w = 0; w < 4; ++w) nw[w] &= chunk_word_mask(c, w);
            store = c > 0;
        }
        if (store) store16(out + y * side + xc, nw);
        lacc += nw[0] + nw[1] + nw[2] + nw[3];  // bytes <= 4R: no carry
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            hp[w] = hc[w];
            hc[w] = hn[w];
            ac[w] = an[w];
        }
    }
    return byte_sum(lacc);
}

// Raw bytes of chunk c of staged row r (row pitch BW bytes) and the words just
// outside it: w[0] = last word of chunk c-1, w[1..4] = chunk c, w[5] = first
// word of chunk c+1.
template <int BW>
__device__ __forceinline__ void load_chunk6(const uint8_t *tile, int r, int c, uint32_t w[6])
{
    const uint8_t *row = tile + r * BW + 16 * c;
    const uint4 v = *reinterpret_cast<const uint4 *>(row);
    w[0] = *reinterpret_cast<const uint32_t *>(row - 4);
    w[1] = v.x;
    w[2] = v.y;
    w[3] = v.z;
    w[4] = v.w;
    w[5] = *reinterpret_cast<const uint32_t *>(row + 16);
}

// Byte-wise horizontal 3-sums of the 4 words v[] given the word before (l) and
// after (r) them: s[w] byte j = v(j - 1) + v(j) + v(j + 1).
__device__ __forceinline__ void hsum4(const uint32_t v[4], uint32_t l, uint32_t r, uint32_t s[4])
{
    s[0] = v[0] + __funnelshift_l(l, v[0], 8) + __funnelshift_r(v[0], v[1], 8);
    s[1] = v[1] + __funnelshift_l(v[0], v[1], 8) + __funnelshift_r(v[1], v[2], 8);
    s[2] = v[2] + __funnelshift_l(v[1], v[2], 8) + __funnelshift_r(v[2], v[3], 8);
    s[3] = v[3] + __funnelshift_l(v[2], v[3], 8) + __funnelshift_r(v[3], r, 8);
}

// m = 3, 16^3 tiles: box 48 x 18 x 18 bytes.  Thread (tx, ty, tz) owns the
// 16-byte chunk tx of row x2 = y0 + ty and walks RZ planes x1 = z0 + tz*RZ ...
// along x1.  The 27-sum (neighbours plus the cell) of a byte is h(V9): V9 is
// the 3 x 3 sum over (x2, x1) -- column sums CY(plane) = row(x2-1) + row(x2) +
// row(x2+1), slid along x1 -- and h one horizontal 3-sum over V9, using the V9
// of the words next to the chunk for its edge bytes (bytes stay <= 27).
// Returns the live cells it wrote.
template <int RHO, int RZ, bool ORK>
__device__ __forceinline__ uint32_t ca3_tile(const uint8_t *tile, int64_t n, int64_t side, const Rule &rule,
                                             uint8_t *__restrict__ out, int64_t x0, int64_t y0, int64_t z0,
                                             bool partial, int tx, int ty, int tz)
{
    static_assert(RHO == 16, "32^3 tiles use ca3_tile32 (swizzled box)");
    constexpr int BW = RHO + 32, BH = RHO + 2;
    const int c = 1 + tx;  // staged chunk (chunk 0 is the left halo)
    // staged row r = zz * BH + yy holds x1 = z0 + zz - 1, x2 = y0 + yy - 1
    const int64_t xc = x0 + 16 * tx;
    const int64_t x2 = y0 + ty;
    const int zb = tz * RZ;  // first output plane of this thread
    auto col_sum = [&](int zz, uint32_t cy[6], uint32_t mid[4]) {
        uint32_t a[6], b[6], d[6];
        const int r = zz * BH + ty;
        load_chunk6<BW>(tile, r, c, a);
        load_chunk6<BW>(tile, r + 1, c, b);
        load_chunk6<BW>(tile, r + 2, c, d);
#pragma unroll
        for (int w = 0; w < 6; ++w) cy[w] = a[w] + b[w] + d[w];
#pragma unroll
        for (int w = 0; w < 4; ++w) mid[w] = b[w + 1];
    };
    uint32_t cp[6], cc[6], ac[4], tmp[4], lacc = 0;
    col_sum(zb, cp, tmp);
    col_sum(zb + 1, cc, ac);
#pragma unroll
    for (int i = 0; i < RZ; ++i) {
        uint32_t cn[6], an[4], v9[6], s[4], nw[4];
        col_sum(zb + i + 2, cn, an);
#pragma unroll
        for (int w = 0; w < 6; ++w) v9[w] = cp[w] + cc[w] + cn[w];
        hsum4(v9 + 1, v9[0], v9[5], s);
        next_state4<ORK>(s, ac, rule, nw);
        const int64_t x1 = z0 + zb + i;
        bool store = true;
        if (partial) {
            const int64_t c64 = n - x1 - x2 - xc + 1;
            const int cnt = (int)(c64 < 0 ? 0 : (c64 > 16 ? 16 : c64));
#pragma unroll
            for (int w = 0; w < 4; ++w) nw[w] &= chunk_word_mask(cnt, w);
            store = cnt > 0;
        }
        if (store) store16(out + (x1 * side + x2) * side + xc, nw);
        lacc += nw[0] + nw[1] + nw[2] + nw[3];
#pragma unroll
        for (int w = 0; w < 6; ++w) {
            cp[w] = cc[w];
            cc[w] = cn[w];
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) ac[w] = an[w];
    }
    return byte_sum(lacc);
}

// m = 3, 32^3 tiles: the staged box is 64 x 34 x 34 bytes, loaded with the
// tensor map's 64-byte swizzle: 16-byte unit u of staged row R = zz * 34 + yy
// (x1 = z0 + zz - 1, x2 = y0 + yy - 1, bytes x0 - 16 ... x0 + 47) sits at unit
// u ^ ((R >> 1) & 3) of the row.
//
// Thread (tx, p, tz) -- tx = lane & 1, p = lane >> 1, tz = warp -- owns the
// 16-byte chunk tx of the output rows x2 = y0 + 2p and y0 + 2p + 1 on the RZ
// planes x1 = z0 + tz*RZ ...  Per staged plane it reads its chunk of the
// staged rows 2p ... 2p + 3 and one halo word of each (the word holding the
// cell just outside the tile on its side), forms the column sums of its two
// output rows and slides them along x1; the 3 x 3 x 3 sum of a byte is then
// one horizontal 3-sum over the summed words.  The summed word just inside
// the partner's chunk comes from lane ^ 1 by shuffle.
//
// Lanes with odd p read their four rows in reverse order, so each 16-byte load
// instruction has half its lanes on even rows and half on odd rows and covers
// all 8 bank groups (no bank conflicts).  The column-sum formulas stay the same;
// only which output row comes first flips.  Returns the live cells it wrote.
template <int RZ, bool ORK>
__device__ __forceinline__ uint32_t ca3_tile32(const uint8_t *tile, int64_t n, int64_t side, const Rule &rule,
                                               uint8_t *__restrict__ out, int64_t x0, int64_t y0, int64_t z0,
                                               bool partial, int tx, int p, int tz)
{
    static_assert(RZ % 4 == 0 || RZ == 2, "runs start on planes that are multiples of 4 (or 2)");
    constexpr int kRow = 64, kPlane = 34 * kRow;
    const int zb = tz * RZ;                         // first output plane of this thread
    const int rev = p & 1;                          // rows read in reverse order
    const uint32_t c16 = 16u * (uint32_t)(1 + tx);  // chunk 1 or 2, in bytes
    // swizzle phase of staged row 2p + r in plane zb + j is (zb + j + p + (r >> 1)) & 3
    const uint32_t ph_lo = 16u * (uint32_t)(zb + p + rev);      // loads 0, 1 (rows r >> 1 == rev)
    const uint32_t ph_hi = 16u * (uint32_t)(zb + p + 1 - rev);  // loads 2, 3
    // the halo word: chunk c ^ 1 (0 or 3), word 3 (left side) or 0 (right side)
    const uint32_t hx = tx ? 16u : 28u;
    const uint8_t *rowp[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rowp[k] = tile + zb * kPlane + (2 * p + (k ^ (3 * rev))) * kRow;
    const int64_t xc = x0 + 16 * tx;
    const int64_t x2f = y0 + 2 * p + rev;      // output row of the first result
    const int64_t x2s = y0 + 2 * p + 1 - rev;  // and of the second

    // column sums of staged plane zb + j: cf = rows 0..2 of the load order,
    // cs = rows 1..3 ([4] = halo word); mf, ms = the centre rows (loads 1, 2)
    auto load_plane = [&](int j, uint32_t cf[5], uint32_t cs[5], uint32_t mf[4], uint32_t ms[4]) {
        uint32_t v[4][4], h[4];
        const uint32_t o_lo = ((ph_lo + 16u * (uint32_t)j) & 48u) ^ c16;
        const uint32_t o_hi = ((ph_hi + 16u * (uint32_t)j) & 48u) ^ c16;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint8_t *row = rowp[k] + j * kPlane;
            const uint32_t o = k < 2 ? o_lo : o_hi;
            const uint4 w = *reinterpret_cast<const uint4 *>(row + o);
            v[k][0] = w.x;
            v[k][1] = w.y;
            v[k][2] = w.z;
            v[k][3] = w.w;
            h[k] = *reinterpret_cast<const uint32_t *>(row + (o ^ hx));
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            cf[w] = v[0][w] + v[1][w] + v[2][w];
            cs[w] = v[1][w] + v[2][w] + v[3][w];
            mf[w] = v[1][w];
            ms[w] = v[2][w];
        }
        cf[4] = h[0] + h[1] + h[2];
        cs[4] = h[1] + h[2] + h[3];
    };
    // next state of one output row from its summed words (v[4] = halo side)
    auto row_next = [&](const uint32_t v[5], const uint32_t alive[4], uint32_t nw[4]) {
        const uint32_t send = tx ? v[0] : v[3];
        const uint32_t got = __shfl_xor_sync(0xffffffffu, send, 1);
        uint32_t s[4];
        hsum4(v, tx ? got : v[4], tx ? v[4] : got, s);
        next_state4<ORK>(s, alive, rule, nw);
    };
    auto put_row = [&](uint8_t *dst, int64_t cnt64, uint32_t nw[4]) {
        if (partial) {
            const int cnt = (int)(cnt64 < 0 ? 0 : (cnt64 > 16 ? 16 : cnt64));
#pragma unroll
            for (int w = 0; w < 4; ++w) nw[w] &= chunk_word_mask(cnt, w);
            if (cnt > 0) store16(dst, nw);
        } else {
            store16(dst, nw);
        }
    };

    uint32_t pf[5], ps[5], qf[5], qs[5], af[4], as[4], tmp[4], lacc = 0;
    load_plane(0, pf, ps, tmp, tmp);
    load_plane(1, qf, qs, af, as);
#pragma unroll
    for (int i = 0; i < RZ; ++i) {
        uint32_t nf[5], ns[5], mf[4], ms[4], vf[5], vs[5], wf[4], ws[4];
        load_plane(i + 2, nf, ns, mf, ms);
#pragma unroll
        for (int w = 0; w < 5; ++w) {
            vf[w] = pf[w] + qf[w] + nf[w];
            vs[w] = ps[w] + qs[w] + ns[w];
        }
        row_next(vf, af, wf);
        row_next(vs, as, ws);
        const int64_t x1 = z0 + zb + i;
        const int64_t rem = n - x1 - xc + 1;  // cells of a row chunk at x2 = 0 inside the simplex
        put_row(out + (x1 * side + x2f) * side + xc, rem - x2f, wf);
        put_row(out + (x1 * side + x2s) * side + xc, rem - x2s, ws);
        lacc += (wf[0] + wf[1]) + (wf[2] + wf[3]) + (ws[0] + ws[1]) + (ws[2] + ws[3]);
#pragma unroll
        for (int w = 0; w < 5; ++w) {
            pf[w] = qf[w];
            ps[w] = qs[w];
            qf[w] = nf[w];
            qs[w] = ns[w];
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            af[w] = mf[w];
            as[w] = ms[w];
        }
    }
    return byte_sum(lacc);
}

// m = 3, 32^3 tiles of the x-stream form: the x-column M of a slab of the
// tile (planes z0 ... z0 + 32 / kStreamZSplit - 1) and its neighbours L
// (x3 - 32) and R (x3 + 32) are staged separately, 32 x 34 x kStreamColPlanes
// bytes each, unswizzled (row R = zz * 34 + yy at byte 32 R; x1 = z0 + zz - 1,
// x2 = y0 + yy - 1, x3 = x0 ... x0 + 31 for M); warp tz walks the planes
// z0 + tz RZ ... z0 + tz RZ + RZ - 1.  The thread layout and sums are those
// of ca3_tile32; the halo word of lane tx = 0 is the last word of
// the L row, of tx = 1 the first word of the R row (0 where has_l / has_r
// is false: the neighbour column lies before x3 = 0 or past the domain).
// Lanes whose row-pair index p has bit 1 set read their rows in reverse
// order: with 32-byte rows that puts the lanes of each 16-byte load on all 8
// bank groups.  Returns the live cells it wrote.
template <int RZ, bool ORK>
__device__ __forceinline__ uint32_t ca3_tile32c(const uint8_t *M, const uint8_t *L, const uint8_t *R, bool has_l,
                                                bool has_r, int64_t n, int64_t side, const Rule &rule,
                                                uint8_t *__restrict__ out, int64_t x0, int64_t y0, int64_t z0,
                                                bool partial, int tx, int p, int tz)
{
    constexpr int kRow = 32, kPlane = 34 * kRow;
    const int zb = tz * RZ;
    const int rev = (p >> 1) & 1;
    const uint8_t *hcol = tx ? R : L;
    const bool has_h = tx ? has_r : has_l;
    const int hoff = tx ? 0 : 28;
    int ro[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ro[k] = zb * kPlane + (2 * p + (k ^ (3 * rev))) * kRow;
    const int64_t xc = x0 + 16 * tx;
    const int64_t x2f = y0 + 2 * p + rev;      // output row of the first result
    const int64_t x2s = y0 + 2 * p + 1 - rev;  // and of the second

    auto load_plane = [&](int j, uint32_t cf[5], uint32_t cs[5], uint32_t mf[4], uint32_t ms[4]) {
        uint32_t v[4][4], h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int o = ro[k] + j * kPlane;
            const uint4 w = *reinterpret_cast<const uint4 *>(M + o + 16 * tx);
            v[k][0] = w.x;
            v[k][1] = w.y;
            v[k][2] = w.z;
            v[k][3] = w.w;
            h[k] = has_h ? *reinterpret_cast<const uint32_t *>(hcol + o + hoff) : 0u;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            cf[w] = v[0][w] + v[1][w] + v[2][w];
            cs[w] = v[1][w] + v[2][w] + v[3][w];
            mf[w] = v[1][w];
            ms[w] = v[2][w];
        }
        cf[4] = h[0] + h[1] + h[2];
        cs[4] = h[1] + h[2] + h[3];
    };
    auto row_next = [&](const uint32_t v[5], const uint32_t alive[4], uint32_t nw[4]) {
        const uint32_t send = tx ? v[0] : v[3];
        const uint32_t got = __shfl_xor_sync(0xffffffffu, send, 1);
        uint32_t sum[4];
        hsum4(v, tx ? got : v[4], tx ? v[4] : got, sum);
        next_state4<ORK>(sum, alive, rule, nw);
    };
    auto put_row = [&](uint8_t *dst, int64_t cnt64, uint32_t nw[4]) {
        if (partial) {
            const int cnt = (int)(cnt64 < 0 ? 0 : (cnt64 > 16 ? 16 : cnt64));
#pragma unroll
            for (int w = 0; w < 4; ++w) nw[w] &= chunk_word_mask(cnt, w);
            if (cnt > 0) store16(dst, nw);
        } else {
            store16(dst, nw);
        }
    };

    uint32_t pf[5], ps[5], qf[5], qs[5], af[4], as[4], tmp[4], lacc = 0;
    load_plane(0, pf, ps, tmp, tmp);
    load_plane(1, qf, qs, af, as);
#pragma unroll
    for (int i = 0; i < RZ; ++i) {
        uint32_t nf[5], ns[5], mf[4], ms[4], vf[5], vs[5], wf[4], ws[4];
        load_plane(i + 2, nf, ns, mf, ms);
#pragma unroll
        for (int w = 0; w < 5; ++w) {
            vf[w] = pf[w] + qf[w] + nf[w];
            vs[w] = ps[w] + qs[w] + ns[w];
        }
        row_next(vf, af, wf);
        row_next(vs, as, ws);
        const int64_t x1 = z0 + zb + i;
        const int64_t rem = n - x1 - xc + 1;
        put_row(out + (x1 * side + x2f) * side + xc, rem - x2f, wf);
        put_row(out + (x1 * side + x2s) * side + xc, rem - x2s, ws);
        lacc += (wf[0] + wf[1]) + (wf[2] + wf[3]) + (ws[0] + ws[1]) + (ws[2] + ws[3]);
#pragma unroll
        for (int w = 0; w < 5; ++w) {
            pf[w] = qf[w];
            ps[w] = qs[w];
            qf[w] = nf[w];
            qs[w] = ns[w];
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            af[w] = mf[w];
            as[w] = ms[w];
        }
    }
    return byte_sum(lacc);
}

}  // namespace sx
