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

// Byte offset of 16-byte chunk c within a staged row r (row pitch BW bytes).
template <int BW, bool SWZ>
__device__ __forceinline__ int chunk_off(int r, int c)
{
    if (SWZ) return r * BW + 16 * (c ^ ((r >> 1) & 3));
    return r * BW + 16 * c;
}

// Horizontal 3-sums of chunk c of staged row r (chunks c-1 and c+1 give the
// neighbour bytes at the chunk's edges).
template <int BW, bool SWZ>
__device__ __forceinline__ void hsum_staged(const uint8_t *tile, int r, int c, uint32_t h[4], uint32_t cc[4])
{
    const uint4 w = *reinterpret_cast<const uint4 *>(tile + chunk_off<BW, SWZ>(r, c));
    const uint32_t lw = *reinterpret_cast<const uint32_t *>(tile + chunk_off<BW, SWZ>(r, c - 1) + 12);
    const uint32_t rw = *reinterpret_cast<const uint32_t *>(tile + chunk_off<BW, SWZ>(r, c + 1));
    h[0] = w.x + __funnelshift_l(lw, w.x, 8) + __funnelshift_r(w.x, w.y, 8);
    h[1] = w.y + __funnelshift_l(w.x, w.y, 8) + __funnelshift_r(w.y, w.z, 8);
    h[2] = w.z + __funnelshift_l(w.y, w.z, 8) + __funnelshift_r(w.z, w.w, 8);
    h[3] = w.w + __funnelshift_l(w.z, w.w, 8) + __funnelshift_r(w.w, rw, 8);
    cc[0] = w.x;
    cc[1] = w.y;
    cc[2] = w.z;
    cc[3] = w.w;
}

// One tile's step from its staged box: thread (tx, ty, tz) owns the 16-byte
// chunk tx of row x2 = y0 + ty and walks RZ planes x1 = z0 + tz*RZ ... along
// x1.  Returns the live cells it wrote.
template <int RHO, int RZ, bool ORK>
__device__ __forceinline__ uint32_t ca3_tile(const uint8_t *tile, int64_t n, int64_t side, const Rule &rule,
                                             uint8_t *__restrict__ out, int64_t x0, int64_t y0, int64_t z0,
                                             bool partial, int tx, int ty, int tz)
{
    constexpr int BW = RHO + 32, BH = RHO + 2;
    constexpr bool SWZ = (BW == 64);
    const int c = 1 + tx;  // staged chunk (chunk 0 is the left halo)
    // staged row r = zz * BH + yy holds x1 = z0 + zz - 1, x2 = y0 + yy - 1
    const int64_t xc = x0 + 16 * tx;
    const int64_t x2 = y0 + ty;
    const int zb = tz * RZ;  // first output plane of this thread
    uint32_t pp[4], pc[4], ac[4], lacc = 0;
    {
        uint32_t h0[4], h1[4], h2[4], cc[4];
        int r = zb * BH + ty;
        hsum_staged<BW, SWZ>(tile, r, c, h0, cc);
        hsum_staged<BW, SWZ>(tile, r + 1, c, h1, cc);
        hsum_staged<BW, SWZ>(tile, r + 2, c, h2, cc);
#pragma unroll
        for (int w = 0; w < 4; ++w) pp[w] = h0[w] + h1[w] + h2[w];
        r += BH;
        hsum_staged<BW, SWZ>(tile, r, c, h0, cc);
        hsum_staged<BW, SWZ>(tile, r + 1, c, h1, ac);
        hsum_staged<BW, SWZ>(tile, r + 2, c, h2, cc);
#pragma unroll
        for (int w = 0; w < 4; ++w) pc[w] = h0[w] + h1[w] + h2[w];
    }
#pragma unroll
    for (int i = 0; i < RZ; ++i) {
        uint32_t h0[4], h1[4], h2[4], cc[4], an[4], pn[4], s[4], nw[4];
        const int r = (zb + i + 2) * BH + ty;
        hsum_staged<BW, SWZ>(tile, r, c, h0, cc);
        hsum_staged<BW, SWZ>(tile, r + 1, c, h1, an);
        hsum_staged<BW, SWZ>(tile, r + 2, c, h2, cc);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            pn[w] = h0[w] + h1[w] + h2[w];
            s[w] = pp[w] + pc[w] + pn[w];
        }
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
        for (int w = 0; w < 4; ++w) {
            pp[w] = pc[w];
            pc[w] = pn[w];
            ac[w] = an[w];
        }
    }
    return byte_sum(lacc);
}

// m = 3, 32^3 tiles, box 64 x 34 x 34 bytes with the 64-byte swizzle.  Thread
// (ty, tz) owns the whole 32-cell row x2 = y0 + ty and walks RZ planes
// x1 = z0 + tz*RZ ... .  The Moore-27 sum (including the cell) is formed as
// h(V9): V9 is the 3 x 3 sum over (x2, x1) of each staged byte, built from
// column sums CY(plane) = row(x2-1) + row(x2) + row(x2+1) slid along x1, and h
// is one horizontal 3-sum over V9 (bytes stay <= 27).  Each staged row is read
// as its four 16-byte chunks; with the swizzle the 8 rows of an 8-lane phase
// hit distinct banks.
template <int RZ, bool ORK>
__device__ __forceinline__ uint32_t ca3_tile32(const uint8_t *tile, int64_t n, int64_t side, const Rule &rule,
                                               uint8_t *__restrict__ out, int64_t x0, int64_t y0, int64_t z0,
                                               bool partial, int ty, int tz)
{
    constexpr int BW = 64, BH = 34;
    const int zb = tz * RZ;  // first output plane (tile-local)
    // words 3 .. 12 of a staged row: the left halo word, the 8 tile words, the right halo word
    auto load_row = [&](int r, uint32_t v[10]) {
        const int sw = (r >> 1) & 3;
        const uint8_t *row = tile + r * BW;
        const uint4 c0 = *reinterpret_cast<const uint4 *>(row + 16 * (0 ^ sw));
        const uint4 c1 = *reinterpret_cast<const uint4 *>(row + 16 * (1 ^ sw));
        const uint4 c2 = *reinterpret_cast<const uint4 *>(row + 16 * (2 ^ sw));
        const uint4 c3 = *reinterpret_cast<const uint4 *>(row + 16 * (3 ^ sw));
        v[0] = c0.w;
        v[1] = c1.x; v[2] = c1.y; v[3] = c1.z; v[4] = c1.w;
        v[5] = c2.x; v[6] = c2.y; v[7] = c2.z; v[8] = c2.w;
        v[9] = c3.x;
    };
    // column sum over x2 - 1, x2, x2 + 1 of staged plane zz; `mid` receives the
    // middle row's 8 tile words (the cells themselves)
    auto col_sum = [&](int zz, uint32_t cy[10], uint32_t mid[8]) {
        uint32_t a[10], b[10], c[10];
        const int r = zz * BH + ty;
        load_row(r, a);
        load_row(r + 1, b);
        load_row(r + 2, c);
#pragma unroll
        for (int w = 0; w < 10; ++w) cy[w] = a[w] + b[w] + c[w];
#pragma unroll
        for (int w = 0; w < 8; ++w) mid[w] = b[w + 1];
    };
    uint32_t cp[10], cc[10], ac[8], tmp[8], lacc = 0;
    col_sum(zb, cp, tmp);
    col_sum(zb + 1, cc, ac);
    const int64_t x2 = y0 + ty;
#pragma unroll
    for (int i = 0; i < RZ; ++i) {
        uint32_t cn[10], an[8], v9[10], s[8], nw[8];
        col_sum(zb + i + 2, cn, an);
#pragma unroll
        for (int w = 0; w < 10; ++w) v9[w] = cp[w] + cc[w] + cn[w];
#pragma unroll
        for (int w = 0; w < 8; ++w)
            s[w] = v9[w + 1] + __funnelshift_l(v9[w], v9[w + 1], 8) + __funnelshift_r(v9[w + 1], v9[w + 2], 8);
        next_state4<ORK>(s, ac, rule, nw);
        next_state4<ORK>(s + 4, ac + 4, rule, nw + 4);
        const int64_t x1 = z0 + zb + i;
        uint8_t *dst = out + (x1 * side + x2) * side + x0;
        if (partial) {
            const int64_t c64 = n - x1 - x2 - x0 + 1;  // domain cells in this 32-cell row
            const int c = (int)(c64 < 0 ? 0 : (c64 > 32 ? 32 : c64));
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                nw[w] &= chunk_word_mask(c, w);
                nw[w + 4] &= chunk_word_mask(c - 16, w);
            }
            if (c > 0) store16(dst, nw);
            if (c > 16) store16(dst + 16, nw + 4);
        } else {
            store16(dst, nw);
            store16(dst + 16, nw + 4);
        }
        lacc += (nw[0] + nw[1]) + (nw[2] + nw[3]) + (nw[4] + nw[5]) + (nw[6] + nw[7]);  // bytes <= 8 RZ
#pragma unroll
        for (int w = 0; w < 10; ++w) {
            cp[w] = cc[w];
            cc[w] = cn[w];
        }
#pragma unroll
        for (int w = 0; w < 8; ++w) ac[w] = an[w];
    }
    return byte_sum(lacc);
}

}  // namespace sx
