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

// Raw bytes of chunk c of staged row r and the words just outside it: w[0] =
// last word of chunk c-1, w[1..4] = chunk c, w[5] = first word of chunk c+1.
template <int BW, bool SWZ>
__device__ __forceinline__ void load_chunk6(const uint8_t *tile, int r, int c, uint32_t w[6])
{
    const uint4 v = *reinterpret_cast<const uint4 *>(tile + chunk_off<BW, SWZ>(r, c));
    w[0] = *reinterpret_cast<const uint32_t *>(tile + chunk_off<BW, SWZ>(r, c - 1) + 12);
    w[1] = v.x;
    w[2] = v.y;
    w[3] = v.z;
    w[4] = v.w;
    w[5] = *reinterpret_cast<const uint32_t *>(tile + chunk_off<BW, SWZ>(r, c + 1));
}

// One tile's step from its staged box: thread (tx, ty, tz) owns the 16-byte
// chunk tx of row x2 = y0 + ty and walks RZ planes x1 = z0 + tz*RZ ... along
// x1.  The 27-sum (neighbours plus the cell) of a byte is h(V9): V9 is the
// 3 x 3 sum over (x2, x1) -- column sums CY(plane) = row(x2-1) + row(x2) +
// row(x2+1), slid along x1 -- and h one horizontal 3-sum over V9, using the
// V9 of the words next to the chunk for its edge bytes (bytes stay <= 27).
// Returns the live cells it wrote.
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
    auto col_sum = [&](int zz, uint32_t cy[6], uint32_t mid[4]) {
        uint32_t a[6], b[6], d[6];
        const int r = zz * BH + ty;
        load_chunk6<BW, SWZ>(tile, r, c, a);
        load_chunk6<BW, SWZ>(tile, r + 1, c, b);
        load_chunk6<BW, SWZ>(tile, r + 2, c, d);
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
#pragma unroll
        for (int w = 0; w < 4; ++w)
            s[w] = v9[w + 1] + __funnelshift_l(v9[w], v9[w + 1], 8) + __funnelshift_r(v9[w + 1], v9[w + 2], 8);
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

}  // namespace sx
