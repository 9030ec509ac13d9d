// tile.cuh -- cell coordinates of a chunk of consecutive cells inside a tile.
#pragma once

#include <stdint.h>

#include "hmap.cuh"

namespace sx {

// Chunk `c` of a tile, chunks of 2^lw cells along x_m (the memory axis),
// chunks ordered with x_m fastest.  For tile X it yields the linear index on
// side D = n + 1 (lin), the element offset on side `side` (addr) and the
// coordinate sum (s) of the chunk's first cell.
template <int M>
struct ChunkPos {
    int64_t lin, addr, sum;
};

template <int M>
__device__ __forceinline__ ChunkPos<M> chunk_pos(const Plan &p, const int32_t *X, uint32_t c, int lw)
{
    const int lr = p.log_rho;
    const int lcr = lr - lw;  // log2(chunks per tile row)
    int32_t t[M];
    t[M - 1] = (int32_t)((c & ((1u << lcr) - 1u)) << lw);
    uint32_t r = c >> lcr;
#pragma unroll
    for (int i = M - 2; i >= 0; --i) {
        t[i] = (int32_t)(r & (uint32_t)(p.rho - 1));
        r >>= lr;
    }
    const int64_t D = p.n + 1;
    ChunkPos<M> q{0, 0, 0};
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int64_t xi = (int64_t)X[i] * p.rho + t[i];
        q.lin = q.lin * D + xi;
        q.addr = q.addr * p.side + xi;
        q.sum += xi;
    }
    return q;
}

}  // namespace sx
