// k_init.cu -- seeded Bernoulli initial state of the automaton and the live
// count of a grid, both fused with the map H (one CUDA block per tile, chunks
// of 16 uint8 cells along x_m with one 16-byte access each).
#include "batch.h"
#include "common.cuh"
#include "hmap.cuh"
#include "kernels.h"
#include "tile.cuh"

namespace sx {

template <int M>
__global__ void __launch_bounds__(256) ca_init_kernel(const Plan p, uint8_t *__restrict__ grid, uint32_t seed,
                                                      uint32_t threshold, uint64_t nblocks,
                                                      unsigned long long *live)
{
    __shared__ uint32_t red[8];
    const uint32_t nchunks = 1u << (M * p.log_rho - 4);
    uint32_t my_live = 0;
    for (uint64_t v = blockIdx.x; v < nblocks; v += gridDim.x) {
        int32_t X[M];
        if (!decode<M>(p, kMapH, v, X)) continue;
        const int64_t s0 = tile_base_sum<M>(p, X);
        if (s0 > p.n) continue;
        const bool partial = s0 + (int64_t)M * (p.rho - 1) > p.n;
        for (uint32_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
            const ChunkPos<M> q = chunk_pos<M>(p, X, c, 4);
            if (partial && q.sum > p.n) continue;  // no domain cell in this chunk
            const uint32_t l0 = (uint32_t)q.lin;
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t word = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int cell = 4 * k + j;
                    const bool alive = splitmix32(seed ^ (l0 + (uint32_t)cell)) < threshold &&
                                       (!partial || q.sum + cell <= p.n);
                    word |= (alive ? 1u : 0u) << (8 * j);
                }
                w[k] = word;
                my_live += __popc(word);
            }
            store16(grid + q.addr, w);
        }
    }
    if (live) block_add_u64(live, my_live, red);
}

template <int M>
__global__ void __launch_bounds__(256) ca_count_kernel(const Plan p, const uint8_t *__restrict__ grid,
                                                       uint64_t nblocks, unsigned long long *live,
                                                       unsigned long long *digest)
{
    __shared__ uint32_t red[8];
    unsigned long long my_dig = 0;
    const uint32_t nchunks = 1u << (M * p.log_rho - 4);
    uint32_t my_live = 0;
    for (uint64_t v = blockIdx.x; v < nblocks; v += gridDim.x) {
        int32_t X[M];
        if (!decode<M>(p, kMapH, v, X)) continue;
        const int64_t s0 = tile_base_sum<M>(p, X);
        if (s0 > p.n) continue;
        const bool partial = s0 + (int64_t)M * (p.rho - 1) > p.n;
        for (uint32_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
            const ChunkPos<M> q = chunk_pos<M>(p, X, c, 4);
            if (partial && q.sum > p.n) continue;
            const uint4 g = *reinterpret_cast<const uint4 *>(grid + q.addr);
            const uint32_t w[4] = {g.x, g.y, g.z, g.w};
            const int64_t rem = p.n - q.sum + 1;
            const int cnt = partial ? (int)(rem < 16 ? rem : 16) : 16;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t wk = w[k] & chunk_word_mask(cnt, k);
                my_live += __popc(wk);
                if (digest) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if ((wk >> (8 * j)) & 1u)
                            my_dig += splitmix32(kDigestSalt ^ ((uint32_t)q.lin + (uint32_t)(4 * k + j)));
                }
            }
        }
    }
    if (live) block_add_u64(live, my_live, red);
    if (digest) {
        // 64-bit sum over the CTA's warps (partial warps included)
        const int lane = threadIdx.x & 31;
        const int in_warp = min(32, (int)blockDim.x - 32 * (int)(threadIdx.x >> 5));
        const uint32_t mask = in_warp == 32 ? 0xffffffffu : ((1u << in_warp) - 1u);
        unsigned long long w = my_dig;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_down_sync(mask, w, o);
            if (lane + o < in_warp) w += other;
        }
        if (lane == 0 && w) atomicAdd(digest, w);
    }
}

static unsigned grid_for(uint64_t nblocks)
{
    const uint64_t cap = 0x7fffffffull;
    return (unsigned)(nblocks < cap ? (nblocks ? nblocks : 1) : cap);
}

cudaError_t launch_ca_init(const Plan &p, uint8_t *grid, uint32_t seed, uint32_t threshold,
                           unsigned long long *live, cudaStream_t st)
{
    const uint64_t nchunks = 1ull << (p.m * p.log_rho - 4);
    const unsigned t = (unsigned)(nchunks < 256 ? nchunks : 256);
    const unsigned g = grid_for(p.h_blocks);
    switch (p.m) {
    case 2: ca_init_kernel<2><<<g, t, 0, st>>>(p, grid, seed, threshold, p.h_blocks, live); break;
    case 3: ca_init_kernel<3><<<g, t, 0, st>>>(p, grid, seed, threshold, p.h_blocks, live); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_ca_count(const Plan &p, const uint8_t *grid, unsigned long long *live, cudaStream_t st,
                            unsigned long long *digest)
{
    const uint64_t nchunks = 1ull << (p.m * p.log_rho - 4);
    const unsigned t = (unsigned)(nchunks < 256 ? nchunks : 256);
    const unsigned g = grid_for(p.h_blocks);
    switch (p.m) {
    case 2: ca_count_kernel<2><<<g, t, 0, st>>>(p, grid, p.h_blocks, live, digest); break;
    case 3: ca_count_kernel<3><<<g, t, 0, st>>>(p, grid, p.h_blocks, live, digest); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sx
