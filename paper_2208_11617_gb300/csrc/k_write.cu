// k_write.cu -- the coordinate-write test fused with the map (Table 1 test 2
// as a store-only kernel), the ACCUM test (Table 1: read, add, write) and the
// coverage (visit-count) kernels.
//
// One CUDA block per tile: the block decodes its tile with H (or the bounding
// box), and its threads write the tile's cells in chunks of 4 consecutive
// cells along x_m with one 16-byte store each.  Tiles that lie wholly inside
// the domain (rho * sum(X) + m (rho - 1) <= n) take the predicate-free path;
// only tiles on the diagonal band test each cell (Sec. 4.1: extra threads only
// at the diagonal).  (Programmatic dependent launch, which the automaton steps
// use, made the back-to-back 2.1 MB writes 20 to 40 % slower.)
#include "common.cuh"
#include "hmap.cuh"
#include "kernels.h"
#include "tile.cuh"

namespace sx {

// The tile of CUDA block v, the same value in every thread of the block.  For
// m >= 3 the generic decodes are long, so warp 0 decodes once and shares the
// result through sX (M + 1 ints of shared memory); m = 2 decodes in every
// thread (the Eq. map2d decode is a few instructions).  Every thread of the
// block must call it.
template <int M>
__device__ __forceinline__ bool block_decode(const Plan &p, int kind, uint64_t v, int32_t *X, int32_t *sX)
{
    if (M < 3) return decode<M>(p, kind, v, X);
    if (threadIdx.x < 32) {
        const bool ok = decode<M>(p, kind, v, X);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int i = 0; i < M; ++i) sX[i] = X[i];
            sX[M] = ok ? 1 : 0;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < M; ++i) X[i] = sX[i];
    const bool ok = sX[M] != 0;
    __syncthreads();  // sX is read by every thread before the next block rewrites it
    return ok;
}

template <int M>
__global__ void __launch_bounds__(256) write_kernel(const Plan p, uint32_t *__restrict__ out, uint32_t seed,
                                                    int kind, uint64_t nblocks, int vec)
{
    const uint32_t nchunks = 1u << (M * p.log_rho - 2);
    __shared__ int32_t sX[M + 1];  // block_decode's shared copy of the tile (m >= 3)
    // m >= 3: when a block's chunks (4 cells each) span whole x1-slabs of the
    // tile (rho^(m-1) cells), a thread's chunks c, c + blockDim.x, ... differ
    // only in x1: their positions follow from the first by three adds
    const int lslab = (M - 1) * p.log_rho;
    const uint32_t step_cells = blockDim.x * 4u;
    const bool stepped = M >= 3 && (step_cells & ((1u << lslab) - 1u)) == 0;
    for (uint64_t v = blockIdx.x; v < nblocks; v += gridDim.x) {
        int32_t X[M];
        if (!block_decode<M>(p, kind, v, X, sX)) continue;
        const int64_t s0 = tile_base_sum<M>(p, X);
        if (s0 > p.n && kind != kMapBBThread) continue;  // tile past the domain
        const bool partial = s0 + (int64_t)M * (p.rho - 1) > p.n;
        int64_t dx = 0, dlin = 0, daddr = 0;
        if (stepped) {
            dx = (int64_t)(step_cells >> lslab);
            dlin = dx;
            daddr = dx;
#pragma unroll
            for (int i = 0; i < M - 1; ++i) {
                dlin *= p.n + 1;
                daddr *= p.side;
            }
        }
        ChunkPos<M> q = chunk_pos<M>(p, X, threadIdx.x, 2);
        for (uint32_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
            if (M < 3 || (!stepped && c != threadIdx.x)) q = chunk_pos<M>(p, X, c, 2);
            const uint32_t l0 = (uint32_t)q.lin;
            if (M < 3) {
                // m = 2 (HBM-bound at full size): the two store forms apart
                if (!partial) {
                    const uint32_t h0 = splitmix32(seed ^ l0), h1 = splitmix32(seed ^ (l0 + 1u));
                    const uint32_t h2 = splitmix32(seed ^ (l0 + 2u)), h3 = splitmix32(seed ^ (l0 + 3u));
                    if (vec) {
                        *reinterpret_cast<uint4 *>(out + q.addr) = make_uint4(h0, h1, h2, h3);
                    } else {
                        out[q.addr] = h0;
                        out[q.addr + 1] = h1;
                        out[q.addr + 2] = h2;
                        out[q.addr + 3] = h3;
                    }
                } else {
                    // diagonal tile: most chunks lie wholly inside or outside the domain
                    const int64_t rem = p.n - q.sum + 1;  // cells of the chunk in the domain
                    if (rem >= 4 && vec) {
                        *reinterpret_cast<uint4 *>(out + q.addr) =
                            make_uint4(splitmix32(seed ^ l0), splitmix32(seed ^ (l0 + 1u)),
                                       splitmix32(seed ^ (l0 + 2u)), splitmix32(seed ^ (l0 + 3u)));
                    } else if (rem > 0) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (j < rem) out[q.addr + j] = splitmix32(seed ^ (l0 + (uint32_t)j));
                    }
                }
            } else {
                // m >= 3 (instruction-bound): cells of the chunk in the domain,
                // 4 off the diagonal band; one hash sequence for every lane
                // with a cell, so a warp whose chunks straddle the diagonal
                // hashes once, not once per store form (7 % faster for the
                // m = 4 write)
                const int64_t rem = partial ? p.n - q.sum + 1 : 4;
                if (rem > 0) {
                    const uint32_t h0 = splitmix32(seed ^ l0), h1 = splitmix32(seed ^ (l0 + 1u));
                    const uint32_t h2 = splitmix32(seed ^ (l0 + 2u)), h3 = splitmix32(seed ^ (l0 + 3u));
                    uint32_t *dst = out + q.addr;
                    if (rem >= 4 && vec) {
                        *reinterpret_cast<uint4 *>(dst) = make_uint4(h0, h1, h2, h3);
                    } else {
                        dst[0] = h0;
                        if (rem > 1) dst[1] = h1;
                        if (rem > 2) dst[2] = h2;
                        if (rem > 3) dst[3] = h3;
                    }
                }
            }
            if (M >= 3) {
                q.lin += dlin;
                q.addr += daddr;
                q.sum += dx;
            }
        }
    }
}

// Write test for m >= 3, one warp per tile: the grid holds kWarpsPerCta warps
// per CTA and each warp takes tiles v = global warp index, + total warps, ...
// Every lane runs the tile's decode itself (the decode is uniform across the
// warp), so there is no barrier between decode and stores and a CTA never
// waits for one of its warps; the warps of an SM overlap one tile's decode
// with other tiles' stores.  Chunk positions come from per-tile bases: the
// hashed row-major index lin (mod 2^32, 32-bit arithmetic) and the element
// offset (64-bit), plus the chunk's offsets inside the tile.
constexpr int kWriteWarps = 8;

template <int M>
__global__ void __launch_bounds__(32 * kWriteWarps) write_kernel_w(const Plan p, uint32_t *__restrict__ out,
                                                                   uint32_t seed, int kind, uint64_t nblocks,
                                                                   int vec)
{
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = 1u << (M * p.log_rho - 2);
    const int lr = p.log_rho, lcr = lr - 2;  // log2(chunks per tile row)
    // strides of axis i: along the array (side^(M-1-i)) and along lin ((n+1)^(M-1-i) mod 2^32)
    int64_t sa[M];
    uint32_t sl[M];
    sa[M - 1] = 1;
    sl[M - 1] = 1u;
#pragma unroll
    for (int i = M - 2; i >= 0; --i) {
        sa[i] = sa[i + 1] * p.side;
        sl[i] = sl[i + 1] * (uint32_t)(p.n + 1);
    }
    const uint64_t stride = (uint64_t)gridDim.x * kWriteWarps;
    for (uint64_t v = (uint64_t)blockIdx.x * kWriteWarps + (threadIdx.x >> 5); v < nblocks; v += stride) {
        int32_t X[M];
        if (!decode<M>(p, kind, v, X)) continue;
        const int64_t s0 = tile_base_sum<M>(p, X);
        if (s0 > p.n && kind != kMapBBThread) continue;  // tile past the domain
        const bool partial = s0 + (int64_t)M * (p.rho - 1) > p.n;
        int64_t abase = 0;
        uint32_t lbase = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            abase += (int64_t)X[i] * p.rho * sa[i];
            lbase += (uint32_t)X[i] * (uint32_t)p.rho * sl[i];
        }
        for (uint32_t c = lane; c < nchunks; c += 32) {
            // offsets of chunk c inside the tile (x_M fastest, 4 cells per chunk)
            int32_t t[M];
            t[M - 1] = (int32_t)((c & ((1u << lcr) - 1u)) << 2);
            uint32_t r = c >> lcr;
#pragma unroll
            for (int i = M - 2; i >= 0; --i) {
                t[i] = (int32_t)(r & (uint32_t)(p.rho - 1));
                r >>= lr;
            }
            int64_t addr = abase;
            uint32_t l0 = lbase;
            int32_t tsum = 0;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                addr += (int64_t)t[i] * sa[i];
                l0 += (uint32_t)t[i] * sl[i];
                tsum += t[i];
            }
            // cells of the chunk in the domain (4 off the diagonal band), one
            // hash sequence for every store form as in write_kernel
            const int64_t rem = partial ? p.n - (s0 + tsum) + 1 : 4;
            if (rem > 0) {
                const uint32_t h0 = splitmix32(seed ^ l0), h1 = splitmix32(seed ^ (l0 + 1u));
                const uint32_t h2 = splitmix32(seed ^ (l0 + 2u)), h3 = splitmix32(seed ^ (l0 + 3u));
                uint32_t *dst = out + addr;
                if (rem >= 4 && vec) {
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(h0, h1, h2, h3);
                } else {
                    dst[0] = h0;
                    if (rem > 1) dst[1] = h1;
                    if (rem > 2) dst[2] = h2;
                    if (rem > 3) dst[3] = h3;
                }
            }
        }
    }
}

// ACCUM (Table 1): every domain cell of `data` gains `add` (mod 2^32).  Same
// decode and chunking as the write test; a chunk is one 16-byte load, four
// adds and one 16-byte store (4-byte accesses where rows are not 16-byte
// aligned, and per cell on the diagonal band).  With G = 4 a thread issues
// the loads of four of its chunks before their stores (used when every thread
// has at least four chunks; with one chunk per thread the extra registers
// cost more occupancy than the loads in flight gain).
template <int M, int G>
__global__ void __launch_bounds__(256) accum_kernel(const Plan p, uint32_t *__restrict__ data, uint32_t add,
                                                    int kind, uint64_t nblocks, int vec)
{
    const uint32_t nchunks = 1u << (M * p.log_rho - 2);
    __shared__ int32_t sX[M + 1];  // block_decode's shared copy of the tile (m >= 3)
    for (uint64_t v = blockIdx.x; v < nblocks; v += gridDim.x) {
        int32_t X[M];
        if (!block_decode<M>(p, kind, v, X, sX)) continue;
        const int64_t s0 = tile_base_sum<M>(p, X);
        if (s0 > p.n && kind != kMapBBThread) continue;
        const bool partial = s0 + (int64_t)M * (p.rho - 1) > p.n;
        if (G > 1 && !partial && vec) {
            // G chunks per thread at a time: their loads are all in flight
            // before the first store
            for (uint32_t c0 = threadIdx.x; c0 < nchunks; c0 += G * blockDim.x) {
                uint4 w[G];
                int64_t a[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const uint32_t c = c0 + (uint32_t)g * blockDim.x;
                    a[g] = c < nchunks ? chunk_pos<M>(p, X, c, 2).addr : -1;
                    if (a[g] >= 0) w[g] = *reinterpret_cast<const uint4 *>(data + a[g]);
                }
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (a[g] >= 0)
                        *reinterpret_cast<uint4 *>(data + a[g]) =
                            make_uint4(w[g].x + add, w[g].y + add, w[g].z + add, w[g].w + add);
            }
            continue;
        }
        for (uint32_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
            const ChunkPos<M> q = chunk_pos<M>(p, X, c, 2);
            if (!partial && vec) {
                uint4 w = *reinterpret_cast<const uint4 *>(data + q.addr);
                w.x += add;
                w.y += add;
                w.z += add;
                w.w += add;
                *reinterpret_cast<uint4 *>(data + q.addr) = w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (!partial || q.sum + j <= p.n) data[q.addr + j] += add;
            }
        }
    }
}

template <int M>
__global__ void __launch_bounds__(256) visit_kernel(const Plan p, uint32_t *__restrict__ counts, int level,
                                                    int kind, uint64_t nblocks)
{
    const uint32_t nchunks = 1u << (M * p.log_rho - 2);
    const int64_t nb = (p.n + p.rho) / p.rho;
    for (uint64_t v = blockIdx.x; v < nblocks; v += gridDim.x) {
        int32_t X[M];
        if (!decode<M>(p, kind, v, X)) continue;
        const int64_t s0 = tile_base_sum<M>(p, X);
        if (s0 > p.n) continue;
        if (level == 0) {
            if (threadIdx.x == 0) {
                int64_t b = 0;
#pragma unroll
                for (int i = 0; i < M; ++i) b = b * nb + X[i];
                atomicAdd(counts + b, 1u);
            }
            continue;
        }
        const bool partial = s0 + (int64_t)M * (p.rho - 1) > p.n;
        for (uint32_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
            const ChunkPos<M> q = chunk_pos<M>(p, X, c, 2);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (!partial || q.sum + j <= p.n) atomicAdd(counts + q.addr + j, 1u);
        }
    }
}

static unsigned grid_for(uint64_t nblocks)
{
    const uint64_t cap = 0x7fffffffull;
    return (unsigned)(nblocks < cap ? (nblocks ? nblocks : 1) : cap);
}

static unsigned threads_for(const Plan &p, int lw)
{
    const uint64_t nchunks = 1ull << (p.m * p.log_rho - lw);
    return (unsigned)(nchunks < 256 ? nchunks : 256);
}

cudaError_t launch_write(const Plan &plan, uint32_t *out, uint32_t seed, int kind, bool vec, cudaStream_t st)
{
    const Plan p = single_grid(plan);
    const uint64_t nb = is_bb(kind) ? p.bb_blocks : p.h_blocks;
    const unsigned g = grid_for(nb), t = threads_for(p, 2);
    // m >= 3: tiles of fewer than 256 chunks one per warp (kWriteWarps per
    // CTA: 1.8x faster for 4^4 tiles); larger ones one per CTA (a warp per
    // tile, or persistent CTAs decoding the next tile ahead, were 1.4x slower
    // for 8^4 tiles).  m = 4 CTAs have 128 threads: with the per-thread
    // position steps (a thread's 8 chunks then lie in consecutive x1-slabs)
    // 1.22x faster than 256 threads, and the bounding box's mostly empty CTAs
    // retire 1.3x faster (64 threads: 13 % slower)
    const bool small = (1ull << (p.m * p.log_rho - 2)) < 256;
    const unsigned gw = grid_for((nb + kWriteWarps - 1) / kWriteWarps);
    switch (p.m * 2 + (small ? 1 : 0)) {
    case 4:
    case 5: write_kernel<2><<<g, t, 0, st>>>(p, out, seed, kind, nb, vec ? 1 : 0); break;
    case 6: write_kernel<3><<<g, t, 0, st>>>(p, out, seed, kind, nb, vec ? 1 : 0); break;
    case 7: write_kernel_w<3><<<gw, 32 * kWriteWarps, 0, st>>>(p, out, seed, kind, nb, vec ? 1 : 0); break;
    case 8: write_kernel<4><<<g, t < 128u ? t : 128u, 0, st>>>(p, out, seed, kind, nb, vec ? 1 : 0); break;
    case 9: write_kernel_w<4><<<gw, 32 * kWriteWarps, 0, st>>>(p, out, seed, kind, nb, vec ? 1 : 0); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_accum(const Plan &plan, uint32_t *data, uint32_t add, int kind, bool vec, cudaStream_t st)
{
    const Plan p = single_grid(plan);
    const uint64_t nb = is_bb(kind) ? p.bb_blocks : p.h_blocks;
    const unsigned g = grid_for(nb), t = threads_for(p, 2);
    const int vc = vec ? 1 : 0;
    const bool grouped = (1ull << (p.m * p.log_rho - 2)) >= 4ull * t;  // >= 4 chunks per thread
    switch (p.m * 10 + (grouped ? 4 : 1)) {
    case 21: accum_kernel<2, 1><<<g, t, 0, st>>>(p, data, add, kind, nb, vc); break;
    case 24: accum_kernel<2, 4><<<g, t, 0, st>>>(p, data, add, kind, nb, vc); break;
    case 31: accum_kernel<3, 1><<<g, t, 0, st>>>(p, data, add, kind, nb, vc); break;
    case 34: accum_kernel<3, 4><<<g, t, 0, st>>>(p, data, add, kind, nb, vc); break;
    case 41: accum_kernel<4, 1><<<g, t, 0, st>>>(p, data, add, kind, nb, vc); break;
    case 44: accum_kernel<4, 4><<<g, t, 0, st>>>(p, data, add, kind, nb, vc); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_visit(const Plan &p, uint32_t *counts, int level, int kind, cudaStream_t st)
{
    const uint64_t nb = is_bb(kind) ? p.bb_blocks : p.h_blocks;
    const unsigned g = grid_for(nb), t = threads_for(p, 2);
    switch (p.m) {
    case 2: visit_kernel<2><<<g, t, 0, st>>>(p, counts, level, kind, nb); break;
    case 3: visit_kernel<3><<<g, t, 0, st>>>(p, counts, level, kind, nb); break;
    case 4: visit_kernel<4><<<g, t, 0, st>>>(p, counts, level, kind, nb); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sx
