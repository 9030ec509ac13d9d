// k_batch.cu -- the batched automaton engine: one persistent launch per step
// over every instance of a batch, fed by a device-side work queue.
//
// The work of a step is the union of the CUDA blocks of every instance's map
// (H in its trapezoid form for m = 2, H3 with the hinge for m = 3), cut into
// work items of up to kBatchChunk consecutive blocks of one instance.  Each
// CTA pops items from a global counter (one atomic per item; the next pop is
// issued while the current item runs), loads the item's instance description
// into shared memory when it changes, decodes each block with that instance's
// map and runs the same per-tile body as the single-instance kernels.
//
// Consecutive passes are launched with programmatic stream serialization: a
// pass starts while the one before it drains, pops its first item, loads the
// instance description and decodes the item's blocks (none of which the
// previous pass writes), and waits for the previous pass to complete only
// before its first access to a grid.  A CTA lets the next pass start once it
// has got past that wait and holds its last item, so at most one pass runs
// ahead.
#include <mutex>

#include "../../include/simplex.h"
#include "batch.h"
#include "ca_tiles.cuh"
#include "common.cuh"
#include "hmap.cuh"
#include "host.h"
#include "kernels.h"
#include "tile.cuh"

namespace sx {

static __device__ uint32_t g_batch_status;
static_assert(kBatchChunk <= 32, "one lane of warp 0 decodes each block of an item");

// Launch sets: set 0 runs the m = 2 bodies and the 16^3 body in 20.8 KB of
// stage (8 CTAs per SM), set 1 the 32^3 body of m = 3 in a 74 KB stage with the
// 64-byte swizzle (3 CTAs per SM).
// Set 0 double-buffers its stage: the TMA load of an item's next tile is in
// flight while the CTA computes the current one.
constexpr int kBatchStageBytes = 160 * 130;  // largest box of set 0: m = 2, 128 x 128 tiles
constexpr int kBatchStage3x32 = 64 * 34 * 34;
__host__ __device__ constexpr int batch_stages(int set) { return set ? 1 : 2; }
__host__ __device__ constexpr int batch_stage_pitch(int set) { return set ? (kBatchStage3x32 + 511) / 512 * 512 : (kBatchStageBytes + 127) / 128 * 128; }
__host__ __device__ constexpr int batch_smem(int set) { return batch_stages(set) * batch_stage_pitch(set) + (set ? 512 : 128); }

__device__ __forceinline__ uint32_t body_box_bytes(int body)
{
    return body == kBody2x64    ? 96u * 66u
           : body == kBody2x128 ? 160u * 130u
           : body == kBody3x16  ? 48u * 18u * 18u
                                : (uint32_t)kBatchStage3x32;
}

// Live cells of one tile of grid `g`, read straight from global memory in
// 16-cell chunks (the count pass that gives live[0]); with `dig` it also sums
// splitmix32(kDigestSalt ^ lin(x)) over the live cells into *dig.
template <int M>
__device__ __forceinline__ uint32_t count_tile(const Plan &p, const int32_t *X, const uint8_t *g, bool partial,
                                               unsigned long long *dig_acc)
{
    const uint32_t nchunks = 1u << (M * p.log_rho - 4);
    uint32_t c_live = 0;
    unsigned long long d = 0;
    for (uint32_t c = threadIdx.x; c < nchunks; c += blockDim.x) {
        const ChunkPos<M> q = chunk_pos<M>(p, X, c, 4);
        if (partial && q.sum > p.n) continue;
        const uint4 w = *reinterpret_cast<const uint4 *>(g + q.addr);
        const int64_t rem = p.n - q.sum + 1;
        const int cnt = partial ? (int)(rem < 16 ? rem : 16) : 16;
        const uint32_t ww[4] = {w.x & chunk_word_mask(cnt, 0), w.y & chunk_word_mask(cnt, 1),
                                w.z & chunk_word_mask(cnt, 2), w.w & chunk_word_mask(cnt, 3)};
        c_live += __popc(ww[0]) + __popc(ww[1]) + __popc(ww[2]) + __popc(ww[3]);
        if (dig_acc) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if ((ww[j >> 2] >> (8 * (j & 3))) & 1u) d += splitmix32(kDigestSalt ^ ((uint32_t)q.lin + (uint32_t)j));
        }
    }
    if (dig_acc) *dig_acc += d;
    return c_live;
}

template <int SET>
__global__ void __launch_bounds__(kBatchThreads, SET ? 3 : 5)
    batch_kernel(const BatchInst *__restrict__ insts, const BatchItem *__restrict__ items, uint32_t nitems,
                 const CUtensorMap *__restrict__ tmaps, uint8_t *__restrict__ arena, int in_parity,
                 unsigned int *__restrict__ queue, unsigned long long *__restrict__ live, int live_stride,
                 int live_index, int count_only, unsigned long long *__restrict__ digest, int pass)
{
    constexpr int NST = batch_stages(SET), kPitch = batch_stage_pitch(SET);
    extern __shared__ uint8_t dsmem[];
    __shared__ BatchInst si;
    __shared__ __align__(8) uint64_t bar[NST];
    __shared__ uint32_t red[32];
    __shared__ uint32_t s_item, s_next;
    __shared__ int s_cur, s_ntiles;
    __shared__ int4 s_tiles[kBatchChunk];  // the item's tiles with cells: X[0..2], partial
    constexpr uintptr_t kAlign = SET ? 512 : 128;
    uint8_t *tile = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + kAlign - 1) & ~(kAlign - 1));
    // stage s at tile + s * kPitch
    const int tid = threadIdx.x;
    uint32_t phase = 0;  // bit s: parity of stage s's next completion
    bool waited = false, triggered = false;  // CTA-uniform

    if (tid == 0) {
        for (int k = 0; k < NST; ++k) mbar_init(&bar[k], 1);
        fence_mbar_init();
        s_cur = -1;
        s_next = atomicAdd(queue, 1u);
    }
    __syncthreads();

    for (;;) {
        if (tid == 0) {
            s_item = s_next;
            if (s_item < nitems) s_next = atomicAdd(queue, 1u);  // prefetch the next pop
        }
        __syncthreads();
        const uint32_t it = s_item;
        if (!triggered && waited && s_next >= nitems) {  // the CTA's last item: the next pass may start
            grid_dep_trigger();
            triggered = true;
        }
        if (it >= nitems) break;
        const BatchItem item = items[it];
        // item.tag: bit 0 flips the input grid, bits 1..12 offset the live-count
        // index, bits 13..18 + 1 = passes the item takes part in (pass p of a
        // multi-step launch sequence reads grid parity ^ p and counts at index + p)
        if ((uint32_t)pass > ((item.tag >> 13) & 63u)) {  // uniform: the job has no step left in this pass
            __syncthreads();  // s_item is read by every thread before thread 0 pops the next item
            continue;
        }
        if ((int)item.inst != s_cur) {
            // load the instance description into shared memory (all threads)
            const uint32_t *src = reinterpret_cast<const uint32_t *>(insts + item.inst);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&si);
            for (int w = tid; w < (int)(sizeof(BatchInst) / 4); w += kBatchThreads) dst[w] = src[w];
            __syncthreads();
            if (tid == 0) {
                s_cur = (int)item.inst;
                if (!count_only) prefetch_tmap(tmaps + si.tmap + (in_parity ^ (int)((item.tag ^ (uint32_t)pass) & 1u)));
            }
        }
        const Plan &p = si.plan;
        const int par = in_parity ^ (int)((item.tag ^ (uint32_t)pass) & 1u);
        const uint8_t *gin = arena + si.grid[par];
        uint8_t *gout = arena + si.grid[par ^ 1];
        uint32_t my_live = 0;
        unsigned long long my_dig = 0;
        if (count_only) {
            if (!waited) {  // the grid may still be written by the previous pass
                grid_dep_wait();
                waited = true;
                if (s_next >= nitems) {  // the CTA's last item: the next pass may start
                    grid_dep_trigger();
                    triggered = true;
                }
            }
            for (uint32_t j = 0; j < item.cnt; ++j) {
                int32_t X[3] = {0, 0, 0};
                const uint64_t v = (uint64_t)item.v0 + j;
                if (!(p.m == 2 ? decode<2>(p, kMapH, v, X) : decode<3>(p, kMapH, v, X))) continue;
                const int64_t s0 = tile_base_sum<3>(p, X);  // X[2] = 0 for m = 2
                if (s0 > p.n) continue;
                const bool partial = s0 + (int64_t)p.m * (p.rho - 1) > p.n;
                unsigned long long *acc = digest ? &my_dig : nullptr;
                my_live += p.m == 2 ? count_tile<2>(p, X, gin, partial, acc) : count_tile<3>(p, X, gin, partial, acc);
            }
        } else if ((si.body == kBody3x32) != (SET == 1)) {  // an item of the other launch set: not run here
            if (tid == 0) atomicOr(&g_batch_status, 2u);
        } else {
            // the item's tiles that hold cells (lane j of warp 0 decodes block
            // v0 + j; a ballot keeps them in block order), then a pipelined
            // walk over them
            if (tid < 32) {
                int4 t = make_int4(0, 0, 0, 0);
                bool hold = false;
                if ((uint32_t)tid < item.cnt && tid < kBatchChunk) {
                    int32_t X[3] = {0, 0, 0};
                    const uint64_t v = (uint64_t)item.v0 + (uint64_t)tid;
                    if (p.m == 2 ? decode<2>(p, kMapH, v, X) : decode<3>(p, kMapH, v, X)) {
                        const int64_t s0 = tile_base_sum<3>(p, X);
                        hold = s0 <= p.n;
                        t = make_int4(X[0], X[1], X[2], s0 + (int64_t)p.m * (p.rho - 1) > p.n ? 1 : 0);
                    }
                }
                const uint32_t held = __ballot_sync(0xffffffffu, hold);
                if (hold) s_tiles[__popc(held & ((1u << tid) - 1u))] = t;
                if (tid == 0) s_ntiles = __popc(held);
            }
            __syncthreads();
            if (!waited) {  // the previous pass writes this pass's input and reads its output
                grid_dep_wait();
                waited = true;
                if (s_next >= nitems) {  // the CTA's last item: the next pass may start
                    grid_dep_trigger();
                    triggered = true;
                }
            }
            const int nt = s_ntiles;
            const uint32_t box = body_box_bytes(si.body);
            const CUtensorMap *tm = tmaps + si.tmap + par;
            auto issue = [&](int k) {  // thread 0: load tile k into stage k % NST
                const int st = k % NST;
                const int4 t = s_tiles[k];
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar[st], box);
                if (p.m == 2)
                    tma_load_2d(tile + st * kPitch, tm, t.y * p.rho - 16, t.x * p.rho - 1, &bar[st]);
                else
                    tma_load_3d(tile + st * kPitch, tm, t.z * p.rho - 16, t.y * p.rho - 1, t.x * p.rho - 1, &bar[st]);
            };
            if (tid == 0)
                for (int k = 0; k < NST && k < nt; ++k) issue(k);
            for (int k = 0; k < nt; ++k) {
                const int st = k % NST;
                const bool done = mbar_wait_bounded(&bar[st], (phase >> st) & 1u, kWaitLimitNs);
                phase ^= 1u << st;
                if (__syncthreads_or(!done)) {
                    if (tid == 0) {
                        atomicOr(&g_batch_status, 1u);
                        // every load still in flight must land before the CTA exits
                        mbar_wait_bounded(&bar[st], ((phase >> st) & 1u) ^ 1u, kWaitLimitNs);
                        for (int k2 = k + 1; k2 < nt && k2 < k + NST; ++k2)
                            mbar_wait_bounded(&bar[k2 % NST], (phase >> (k2 % NST)) & 1u, kWaitLimitNs);
                    }
                    return;
                }
                const int4 t = s_tiles[k];
                const int32_t X[3] = {t.x, t.y, t.z};
                const bool partial = t.w != 0;
                const uint8_t *stile = tile + st * kPitch;
                const bool ork = si.rule.or_k != 0;
                if constexpr (SET == 1) {
                    const int64_t z0 = (int64_t)X[0] * 32, y0 = (int64_t)X[1] * 32, x0 = (int64_t)X[2] * 32;
                    my_live += ork ? ca3_tile32<8, true>(stile, p.n, p.side, si.rule, gout, x0, y0, z0, partial,
                                                         tid & 1, (tid >> 1) & 15, tid >> 5)
                                   : ca3_tile32<8, false>(stile, p.n, p.side, si.rule, gout, x0, y0, z0, partial,
                                                          tid & 1, (tid >> 1) & 15, tid >> 5);
                } else {
                    switch (si.body) {
                    case kBody2x64:
                        my_live += ork ? ca2_tile<64, 2, true>(stile, p.n, p.side, si.rule, gout, (int64_t)X[1] * 64,
                                                               (int64_t)X[0] * 64, partial, tid & 3, tid >> 2)
                                       : ca2_tile<64, 2, false>(stile, p.n, p.side, si.rule, gout, (int64_t)X[1] * 64,
                                                                (int64_t)X[0] * 64, partial, tid & 3, tid >> 2);
                        break;
                    case kBody2x128:
                        my_live += ork ? ca2_tile<128, 8, true>(stile, p.n, p.side, si.rule, gout,
                                                                (int64_t)X[1] * 128, (int64_t)X[0] * 128, partial,
                                                                tid & 7, tid >> 3)
                                       : ca2_tile<128, 8, false>(stile, p.n, p.side, si.rule, gout,
                                                                 (int64_t)X[1] * 128, (int64_t)X[0] * 128, partial,
                                                                 tid & 7, tid >> 3);
                        break;
                    default:
                        my_live += ork ? ca3_tile<16, 2, true>(stile, p.n, p.side, si.rule, gout, (int64_t)X[2] * 16,
                                                               (int64_t)X[1] * 16, (int64_t)X[0] * 16, partial, 0,
                                                               tid & 15, tid >> 4)
                                       : ca3_tile<16, 2, false>(stile, p.n, p.side, si.rule, gout,
                                                                (int64_t)X[2] * 16, (int64_t)X[1] * 16,
                                                                (int64_t)X[0] * 16, partial, 0, tid & 15, tid >> 4);
                        break;
                    }
                }
                __syncthreads();  // stage st fully read before it is loaded again
                if (tid == 0 && k + NST < nt) issue(k + NST);
            }
        }
        if (live)
            block_add_u64(live + (uint64_t)item.inst * live_stride + live_index + ((item.tag >> 1) & 0xfffu) + pass,
                          my_live, red);
        if (digest) {
            unsigned long long w = my_dig;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
            if ((tid & 31) == 0 && w) atomicAdd(digest + item.inst, w);
        }
        __syncthreads();
    }
}

// Flat m = 2 pass: one CTA per block of every m = 2 instance's map that holds
// cells (tiles[blockIdx.x] names the instance and the block), the launch model
// of the single-instance step: the CTA decodes its block with the instance's H
// (trapezoid form), stages the tile plus halo with one TMA load and runs the
// instance's tile body (64^2 or 128^2).  Consecutive passes are launched with
// programmatic stream serialization: a CTA decodes before it waits for the
// previous pass, and lets the next one start once past that wait.
constexpr int kFlatStage = 160 * 130;  // the 128 x 128 box, the larger of the two bodies

__global__ void __launch_bounds__(kBatchThreads, 10)
    batch_flat2_kernel(const BatchInst *__restrict__ insts, const BatchTile *__restrict__ tiles,
                       const CUtensorMap *__restrict__ tmaps, uint8_t *__restrict__ arena, int in_parity,
                       unsigned long long *__restrict__ live, int live_stride, int live_index)
{
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t red[32];
    uint8_t *tile = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x;
    const BatchTile bt = tiles[blockIdx.x];
    const BatchInst &bi = insts[bt.inst];
    const Plan &p = bi.plan;
    int32_t X[2] = {0, 0};
    const bool ok_map = decode<2>(p, kMapH, bt.v, X);
    const int rho = p.rho;
    const int64_t y0 = (int64_t)X[0] * rho, x0 = (int64_t)X[1] * rho;
    const bool partial = y0 + x0 + 2 * (rho - 1) > p.n;
    const int64_t n = p.n, side = p.side;
    const CUtensorMap *tm = tmaps + bi.tmap + in_parity;
    uint8_t *gout = arena + bi.grid[in_parity ^ 1];
    const bool body128 = bi.body == kBody2x128;
    if (tid == 0) {
        prefetch_tmap(tm);
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    grid_dep_wait();     // the previous pass writes this pass's input and reads its output
    grid_dep_trigger();  // the next pass may start (at most one pass ahead)
    if (!ok_map || y0 + x0 > n) return;  // never listed: every tile of the table holds cells
    if (tid == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar, body128 ? 160u * 130u : 96u * 66u);
        tma_load_2d(tile, tm, (int32_t)(x0 - 16), (int32_t)(y0 - 1), &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0u, kWaitLimitNs);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicOr(&g_batch_status, 4u);
            mbar_wait_bounded(&bar, 0u, kWaitLimitNs);
        }
        return;
    }
    const bool ork = bi.rule.or_k != 0;
    uint32_t my_live;
    if (body128)
        my_live = ork ? ca2_tile<128, 8, true>(tile, n, side, bi.rule, gout, x0, y0, partial, tid & 7, tid >> 3)
                      : ca2_tile<128, 8, false>(tile, n, side, bi.rule, gout, x0, y0, partial, tid & 7, tid >> 3);
    else
        my_live = ork ? ca2_tile<64, 2, true>(tile, n, side, bi.rule, gout, x0, y0, partial, tid & 3, tid >> 2)
                      : ca2_tile<64, 2, false>(tile, n, side, bi.rule, gout, x0, y0, partial, tid & 3, tid >> 2);
    if (live)
        block_add_u64(live + (uint64_t)bt.inst * (uint64_t)live_stride + (uint64_t)live_index, my_live, red);
}

cudaError_t launch_batch_flat2(const BatchInst *insts, const BatchTile *tiles, uint32_t ntiles,
                               const CUtensorMap *tmaps, uint8_t *arena, int in_parity, unsigned long long *live,
                               int live_stride, int live_index, cudaStream_t st)
{
    if (!ntiles) return cudaSuccess;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    constexpr int smem = kFlatStage + 128;
    if (!(dev >= 0 && dev < 64 && attr_set[dev])) {
        e = cudaFuncSetAttribute(batch_flat2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    return launch_pdl(batch_flat2_kernel, dim3(ntiles), dim3(kBatchThreads), (size_t)smem, st, insts, tiles, tmaps,
                      arena, in_parity, live, live_stride, live_index);
}

cudaError_t batch_prepare()
{
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(batch_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem(0));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem(1));
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

// Resident CTAs of the persistent launch of set `set` on the current device
// (SM count x occupancy), looked up once per device.
cudaError_t batch_resident_ctas(uint64_t *out, int set)
{
    static uint64_t cached[2][64] = {};
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    set = set ? 1 : 0;
    if (dev >= 0 && dev < 64 && cached[set][dev]) {
        *out = cached[set][dev];
        return cudaSuccess;
    }
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = set ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<1>, kBatchThreads, batch_smem(1))
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<0>, kBatchThreads, batch_smem(0));
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    *out = (uint64_t)sms * (uint64_t)per_sm;
    if (dev >= 0 && dev < 64) cached[set][dev] = *out;
    return cudaSuccess;
}

cudaError_t launch_batch_pass(const BatchInst *insts, const BatchItem *items, uint32_t nitems,
                              const CUtensorMap *tmaps, uint8_t *arena, int in_parity, unsigned int *queue,
                              unsigned long long *live, int live_stride, int live_index, bool count_only,
                              cudaStream_t st, unsigned long long *digest, int set, int pass)
{
    cudaError_t e = batch_prepare();
    if (e != cudaSuccess) return e;
    set = (set && !count_only) ? 1 : 0;
    uint64_t g = 0;
    if ((e = batch_resident_ctas(&g, set)) != cudaSuccess) return e;  // persistent: every CTA resident
    if (g > nitems) g = nitems ? nitems : 1;
    // programmatic stream serialization: the pass may start while the kernel
    // before it drains (the kernel waits before it touches a grid)
    const int co = count_only ? 1 : 0;
    if (set)
        return launch_pdl(batch_kernel<1>, dim3((unsigned)g), dim3(kBatchThreads), (size_t)batch_smem(1), st, insts,
                          items, nitems, tmaps, arena, in_parity, queue, live, live_stride, live_index, 0, digest,
                          pass);
    return launch_pdl(batch_kernel<0>, dim3((unsigned)g), dim3(kBatchThreads), (size_t)batch_smem(0), st, insts,
                      items, nitems, tmaps, arena, in_parity, queue, live, live_stride, live_index, co, digest, pass);
}

cudaError_t batch_read_status(uint32_t *out)
{
    uint32_t zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_batch_status, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_batch_status, &zero, sizeof(uint32_t));
}

}  // namespace sx

// ---------------------------------------------------------------------------
// Allocation-free batched run.
//
// simplex_batch_run needs an arena from the caller for the batch's descriptors,
// work items, TMA maps and work-queue counters.  Some callers cannot provide
// one: a host that owns every byte of device memory through its own pool or
// budget and hands libraries fixed buffers only, or a latency-critical loop
// that must not pay for an allocator call (cudaMalloc can synchronise the
// device) on its hot path.  For them the scratch lives in this fixed-size
// array instead; the caller passes only the grids (the inputs and outputs).
// The array exists once per device that loads the library and stays allocated
// until the process exits.
namespace sx {

constexpr uint64_t kStaticScratchBytes = 8ull << 20;  // 8 MiB

static __device__ __align__(256) uint8_t g_batch_static_scratch[kStaticScratchBytes];

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress with that device current), and what the
// array holds there: the batch (its serial) and grids whose descriptors, work
// items and tensor maps the last complete upload put in.  Guarded by
// g_static_mu, which a call holds while it fills the array and enqueues its
// work.
static std::mutex g_static_mu;
static uint8_t *g_static_addr[64] = {};
static uint64_t g_static_serial[64] = {};
static const uint8_t *g_static_grids[64] = {};

static cudaError_t static_scratch_address(int dev, uint8_t **out)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_batch_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = static_cast<uint8_t *>(p);
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

}  // namespace sx

extern "C" int simplex_batch_run_static(simplex_batch_t batch, uint8_t *grids, uint64_t grids_bytes, int parity,
                                        int steps, unsigned long long *live, void *stream)
{
    using namespace sxh;
    BatchView bv;
    int rc = batch_view(batch, &bv);
    if (rc) return rc;
    if (!grids) return fail(SIMPLEX_EINVAL, "grids is NULL");
    if ((reinterpret_cast<uintptr_t>(grids) & 255u) != 0) return fail(SIMPLEX_EINVAL, "grids must be 256-byte aligned");
    if (grids_bytes < bv.grids_bytes)
        return fail(SIMPLEX_EINVAL, "grids too small: %llu bytes, the batch's grids need %llu",
                    (unsigned long long)grids_bytes, (unsigned long long)bv.grids_bytes);
    if (parity != 0 && parity != 1) return fail(SIMPLEX_EINVAL, "parity must be 0 or 1 (got %d)", parity);
    if (steps < 1 || steps > sx::kBatchMaxSteps)
        return fail(SIMPLEX_EINVAL, "steps must be in [1, %d] (got %d)", sx::kBatchMaxSteps, steps);
    if (bv.has_planes)
        return fail(SIMPLEX_EUNSUPPORTED, "the fixed scratch does not hold plane-stream instances (m = 3, block 128): "
                                          "use simplex_batch_bind / simplex_batch_run");
    // scratch layout: descriptors, work items, tensor maps, queue counters
    auto up = [](uint64_t x) { return (x + 255) / 256 * 256; };
    const uint64_t off_items = up(sizeof(sx::BatchInst) * bv.count);
    const uint64_t off_tmaps = up(off_items + sizeof(sx::BatchItem) * bv.nitems);
    const uint64_t off_queue = up(off_tmaps + sizeof(CUtensorMap) * 2 * bv.count);
    const uint64_t need = off_queue + sizeof(unsigned int) * 2 * (uint64_t)(steps + 1);
    if (need > sx::kStaticScratchBytes)
        return fail(SIMPLEX_EINVAL,
                    "batch too large for the fixed scratch: needs %llu bytes of descriptors, work items and "
                    "queue counters, the limit is %llu (use simplex_batch_bind / simplex_batch_run)",
                    (unsigned long long)need, (unsigned long long)sx::kStaticScratchBytes);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(sx::g_static_mu);
    uint8_t *scratch = nullptr;
    e = sx::static_scratch_address(dev, &scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static batch scratch)");
    // the grid offsets of the descriptors count from the arena start; the
    // caller's buffer starts at the grids, so shift the base accordingly
    uint8_t *base = grids - bv.grids_offset;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((e = sx::batch_prepare()) != cudaSuccess) return cuda_fail(e, "setting the batch kernel's shared memory");
    unsigned int *queue = reinterpret_cast<unsigned int *>(scratch + off_queue);
    // descriptors, work items and tensor maps depend only on the batch and the
    // grids' address: when the array already holds them (the last complete
    // upload on this device was for the same batch and grids), only the queue
    // counters are reset
    const bool fresh = !(sx::g_static_serial[dev] == bv.serial && sx::g_static_grids[dev] == grids);
    if (fresh) {
        sx::g_static_serial[dev] = 0;  // the array is about to change
        sx::g_static_grids[dev] = nullptr;
        if ((e = cudaMemcpyAsync(scratch, bv.insts, sizeof(sx::BatchInst) * bv.count, cudaMemcpyHostToDevice,
                                 st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(scratch + off_items, bv.items, sizeof(sx::BatchItem) * bv.nitems,
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "filling the static batch scratch");
        // TMA maps of the caller's grids, encoded in a fixed host buffer and
        // copied in pieces (a copy from pageable memory has read its source on
        // return)
        CUtensorMap piece[32];
        for (size_t k0 = 0; k0 < 2 * bv.count; k0 += 32) {
            const size_t k1 = k0 + 32 < 2 * bv.count ? k0 + 32 : 2 * bv.count;
            for (size_t k = k0; k < k1; ++k) {
                rc = make_tensor_map(bv.insts[k / 2].plan, base + bv.insts[k / 2].grid[k % 2], &piece[k - k0],
                                     bv.insts[k / 2].plan.rho + 2);
                if (rc) return rc;
            }
            if ((e = cudaMemcpyAsync(scratch + off_tmaps + sizeof(CUtensorMap) * k0, piece,
                                     sizeof(CUtensorMap) * (k1 - k0), cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_fail(e, "filling the static batch scratch");
        }
        sx::g_static_serial[dev] = bv.serial;
        sx::g_static_grids[dev] = grids;
    }
    if ((e = cudaMemsetAsync(queue, 0, sizeof(unsigned int) * 2 * (size_t)(steps + 1), st)) != cudaSuccess)
        return cuda_fail(e, "resetting the static batch queue counters");
    const sx::BatchInst *insts = reinterpret_cast<const sx::BatchInst *>(scratch);
    const sx::BatchItem *items = reinterpret_cast<const sx::BatchItem *>(scratch + off_items);
    const CUtensorMap *tm = reinterpret_cast<const CUtensorMap *>(scratch + off_tmaps);
    if (live &&
        (e = cudaMemsetAsync(live, 0, sizeof(unsigned long long) * bv.count * (size_t)(steps + 1), st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(live)");
    rc = enqueue_batch_passes(insts, items, bv.nitems, bv.nitems0, tm, base, queue, queue + steps + 1, steps, live,
                              parity, st);
    if (rc) return rc;
    return SIMPLEX_OK;
}
