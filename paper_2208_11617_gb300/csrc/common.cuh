// common.cuh -- device helpers shared by the kernels: the hash, TMA and
// mbarrier wrappers (inline PTX for sm_103a), bounded waits, reductions.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rule.h"

namespace sx {

// splitmix32: the golden-ratio counter step (add 0x9E3779B9) followed by the
// MurmurHash3 32-bit finaliser.  Not part of the paper; it defines the
// synthetic cell values and initial states.
__device__ __forceinline__ uint32_t splitmix32(uint32_t z)
{
    z += 0x9E3779B9u;
    z = (z ^ (z >> 16)) * 0x85EBCA6Bu;
    z = (z ^ (z >> 13)) * 0xC2B2AE35u;
    return z ^ (z >> 16);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this CTA's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One plain arrival (no transaction bytes) on `bar`.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// `count` plain arrivals at once (count >= 1).
__device__ __forceinline__ void mbar_arrive_n(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier to complete, giving up after
// `limit_ns` nanoseconds of wall time (or 2^22 polls, whichever comes first).
// Returns false if it gave up.
static __device__ __noinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// One TMA tiled load of a box into shared memory, completing on `bar`.
// Coordinates are element indices, innermost first; x must be a multiple of
// 16 bytes / element size.  Cells outside the tensor read as zero.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            int32_t z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Programmatic dependent launch (sm_90 and later).  A grid launched with
// programmatic stream serialization may start while the kernel before it in
// the stream is still running: grid_dep_wait() blocks until that kernel has
// completed and its writes are visible, and grid_dep_trigger() lets the next
// such grid start once every CTA of this one has called it or exited.  Both
// return at once for a grid launched without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches `kernel` with programmatic stream serialization (see above).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Sum of v over the CTA, added to *dst by one thread (skipped when zero).
// Every thread of the CTA must call it.
__device__ __forceinline__ void block_add_u64(unsigned long long *dst, uint32_t v, uint32_t *scratch32)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    const int in_warp = min(32, (int)blockDim.x - 32 * warp);
    const uint32_t mask = in_warp == 32 ? 0xffffffffu : ((1u << in_warp) - 1u);
    const uint32_t w = __reduce_add_sync(mask, v);
    if (lane == 0) scratch32[warp] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int i = 0; i < nwarps; ++i) s += scratch32[i];
        if (s) atomicAdd(dst, s);
    }
}

// Byte mask keeping the first `c` bytes (0..16) of a 16-byte chunk, word w.
__device__ __forceinline__ uint32_t chunk_word_mask(int c, int w)
{
    const int ci = min(max(c - 4 * w, 0), 4);
    return ci >= 4 ? 0xffffffffu : ((1u << (8 * ci)) - 1u);
}

// Next state of 4 x 4 cells: s[w] holds, per byte, the number of live cells in
// the 3^m neighbourhood including the cell itself (<= 27); alive[w] holds the
// cells (0/1 per byte).  Bytes stay below 0x20, so adding 0x7F per byte never
// carries and sets bit 7 exactly where s differs from the tested value.
__device__ __forceinline__ void apply_rule4(const uint32_t s[4], const uint32_t alive[4], const Rule &r,
                                            uint32_t nw[4])
{
    uint32_t a7[4], acc[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        a7[w] = alive[w] << 7;
        acc[w] = 0;
    }
    for (int j = 0; j < r.nk; ++j) {
        const uint32_t K = r.kbytes[j], B = r.bsel[j], S = r.ssel[j];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t nz = (s[w] ^ K) + 0x7F7F7F7Fu;
            const uint32_t cond = (B & ~a7[w]) | (S & a7[w]);
            acc[w] |= ~nz & cond;
        }
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) nw[w] = (acc[w] >> 7) & 0x01010101u;
}

// Next state for the "or-k" rules (Rule::or_k != 0): with c = s - alive the
// live-neighbour count, a cell is alive next iff (c | alive) == k.  For k odd
// this is exactly birth on k and survival on k-1 or k.
__device__ __forceinline__ void apply_rule4_ork(const uint32_t s[4], const uint32_t alive[4], uint32_t kbytes,
                                                uint32_t nw[4])
{
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t c = s[w] - alive[w];                      // bytes never borrow: s >= alive
        const uint32_t y = ((c | alive[w]) ^ kbytes) + 0x7F7F7F7Fu;  // bit 7 set iff byte != k
        nw[w] = (~y >> 7) & 0x01010101u;
    }
}

template <bool ORK>
__device__ __forceinline__ void next_state4(const uint32_t s[4], const uint32_t alive[4], const Rule &r,
                                            uint32_t nw[4])
{
    if (ORK)
        apply_rule4_ork(s, alive, r.or_k, nw);
    else
        apply_rule4(s, alive, r, nw);
}

// Dead-byte words of a 16-cell chunk of which the first `cnt` cells lie in the
// domain: bit 7 of byte i of dead[w] is set iff 4 w + i >= cnt.  Byte i of
// word w holds 4 w + i + 128 - min(max(cnt, 0), 16), which stays in
// 112 ... 143 (no carries) and reaches 128 exactly from cell cnt on.
__device__ __forceinline__ void chunk_dead4(int cnt, uint32_t dead[4])
{
    const uint32_t k = (uint32_t)(128 - min(max(cnt, 0), 16)) * 0x01010101u;
#pragma unroll
    for (int w = 0; w < 4; ++w) dead[w] = k + (0x03020100u + 0x04040404u * (uint32_t)w);
}

// apply_rule4_ork / apply_rule4 with the bytes whose bit 7 is set in dead[]
// forced to 0 (cells past the domain's edge).
__device__ __forceinline__ void apply_rule4_ork_masked(const uint32_t s[4], const uint32_t alive[4], uint32_t kbytes,
                                                       const uint32_t dead[4], uint32_t nw[4])
{
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t c = s[w] - alive[w];
        const uint32_t y = ((c | alive[w]) ^ kbytes) + 0x7F7F7F7Fu;  // bit 7 set iff byte != k
        nw[w] = (~(y | dead[w]) >> 7) & 0x01010101u;
    }
}

__device__ __forceinline__ void apply_rule4_masked(const uint32_t s[4], const uint32_t alive[4], const Rule &r,
                                                   const uint32_t dead[4], uint32_t nw[4])
{
    apply_rule4(s, alive, r, nw);
#pragma unroll
    for (int w = 0; w < 4; ++w) nw[w] &= ~(dead[w] >> 7);
}

template <bool ORK>
__device__ __forceinline__ void next_state4_masked(const uint32_t s[4], const uint32_t alive[4], const Rule &r,
                                                   const uint32_t dead[4], uint32_t nw[4])
{
    if (ORK)
        apply_rule4_ork_masked(s, alive, r.or_k, dead, nw);
    else
        apply_rule4_masked(s, alive, r, dead, nw);
}

// Sum of the four bytes of a word (each byte <= 255, no overflow).
__device__ __forceinline__ uint32_t byte_sum(uint32_t v)
{
    return (v & 0xffu) + ((v >> 8) & 0xffu) + ((v >> 16) & 0xffu) + (v >> 24);
}

// Horizontal 3-sums of one 16-byte row chunk in shared memory: h[w] byte j =
// cell(j-1) + cell(j) + cell(j+1), using the 4 bytes before and after the
// chunk for the edge cells.  c[] receives the chunk itself.
__device__ __forceinline__ void hsum_row(const uint8_t *chunk, uint32_t h[4], uint32_t c[4])
{
    const uint4 w = *reinterpret_cast<const uint4 *>(chunk);
    const uint32_t lw = *reinterpret_cast<const uint32_t *>(chunk - 4);
    const uint32_t rw = *reinterpret_cast<const uint32_t *>(chunk + 16);
    h[0] = w.x + __funnelshift_l(lw, w.x, 8) + __funnelshift_r(w.x, w.y, 8);
    h[1] = w.y + __funnelshift_l(w.x, w.y, 8) + __funnelshift_r(w.y, w.z, 8);
    h[2] = w.z + __funnelshift_l(w.y, w.z, 8) + __funnelshift_r(w.z, w.w, 8);
    h[3] = w.w + __funnelshift_l(w.z, w.w, 8) + __funnelshift_r(w.w, rw, 8);
    c[0] = w.x;
    c[1] = w.y;
    c[2] = w.z;
    c[3] = w.w;
}

__device__ __forceinline__ void store16(uint8_t *dst, const uint32_t v[4])
{
    *reinterpret_cast<uint4 *>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
}

constexpr uint64_t kWaitLimitNs = 200ull * 1000ull * 1000ull;  // 200 ms per TMA wait

}  // namespace sx
