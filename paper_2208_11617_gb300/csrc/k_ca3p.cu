// k_ca3p.cu -- one step of the automaton on the 3-simplex (Table 1 test 4 on
// the tetrahedron, fixed-dead boundary, Sec. 5.1), plane-stream form
// (launch 3).
//
// Persistent CTAs (kPlCtasPerSm per SM: four consumer warps and one producer
// warp each) take work units from a device counter; a unit is one brick of kPlaneTY rows x2 by kPlaneTX
// cells x3 over one segment of planes x1 (plane_unit_decode).  The CTA
// streams the brick along x1: every input plane of the brick (its 32 rows and
// 128 cells plus the one-cell halo: 34 rows of up to 160 bytes, the box
// starting 16 bytes left of the brick because a TMA x coordinate must be
// 16-byte aligned) comes in by one TMA tiled load into a ring of kPlSlots
// stages, is read from shared memory once, and is reduced at once to column
// sums over x2 that slide along x1 in registers.  So every staged byte is
// read once, and the 3 x 3 x 3 sum of a cell is three column sums (planes
// x1 - 1, x1, x1 + 1) plus one horizontal 3-sum, all byte-parallel in 32-bit
// words (cells are 0/1, sums stay below 32: no carries between bytes).
//
// Thread (c, p) -- c = tid & 7, p = tid >> 3 -- owns the 16-byte chunk c of
// the brick's rows 2p and 2p + 1: per plane it loads its chunk of the four
// staged rows 2p ... 2p + 3 and one halo word (lane c = 0 the word left of
// the brick, c = 7 the word right of it), and takes the neighbouring
// chunks' edge words from lanes c - 1 and c + 1 by shuffle.  The register
// sets of three consecutive planes rotate through a loop unrolled three
// times, so nothing is copied between planes.
//
// Box width.  The cells of a staged plane x1 that lie in the domain have
// x3 <= n - x1 - (y0 - 1), so the box only has to reach that far: the
// producer picks the narrowest of kPlWidths tensor maps (box widths 48, 80,
// 112, 144 and 160 bytes) that covers it, and the consumers treat chunks
// past the box as zero (they are zero in the grid: outside the domain).  On
// the bricks along the diagonal this halves the bytes read; a staged plane
// with no domain cell in reach (before x1 = 0, past the brick's apex) is not
// loaded at all.
//
// The producer is lane 0 of the last warp.  Each stage has a `full` mbarrier
// (the producer's arrival with the load's bytes, or a plain arrival for a
// plane it does not load) and an `empty` one (one arrival per consumer warp
// once the warp has read the stage); the producer refills stage s with the
// plane kPlSlots ahead as soon as `empty` says every consumer warp is done
// with it, fetching the next unit from the counter one unit in advance, so
// the consumer warps never wait for one another.  A unit of output planes
// b ... e stages planes b - 1 ... e + 1; the first two only fill the sums.
// Every wait is bounded: a warp whose wait runs out sets an abort flag that
// stops the others, the CTA records the status word, waits (bounded) for the
// loads it issued and leaves.  The last CTA to finish puts the counter back
// to zero.
#include "ca_tiles.cuh"
#include "common.cuh"
#include "hmap.cuh"
#include "kernels.h"

namespace sx {

static __device__ uint32_t g_ca3p_status;

constexpr int kPlSlots = 10;
constexpr int kPlCtasPerSm = 4;
constexpr int kPlConsumerWarps = (kPlaneTX / 16) * (kPlaneTY / 2) / 32;  // 8 chunks x 16 row pairs
constexpr int kPlThreads = 32 * (kPlConsumerWarps + 1);                  // plus the producer warp
constexpr int kPlRows = kPlaneTY + 2;
constexpr int kPlMaxW = kPlaneTX + 32;
constexpr uint32_t kPlSlotBytes = ((uint32_t)(kPlRows * kPlMaxW) + 127u) / 128u * 128u;
constexpr int kPlSmem = kPlSlots * (int)kPlSlotBytes + 128;
static_assert(kPlConsumerWarps == 4, "the thread layout assumes 8 chunks x 16 row pairs");
static_assert(kPlMaxW == 160 && kPlaneTY == 32, "the halo-word offsets assume 160-byte rows");
static_assert(kPlCtasPerSm * (kPlSmem + 2048) <= 228 * 1024, "the ring of four CTAs exceeds an SM's shared memory");

// Phase codes of a staged plane (meta .w bits 8..9).
constexpr int kPhFirst = 0, kPhSecond = 1, kPhOut = 2, kPhEnd = 3;

__host__ __device__ constexpr int plane_box_width(int i) { return i < kPlWidths - 1 ? 48 + 32 * i : kPlMaxW; }

// BATCH: one pass of the batched engine over the plane-stream units of many
// m = 3 instances (bt.units, each naming its instance); every instance has its
// own size, grids, tensor maps (bt.ptmaps + its BatchInst::tmap: the widths of
// grid 0, then those of grid 1), rule and live counter.  Otherwise one
// instance: the units come from `sched` and the maps from `maps`.
template <bool ORK, bool BATCH>
__global__ void __launch_bounds__(kPlThreads, kPlCtasPerSm)
    ca3_step_planes(const __grid_constant__ PlaneMaps maps, uint8_t *__restrict__ out, const int64_t n,
                    const int64_t side, const Rule rule, const __grid_constant__ PlaneSched sched,
                    unsigned long long *__restrict__ live, unsigned long long *__restrict__ queue,
                    const PlaneBatch bt)
{
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t full[kPlSlots], empty[kPlSlots];
    // per stage: the address of the output row (x1 - 1, y0, x0) as two 32-bit
    // halves; n - (x1 - 1) + 1 - y0 - x0 (a cell of that plane is in the
    // domain iff its offsets inside the brick sum below it); width | phase << 8
    __shared__ int4 meta[kPlSlots];
    // BATCH: the stage's instance, its or-k rule word (0: the general tables) and its side
    __shared__ int4 meta2[BATCH ? kPlSlots : 1];
    __shared__ uint32_t red[32];
    __shared__ volatile int abort_flag;
    uint8_t *ring = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t lsum = 0;
    uint64_t issued = 0;  // producer: stages filled (loads and markers)

    if (tid == 0) {
        if (!BATCH)
            for (int i = 0; i < kPlWidths; ++i) prefetch_tmap(&maps.m[i]);
        for (int s = 0; s < kPlSlots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kPlConsumerWarps);
        }
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    if (warp == kPlConsumerWarps) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            unsigned long long next_w = atomicAdd(queue, 1ull);
            int32_t py0 = 0, px0 = 0, pb = 0, pe = -1, px1 = 0;
            bool have = false;
            // the unit's instance (BATCH; else the launch's own)
            int64_t pn = n, pside = side;
            uint8_t *pout = out;
            const CUtensorMap *ptm = maps.m;
            int32_t pinst = 0;
            uint32_t pork = 0;
            const uint64_t nunits = BATCH ? (uint64_t)bt.nunits : sched.units;
            for (uint64_t k = 0;; ++k) {
                const int s = (int)(k % kPlSlots);
                if (k >= (uint64_t)kPlSlots && !mbar_try_wait(&empty[s], (uint32_t)((k / kPlSlots - 1) & 1)) &&
                    !mbar_wait_bounded(&empty[s], (uint32_t)((k / kPlSlots - 1) & 1), kWaitLimitNs)) {
                    abort_flag = 1;
                    break;
                }
                while (!have) {
                    const unsigned long long w = next_w;
                    if (w >= nunits) break;
                    next_w = atomicAdd(queue, 1ull);
                    PlaneUnit u;
                    if constexpr (BATCH) {
                        const BatchPlaneUnit bu = bt.units[w];
                        const BatchInst &bi = bt.insts[bu.inst];
                        u = PlaneUnit{(int32_t)(bu.yx & 0xffffu), (int32_t)(bu.yx >> 16), bu.b, bu.e};
                        pinst = (int32_t)bu.inst;
                        pn = bi.plan.n;
                        pside = bi.plan.side;
                        pout = bt.arena + bi.grid[bt.in_parity ^ 1];
                        ptm = bt.ptmaps + bi.tmap + bt.in_parity * kPlWidths;
                        pork = bi.rule.or_k;
                    } else {
                        if (!plane_unit_decode(sched, w, u)) continue;
                    }
                    py0 = u.y0;
                    px0 = u.x0;
                    pb = u.b;
                    pe = u.e;
                    px1 = pb - 1;
                    have = true;
                }
                if (!have) {  // no more work: one end marker
                    meta[s] = make_int4(0, 0, 0, kPhEnd << 8);
                    mbar_arrive(&full[s]);
                    issued = k + 1;
                    break;
                }
                const int ph = px1 == pb - 1 ? kPhFirst : (px1 == pb ? kPhSecond : kPhOut);
                // bytes of the box that can hold domain cells: from x0 - 16 up to
                // n - x1 - (y0 - 1) inclusive
                const int64_t need = (pn - px1 - py0 + 2) - (int64_t)(px0 - 16);
                int wi = -1;
                if (!BATCH && px1 >= 0 && px1 <= pn && sched.kind == kMapBBThread) {
                    wi = kPlWidths - 1;  // the paper's bounding box: every brick staged in full
                } else if (px1 >= 0 && px1 <= pn && need > 16) {
                    wi = 0;
                    while (wi < kPlWidths - 1 && (int64_t)plane_box_width(wi) < need) ++wi;
                }
                const int W = wi < 0 ? 0 : plane_box_width(wi);
                const uint64_t orow =
                    reinterpret_cast<uint64_t>(pout + ((((int64_t)px1 - 1) * pside + py0) * pside + px0));
                meta[s] = make_int4((int)(uint32_t)orow, (int)(uint32_t)(orow >> 32), (int)(pn - px1 + 2 - py0 - px0),
                                    W | (ph << 8));
                if (BATCH) meta2[s] = make_int4(pinst, (int)pork, (int)pside, 0);
                if (wi < 0) {
                    mbar_arrive(&full[s]);  // nothing to load: the phase completes with no bytes
                } else {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&full[s], (uint32_t)(kPlRows * W));
                    tma_load_3d(ring + s * kPlSlotBytes, ptm + wi, px0 - 16, py0 - 1, px1, &full[s]);
                }
                issued = k + 1;
                if (++px1 > pe + 1) have = false;
            }
        }
    } else {
        // ---------------------------------------------------------------- consumers
        const int c = tid & 7, p = tid >> 3;
        // column sums of the three newest staged planes (rotating): words 0..3
        // of row 2p (f) and of row 2p + 1 (s), [4] the halo word; and the
        // centre rows (the cells' own states)
        uint32_t sf[3][5], ss[3][5], af[3][4], as[3][4];
        int slot = 0;
        uint32_t parity = 0;
        const int ho = c == 0 ? 12 : 16 + kPlaneTX;  // this lane's halo word (left or right of the brick)
        const int64_t toff = (int64_t)(2 * p) * side + 16 * c;  // first output cell of the thread in a brick plane
        const int tq = 2 * p + 16 * c;                         // its offsets inside the brick, summed
        int cur = -1;  // BATCH: the instance lsum counts for
        auto flush = [&]() {  // BATCH: the warp's live cells of instance `cur` to its counter
            const uint32_t tot = __reduce_add_sync(0xffffffffu, lsum);
            if (lane == 0 && tot && cur >= 0 && bt.live)
                atomicAdd(bt.live + (uint64_t)cur * (uint64_t)bt.live_stride + (uint64_t)bt.live_index,
                          (unsigned long long)tot);
            lsum = 0;
        };
        for (;;) {
            bool stop = false;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (!mbar_try_wait(&full[slot], parity) &&
                    (abort_flag || !mbar_wait_bounded(&full[slot], parity, kWaitLimitNs))) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                const int4 md = meta[slot];
                const int4 md2 = BATCH ? meta2[slot] : make_int4(0, 0, 0, 0);
                const int W = md.w & 255, ph = md.w >> 8;
                if (ph == kPhEnd) {
                    stop = true;
                    break;
                }
                uint32_t v[4][4], h[4];
                const uint8_t *base = ring + slot * kPlSlotBytes + 2 * p * W;
                if (W == kPlMaxW) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint4 q = *reinterpret_cast<const uint4 *>(base + k * kPlMaxW + 16 + 16 * c);
                        v[k][0] = q.x;
                        v[k][1] = q.y;
                        v[k][2] = q.z;
                        v[k][3] = q.w;
                        h[k] = *reinterpret_cast<const uint32_t *>(base + k * kPlMaxW + ho);
                    }
                } else {
                    const bool has_c = 16 * c + 32 <= W, has_h = c == 0 && W > 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        uint4 q = make_uint4(0u, 0u, 0u, 0u);
                        if (has_c) q = *reinterpret_cast<const uint4 *>(base + k * W + 16 + 16 * c);
                        v[k][0] = q.x;
                        v[k][1] = q.y;
                        v[k][2] = q.z;
                        v[k][3] = q.w;
                        h[k] = has_h ? *reinterpret_cast<const uint32_t *>(base + k * W + 12) : 0u;
                    }
                }
                // this warp is done with the stage
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                // sums of this plane into set j; only lanes c = 0 (left) and
                // c = 7 (right) use their halo word
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    sf[j][w] = v[0][w] + v[1][w] + v[2][w];
                    ss[j][w] = v[1][w] + v[2][w] + v[3][w];
                    af[j][w] = v[1][w];
                    as[j][w] = v[2][w];
                }
                sf[j][4] = h[0] + h[1] + h[2];
                ss[j][4] = h[1] + h[2] + h[3];
                if (ph == kPhOut) {
                    // output plane x1 - 1 (x1 the staged plane) from the sets
                    // of planes x1 - 2 (j + 1), x1 - 1 (j + 2) and x1 (j)
                    const int P = (j + 1) % 3, Q = (j + 2) % 3;
                    const bool partial = md.z < kPlaneTY + kPlaneTX - 1;  // not every cell of the brick plane
                    const int64_t rs = BATCH ? (int64_t)md2.z : side;  // row stride of the output grid
                    uint8_t *dst = reinterpret_cast<uint8_t *>(((uint64_t)(uint32_t)md.y << 32) | (uint32_t)md.x) +
                                   (BATCH ? (int64_t)(2 * p) * rs + 16 * c : toff);
                    if (BATCH && md2.x != cur) {
                        flush();
                        cur = md2.x;
                    }
                    uint32_t acc = 0;
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        uint32_t V[5], S[4], nw[4];
#pragma unroll
                        for (int w = 0; w < 5; ++w)
                            V[w] = r == 0 ? sf[P][w] + sf[Q][w] + sf[j][w] : ss[P][w] + ss[Q][w] + ss[j][w];
                        const uint32_t lft = __shfl_up_sync(0xffffffffu, V[3], 1, 8);
                        const uint32_t rgt = __shfl_down_sync(0xffffffffu, V[0], 1, 8);
                        hsum4(V, c == 0 ? V[4] : lft, c == 7 ? V[4] : rgt, S);
                        if constexpr (BATCH) {
                            if (md2.y)
                                apply_rule4_ork(S, r == 0 ? af[Q] : as[Q], (uint32_t)md2.y, nw);
                            else
                                apply_rule4(S, r == 0 ? af[Q] : as[Q], bt.insts[md2.x].rule, nw);
                        } else {
                            next_state4<ORK>(S, r == 0 ? af[Q] : as[Q], rule, nw);
                        }
                        if (partial) {
                            const int cnt = md.z - tq - r;  // cells of the chunk in the domain
                            if (cnt < 16) {
                                const int c8 = 8 * cnt;
#pragma unroll
                                for (int w = 0; w < 4; ++w)
                                    nw[w] &= __funnelshift_rc(0xffffffffu, 0u, (uint32_t)max(0, 32 * w + 32 - c8));
                            }
                            if (cnt > 0) store16(dst + r * rs, nw);
                        } else {
                            store16(dst + r * rs, nw);
                        }
                        acc += (nw[0] + nw[1]) + (nw[2] + nw[3]);
                    }
                    lsum += (acc * 0x01010101u) >> 24;  // bytes <= 8: their sum fits the top byte
                }
                if (++slot == kPlSlots) {
                    slot = 0;
                    parity ^= 1u;
                }
            }
            if (stop) break;
        }
        if (BATCH) flush();
    }

    __syncthreads();
    if (tid == kPlConsumerWarps * 32) {
        if (abort_flag) {
            atomicOr(&g_ca3p_status, 1u);
            // the last fill issued into each stage must land before the CTA exits
            for (int j = 1; j <= kPlSlots && (uint64_t)j <= issued; ++j) {
                const uint64_t q = issued - j;
                mbar_wait_bounded(&full[q % kPlSlots], (uint32_t)((q / kPlSlots) & 1), kWaitLimitNs);
            }
        }
        // the last CTA out resets the work counter (every fetch of this launch is done)
        __threadfence();
        if (atomicAdd(&queue[1], 1ull) == (unsigned long long)gridDim.x - 1ull) {
            queue[0] = 0;
            queue[1] = 0;
            __threadfence();
        }
    }
    if (!BATCH && live) block_add_u64(live, lsum, red);
}

template <bool ORK, bool BATCH>
static cudaError_t prepare_planes_one()
{
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(ca3_step_planes<ORK, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPlSmem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

cudaError_t ca3_planes_prepare()
{
    cudaError_t e = prepare_planes_one<false, false>();
    if (e == cudaSuccess) e = prepare_planes_one<true, false>();
    return e != cudaSuccess ? e : prepare_planes_one<false, true>();
}

int plane_box_widths(int *w)
{
    for (int i = 0; i < kPlWidths; ++i) w[i] = plane_box_width(i);
    return kPlWidths;
}

// Resident CTAs of the plane-stream kernel on the current device (SMs x occupancy).
static cudaError_t planes_resident(uint64_t *out)
{
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ca3_step_planes<true, false>, kPlThreads,
                                                           kPlSmem)) != cudaSuccess)
        return e;
    *out = (uint64_t)sms * (uint64_t)(occ < 1 ? 1 : occ);
    return cudaSuccess;
}

cudaError_t launch_ca3_planes(const PlaneSched &sched, const PlaneMaps &maps, int64_t n, int64_t side, uint8_t *out,
                              const Rule &rule, unsigned long long *live, unsigned long long *queue, cudaStream_t st)
{
    if (!queue) return cudaErrorInvalidValue;
    cudaError_t e = ca3_planes_prepare();
    if (e != cudaSuccess) return e;
    uint64_t resident = 0;
    if ((e = planes_resident(&resident)) != cudaSuccess) return e;
    const uint64_t g = sched.units < resident ? (sched.units ? sched.units : 1) : resident;
    const PlaneBatch none = {};
    if (rule.or_k)
        ca3_step_planes<true, false><<<(unsigned)g, kPlThreads, kPlSmem, st>>>(maps, out, n, side, rule, sched, live,
                                                                               queue, none);
    else
        ca3_step_planes<false, false><<<(unsigned)g, kPlThreads, kPlSmem, st>>>(maps, out, n, side, rule, sched,
                                                                                live, queue, none);
    return cudaGetLastError();
}

cudaError_t launch_batch_planes(const PlaneBatch &bt, unsigned long long *queue, cudaStream_t st)
{
    if (!queue || !bt.nunits) return bt.nunits ? cudaErrorInvalidValue : cudaSuccess;
    cudaError_t e = ca3_planes_prepare();
    if (e != cudaSuccess) return e;
    uint64_t resident = 0;
    if ((e = planes_resident(&resident)) != cudaSuccess) return e;
    const uint64_t g = (uint64_t)bt.nunits < resident ? (uint64_t)bt.nunits : resident;
    static const PlaneMaps no_maps = {};
    static const PlaneSched no_sched = {};
    static const Rule no_rule = {};
    ca3_step_planes<false, true><<<(unsigned)g, kPlThreads, kPlSmem, st>>>(no_maps, nullptr, 0, 0, no_rule, no_sched,
                                                                           nullptr, queue, bt);
    return cudaGetLastError();
}

cudaError_t ca3p_read_status(uint32_t *out)
{
    uint32_t zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_ca3p_status, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_ca3p_status, &zero, sizeof(uint32_t));
}

}  // namespace sx
