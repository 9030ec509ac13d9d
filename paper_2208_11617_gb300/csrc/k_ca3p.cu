// k_ca3p.cu -- one step of the automaton on the 3-simplex (Table 1 test 4 on
// the tetrahedron, fixed-dead boundary, Sec. 5.1), plane-stream form
// (launch 3).
//
// Persistent CTAs (kPlCtasPerSm per SM: four consumer warps and one producer
// warp each) take work units from a device counter; a unit is one brick of
// kPlaneTY rows x2 by kPlaneTX cells x3 over one segment of planes x1
// (plane_unit_decode).  The CTA streams the brick along x1.  A stage is one
// TMA tiled load of kPlPlanes consecutive input planes of the brick: per plane
// its 32 rows and 128 cells plus the one-cell halo, 34 rows of up to 160
// bytes, the box starting 16 bytes left of the brick because a TMA x
// coordinate must be 16-byte aligned.  Stages go into a ring of kPlStages;
// each staged plane is read from shared memory once and reduced at once to
// column sums over x2 that slide along x1 in registers.  So every staged byte
// is read once, and the 3 x 3 x 3 sum of a cell is three column sums (planes
// x1 - 1, x1, x1 + 1) plus one horizontal 3-sum, all byte-parallel in 32-bit
// words (cells are 0/1, sums stay below 32: no carries between bytes).
//
// Consumer warp w owns the warp tile of 16 rows (wy = w / 2) by 64 cells
// (wx = w % 2) of the brick; its lane (c, p) -- c = lane & 3, p = lane >> 2
// -- owns the 16-byte chunk C = 4 wx + c of the brick rows 2P and 2P + 1,
// P = 8 wy + p.  Per plane a lane loads its chunk of the four staged rows
// 2P ... 2P + 3 and one halo word (c = 0 the word left of the warp tile, c =
// 3 the word right of it: inside the box, or the box's halo at the brick's
// edges) and takes the neighbouring chunks' edge words from lanes c - 1 and
// c + 1 by shuffle.  A warp whose tile holds no domain cell on an output
// plane (on the bricks along the diagonal) skips that plane's output: 2-3 %
// faster than warps of 8 rows by the whole brick width, which never skip,
// although the narrower boxes now cost some shared-memory bank conflicts
// (a quarter warp reads two row pairs 2W bytes apart; boxes narrowed to
// widths 32 modulo 64 only, which avoid them, read more and were 5 %
// slower).  The register sets of three consecutive planes rotate through a
// loop unrolled over three stages (six planes), so nothing is copied between
// planes.
//
// Box width.  The cells of a staged plane x1 that lie in the domain have
// x3 <= n - x1 - (y0 - 1), so the box only has to reach that far: the
// producer picks the narrowest of kPlWidths tensor maps (box widths 48, 80,
// 112, 144 and 160 bytes) that covers the stage's first plane, and the
// consumers read chunks past the box as zero (they are zero in the grid:
// outside the domain).  On the bricks along the diagonal this halves the
// bytes read; a stage with no domain cell in reach (past the brick's apex)
// is not loaded at all.
//
// The producer is lane 0 of the last warp; its warp first copies the
// schedule's segment tables into shared memory, where the unit decode
// searches them.  Each stage has a `full` mbarrier (the producer's arrival
// with the load's bytes, or a plain arrival for a stage it does not load)
// and an `empty` one (one arrival per consumer warp once the warp has read
// the stage); the producer refills a stage as soon as `empty` says every
// consumer warp is done with it, takes the next unit from the counter one
// unit in advance and decodes it as soon as the current unit's last stage
// is issued, so the consumer warps never wait for one another.  A unit of
// output planes b ... e stages planes b - 1 ... e + 1 (rounded up to whole
// stages; a plane past e + 1 only fills sums); the first two only fill the
// sums.  Every wait is bounded: a warp whose wait runs out sets an abort flag
// that stops the others, the CTA records the status word, waits (bounded)
// for the loads it issued and leaves.  The last CTA to finish puts the
// counter back to zero.
#include "ca_tiles.cuh"
#include "common.cuh"
#include "hmap.cuh"
#include "kernels.h"

namespace sx {

static __device__ uint32_t g_ca3p_status;

constexpr int kPlStages = 4;  // five per CTA were 5 % slower, three or six (three CTAs per SM) no faster
constexpr int kPlCtasPerSm = 4;
constexpr int kPlTileRows = 16, kPlTileCols = 64;  // a consumer warp's tile of the brick
constexpr int kPlConsumerWarps = (kPlaneTY / kPlTileRows) * (kPlaneTX / kPlTileCols);
constexpr int kPlThreads = 32 * (kPlConsumerWarps + 1);                  // plus the producer warp
constexpr int kPlRows = kPlaneTY + 2;
constexpr int kPlMaxW = kPlaneTX + 32;
constexpr uint32_t kPlStageBytes = (uint32_t)(kPlPlanes * kPlRows * kPlMaxW);
constexpr int kPlRingSmem = kPlStages * (int)kPlStageBytes + 128;  // plus 128 bytes to align the ring
// the most shared memory a launch asks for: the ring and the largest segment tables
constexpr int kPlMaxSmem = kPlRingSmem + kPlaneSegWords * (int)sizeof(int32_t);
static_assert(kPlPlanes == 2, "the consumer loop handles two planes per stage");
static_assert(kPlStageBytes % 128 == 0, "every stage starts on a 128-byte boundary");
static_assert(kPlConsumerWarps == 4 && kPlTileRows * kPlTileCols == 32 * 2 * 16,
              "a warp tile is 8 row pairs x 4 chunks, one chunk pair per lane");
static_assert(kPlMaxW == 160 && kPlaneTY == 32, "the halo-word offsets assume 160-byte rows");

// Phase codes of a staged plane (meta .w: first plane bits 8..9, second
// plane bits 10..11).  kPhFirst: the plane only fills sums (the first of a
// unit, or a plane past the unit's end); kPhSecond: the second of a unit;
// kPhOut: the plane completes the sums of output plane x1 - 1; kPhEnd (first
// plane only): no more work.
constexpr int kPhFirst = 0, kPhSecond = 1, kPhOut = 2, kPhEnd = 3;
static_assert(kPhFirst == 0 && kPhSecond == 1 && kPhOut == 2, "the producer's phase is min(x1 - b + 1, kPhOut)");

__host__ __device__ constexpr int plane_box_width(int i) { return i < kPlWidths - 1 ? 48 + 32 * i : kPlMaxW; }

// Dynamic shared memory of one launch: the ring, then (single instance) the
// schedule's segment tables, seg_b[nseg + 1] and seg_u[nseg + 1].
__host__ __device__ constexpr int plane_smem_bytes(int nseg, bool batch)
{
    return kPlRingSmem + (batch ? 0 : 2 * (nseg + 1) * (int)sizeof(int32_t));
}

// Shared-memory loads at 32-bit shared addresses.  volatile: they stay after
// the stage's mbarrier wait and before the warp's release arrival.
__device__ __forceinline__ void lds128(uint32_t a, uint32_t v[4])
{
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(a));
}

__device__ __forceinline__ uint32_t lds32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// BATCH: one pass of the batched engine over the plane-stream units of many
// m = 3 instances (bt.units, each naming its instance); every instance has its
// own size, grids, tensor maps (bt.ptmaps + its BatchInst::tmap: the widths of
// grid 0, then those of grid 1), rule and live counter.  Otherwise one
// instance: the units come from `sched` (segment tables `segs` in device
// memory) and the maps from `maps`.
template <bool ORK, bool BATCH>
__global__ void __launch_bounds__(kPlThreads, kPlCtasPerSm)
    ca3_step_planes(const __grid_constant__ PlaneMaps maps, uint8_t *__restrict__ out, const int64_t n,
                    const int64_t side, const Rule rule, const __grid_constant__ PlaneSched sched,
                    const int32_t *__restrict__ segs, unsigned long long *__restrict__ live,
                    unsigned long long *__restrict__ queue, const PlaneBatch bt)
{
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t full[kPlStages], empty[kPlStages];
    // per stage: the address of the output row (x1 - 1, y0, x0) of its first
    // plane x1 as two 32-bit halves; n - (x1 - 1) + 1 - y0 - x0 (a cell of
    // that output plane is in the domain iff its offsets inside the brick sum
    // below it); width | phase of the first plane << 8 | of the second << 10
    __shared__ int4 meta[kPlStages];
    // BATCH: the stage's instance, its or-k rule word (0: the general tables) and its side
    __shared__ int4 meta2[BATCH ? kPlStages : 1];
    __shared__ uint32_t red[32];
    __shared__ __align__(16) uint8_t zb[16];  // zeros: what a chunk outside the staged box reads
    __shared__ volatile int abort_flag;
    uint8_t *ring = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 127) & ~uintptr_t(127));
    int32_t *sseg = reinterpret_cast<int32_t *>(dsmem + kPlRingSmem);  // seg_b[nseg + 1], seg_u[nseg + 1]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t lsum = 0;
    uint64_t issued = 0;  // producer: stages filled (loads and markers)

    if (tid == 0) {
        if (!BATCH)
            for (int i = 0; i < kPlWidths; ++i) prefetch_tmap(&maps.m[i]);
        for (int s = 0; s < kPlStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kPlConsumerWarps);
        }
        fence_mbar_init();
        abort_flag = 0;
    }
    if (tid < 4) reinterpret_cast<uint32_t *>(zb)[tid] = 0u;
    __syncthreads();

    if (warp == kPlConsumerWarps) {
        // ---------------------------------------------------------------- producer
        const int ns = BATCH ? 0 : sched.nseg + 1;
        if (!BATCH) {
            for (int i = lane; i < ns; i += 32) {
                sseg[i] = segs[i];
                sseg[ns + i] = segs[kPlaneSegTable + i];
            }
            __syncwarp();
        }
        if (lane == 0) {
            unsigned long long next_w = atomicAdd(queue, 1ull);
            // the current unit: rows y0.., cells x0.., output planes b ... e;
            // px1 the first plane of the next stage
            int32_t py0 = 0, px0 = 0, pb = 0, pe = -1, px1 = 0;
            int32_t pq = 0;                   // n - px1 + 2 - y0 - x0
            uint64_t orow = 0, ostride = 0;   // output row (px1 - 1, y0, x0); bytes per plane
            int64_t pn = n;
            const CUtensorMap *ptm = maps.m;
            int32_t pinst = 0, pside = (int32_t)side;
            uint32_t pork = 0;
            const uint64_t nunits = BATCH ? (uint64_t)bt.nunits : sched.units;
            const bool full_box = !BATCH && sched.kind == kMapBBThread;
            const int32_t *seg_b = sseg;
            const uint32_t *seg_u = reinterpret_cast<const uint32_t *>(sseg + ns);
            // Takes the next unit from the counter (the one fetched a unit
            // earlier, so the atomic's latency is hidden) and decodes it;
            // false once the queue is exhausted.
            auto next_unit = [&]() -> bool {
                for (;;) {
                    const unsigned long long w = next_w;
                    if (w >= nunits) return false;
                    next_w = atomicAdd(queue, 1ull);
                    PlaneUnit u;
                    uint8_t *pout = out;
                    if constexpr (BATCH) {
                        const BatchPlaneUnit bu = bt.units[w];
                        const BatchInst &bi = bt.insts[bu.inst];
                        u = PlaneUnit{(int32_t)(bu.yx & 0xffffu), (int32_t)(bu.yx >> 16), bu.b, bu.e};
                        pinst = (int32_t)bu.inst;
                        pn = bi.plan.n;
                        pside = (int32_t)bi.plan.side;
                        pout = bt.arena + bi.grid[bt.in_parity ^ 1];
                        ptm = bt.ptmaps + bi.tmap + bt.in_parity * kPlWidths;
                        pork = bi.rule.or_k;
                    } else {
                        if (!plane_unit_decode(sched, seg_b, seg_u, w, u)) continue;
                    }
                    py0 = u.y0;
                    px0 = u.x0;
                    pb = u.b;
                    pe = u.e;
                    px1 = pb - 1;
                    pq = (int32_t)(pn - px1 + 2 - py0 - px0);
                    ostride = (uint64_t)pside * (uint64_t)pside;
                    orow = reinterpret_cast<uint64_t>(pout) +
                           (uint64_t)((((int64_t)px1 - 1) * pside + py0) * (int64_t)pside + px0);
                    return true;
                }
            };
            bool have = next_unit();
            int s = 0;
            uint32_t eph = 1;  // parity of empty[s] to wait for (from the second pass over the ring on)
            for (uint32_t k = 0;; ++k) {
                if (k >= (uint32_t)kPlStages && !mbar_try_wait(&empty[s], eph) &&
                    !mbar_wait_bounded(&empty[s], eph, kWaitLimitNs)) {
                    abort_flag = 1;
                    break;
                }
                if (!have) {  // no more work: one end marker
                    meta[s] = make_int4(0, 0, 0, kPhEnd << 8);
                    mbar_arrive(&full[s]);
                    issued = k + 1;
                    break;
                }
                // planes px1 and px1 + 1; the second past the unit's end only fills sums
                const int ph0 = min(px1 - pb + 1, (int)kPhOut);
                const int ph1 = px1 + 1 <= pe + 1 ? min(px1 - pb + 2, (int)kPhOut) : kPhFirst;
                // the box reaches from x0 - 16 to the last cell of the first
                // plane that can be in the domain, x0 + pq - 1: pq + 16 bytes;
                // boxes of 48, 80, 112, 144 or 160 bytes (index (pq - 1) / 32,
                // at most 4).  No load when neither plane lies in 0 ... n.
                int wi = -1;
                if (px1 + 1 >= 0 && px1 <= pn) {
                    if (full_box)
                        wi = kPlWidths - 1;  // the paper's bounding box: every brick staged in full
                    else if (pq > 0)
                        wi = min((pq - 1) >> 5, kPlWidths - 1);
                }
                const int W = wi < 0 ? 0 : plane_box_width(wi);
                meta[s] = make_int4((int)(uint32_t)orow, (int)(uint32_t)(orow >> 32), pq,
                                    W | (ph0 << 8) | (ph1 << 10));
                if (BATCH) meta2[s] = make_int4(pinst, (int)pork, pside, 0);
                // The consumers' reads of this stage's previous contents are
                // ordered before this fill by the empty barrier (their warps'
                // release arrivals, the wait's acquire).
                if (wi < 0) {
                    mbar_arrive(&full[s]);  // nothing to load: the phase completes with no bytes
                } else {
                    mbar_arrive_expect_tx(&full[s], (uint32_t)(kPlPlanes * kPlRows * W));
                    tma_load_3d(ring + s * kPlStageBytes, ptm + wi, px0 - 16, py0 - 1, px1, &full[s]);
                }
                issued = k + 1;
                if (++s == kPlStages) {
                    s = 0;
                    eph ^= 1u;
                }
                orow += kPlPlanes * ostride;
                pq -= kPlPlanes;
                px1 += kPlPlanes;
                // the unit's last stage is issued: decode the next unit now,
                // while the ring is full, not after the next stage frees
                if (px1 > pe + 1) have = next_unit();
            }
        }
    } else {
        // ---------------------------------------------------------------- consumers
        const int wx = warp % (kPlaneTX / kPlTileCols), wy = warp / (kPlaneTX / kPlTileCols);
        const int c = lane & 3, C = 4 * wx + c;              // chunk inside the warp tile / the brick
        const int P = (kPlTileRows / 2) * wy + (lane >> 2);  // row pair inside the brick
        // column sums of the three newest staged planes (rotating): words 0..3
        // of row 2P (f) and of row 2P + 1 (s), [4] the halo word; and the
        // centre rows (the cells' own states)
        uint32_t sf[3][5], ss[3][5], af[3][4], as[3][4];
        int slot = 0;
        uint32_t parity = 0;
        // this lane's halo word as a byte offset in a staged row (c = 0: the
        // word left of the warp tile, c = 3: the word right of it) and the box
        // width from which it lies inside the box; lanes c = 1, 2 read zeros
        // and do not use theirs
        const int ho = c == 0 ? 12 + kPlTileCols * wx : 16 + kPlTileCols * (wx + 1);
        const int hw = c == 0 || c == 3 ? ho + 4 : 1 << 20;
        const int cw = 16 * C + 32;  // box width from which this lane's chunk lies inside the box
        const uint32_t ring_sa = smem_u32(ring), zb_sa = smem_u32(zb);
        const int64_t toff = (int64_t)(2 * P) * side + 16 * C;  // first output cell of the thread in a brick plane
        const int64_t pstride = side * side;                   // bytes per output plane
        const int tq = 2 * P + 16 * C;                         // its offsets inside the brick, summed
        const int tmin = kPlTileRows * wy + kPlTileCols * wx;  // the warp tile's least offset sum
        int cur = -1;  // BATCH: the instance lsum counts for
        uint32_t acc = 0;  // live cells written, per byte, over at most six planes (bytes <= 48)
        auto flush = [&]() {  // BATCH: the warp's live cells of instance `cur` to its counter
            lsum += (acc * 0x01010101u) >> 24;
            acc = 0;
            const uint32_t tot = __reduce_add_sync(0xffffffffu, lsum);
            if (lane == 0 && tot && cur >= 0 && bt.live)
                atomicAdd(bt.live + (uint64_t)cur * (uint64_t)bt.live_stride + (uint64_t)bt.live_index,
                          (unsigned long long)tot);
            lsum = 0;
        };
        for (;;) {
            bool stop = false;
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                if (!mbar_try_wait(&full[slot], parity) &&
                    (abort_flag || !mbar_wait_bounded(&full[slot], parity, kWaitLimitNs))) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                const int4 md = meta[slot];
                const int4 md2 = BATCH ? meta2[slot] : make_int4(0, 0, 0, 0);
                const int W = md.w & 255;
                if (((md.w >> 8) & 3) == kPhEnd) {
                    stop = true;
                    break;
                }
                // Row k of the lane's chunk of plane q sits at pc + q * qc +
                // k * sc, its halo word at hc + q * qh + k * sh; a chunk (or
                // halo word) outside the box reads the 16 zero bytes zb with
                // stride 0 (the grid is zero there: outside the domain).  Every
                // lane thus loads unconditionally.
                const uint32_t rowb = ring_sa + (uint32_t)(slot * (int)kPlStageBytes + 2 * P * W);
                const bool has_c = cw <= W, has_h = hw <= W;
                const uint32_t pc = has_c ? rowb + (uint32_t)(16 + 16 * C) : zb_sa;
                const uint32_t hc = has_h ? rowb + (uint32_t)ho : zb_sa;
                const uint32_t sc = has_c ? (uint32_t)W : 0u, sh = has_h ? (uint32_t)W : 0u;
                const uint64_t dbase = ((uint64_t)(uint32_t)md.y << 32) | (uint32_t)md.x;
                const int64_t rs = BATCH ? (int64_t)md2.z : side;  // row stride of the output grid
                const int64_t ps = BATCH ? rs * rs : pstride;
                if (BATCH && md2.x != cur) {
                    flush();
                    cur = md2.x;
                }
#pragma unroll
                for (int q = 0; q < kPlPlanes; ++q) {
                    const int j = (kPlPlanes * jj + q) % 3;  // this plane's register set
                    const int ph = (md.w >> (8 + 2 * q)) & 3;
                    uint32_t v[4][4], h[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        lds128(pc + (uint32_t)q * (uint32_t)kPlRows * sc + (uint32_t)k * sc, v[k]);
                        h[k] = lds32(hc + (uint32_t)q * (uint32_t)kPlRows * sh + (uint32_t)k * sh);
                    }
                    if (q == kPlPlanes - 1) {
                        // this warp is done with the stage
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&empty[slot]);
                    }
                    // sums of this plane into set j; only lanes c = 0 (left)
                    // and c = 3 (right) use their halo word
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        sf[j][w] = v[0][w] + v[1][w] + v[2][w];
                        ss[j][w] = v[1][w] + v[2][w] + v[3][w];
                        af[j][w] = v[1][w];
                        as[j][w] = v[2][w];
                    }
                    sf[j][4] = h[0] + h[1] + h[2];
                    ss[j][4] = h[1] + h[2] + h[3];
                    const int qz = md.z - q;  // n - (x1 - 1) + 1 - y0 - x0 of this plane
                    if (ph == kPhOut && tmin < qz) {
                        // output plane x1 - 1 (x1 the staged plane) from the
                        // sets of planes x1 - 2 (j + 1), x1 - 1 (j + 2) and x1
                        // (j); a warp tile with no domain cell skips it
                        const int P3 = (j + 1) % 3, Q = (j + 2) % 3;
                        const bool partial = qz < kPlaneTY + kPlaneTX - 1;  // not every cell of the brick plane
                        uint8_t *dst = reinterpret_cast<uint8_t *>(dbase) + q * ps +
                                       (BATCH ? (int64_t)(2 * P) * rs + 16 * C : toff);
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            uint32_t V[5], S[4], nw[4];
#pragma unroll
                            for (int w = 0; w < 5; ++w)
                                V[w] = r == 0 ? sf[P3][w] + sf[Q][w] + sf[j][w] : ss[P3][w] + ss[Q][w] + ss[j][w];
                            const uint32_t lft = __shfl_up_sync(0xffffffffu, V[3], 1, 4);
                            const uint32_t rgt = __shfl_down_sync(0xffffffffu, V[0], 1, 4);
                            hsum4(V, c == 0 ? V[4] : lft, c == 3 ? V[4] : rgt, S);
                            const uint32_t *A = r == 0 ? af[Q] : as[Q];
                            if constexpr (BATCH) {
                                // ORK: every instance's rule is or-k (its word in
                                // md2.y); else or-k or the general tables per instance
                                const int cnt = partial ? qz - tq - r : 16;
                                uint32_t dead[4];
                                chunk_dead4(cnt, dead);
                                if (ORK || md2.y)
                                    apply_rule4_ork_masked(S, A, (uint32_t)md2.y, dead, nw);
                                else
                                    apply_rule4_masked(S, A, bt.insts[md2.x].rule, dead, nw);
                                if (cnt > 0) store16(dst + r * rs, nw);
                            } else if (partial) {
                                // cells of the chunk in the domain: the first cnt
                                const int cnt = qz - tq - r;
                                uint32_t dead[4];
                                chunk_dead4(cnt, dead);
                                next_state4_masked<ORK>(S, A, rule, dead, nw);
                                if (cnt > 0) store16(dst + r * rs, nw);
                            } else {
                                next_state4<ORK>(S, A, rule, nw);
                                store16(dst + r * rs, nw);
                            }
                            acc += (nw[0] + nw[1]) + (nw[2] + nw[3]);
                        }
                    }
                }
                if (++slot == kPlStages) {
                    slot = 0;
                    parity ^= 1u;
                }
            }
            lsum += (acc * 0x01010101u) >> 24;  // bytes <= 48: their sum fits the top byte
            acc = 0;
            if (stop) break;
        }
        if (BATCH) flush();
    }

    __syncthreads();
    if (tid == kPlConsumerWarps * 32) {
        if (abort_flag) {
            atomicOr(&g_ca3p_status, 1u);
            // the last fill issued into each stage must land before the CTA exits
            for (int j = 1; j <= kPlStages && (uint64_t)j <= issued; ++j) {
                const uint64_t q = issued - j;
                mbar_wait_bounded(&full[q % kPlStages], (uint32_t)((q / kPlStages) & 1), kWaitLimitNs);
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
    e = cudaFuncSetAttribute(ca3_step_planes<ORK, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPlMaxSmem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

cudaError_t ca3_planes_prepare()
{
    cudaError_t e = prepare_planes_one<false, false>();
    if (e == cudaSuccess) e = prepare_planes_one<true, false>();
    if (e == cudaSuccess) e = prepare_planes_one<true, true>();
    return e != cudaSuccess ? e : prepare_planes_one<false, true>();
}

int plane_box_widths(int *w)
{
    for (int i = 0; i < kPlWidths; ++i) w[i] = plane_box_width(i);
    return kPlWidths;
}

// Resident CTAs of the plane-stream kernel with `smem` bytes of dynamic
// shared memory on the current device (SMs x occupancy).
static cudaError_t planes_resident(int smem, uint64_t *out)
{
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ca3_step_planes<true, false>, kPlThreads, smem)) !=
        cudaSuccess)
        return e;
    *out = (uint64_t)sms * (uint64_t)(occ < 1 ? 1 : occ);
    return cudaSuccess;
}

cudaError_t launch_ca3_planes(const PlaneSched &sched, const int32_t *segs, const PlaneMaps &maps, int64_t n,
                              int64_t side, uint8_t *out, const Rule &rule, unsigned long long *live,
                              unsigned long long *queue, cudaStream_t st)
{
    if (!queue || !segs || sched.nseg < 1 || sched.nseg > kPlaneMaxSegs) return cudaErrorInvalidValue;
    cudaError_t e = ca3_planes_prepare();
    if (e != cudaSuccess) return e;
    const int smem = plane_smem_bytes(sched.nseg, false);
    uint64_t resident = 0;
    if ((e = planes_resident(smem, &resident)) != cudaSuccess) return e;
    const uint64_t g = sched.units < resident ? (sched.units ? sched.units : 1) : resident;
    const PlaneBatch none = {};
    if (rule.or_k)
        ca3_step_planes<true, false><<<(unsigned)g, kPlThreads, smem, st>>>(maps, out, n, side, rule, sched, segs,
                                                                            live, queue, none);
    else
        ca3_step_planes<false, false><<<(unsigned)g, kPlThreads, smem, st>>>(maps, out, n, side, rule, sched, segs,
                                                                             live, queue, none);
    return cudaGetLastError();
}

cudaError_t launch_batch_planes(const PlaneBatch &bt, unsigned long long *queue, cudaStream_t st)
{
    if (!queue || !bt.nunits) return bt.nunits ? cudaErrorInvalidValue : cudaSuccess;
    cudaError_t e = ca3_planes_prepare();
    if (e != cudaSuccess) return e;
    const int smem = plane_smem_bytes(0, true);
    uint64_t resident = 0;
    if ((e = planes_resident(smem, &resident)) != cudaSuccess) return e;
    const uint64_t g = (uint64_t)bt.nunits < resident ? (uint64_t)bt.nunits : resident;
    static const PlaneMaps no_maps = {};
    static const PlaneSched no_sched = {};
    static const Rule no_rule = {};
    if (bt.all_ork)
        ca3_step_planes<true, true><<<(unsigned)g, kPlThreads, smem, st>>>(no_maps, nullptr, 0, 0, no_rule, no_sched,
                                                                           nullptr, nullptr, queue, bt);
    else
        ca3_step_planes<false, true><<<(unsigned)g, kPlThreads, smem, st>>>(no_maps, nullptr, 0, 0, no_rule,
                                                                            no_sched, nullptr, nullptr, queue, bt);
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
