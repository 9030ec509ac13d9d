// k_ca3.cu -- one step of a life-like automaton on the 3-simplex, fused with
// the map (Table 1 test 4 on the tetrahedron, fixed-dead boundary, Sec. 5.1).
//
// One CUDA block per tile of RHO^3 uint8 cells (axes x1 slow .. x3 fast).  The
// block decodes its tile with H (Sec. 4.3 packing with the hinge, or the
// generic beta = 3 cubes) or the bounding box, stages the tile plus a one-cell
// halo with a single 3-D TMA tiled load of (RHO + 32) x (RHO + 2) x (RHO + 2)
// bytes, and its threads walk the planes along x1 keeping 3 x 3 column sums of
// the staged rows in registers: the Moore-26 sum of a cell is one horizontal
// 3-sum over the column sums of three consecutive planes, all byte-parallel in
// 32-bit registers.
//
// For RHO = 32 the staged rows are 64 bytes and the tensor map uses the 64-byte
// swizzle (16-byte unit u of staged row R sits at u ^ ((R >> 1) & 3)); each
// thread owns two output rows (ca3_tile32) and the lanes of one 16-byte load
// instruction spread over all shared-memory banks.  Grid-form steps are
// launched with programmatic stream serialization (the next step's CTAs may
// start and decode their tiles once every CTA of this one has got past its
// own wait, and wait for it to complete before their first load).  The file also holds the
// x-stream form (ca3_step_stream, launch 2): persistent CTAs that stream runs
// of tiles along x3 through a ring of 32-byte-wide x-columns.
#include "ca_tiles.cuh"
#include "common.cuh"
#include "hmap.cuh"
#include "kernels.h"

namespace sx {

static __device__ uint32_t g_ca3_status;

// CTAs per SM the kernel is built for (shared memory allows 3 at RHO = 32).
// (Two CTAs of 16 planes per 32^3 tile, five per SM, ran 2 % slower.)
template <int RHO>
constexpr int ca3_min_blocks() { return RHO == 32 ? 3 : 12; }

// Threads per tile: RHO = 32 -- 32 lanes (2 chunks x 16 row pairs) per run of
// RZ planes; RHO = 16 -- one thread per (chunk, row, run of RZ planes).
// Planes per thread run for 32^3 tiles in the grid form (128 threads per tile
// at 8, 256 at 4).
constexpr int kCa3Rz32 = 8;

template <int RHO, int RZ>
constexpr int ca3_threads() { return RHO == 32 ? 32 * (RHO / RZ) : (RHO / 16) * RHO * (RHO / RZ); }

// Staged box bytes and the alignment its swizzle needs.
template <int RHO>
__host__ __device__ constexpr uint32_t ca3_box_bytes() { return (RHO + 32) * (RHO + 2) * (RHO + 2); }
template <int RHO>
__host__ __device__ constexpr int ca3_box_align() { return RHO == 32 ? 512 : 128; }

template <int RHO, int RZ, bool ORK>
__global__ void __launch_bounds__(ca3_threads<RHO, RZ>(), ca3_min_blocks<RHO>())
    ca3_step_kernel(const __grid_constant__ CUtensorMap tin, uint8_t *__restrict__ out, const Plan p,
                    const Rule rule, int kind, uint64_t nblocks, unsigned long long *__restrict__ live)
{
    constexpr int TX = RHO / 16;
    constexpr uint32_t kBoxBytes = ca3_box_bytes<RHO>();
    constexpr uintptr_t kAlign = ca3_box_align<RHO>();
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t red[32];
    uint8_t *tile = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + kAlign - 1) & ~(kAlign - 1));

    const int tid = threadIdx.x;
    const int tx = tid % TX;
    const int ty = (tid / TX) % RHO;         // x2 within the tile
    const int tz = tid / (TX * RHO);         // plane segment along x1
    uint32_t phase = 0, my_live = 0;
    if (tid == 0) {
        prefetch_tmap(&tin);
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool waited = false;  // CTA-uniform

    for (uint64_t v = blockIdx.x; v < nblocks; v += gridDim.x) {
        int32_t X[3];
        if (!decode<3>(p, kind, v, X)) continue;
        const int64_t z0 = (int64_t)X[0] * RHO, y0 = (int64_t)X[1] * RHO, x0 = (int64_t)X[2] * RHO;
        if (z0 + y0 + x0 > p.n && kind != kMapBBThread) continue;
        const bool partial = z0 + y0 + x0 + 3 * (RHO - 1) > p.n;
        if (!waited) {  // the previous step writes this step's input and reads its output
            grid_dep_wait();
            grid_dep_trigger();  // the next step may start (at most one step ahead)
            waited = true;
        }
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar, kBoxBytes);
            tma_load_3d(tile, &tin, (int32_t)(x0 - 16), (int32_t)(y0 - 1), (int32_t)(z0 - 1), &bar);
        }
        const bool ok = mbar_wait_bounded(&bar, phase, kWaitLimitNs);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&g_ca3_status, 1u);
                mbar_wait_bounded(&bar, phase ^ 1u, kWaitLimitNs);
            }
            return;
        }

        if constexpr (RHO == 32)
            my_live += ca3_tile32<RZ, ORK>(tile, p.n, p.side, rule, out, x0, y0, z0, partial, tid & 1, (tid >> 1) & 15,
                                           tid >> 5);
        else
            my_live += ca3_tile<RHO, RZ, ORK>(tile, p.n, p.side, rule, out, x0, y0, z0, partial, tx, ty, tz);
        __syncthreads();
    }
    if (live) block_add_u64(live, my_live, red);
}

// ---------------------------------------------------------------------------
// x-stream form (32^3 tiles): one CTA per SM takes work units from a device
// counter.  A tile column (X1, X2) (xrun_decode: H2 over the triangle of
// columns, or the bounding square) is cut into runs of up to seg_len tiles
// along x3, and every run into kStreamZSplit slabs of 32 / kStreamZSplit
// planes along x1: unit w is slab w % kStreamZSplit of run w / kStreamZSplit,
// so the slabs of one run go to different CTAs at about the same time and
// share their halo planes in L2.  A slab run of tiles X3 = a ... b needs the
// x-columns a - 1 ... b + 1 (32 x 34 x kStreamColPlanes bytes each: the
// slab's cells plus the x1/x2 halo), so every column is read once per run
// instead of each tile reading a box with 16-byte x halos on both sides (3
// sectors of 32 bytes per 32-byte row).
//
// The last warp (one lane) is the producer.  Per run it first publishes a
// header (the run and the sequence number of its first column) in a ring of
// kStreamHeaders entries (hfull: one plain arrival; hempty: one arrival per
// consumer warp once it has read the header), then TMA-loads the run's columns
// in order into a ring of kStreamSlots stages (full: the bytes; empty: see
// below).  After the last unit it publishes an end header (a > b).
// The consumers form kStreamGroups groups of kStreamGroupWarps warps; group g
// takes the tiles g, g + G, ... of the CTA's tile sequence, so G slab tiles
// are computed at once, each by 2 warps walking 8 planes per thread.  Column c
// of a run is the centre of tile c and a neighbour of tiles c - 1 and c + 1:
// every column has exactly three uses (a tile at a run's end also performs the
// uses of the tiles missing beyond it), so empty completes after 3 x
// kStreamGroupWarps warp arrivals, when every tile reading the column is done;
// a column is never refilled while a group that has not reached its tile still
// needs it.  Every wait is bounded; a timeout sets the status word and an
// abort flag that stops both sides, and the producer then waits (bounded) for
// the loads it issued before the CTA exits.  The last CTA to finish puts the
// work counter back to zero.
constexpr int kStreamSlots = 11;
constexpr int kStreamHeaders = 8;
constexpr int kStreamGroups = 5;
constexpr int kStreamGroupWarps = 32 / kStreamZSplit / 8;  // 2 chunks x 16 row pairs x runs of 8 planes
constexpr int kStreamConsumers = kStreamGroups * kStreamGroupWarps * 32;
constexpr int kStreamThreads = kStreamConsumers + 32;
constexpr uint32_t kColBytes = 32u * 34u * (uint32_t)kStreamColPlanes;  // 19,584 = 153 x 128
constexpr int kStreamSmem = kStreamSlots * (int)kColBytes + 128;
static_assert(kColBytes % 128 == 0, "ring slots must stay 128-byte aligned");
static_assert(kStreamSmem <= 227 * 1024, "ring exceeds the shared memory of one CTA");

template <bool ORK>
__global__ void __launch_bounds__(kStreamThreads, 1)
    ca3_step_stream(const __grid_constant__ CUtensorMap tcol, uint8_t *__restrict__ out, const Plan p,
                    const Rule rule, int kind, uint64_t units, unsigned long long *__restrict__ live,
                    unsigned long long *__restrict__ queue)
{
    constexpr int S = kStreamSlots, HN = kStreamHeaders, G = kStreamGroups;
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t full[S], empty[S], hfull[HN], hempty[HN];
    __shared__ int4 hdr[HN];             // X1, X2, a, b of the run (a > b: no more work)
    __shared__ unsigned long long hseq[HN];  // sequence number of the run's first column
    __shared__ uint32_t red[32];
    __shared__ volatile int abort_flag;
    uint8_t *ring = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t my_live = 0;
    uint64_t issued = 0;  // producer: columns loaded
    if (tid == 0) {
        prefetch_tmap(&tcol);
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 3 * kStreamGroupWarps);
        }
        for (int h = 0; h < HN; ++h) {
            mbar_init(&hfull[h], 1);
            mbar_init(&hempty[h], G * kStreamGroupWarps);
        }
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    if (warp == kStreamConsumers / 32) {
        // producer
        if (lane == 0) {
            uint64_t seq = 0, nh = 0;
            bool ok = true;
            auto header = [&](int4 r) {  // publish header nh
                const int h = (int)(nh % HN);
                if (nh >= (uint64_t)HN &&
                    !mbar_wait_bounded(&hempty[h], (uint32_t)((nh / HN - 1) & 1), kWaitLimitNs))
                    return false;
                hdr[h] = r;
                hseq[h] = seq;
                ++nh;
                mbar_arrive(&hfull[h]);
                return true;
            };
            while (ok) {
                const uint64_t w = atomicAdd(&queue[0], 1ull);
                if (w >= units) break;
                XRun r;
                if (!xrun_decode(p, kind, w / kStreamZSplit, r)) continue;
                // slab zs: planes z0 ... z0 + 32 / kStreamZSplit - 1; its tiles
                // hold cells while X3 * 32 <= n - z0 - y0
                const int32_t zs = r.X1 * kStreamZSplit + (int32_t)(w % kStreamZSplit);
                const int64_t reach = (p.n - (int64_t)zs * (32 / kStreamZSplit) - (int64_t)r.X2 * 32) >> 5;
                if (reach < (int64_t)r.b) r.b = (int32_t)reach;
                if (r.b < r.a) continue;
                if (!(ok = header(make_int4(zs, r.X2, r.a, r.b)))) break;
                // the slab's right-halo column past its run holds live cells only
                // if x3 = c * 32 can be reached from the halo rows (x1 >= z0 - 1,
                // x2 >= y0 - 1); else it is all zeros and is not loaded (the
                // consumers see it as absent: stream_has_right)
                const int64_t hreach = p.n - (int64_t)zs * (32 / kStreamZSplit) - (int64_t)r.X2 * 32 + 2;
                for (int32_t c = r.a - 1; c <= r.b + 1; ++c, ++seq) {
                    const int s = (int)(seq % S);
                    if (seq >= (uint64_t)S &&
                        !(ok = mbar_wait_bounded(&empty[s], (uint32_t)((seq / S - 1) & 1), kWaitLimitNs)))
                        break;
                    if (c == r.b + 1 && (int64_t)c * 32 > hreach) {
                        mbar_arrive(&full[s]);  // an empty column: the phase completes with no bytes
                        continue;
                    }
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&full[s], kColBytes);
                    tma_load_3d(ring + s * kColBytes, &tcol, c * 32, r.X2 * 32 - 1, zs * (32 / kStreamZSplit) - 1,
                                &full[s]);
                }
            }
            issued = seq;
            if (ok) ok = header(make_int4(0, 0, 1, 0));
            if (!ok) abort_flag = 1;
        }
    } else {
        // consumers
        const int grp = warp / kStreamGroupWarps, tz = warp % kStreamGroupWarps;
        const int tx = lane & 1, pr = lane >> 1;
        uint64_t nh = 0;
        uint32_t t0 = 0;  // tiles of the sequence before the current run
        for (;;) {
            const int h = (int)(nh % HN);
            if (abort_flag || !mbar_wait_bounded(&hfull[h], (uint32_t)((nh / HN) & 1), kWaitLimitNs)) {
                abort_flag = 1;
                break;
            }
            const int4 r = hdr[h];
            const uint64_t seq = hseq[h];
            __syncwarp();
            if (lane == 0) mbar_arrive(&hempty[h]);
            ++nh;
            if (r.z > r.w) break;  // end header
            const int64_t z0 = (int64_t)r.x * (32 / kStreamZSplit), y0 = (int64_t)r.y * 32;
            bool ok = true;
            const int32_t first = r.z + (int32_t)((uint32_t)(grp - (int)(t0 % G) + G) % G);
            for (int32_t x3 = first; x3 <= r.w && ok; x3 += G) {
                const uint64_t c = seq + (uint64_t)(x3 - r.z) + 1;  // centre column of this tile
                for (uint64_t q = c - 1; q <= c + 1 && ok; ++q)
                    ok = !abort_flag && mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), kWaitLimitNs);
                if (!ok) break;
                const int64_t x0 = (int64_t)x3 * 32;
                const bool partial = z0 + y0 + x0 + (32 / kStreamZSplit - 1) + 2 * 31 > p.n;
                my_live += ca3_tile32c<8, ORK>(ring + (c % S) * kColBytes, ring + ((c - 1) % S) * kColBytes,
                                               ring + ((c + 1) % S) * kColBytes, x3 > 0,
                                               x0 + 32 <= p.n - z0 - y0 + 2, p.n, p.side,
                                               rule, out, x0, y0, z0, partial, tx, pr, tz);
                __syncwarp();
                if (lane == 0) {
                    const bool fst = x3 == r.z, lst = x3 == r.w;
                    mbar_arrive_n(&empty[(c - 1) % S], fst ? 3u : 1u);
                    mbar_arrive_n(&empty[c % S], 1u + (fst ? 1u : 0u) + (lst ? 1u : 0u));
                    mbar_arrive_n(&empty[(c + 1) % S], lst ? 3u : 1u);
                }
            }
            if (!ok) {
                abort_flag = 1;
                break;
            }
            t0 += (uint32_t)(r.w - r.z + 1);
        }
    }
    __syncthreads();
    if (tid == kStreamConsumers) {
        if (abort_flag) {
            atomicOr(&g_ca3_status, 2u);
            // the last fill issued into each stage must land before the CTA exits
            for (int j = 1; j <= S && (uint64_t)j <= issued; ++j) {
                const uint64_t q = issued - j;
                mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), kWaitLimitNs);
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
    if (live) block_add_u64(live, my_live, red);
}

bool ca3_supports(int rho) { return rho == 16 || rho == 32; }

int ca3_box_planes(const Plan &p)
{
    return p.persistent == 1 ? kStreamColPlanes : p.rho + 2;
}

// The 64-byte swizzle the tensor map must use for this tile side (see above).
bool ca3_swizzled(int rho) { return rho == 32; }

template <int RHO, int RZ, bool ORK>
static cudaError_t prepare_one()
{
    constexpr int smem = ca3_box_bytes<RHO>() + ca3_box_align<RHO>();
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(ca3_step_kernel<RHO, RZ, ORK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

template <int RHO, int RZ>
static cudaError_t prepare_t()
{
    cudaError_t e = prepare_one<RHO, RZ, false>();
    return e != cudaSuccess ? e : prepare_one<RHO, RZ, true>();
}

template <int RHO, int RZ>
static cudaError_t launch_t(const Plan &p, const CUtensorMap &tin, uint8_t *out, const Rule &rule, int kind,
                            unsigned long long *live, cudaStream_t st)
{
    constexpr int T = ca3_threads<RHO, RZ>();
    constexpr int smem = ca3_box_bytes<RHO>() + ca3_box_align<RHO>();
    cudaError_t e = prepare_t<RHO, RZ>();
    if (e != cudaSuccess) return e;
    const uint64_t nb = is_bb(kind) ? p.bb_blocks : p.h_blocks;
    const unsigned g = (unsigned)(nb < 0x7fffffffull ? (nb ? nb : 1) : 0x7fffffffull);
    if (rule.or_k)
        return launch_pdl(ca3_step_kernel<RHO, RZ, true>, dim3(g), dim3(T), (size_t)smem, st, tin, out, p, rule, kind,
                          nb, live);
    return launch_pdl(ca3_step_kernel<RHO, RZ, false>, dim3(g), dim3(T), (size_t)smem, st, tin, out, p, rule, kind,
                      nb, live);
}

template <bool ORK>
static cudaError_t prepare_stream_one()
{
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(ca3_step_stream<ORK>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamSmem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

static cudaError_t launch_stream(const Plan &p, const CUtensorMap &tcol, uint8_t *out, const Rule &rule, int kind,
                                 unsigned long long *live, unsigned long long *queue, cudaStream_t st)
{
    if (!queue) return cudaErrorInvalidValue;
    cudaError_t e = prepare_stream_one<false>();
    if (e == cudaSuccess) e = prepare_stream_one<true>();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const uint64_t units = xrun_units(p, kind) * kStreamZSplit;
    const uint64_t g = units < (uint64_t)sms ? (units ? units : 1) : (uint64_t)sms;  // one CTA per SM
    if (rule.or_k)
        ca3_step_stream<true><<<(unsigned)g, kStreamThreads, kStreamSmem, st>>>(tcol, out, p, rule, kind, units, live,
                                                                                 queue);
    else
        ca3_step_stream<false><<<(unsigned)g, kStreamThreads, kStreamSmem, st>>>(tcol, out, p, rule, kind, units, live,
                                                                                  queue);
    return cudaGetLastError();
}

cudaError_t launch_ca3_step(const Plan &p, const CUtensorMap &tin, uint8_t *out, const Rule &rule, int kind,
                            unsigned long long *live, unsigned long long *queue, cudaStream_t st)
{
    if (p.persistent == 1 && p.rho == 32) return launch_stream(p, tin, out, rule, kind, live, queue, st);
    switch (p.rho) {
    case 16: return launch_t<16, 4>(p, tin, out, rule, kind, live, st);
    case 32: return launch_t<32, kCa3Rz32>(p, tin, out, rule, kind, live, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t ca3_prepare(int rho)
{
    if (rho == 32) {
        cudaError_t e = prepare_stream_one<false>();
        if (e == cudaSuccess) e = prepare_stream_one<true>();
        if (e != cudaSuccess) return e;
    }
    switch (rho) {
    case 16: return prepare_t<16, 4>();
    case 32: return prepare_t<32, kCa3Rz32>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t ca3_read_status(uint32_t *out)
{
    uint32_t zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_ca3_status, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_ca3_status, &zero, sizeof(uint32_t));
}

}  // namespace sx
