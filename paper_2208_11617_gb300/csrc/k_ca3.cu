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
// instruction spread over all shared-memory banks.
#include "ca_tiles.cuh"
#include "common.cuh"
#include "hmap.cuh"
#include "kernels.h"

namespace sx {

static __device__ uint32_t g_ca3_status;

// CTAs per SM the kernel is built for (shared memory allows 3 at RHO = 32).
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

    for (uint64_t v = blockIdx.x; v < nblocks; v += gridDim.x) {
        int32_t X[3];
        if (!decode<3>(p, kind, v, X)) continue;
        const int64_t z0 = (int64_t)X[0] * RHO, y0 = (int64_t)X[1] * RHO, x0 = (int64_t)X[2] * RHO;
        if (z0 + y0 + x0 > p.n) continue;
        const bool partial = z0 + y0 + x0 + 3 * (RHO - 1) > p.n;
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
// Persistent form: one CTA per SM walks the map's blocks v = blockIdx.x,
// blockIdx.x + gridDim.x, ... (the same H or bounding-box decode) through a
// ring of S shared-memory stages.  Thread 0 keeps S - 1 TMA loads in flight
// ahead of the tile the CTA is computing, so loads and compute overlap
// instead of every CTA waiting for its own load.
template <int RHO, int T>
struct Ca3Persist {
    static_assert(RHO == 32, "the persistent form stages 32^3 tiles");
    static constexpr int ZS = T / 32;  // plane runs per tile (32 lanes each)
    static constexpr int RZ = RHO / ZS;
    static constexpr uint32_t kBox = ca3_box_bytes<RHO>();
    static constexpr uint32_t kStage = (kBox + 511u) & ~511u;
    static constexpr int S = (3 * kStage + 512 <= 227 * 1024) ? 3 : 2;
    static constexpr int kSmem = S * kStage + 512;
};

template <int RHO, int T, bool ORK>
__global__ void __launch_bounds__(T, 1)
    ca3_step_persistent(const __grid_constant__ CUtensorMap tin, uint8_t *__restrict__ out, const Plan p,
                        const Rule rule, int kind, uint64_t nblocks, unsigned long long *__restrict__ live)
{
    using C = Ca3Persist<RHO, T>;
    constexpr int S = C::S;
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ int4 info[S];  // x0, y0, z0 of the staged tile; w: 1 = valid, 2 = partial
    __shared__ uint32_t red[32];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 511) & ~uintptr_t(511));
    const int tid = threadIdx.x;
    uint64_t vnext = blockIdx.x;  // producer state (thread 0)
    uint32_t my_live = 0;

    // thread 0: find the next block with a tile and start its load into stage s
    auto produce = [&](int s) {
        while (vnext < nblocks) {
            const uint64_t v = vnext;
            vnext += gridDim.x;
            int32_t X[3];
            if (!decode<3>(p, kind, v, X)) continue;
            const int64_t z0 = (int64_t)X[0] * RHO, y0 = (int64_t)X[1] * RHO, x0 = (int64_t)X[2] * RHO;
            if (z0 + y0 + x0 > p.n) continue;
            const bool partial = z0 + y0 + x0 + 3 * (RHO - 1) > p.n;
            info[s] = make_int4((int)x0, (int)y0, (int)z0, 1 | (partial ? 2 : 0));
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&full[s], C::kBox);
            tma_load_3d(base + s * C::kStage, &tin, (int32_t)(x0 - 16), (int32_t)(y0 - 1), (int32_t)(z0 - 1),
                        &full[s]);
            return;
        }
        info[s] = make_int4(0, 0, 0, 0);
    };

    if (tid == 0) {
        prefetch_tmap(&tin);
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
        for (int s = 0; s < S; ++s) produce(s);
    }
    __syncthreads();

    for (int k = 0;; ++k) {
        const int s = k % S;
        const int4 inf = info[s];
        if (!(inf.w & 1)) break;  // the producer ran out of tiles (uniform)
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k / S) & 1), kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&g_ca3_status, 1u);
                // wait (bounded) for every load still in flight before leaving
                for (int j = 0; j < S; ++j)
                    if (info[(k + j) % S].w & 1)
                        mbar_wait_bounded(&full[(k + j) % S], (uint32_t)(((k + j) / S) & 1), kWaitLimitNs);
            }
            return;
        }
        my_live += ca3_tile32<C::RZ, ORK>(base + s * C::kStage, p.n, p.side, rule, out, inf.x, inf.y, inf.z,
                                           (inf.w & 2) != 0, tid & 1, (tid >> 1) & 15, tid >> 5);
        __syncthreads();  // stage s fully read
        if (tid == 0) produce(s);
    }
    if (live) block_add_u64(live, my_live, red);
}

bool ca3_supports(int rho) { return rho == 16 || rho == 32; }

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
    const uint64_t nb = kind == kMapBB ? p.bb_blocks : p.h_blocks;
    const unsigned g = (unsigned)(nb < 0x7fffffffull ? (nb ? nb : 1) : 0x7fffffffull);
    if (rule.or_k)
        ca3_step_kernel<RHO, RZ, true><<<g, T, smem, st>>>(tin, out, p, rule, kind, nb, live);
    else
        ca3_step_kernel<RHO, RZ, false><<<g, T, smem, st>>>(tin, out, p, rule, kind, nb, live);
    return cudaGetLastError();
}

constexpr int kCa3PersistThreads = 256;

template <bool ORK>
static cudaError_t prepare_persist_one()
{
    using C = Ca3Persist<32, kCa3PersistThreads>;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(ca3_step_persistent<32, kCa3PersistThreads, ORK>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

static cudaError_t launch_persist(const Plan &p, const CUtensorMap &tin, uint8_t *out, const Rule &rule, int kind,
                                  unsigned long long *live, cudaStream_t st)
{
    using C = Ca3Persist<32, kCa3PersistThreads>;
    cudaError_t e = prepare_persist_one<false>();
    if (e == cudaSuccess) e = prepare_persist_one<true>();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const uint64_t nb = kind == kMapBB ? p.bb_blocks : p.h_blocks;
    const uint64_t g = nb < (uint64_t)sms ? (nb ? nb : 1) : (uint64_t)sms;  // one CTA per SM
    if (rule.or_k)
        ca3_step_persistent<32, kCa3PersistThreads, true><<<(unsigned)g, kCa3PersistThreads, C::kSmem, st>>>(
            tin, out, p, rule, kind, nb, live);
    else
        ca3_step_persistent<32, kCa3PersistThreads, false><<<(unsigned)g, kCa3PersistThreads, C::kSmem, st>>>(
            tin, out, p, rule, kind, nb, live);
    return cudaGetLastError();
}

cudaError_t launch_ca3_step(const Plan &p, const CUtensorMap &tin, uint8_t *out, const Rule &rule, int kind,
                            unsigned long long *live, cudaStream_t st)
{
    if (p.persistent && p.rho == 32) return launch_persist(p, tin, out, rule, kind, live, st);
    switch (p.rho) {
    case 16: return launch_t<16, 4>(p, tin, out, rule, kind, live, st);
    case 32: return launch_t<32, kCa3Rz32>(p, tin, out, rule, kind, live, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t ca3_prepare(int rho)
{
    if (rho == 32) {
        cudaError_t e = prepare_persist_one<false>();
        if (e == cudaSuccess) e = prepare_persist_one<true>();
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
