// k_ca2.cu -- one step of a life-like automaton on the 2-simplex, fused with
// the map (Table 1 test 4, Sec. 5.1).
//
// One CUDA block per tile of RHO x RHO uint8 cells.  The block
//   1. decodes its tile with H (Eq. map2d + diagonal row) or the bounding box;
//   2. stages the tile plus a one-cell halo in shared memory with a single TMA
//      tiled load of (RHO + 32) x (RHO + 2) bytes: the box starts 16 bytes left
//      of the tile (TMA x coordinates must be 16-byte aligned) and one row
//      above; cells outside the array read as 0;
//   3. lets each thread walk down R rows of one 16-byte column chunk, keeping
//      the horizontal 3-sums of three rows in registers, so the Moore sum of
//      16 cells comes from byte-parallel 32-bit adds (cells are 0/1, sums
//      never carry across bytes);
//   4. applies the rule byte-parallel and writes 16 cells per 16-byte store;
//   5. adds its live cells to the step's counter: new states (0/1 bytes) are
//      summed byte-wise per thread, folded once per tile, reduced per CTA and
//      added with one atomic per CTA.
// Only tiles on the diagonal band mask cells past x1 + x2 = n.  Steps are
// launched with programmatic stream serialization: once every CTA of a step
// has got past its own wait for the step before, the next step's CTAs may
// start, decode their tiles and wait for the step to complete before their
// first load.
#include "ca_tiles.cuh"
#include "common.cuh"
#include "hmap.cuh"
#include "kernels.h"

namespace sx {

static __device__ uint32_t g_ca2_status;

// CTAs per SM the kernel is built for (the 128 x 128 tile's shared memory
// allows 10; smaller tiles are limited by threads).
template <int RHO>
constexpr int ca2_min_blocks() { return RHO == 128 ? 10 : 16; }

template <int RHO, int R, bool ORK>
__global__ void __launch_bounds__(RHO * RHO / (16 * R), ca2_min_blocks<RHO>())
    ca2_step_kernel(const __grid_constant__ CUtensorMap tin, uint8_t *__restrict__ out, const Plan p,
                    const Rule rule, int kind, uint64_t nblocks, unsigned long long *__restrict__ live)
{
    constexpr int TX = RHO / 16;                // 16-byte chunks per tile row
    constexpr int BW = RHO + 32;                // staged row: 16-byte halo each side
    constexpr int BH = RHO + 2;                 // staged rows: one halo row each side
    constexpr uint32_t kBoxBytes = BW * BH;
    extern __shared__ uint8_t dsmem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t red[32];
    uint8_t *tile = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsmem) + 127) & ~uintptr_t(127));

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    uint32_t phase = 0, my_live = 0;
    if (tid == 0) {
        prefetch_tmap(&tin);
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool waited = false;  // CTA-uniform

    for (uint64_t v = blockIdx.x; v < nblocks; v += gridDim.x) {
        int32_t X[2];
        if (!decode<2>(p, kind, v, X)) continue;
        const int64_t y0 = (int64_t)X[0] * RHO, x0 = (int64_t)X[1] * RHO;
        if (y0 + x0 > p.n && kind != kMapBBThread) continue;  // tile past the domain
        const bool partial = y0 + x0 + 2 * (RHO - 1) > p.n;
        if (!waited) {  // the previous step writes this step's input and reads its output
            grid_dep_wait();
            grid_dep_trigger();  // the next step may start (at most one step ahead)
            waited = true;
        }
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar, kBoxBytes);
            tma_load_2d(tile, &tin, (int32_t)(x0 - 16), (int32_t)(y0 - 1), &bar);
        }
        const bool ok = mbar_wait_bounded(&bar, phase, kWaitLimitNs);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&g_ca2_status, 1u);
                mbar_wait_bounded(&bar, phase ^ 1u, kWaitLimitNs);
            }
            return;
        }

        my_live += ca2_tile<RHO, R, ORK>(tile, p.n, p.side, rule, out, x0, y0, partial, tx, ty);
        __syncthreads();  // the tile is fully read before the next load reuses it
    }
    if (live) block_add_u64(live, my_live, red);
}

// Self-test of the bounded wait: one CTA waits on an mbarrier that nothing
// completes, gives up after limit_ns, records status bit 2 and returns.
__global__ void wait_selftest_kernel(uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(&g_ca2_status, 2u);
}

cudaError_t launch_wait_selftest(uint64_t limit_ns, cudaStream_t st)
{
    wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns);
    return cudaGetLastError();
}

bool ca2_supports(int rho) { return rho == 32 || rho == 64 || rho == 128; }

template <int RHO, int R, bool ORK>
static cudaError_t prepare_one()
{
    constexpr int smem = (RHO + 32) * (RHO + 2) + 128;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && attr_set[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(ca2_step_kernel<RHO, R, ORK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_set[dev] = true;
    return e;
}

template <int RHO, int R>
static cudaError_t prepare_t()
{
    cudaError_t e = prepare_one<RHO, R, false>();
    return e != cudaSuccess ? e : prepare_one<RHO, R, true>();
}

template <int RHO, int R>
static cudaError_t launch_t(const Plan &p, const CUtensorMap &tin, uint8_t *out, const Rule &rule, int kind,
                            unsigned long long *live, cudaStream_t st)
{
    constexpr int T = RHO * RHO / (16 * R);
    constexpr int smem = (RHO + 32) * (RHO + 2) + 128;
    cudaError_t e = prepare_t<RHO, R>();
    if (e != cudaSuccess) return e;
    const uint64_t nb = is_bb(kind) ? p.bb_blocks : p.h_blocks;
    const unsigned g = (unsigned)(nb < 0x7fffffffull ? (nb ? nb : 1) : 0x7fffffffull);
    if (rule.or_k)
        return launch_pdl(ca2_step_kernel<RHO, R, true>, dim3(g), dim3(T), (size_t)smem, st, tin, out, p, rule, kind,
                          nb, live);
    return launch_pdl(ca2_step_kernel<RHO, R, false>, dim3(g), dim3(T), (size_t)smem, st, tin, out, p, rule, kind, nb,
                      live);
}

cudaError_t launch_ca2_step(const Plan &p, const CUtensorMap &tin, uint8_t *out, const Rule &rule, int kind,
                            unsigned long long *live, cudaStream_t st)
{
    switch (p.rho) {
    case 32: return launch_t<32, 2>(p, tin, out, rule, kind, live, st);
    case 64: return launch_t<64, 4>(p, tin, out, rule, kind, live, st);
    case 128: return launch_t<128, 8>(p, tin, out, rule, kind, live, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t ca2_prepare(int rho)
{
    switch (rho) {
    case 32: return prepare_t<32, 2>();
    case 64: return prepare_t<64, 4>();
    case 128: return prepare_t<128, 8>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t ca2_read_status(uint32_t *out)
{
    uint32_t zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_ca2_status, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_ca2_status, &zero, sizeof(uint32_t));
}

}  // namespace sx
