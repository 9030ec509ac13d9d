// k_diag.cu -- the paper's diagnostic tests (Table 1): MAP, the map alone, and
// EDM, the Euclidean distance matrix on the 2-simplex (Sec. 5.1).
//
// MAP.  One CUDA block of rho^m threads per block of the map, one thread per
// cell (the paper's execution model, Sec. 2): the block decodes its tile with
// H or the bounding box, every thread forms its cell coordinate and the
// predicate x_1 + ... + x_m <= n, and the result is kept alive by an empty
// asm statement that consumes it (the paper uses a volatile variable), so the
// kernel does no memory traffic and its time is the map plus the cost of
// launching and retiring the grid's blocks.  With `cells` given, each block
// adds the number of its simplex cells to *cells (the coverage check: the
// total must be C(n + m, m)).
//
// EDM (m = 2).  Cell x = (x1, x2) of the 2-simplex stands for the pair of
// points (i, j) = (x1, n - x2), i <= j, and receives d(p_i, p_j) as float32:
// the upper triangle of the distance matrix of n + 1 points, diagonal
// included.  One block per tile of rho x rho cells; every thread reads its
// points straight from global memory (3-D points get an unrolled kernel),
// computes 4 consecutive cells along x2 and writes them with one 16-byte
// store (4-byte stores where rows are not 16-byte aligned or on the
// diagonal).  Arithmetic is fp32 in a fixed order without contraction
// (d^2 = sum over k of (p_ik - p_jk)^2, k = 0, 1, ...) and a correctly
// rounded square root.
#include "common.cuh"
#include "hmap.cuh"
#include "kernels.h"

namespace sx {

template <int M>
__global__ void map_kernel(const Plan p, int kind, uint64_t nblocks, unsigned long long *__restrict__ cells)
{
    __shared__ uint32_t red[32];
    const uint64_t v = blockIdx.x;
    int32_t X[M];
    if (v >= nblocks || !decode<M>(p, kind, v, X)) return;  // block-uniform
    const uint32_t t = threadIdx.x;
    int64_t s = 0, lin = 0;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int sh = (M - 1 - i) * p.log_rho;
        const int64_t xi = (int64_t)X[i] * p.rho + (int64_t)((t >> sh) & (uint32_t)(p.rho - 1));
        s += xi;
        lin = lin * p.side + xi;
    }
    const bool inside = s <= p.n;
    if (cells) {
        block_add_u64(cells, inside ? 1u : 0u, red);
    } else {
        const uint32_t r = inside ? (uint32_t)lin : 0xffffffffu;
        asm volatile("" ::"r"(r));
    }
}

template <int M>
static cudaError_t launch_map_t(const Plan &p, int kind, unsigned long long *cells, cudaStream_t st)
{
    const uint64_t nb = is_bb(kind) ? p.bb_blocks : p.h_blocks;
    const uint32_t threads = 1u << (M * p.log_rho);
    if (nb > 0x7fffffffull || threads > 1024) return cudaErrorInvalidConfiguration;
    map_kernel<M><<<(unsigned)(nb ? nb : 1), threads, 0, st>>>(p, kind, nb, cells);
    return cudaGetLastError();
}

cudaError_t launch_map_test(const Plan &plan, int kind, unsigned long long *cells, cudaStream_t st)
{
    const Plan p = single_grid(plan);
    switch (p.m) {
    case 2: return launch_map_t<2>(p, kind, cells, st);
    case 3: return launch_map_t<3>(p, kind, cells, st);
    case 4: return launch_map_t<4>(p, kind, cells, st);
    default: return cudaErrorInvalidValue;
    }
}

constexpr int kEdmMaxDim = 16;

template <int RHO, int DIM>
__global__ void __launch_bounds__(RHO * RHO / 4)
    edm_kernel(const Plan p, int kind, const float *__restrict__ pts, int dim_rt, float *__restrict__ out, int vec)
{
    const int dim = DIM > 0 ? DIM : dim_rt;
    int32_t X[2];
    if (!decode<2>(p, kind, blockIdx.x, X)) return;
    const int64_t x1_0 = (int64_t)X[0] * RHO, x2_0 = (int64_t)X[1] * RHO;
    if (x1_0 + x2_0 > p.n && kind != kMapBBThread) return;
    const bool partial = x1_0 + x2_0 + 2 * (RHO - 1) > p.n;
    constexpr int kChunks = RHO / 4;
    const int row = threadIdx.x / kChunks, ch = threadIdx.x - row * kChunks;
    const int64_t x1 = x1_0 + row, x2 = x2_0 + 4 * ch;
    const int64_t valid = p.n - x1 - x2 + 1;  // cells of the chunk inside the simplex
    if (partial && valid <= 0) return;
    // point i = x1 and points j = n - x2 - c, read straight from global memory
    // (the points are a few hundred KB: L1 and L2 hits after the first touch)
    const float *a = pts + x1 * dim;
    float d[4];
    if (DIM > 0 && (!partial || valid >= 4)) {
        // all four j exist: point j0 - c sits c * DIM floats below point j0
        float ai[DIM > 0 ? DIM : 1];
#pragma unroll
        for (int k = 0; k < DIM; ++k) ai[k] = __ldg(a + k);
        const float *b0 = pts + (p.n - x2) * DIM;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const float df = __fsub_rn(ai[k], __ldg(b0 - c * DIM + k));
                acc = __fadd_rn(acc, __fmul_rn(df, df));
            }
            d[c] = __fsqrt_rn(acc);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = p.n - x2 - c;
            const float *b = pts + (j >= 0 ? j : 0) * dim;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < (DIM > 0 ? DIM : kEdmMaxDim); ++k) {
                if (DIM == 0 && k >= dim) break;
                const float df = __fsub_rn(__ldg(a + k), __ldg(b + k));
                acc = __fadd_rn(acc, __fmul_rn(df, df));
            }
            d[c] = __fsqrt_rn(acc);
        }
    }
    float *dst = out + x1 * p.side + x2;
    if (vec && (!partial || valid >= 4)) {
        *reinterpret_cast<float4 *>(dst) = make_float4(d[0], d[1], d[2], d[3]);
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c < valid) dst[c] = d[c];
    }
}

bool edm_supports(int rho) { return rho == 16 || rho == 32 || rho == 64; }

cudaError_t launch_edm(const Plan &plan, const float *pts, int dim, float *out, int kind, bool vec, cudaStream_t st)
{
    const Plan p = single_grid(plan);
    if (dim < 1 || dim > kEdmMaxDim) return cudaErrorInvalidValue;
    const uint64_t nb = is_bb(kind) ? p.bb_blocks : p.h_blocks;
    if (nb > 0x7fffffffull) return cudaErrorInvalidConfiguration;
    const unsigned g = (unsigned)(nb ? nb : 1);
    const int v = vec ? 1 : 0;
    switch (p.rho * 100 + (dim == 3 ? 3 : 0)) {
    case 1603: edm_kernel<16, 3><<<g, 64, 0, st>>>(p, kind, pts, dim, out, v); break;
    case 3203: edm_kernel<32, 3><<<g, 256, 0, st>>>(p, kind, pts, dim, out, v); break;
    case 6403: edm_kernel<64, 3><<<g, 1024, 0, st>>>(p, kind, pts, dim, out, v); break;
    case 1600: edm_kernel<16, 0><<<g, 64, 0, st>>>(p, kind, pts, dim, out, v); break;
    case 3200: edm_kernel<32, 0><<<g, 256, 0, st>>>(p, kind, pts, dim, out, v); break;
    case 6400: edm_kernel<64, 0><<<g, 1024, 0, st>>>(p, kind, pts, dim, out, v); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sx
