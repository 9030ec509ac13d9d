// tmap.cpp -- TMA tensor maps of the automaton grids (cuTensorMapEncodeTiled
// through the runtime's driver entry point): the box and the L2 fill size the
// kernels' staged loads depend on.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/simplex.h"
#include "hmap.cuh"
#include "host.h"
#include "kernels.h"

namespace sxh {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// Tensor map over a uint8 grid: extent n + 1 along every axis (cells past the
// domain's bounding box read as zero), row pitch `side`, box of the tile plus
// its halo: (rho + 32) x (rho + 2) [x box_planes], or for the m = 3 x-stream
// form one x-column of a slab: rho x (rho + 2) x box_planes.  L2 fills are promoted to 64
// bytes for m = 2 and 128 bytes for m = 3: wider fills fetched bytes of rows
// that no box in flight reads (the 128 x 128 step was 4 % slower and noisier
// at 256 bytes, the 32^3 step 9 % slower).
int make_tensor_map(const sx::Plan &p, const void *base, CUtensorMap *tm, int box_planes)
{
    auto fn = encode_fn();
    if (!fn) return fail(SIMPLEX_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (p.m == 3 && (box_planes < 3 || box_planes > p.rho + 2))
        return fail(SIMPLEX_EINVAL, "m = 3 box depth %d outside 3 ... rho + 2", box_planes);
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3], estr[3] = {1, 1, 1};
    for (int i = 0; i < p.m; ++i) dims[i] = (cuuint64_t)(p.n + 1);
    strides[0] = (cuuint64_t)p.side;
    if (p.m == 3) strides[1] = (cuuint64_t)(p.side * p.side);
    // the m = 3 x-stream form stages x-columns of the tile's own width
    const bool xcols = p.m == 3 && p.persistent == 1;
    box[0] = (cuuint32_t)(xcols ? p.rho : p.rho + 32);
    box[1] = (cuuint32_t)(p.rho + 2);
    box[2] = (cuuint32_t)box_planes;
    const CUtensorMapSwizzle swz = (p.m == 3 && !xcols && sx::ca3_swizzled(p.rho)) ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                                  : CU_TENSOR_MAP_SWIZZLE_NONE;
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, (cuuint32_t)p.m, const_cast<void *>(base), dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                    p.m == 3 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B : CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SIMPLEX_ECUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return SIMPLEX_OK;
}

// The tensor maps of the m = 3 plane-stream form: extent n + 1 along every
// axis, one box of 34 rows x one plane per width of plane_box_widths, no
// swizzle (the consumers read rows at the box's own pitch).  No L2 fill
// promotion: a box narrowed to the domain's reach on a diagonal brick would
// otherwise fetch whole 128-byte lines past it (DRAM reads 1.37x the cells
// with 128-byte fills against 1.10x expected from 32-byte sectors).
int make_plane_maps(const sx::Plan &p, const void *base, sx::PlaneMaps *maps)
{
    auto fn = encode_fn();
    if (!fn) return fail(SIMPLEX_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (p.m != 3) return fail(SIMPLEX_EINVAL, "the plane-stream form is an m = 3 step");
    int widths[sx::kPlWidths];
    sx::plane_box_widths(widths);
    cuuint64_t dims[3] = {(cuuint64_t)(p.n + 1), (cuuint64_t)(p.n + 1), (cuuint64_t)(p.n + 1)};
    cuuint64_t strides[2] = {(cuuint64_t)p.side, (cuuint64_t)(p.side * p.side)};
    cuuint32_t estr[3] = {1, 1, 1};
    for (int i = 0; i < sx::kPlWidths; ++i) {
        cuuint32_t box[3] = {(cuuint32_t)widths[i], (cuuint32_t)(sx::kPlaneTY + 2), (cuuint32_t)sx::kPlPlanes};
        CUresult r = fn(&maps->m[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return fail(SIMPLEX_ECUDA, "cuTensorMapEncodeTiled failed for box width %d (CUresult %d)", widths[i], (int)r);
    }
    return SIMPLEX_OK;
}

}  // namespace sxh
