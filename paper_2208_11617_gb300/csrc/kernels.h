// kernels.h -- host-side launchers of the CUDA kernels (one per .cu file).
// Each returns a cudaError_t from the launch; arguments are validated by the
// C ABI layer before they get here.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "batch.h"
#include "hmap.cuh"
#include "rule.h"

namespace sx {

cudaError_t launch_write(const Plan &p, uint32_t *out, uint32_t seed, int kind, bool vec, cudaStream_t st);
cudaError_t launch_accum(const Plan &p, uint32_t *data, uint32_t add, int kind, bool vec, cudaStream_t st);

cudaError_t launch_visit(const Plan &p, uint32_t *counts, int level, int kind, cudaStream_t st);

cudaError_t launch_ca_init(const Plan &p, uint8_t *grid, uint32_t seed, uint32_t threshold,
                           unsigned long long *live, cudaStream_t st);

// Live cells of a grid added to *live (if given); with `digest`, the sum over
// live cells x of splitmix32(kDigestSalt ^ lin(x)) is added to *digest.
cudaError_t launch_ca_count(const Plan &p, const uint8_t *grid, unsigned long long *live, cudaStream_t st,
                            unsigned long long *digest = nullptr);

// TMA-staged automaton steps; `tin` maps the input grid (see make_tensor_map).
bool ca2_supports(int rho);
bool ca3_supports(int rho);
bool ca3_swizzled(int rho);  // tensor map needs CU_TENSOR_MAP_SWIZZLE_64B
// m = 3 x-stream form: every 32^3 tile is processed as kStreamZSplit slabs
// along x1, and its x-columns are staged as boxes of 32 x 34 x
// kStreamColPlanes bytes (one slab plus its two halo planes).
constexpr int kStreamZSplit = 2;
constexpr int kStreamColPlanes = 32 / kStreamZSplit + 2;
// Depth along x1 of the box the single-instance m = 3 step stages: the
// x-stream column of a slab, or the whole tile plus halo (grid form).
int ca3_box_planes(const Plan &p);
cudaError_t launch_ca2_step(const Plan &p, const CUtensorMap &tin, uint8_t *out, const Rule &rule,
                            int kind, unsigned long long *live, cudaStream_t st);
// queue: two zeroed 64-bit counters (work counter, CTAs done) that the x-stream
// form (p.persistent) uses and leaves zeroed; unused by the grid form.
cudaError_t launch_ca3_step(const Plan &p, const CUtensorMap &tin, uint8_t *out, const Rule &rule,
                            int kind, unsigned long long *live, unsigned long long *queue, cudaStream_t st);

// m = 3 plane-stream form (launch 3, k_ca3p.cu): bricks of kPlaneTY x
// kPlaneTX cells streamed along x1.  Each stage is one TMA box of kPlPlanes
// planes of 34 rows by one of kPlWidths widths (plane_box_widths: 48 ... 160
// bytes);
// maps.m[i] maps the input grid with box width i.  queue: two zeroed 64-bit
// counters, left zeroed.  segs: sched's segment tables in device memory
// (kPlaneSegWords words: seg_b, then seg_u).
constexpr int kPlWidths = 5;
constexpr int kPlPlanes = 2;  // planes x1 per TMA box (the box's depth)
struct PlaneMaps {
    CUtensorMap m[kPlWidths];
};
int plane_box_widths(int *w);  // fills kPlWidths widths in bytes, returns kPlWidths
cudaError_t launch_ca3_planes(const PlaneSched &sched, const int32_t *segs, const PlaneMaps &maps, int64_t n,
                              int64_t side, uint8_t *out, const Rule &rule, unsigned long long *live,
                              unsigned long long *queue, cudaStream_t st);
cudaError_t ca3_planes_prepare();
cudaError_t ca3p_read_status(uint32_t *out);
// One step of every plane-stream instance of a batch (kBody3plane units).
cudaError_t launch_batch_planes(const PlaneBatch &bt, unsigned long long *queue, cudaStream_t st);

// Sets the kernels' shared-memory limits for the current device (before any
// stream capture).
cudaError_t ca2_prepare(int rho);
cudaError_t ca3_prepare(int rho);

// Diagnostics of Table 1: MAP (rho^m threads per block, one per cell; with
// `cells`, the simplex cells of every block are added to *cells) and EDM on
// the 2-simplex (fp32 distances of points (x1, n - x2), dim <= 16).
cudaError_t launch_map_test(const Plan &p, int kind, unsigned long long *cells, cudaStream_t st);
bool edm_supports(int rho);
cudaError_t launch_edm(const Plan &p, const float *pts, int dim, float *out, int kind, bool vec, cudaStream_t st);

// One CTA whose mbarrier wait runs out after limit_ns (tests the bounded-wait path).
cudaError_t launch_wait_selftest(uint64_t limit_ns, cudaStream_t st);

// Batched engine: one persistent pass (count_only: live counts of the input
// grids, plus a result digest when `digest` is given; else one automaton step
// in -> out) over every work item.  `set` 1 runs the items of 32^3 tiles of
// m = 3 (kBody3x32), set 0 every other body; a count pass runs any item in set
// 0.  `pass` p > 0 is step p of a sequence launched over the same items: an
// item takes part while p < its pass count (tag bits 13..18, plus 1), reading
// grid parity ^ p and counting at its live index + p.
cudaError_t batch_prepare();
cudaError_t launch_batch_pass(const BatchInst *insts, const BatchItem *items, uint32_t nitems,
                              const CUtensorMap *tmaps, uint8_t *arena, int in_parity, unsigned int *queue,
                              unsigned long long *live, int live_stride, int live_index, bool count_only,
                              cudaStream_t st, unsigned long long *digest = nullptr, int set = 0, int pass = 0);
// The flat m = 2 pass of a bound batch: one CTA per tiles[] entry.
cudaError_t launch_batch_flat2(const BatchInst *insts, const BatchTile *tiles, uint32_t ntiles,
                               const CUtensorMap *tmaps, uint8_t *arena, int in_parity, unsigned long long *live,
                               int live_stride, int live_index, cudaStream_t st);
cudaError_t batch_read_status(uint32_t *out);
// CTAs of the batched kernel's launch set resident at once on the current device (SMs x occupancy).
cudaError_t batch_resident_ctas(uint64_t *out, int set = 0);

// Device error words of the TMA kernels (bounded waits that gave up).
// Reads and clears; synchronous.
cudaError_t ca2_read_status(uint32_t *out);
cudaError_t ca3_read_status(uint32_t *out);

}  // namespace sx
