// host.h -- host-side helpers shared by the C ABI translation units
// (api.cpp, batch.cpp): error reporting, planning, rules and tensor maps.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "batch.h"
#include "hmap.cuh"
#include "kernels.h"
#include "rule.h"

namespace sxh {

extern thread_local std::string g_last_error;

// Records a message for simplex_last_error() and returns `code`.
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// Validates the arguments and fills the launch plan (host memory only).
int build_plan(int m, int64_t n, int r_inv, int beta, int block, int64_t side, int band, sx::Plan *p,
               int layout = 0);

// The byte-sliced rule tables for birth/survive masks of an m-dimensional automaton.
sx::Rule make_rule(int m, uint32_t birth, uint32_t survive);

// TMA tensor map over a uint8 grid of the plan's layout (extent n + 1 per
// axis, pitch side), box = tile + halo; SIMPLEX_OK or an error code.
// box_planes: depth along x1 of an m = 3 box (ignored for m = 2).
int make_tensor_map(const sx::Plan &p, const void *base, CUtensorMap *tm, int box_planes);

// The tensor maps of the m = 3 plane-stream step (one per box width).
int make_plane_maps(const sx::Plan &p, const void *base, sx::PlaneMaps *maps);

// Read-only view of a batch's host-side plans and work items; grid offsets in
// the BatchInst records count from the start of the arena, and the grids
// occupy [grids_offset, grids_offset + grids_bytes).
struct BatchView {
    const sx::BatchInst *insts;
    size_t count;
    const sx::BatchItem *items;
    size_t nitems;
    size_t nitems0;  // items of launch set 0 come first, then those of set 1 (32^3 tiles of m = 3)
    uint64_t grids_offset, grids_bytes;
    uint64_t serial;  // unique per batch of this process: equal serials mean equal plans and items
    bool has_planes;  // the batch holds plane-stream instances (kBody3plane)
};

// The step passes of a run: per step, launch set 0 over items [0, nitems0)
// with queue counter q0[s] and set 1 over the rest with q1[s]; a count pass
// over every item first (queue q0[0]) when `live` is given.  The counters
// must be zero.
// Optional parts of a bound batch's passes.  Items of set 1 end at nitems1
// (the rest, up to nitems, take part in count passes only).  With `tiles`,
// set 0's step passes run items [0, nitems0_step) and the m = 2 items after
// them run as one flat pass over `tiles` instead.  With `planes`, every step
// also runs one plane-stream pass (work counters `pqueue`, zero and left zero).
struct BatchExtras {
    size_t nitems1 = (size_t)-1;
    size_t nitems0_step = (size_t)-1;
    const sx::BatchTile *tiles = nullptr;
    uint32_t ntiles = 0;
    const sx::PlaneBatch *planes = nullptr;
    unsigned long long *pqueue = nullptr;
    // a second stream and two events: when set and the batch holds both m = 2
    // tiles and m = 3 work, the m = 3 launches of every step run on `side`,
    // forked from and joined back to the main stream, beside the m = 2 ones
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
int enqueue_batch_passes(const sx::BatchInst *insts, const sx::BatchItem *items, size_t nitems, size_t nitems0,
                         const CUtensorMap *tmaps, uint8_t *arena, unsigned int *q0, unsigned int *q1, int steps,
                         unsigned long long *live, int parity, cudaStream_t st, const BatchExtras *ex = nullptr);
int batch_view(struct simplex_batch *b, BatchView *out);

}  // namespace sxh
