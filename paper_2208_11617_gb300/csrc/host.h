// host.h -- host-side helpers shared by the C ABI translation units
// (api.cpp, batch.cpp): error reporting, planning, rules and tensor maps.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "batch.h"
#include "hmap.cuh"
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
int make_tensor_map(const sx::Plan &p, const void *base, CUtensorMap *tm);

// Read-only view of a batch's host-side plans and work items; grid offsets in
// the BatchInst records count from the start of the arena, and the grids
// occupy [grids_offset, grids_offset + grids_bytes).
struct BatchView {
    const sx::BatchInst *insts;
    size_t count;
    const sx::BatchItem *items;
    size_t nitems;
    uint64_t grids_offset, grids_bytes;
};
int batch_view(struct simplex_batch *b, BatchView *out);

}  // namespace sxh
