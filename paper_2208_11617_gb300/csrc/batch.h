// batch.h -- device-resident description of a batch of automaton instances
// (host and device).  The batched engine keeps, in one arena of device memory:
//   BatchInst[count]        each instance's map, rule and grid offsets
//   BatchItem[nitems]       the work items (runs of blocks of one instance)
//   CUtensorMap[2 * count]  TMA maps of each instance's two grids
//   queue[2 (kBatchMaxSteps+1)] work-queue counters, one per pass of a run
//                           and launch (32^3 tiles of m = 3 run in a second
//                           launch per step)
//   grids                   two side^m uint8 grids per instance
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "hmap.cuh"
#include "rule.h"

namespace sx {

// Tile bodies the batched kernel implements (all with 128-thread CTAs).
enum BatchBody : int32_t {
    kBody2x64 = 0,   // m = 2, 64 x 64 tiles
    kBody2x128 = 1,  // m = 2, 128 x 128 tiles
    kBody3x16 = 2,   // m = 3, 16^3 tiles
    kBody3x32 = 3,   // m = 3, 32^3 tiles (a launch of its own: 74 KB stage)
    kBody3plane = 4, // m = 3, plane stream: 32 x 128 bricks streamed along x1 (a launch of its own)
};

constexpr int kBatchThreads = 128;
constexpr int kBatchChunk = 8;         // CUDA blocks of one instance per work item
constexpr int kBatchMaxSteps = 4096;   // steps per simplex_batch_run call

// One work item of the device queue: up to kBatchChunk consecutive CUDA
// blocks v0 .. v0 + cnt - 1 of instance `inst`'s map.  `tag` lets instances
// that are at different steps share one launch: bit 0 flips the grid the
// instance reads, bits 1..12 add to the live-count index of the pass, bits
// 13..18 + 1 = how many passes of a multi-step sequence the item takes part in.
struct BatchItem {
    uint32_t inst, v0, cnt, tag;
};

// Salt of the result digest: sum over live cells x of splitmix32(kDigestSalt ^ lin(x)).
constexpr uint32_t kDigestSalt = 0x00D16E57u;

// One CTA of the batched engine's flat m = 2 launch: block v of instance
// `inst`'s map (H in trapezoid form, decoded on the device).
struct BatchTile {
    uint32_t inst, v;
};

// One plane-stream work unit of a batch: instance `inst`, brick rows
// y0 = yx & 0xffff ..., cells x0 = yx >> 16 ..., output planes b ... e.
struct BatchPlaneUnit {
    uint32_t inst, yx;
    int32_t b, e;
};

struct BatchInst {
    Plan plan;
    Rule rule;
    uint64_t grid[2];  // byte offsets of the two grids in the arena
    int32_t body;      // BatchBody
    int32_t tmap;      // index of the tensor map of grid 0 (grid 1 follows); kBody3plane: of the first
                       // of grid 0's plane maps in the plane-map array (kPlWidths per grid)
};

// One pass of the plane-stream kernel over a batch's plane units (k_ca3p.cu).
struct PlaneBatch {
    const BatchInst *insts;
    const BatchPlaneUnit *units;
    uint32_t nunits;
    int32_t in_parity;           // grid each instance reads; the result goes to the other
    int32_t all_ork;             // every plane-stream instance has an or-k rule (Rule::or_k)
    const CUtensorMap *ptmaps;   // the plane maps of every kBody3plane instance
    uint8_t *arena;              // grid offsets count from here
    unsigned long long *live;    // live[inst * live_stride + live_index] += live cells written
    int32_t live_stride, live_index;
};

}  // namespace sx
