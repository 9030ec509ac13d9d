// batch.cpp -- C ABI of the batched engine (include/simplex.h): planning of
// every instance, arena layout, descriptor upload, graph capture of runs.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/simplex.h"
#include "batch.h"
#include "host.h"
#include "kernels.h"

using namespace sxh;

namespace {

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint64_t binom(uint64_t n, int k)
{
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return (uint64_t)r;
}

struct RunGraph {
    int steps;
    unsigned long long *live;
    int parity;
    cudaGraphExec_t exec;
};

}  // namespace

struct simplex_batch {
    std::vector<simplex_instance_t> spec;
    std::vector<sx::BatchInst> insts;
    // items of set 0 (m = 3 16^3 tiles, then m = 2 tiles), set 1, count passes only
    std::vector<sx::BatchItem> items;
    size_t nitems0_step = 0, nitems0 = 0, nitems1 = 0;  // end of set 0's m = 3 items, of set 0's, of set 1's
    // m = 2 instances: their blocks holding cells, for the flat pass of a bound batch
    std::vector<sx::BatchTile> tiles2;
    uint64_t off_tiles2 = 0;
    // plane-stream instances (kBody3plane): their work units, in instance order
    std::vector<sx::BatchPlaneUnit> punits;
    size_t nplane = 0;
    uint64_t off_punits = 0, off_ptmaps = 0, off_pqueue = 0;
    std::vector<uint64_t> grid_bytes;
    uint64_t blocks = 0, cells = 0;
    // arena layout (byte offsets)
    uint64_t off_insts = 0, off_items = 0, off_tmaps = 0, off_queue = 0, off_grids = 0, bytes = 0;
    uint8_t *arena = nullptr;
    int device = -1;
    int parity = 0;
    cudaStream_t capture = nullptr;
    // the m = 3 chain's stream and its fork / join events (created on the first run)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    std::vector<RunGraph> graphs;
    uint64_t serial = 0;  // unique per batch created in this process (never reused)
};

namespace {

// Planes per slab of a batched plane-stream instance (8: the m = 3 pass over
// the workload's instances ran 13 % faster than with 16, 32 was slower).
constexpr int32_t kBatchPlaneSlab = 8;

int check_batch(simplex_batch_t b, bool bound)
{
    if (!b) return fail(SIMPLEX_EINVAL, "batch is NULL");
    if (bound && !b->arena) return fail(SIMPLEX_EINVAL, "batch is not bound to an arena (simplex_batch_bind)");
    return SIMPLEX_OK;
}

// The whole run as stream work on `st`.
int enqueue_batch_run(simplex_batch_t b, int steps, unsigned long long *live, int parity, cudaStream_t st)
{
    const sx::BatchInst *insts = reinterpret_cast<const sx::BatchInst *>(b->arena + b->off_insts);
    const sx::BatchItem *items = reinterpret_cast<const sx::BatchItem *>(b->arena + b->off_items);
    const CUtensorMap *tmaps = reinterpret_cast<const CUtensorMap *>(b->arena + b->off_tmaps);
    unsigned int *queue = reinterpret_cast<unsigned int *>(b->arena + b->off_queue);
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned int) * 2 * (size_t)(steps + 1), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(queue)");
    if (live) {
        e = cudaMemsetAsync(live, 0, sizeof(unsigned long long) * b->insts.size() * (size_t)(steps + 1), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(live)");
    }
    sx::PlaneBatch pb = {};
    BatchExtras ex;
    ex.nitems1 = b->nitems1;
    if (!b->punits.empty()) {
        pb.insts = insts;
        pb.units = reinterpret_cast<const sx::BatchPlaneUnit *>(b->arena + b->off_punits);
        pb.nunits = (uint32_t)b->punits.size();
        pb.ptmaps = reinterpret_cast<const CUtensorMap *>(b->arena + b->off_ptmaps);
        pb.arena = b->arena;
        pb.all_ork = 1;
        for (const auto &bi : b->insts)
            if (bi.body == sx::kBody3plane && !bi.rule.or_k) pb.all_ork = 0;
        ex.planes = &pb;
        ex.pqueue = reinterpret_cast<unsigned long long *>(b->arena + b->off_pqueue);
    }
    ex.side = b->side;
    ex.fork = b->fork;
    ex.join = b->join;
    if (!b->tiles2.empty()) {
        ex.nitems0_step = b->nitems0_step;
        ex.tiles = reinterpret_cast<const sx::BatchTile *>(b->arena + b->off_tiles2);
        ex.ntiles = (uint32_t)b->tiles2.size();
    }
    return enqueue_batch_passes(insts, items, b->items.size(), b->nitems0, tmaps, b->arena, queue,
                                queue + steps + 1, steps, live, parity, st, &ex);
}

}  // namespace

namespace sxh {

int enqueue_batch_passes(const sx::BatchInst *insts, const sx::BatchItem *items, size_t nitems, size_t nitems0,
                         const CUtensorMap *tmaps, uint8_t *arena, unsigned int *q0, unsigned int *q1, int steps,
                         unsigned long long *live, int parity, cudaStream_t st, const BatchExtras *ex)
{
    cudaError_t e;
    const BatchExtras none;
    if (!ex) ex = &none;
    const size_t nitems1 = ex->nitems1 == (size_t)-1 ? nitems : ex->nitems1;
    const size_t nstep0 = ex->tiles && ex->nitems0_step != (size_t)-1 ? ex->nitems0_step : nitems0;
    const sx::PlaneBatch *planes = ex->planes;
    if (live) {
        e = sx::launch_batch_pass(insts, items, (uint32_t)nitems, tmaps, arena, parity, q0, live, steps + 1, 0, true,
                                  st);
        if (e != cudaSuccess) return cuda_fail(e, "batch count launch");
    }
    // With m = 2 tiles and m = 3 work both present, the two chains of launches
    // (m = 2: the flat tile pass; m = 3: set 0's 16^3 items, set 1, the plane
    // stream) touch disjoint instances, counters and live slots, so the m = 3
    // chain may run on a second stream beside the m = 2 one: each fills the
    // SMs the other leaves idle (its tail, its latency-bound stretches).
    const bool has_m2 = ex->tiles && ex->ntiles;
    const bool has_m3 = nstep0 || nitems1 > nitems0 || (planes && planes->nunits);
    cudaStream_t s3 = st;
    if (ex->side && ex->fork && ex->join && has_m2 && has_m3) {
        if ((e = cudaEventRecord(ex->fork, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord(fork)");
        if ((e = cudaStreamWaitEvent(ex->side, ex->fork, 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent(fork)");
        s3 = ex->side;
    }
    for (int s = 1; s <= steps; ++s) {
        const int in = (parity + s - 1) & 1;
        if (nstep0) {
            e = sx::launch_batch_pass(insts, items, (uint32_t)nstep0, tmaps, arena, in, q0 + s, live, steps + 1, s,
                                      false, s3, nullptr, 0);
            if (e != cudaSuccess) return cuda_fail(e, "batch step launch");
        }
        if (has_m2) {
            e = sx::launch_batch_flat2(insts, ex->tiles, ex->ntiles, tmaps, arena, in, live, steps + 1, s, st);
            if (e != cudaSuccess) return cuda_fail(e, "batch step launch (m = 2 tiles)");
        }
        if (nitems1 > nitems0) {
            e = sx::launch_batch_pass(insts, items + nitems0, (uint32_t)(nitems1 - nitems0), tmaps, arena, in, q1 + s,
                                      live, steps + 1, s, false, s3, nullptr, 1);
            if (e != cudaSuccess) return cuda_fail(e, "batch step launch (32^3 tiles)");
        }
        if (planes && planes->nunits) {
            sx::PlaneBatch pb = *planes;
            pb.in_parity = in;
            pb.live = live;
            pb.live_stride = steps + 1;
            pb.live_index = s;
            e = sx::launch_batch_planes(pb, ex->pqueue, s3);
            if (e != cudaSuccess) return cuda_fail(e, "batch step launch (plane stream)");
        }
    }
    if (s3 != st) {
        if ((e = cudaEventRecord(ex->join, s3)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord(join)");
        if ((e = cudaStreamWaitEvent(st, ex->join, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent(join)");
    }
    return SIMPLEX_OK;
}

int batch_view(simplex_batch_t b, BatchView *out)
{
    if (!b) return fail(SIMPLEX_EINVAL, "batch is NULL");
    out->insts = b->insts.data();
    out->count = b->insts.size();
    out->items = b->items.data();
    out->nitems = b->items.size();
    out->nitems0 = b->nitems0;
    out->grids_offset = b->off_grids;
    out->grids_bytes = b->bytes - b->off_grids;
    out->serial = b->serial;
    out->has_planes = !b->punits.empty();
    return SIMPLEX_OK;
}

}  // namespace sxh

extern "C" {

int simplex_batch_create(const simplex_instance_t *instances, int count, simplex_batch_t *out)
{
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!instances || count <= 0) return fail(SIMPLEX_EINVAL, "need at least one instance");
    if (count > (1 << 24)) return fail(SIMPLEX_EINVAL, "too many instances (%d)", count);
    simplex_batch *b = new (std::nothrow) simplex_batch();
    if (!b) return fail(SIMPLEX_ENOMEM, "host allocation failed");
    try {
        b->spec.assign(instances, instances + count);
        b->insts.resize(count);
        b->grid_bytes.resize(count);
    } catch (...) {
        delete b;
        return fail(SIMPLEX_ENOMEM, "host allocation failed");
    }
    uint64_t grid_off = 0;
    std::vector<sx::BatchItem> items0m2;  // set 0 items of m = 2 instances, after set 0's m = 3 items
    std::vector<sx::BatchItem> items1;    // items of launch set 1, appended after set 0's
    std::vector<sx::BatchItem> items2;    // count-only items (plane-stream instances), appended last
    for (int i = 0; i < count; ++i) {
        const simplex_instance_t &in = instances[i];
        sx::BatchInst &bi = b->insts[i];
        std::memset(&bi, 0, sizeof bi);
        int body = -1;
        if (in.m == 2 && in.block == 64) body = sx::kBody2x64;
        if (in.m == 2 && in.block == 128) body = sx::kBody2x128;
        if (in.m == 3 && in.block == 16) body = sx::kBody3x16;
        if (in.m == 3 && in.block == 32) body = sx::kBody3x32;
        if (in.m == 3 && in.block == 128) body = sx::kBody3plane;
        if (body < 0) {
            delete b;
            return fail(SIMPLEX_EINVAL, "instance %d: the batched engine runs m = 2 with block 64 or 128 and m = 3 "
                                        "with block 16, 32 or 128 (the plane stream) (got m = %d, block = %d)",
                        i, in.m, in.block);
        }
        // rows start on 128-byte lines: a box row then touches only the
        // 32-byte sectors it reads (with rows 16-byte aligned the m = 2 flat
        // pass ran 3 % slower, the whole batch 4 %)
        const int64_t side = (in.n + 128) / 128 * 128;
        int band = 0;
        if (in.m == 2) {
            band = in.band;
            if (band <= 0) {  // automatic: 8 tile rows, fewer for small domains
                const int64_t nb = (in.n + in.block) / in.block;
                band = 1;
                while (band < 8 && band * 2 <= nb) band *= 2;
            }
        }
        // plane-stream instances keep a 32^3 H3 plan for the count pass (live[0], digests)
        const int rho = body == sx::kBody3plane ? 32 : in.block;
        int rc = build_plan(in.m, in.n, 2, in.beta, rho, side, band, &bi.plan);
        if (rc) {
            std::string msg = g_last_error;
            delete b;
            return fail(rc, "instance %d: %s", i, msg.c_str());
        }
        bi.rule = make_rule(in.m, in.birth, in.survive);
        bi.body = body;
        bi.tmap = 2 * i;
        if (body == sx::kBody3plane) {
            sx::PlaneSched ps;
            if (!sx::plane_sched_build(in.n, sx::kMapH, &ps, kBatchPlaneSlab) || in.n >= 65535) {
                delete b;
                return fail(SIMPLEX_EINVAL, "instance %d: n = %lld is too large for a batched plane stream", i,
                            (long long)in.n);
            }
            bi.tmap = (int32_t)(2 * sx::kPlWidths * b->nplane++);
            try {
                for (uint64_t w = 0; w < ps.units; ++w) {
                    sx::PlaneUnit u;
                    sx::plane_unit_decode(ps, w, u);
                    b->punits.push_back(sx::BatchPlaneUnit{(uint32_t)i, (uint32_t)u.y0 | ((uint32_t)u.x0 << 16), u.b,
                                                           u.e});
                }
            } catch (...) {
                delete b;
                return fail(SIMPLEX_ENOMEM, "host allocation failed");
            }
        }
        uint64_t gb = 1;
        for (int d = 0; d < in.m; ++d) gb *= (uint64_t)side;
        b->grid_bytes[i] = gb;
        bi.grid[0] = grid_off;
        grid_off += align_up(gb, 256);
        bi.grid[1] = grid_off;
        grid_off += align_up(gb, 256);
        b->blocks += bi.plan.h_blocks;
        b->cells += binom((uint64_t)in.n + (uint64_t)in.m, in.m);
        // work items: runs of up to kBatchChunk consecutive blocks whose tiles
        // hold cells (the host evaluates the kernels' own decode; blocks that
        // exit -- packing waste, overhang, tiles past the padded lattice's
        // domain -- get no item, and the kernel still decodes every block)
        auto holds_cells = [&](uint64_t v) {
            int32_t X[sx::kMaxM] = {0, 0, 0, 0};
            bool ok = false;
            switch (bi.plan.m) {
            case 2: ok = sx::decode<2>(bi.plan, sx::kMapH, v, X); break;
            case 3: ok = sx::decode<3>(bi.plan, sx::kMapH, v, X); break;
            default: ok = sx::decode<4>(bi.plan, sx::kMapH, v, X); break;
            }
            int64_t sum = 0;
            for (int d = 0; d < bi.plan.m; ++d) sum += X[d];
            return ok && sum * bi.plan.rho <= bi.plan.n;
        };
        // plane-stream instances: block items for the count pass only
        std::vector<sx::BatchItem> &dst = body == sx::kBody3x32     ? items1
                                          : body == sx::kBody3plane ? items2
                                          : in.m == 2               ? items0m2
                                                                    : b->items;
        for (uint64_t v = 0; v < bi.plan.h_blocks;) {
            if (!holds_cells(v)) {
                ++v;
                continue;
            }
            const uint64_t v0 = v;
            while (v < bi.plan.h_blocks && v - v0 < (uint64_t)sx::kBatchChunk && holds_cells(v)) ++v;
            dst.push_back(sx::BatchItem{(uint32_t)i, (uint32_t)v0, (uint32_t)(v - v0), 0u});
        }
        if (in.m == 2)
            for (uint64_t v = 0; v < bi.plan.h_blocks; ++v)
                if (holds_cells(v)) b->tiles2.push_back(sx::BatchTile{(uint32_t)i, (uint32_t)v});
    }
    // plane units longest first (the queue's last units are the short ones);
    // equal lengths keep instance and slab order
    std::stable_sort(b->punits.begin(), b->punits.end(),
                     [](const sx::BatchPlaneUnit &x, const sx::BatchPlaneUnit &y) { return x.e - x.b > y.e - y.b; });
    b->nitems0_step = b->items.size();
    b->items.insert(b->items.end(), items0m2.begin(), items0m2.end());
    b->nitems0 = b->items.size();
    b->items.insert(b->items.end(), items1.begin(), items1.end());
    b->nitems1 = b->items.size();
    b->items.insert(b->items.end(), items2.begin(), items2.end());
    if (b->items.size() >= 0xffffff00ull) {
        delete b;
        return fail(SIMPLEX_EINVAL, "too many work items (%zu)", b->items.size());
    }
    // arena layout
    uint64_t off = 0;
    b->off_insts = off;
    off = align_up(off + sizeof(sx::BatchInst) * (uint64_t)count, 256);
    b->off_items = off;
    off = align_up(off + sizeof(sx::BatchItem) * b->items.size(), 256);
    b->off_tmaps = off;
    off = align_up(off + sizeof(CUtensorMap) * 2ull * (uint64_t)count, 256);
    b->off_queue = off;
    off = align_up(off + sizeof(unsigned int) * 2ull * (uint64_t)(sx::kBatchMaxSteps + 1), 256);
    b->off_tiles2 = off;
    off = align_up(off + sizeof(sx::BatchTile) * b->tiles2.size(), 256);
    b->off_punits = off;
    off = align_up(off + sizeof(sx::BatchPlaneUnit) * b->punits.size(), 256);
    b->off_ptmaps = off;
    off = align_up(off + sizeof(CUtensorMap) * 2ull * sx::kPlWidths * b->nplane, 256);
    b->off_pqueue = off;
    off = align_up(off + 2 * sizeof(unsigned long long), 256);
    b->off_grids = off;
    for (auto &bi : b->insts) {
        bi.grid[0] += off;
        bi.grid[1] += off;
    }
    b->bytes = off + grid_off;
    static std::atomic<uint64_t> next_serial{0};
    b->serial = ++next_serial;
    *out = b;
    return SIMPLEX_OK;
}

int simplex_batch_destroy(simplex_batch_t b)
{
    if (!b) return SIMPLEX_OK;
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    delete b;
    return SIMPLEX_OK;
}

int simplex_batch_info(simplex_batch_t b, simplex_batch_info_t *out)
{
    int rc;
    if ((rc = check_batch(b, false))) return rc;
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof *out);
    out->count = (int32_t)b->insts.size();
    out->parity = b->parity;
    out->items = b->items.size();
    out->blocks = b->blocks;
    out->cells = b->cells;
    out->arena_bytes = b->bytes;
    out->grids_offset = b->off_grids;
    out->grids_bytes = b->bytes - b->off_grids;
    return SIMPLEX_OK;
}

int simplex_batch_bind(simplex_batch_t b, void *arena, uint64_t arena_bytes, void *stream)
{
    int rc;
    if ((rc = check_batch(b, false))) return rc;
    if (!arena) return fail(SIMPLEX_EINVAL, "arena is NULL");
    if ((reinterpret_cast<uintptr_t>(arena) & 255u) != 0) return fail(SIMPLEX_EINVAL, "arena must be 256-byte aligned");
    if (arena_bytes < b->bytes)
        return fail(SIMPLEX_EINVAL, "arena too small: %llu bytes, need %llu", (unsigned long long)arena_bytes,
                    (unsigned long long)b->bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t *base = static_cast<uint8_t *>(arena);
    std::vector<CUtensorMap> tmaps(2 * b->insts.size());
    for (size_t i = 0; i < b->insts.size(); ++i)
        for (int g = 0; g < 2; ++g) {
            rc = make_tensor_map(b->insts[i].plan, base + b->insts[i].grid[g], &tmaps[2 * i + g],
                                 b->insts[i].plan.rho + 2);
            if (rc) return rc;
        }
    std::vector<sx::PlaneMaps> pmaps(2 * b->nplane);
    for (size_t i = 0; i < b->insts.size(); ++i) {
        if (b->insts[i].body != sx::kBody3plane) continue;
        for (int g = 0; g < 2; ++g) {
            rc = make_plane_maps(b->insts[i].plan, base + b->insts[i].grid[g],
                                 &pmaps[b->insts[i].tmap / sx::kPlWidths + g]);
            if (rc) return rc;
        }
    }
    static_assert(sizeof(sx::PlaneMaps) == sizeof(CUtensorMap) * sx::kPlWidths, "plane maps must be contiguous");
    cudaError_t e;
    if (!b->punits.empty() &&
        ((e = cudaMemcpyAsync(base + b->off_punits, b->punits.data(), sizeof(sx::BatchPlaneUnit) * b->punits.size(),
                              cudaMemcpyHostToDevice, st)) != cudaSuccess ||
         (e = cudaMemcpyAsync(base + b->off_ptmaps, pmaps.data(), sizeof(sx::PlaneMaps) * pmaps.size(),
                              cudaMemcpyHostToDevice, st)) != cudaSuccess))
        return cuda_fail(e, "binding the batch arena (plane stream)");
    if (!b->tiles2.empty() &&
        (e = cudaMemcpyAsync(base + b->off_tiles2, b->tiles2.data(), sizeof(sx::BatchTile) * b->tiles2.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "binding the batch arena (m = 2 tiles)");
    if ((e = cudaMemsetAsync(base + b->off_pqueue, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + b->off_insts, b->insts.data(), sizeof(sx::BatchInst) * b->insts.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + b->off_items, b->items.data(), sizeof(sx::BatchItem) * b->items.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + b->off_tmaps, tmaps.data(), sizeof(CUtensorMap) * tmaps.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + b->off_grids, 0, b->bytes - b->off_grids, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "binding the batch arena");
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
    b->arena = base;
    b->parity = 0;
    return SIMPLEX_OK;
}

int simplex_batch_init(simplex_batch_t b, void *stream)
{
    int rc;
    if ((rc = check_batch(b, true))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (size_t i = 0; i < b->insts.size(); ++i) {
        const simplex_instance_t &in = b->spec[i];
        cudaError_t e = sx::launch_ca_init(b->insts[i].plan, b->arena + b->insts[i].grid[0], in.seed, in.threshold,
                                           nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch init launch");
    }
    b->parity = 0;
    return SIMPLEX_OK;
}

int simplex_batch_run(simplex_batch_t b, int steps, unsigned long long *live, int use_graph, void *stream)
{
    int rc;
    if ((rc = check_batch(b, true))) return rc;
    if (steps < 1 || steps > sx::kBatchMaxSteps)
        return fail(SIMPLEX_EINVAL, "steps must be in [1, %d] (got %d)", sx::kBatchMaxSteps, steps);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = sx::batch_prepare();
    if (e != cudaSuccess) return cuda_fail(e, "setting the batch kernel's shared-memory limit");
    if (!b->side) {
        if ((e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreateWithFlags(side)");
        if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreateWithFlags");
    }
    if (!use_graph) {
        rc = enqueue_batch_run(b, steps, live, b->parity, st);
        if (rc) return rc;
        b->parity = (b->parity + steps) & 1;
        return SIMPLEX_OK;
    }
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (b->device >= 0 && b->device != dev)
        return fail(SIMPLEX_EINVAL, "batch was first run with graphs on device %d, now %d", b->device, dev);
    if (!b->capture) {
        if ((e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        b->device = dev;
    }
    cudaGraphExec_t exec = nullptr;
    for (auto &g : b->graphs)
        if (g.steps == steps && g.live == live && g.parity == b->parity) exec = g.exec;
    if (!exec) {
        if ((e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamBeginCapture");
        rc = enqueue_batch_run(b, steps, live, b->parity, b->capture);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        if (b->graphs.size() >= 8) {
            cudaGraphExecDestroy(b->graphs.front().exec);
            b->graphs.erase(b->graphs.begin());
        }
        b->graphs.push_back(RunGraph{steps, live, b->parity, exec});
    }
    if ((e = cudaGraphLaunch(exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    b->parity = (b->parity + steps) & 1;
    return SIMPLEX_OK;
}

int simplex_batch_grid(simplex_batch_t b, int i, uint8_t **grid, int64_t *side)
{
    int rc;
    if ((rc = check_batch(b, true))) return rc;
    if (i < 0 || i >= (int)b->insts.size()) return fail(SIMPLEX_EINVAL, "instance index %d out of range", i);
    if (!grid || !side) return fail(SIMPLEX_EINVAL, "grid and side must not be NULL");
    *grid = b->arena + b->insts[i].grid[b->parity];
    *side = b->insts[i].plan.side;
    return SIMPLEX_OK;
}

}  // extern "C"
