// server.cpp -- continuous-batching server for automaton jobs (C ABI in
// include/simplex.h).
//
// Jobs (an m-simplex automaton of size n run for a number of steps) arrive
// over time.  The server keeps every admitted job's two grids resident in a
// device arena whose grid pool is capped by an HBM budget, and works in
// rounds: each round is round_steps launches of the batched persistent
// kernel, launch k advancing every resident job that still has steps left by
// one step, whatever step each job is at (per-item tags select each job's
// input grid and live-count slot).  Several steps per round keep the
// per-round costs (item upload, digest pass, result copies, event) off most
// steps, so a job's latency approaches its run time alone.  With at most
// direct_jobs jobs resident the server works in direct chunks instead: each
// job's next steps go out as single-instance step launches on its own grids
// and tensor maps, on a side stream of its own, so light jobs run
// concurrently and a new arrival does not queue behind another job's chunk
// (a persistent batched pass costs more than a few jobs' own launches).  Between
// rounds the host loop admits jobs that have arrived (first come, first
// served) as soon as a slot and enough pool memory are free, and retires jobs
// whose last step has completed (their results -- live counts of every step
// and a digest of the final grid -- are copied to host memory and their
// memory returns to the pool).  Completion times are device times (CUDA
// events), arrival times come from the trace.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <thread>
#include <vector>

#include "../../include/simplex.h"
#include "batch.h"
#include "host.h"
#include "kernels.h"
#include "pool.h"

using namespace sxh;

namespace {

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint64_t binom(uint64_t n, int k)
{
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return (uint64_t)r;
}

enum JobStatus : int32_t { kPending = 0, kActive = 1, kDone = 2, kRejected = 3 };

struct ServerJob {
    simplex_job_t spec;
    double arrival_ms = 0, admit_ms = 0, done_ms = 0;
    double seen_ms = 0;  // host time at which the serving loop found the job complete
    int32_t status = kPending;
    int slot = -1;
    uint64_t off = 0, bytes = 0;
    int step = 0, parity = 0;
    uint64_t digest = 0;
    std::vector<uint64_t> live;
    uint64_t cells = 0;
    uint64_t items = 0;  // work items per round
    bool busy = false;   // a direct chunk of its steps is in flight on a side stream
};

struct Round {
    cudaEvent_t ev0 = nullptr, ev = nullptr;  // before its first operation, after its last
    std::vector<int64_t> finishing;
};

// A direct chunk: the next steps of one job (and, when they are its last,
// its digest and result copies) on a side stream of its own.
struct Chunk {
    int64_t job = -1;
    cudaEvent_t ev0 = nullptr, ev = nullptr;
    bool finishing = false;
};

// Side streams of the direct chunks: job slot s uses side[s % kSideStreams],
// so the chunks of different light jobs run concurrently.
constexpr int kSideStreams = 8;

// Tile side of a job's plan for the batched passes (the sides the batched
// kernel's bodies cover).
int tile_for(int m, int64_t n) { return m == 2 ? (n >= 1024 ? 128 : 64) : 16; }

// Tile side of a job's direct chunks (single-instance step launches), from
// per-step times of 64 such launches on GB300: m = 2 runs fastest on 64 x 64
// tiles up to n ~ 2500 (n = 1500: 3.0 us a step, 3.7 us on 128 x 128) and on
// 128 x 128 beyond; m = 3 on 16^3 tiles up to n ~ 350 and on 32^3 beyond
// (n = 511: 18.6 us a step, 22.8 us on 16^3).  Both plans address the same
// grids: a job may take batched passes and direct chunks in any order.
int direct_tile_for(int m, int64_t n) { return m == 2 ? (n >= 2560 ? 128 : 64) : (n >= 352 ? 32 : 16); }

// Trapezoid band height of an m = 2 plan: 8 tiles, fewer when the triangle
// is smaller than two bands; 0 (no bands) for m = 3.
int band_for(int m, int64_t n, int block)
{
    if (m != 2) return 0;
    const int64_t nb = (n + block) / block;
    int band = 1;
    while (band < 8 && band * 2 <= nb) band *= 2;
    return band;
}

// Work-queue counters: round r uses group r % (max_inflight + 1) of
// round_steps + 1 counters (its step passes, then its digest pass), zeroed by
// a memset at the start of the round: the groups of the rounds still in
// flight are not touched.
constexpr int kDefaultRoundSteps = 16;
constexpr int kMaxRoundSteps = 64;

int round_steps(const simplex_server_params_t &p) { return p.round_steps ? p.round_steps : kDefaultRoundSteps; }

constexpr int kDefaultDirectJobs = 24, kMaxDirectJobs = 64;
int direct_jobs(const simplex_server_params_t &p) { return p.direct_jobs ? p.direct_jobs : kDefaultDirectJobs; }

}  // namespace

struct simplex_server {
    simplex_server_params_t prm;
    uint8_t *arena = nullptr;
    uint64_t off_insts = 0, off_tmaps = 0, off_items = 0, off_queue = 0, off_live = 0, off_digest = 0,
             off_pool = 0, bytes = 0;
    uint64_t max_items = 0;
    FreeList pool;
    std::vector<int> free_slots;
    std::vector<sx::BatchInst> slot_inst;        // host copies uploaded at admission
    std::vector<CUtensorMap> slot_tmap;          // 2 per slot
    std::vector<sx::Plan> slot_dplan;            // plan of the direct chunks (direct_tile_for)
    std::vector<CUtensorMap> slot_dtmap;         // its tensor maps, 2 per slot
    std::vector<ServerJob> jobs;
    std::deque<int64_t> pending;
    std::vector<int64_t> active;
    uint64_t active_items = 0;                   // blocks of one round over the active jobs
    uint64_t ctas = 1216;                        // resident CTAs of a batched launch
    std::deque<Round> inflight;
    std::vector<cudaEvent_t> spare_events;
    std::vector<sx::BatchItem> items, fin_items;
    sx::BatchItem *stage = nullptr;              // pinned ring: (max_inflight + 1) x 2 x max_items
    uint64_t round_no = 0;                       // selects the work-queue counters of a round
    double host_round_ms = 0;                    // host time spent issuing rounds
    unsigned long long *host_live = nullptr;     // pinned [max_jobs][max_steps + 1]
    unsigned long long *host_digest = nullptr;   // pinned [max_jobs]
    cudaEvent_t t0 = nullptr;
    std::chrono::steady_clock::time_point h0;
    // stats
    uint64_t rounds = 0, cell_updates = 0, active_sum = 0;
    double wall_ms = 0;
    double gpu_round_ms = 0;                     // device time of the retired rounds
    uint64_t launches = 0;                       // kernels launched (init, steps, passes, digests)
    std::vector<Chunk> chunks;                   // direct chunks in flight
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t main_ev = nullptr;               // orders a chunk after the main stream's work
    // the stream of the current trace or online session; online calls need
    // simplex_server_begin first
    cudaStream_t stream = nullptr;
    bool stream_set = false;
};

namespace {

uint64_t layout(const simplex_server_params_t &p, simplex_server *s)
{
    const uint64_t slots = (uint64_t)p.max_jobs;
    uint64_t off = 0;
    const uint64_t max_items = (uint64_t)p.max_items;
    if (s) s->off_insts = off;
    off = align_up(off + sizeof(sx::BatchInst) * slots, 256);
    if (s) s->off_tmaps = off;
    off = align_up(off + sizeof(CUtensorMap) * 2 * slots, 256);
    if (s) s->off_items = off;
    const uint64_t K = (uint64_t)round_steps(p);
    off = align_up(off + sizeof(sx::BatchItem) * max_items * 2, 256);  // round items + finishing items
    if (s) s->off_queue = off;
    off = align_up(off + sizeof(unsigned int) * (K + 1) * (uint64_t)(p.max_inflight + 1), 256);
    if (s) s->off_live = off;
    off = align_up(off + sizeof(unsigned long long) * slots * (uint64_t)(p.max_steps + 1), 256);
    if (s) s->off_digest = off;
    off = align_up(off + sizeof(unsigned long long) * slots, 256);
    if (s) {
        s->off_pool = off;
        s->max_items = max_items;
    }
    return off + p.hbm_budget;
}

int check_params(const simplex_server_params_t *p)
{
    if (!p) return fail(SIMPLEX_EINVAL, "params is NULL");
    if (p->hbm_budget < (1ull << 20)) return fail(SIMPLEX_EINVAL, "hbm_budget must be at least 1 MiB");
    if (p->max_jobs < 1 || p->max_jobs > (1 << 20)) return fail(SIMPLEX_EINVAL, "max_jobs must be in [1, 2^20]");
    if (p->max_steps < 1 || p->max_steps > 4095) return fail(SIMPLEX_EINVAL, "max_steps must be in [1, 4095]");
    if (p->max_items < 1024 || p->max_items > (1 << 26)) return fail(SIMPLEX_EINVAL, "max_items must be in [1024, 2^26]");
    if (p->max_inflight < 1 || p->max_inflight > 64) return fail(SIMPLEX_EINVAL, "max_inflight must be in [1, 64]");
    if (p->round_steps < 0 || p->round_steps > kMaxRoundSteps)
        return fail(SIMPLEX_EINVAL, "round_steps must be in [0, %d]", kMaxRoundSteps);
    if (p->direct_jobs < -1 || p->direct_jobs > kMaxDirectJobs)
        return fail(SIMPLEX_EINVAL, "direct_jobs must be in [-1, %d]", kMaxDirectJobs);
    return SIMPLEX_OK;
}

double host_ms(simplex_server *s)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s->h0).count();
}

// Tries to admit job j: a slot, pool memory for both grids, plan, tensor maps,
// zeroed grids, initial state.  Returns 1 admitted, 0 must wait, <0 error.
int admit(simplex_server *s, int64_t j, cudaStream_t st)
{
    ServerJob &job = s->jobs[j];
    const simplex_job_t &sp = job.spec;
    if (s->free_slots.empty()) return 0;
    const int block = tile_for(sp.m, sp.n);
    const int64_t side = (sp.n + 16) / 16 * 16;
    uint64_t gb = 1;
    for (int d = 0; d < sp.m; ++d) gb *= (uint64_t)side;
    const uint64_t bytes = 2 * align_up(gb, 256);
    if (bytes > s->prm.hbm_budget) return -2;  // can never fit
    // work items per round: plan first (host only), then check the round budget
    sx::Plan plan, dplan;
    const int dblock = direct_tile_for(sp.m, sp.n);
    if (build_plan(sp.m, sp.n, 2, 2, block, side, band_for(sp.m, sp.n, block), &plan)) return -1;
    if (dblock == block) dplan = plan;
    else if (build_plan(sp.m, sp.n, 2, 2, dblock, side, band_for(sp.m, sp.n, dblock), &dplan)) return -1;
    const uint64_t nitems = plan.h_blocks;  // work items at the finest chunk (one block each)
    if (nitems > s->max_items) return -2;                   // can never fit in a round
    if (s->active_items + nitems > s->max_items) return 0;  // wait for the round to shrink
    uint64_t off = 0;
    if (!s->pool.alloc(bytes, &off)) return 0;
    const int slot = s->free_slots.back();
    s->free_slots.pop_back();
    sx::BatchInst &bi = s->slot_inst[slot];
    std::memset(&bi, 0, sizeof bi);
    bi.plan = plan;
    int rc;
    bi.rule = make_rule(sp.m, sp.birth, sp.survive);
    bi.body = sp.m == 2 ? (block == 64 ? sx::kBody2x64 : sx::kBody2x128) : sx::kBody3x16;
    bi.tmap = 2 * slot;
    bi.grid[0] = s->off_pool + off;
    bi.grid[1] = s->off_pool + off + align_up(gb, 256);
    s->slot_dplan[slot] = dplan;
    for (int g = 0; g < 2; ++g) {
        rc = make_tensor_map(bi.plan, s->arena + bi.grid[g], &s->slot_tmap[2 * slot + g], bi.plan.rho + 2);
        if (rc == SIMPLEX_OK)
            rc = make_tensor_map(dplan, s->arena + bi.grid[g], &s->slot_dtmap[2 * slot + g], dplan.rho + 2);
        if (rc) {
            // the slot and pool memory go back: the job is not admitted
            s->free_slots.push_back(slot);
            s->pool.release(off, bytes);
            return -1;
        }
    }
    cudaError_t e;
    unsigned long long *live = reinterpret_cast<unsigned long long *>(s->arena + s->off_live) +
                               (uint64_t)slot * (uint64_t)(s->prm.max_steps + 1);
    unsigned long long *dig = reinterpret_cast<unsigned long long *>(s->arena + s->off_digest) + slot;
    if ((e = cudaMemcpyAsync(s->arena + s->off_insts + sizeof(sx::BatchInst) * slot, &bi, sizeof bi,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s->arena + s->off_tmaps + sizeof(CUtensorMap) * 2 * slot, &s->slot_tmap[2 * slot],
                             sizeof(CUtensorMap) * 2, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(s->arena + bi.grid[0], 0, bytes, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(live, 0, sizeof(unsigned long long) * (size_t)(s->prm.max_steps + 1), st)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(dig, 0, sizeof(unsigned long long), st)) != cudaSuccess ||
        (e = sx::launch_ca_init(bi.plan, s->arena + bi.grid[0], sp.seed, sp.threshold, live, st)) != cudaSuccess) {
        cuda_fail(e, "admitting a job");
        return -1;
    }
    s->launches += 1;
    job.status = kActive;
    job.slot = slot;
    job.off = off;
    job.bytes = bytes;
    job.step = 0;
    job.parity = 0;
    job.admit_ms = host_ms(s);
    job.items = nitems;
    s->active_items += nitems;
    s->active.push_back(j);
    return 1;
}

// One round: advance every active job by one step; jobs reaching their step
// count get a digest pass and their results queued for copy to the host.
int launch_round_impl(simplex_server *s, cudaStream_t st);

// An event from the pool (created when the pool is empty).
cudaError_t take_event(simplex_server *s, cudaEvent_t *ev)
{
    if (s->spare_events.empty()) {
        cudaEvent_t e0;
        const cudaError_t e = cudaEventCreate(&e0);
        if (e != cudaSuccess) return e;
        s->spare_events.push_back(e0);
    }
    *ev = s->spare_events.back();
    s->spare_events.pop_back();
    return cudaSuccess;
}

// Launches a direct chunk for active job j on its side stream: its next
// min(r, 4 K) steps as single-instance step launches (the same kernels and
// results as simplex_ca_step), and after its last step the digest of the
// final grid and the copies of its results.  The side stream first waits for
// everything already queued on the main stream (the job's admission, and the
// batched rounds it took part in).
int launch_chunk(simplex_server *s, int64_t j, cudaStream_t st)
{
    ServerJob &job = s->jobs[j];
    const sx::BatchInst &bi = s->slot_inst[job.slot];
    const sx::Plan &dp = s->slot_dplan[job.slot];
    cudaStream_t cs = s->side[job.slot % kSideStreams];
    const int np = std::min(std::min(kMaxRoundSteps, 4 * round_steps(s->prm)), job.spec.steps - job.step);
    unsigned long long *live_row =
        reinterpret_cast<unsigned long long *>(s->arena + s->off_live) + (size_t)job.slot * (size_t)(s->prm.max_steps + 1);
    unsigned long long *dig = reinterpret_cast<unsigned long long *>(s->arena + s->off_digest) + job.slot;
    Chunk c;
    c.job = j;
    cudaError_t e;
    if ((e = cudaEventRecord(s->main_ev, st)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, s->main_ev, 0)) != cudaSuccess ||
        (e = take_event(s, &c.ev0)) != cudaSuccess || (e = cudaEventRecord(c.ev0, cs)) != cudaSuccess)
        return cuda_fail(e, "starting a direct chunk");
    // step k reads grid parity ^ k and counts at step index + k, as a batched pass does
    for (int k = 0; k < np; ++k) {
        const int par = job.parity ^ (k & 1);
        uint8_t *out = s->arena + bi.grid[par ^ 1];
        const CUtensorMap &tm = s->slot_dtmap[2 * job.slot + par];
        e = dp.m == 2 ? sx::launch_ca2_step(dp, tm, out, bi.rule, sx::kMapH, live_row + job.step + 1 + k, cs)
                      : sx::launch_ca3_step(dp, tm, out, bi.rule, sx::kMapH, live_row + job.step + 1 + k, nullptr, cs);
        if (e != cudaSuccess) return cuda_fail(e, "launching a job's step");
        s->launches += 1;
    }
    job.step += np;
    job.parity ^= np & 1;
    s->cell_updates += job.cells * (uint64_t)np;
    c.finishing = job.step == job.spec.steps;
    if (c.finishing) {
        const size_t row = (size_t)(s->prm.max_steps + 1);
        if ((e = sx::launch_ca_count(bi.plan, s->arena + bi.grid[job.parity], nullptr, cs, dig)) != cudaSuccess)
            return cuda_fail(e, "launching a job's digest");
        s->launches += 1;
        if ((e = cudaMemcpyAsync(s->host_live + job.slot * row, live_row,
                                 sizeof(unsigned long long) * (size_t)(job.spec.steps + 1), cudaMemcpyDeviceToHost,
                                 cs)) != cudaSuccess ||
            (e = cudaMemcpyAsync(s->host_digest + job.slot, dig, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 cs)) != cudaSuccess)
            return cuda_fail(e, "copying job results");
    }
    if ((e = take_event(s, &c.ev)) != cudaSuccess || (e = cudaEventRecord(c.ev, cs)) != cudaSuccess)
        return cuda_fail(e, "recording the end of a direct chunk");
    job.busy = true;
    s->active_sum += s->active.size();  // resident jobs sharing the GPU at this launch
    if (c.finishing) {  // the job leaves the active set now; its memory is released at retirement
        s->active.erase(std::find(s->active.begin(), s->active.end(), j));
        s->active_items -= job.items;
    }
    s->chunks.push_back(c);
    s->rounds += 1;
    return SIMPLEX_OK;
}

int launch_round(simplex_server *s, cudaStream_t st)
{
    const auto t = std::chrono::steady_clock::now();
    const int rc = launch_round_impl(s, st);
    s->host_round_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t).count();
    return rc;
}

int launch_round_impl(simplex_server *s, cudaStream_t st)
{
    const int K = round_steps(s->prm);
    s->items.clear();
    s->fin_items.clear();
    Round r;
    cudaError_t e;
    // the round's events go back to the pool on every early return
    struct Guard {
        simplex_server *s;
        Round *r;
        bool armed;
        ~Guard()
        {
            if (!armed) return;
            if (r->ev0) s->spare_events.push_back(r->ev0);
            if (r->ev) s->spare_events.push_back(r->ev);
        }
    } guard{s, &r, true};
    if ((e = take_event(s, &r.ev0)) != cudaSuccess || (e = cudaEventRecord(r.ev0, st)) != cudaSuccess)
        return cuda_fail(e, "recording the start of a serving round");
    // blocks per work item: 8 when a pass has work for every resident CTA
    // several times over, fewer (down to 1) when it has not, so that a light
    // pass is spread over more CTAs instead of queueing blocks behind each other
    // (jobs with a direct chunk in flight sit this round out)
    uint64_t blocks = 0, members = 0;
    for (int64_t j : s->active)
        if (!s->jobs[j].busy) {
            blocks += s->slot_inst[s->jobs[j].slot].plan.h_blocks;
            ++members;
        }
    uint64_t chunk = blocks / (2 * s->ctas + 1);
    chunk = chunk < 1 ? 1 : (chunk > (uint64_t)sx::kBatchChunk ? (uint64_t)sx::kBatchChunk : chunk);
    // one item list for the round's passes: a job with r steps left takes part
    // in the first min(r, K) passes (tag bits 13..18); pass k reads parity ^ k
    // and counts at step index + k
    int passes = 0;
    for (int64_t j : s->active) {
        ServerJob &job = s->jobs[j];
        if (job.busy) continue;
        const sx::BatchInst &bi = s->slot_inst[job.slot];
        const int np = std::min(K, job.spec.steps - job.step);
        passes = std::max(passes, np);
        const uint32_t tag = (uint32_t)job.parity | ((uint32_t)(job.step + 1) << 1) | ((uint32_t)(np - 1) << 13);
        for (uint64_t v0 = 0; v0 < bi.plan.h_blocks; v0 += chunk) {
            const uint64_t cnt = std::min<uint64_t>(chunk, bi.plan.h_blocks - v0);
            s->items.push_back(sx::BatchItem{(uint32_t)job.slot, (uint32_t)v0, (uint32_t)cnt, tag});
        }
        job.step += np;
        job.parity ^= np & 1;
        s->cell_updates += job.cells * (uint64_t)np;
        if (job.step == job.spec.steps) {
            r.finishing.push_back(j);
            for (uint64_t v0 = 0; v0 < bi.plan.h_blocks; v0 += sx::kBatchChunk) {
                const uint64_t cnt = std::min<uint64_t>(sx::kBatchChunk, bi.plan.h_blocks - v0);
                s->fin_items.push_back(sx::BatchItem{(uint32_t)job.slot, (uint32_t)v0, (uint32_t)cnt,
                                                     (uint32_t)job.parity});
            }
        }
    }
    if (s->items.size() > s->max_items || s->fin_items.size() > s->max_items)
        return fail(SIMPLEX_ENOMEM, "a round needs %zu work items, max_items is %llu", s->items.size(),
                    (unsigned long long)s->max_items);
    s->active_sum += members;
    const sx::BatchInst *insts = reinterpret_cast<const sx::BatchInst *>(s->arena + s->off_insts);
    const CUtensorMap *tmaps = reinterpret_cast<const CUtensorMap *>(s->arena + s->off_tmaps);
    sx::BatchItem *items = reinterpret_cast<sx::BatchItem *>(s->arena + s->off_items);
    sx::BatchItem *fitems = items + s->max_items;
    unsigned int *queue = reinterpret_cast<unsigned int *>(s->arena + s->off_queue);
    unsigned long long *live = reinterpret_cast<unsigned long long *>(s->arena + s->off_live);
    unsigned long long *dig = reinterpret_cast<unsigned long long *>(s->arena + s->off_digest);
    const uint64_t ring = (uint64_t)(s->prm.max_inflight + 1);
    unsigned int *q = queue + (size_t)(K + 1) * (s->round_no % ring);
    // stage in pinned memory so the copies run asynchronously; a ring slot is
    // rewritten max_inflight + 1 rounds later, when the round that read it has
    // completed (the run loop never keeps more than max_inflight in flight)
    sx::BatchItem *stage = s->stage + (s->round_no % ring) * 2 * s->max_items;
    std::memcpy(stage, s->items.data(), sizeof(sx::BatchItem) * s->items.size());
    if ((e = cudaMemsetAsync(q, 0, sizeof(unsigned int) * (size_t)(K + 1), st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(items, stage, sizeof(sx::BatchItem) * s->items.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return cuda_fail(e, "launching a serving round");
    for (int k = 0; k < passes; ++k) {
        if ((e = sx::launch_batch_pass(insts, items, (uint32_t)s->items.size(), tmaps, s->arena, 0, q + k, live,
                                       s->prm.max_steps + 1, 0, false, st, nullptr, 0, k)) != cudaSuccess)
            return cuda_fail(e, "launching a serving round");
        s->launches += 1;
    }
    if (!s->fin_items.empty()) {
        std::memcpy(stage + s->max_items, s->fin_items.data(), sizeof(sx::BatchItem) * s->fin_items.size());
        if ((e = cudaMemcpyAsync(fitems, stage + s->max_items, sizeof(sx::BatchItem) * s->fin_items.size(),
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = sx::launch_batch_pass(insts, fitems, (uint32_t)s->fin_items.size(), tmaps, s->arena, 0, q + K,
                                       nullptr, 0, 0, true, st, dig)) != cudaSuccess)
            return cuda_fail(e, "launching the digest pass");
        s->launches += 1;
        for (int64_t j : r.finishing) {
            const int slot = s->jobs[j].slot;
            const size_t row = (size_t)(s->prm.max_steps + 1);
            if ((e = cudaMemcpyAsync(s->host_live + slot * row, live + slot * row,
                                     sizeof(unsigned long long) * (size_t)(s->jobs[j].spec.steps + 1),
                                     cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(s->host_digest + slot, dig + slot, sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return cuda_fail(e, "copying job results");
        }
        // finishing jobs leave the active set now; their memory is released at retirement
        std::vector<int64_t> still;
        still.reserve(s->active.size());
        for (int64_t j : s->active) {
            if (s->jobs[j].step < s->jobs[j].spec.steps) still.push_back(j);
            else s->active_items -= s->jobs[j].items;
        }
        s->active.swap(still);
    }
    if ((e = take_event(s, &r.ev)) != cudaSuccess || (e = cudaEventRecord(r.ev, st)) != cudaSuccess)
        return cuda_fail(e, "recording the end of a serving round");
    guard.armed = false;
    s->inflight.push_back(std::move(r));
    s->rounds += 1;
    s->round_no += 1;
    return SIMPLEX_OK;
}

// A job whose last step has completed: results from the pinned copies, its
// memory and slot back to the pool.
void finish_job(simplex_server *s, int64_t j, float done_ms)
{
    ServerJob &job = s->jobs[j];
    const size_t row = (size_t)(s->prm.max_steps + 1);
    job.live.assign(s->host_live + job.slot * row, s->host_live + job.slot * row + job.spec.steps + 1);
    job.digest = s->host_digest[job.slot];
    job.done_ms = done_ms;
    job.seen_ms = host_ms(s);
    job.status = kDone;
    job.busy = false;
    s->pool.release(job.off, job.bytes);
    s->free_slots.push_back(job.slot);
    job.slot = -1;
}

// Retires the direct chunks that have completed.  Returns the number of jobs
// that finished (or <0); *completed += the chunks retired.
int retire_chunks(simplex_server *s, int *completed)
{
    int finished = 0;
    for (size_t i = 0; i < s->chunks.size();) {
        Chunk &c = s->chunks[i];
        cudaError_t e = cudaEventQuery(c.ev);
        if (e == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (e != cudaSuccess) return cuda_fail(e, "waiting for a direct chunk");
        float ms = 0, dur = 0;
        if ((e = cudaEventElapsedTime(&ms, s->t0, c.ev)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&dur, c.ev0, c.ev)) != cudaSuccess)
            return cuda_fail(e, "cudaEventElapsedTime");
        s->gpu_round_ms += dur;
        if (c.finishing) {
            finish_job(s, c.job, ms);
            ++finished;
        } else {
            s->jobs[c.job].busy = false;
        }
        s->spare_events.push_back(c.ev);
        s->spare_events.push_back(c.ev0);
        c = s->chunks.back();
        s->chunks.pop_back();
        ++*completed;
    }
    return finished;
}

// Retires the oldest in-flight rounds whose event has completed (or, with
// `wait`, the oldest one regardless).  Returns the number of jobs that
// finished, or <0; *completed += the rounds retired.
int retire(simplex_server *s, bool wait, int *completed)
{
    int n = 0, finished = 0;
    while (!s->inflight.empty()) {
        Round &r = s->inflight.front();
        cudaError_t e = wait && n == 0 ? cudaEventSynchronize(r.ev) : cudaEventQuery(r.ev);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return cuda_fail(e, "waiting for a serving round");
        float ms = 0, dur = 0;
        if ((e = cudaEventElapsedTime(&ms, s->t0, r.ev)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&dur, r.ev0, r.ev)) != cudaSuccess)
            return cuda_fail(e, "cudaEventElapsedTime");
        s->gpu_round_ms += dur;
        for (int64_t j : r.finishing) {
            finish_job(s, j, ms);
            ++finished;
        }
        s->spare_events.push_back(r.ev);
        s->spare_events.push_back(r.ev0);
        s->inflight.pop_front();
        ++n;
    }
    *completed += n;
    return finished;
}

// Clears the job table and statistics and starts the server's clocks (host
// and device) for a new trace or online session.
int reset_session(simplex_server *s, cudaStream_t st)
{
    s->jobs.clear();
    s->pending.clear();
    s->rounds = s->cell_updates = s->active_sum = 0;
    s->active_items = 0;
    s->host_round_ms = 0;
    s->gpu_round_ms = 0;
    s->launches = 0;
    s->wall_ms = 0;
    s->pool.reset(s->prm.hbm_budget);
    cudaError_t e = sx::batch_prepare();
    if (e != cudaSuccess) return cuda_fail(e, "setting the batch kernel's shared memory");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "synchronising before a trace");
    s->round_no = 0;
    if ((e = sx::batch_resident_ctas(&s->ctas)) != cudaSuccess) return cuda_fail(e, "occupancy query");
    if ((e = cudaEventRecord(s->t0, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    s->h0 = std::chrono::steady_clock::now();
    s->stream = st;
    return SIMPLEX_OK;
}

int check_job(const simplex_server *s, const simplex_job_t &sp, int64_t i)
{
    if ((sp.m != 2 && sp.m != 3) || sp.n < 0 || sp.steps < 1 || sp.steps > s->prm.max_steps)
        return fail(SIMPLEX_EINVAL, "job %lld: m must be 2 or 3, n >= 0, steps in [1, %d]", (long long)i,
                    s->prm.max_steps);
    return SIMPLEX_OK;
}

// One turn of the serving loop.  Retirement of the rounds and chunks that have
// completed.  Admission: jobs that have arrived, first come first served, as
// slots and pool memory allow.  Work: with at most
// direct_jobs jobs resident, a direct chunk for every resident job that has
// none in flight; otherwise one batched round over those jobs when fewer than
// max_inflight rounds are queued.  Retirement of the rounds and chunks that
// have completed -- with `block`, waiting for one to complete when nothing
// else can progress.  *done += the jobs that finished (done or rejected).
int serve_turn(simplex_server *s, cudaStream_t st, bool realtime, bool block, int64_t *done)
{
    // retire what has completed first: a job's results become readable before
    // this turn spends host time on admissions and launches, and its memory
    // and slot are free for them
    int completed = 0;
    int r = retire(s, false, &completed);
    if (r < 0) return SIMPLEX_ECUDA;
    *done += r;
    if ((r = retire_chunks(s, &completed)) < 0) return SIMPLEX_ECUDA;
    *done += r;
    const double now = host_ms(s);
    while (!s->pending.empty()) {
        const int64_t j = s->pending.front();
        if (realtime && s->jobs[j].arrival_ms > now) break;
        const int a = admit(s, j, st);
        if (a < 0) {
            if (a == -2) {
                s->jobs[j].status = kRejected;
                s->pending.pop_front();
                ++*done;
                continue;
            }
            return SIMPLEX_ECUDA;
        }
        if (a == 0) break;
        s->pending.pop_front();
    }
    const int dj = direct_jobs(s->prm);
    const bool direct = dj > 0 && s->active.size() <= (size_t)dj;
    bool idle_job = false;  // a resident job with nothing in flight
    for (int64_t j : s->active) idle_job |= !s->jobs[j].busy;
    if (direct) {
        const std::vector<int64_t> act = s->active;  // launch_chunk may shrink the active set
        for (int64_t j : act)
            if (!s->jobs[j].busy) {
                const int rc = launch_chunk(s, j, st);
                if (rc) return rc;
                // a chunk is tens of launches of host time: chunks that complete
                // meanwhile are retired (their jobs seen done) between two chunks
                if ((r = retire_chunks(s, &completed)) < 0) return SIMPLEX_ECUDA;
                *done += r;
            }
        idle_job = false;
    } else if (idle_job && (int)s->inflight.size() < s->prm.max_inflight) {
        const int rc = launch_round(s, st);
        if (rc) return rc;
        idle_job = false;
        for (int64_t j : s->active) idle_job |= !s->jobs[j].busy;
        idle_job = idle_job && (int)s->inflight.size() < s->prm.max_inflight;
    }
    if ((r = retire(s, false, &completed)) < 0) return SIMPLEX_ECUDA;
    *done += r;
    if ((r = retire_chunks(s, &completed)) < 0) return SIMPLEX_ECUDA;
    *done += r;
    // nothing can be launched until something completes: wait for one
    const bool busy_gpu = !s->inflight.empty() || !s->chunks.empty();
    const bool arrived = !s->pending.empty() && (!realtime || s->jobs[s->pending.front()].arrival_ms <= host_ms(s));
    // (in real time the wait also ends when a job arrives that can take a
    // free slot: it is admitted, and in direct mode started, without waiting
    // for another job's chunk or round to end)
    if (block && completed == 0 && busy_gpu && !idle_job &&
        ((int)s->inflight.size() >= s->prm.max_inflight || !arrived || s->free_slots.empty())) {
        while (completed == 0) {
            if ((r = retire(s, false, &completed)) < 0) return SIMPLEX_ECUDA;
            *done += r;
            if ((r = retire_chunks(s, &completed)) < 0) return SIMPLEX_ECUDA;
            *done += r;
            if (completed) break;
            if (realtime) {
                if (!s->pending.empty() && !s->free_slots.empty() &&
                    s->jobs[s->pending.front()].arrival_ms <= host_ms(s))
                    break;
            } else if (s->chunks.empty() && !s->inflight.empty()) {
                if ((r = retire(s, true, &completed)) < 0) return SIMPLEX_ECUDA;  // only rounds: block on the oldest
                *done += r;
            }
        }
    }
    return SIMPLEX_OK;
}

}  // namespace

extern "C" {

int simplex_server_arena_bytes(const simplex_server_params_t *params, uint64_t *out)
{
    int rc = check_params(params);
    if (rc) return rc;
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    *out = layout(*params, nullptr);
    return SIMPLEX_OK;
}

int simplex_server_create(const simplex_server_params_t *params, void *arena, uint64_t arena_bytes,
                          simplex_server_t *out)
{
    int rc = check_params(params);
    if (rc) return rc;
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!arena || (reinterpret_cast<uintptr_t>(arena) & 255u))
        return fail(SIMPLEX_EINVAL, "arena must be a 256-byte aligned device pointer");
    simplex_server *s = new (std::nothrow) simplex_server();
    if (!s) return fail(SIMPLEX_ENOMEM, "host allocation failed");
    s->prm = *params;
    const uint64_t need = layout(*params, s);
    if (arena_bytes < need) {
        delete s;
        return fail(SIMPLEX_EINVAL, "arena too small: %llu bytes, need %llu", (unsigned long long)arena_bytes,
                    (unsigned long long)need);
    }
    s->arena = static_cast<uint8_t *>(arena);
    s->bytes = need;
    s->pool.reset(params->hbm_budget);
    try {
        s->slot_inst.resize(params->max_jobs);
        s->slot_tmap.resize(2 * (size_t)params->max_jobs);
        s->slot_dplan.resize(params->max_jobs);
        s->slot_dtmap.resize(2 * (size_t)params->max_jobs);
        for (int i = params->max_jobs - 1; i >= 0; --i) s->free_slots.push_back(i);
    } catch (...) {
        delete s;
        return fail(SIMPLEX_ENOMEM, "host allocation failed");
    }
    cudaError_t e;
    const size_t row = (size_t)(params->max_steps + 1);
    if ((e = cudaMallocHost(&s->host_live, sizeof(unsigned long long) * row * params->max_jobs)) != cudaSuccess ||
        (e = cudaMallocHost(&s->host_digest, sizeof(unsigned long long) * params->max_jobs)) != cudaSuccess ||
        (e = cudaMallocHost(&s->stage, sizeof(sx::BatchItem) * 2 * (size_t)params->max_items *
                                           (size_t)(params->max_inflight + 1))) != cudaSuccess ||
        (e = cudaEventCreate(&s->t0)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s->main_ev, cudaEventDisableTiming)) != cudaSuccess) {
        if (s->host_live) cudaFreeHost(s->host_live);
        if (s->host_digest) cudaFreeHost(s->host_digest);
        if (s->stage) cudaFreeHost(s->stage);
        if (s->t0) cudaEventDestroy(s->t0);
        delete s;
        return cuda_fail(e, "allocating the server's pinned result buffers");
    }
    for (auto &cs : s->side)
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
            simplex_server_destroy(s);
            return cuda_fail(e, "creating the server's side streams");
        }
    *out = s;
    return SIMPLEX_OK;
}

int simplex_server_destroy(simplex_server_t s)
{
    if (!s) return SIMPLEX_OK;
    for (auto &r : s->inflight) {
        cudaEventSynchronize(r.ev);
        cudaEventDestroy(r.ev);
        cudaEventDestroy(r.ev0);
    }
    for (auto &c : s->chunks) {
        cudaEventSynchronize(c.ev);
        cudaEventDestroy(c.ev);
        cudaEventDestroy(c.ev0);
    }
    for (auto ev : s->spare_events) cudaEventDestroy(ev);
    for (auto cs : s->side)
        if (cs) cudaStreamDestroy(cs);
    if (s->main_ev) cudaEventDestroy(s->main_ev);
    if (s->t0) cudaEventDestroy(s->t0);
    if (s->host_live) cudaFreeHost(s->host_live);
    if (s->host_digest) cudaFreeHost(s->host_digest);
    if (s->stage) cudaFreeHost(s->stage);
    delete s;
    return SIMPLEX_OK;
}

int simplex_server_run(simplex_server_t s, const simplex_job_t *jobs, const double *arrival_s, int count,
                       int realtime, void *stream)
{
    if (!s) return fail(SIMPLEX_EINVAL, "server is NULL");
    if (count < 0 || (!jobs && count > 0)) return fail(SIMPLEX_EINVAL, "jobs is NULL or count < 0");
    if (!s->active.empty() || !s->inflight.empty() || !s->pending.empty() || !s->chunks.empty())
        return fail(SIMPLEX_EINVAL, "the server is still running another trace");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < count; ++i) {
        const int rc = check_job(s, jobs[i], i);
        if (rc) return rc;
    }
    int rc = reset_session(s, st);
    if (rc) return rc;
    s->stream_set = false;  // a trace is not an online session
    // queue every job in arrival order
    s->jobs.resize(count);
    std::vector<int64_t> order(count);
    for (int i = 0; i < count; ++i) {
        s->jobs[i].spec = jobs[i];
        s->jobs[i].arrival_ms = arrival_s ? arrival_s[i] * 1e3 : 0.0;
        s->jobs[i].cells = binom((uint64_t)jobs[i].n + (uint64_t)jobs[i].m, jobs[i].m);
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return s->jobs[a].arrival_ms < s->jobs[b].arrival_ms; });
    for (int64_t j : order) s->pending.push_back(j);
    int64_t done = 0;
    while (done < count) {
        if ((rc = serve_turn(s, st, realtime != 0, true, &done))) return rc;
        if (s->active.empty() && s->inflight.empty() && s->chunks.empty() && !s->pending.empty() && realtime) {
            // nothing on the GPU (a job's last chunk is not in the active set,
            // so chunks are checked too: sleeping past one would hold its
            // completion until the next arrival): sleep until 0.2 ms before the
            // next arrival, then spin: a sleep can overshoot by tens of
            // microseconds, which would add to that job's latency
            const double wait_ms = s->jobs[s->pending.front()].arrival_ms - host_ms(s);
            if (wait_ms > 0.3)
                std::this_thread::sleep_for(std::chrono::microseconds((int64_t)((wait_ms - 0.2) * 1000)));
        }
    }
    s->wall_ms = host_ms(s);
    return SIMPLEX_OK;
}

int simplex_server_begin(simplex_server_t s, void *stream)
{
    if (!s) return fail(SIMPLEX_EINVAL, "server is NULL");
    if (!s->active.empty() || !s->inflight.empty() || !s->pending.empty() || !s->chunks.empty())
        return fail(SIMPLEX_EINVAL, "the server still has jobs in progress");
    const int rc = reset_session(s, static_cast<cudaStream_t>(stream));
    s->stream_set = rc == SIMPLEX_OK;
    return rc;
}

int simplex_server_submit(simplex_server_t s, const simplex_job_t *job, int64_t *id)
{
    if (!s) return fail(SIMPLEX_EINVAL, "server is NULL");
    if (!job || !id) return fail(SIMPLEX_EINVAL, "job and id must not be NULL");
    if (!s->stream_set) return fail(SIMPLEX_EINVAL, "call simplex_server_begin before submitting jobs");
    const int64_t i = (int64_t)s->jobs.size();
    int rc = check_job(s, *job, i);
    if (rc) return rc;
    ServerJob j;
    j.spec = *job;
    j.arrival_ms = host_ms(s);
    j.cells = binom((uint64_t)job->n + (uint64_t)job->m, job->m);
    s->jobs.push_back(j);
    s->pending.push_back(i);
    *id = i;
    return SIMPLEX_OK;
}

int simplex_server_poll(simplex_server_t s, int *finished)
{
    if (!s) return fail(SIMPLEX_EINVAL, "server is NULL");
    if (!s->stream_set) return fail(SIMPLEX_EINVAL, "call simplex_server_begin first");
    int64_t done = 0;
    const int rc = serve_turn(s, s->stream, true, false, &done);
    if (rc) return rc;
    s->wall_ms = host_ms(s);
    if (finished) *finished = (int)done;
    return SIMPLEX_OK;
}

int simplex_server_wait(simplex_server_t s, int64_t id)
{
    if (!s) return fail(SIMPLEX_EINVAL, "server is NULL");
    if (!s->stream_set) return fail(SIMPLEX_EINVAL, "call simplex_server_begin first");
    if (id >= (int64_t)s->jobs.size()) return fail(SIMPLEX_EINVAL, "no job %lld", (long long)id);
    auto finished = [&]() {
        if (id >= 0) return s->jobs[id].status == kDone || s->jobs[id].status == kRejected;
        return s->active.empty() && s->inflight.empty() && s->pending.empty() && s->chunks.empty();
    };
    while (!finished()) {
        int64_t done = 0;
        const int rc = serve_turn(s, s->stream, true, true, &done);
        if (rc) return rc;
    }
    s->wall_ms = host_ms(s);
    return SIMPLEX_OK;
}

int simplex_server_result(simplex_server_t s, int64_t job, simplex_job_result_t *out, unsigned long long *live)
{
    if (!s) return fail(SIMPLEX_EINVAL, "server is NULL");
    if (job < 0 || job >= (int64_t)s->jobs.size()) return fail(SIMPLEX_EINVAL, "job %lld out of range", (long long)job);
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    const ServerJob &j = s->jobs[job];
    std::memset(out, 0, sizeof *out);
    out->status = j.status;
    out->steps = j.spec.steps;
    out->arrival_ms = j.arrival_ms;
    out->admit_ms = j.admit_ms;
    out->done_ms = j.done_ms;
    out->seen_ms = j.seen_ms;
    out->digest = j.digest;
    out->live_final = j.live.empty() ? 0 : j.live.back();
    if (live && !j.live.empty()) std::memcpy(live, j.live.data(), sizeof(unsigned long long) * j.live.size());
    return SIMPLEX_OK;
}

int simplex_server_stats(simplex_server_t s, simplex_server_stats_t *out)
{
    if (!s) return fail(SIMPLEX_EINVAL, "server is NULL");
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof *out);
    std::vector<double> lat, seen;
    for (const auto &j : s->jobs)
        if (j.status == kDone) {
            lat.push_back(j.done_ms - j.arrival_ms);
            seen.push_back(j.seen_ms - j.arrival_ms);
        } else if (j.status == kRejected) {
            out->rejected += 1;
        }
    out->submitted = s->jobs.size();
    out->completed = lat.size();
    out->rounds = s->rounds;
    out->cell_updates = s->cell_updates;
    out->wall_ms = s->wall_ms;
    out->mean_active = s->rounds ? (double)s->active_sum / (double)s->rounds : 0.0;
    out->peak_pool_bytes = s->pool.peak();
    out->host_issue_ms = s->host_round_ms;
    out->gpu_round_ms = s->rounds ? s->gpu_round_ms / (double)s->rounds : 0.0;
    out->launches = s->launches;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto q = [&](double f) { return lat[std::min(lat.size() - 1, (size_t)(f * (double)(lat.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p90_ms = q(0.90);
        out->p99_ms = q(0.99);
        out->max_ms = lat.back();
        double sum = 0;
        for (double x : lat) sum += x;
        out->mean_ms = sum / (double)lat.size();
        std::sort(seen.begin(), seen.end());
        auto qs = [&](double f) {
            return seen[std::min(seen.size() - 1, (size_t)(f * (double)(seen.size() - 1) + 0.5))];
        };
        out->host_p50_ms = qs(0.50);
        out->host_p99_ms = qs(0.99);
    }
    return SIMPLEX_OK;
}

}  // extern "C"
