// api.cpp -- the C ABI of libsimplex (include/simplex.h): argument checks, the
// host-side launch plan, TMA tensor maps, CUDA-graph capture of automaton
// runs, and the error model (status codes + thread-local message; nothing
// aborts, no device trap).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/simplex.h"
#include "hmap.cuh"
#include "host.h"
#include "kernels.h"

namespace sxh {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(SIMPLEX_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

}  // namespace sxh

using namespace sxh;

namespace {

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

int ilog2_i64(int64_t x)
{
    int l = 0;
    while ((int64_t(1) << (l + 1)) <= x) ++l;
    return l;
}

uint64_t ipow(uint64_t b, int e)
{
    uint64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

uint64_t binom(uint64_t n, int k)
{
    // C(n, k) for small k, exact in 128-bit intermediate
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return (uint64_t)r;
}

// Trapezoid band height (tiles) the automatic plan uses for m = 2.
constexpr int kDefaultBand = 8;
// m = 3 x-stream form: tiles per run along x3 (a run reads 2 extra x-columns)
constexpr int kStreamRun = 16;

struct GraphEntry {
    uint8_t *a, *b;
    int steps;
    uint32_t birth, survive;
    unsigned long long *live;
    int mode;
    cudaGraphExec_t exec;
};

}  // namespace

struct simplex_map {
    sx::Plan plan;
    int r_inv;
    int device = -1;
    cudaStream_t capture = nullptr;
    std::vector<GraphEntry> graphs;
    // m = 3 x-stream and plane-stream forms: work counter and CTAs-done
    // counter (zero between launches)
    unsigned long long *queue = nullptr;
    int queue_device = -1;
    // m = 3 plane-stream form: the unit schedule of each mode (built on first use)
    sx::PlaneSched *sched[3] = {nullptr, nullptr, nullptr};
};

namespace sxh {

int build_plan(int m, int64_t n, int r_inv, int beta, int block, int64_t side, int band, sx::Plan *p, int layout)
{
    if (m < 2 || m > 4) return fail(SIMPLEX_EINVAL, "m must be 2, 3 or 4 (got %d)", m);
    if (n < 0) return fail(SIMPLEX_EINVAL, "n must be >= 0 (got %lld)", (long long)n);
    if (r_inv != 2 && !(r_inv == 3 && m == 2))
        return fail(SIMPLEX_EUNSUPPORTED,
                    "r = 1/%d is not implemented for m = %d (r = 1/2 for every m, r = 1/3 for m = 2)", r_inv, m);
    const bool beta_ok = r_inv == 3 ? beta == 3
                                    : (m == 2 && beta == 2) || (m == 3 && (beta == 2 || beta == 3)) ||
                                          (m == 4 && beta == 4);
    if (!beta_ok)
        return fail(SIMPLEX_EUNSUPPORTED,
                    "beta = %d does not give a covering map for m = %d, r = 1/%d (r = 1/2: m=2: 2; m=3: 2 or 3; "
                    "m=4: 4; r = 1/3, m = 2: 3)", beta, m, r_inv);
    if (r_inv == 3 && band > 0)
        return fail(SIMPLEX_EINVAL, "the trapezoid form (band > 0) is an r = 1/2 map; r = 1/3 takes band 0 or -1");
    if (!is_pow2(block) || block < 4 || block > 256)
        return fail(SIMPLEX_EINVAL, "block must be a power of two in [4, 256] (got %d)", block);
    if (side < n + 1) return fail(SIMPLEX_EINVAL, "side (%lld) must be >= n + 1", (long long)side);
    const int64_t nb = (n + block) / block;  // ceil((n+1)/rho)
    int64_t N = 1;
    int logN = 0;
    while (N < nb) {
        N <<= 1;
        ++logN;
    }
    if (logN > 15) return fail(SIMPLEX_EINVAL, "n / block too large: %lld tiles per axis (max 32768)", (long long)nb);
    // array size in elements must fit comfortably in 63 bits
    {
        long double tot = 1;
        for (int i = 0; i < m; ++i) tot *= (long double)side;
        if (tot > 4.0e18L) return fail(SIMPLEX_EINVAL, "side^m too large");
    }

    std::memset(p, 0, sizeof *p);
    p->m = m;
    p->rho = block;
    p->log_rho = ilog2_i64(block);
    p->N = (int32_t)N;
    p->logN = logN;
    p->beta = beta;
    p->n = n;
    p->side = side;
    p->bb_blocks = ipow((uint64_t)N, m);
    p->rinv = r_inv;
    p->seg_len = (int32_t)(N < kStreamRun ? N : kStreamRun);
    const uint64_t h2 = sx::h2_cover_blocks((int32_t)N);
    if (m != 2 && band > 0)
        return fail(SIMPLEX_EINVAL, "band (trapezoid height) applies to m = 2 only (got %d for m = %d)", band, m);
    if (r_inv == 3) {
        int64_t N3 = 1;
        int L3 = 0;
        while (N3 < nb) {
            N3 *= 3;
            ++L3;
        }
        p->N3 = (int32_t)N3;
        p->L3 = L3;
        p->h_blocks = (uint64_t)N3 * (uint64_t)(N3 + 1) / 2;
    } else if (m == 2 && band > 0) {
        if (!is_pow2(band) || band > 32768)
            return fail(SIMPLEX_EINVAL, "band must be a power of two <= 32768 (got %d)", band);
        const int64_t Ne = (nb + band - 1) / band * band;
        p->band = band;
        p->log_band = ilog2_i64(band);
        p->Ne = (int32_t)Ne;
        p->nbands = (int32_t)(Ne / band);
        p->h_blocks = (uint64_t)Ne * (uint64_t)(Ne + 1) / 2;
    } else if (m == 2) {
        p->h_blocks = h2;
    } else if (m == 3 && beta == 2) {
        const uint64_t half = (uint64_t)N / 2;
        p->h3_cube = half * half * half;
        p->h3_exact = layout == 1 ? 1 : 0;
        if (p->h3_exact)
            p->h3_layer = N >= 4 ? sx::h3_level_prefix((int32_t)N, logN + 1) : 0;
        else
            p->h3_layer = N >= 4 ? half * ((uint64_t)N / 4) * (half - 1) : 0;
        p->h_blocks = p->h3_cube + p->h3_layer + h2;
    } else {
        uint64_t total = h2;
        for (int d = 3; d <= m; ++d) {
            uint64_t acc = 0;
            p->level_end[d - 3][0] = 0;
            for (int k = 1; k <= logN; ++k) {
                acc += ipow((uint64_t)d, k - 1) * ipow((uint64_t)(N >> k), d);
                p->level_end[d - 3][k] = acc;
            }
            p->cube_total[d - 3] = acc;
            total += acc;
        }
        p->h_blocks = total;
    }
    return SIMPLEX_OK;
}

sx::Rule make_rule(int m, uint32_t birth, uint32_t survive)
{
    sx::Rule r;
    std::memset(&r, 0, sizeof r);
    const int kmax = m == 2 ? 9 : 27;  // largest neighbourhood sum including the cell
    for (int s = 0; s <= kmax; ++s) {
        const bool b = s <= kmax - 1 && ((birth >> s) & 1u);
        const bool sv = s >= 1 && ((survive >> (s - 1)) & 1u);
        if (!b && !sv) continue;
        r.kbytes[r.nk] = 0x01010101u * (uint32_t)s;
        r.bsel[r.nk] = b ? 0xffffffffu : 0u;
        r.ssel[r.nk] = sv ? 0xffffffffu : 0u;
        ++r.nk;
    }
    // "or-k" form: born with k, survive with k-1 or k, k odd
    const int nmax = m == 2 ? 8 : 26;
    for (int k = 1; k <= nmax; k += 2)
        if (birth == (1u << k) && survive == ((1u << (k - 1)) | (1u << k))) r.or_k = 0x01010101u * (uint32_t)k;
    return r;
}

}  // namespace sxh

namespace {

bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

int check_map(simplex_map_t map)
{
    if (!map) return fail(SIMPLEX_EINVAL, "map is NULL");
    return SIMPLEX_OK;
}

int check_mode(int mode)
{
    if (mode != SIMPLEX_MODE_H && mode != SIMPLEX_MODE_BB && mode != SIMPLEX_MODE_BB_THREAD)
        return fail(SIMPLEX_EINVAL, "mode must be SIMPLEX_MODE_H, SIMPLEX_MODE_BB or SIMPLEX_MODE_BB_THREAD (got %d)",
                    mode);
    return SIMPLEX_OK;
}

int check_ca_layout(const sx::Plan &p, const void *grid, const char *name)
{
    if (p.m != 2 && p.m != 3) return fail(SIMPLEX_EINVAL, "the automaton is implemented for m = 2 and 3 (map has m = %d)", p.m);
    if (!grid) return fail(SIMPLEX_EINVAL, "%s is NULL", name);
    if (!aligned16(grid)) return fail(SIMPLEX_EINVAL, "%s must be 16-byte aligned", name);
    if (p.side % 16 != 0) return fail(SIMPLEX_EINVAL, "the automaton needs side %% 16 == 0 (side = %lld)", (long long)p.side);
    if (p.rho < 16) return fail(SIMPLEX_EINVAL, "the automaton needs block >= 16 (block = %d)", p.rho);
    return SIMPLEX_OK;
}

// The x-stream form's work counters: allocated (zeroed) on first use on the
// current device; not during stream capture (simplex_ca_run calls this first).
int ensure_queue(simplex_map_t map)
{
    if (!(map->plan.m == 3 && map->plan.persistent)) return SIMPLEX_OK;
    if (map->plan.persistent == 2) {
        for (int k = 0; k < 3; ++k) {
            if (map->sched[k]) continue;
            sx::PlaneSched *s = new (std::nothrow) sx::PlaneSched();
            if (!s) return fail(SIMPLEX_ENOMEM, "host allocation failed");
            if (!sx::plane_sched_build(map->plan.n, k, s)) {
                delete s;
                return fail(SIMPLEX_EUNSUPPORTED, "n = %lld needs more plane-stream segments or units than supported",
                            (long long)map->plan.n);
            }
            map->sched[k] = s;
        }
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (map->queue) {
        if (map->queue_device != dev)
            return fail(SIMPLEX_EINVAL, "the map's work counters live on device %d, not %d", map->queue_device, dev);
        return SIMPLEX_OK;
    }
    // two counters, then (plane stream) the segment tables of the three map
    // kinds, which the kernel's producer searches through L1
    const size_t tables = map->plan.persistent == 2 ? 3 * sx::kPlaneSegWords * sizeof(int32_t) : 0;
    void *q = nullptr;
    if ((e = cudaMalloc(&q, 2 * sizeof(unsigned long long) + tables)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(work counters)");
    if ((e = cudaMemset(q, 0, 2 * sizeof(unsigned long long))) != cudaSuccess) {
        cudaFree(q);
        return cuda_fail(e, "cudaMemset(work counters)");
    }
    if (tables) {
        std::vector<int32_t> h(3 * sx::kPlaneSegWords, 0);
        for (int k = 0; k < 3; ++k) {
            std::memcpy(h.data() + k * sx::kPlaneSegWords, map->sched[k]->seg_b, sizeof(map->sched[k]->seg_b));
            std::memcpy(h.data() + k * sx::kPlaneSegWords + sx::kPlaneSegTable, map->sched[k]->seg_u,
                        sizeof(map->sched[k]->seg_u));
        }
        e = cudaMemcpy(static_cast<unsigned long long *>(q) + 2, h.data(), tables, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(q);
            return cuda_fail(e, "cudaMemcpy(plane-stream segment tables)");
        }
    }
    map->queue = static_cast<unsigned long long *>(q);
    map->queue_device = dev;
    return SIMPLEX_OK;
}

int step_once(simplex_map_t map, const uint8_t *in, uint8_t *out, const sx::Rule &rule,
              unsigned long long *live, int mode, cudaStream_t st)
{
    const sx::Plan &p = map->plan;
    int rc = ensure_queue(map);
    if (rc) return rc;
    if (p.m == 3 && p.persistent == 2) {
        sx::PlaneMaps maps;
        if ((rc = make_plane_maps(p, in, &maps))) return rc;
        const int32_t *segs = reinterpret_cast<const int32_t *>(map->queue + 2) + mode * sx::kPlaneSegWords;
        cudaError_t e =
            sx::launch_ca3_planes(*map->sched[mode], segs, maps, p.n, p.side, out, rule, live, map->queue, st);
        if (e != cudaSuccess) return cuda_fail(e, "automaton step launch");
        return SIMPLEX_OK;
    }
    CUtensorMap tm;
    rc = make_tensor_map(p, in, &tm, sx::ca3_box_planes(p));
    if (rc) return rc;
    cudaError_t e = p.m == 2 ? sx::launch_ca2_step(p, tm, out, rule, mode, live, st)
                             : sx::launch_ca3_step(p, tm, out, rule, mode, live, map->queue, st);
    if (e != cudaSuccess) return cuda_fail(e, "automaton step launch");
    return SIMPLEX_OK;
}

int check_step_args(simplex_map_t map, const uint8_t *in, const uint8_t *out, int mode)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_mode(mode))) return rc;
    const sx::Plan &p = map->plan;
    if ((rc = check_ca_layout(p, in, "in")) || (rc = check_ca_layout(p, out, "out"))) return rc;
    if (in == out) return fail(SIMPLEX_EINVAL, "in and out must be distinct buffers");
    const bool ok = p.m == 2 ? sx::ca2_supports(p.rho) : sx::ca3_supports(p.rho);
    if (!ok)
        return fail(SIMPLEX_EUNSUPPORTED, "automaton step for m = %d supports block %s (got %d)", p.m,
                    p.m == 2 ? "32, 64, 128" : "16, 32", p.rho);
    return SIMPLEX_OK;
}

// The whole run as stream work: zero live, count live[0], then the steps.
int enqueue_run(simplex_map_t map, uint8_t *a, uint8_t *b, int steps, const sx::Rule &rule,
                unsigned long long *live, int mode, cudaStream_t st)
{
    if (live) {
        cudaError_t e = cudaMemsetAsync(live, 0, sizeof(unsigned long long) * (size_t)(steps + 1), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(live)");
        e = sx::launch_ca_count(map->plan, a, live, st);
        if (e != cudaSuccess) return cuda_fail(e, "live count launch");
    }
    for (int s = 1; s <= steps; ++s) {
        const uint8_t *src = (s & 1) ? a : b;
        uint8_t *dst = (s & 1) ? b : a;
        int rc = step_once(map, src, dst, rule, live ? live + s : nullptr, mode, st);
        if (rc) return rc;
    }
    return SIMPLEX_OK;
}

}  // namespace

namespace {

// Host <-> device transfers of the domain only (Sec. 2, Eq. 1: every grid is
// zero past the simplex and the steps keep it so, so only the prefix of each
// row that holds domain cells has to move).  m = 2: rows x1 = 0 ... n in
// kCopyBands2 bands, each one pitched 2-D copy as wide as its longest row
// (n - r0 + 1 cells).  m = 3: kCopyBands3 bands of planes x1, each cut into
// kCopySub3 ranges of rows x2, each one pitched 3-D copy as wide as its
// longest row.  For n = 32767 (m = 2) this moves 0.55 GB instead of the
// 1.07 GB array, for n = 1023 (m = 3) 0.22 GB instead of 1.07 GB.
constexpr int64_t kCopyBands2 = 32, kCopyBands3 = 16, kCopySub3 = 8;

// Calls f(x1_0, x1_1, x2_0, x2_1, width) for every copy box (m = 2: x1 is
// the row, the x2 range is [0, 1)).
template <typename F>
void for_each_copy_box(const sx::Plan &p, F f)
{
    const int64_t R = p.n + 1;
    if (p.m == 2) {
        const int64_t B = std::min(kCopyBands2, R);
        for (int64_t k = 0; k < B; ++k) {
            const int64_t r0 = R * k / B, r1 = R * (k + 1) / B;
            if (r1 > r0) f(r0, r1, 0, 1, p.n - r0 + 1);
        }
        return;
    }
    const int64_t B = std::min(kCopyBands3, R);
    for (int64_t k = 0; k < B; ++k) {
        const int64_t a0 = R * k / B, a1 = R * (k + 1) / B;
        if (a1 <= a0) continue;
        const int64_t L = p.n - a0 + 1, J = std::min(kCopySub3, L);  // rows x2 = 0 ... n - a0
        for (int64_t j = 0; j < J; ++j) {
            const int64_t b0 = L * j / J, b1 = L * (j + 1) / J;
            if (b1 > b0) f(a0, a1, b0, b1, p.n - a0 - b0 + 1);
        }
    }
}

uint64_t domain_copy_bytes(const sx::Plan &p)
{
    uint64_t s = 0;
    for_each_copy_box(p, [&](int64_t a0, int64_t a1, int64_t b0, int64_t b1, int64_t w) {
        s += (uint64_t)((a1 - a0) * (b1 - b0) * w);
    });
    return s;
}

// All copies go on `st` (spreading them over four streams gave the same
// rate: the host link, not one copy engine, is the limit).
cudaError_t copy_domain(const sx::Plan &p, uint8_t *dst, const uint8_t *src, cudaMemcpyKind kind, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    const size_t side = (size_t)p.side;
    for_each_copy_box(p, [&](int64_t a0, int64_t a1, int64_t b0, int64_t b1, int64_t w) {
        if (e != cudaSuccess) return;
        if (p.m == 2) {
            e = cudaMemcpy2DAsync(dst + (size_t)a0 * side, side, src + (size_t)a0 * side, side, (size_t)w,
                                  (size_t)(a1 - a0), kind, st);
            return;
        }
        cudaMemcpy3DParms c = {};
        c.srcPtr = make_cudaPitchedPtr(const_cast<uint8_t *>(src), side, side, side);
        c.dstPtr = make_cudaPitchedPtr(dst, side, side, side);
        c.srcPos = make_cudaPos(0, (size_t)b0, (size_t)a0);
        c.dstPos = c.srcPos;
        c.extent = make_cudaExtent((size_t)w, (size_t)(b1 - b0), (size_t)(a1 - a0));
        c.kind = kind;
        e = cudaMemcpy3DAsync(&c, st);
    });
    return e;
}

}  // namespace

extern "C" {

int simplex_map_create_ex(const simplex_map_params_t *params, simplex_map_t *out)
{
    if (!params || !out) return fail(SIMPLEX_EINVAL, "params and out must not be NULL");
    *out = nullptr;
    if (params->launch < 0 || params->launch > 3)
        return fail(SIMPLEX_EINVAL,
                    "params->launch must be 0 (automatic), 1 (grid), 2 (x-stream) or 3 (plane stream), got %d",
                    params->launch);
    const int64_t side = params->side ? params->side : params->n + 1;
    int band = params->band;
    if (band == 0) band = (params->m == 2 && params->r_inv == 2) ? kDefaultBand : 0;  // automatic
    if (band < 0) band = 0;                                   // single H2 grid
    sx::Plan p;
    if (params->layout != 0 && !(params->layout == 1 && params->m == 3 && params->beta == 2))
        return fail(SIMPLEX_EINVAL, "layout 1 (one block range per stack level) applies to m = 3, beta = 2 only "
                    "(got layout %d, m = %d, beta = %d)", params->layout, params->m, params->beta);
    int rc = build_plan(params->m, params->n, params->r_inv, params->beta, params->block, side, band, &p,
                        params->layout);
    if (rc == SIMPLEX_OK) {
        // automatic: the grid form (one CTA per block of the map, the paper's
        // model); the x-stream form on request (m = 3, block 32)
        const bool can_persist = p.m == 3 && p.rho == 32;
        if (params->launch == 2 && !can_persist)
            return fail(SIMPLEX_EUNSUPPORTED, "the x-stream automaton step exists for m = 3, block 32");
        if (params->launch == 3) {
            if (p.m != 3) return fail(SIMPLEX_EUNSUPPORTED, "the plane-stream automaton step exists for m = 3");
            sx::PlaneSched probe;
            if (!sx::plane_sched_build(p.n, sx::kMapBB, &probe))
                return fail(SIMPLEX_EUNSUPPORTED, "n = %lld needs more plane-stream segments or units than supported",
                            (long long)p.n);
        }
        p.persistent = params->launch == 2 ? 1 : (params->launch == 3 ? 2 : 0);
    }
    if (rc) return rc;
    simplex_map *map = new (std::nothrow) simplex_map();
    if (!map) return fail(SIMPLEX_ENOMEM, "host allocation failed");
    map->plan = p;
    map->r_inv = params->r_inv;
    *out = map;
    return SIMPLEX_OK;
}

int simplex_map_create_padded(int m, int64_t n, int r_inv, int beta, int block, int64_t side, simplex_map_t *out)
{
    const simplex_map_params_t prm = {m, r_inv, beta, block, n, side, 0, 0, 0};
    return simplex_map_create_ex(&prm, out);
}

int simplex_map_create(int m, int64_t n, int r_inv, int beta, int block, simplex_map_t *out)
{
    return simplex_map_create_padded(m, n, r_inv, beta, block, n + 1, out);
}

int simplex_map_destroy(simplex_map_t map)
{
    if (!map) return SIMPLEX_OK;
    for (auto &g : map->graphs) cudaGraphExecDestroy(g.exec);
    if (map->capture) cudaStreamDestroy(map->capture);
    if (map->queue) cudaFree(map->queue);
    for (auto *s : map->sched) delete s;
    delete map;
    return SIMPLEX_OK;
}

int simplex_map_info(simplex_map_t map, simplex_map_info_t *out)
{
    int rc;
    if ((rc = check_map(map))) return rc;
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    const sx::Plan &p = map->plan;
    std::memset(out, 0, sizeof *out);
    out->m = p.m;
    out->r_inv = map->r_inv;
    out->beta = p.beta;
    out->block = p.rho;
    out->n = p.n;
    out->side = p.side;
    out->N = p.N;
    out->log2N = p.logN;
    out->band = p.band;
    out->Ne = p.Ne;
    out->launch = p.persistent == 2 ? 3 : (p.persistent ? 2 : 1);
    out->layout = p.h3_exact;
    out->cells = binom((uint64_t)p.n + (uint64_t)p.m, p.m);
    out->useful_blocks = binom((uint64_t)(p.n / p.rho) + (uint64_t)p.m, p.m);
    out->host_copy_bytes = (p.m == 2 || p.m == 3) ? domain_copy_bytes(p) : 0;
    if (p.m == 3 && p.persistent == 2) {
        sx::PlaneSched sh, sb;
        if (sx::plane_sched_build(p.n, sx::kMapH, &sh)) out->plane_units = sh.units;
        if (sx::plane_sched_build(p.n, sx::kMapBB, &sb)) out->plane_units_bb = sb.units;
    }
    out->h_blocks = p.h_blocks;
    out->bb_blocks = p.bb_blocks;
    // Eq. generic-m with r = 1/2: (N^m - beta^log2 N) / (2^m - beta); the
    // r = 1/3 map of m = 2 lays three squares per split instead of one:
    // 3 (N3^2 - 3^L3) / (3^2 - 3)
    if (p.rinv == 3)
        out->h_set_blocks = 3 * ((uint64_t)p.N3 * (uint64_t)p.N3 - ipow(3, p.L3)) / 6;
    else
        out->h_set_blocks = (ipow((uint64_t)p.N, p.m) - ipow((uint64_t)p.beta, p.logN)) /
                            ((uint64_t(1) << p.m) - (uint64_t)p.beta);
    return SIMPLEX_OK;
}

int simplex_map_block(simplex_map_t map, int mode, uint64_t v, int32_t *coord, int *valid)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_mode(mode))) return rc;
    if (!coord || !valid) return fail(SIMPLEX_EINVAL, "coord and valid must not be NULL");
    const sx::Plan &p = map->plan;
    const uint64_t nb = sx::is_bb(mode) ? p.bb_blocks : p.h_blocks;
    if (v >= nb) return fail(SIMPLEX_EINVAL, "block index %llu out of range (%llu blocks)",
                             (unsigned long long)v, (unsigned long long)nb);
    int32_t X[sx::kMaxM] = {0, 0, 0, 0};
    bool ok = false;
    switch (p.m) {
    case 2: ok = sx::decode<2>(p, mode, v, X); break;
    case 3: ok = sx::decode<3>(p, mode, v, X); break;
    case 4: ok = sx::decode<4>(p, mode, v, X); break;
    }
    for (int i = 0; i < p.m; ++i) coord[i] = X[i];
    if (ok) {
        int64_t s = 0;
        for (int i = 0; i < p.m; ++i) s += X[i];
        ok = s * p.rho <= p.n;
    }
    *valid = ok ? 1 : 0;
    return SIMPLEX_OK;
}

int simplex_map_unit(simplex_map_t map, int mode, uint64_t w, int32_t *unit, int *valid)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_mode(mode))) return rc;
    if (!unit || !valid) return fail(SIMPLEX_EINVAL, "unit and valid must not be NULL");
    const sx::Plan &p = map->plan;
    if (!(p.m == 3 && p.persistent == 2)) return fail(SIMPLEX_EINVAL, "the map is not a plane-stream (launch 3) map");
    sx::PlaneSched s;
    if (!sx::plane_sched_build(p.n, mode, &s)) return fail(SIMPLEX_EUNSUPPORTED, "plane-stream schedule too large");
    if (w >= s.units)
        return fail(SIMPLEX_EINVAL, "unit index %llu out of range (%llu units)", (unsigned long long)w,
                    (unsigned long long)s.units);
    sx::PlaneUnit u;
    const bool ok = sx::plane_unit_decode(s, w, u);
    unit[0] = u.y0;
    unit[1] = u.x0;
    unit[2] = u.b;
    unit[3] = u.e;
    *valid = ok ? 1 : 0;
    return SIMPLEX_OK;
}

int simplex_write(simplex_map_t map, uint32_t *out, uint32_t seed, int mode, void *stream)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_mode(mode))) return rc;
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    if ((reinterpret_cast<uintptr_t>(out) & 3u) != 0) return fail(SIMPLEX_EINVAL, "out must be 4-byte aligned");
    const sx::Plan &p = map->plan;
    const bool vec = aligned16(out) && (p.side % 4 == 0);
    cudaError_t e = sx::launch_write(p, out, seed, mode, vec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "write launch");
    return SIMPLEX_OK;
}

int simplex_accum(simplex_map_t map, uint32_t *data, uint32_t add, int mode, void *stream)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_mode(mode))) return rc;
    if (!data) return fail(SIMPLEX_EINVAL, "data is NULL");
    if ((reinterpret_cast<uintptr_t>(data) & 3u) != 0) return fail(SIMPLEX_EINVAL, "data must be 4-byte aligned");
    const sx::Plan &p = map->plan;
    const bool vec = aligned16(data) && (p.side % 4 == 0);
    cudaError_t e = sx::launch_accum(p, data, add, mode, vec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "ACCUM launch");
    return SIMPLEX_OK;
}

int simplex_map_test(simplex_map_t map, unsigned long long *cells, int mode, void *stream)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_mode(mode))) return rc;
    const sx::Plan &p = map->plan;
    if (p.m * p.log_rho > 10)
        return fail(SIMPLEX_EINVAL, "the MAP test runs block^m threads per CUDA block: needs block^m <= 1024 "
                    "(m = %d, block = %d)", p.m, p.rho);
    cudaError_t e = sx::launch_map_test(p, mode, cells, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "MAP test launch");
    return SIMPLEX_OK;
}

int simplex_edm(simplex_map_t map, const float *points, int dim, float *out, int mode, void *stream)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_mode(mode))) return rc;
    const sx::Plan &p = map->plan;
    if (p.m != 2) return fail(SIMPLEX_EINVAL, "EDM is defined on the 2-simplex (map has m = %d)", p.m);
    if (!sx::edm_supports(p.rho)) return fail(SIMPLEX_EINVAL, "EDM needs block 16, 32 or 64 (got %d)", p.rho);
    if (dim < 1 || dim > 16) return fail(SIMPLEX_EINVAL, "dim must be in [1, 16] (got %d)", dim);
    if (!points || !out) return fail(SIMPLEX_EINVAL, "points and out must not be NULL");
    if ((reinterpret_cast<uintptr_t>(out) & 3u) != 0 || (reinterpret_cast<uintptr_t>(points) & 3u) != 0)
        return fail(SIMPLEX_EINVAL, "points and out must be 4-byte aligned");
    const bool vec = aligned16(out) && p.side % 4 == 0;
    cudaError_t e = sx::launch_edm(p, points, dim, out, mode, vec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "EDM launch");
    return SIMPLEX_OK;
}

int simplex_ca_init(simplex_map_t map, uint8_t *grid, uint32_t seed, uint32_t threshold,
                    unsigned long long *live, void *stream)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_ca_layout(map->plan, grid, "grid"))) return rc;
    cudaError_t e = sx::launch_ca_init(map->plan, grid, seed, threshold, live, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "init launch");
    return SIMPLEX_OK;
}

int simplex_ca_step(simplex_map_t map, const uint8_t *in, uint8_t *out, uint32_t birth, uint32_t survive,
                    unsigned long long *live, int mode, void *stream)
{
    int rc = check_step_args(map, in, out, mode);
    if (rc) return rc;
    const sx::Rule rule = make_rule(map->plan.m, birth, survive);
    return step_once(map, in, out, rule, live, mode, static_cast<cudaStream_t>(stream));
}

int simplex_ca_run(simplex_map_t map, uint8_t *a, uint8_t *b, int steps, uint32_t birth, uint32_t survive,
                   unsigned long long *live, int use_graph, int mode, void *stream)
{
    int rc = check_step_args(map, a, b, mode);
    if (rc) return rc;
    if (steps < 0) return fail(SIMPLEX_EINVAL, "steps must be >= 0 (got %d)", steps);
    const sx::Rule rule = make_rule(map->plan.m, birth, survive);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!use_graph) return enqueue_run(map, a, b, steps, rule, live, mode, st);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (map->device >= 0 && map->device != dev)
        return fail(SIMPLEX_EINVAL, "map was first used with graphs on device %d, now %d", map->device, dev);
    if (!map->capture) {
        e = cudaStreamCreateWithFlags(&map->capture, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
        map->device = dev;
    }
    e = map->plan.m == 2 ? sx::ca2_prepare(map->plan.rho) : sx::ca3_prepare(map->plan.rho);
    if (e == cudaSuccess && map->plan.m == 3 && map->plan.persistent == 2) e = sx::ca3_planes_prepare();
    if (e != cudaSuccess) return cuda_fail(e, "setting the kernel shared-memory limit");
    if ((rc = ensure_queue(map))) return rc;
    cudaGraphExec_t exec = nullptr;
    for (auto &g : map->graphs)
        if (g.a == a && g.b == b && g.steps == steps && g.birth == birth && g.survive == survive && g.live == live &&
            g.mode == mode)
            exec = g.exec;
    if (!exec) {
        e = cudaStreamBeginCapture(map->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        rc = enqueue_run(map, a, b, steps, rule, live, mode, map->capture);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(map->capture, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        if (map->graphs.size() >= 8) {
            cudaGraphExecDestroy(map->graphs.front().exec);
            map->graphs.erase(map->graphs.begin());
        }
        map->graphs.push_back(GraphEntry{a, b, steps, birth, survive, live, mode, exec});
    }
    e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return SIMPLEX_OK;
}

int simplex_ca_run_host(simplex_map_t map, const uint8_t *host_in, uint8_t *host_out, uint8_t *a, uint8_t *b,
                        int steps, uint32_t birth, uint32_t survive, unsigned long long *dev_live,
                        unsigned long long *host_live, int use_graph, int mode, void *stream)
{
    int rc;
    if ((rc = check_map(map))) return rc;
    if (!host_in || !host_out) return fail(SIMPLEX_EINVAL, "host_in and host_out must not be NULL");
    if (host_live && !dev_live) return fail(SIMPLEX_EINVAL, "host_live needs dev_live");
    const sx::Plan &p = map->plan;
    if ((rc = check_ca_layout(p, a, "a")) || (rc = check_ca_layout(p, b, "b"))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = copy_domain(p, a, host_in, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copying the domain of host_in to a");
    rc = simplex_ca_run(map, a, b, steps, birth, survive, dev_live, use_graph, mode, stream);
    if (rc) return rc;
    const uint8_t *fin = (steps % 2 == 0) ? a : b;
    e = copy_domain(p, host_out, fin, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "copying the domain of the final grid to host_out");
    if (host_live) {
        e = cudaMemcpyAsync(host_live, dev_live, sizeof(unsigned long long) * (size_t)(steps + 1),
                            cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(live -> host_live)");
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return SIMPLEX_OK;
}

int simplex_visit_count(simplex_map_t map, uint32_t *counts, int level, int mode, void *stream)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_mode(mode))) return rc;
    if (!counts) return fail(SIMPLEX_EINVAL, "counts is NULL");
    if (level != SIMPLEX_LEVEL_BLOCK && level != SIMPLEX_LEVEL_CELL)
        return fail(SIMPLEX_EINVAL, "level must be SIMPLEX_LEVEL_BLOCK or SIMPLEX_LEVEL_CELL (got %d)", level);
    cudaError_t e = sx::launch_visit(map->plan, counts, level, mode, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "visit-count launch");
    return SIMPLEX_OK;
}

int simplex_ca_digest(simplex_map_t map, const uint8_t *grid, unsigned long long *digest, unsigned long long *live,
                      void *stream)
{
    int rc;
    if ((rc = check_map(map)) || (rc = check_ca_layout(map->plan, grid, "grid"))) return rc;
    if (!digest) return fail(SIMPLEX_EINVAL, "digest is NULL");
    cudaError_t e = sx::launch_ca_count(map->plan, grid, live, static_cast<cudaStream_t>(stream), digest);
    if (e != cudaSuccess) return cuda_fail(e, "digest launch");
    return SIMPLEX_OK;
}

int simplex_device_status(uint32_t *out)
{
    if (!out) return fail(SIMPLEX_EINVAL, "out is NULL");
    uint32_t s2 = 0, s3 = 0;
    cudaError_t e = sx::ca2_read_status(&s2);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
    e = sx::ca3_read_status(&s3);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
    uint32_t s3p = 0;
    e = sx::ca3p_read_status(&s3p);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
    s3 |= s3p;
    uint32_t sb = 0;
    e = sx::batch_read_status(&sb);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status word");
    *out = s2 | s3 | sb;
    if (*out) return fail(SIMPLEX_ETIMEOUT, "a kernel gave up a bounded wait for its TMA load (status 0x%x)", *out);
    return SIMPLEX_OK;
}

int simplex_selftest_wait_timeout(uint64_t limit_ns, void *stream)
{
    if (limit_ns < 1000ull || limit_ns > 1000000000ull)
        return fail(SIMPLEX_EINVAL, "limit_ns must be in [1 us, 1 s] (got %llu)", (unsigned long long)limit_ns);
    cudaError_t e = sx::launch_wait_selftest(limit_ns, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
    return SIMPLEX_OK;
}

const char *simplex_last_error(void) { return g_last_error.c_str(); }

const char *simplex_version(void) { return "libsimplex 0.1 (sm_103a)"; }

}  // extern "C"
