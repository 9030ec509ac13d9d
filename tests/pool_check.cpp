// pool_check.cpp -- randomized check of the serving engine's grid-pool
// allocator (paper_2208_11617_gb300/csrc/pool.h) against a brute-force model:
// the live allocations as a list of ranges.  Built and run by test_pool.py.
//
// After every operation: offsets are 256-byte aligned and inside the pool,
// no two live ranges overlap, used() is the sum of the live (rounded) sizes
// and peak() its maximum so far; an allocation succeeds exactly when some
// gap between live ranges holds it, and then at the lowest such gap (first
// fit); after everything is released one allocation of the whole pool fits
// (the free ranges coalesced).  Exit status 0 = all checks held.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <random>
#include <vector>

#include "../paper_2208_11617_gb300/csrc/pool.h"

struct Live {
    uint64_t off, bytes;  // bytes rounded up to 256
};

static int fails = 0;
#define CHECK(c, ...)                                  \
    do {                                               \
        if (!(c)) {                                    \
            fputs("check failed: " #c " -- ", stderr);   \
            fprintf(stderr, __VA_ARGS__);              \
            fprintf(stderr, "\n");                     \
            if (++fails > 10) exit(1);                 \
        }                                              \
    } while (0)

static uint64_t round256(uint64_t x) { return (x + 255) / 256 * 256; }

// lowest offset of a gap of at least `need` bytes among the live ranges in
// [0, size), or UINT64_MAX
static uint64_t first_fit(std::vector<Live> live, uint64_t size, uint64_t need)
{
    std::sort(live.begin(), live.end(), [](const Live &a, const Live &b) { return a.off < b.off; });
    uint64_t at = 0;
    for (const Live &l : live) {
        if (l.off >= at && l.off - at >= need) return at;
        at = std::max(at, l.off + l.bytes);
    }
    return size >= at && size - at >= need ? at : UINT64_MAX;
}

static void run(uint64_t size, uint64_t max_req, int ops, uint32_t seed)
{
    std::mt19937_64 rng(seed);
    sxh::FreeList pool;
    pool.reset(size);
    std::vector<Live> live;
    uint64_t used = 0, peak = 0;
    for (int op = 0; op < ops; ++op) {
        const bool do_alloc = live.empty() || (rng() % 100) < 55;
        if (do_alloc) {
            const uint64_t req = 1 + rng() % max_req;
            const uint64_t need = round256(req);
            const uint64_t want = first_fit(live, size, need);
            uint64_t off = 0;
            const bool ok = pool.alloc(req, &off);
            CHECK(ok == (want != UINT64_MAX), "seed %u op %d: alloc(%llu) returned %d", seed, op,
                  (unsigned long long)req, (int)ok);
            if (ok) {
                CHECK(off == want, "seed %u op %d: offset %llu, first fit %llu", seed, op, (unsigned long long)off,
                      (unsigned long long)want);
                CHECK(off % 256 == 0 && off + need <= size, "seed %u op %d: range %llu + %llu outside the pool", seed,
                      op, (unsigned long long)off, (unsigned long long)need);
                for (const Live &l : live)
                    CHECK(off + need <= l.off || l.off + l.bytes <= off, "seed %u op %d: overlap", seed, op);
                live.push_back({off, need});
                used += need;
                peak = std::max(peak, used);
            }
        } else {
            const size_t k = rng() % live.size();
            // release with the size the caller asked for (any value that rounds the same)
            pool.release(live[k].off, live[k].bytes - (rng() % 256));
            used -= live[k].bytes;
            live[k] = live.back();
            live.pop_back();
        }
        CHECK(pool.used() == used, "seed %u op %d: used %llu, expected %llu", seed, op,
              (unsigned long long)pool.used(), (unsigned long long)used);
        CHECK(pool.peak() == peak, "seed %u op %d: peak", seed, op);
    }
    for (const Live &l : live) pool.release(l.off, l.bytes);
    CHECK(pool.used() == 0, "seed %u: used after releasing everything", seed);
    uint64_t off = 1;
    const uint64_t whole = size / 256 * 256;
    CHECK(pool.alloc(whole, &off) && off == 0, "seed %u: the whole pool does not fit after releasing all", seed);
}

int main()
{
    // pools of a few requests (often full) and of many, sizes not multiples of 256
    const uint64_t sizes[] = {4096, 1 << 20, (1 << 20) + 100, 64ull << 20};
    const uint64_t reqs[] = {1000, 70000, 300000, 4ull << 20};
    for (int i = 0; i < 4; ++i)
        for (uint32_t seed = 1; seed <= 6; ++seed) run(sizes[i], reqs[i], 3000, seed * 7919 + i);
    if (fails) return 1;
    printf("ok\n");
    return 0;
}
