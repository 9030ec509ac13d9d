// pool.h -- the serving engine's allocator for the grids of resident jobs
// (host bookkeeping only; the pool itself is a range of the device arena).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <iterator>
#include <map>

namespace sxh {

// First-fit allocator over the grid pool [0, size), 256-byte granules; free
// ranges are coalesced on release.
class FreeList {
  public:
    void reset(uint64_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
        used_ = 0;
        peak_ = 0;
    }
    bool alloc(uint64_t bytes, uint64_t *off)
    {
        bytes = granule_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        return false;
    }
    void release(uint64_t off, uint64_t bytes)
    {
        bytes = granule_up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    uint64_t used() const { return used_; }
    uint64_t peak() const { return peak_; }

  private:
    static uint64_t granule_up(uint64_t x) { return (x + 255) / 256 * 256; }
    std::map<uint64_t, uint64_t> free_;  // free ranges: offset -> bytes
    uint64_t size_ = 0, used_ = 0, peak_ = 0;
};

}  // namespace sxh
