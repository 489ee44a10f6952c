// range_alloc.h -- first-fit allocator of contiguous ranges of state-pool
// slots, used by the serving loop to place admitted jobs.  Host code only
// (no CUDA), so it is also compiled on its own by a CPU test.
#pragma once

#include <cstdint>
#include <iterator>
#include <map>

namespace nb {

// Free ranges are kept as start -> length, non-overlapping and coalesced
// (no two free ranges touch).  alloc takes the lowest-addressed free range
// that fits; release returns a range and merges it with free neighbours.
struct RangeAlloc {
    std::map<int64_t, int64_t> free_;     // start -> length
    explicit RangeAlloc(int64_t cap = 0) { if (cap > 0) free_[0] = cap; }
    // start of a range of n slots, or -1 when no free range holds n
    int64_t alloc(int64_t n)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                const int64_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > n) free_[off + n] = len - n;
                return off;
            }
        return -1;
    }
    // give back [off, off + n), a range alloc returned and not yet released
    void release(int64_t off, int64_t n)
    {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace nb
