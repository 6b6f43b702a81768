/*
 * First-fit allocator of unit ranges, the admission bookkeeping of the
 * runtime's heap pool (units: 256 KiB slabs) and ring pool (units: slots).
 * Plain C++ (no CUDA), so the CPU tests exercise it directly.
 */
#ifndef GF_RANGE_ALLOC_H
#define GF_RANGE_ALLOC_H
#include <stdint.h>
#include <iterator>
#include <map>

/* Free ranges of [0, total), kept disjoint and never touching (neighbours
 * merge on release).  alloc takes the first range long enough; release of a
 * range that is not allocated is the caller's error.  Not thread-safe: the
 * runtime holds its admission lock around every call. */
struct RangeAlloc {
    uint64_t total = 0;
    std::map<uint64_t, uint64_t> free_;   /* start -> length, disjoint, not touching */
    void init(uint64_t n)
    {
        total = n;
        free_.clear();
        if (n)
            free_[0] = n;
    }
    bool alloc(uint64_t n, uint64_t *out)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n)
                continue;
            const uint64_t a = it->first, l = it->second;
            free_.erase(it);
            if (l > n)
                free_[a + n] = l - n;
            *out = a;
            return true;
        }
        return false;
    }
    void release(uint64_t a, uint64_t n)
    {
        if (!n)
            return;
        auto it = free_.emplace(a, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && a + n == nx->first) {
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

#endif
