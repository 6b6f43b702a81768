/* CPU check of the admission range allocator (host/range_alloc.h) against a
 * brute-force model: a bitmap of units and the first-fit rule written out
 * unit by unit.  Random alloc / release sequences over pools of several
 * sizes; every answer (granted or refused, and the start) must match the
 * model, and the free list must stay disjoint, sorted and merged. */
#include <stdio.h>
#include <stdlib.h>
#include <vector>

#include "host/range_alloc.h"

static uint64_t rng = 88172645463325252ull;
static uint64_t next_u()
{
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return rng;
}

/* first start s with units [s, s + n) all free, or -1 */
static long long model_first_fit(const std::vector<char> &used, uint64_t n)
{
    const uint64_t T = used.size();
    for (uint64_t s = 0; s + n <= T; s++) {
        uint64_t k = 0;
        while (k < n && !used[s + k])
            k++;
        if (k == n)
            return (long long)s;
    }
    return -1;
}

int main()
{
    int checks = 0;
    for (uint64_t total : {1ull, 7ull, 64ull, 1000ull, 4096ull}) {
        RangeAlloc ra;
        ra.init(total);
        std::vector<char> used(total, 0);
        std::vector<std::pair<uint64_t, uint64_t>> live;
        for (int step = 0; step < 20000; step++) {
            if (!live.empty() && (next_u() % 3 == 0)) {
                const size_t k = next_u() % live.size();
                const auto r = live[k];
                live[k] = live.back();
                live.pop_back();
                ra.release(r.first, r.second);
                for (uint64_t u = r.first; u < r.first + r.second; u++)
                    used[u] = 0;
            } else {
                const uint64_t n = 1 + next_u() % (total < 64 ? total : total / 8);
                uint64_t got = ~0ull;
                const bool ok = ra.alloc(n, &got);
                const long long want = model_first_fit(used, n);
                if (ok != (want >= 0) || (ok && (long long)got != want)) {
                    printf("FAIL total %llu step %d n %llu: got %d/%llu want %lld\n", (unsigned long long)total, step,
                           (unsigned long long)n, (int)ok, (unsigned long long)got, want);
                    return 1;
                }
                if (ok) {
                    live.push_back({got, n});
                    for (uint64_t u = got; u < got + n; u++)
                        used[u] = 1;
                }
            }
            /* the free list: sorted, disjoint, not touching, and exactly the model's free units */
            uint64_t prev_end = 0, free_units = 0;
            bool first = true;
            for (const auto &f : ra.free_) {
                if (f.second == 0 || (!first && f.first <= prev_end) || f.first + f.second > total) {
                    printf("FAIL total %llu step %d: bad free list\n", (unsigned long long)total, step);
                    return 1;
                }
                for (uint64_t u = f.first; u < f.first + f.second; u++)
                    if (used[u]) {
                        printf("FAIL total %llu step %d: unit %llu free and used\n", (unsigned long long)total, step,
                               (unsigned long long)u);
                        return 1;
                    }
                free_units += f.second;
                prev_end = f.first + f.second;
                first = false;
            }
            uint64_t model_free = 0;
            for (char c : used)
                model_free += !c;
            if (free_units != model_free) {
                printf("FAIL total %llu step %d: %llu free units, model %llu\n", (unsigned long long)total, step,
                       (unsigned long long)free_units, (unsigned long long)model_free);
                return 1;
            }
            checks++;
        }
        for (const auto &r : live)
            ra.release(r.first, r.second);
        if (ra.free_.size() != 1 || ra.free_.begin()->first != 0 || ra.free_.begin()->second != total) {
            printf("FAIL total %llu: pool not whole after releasing everything\n", (unsigned long long)total);
            return 1;
        }
    }
    printf("OK %d checks\n", checks);
    return 0;
}
