// Host-side check of the device arena's suballocator (csrc/arena.h) against a brute-force
// model: a map of 256-byte units, first fit by address, and maximal free runs.
#include <stdint.h>
#include <stdio.h>

#include <map>
#include <vector>

#include "arena.h"

namespace {

uint64_t rng_state = 0x9e3779b97f4a7c15ull;
uint64_t next_u64() {  // splitmix64
    uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

// Returns 0 on success, else the failing step (>0).
extern "C" int arena_check(int units, int steps, unsigned long long seed) {
    rng_state = seed;
    const size_t A = dafmm::OffsetArena::kAlign;
    dafmm::OffsetArena a((size_t)units * A + 17);  // a ragged size is rounded down
    if (a.size() != (size_t)units * A) return 1;
    std::vector<int> owner(units, -1);  // model: unit -> live block id
    std::map<int, std::pair<size_t, size_t>> live;  // id -> (offset, bytes)
    int next_id = 0;
    for (int s = 0; s < steps; ++s) {
        const bool do_alloc = live.empty() || (next_u64() % 100) < 55;
        if (do_alloc) {
            const size_t k = (size_t)(next_u64() % (size_t)(units / 4 + 1));
            const size_t req = k ? k * A - (next_u64() % 3) * 7 : (next_u64() % 2) * 5;
            const size_t need = req == 0 ? 1 : (req + A - 1) / A;  // units
            // model first fit
            long fit = -1;
            for (int u = 0, run = 0; u < units; ++u) {
                run = owner[u] < 0 ? run + 1 : 0;
                if ((size_t)run == need) {
                    fit = u - (long)need + 1;
                    break;
                }
            }
            size_t off = 0;
            const bool ok = a.alloc(req, &off);
            if (ok != (fit >= 0)) return 1000000 + s;
            if (!ok) continue;
            if (off != (size_t)fit * A) return 2000000 + s;
            for (size_t u = 0; u < need; ++u) owner[fit + u] = next_id;
            live[next_id++] = {off, need * A};
        } else {
            auto it = live.begin();
            std::advance(it, (long)(next_u64() % live.size()));
            const size_t got = a.release(it->second.first);
            if (got != it->second.second) return 3000000 + s;
            for (size_t u = 0; u < got / A; ++u) owner[it->second.first / A + u] = -1;
            live.erase(it);
            if (a.release(12345 * A + 1) != 0) return 4000000 + s;  // not a live block
        }
        // invariants: used bytes, number of maximal free runs, largest free run
        size_t used = 0, runs = 0, largest = 0, run = 0;
        for (int u = 0; u < units; ++u) {
            if (owner[u] >= 0) {
                used += A;
                run = 0;
            } else {
                if (run == 0) ++runs;
                ++run;
                largest = run > largest ? run : largest;
            }
        }
        if (a.used() != used || a.free_blocks() != runs || a.largest_free() != largest * A ||
            a.live_blocks() != live.size())
            return 5000000 + s;
    }
    return 0;
}
