// Host-side check of the serving loop's admission policy (csrc/serve_policy.h) on random
// queues: every stated rule is tested against a direct restatement.
#include <stdint.h>

#include <vector>

#include "serve_policy.h"

namespace {
uint64_t st = 1;
uint64_t rnd() {  // splitmix64
    uint64_t z = (st += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
}  // namespace

// 0 on success, else the failing trial * 10 + rule.
extern "C" int policy_check(int trials, unsigned long long seed) {
    st = seed;
    for (int t = 0; t < trials; ++t) {
        std::vector<dafmm::PendingRequest> q(rnd() % 12);
        for (auto& r : q) {
            r.cls = (int64_t)(rnd() % 3);
            r.n = (int64_t)(rnd() % 1000);
            r.bytes = (size_t)(rnd() % 500);
        }
        const size_t free_b = rnd() % 2000;
        const int mb = 1 + (int)(rnd() % 5);
        const int64_t mp = (int64_t)(rnd() % 3000);
        const std::vector<size_t> sel = dafmm::select_batch(q, free_b, mb, mp);
        // rule 1: empty exactly when the queue is empty or the head does not fit
        const bool expect_empty = q.empty() || q[0].bytes > free_b;
        if (sel.empty() != expect_empty) return t * 10 + 1;
        if (sel.empty()) continue;
        // rule 2: head first, indices increasing, one class, within max_batch
        if (sel[0] != 0 || (int)sel.size() > mb) return t * 10 + 2;
        size_t bytes = 0;
        int64_t parts = 0;
        for (size_t k = 0; k < sel.size(); ++k) {
            if (k && sel[k] <= sel[k - 1]) return t * 10 + 2;
            if (q[sel[k]].cls != q[0].cls) return t * 10 + 2;
            bytes += q[sel[k]].bytes;
            parts += q[sel[k]].n;
        }
        // rule 3: memory always fits; particles fit unless the head alone is taken
        if (bytes > free_b) return t * 10 + 3;
        if (sel.size() > 1 && parts > mp) return t * 10 + 3;
        // rule 4: no same-class request between selected ones was skipped, and the job
        // stopped for a reason (batch full, queue exhausted, or the next one did not fit)
        size_t next = 1;
        for (size_t k = 1; k < sel.size(); ++k) {
            for (size_t i = next; i < sel[k]; ++i)
                if (q[i].cls == q[0].cls) return t * 10 + 4;
            next = sel[k] + 1;
        }
        if ((int)sel.size() < mb) {
            for (size_t i = next; i < q.size(); ++i) {
                if (q[i].cls != q[0].cls) continue;
                if (parts + q[i].n <= mp && bytes + q[i].bytes <= free_b) return t * 10 + 4;
                break;
            }
        }
    }
    return 0;
}
