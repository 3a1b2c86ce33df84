// serve_policy.h -- which queued requests the serving loop admits next (plain host code).
//
// Requests wait in arrival order.  When a slot (a CUDA stream) is free, the loop forms one
// job -- a forest solved by one build and one evaluation -- from the queue:
//   * the job takes the class (expansion order, precision, leaf size) of the oldest request;
//   * it then takes, oldest first, further requests of that class while the job holds fewer
//     than max_batch requests and at most max_particles particles, and while the summed
//     device-memory estimates fit in free_bytes; it stops at the first request of the class
//     that does not fit, so that no request of a class overtakes an older one of the same
//     class; requests of other classes are skipped and keep their places;
//   * the oldest request is always taken when its own estimate fits, even if it alone holds
//     more than max_particles particles;
//   * when the oldest request does not fit, nothing is admitted: the loop waits for running
//     jobs to return memory (and fails the request when nothing runs and it still does not
//     fit the empty pool).
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <vector>

namespace dafmm {

struct PendingRequest {
    int64_t cls;    // order, precision and leaf size packed into one key
    int64_t n;      // particles
    size_t bytes;   // device-memory estimate of solving it
};

// Indices into `queue` (oldest first) of the next job; empty when the oldest does not fit.
inline std::vector<size_t> select_batch(const std::vector<PendingRequest>& queue, size_t free_bytes, int max_batch,
                                        int64_t max_particles) {
    std::vector<size_t> out;
    if (queue.empty() || max_batch < 1) return out;
    const PendingRequest& head = queue[0];
    if (head.bytes > free_bytes) return out;
    out.push_back(0);
    size_t bytes = head.bytes;
    int64_t parts = head.n;
    for (size_t i = 1; i < queue.size() && (int)out.size() < max_batch; ++i) {
        const PendingRequest& r = queue[i];
        if (r.cls != head.cls) continue;
        if (parts + r.n > max_particles || bytes + r.bytes > free_bytes) break;
        out.push_back(i);
        bytes += r.bytes;
        parts += r.n;
    }
    return out;
}

}  // namespace dafmm
