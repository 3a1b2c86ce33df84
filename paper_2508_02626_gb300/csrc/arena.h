// arena.h -- first-fit suballocator over one device reservation.
//
// A pooled context reserves its whole HBM budget with one cudaMalloc and carves every tree,
// expansion and scratch array out of it.  Unlike cudaFree, returning a block never
// synchronises the device, so a serving loop can retire finished solves while others run.
// The arena works on byte offsets only (plain host code, no CUDA), blocks are 256-byte
// aligned, the lowest-addressed free block that fits is taken, and freed blocks merge with
// free neighbours.  Not thread-safe: the owning context serialises its calls.
#pragma once
#include <stddef.h>

#include <iterator>
#include <map>

namespace dafmm {

class OffsetArena {
public:
    static constexpr size_t kAlign = 256;

    explicit OffsetArena(size_t size = 0) { reset(size); }

    void reset(size_t size) {
        free_.clear();
        live_.clear();
        size_ = size / kAlign * kAlign;
        used_ = 0;
        if (size_) free_[0] = size_;
    }

    // A block of at least `bytes` (rounded up to kAlign; 0 counts as kAlign); false when no
    // free block is large enough.
    bool alloc(size_t bytes, size_t* off) {
        bytes = bytes == 0 ? kAlign : (bytes + kAlign - 1) / kAlign * kAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t o = it->first, sz = it->second;
            free_.erase(it);
            if (sz > bytes) free_[o + bytes] = sz - bytes;
            live_[o] = bytes;
            used_ += bytes;
            *off = o;
            return true;
        }
        return false;
    }

    // Returns the block at `off` to the free list; its size, or 0 when `off` is not a live block.
    size_t release(size_t off) {
        auto it = live_.find(off);
        if (it == live_.end()) return 0;
        const size_t sz = it->second;
        live_.erase(it);
        used_ -= sz;
        size_t o = off, s = sz;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && nx->first == off + sz) {
            s += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                o = pv->first;
                s += pv->second;
                free_.erase(pv);
            }
        }
        free_[o] = s;
        return sz;
    }

    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t live_blocks() const { return live_.size(); }
    size_t free_blocks() const { return free_.size(); }
    size_t largest_free() const {
        size_t m = 0;
        for (const auto& kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }

private:
    std::map<size_t, size_t> free_;  // offset -> size, disjoint, never adjacent
    std::map<size_t, size_t> live_;  // offset -> size
    size_t size_ = 0, used_ = 0;
};

}  // namespace dafmm
