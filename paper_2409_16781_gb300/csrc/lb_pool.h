// First-fit byte-range allocator with coalescing (host code): the batch
// pool's bookkeeping of which parts of its device buffer hold slots.  Every
// request is rounded up to ALIGN bytes; offsets are multiples of ALIGN.
// Header-only and free of CUDA, so that it is checked on the CPU against a
// brute-force model of the pool.
#pragma once
#include <cstddef>
#include <iterator>
#include <map>

namespace lbgb {

template <size_t ALIGN>
class Pool {
   public:
    static size_t round_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

    // The pool [0, size); size a multiple of ALIGN.  Forgets every allocation.
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
    }
    // Lowest offset of a free range that holds round_up(bytes); false if none.
    bool alloc(size_t bytes, size_t* off) {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    // Return [off, off + round_up(bytes)), merging it with free neighbours.
    void release(size_t off, size_t bytes) {
        bytes = round_up(bytes);
        auto it = free_.emplace(off, bytes).first;
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
    size_t free_bytes() const {
        size_t s = 0;
        for (auto& kv : free_) s += kv.second;
        return s;
    }
    size_t free_ranges() const { return free_.size(); }
    size_t size() const { return size_; }

   private:
    std::map<size_t, size_t> free_;  // offset -> length of each free range
    size_t size_ = 0;
};

}  // namespace lbgb
