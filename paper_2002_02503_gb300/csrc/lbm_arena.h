// lbm_arena.h -- first-fit allocator of a pool's arena: offsets into one caller-owned
// device region, with a free list of (offset, size) runs kept coalesced, so that every run in
// it is a maximal free run and a release next to free space merges with it.  Host-only code
// (no CUDA); the pool serialises its calls.
#pragma once

#include <stddef.h>

#include <iterator>
#include <map>

namespace lbm {

struct Arena {
    char *base = nullptr;
    size_t bytes = 0;
    std::map<size_t, size_t> free_;  // offset -> size, coalesced

    void init(char *b, size_t n) {
        base = b;
        bytes = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    // The lowest free run of at least n bytes; false if none.
    bool alloc(size_t n, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t roff = it->first + n;
                free_.erase(it);
                if (rest) free_[roff] = rest;
                return true;
            }
        }
        return false;
    }
    // Returns [off, off + n), which alloc handed out, merging it with free neighbours.
    void release(size_t off, size_t n) {
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
    size_t free_bytes() const {
        size_t s = 0;
        for (auto &kv : free_) s += kv.second;
        return s;
    }
};

}  // namespace lbm
