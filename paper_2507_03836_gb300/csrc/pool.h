// First-fit allocator over one device range (host bookkeeping only), used by the serving loop to carve
// per-request scratch out of its budget.  Plain C++ with no CUDA dependency, so it also compiles into
// host-only tests.  Sizes are rounded up to 256 bytes; freed neighbours coalesce.
#pragma once
#include <stdint.h>

#include <iterator>
#include <map>

namespace fh {

struct Pool {
    char* base = nullptr;
    uint64_t bytes = 0, used = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> size
    void init(char* b, uint64_t n) {
        base = b; bytes = n; used = 0;
        free_.clear();
        if (n) free_[0] = n;
    }
    bool alloc(uint64_t n, uint64_t* off) {
        n = (n + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                uint64_t rest = it->second - n, o = it->first + n;
                free_.erase(it);
                if (rest) free_[o] = rest;
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        n = (n + 255) / 256 * 256;
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
};

}  // namespace fh
