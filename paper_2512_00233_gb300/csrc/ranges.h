// First-fit allocator of [0, cap) ranges with coalescing on free: the vertex
// and entry ranges of the batch engine's device arena and the ranges of its
// page-locked staging pool.  Host-only C++ (no CUDA), not thread-safe: the
// engine calls it under its mutex.
#pragma once

#include <algorithm>
#include <iterator>
#include <map>

namespace kc {

class Ranges {
  public:
    // Everything free again; the peak is kept (it is a high-water mark).
    void reset(long long cap) {
        free_.clear();
        if (cap > 0) free_[0] = cap;
        cap_ = cap;
        used_ = 0;
    }
    long long take(long long len) {
        if (len <= 0) return 0;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                const long long at = it->first, rest = it->second - len;
                free_.erase(it);
                if (rest > 0) free_[at + len] = rest;
                used_ += len;
                peak_ = std::max(peak_, used_);
                return at;
            }
        }
        return -1;
    }
    void give(long long at, long long len) {
        if (len <= 0) return;
        used_ -= len;
        auto next = free_.lower_bound(at);
        if (next != free_.end() && at + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == at) {
                prev->second += len;
                return;
            }
        }
        free_[at] = len;
    }
    long long largest() const {
        long long b = 0;
        for (auto& kv : free_) b = std::max(b, kv.second);
        return b;
    }
    long long peak() const { return peak_; }
    long long used() const { return used_; }

  private:
    std::map<long long, long long> free_;
    long long cap_ = 0, used_ = 0, peak_ = 0;
};

}  // namespace kc
