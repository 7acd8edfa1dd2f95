// First-fit placement of byte ranges inside one fixed span [0, size): the
// bookkeeping of the serving arena (the custom device memory pool of section
// 4.1.2), kept free of CUDA so that it builds and is tested on the host.
//
// Ranges are whole 256-byte granules.  alloc() takes the lowest free range
// that fits; release() returns a range and merges it with free neighbours, so
// the free list never holds two adjacent ranges.  Not thread-safe: the owner
// locks.
#pragma once

#include <cstddef>
#include <map>

namespace jgb {

class FirstFit {
 public:
  static constexpr size_t kGranule = 256;

  static size_t round_up(size_t n) { return (n + kGranule - 1) & ~(kGranule - 1); }

  // Starts with the whole span free; size is rounded down to whole granules.
  void reset(size_t size) {
    size_ = size & ~(kGranule - 1);
    in_use_ = 0;
    free_.clear();
    used_.clear();
    if (size_) free_[0] = size_;
  }

  // Offset of a new range of at least n bytes, or npos when no free range
  // fits (n = 0 takes one granule).
  size_t alloc(size_t n) {
    n = round_up(n ? n : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const size_t off = it->first, sz = it->second;
      free_.erase(it);
      if (sz > n) free_[off + n] = sz - n;
      used_[off] = n;
      in_use_ += n;
      return off;
    }
    return npos;
  }

  // Returns the range that starts at off; false (and no change) when no
  // range starts there.
  bool release(size_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return false;
    size_t n = u->second, start = off;
    used_.erase(u);
    in_use_ -= n;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && next->first == off + n) {
      n += next->second;
      free_.erase(next);
    }
    auto prev = free_.lower_bound(off);
    if (prev != free_.begin()) {
      --prev;
      if (prev->first + prev->second == off) {
        start = prev->first;
        n += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = n;
    return true;
  }

  size_t size() const { return size_; }
  size_t in_use() const { return in_use_; }
  const std::map<size_t, size_t>& free_ranges() const { return free_; }
  const std::map<size_t, size_t>& used_ranges() const { return used_; }

  static constexpr size_t npos = ~(size_t)0;

 private:
  size_t size_ = 0, in_use_ = 0;
  std::map<size_t, size_t> free_, used_;  // offset -> bytes
};

}  // namespace jgb
