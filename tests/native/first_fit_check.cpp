// Check of the serving arena's first-fit placement (first_fit.h) against a
// brute-force model: one owner entry per 256-byte granule, first fit found by
// scanning from offset 0.  Random sequences of allocations (including zero
// and span-sized requests) and releases (including offsets that were never
// returned) must give the same offsets as the model, and after every step the
// free list must be exactly the model's free granules as maximal runs.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "first_fit.h"

using jgb::FirstFit;

static long failures = 0;

static void fail(const char* what, long step) {
  if (failures++ < 10) std::printf("mismatch at step %ld: %s\n", step, what);
}

struct Model {
  std::vector<long> owner;  // per granule: id of the range holding it, -1 free
  long next_id = 0;
  explicit Model(size_t granules) : owner(granules, -1) {}
  size_t alloc(size_t n) {
    const size_t k = (n ? n : 1) / FirstFit::kGranule + (((n ? n : 1) % FirstFit::kGranule) != 0);
    for (size_t s = 0; s + k <= owner.size(); ++s) {
      size_t j = 0;
      while (j < k && owner[s + j] < 0) ++j;
      if (j == k) {
        for (size_t q = 0; q < k; ++q) owner[s + q] = next_id;
        ++next_id;
        return s * FirstFit::kGranule;
      }
      s += j;  // skip past the granule that blocked this start
    }
    return FirstFit::npos;
  }
  bool release(size_t off) {
    if (off % FirstFit::kGranule) return false;
    const size_t g = off / FirstFit::kGranule;
    if (g >= owner.size() || owner[g] < 0) return false;
    if (g > 0 && owner[g - 1] == owner[g]) return false;  // not the start of its range
    const long id = owner[g];
    for (size_t q = g; q < owner.size() && owner[q] == id; ++q) owner[q] = -1;
    return true;
  }
};

static void compare(const FirstFit& ff, const Model& m, long step) {
  // free ranges: maximal runs of free granules, in order
  std::vector<std::pair<size_t, size_t>> runs;
  size_t in_use = 0;
  for (size_t g = 0; g < m.owner.size();) {
    if (m.owner[g] >= 0) {
      in_use += FirstFit::kGranule;
      ++g;
      continue;
    }
    size_t e = g;
    while (e < m.owner.size() && m.owner[e] < 0) ++e;
    runs.push_back({g * FirstFit::kGranule, (e - g) * FirstFit::kGranule});
    g = e;
  }
  if (ff.in_use() != in_use) fail("bytes in use", step);
  if (ff.free_ranges().size() != runs.size()) {
    fail("number of free ranges", step);
    return;
  }
  size_t i = 0;
  for (const auto& kv : ff.free_ranges()) {
    if (kv.first != runs[i].first || kv.second != runs[i].second) fail("free range", step);
    ++i;
  }
  size_t used = 0;
  for (const auto& kv : ff.used_ranges()) used += kv.second;
  if (used != in_use) fail("used ranges", step);
}

int main(int argc, char** argv) {
  const long steps = argc > 1 ? std::atol(argv[1]) : 200000;
  std::mt19937_64 g(20230302);
  long ops = 0, misses = 0;
  for (size_t granules : {1ul, 2ul, 7ul, 64ul, 1000ul}) {
    FirstFit ff;
    ff.reset(granules * FirstFit::kGranule + 100);  // a ragged tail is dropped
    Model m(granules);
    compare(ff, m, -1);
    std::vector<size_t> live;
    for (long s = 0; s < steps / 5; ++s) {
      const unsigned r = (unsigned)(g() % 100);
      if (r < 55 || live.empty()) {
        size_t n;
        const unsigned kind = (unsigned)(g() % 10);
        if (kind == 0) n = 0;
        else if (kind == 1) n = granules * FirstFit::kGranule;               // the whole span
        else if (kind == 2) n = (size_t)(g() % (granules * FirstFit::kGranule + 512));
        else n = 1 + (size_t)(g() % (4 * FirstFit::kGranule));
        const size_t a = ff.alloc(n), b = m.alloc(n);
        if (a != b) fail("alloc offset", s);
        if (a == FirstFit::npos) ++misses;
        else live.push_back(a);
      } else if (r < 95) {
        const size_t k = (size_t)(g() % live.size());
        const size_t off = live[k];
        live[k] = live.back();
        live.pop_back();
        const bool a = ff.release(off), b = m.release(off);
        if (!a || !b) fail("release of a live range", s);
      } else {
        // an offset that was never handed out (or is already free) changes nothing
        const size_t off = (size_t)(g() % (granules * FirstFit::kGranule + 1024));
        bool held = false;
        for (size_t o : live) held |= o == off;
        if (!held) {
          if (ff.release(off)) fail("release of a foreign offset succeeded", s);
        }
      }
      ++ops;
      compare(ff, m, s);
    }
  }
  std::printf("ops %ld misses %ld failures %ld\n", ops, misses, failures);
  return failures ? 1 : 0;
}
