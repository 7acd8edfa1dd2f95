// Dealing the lines of a set of blocks out to warps in equal runs: the work
// items of the 2D FP64 march kernels under option march 3 (engine.cu).
// Host-only C++, no CUDA, so that it is checked on the CPU
// (tests/native/deal_runs_check.cpp).
#pragma once

#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

namespace jgb {

// A run's piece inside one block: lines y0 .. y0 + n - 1 of block `block`.
struct RunPiece {
  int block;
  int y0;
  int n;
};

// blocks: (block index, lines) in table order.  The lines, counted in steps of
// `unit` lines (a block's last step may be shorter), are dealt out in equal
// runs, one per warp, in block order: `target` warps (as many as the kernel
// keeps resident), but no fewer steps per run than min_lines takes, and more
// warps only where a run would exceed max_lines.  A run that crosses a block
// boundary becomes two pieces (more for blocks shorter than a run).  Warp w
// computes pieces start[w] .. start[w + 1] - 1 (indices into `pieces`, which
// is appended to; start gets one entry per warp plus the end).
inline void deal_runs(const std::vector<std::pair<int, int>>& blocks, int64_t target, int unit, int min_lines,
                      int max_lines, std::vector<RunPiece>& pieces, std::vector<int>& start) {
  unit = std::max(unit, 1);
  int64_t total = 0;  // steps over all blocks
  for (const auto& b : blocks) total += (std::max(b.second, 0) + unit - 1) / unit;
  if (total == 0) return;
  const int64_t smax = std::max(max_lines / unit, 1);
  const int64_t smin = std::max((min_lines + unit - 1) / unit, 1);
  const int64_t nw = std::max<int64_t>(std::min<int64_t>(std::max<int64_t>(target, 1), (total + smin - 1) / smin),
                                       (total + smax - 1) / smax);
  size_t bk = 0;
  int64_t used = 0;  // steps of blocks[bk] already dealt
  for (int64_t w = 0; w < nw; ++w) {
    start.push_back((int)pieces.size());
    int64_t need = (w + 1) * total / nw - w * total / nw;
    while (need > 0 && bk < blocks.size()) {
      const int lines = std::max(blocks[bk].second, 0);
      const int64_t steps = (lines + unit - 1) / unit;
      if (steps == 0) {
        ++bk;
        continue;
      }
      const int64_t take = std::min(need, steps - used);
      const int a = (int)(used * unit), e = (int)std::min<int64_t>((used + take) * unit, lines);
      pieces.push_back(RunPiece{blocks[bk].first, a, e - a});
      used += take;
      need -= take;
      if (used == steps) {
        ++bk;
        used = 0;
      }
    }
  }
  start.push_back((int)pieces.size());
}

}  // namespace jgb
