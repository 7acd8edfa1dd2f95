// Check of the dealing of lines to warps (deal_runs.h) against its contract on
// random block lists: every line of every block covered once, in block order,
// by pieces inside one block each, starting on a step boundary; warps in the
// stated count; every warp's run the same number of steps as the others to
// within one, and no run longer than the longest allowed.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "deal_runs.h"

static long failures = 0;

static void fail(const char* what, long trial) {
  if (failures++ < 10) std::printf("trial %ld: %s\n", trial, what);
}

int main(int argc, char** argv) {
  const long trials = argc > 1 ? std::atol(argv[1]) : 20000;
  std::mt19937_64 rng(2311);
  for (long trial = 0; trial < trials; ++trial) {
    const int nb = 1 + (int)(rng() % (trial % 7 == 0 ? 300 : 12));
    std::vector<std::pair<int, int>> blocks;
    for (int b = 0; b < nb; ++b) {
      const int kind = (int)(rng() % 4);
      const int lines = kind == 0 ? 1 + (int)(rng() % 8) : kind == 1 ? 1 + (int)(rng() % 700) : 512;
      blocks.push_back({3 * b + 1, lines});
    }
    const int unit = (rng() & 1) ? 1 : 8;
    const int64_t target = 1 + (int64_t)(rng() % 5000);
    const int min_lines = 8, max_lines = 64;
    std::vector<jgb::RunPiece> pieces;
    std::vector<int> start;
    jgb::deal_runs(blocks, target, unit, min_lines, max_lines, pieces, start);

    int64_t total = 0;
    for (const auto& b : blocks) total += (b.second + unit - 1) / unit;
    const int64_t smax = max_lines / unit, smin = (min_lines + unit - 1) / unit;
    int64_t nw = std::min<int64_t>(target, (total + smin - 1) / smin);
    nw = std::max<int64_t>(nw, (total + smax - 1) / smax);
    if ((int64_t)start.size() != nw + 1) {
      fail("warp count", trial);
      continue;
    }
    if (start.front() != 0 || start.back() != (int)pieces.size()) fail("start bounds", trial);
    // coverage in block order
    size_t bk = 0;
    int next = 0;  // next line expected in blocks[bk]
    for (const auto& q : pieces) {
      while (bk < blocks.size() && next == blocks[bk].second) {
        ++bk;
        next = 0;
      }
      if (bk >= blocks.size()) {
        fail("piece past the last block", trial);
        break;
      }
      if (q.block != blocks[bk].first) fail("piece out of block order", trial);
      if (q.y0 != next) fail("gap or overlap", trial);
      if (q.n < 1 || q.y0 + q.n > blocks[bk].second) fail("piece outside its block", trial);
      if (q.y0 % unit != 0) fail("piece not on a step boundary", trial);
      next = q.y0 + q.n;
    }
    if (!(bk == blocks.size() - 1 && next == blocks.back().second)) fail("lines left over", trial);
    // equal runs
    int64_t lo = -1, hi = -1;
    for (int64_t w = 0; w < nw; ++w) {
      int64_t steps = 0, lines = 0;
      for (int k = start[w]; k < start[w + 1]; ++k) {
        if (k < start[w] || k >= (int)pieces.size()) {
          fail("start order", trial);
          break;
        }
        steps += (pieces[k].n + unit - 1) / unit;
        lines += pieces[k].n;
      }
      if (lines > max_lines) fail("run too long", trial);
      if (lo < 0 || steps < lo) lo = steps;
      if (hi < 0 || steps > hi) hi = steps;
    }
    if (hi - lo > 1) fail("runs not equal to within one step", trial);
  }
  std::printf("trials %ld failures %ld\n", trials, failures);
  return failures == 0 ? 0 : 1;
}
