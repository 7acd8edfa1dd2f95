// Bit-for-bit check of the kernels' exact FP64 scalings (exact_f64.cuh)
// against the host's IEEE-754 division: random bit patterns over the whole
// finite range, integers, near-halfway products and the edges of the fast
// range.  Prints "mismatches N" and exits non-zero on any mismatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "exact_f64.cuh"

using namespace jgb;

static long bad = 0, checked = 0;

static void check(double t) {
  const uint64_t u = f64_bits(t);
  if (!std::isfinite(t)) return;
  ++checked;
  if (sixth_fast(u) && f64_bits(sixth_bits(u)) != f64_bits(t / 6.0)) {
    if (bad < 10) std::printf("t/6 mismatch for %a: %a vs %a\n", t, sixth_bits(u), t / 6.0);
    ++bad;
  }
  if (quarter_fast(u) && f64_bits(quarter_bits(u)) != f64_bits(t / 4.0)) {
    if (bad < 10) std::printf("t/4 mismatch for %a\n", t);
    ++bad;
  }
}

int main(int argc, char** argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 1000000;
  std::mt19937_64 g(20230305);
  for (long i = 0; i < n; ++i) check(f64_from_bits(g()));
  std::uniform_real_distribution<double> U(-8.0, 8.0);
  for (long i = 0; i < n; ++i) check(U(g));
  for (long k = -200000; k <= 200000; ++k) {
    check((double)k);
    check((double)k * 0.125);
    check(3.0 * (double)k + 1.5);  // multiples of 3 and odd halves
  }
  // significands that are multiples of 3 (exact quotients) and their neighbours
  for (long k = 1; k < 200000; ++k) {
    const double m = std::ldexp((double)(3 * k), 52 - (int)std::ilogb((double)(3 * k)));
    check(m);
    check(std::nextafter(m, 0.0));
    check(std::nextafter(m, 1e300));
  }
  // edges of the fast ranges
  for (int e = 1; e < 8; ++e)
    for (long k = 0; k < 1000; ++k) check(f64_from_bits(((uint64_t)e << 52) | (uint64_t)(k * 4503599627370ull)));
  check(f64_from_bits(0x7FEFFFFFFFFFFFFFull));
  std::printf("checked %ld mismatches %ld\n", checked, bad);
  return bad != 0;
}
