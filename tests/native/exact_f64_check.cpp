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

static long add_checked = 0, add_fast = 0;

static void check_add(double x, double y) {
  bool ok = false;
  const uint64_t r = add_bits(f64_bits(x), f64_bits(y), ok);
  if (!std::isfinite(x) || !std::isfinite(y)) return;
  ++add_checked;
  if (!ok) return;
  ++add_fast;
  const double ref = x + y;
  if (r != f64_bits(ref)) {
    if (bad < 10) std::printf("add mismatch %a + %a: %a vs %a\n", x, y, f64_from_bits(r), ref);
    ++bad;
  }
}

static long conv_checked = 0, x6_fast = 0;

static void check_conv(double d, float f) {
  bool ok;
  ++conv_checked;
  uint32_t fb;
  memcpy(&fb, &f, 4);
  const uint64_t db = f32_to_f64_bits(fb, ok);
  if (ok && db != f64_bits((double)f)) {
    if (bad < 10) std::printf("f2d mismatch %a\n", (double)f);
    ++bad;
  }
  const uint32_t r = f64_to_f32_bits(f64_bits(d), ok);
  const float ref = (float)d;
  uint32_t rb;
  memcpy(&rb, &ref, 4);
  if (ok && r != rb) {
    if (bad < 10) std::printf("d2f mismatch %a: %08x vs %08x\n", d, r, rb);
    ++bad;
  }
  const uint64_t q = times4_bits(f64_bits(d), ok);
  if (ok && q != f64_bits(d * 4.0)) {
    if (bad < 10) std::printf("x4 mismatch %a\n", d);
    ++bad;
  }
  const uint64_t q6 = times6_bits(f64_bits(d), ok);
  if (ok && q6 != f64_bits(d * 6.0)) {
    if (bad < 10) std::printf("x6 mismatch %a: %a vs %a\n", d, f64_from_bits(q6), d * 6.0);
    ++bad;
  }
  if (ok) ++x6_fast;
}

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
  // additions: random bit patterns, nearby magnitudes (cancellation), ties,
  // zeros of both signs, exponent gaps around 53..64
  for (long i = 0; i < n; ++i) {
    const double x = f64_from_bits(g()), y = f64_from_bits(g());
    check_add(x, y);
    check_add(x, -x * (1.0 + std::ldexp(1.0, -(int)(g() % 60))));
    check_add(U(g), U(g));
    check_add(U(g), -U(g));
    check_add(U(g) * 1e10, U(g));
    check_add(x, std::ldexp(y, -(int)(g() % 70)));
  }
  for (long k = -3000; k <= 3000; ++k)
    for (long j = -40; j <= 40; ++j) {
      check_add((double)k, (double)j * 0.5);
      check_add((double)k * 0.1, -(double)j * 0.1);
    }
  const double zs[] = {0.0, -0.0, 1.0, -1.0, 3.5, -2.25};
  for (double x : zs)
    for (double y : zs) check_add(x, y);
  for (int e = 0; e < 70; ++e) {
    check_add(1.0, std::ldexp(1.0, -e));
    check_add(1.0, -std::ldexp(1.0, -e));
    check_add(1.0, std::ldexp(1.5, -e));
    check_add(1.0 + std::ldexp(1.0, -52), std::ldexp(1.0, -e));
  }
  check_add(0x1.fffffffffffffp+1023, 0x1.fffffffffffffp+1023);  // overflow -> not fast
  check_add(0x1p-1022, -0x1.0000000000001p-1022);               // subnormal result -> not fast
  std::printf("adds %ld fast %ld\n", add_checked, add_fast);
  // conversions: random doubles in and around the float range, halfway cases
  for (long i = 0; i < n; ++i) {
    const double d = f64_from_bits(g());
    uint32_t fb = (uint32_t)g();
    float f;
    memcpy(&f, &fb, 4);
    check_conv(d, f);
    const double u = std::ldexp(U(g), (int)(g() % 300) - 150);
    check_conv(u, (float)u);
    const float ff = (float)U(g);
    const double half = (double)ff + std::ldexp((double)std::nextafter(ff, 1e30f) - (double)ff, -1);
    check_conv(half, ff);
    check_conv(-half, -ff);
  }
  check_conv(0.0, 0.0f);
  check_conv(-0.0, -0.0f);
  check_conv(3.4028235677973366e38, 3.4028235e38f);  // rounds past FLT_MAX -> not fast
  // x6 at the edges of its fast range: largest exponents, smallest normals
  for (uint64_t e = 2038; e <= 2046; ++e)
    for (long k = 0; k < 2000; ++k) {
      const double d = f64_from_bits((e << 52) | (g() & 0x000FFFFFFFFFFFFFull));
      check_conv(d, 0.0f);
      check_conv(-d, 0.0f);
    }
  for (uint64_t e = 1; e <= 4; ++e)
    for (long k = 0; k < 2000; ++k) check_conv(f64_from_bits((e << 52) | (g() & 0x000FFFFFFFFFFFFFull)), 0.0f);
  check_conv(f64_from_bits(0x7FEFFFFFFFFFFFFFull), 0.0f);
  std::printf("conversions %ld (x6 fast %ld)\n", conv_checked, x6_fast);
  std::printf("checked %ld mismatches %ld\n", checked, bad);
  return bad != 0;
}
