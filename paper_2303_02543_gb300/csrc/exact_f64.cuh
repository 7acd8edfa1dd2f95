// Exact FP64 scalings that run on the integer pipe.
//
// On GB300 the FP64 pipe issues about 2 operations per clock per SM (one
// sixty-fourth of the FP32 rate), so a Jacobi sweep in FP64 is bound by its
// FP64 additions rather than by HBM.  The two divisions of the update,
// t / 4 (2D) and t / 6 (3D), are done here on the integer pipe instead.  Both
// return exactly the IEEE-754 round-to-nearest-even quotient; operands whose
// result would leave the normal range (zero, subnormal, tiny, inf, NaN) take
// the ordinary FP64 operation.  The helpers are host+device so the CPU test
// suite can compare them bit for bit with IEEE division.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define JGB_HD __host__ __device__ __forceinline__
#else
#define JGB_HD static inline
#endif

namespace jgb {

JGB_HD uint64_t f64_bits(double v) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t u;
  memcpy(&u, &v, 8);
  return u;
#endif
}

JGB_HD double f64_from_bits(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double v;
  memcpy(&v, &u, 8);
  return v;
#endif
}

JGB_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// True when t / 4 can be formed by lowering the exponent field by 2: the
// biased exponent e satisfies 3 <= e <= 2046 (result normal, t finite).
JGB_HD bool quarter_fast(uint64_t b) {
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  return (e - 3u) < 0x7fcu;
}

// t / 4 for a t with quarter_fast(bits(t)).
JGB_HD double quarter_bits(uint64_t b) { return f64_from_bits(b - (2ull << 52)); }

// True when t / 6 stays in the normal range: biased exponent 4 <= e <= 2046.
JGB_HD bool sixth_fast(uint64_t b) {
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  return (e - 4u) < 0x7fbu;
}

// t / 6, correctly rounded, for a t with sixth_fast(bits(t)).
//
// t = M 2^(e-1075) with the 53-bit significand M.  With N = 16 M (< 2^57)
// the quotient is t / 6 = (N / 3) 2^(e-1080).  Q = floor(N / 3) comes from a
// multiply by the invariant 0xAAAAAAAAAAAAAAAB = (2^65 + 1) / 3 (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994).
// Q lies in [2^54.4, 2^55.4); dropping sh = 2 or 3 low bits leaves 53.  The
// exact quotient N/3 is never halfway between two results (a tie needs 3 | N,
// and then Q has four trailing zero bits), so adding half a unit and
// truncating rounds to nearest-even.  A carry out of the significand moves
// into the exponent field by itself.
JGB_HD double sixth_bits(uint64_t b) {
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  const uint64_t M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const uint64_t N = M << 4;
  const uint64_t Q = umulhi64(N, 0xAAAAAAAAAAAAAAABull) >> 1;
  const uint32_t sh = 2u + (uint32_t)(Q >> 55);
  const uint64_t q = (Q + (1ull << (sh - 1))) >> sh;
  const uint64_t hi = (b & 0x8000000000000000ull) | ((uint64_t)(e - 6u + sh) << 52);
  return f64_from_bits(hi + q);
}

}  // namespace jgb
