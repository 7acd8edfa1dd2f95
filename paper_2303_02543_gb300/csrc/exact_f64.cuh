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

JGB_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
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

// a + b rounded to nearest-even, on the integer pipe.  Fast path: the larger
// operand normal, the smaller normal or zero, the result normal; `ok` is
// false otherwise and the caller must take the hardware addition.
//
// Textbook binary floating-point addition: order by magnitude, align the
// smaller significand with its shifted-out bits jammed into the lowest bit
// (10 guard bits), add or subtract, renormalise (one right shift after a
// carry, a count of leading zeros after cancellation), round to nearest with
// ties to even, repack.
JGB_HD uint64_t add_bits(uint64_t a, uint64_t b, bool& ok) {
  const uint64_t kMag = 0x7FFFFFFFFFFFFFFFull, kFrac = 0x000FFFFFFFFFFFFFull, kHid = 0x0010000000000000ull;
  uint64_t ma = a & kMag, mb = b & kMag;
  if (ma < mb) {
    const uint64_t t = a;
    a = b;
    b = t;
    const uint64_t u = ma;
    ma = mb;
    mb = u;
  }
  const uint32_t ea = (uint32_t)(ma >> 52), eb = (uint32_t)(mb >> 52);
  if (mb == 0) {  // b = +-0: a + b = a, and +-0 + +-0 follows the sign rule
    ok = true;
    return ma == 0 ? (a & b) : a;
  }
  ok = (ea - 1u < 0x7FEu) && (eb - 1u < 0x7FEu);
  const uint64_t A = ((a & kFrac) | kHid) << 10;  // leading bit at 62
  const uint64_t B = ((b & kFrac) | kHid) << 10;
  const uint32_t d = ea - eb;
  uint64_t Bs;
  if (d == 0) Bs = B;
  else if (d < 64) Bs = (B >> d) | (uint64_t)((B << (64 - d)) != 0);
  else Bs = 1;
  int32_t e = (int32_t)ea;
  uint64_t S;
  if (((a ^ b) >> 63) == 0) {
    S = A + Bs;
    if (S >> 63) {
      S = (S >> 1) | (S & 1);
      e += 1;
    }
  } else {
    S = A - Bs;
    if (S == 0) return 0;  // exact cancellation: +0
    const int lz = clz64(S) - 1;
    S <<= lz;
    e -= lz;
  }
  uint64_t M = S >> 10;
  const uint32_t rem = (uint32_t)(S & 0x3FF);
  M += (uint64_t)((rem > 0x200u) | ((rem == 0x200u) & (uint32_t)(M & 1)));
  if (M >> 53) {
    M >>= 1;
    e += 1;
  }
  ok = ok && e >= 1 && e <= 0x7FE;
  return (a & 0x8000000000000000ull) | (((uint64_t)(uint32_t)(e - 1) << 52) + M);
}

// float -> double, exact, for normal floats and zeros (ok false otherwise).
JGB_HD uint64_t f32_to_f64_bits(uint32_t f, bool& ok) {
  const uint32_t e = (f >> 23) & 0xFFu, m = f & 0x7FFFFFu;
  const uint64_t sign = (uint64_t)(f >> 31) << 63;
  if (e == 0 && m == 0) {
    ok = true;
    return sign;
  }
  ok = e - 1u < 254u;
  return sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
}

// double -> float rounded to nearest-even when the result is a normal float
// or a zero of a zero input (ok false otherwise).
JGB_HD uint32_t f64_to_f32_bits(uint64_t d, bool& ok) {
  const uint32_t sign = (uint32_t)(d >> 63) << 31;
  const uint32_t e = (uint32_t)(d >> 52) & 0x7FFu;
  const uint64_t mant = d & 0x000FFFFFFFFFFFFFull;
  if (e == 0 && mant == 0) {
    ok = true;
    return sign;
  }
  const uint32_t m23 = (uint32_t)(mant >> 29);
  const uint32_t rem = (uint32_t)(mant & 0x1FFFFFFFu);
  const uint32_t up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (m23 & 1u));
  const uint32_t E = e - 896u;                      // biased float exponent
  const uint32_t f = (E << 23) + m23 + up;          // a carry moves into the exponent
  ok = (e - 897u < 254u) && ((f >> 23) - 1u < 254u);
  return sign | f;
}

// 4 x, exact, for normal x with 4x normal and for zeros (ok false otherwise).
JGB_HD uint64_t times4_bits(uint64_t b, bool& ok) {
  const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
  if ((b & 0x7FFFFFFFFFFFFFFFull) == 0) {
    ok = true;
    return b;
  }
  ok = e - 1u < 0x7FCu;
  return b + (2ull << 52);
}

// 6 x rounded to nearest-even, for normal x with 6x normal and for zeros
// (ok false otherwise).  x = M 2^(e-1075) with the 53-bit significand M, so
// 6x = P 2^(e-1074) with P = 3M in [1.5 2^53, 1.5 2^54): P keeps 54 or 55
// bits, of which the lowest sh = 1 or 2 are dropped with round-to-nearest,
// ties to even; the biased exponent of the result is e + 1 + sh, and a carry
// out of the significand moves into the exponent field by itself.
JGB_HD uint64_t times6_bits(uint64_t b, bool& ok) {
  const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
  if ((b & 0x7FFFFFFFFFFFFFFFull) == 0) {
    ok = true;
    return b;
  }
  ok = e - 1u < 2042u;
  const uint64_t M = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const uint64_t P = M * 3u;
  const uint32_t sh = 1u + (uint32_t)(P >> 54);
  const uint64_t rem = P & ((1ull << sh) - 1u), half = 1ull << (sh - 1u);
  uint64_t q = P >> sh;
  q += (uint64_t)((rem > half) | ((rem == half) & (uint32_t)(q & 1u)));
  return (b & 0x8000000000000000ull) + ((uint64_t)(e + sh) << 52) + q;
}

}  // namespace jgb
