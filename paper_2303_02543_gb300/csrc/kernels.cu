// CUDA kernels (sm_103a) for the over-decomposed Jacobi relaxation.
//
// Section 4.3 describes each iteration of the Jacobi3D proxy as: pack the
// faces of every cuboid, move them to the neighbours, unpack them into the
// halos, then run the Jacobi update once all halos are in.  Section 4.4 cuts
// the domain into more pieces than processors.  Here every block of the
// decomposition is a task that warps pick from a work table; the update and
// the halo exchange are fused (each block writes its boundary layer straight
// into its neighbours' ghost cells of the destination buffer) or run as
// separate pack / unpack kernels.  Both give bit-identical fields.
//
// Canonical arithmetic of one update (W/E, S/N, D/U = -/+ neighbours along
// x, y, z; every operation one IEEE round-to-nearest-even, no contraction):
//   2D: t = ((W + S) + (E + N)) + f,            x' = t / 4
//   3D: t = (((W + D) + (E + U)) + (S + N)) + f, x' = t / 6
//   residual r = t - (2d) x, reduced as sum r^2.
// The pair (E + N) of a point is the pair (W + S) of its diagonal neighbour
// one row up and one column right (2D; in 3D the same holds along x and z),
// so a warp marching along the last axis forms each such pair once and
// passes it on: 3 FP64 additions per 2D update instead of 4, plus one edge
// pair per warp row (per block row with the march items of k_f64_march).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "exact_f64.cuh"
#include "jacobi_internal.h"

namespace jgb {

#define FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// scalar helpers

// a + b rounded to nearest even, issued as fma(a, 1, b): the product a * 1 is
// exact, so the result is bit-identical to __dadd_rn(a, b) for every input.
// It is written in PTX because the compiler would turn fma(a, 1.0, b) back
// into an add.
//
// On GB300 an FP64 FMA whose multiplier is a register issues at the full FP64
// rate (2.0 lanes per clock per SM, measured 628 G/s), while the FP64 add, the
// FP64 multiply and an FMA whose multiplier is an immediate or a constant-bank
// operand issue at 1.68 (529 G/s).  The hot kernels therefore call dadd1 with
// `one` = 1.0 loaded once per thread from global memory (load_one), so that
// the compiler cannot see its value and fold it into an immediate; dadd is
// the plain form for the cold paths.
__device__ __forceinline__ double dadd(double a, double b) {
  double r;
  asm("fma.rn.f64 %0, %1, 0d3FF0000000000000, %2;" : "=d"(r) : "d"(a), "d"(b));
  return r;
}
__device__ __forceinline__ double dadd1(double a, double b, double one) {
  double r;
  asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(one), "d"(b));
  return r;
}
// a * m + b rounded once, m a multiplier held in a register (the residual's
// t - 4 c in 2D as fma(c, -4, t): 4 c is exact, so this is the rounding of
// the subtraction, in one FP64 instruction)
__device__ __forceinline__ double dfma1(double a, double m, double b) {
  double r;
  asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(m), "d"(b));
  return r;
}
__device__ double g_fp64_one = 1.0;
__device__ __forceinline__ double load_one() { return __ldg(&g_fp64_one); }

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2 by the
// TMA unit: one instruction per line, no registers, no completion to wait for.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The rare-case paths behind the warp votes below are out-of-line calls: the
// compiler would otherwise compute them for every point and select afterwards,
// an FP64 multiply (or a whole FP64 division) per point on a pipe that is the
// bottleneck.
__device__ __noinline__ double slow_quarter(double t) { return __dmul_rn(t, 0.25); }
__device__ __noinline__ double slow_sixth(double t) { return __ddiv_rn(t, 6.0); }
__device__ __noinline__ double slow_times4(double c) { return __dmul_rn(4.0, c); }
__device__ __noinline__ double slow_times6(double c) { return __dmul_rn(6.0, c); }
__device__ __noinline__ double slow_f2d(float v) { return (double)v; }
__device__ __noinline__ float slow_d2f(double v) { return __double2float_rn(v); }

// t / 4, exact: exponent decrement on the integer pipe, FP64 multiply only when
// some live lane of the warp needs it (zero, subnormal, inf/NaN).  A lane that
// holds no point (`live` false: its result is never stored) never calls for
// the slow path: its t is typically 0.
__device__ __forceinline__ double div_2d(double t, bool live = true) {
  const uint64_t b = f64_bits(t);
  const bool fast = quarter_fast(b) || !live;
  double q = quarter_bits(b);
  if (!__all_sync(FULL_MASK, fast)) {
    if (!fast) q = slow_quarter(t);
  }
  return q;
}

// t / 6, correctly rounded, integer pipe (see exact_f64.cuh); IEEE division
// only when some live lane of the warp leaves the fast range.
__device__ __forceinline__ double div_3d(double t, bool live = true) {
  const uint64_t b = f64_bits(t);
  const bool fast = sixth_fast(b) || !live;
  double q = sixth_bits(b);
  if (!__all_sync(FULL_MASK, fast)) {
    if (!fast) q = slow_sixth(t);
  }
  return q;
}

template <int DIM>
__device__ __forceinline__ double jdiv(double t, bool live = true) {
  if constexpr (DIM == 2) return div_2d(t, live);
  else return div_3d(t, live);
}

template <int DIM>
__device__ __forceinline__ float jdivf(float t) {
  if constexpr (DIM == 2) return __fmul_rn(t, 0.25f);
  else return __fdiv_rn(t, 6.0f);
}

// low-precision element access ------------------------------------------------

struct bf16x4 {
  __nv_bfloat162 a, b;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// 4 consecutive elements (16-byte aligned for float, 8-byte for bf16)
__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  bf16x4 v;
  memcpy(&v, &u, 8);
  const float2 lo = __bfloat1622float2(v.a), hi = __bfloat1622float2(v.b);
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
  bf16x4 o;
  o.a = __floats2bfloat162_rn(v.x, v.y);
  o.b = __floats2bfloat162_rn(v.z, v.w);
  uint2 u;
  memcpy(&u, &o, 8);
  *reinterpret_cast<uint2*>(p) = u;
}

__device__ __forceinline__ float comp(const float4& v, int k) {
  return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// Store the valid leading elements of a 4-vector (all 4 in one store when valid).
template <typename T>
__device__ __forceinline__ void st4_valid(T* p, float4 v, int nvalid) {
  if (nvalid >= 4) {
    st4(p, v);
  } else {
    if (nvalid > 0) p[0] = from_f<T>(v.x);
    if (nvalid > 1) p[1] = from_f<T>(v.y);
    if (nvalid > 2) p[2] = from_f<T>(v.z);
  }
}

// ---------------------------------------------------------------------------
// Geometry of one warp item.  The warp marches along the last axis (y in 2D,
// z in 3D); in 3D the row y is fixed.  "Line m" is the row of the warp at
// march index m (m = -1 and m = extent are ghost lines).

template <int DIM>
struct Geo {
  int64_t base;   // element offset of the line at march index 0 minus one line step
  int64_t step;   // elements between consecutive lines along the march
  int64_t side;   // 3D: elements from a line to the same x on row y+1 (= pitch)
  int extent;     // interior extent along the march axis
  int col_stride; // x-ghost column index = m * col_stride + col_off
  int col_off;

  __device__ __forceinline__ Geo(const BlockDev& B, int y) {
    if constexpr (DIM == 2) {
      step = B.pitch;
      base = B.off;
      side = 0;
      extent = B.by;
      col_stride = 1;
      col_off = 0;
    } else {
      step = B.plane;
      base = B.off + (int64_t)(y + 1) * B.pitch;
      side = B.pitch;
      extent = B.bz;
      col_stride = B.by;
      col_off = y;
    }
  }
  // offset of x = 0 on line m
  __device__ __forceinline__ int64_t line(int m) const { return base + (int64_t)(m + 1) * step; }
  __device__ __forceinline__ int col(int m) const { return m * col_stride + col_off; }
};

// Ghost targets of the halo push for one warp item (destination buffer).
struct PushTargets {
  int64_t lo_line, hi_line;   // march-axis faces: offset of x = 0 in the neighbour's ghost line
  int64_t lo_side, hi_side;   // 3D side faces (y): per-plane offset base, -1 if none
  int64_t w_col, e_col;       // x faces: neighbour ghost column base (add col(m)), -1 if none
  int64_t lo_side_step, hi_side_step;
};

// MODE of the FP64 kernel
// kModeOuterR: the residual pass of the split outer step (reads x_new, stores
// r in the low type and the partials; writes no x)
enum { kModeSweep = 0, kModeResid = 1, kModeOuter = 2, kModeOuterR = 3 };

// Load policies.  COH = false: read-only path (__ldg), valid when nothing
// writes the array during the launch.  COH = true: L2-only loads (__ldcg),
// for the persistent kernel where other CTAs rewrite the arrays while it runs.
template <bool COH>
__device__ __forceinline__ double ldd(const double* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ double2 ldd2(const double* p) {
  if constexpr (COH) return __ldcg(reinterpret_cast<const double2*>(p));
  else return __ldg(reinterpret_cast<const double2*>(p));
}
template <bool COH>
__device__ __forceinline__ float ldf(const float* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) {
  const unsigned short* q = reinterpret_cast<const unsigned short*>(p);
  unsigned short u;
  if constexpr (COH) u = __ldcg(q);
  else u = __ldg(q);
  return __bfloat162float(__ushort_as_bfloat16(u));
}
template <bool COH>
__device__ __forceinline__ float4 ldf4(const float* p) {
  if constexpr (COH) return __ldcg(reinterpret_cast<const float4*>(p));
  else return __ldg(reinterpret_cast<const float4*>(p));
}
template <bool COH>
__device__ __forceinline__ float4 ldf4(const __nv_bfloat16* p) {
  uint2 u;
  if constexpr (COH) u = __ldcg(reinterpret_cast<const uint2*>(p));
  else u = __ldg(reinterpret_cast<const uint2*>(p));
  bf16x4 v;
  memcpy(&v, &u, 8);
  const float2 lo = __bfloat1622float2(v.a), hi = __bfloat1622float2(v.b);
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// float -> double and double -> float (nearest-even) on the integer pipe when
// every lane of the warp is in the normal range, else the conversion
// instruction (which runs on the FP64 pipe); bit-identical either way.
// Like every helper here that votes across the warp (div_2d, div_3d,
// twod_x, dadd_int), these must be called by all 32 lanes together.
__device__ __forceinline__ double f2d(float v) {
  bool ok;
  double r = f64_from_bits(f32_to_f64_bits(__float_as_uint(v), ok));
  if (!__all_sync(FULL_MASK, ok)) {
    if (!ok) r = slow_f2d(v);
  }
  return r;
}
__device__ __forceinline__ float d2f(double v) {
  bool ok;
  float r = __uint_as_float(f64_to_f32_bits(f64_bits(v), ok));
  if (!__all_sync(FULL_MASK, ok)) {
    if (!ok) r = slow_d2f(v);
  }
  return r;
}
// (2d) x of the residual on the integer pipe: 4x exactly in 2D, 6x rounded
// to nearest-even in 3D (exact_f64.cuh); the FP64 product only when a lane
// leaves the fast range.
template <int DIM>
__device__ __forceinline__ double twod_x(double c) {
  if constexpr (DIM == 2) {
    bool ok;
    double r = f64_from_bits(times4_bits(f64_bits(c), ok));
    if (!__all_sync(FULL_MASK, ok)) {
      if (!ok) r = slow_times4(c);
    }
    return r;
  } else {
    bool ok;
    double r = f64_from_bits(times6_bits(f64_bits(c), ok));
    if (!__all_sync(FULL_MASK, ok)) {
      if (!ok) r = slow_times6(c);
    }
    return r;
  }
}

// Loader of "the field value" at an element offset: x, or x + e in the outer
// refinement step (the updated iterate x_new = x + e, formed on the fly).
// Loads are split into fetch (issue the loads into registers) and fin (the
// additions of x + e), so a kernel can issue the loads of a later line and
// only wait for them where it consumes the values.
template <int MODE, typename TE, bool COH>
struct F64Src {
  const double* __restrict__ x;
  const TE* __restrict__ e;
  bool apply;
  double unit;  // 1.0 in a register (see dadd1)

  struct Raw1 {
    double v;
    float e;
  };
  struct Raw2 {
    double a, b;
    float ea, eb;
  };

  __device__ __forceinline__ void fetch1(int64_t o, Raw1& r) const {
    r.v = ldd<COH>(x + o);
    r.e = 0.f;
    if constexpr (MODE == kModeOuter) {
      if (apply) r.e = ldf<COH>(e + o);
    }
  }
  // Called from lane-divergent code (edge lanes only): no warp-collective
  // operation may appear here, so the conversion is the plain instruction.
  __device__ __forceinline__ double fin1(const Raw1& r) const {
    if constexpr (MODE == kModeOuter) {
      if (apply) return dadd1(r.v, (double)r.e, unit);
    }
    return r.v;
  }
  __device__ __forceinline__ double one(int64_t o) const {
    Raw1 r;
    fetch1(o, r);
    return fin1(r);
  }
  // `valid` only predicates the loads
  __device__ __forceinline__ void fetch2(int64_t o, bool valid, Raw2& r) const {
    r.a = 0.0;
    r.b = 0.0;
    r.ea = 0.f;
    r.eb = 0.f;
    if (valid) {
      const double2 v = ldd2<COH>(x + o);
      r.a = v.x;
      r.b = v.y;
      if constexpr (MODE == kModeOuter) {
        if (apply) {
          r.ea = ldf<COH>(e + o);
          r.eb = ldf<COH>(e + o + 1);
        }
      }
    }
  }
  // Called by every lane of the warp, so the warp-voting integer conversion
  // f2d is allowed.
  __device__ __forceinline__ void fin2(const Raw2& r, double& a, double& b) const {
    a = r.a;
    b = r.b;
    if constexpr (MODE == kModeOuter) {
      if (apply) {  // uniform: one flag per solve
        a = dadd1(a, f2d(r.ea), unit);
        b = dadd1(b, f2d(r.eb), unit);
      }
    }
  }
  __device__ __forceinline__ void two(int64_t o, bool valid, double& a, double& b) const {
    Raw2 r;
    fetch2(o, valid, r);
    fin2(r, a, b);
  }
};

template <typename TR>
__device__ __forceinline__ void store_r(TR* p, float rf);
template <>
__device__ __forceinline__ void store_r<float>(float* p, float rf) { *p = rf; }
template <>
__device__ __forceinline__ void store_r<__nv_bfloat16>(__nv_bfloat16* p, float rf) { *p = __float2bfloat16_rn(rf); }

template <int DIM>
__device__ __forceinline__ void push_targets(PushTargets& T, const BlockDev& B, const BlockDev* __restrict__ blocks,
                                             int y) {
  const int lo = DIM == 2 ? 2 : 4, hi = lo + 1;
  T.lo_line = T.hi_line = -1;
  if (B.nbr[lo] >= 0) {
    const BlockDev& N = blocks[B.nbr[lo]];
    const Geo<DIM> GN(N, y);
    T.lo_line = GN.line(GN.extent);
  }
  if (B.nbr[hi] >= 0) {
    const BlockDev& N = blocks[B.nbr[hi]];
    const Geo<DIM> GN(N, y);
    T.hi_line = GN.line(-1);
  }
  T.lo_side = T.hi_side = -1;
  T.lo_side_step = T.hi_side_step = 0;
  if constexpr (DIM == 3) {
    if (y == 0 && B.nbr[2] >= 0) {
      const BlockDev& N = blocks[B.nbr[2]];
      T.lo_side = N.off + (int64_t)(N.by + 1) * N.pitch;
      T.lo_side_step = N.plane;
    }
    if (y == B.by - 1 && B.nbr[3] >= 0) {
      const BlockDev& N = blocks[B.nbr[3]];
      T.hi_side = N.off;
      T.hi_side_step = N.plane;
    }
  }
  T.w_col = T.e_col = -1;
  if (B.nbr[0] >= 0) {
    const BlockDev& N = blocks[B.nbr[0]];
    T.w_col = N.xoff + (int64_t)N.by * N.bz;  // the west neighbour's east ghost column
  }
  if (B.nbr[1] >= 0) T.e_col = blocks[B.nbr[1]].xoff;  // the east neighbour's west column
}

// ---------------------------------------------------------------------------
// FP64 work item: sweep (x' = t / 2d), residual only, or the refinement outer
// step (x_new = x + e; r = b - A x_new; store x_new, r in low precision).
// Two points per lane, 64 per warp row.  Every load of line m+1 is issued
// while line m is computed.

// a + b for every lane, on the integer pipe when every lane of the warp is on
// the software fast path (exact_f64.cuh), else on the FP64 pipe.
__device__ __noinline__ double slow_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dadd_int(double a, double b) {
  bool ok;
  double r = f64_from_bits(add_bits(f64_bits(a), f64_bits(b), ok));
  if (!__all_sync(FULL_MASK, ok)) {
    if (!ok) r = slow_add(a, b);
  }
  return r;
}

// EMU: how many of the seven FP64 additions of a warp step run on the
// integer pipe instead (0; 2 = the two source additions; 3 = also the edge
// pair of lane 0).  The FP64 pipe issues about 2 operations per clock per SM
// on GB300 while the integer pipe is idle; results are bit-identical.
//
// MARCH: the item is one of several segments of a block row range that the
// same warp computes left to right.  Lane 31 keeps its pair P(m-1, x+1) of
// every line in `wr`; for the next segment that pair is P(m-1, xs-1), the
// (W + S) pair lane 0 would otherwise form, so lane 0 reads it from `rd`
// (bit for bit the same value: addition is commutative) and the warp issues
// one FP64 addition fewer per line.
//
// COLP (the block's first segment): the (W + S) pairs of the block's first
// column, x[m][-1] + x[m-1][0], are formed kMarchLines lines at a time, one
// line per lane, into the warp's shared buffer `colp`, and lane 0 reads them
// there: one warp FP64 instruction per kMarchLines lines instead of one per
// line (the same values: the same operands in the same order).
template <int DIM, int MODE, bool PUSH, bool RESID, typename TE, typename TR, bool COH, int EMU = 0,
          bool MARCH = false, bool COLP = false>
__device__ __forceinline__ void f64_item(const WorkItem& it, const BlockDev* __restrict__ blocks,
                                         const SolveDev* __restrict__ solves, int kpar, int epar,
                                         const double* rd = nullptr, double* wr = nullptr, int pf = 0,
                                         double* colp = nullptr) {
  constexpr bool WRITE = MODE != kModeResid && MODE != kModeOuterR;
  constexpr bool STORE_R = MODE == kModeOuter || MODE == kModeOuterR;
  const int lane = threadIdx.x & 31;
  const BlockDev B = blocks[it.block];
  const SolveDev* S = solves + B.solve;
  const int par = (S->phase + kpar) & 1;
  const double one = load_one();
  auto add = [one](double u, double v) { return dadd1(u, v, one); };
  double mfour = 0.0, mone = 0.0;  // -4 and -1 in registers (residual)
  if constexpr (RESID || STORE_R) {
    mfour = __dmul_rn(one, -4.0);
    mone = __dmul_rn(one, -1.0);
  }
  F64Src<MODE, TE, COH> src;
  src.unit = one;
  src.x = S->x[par];
  src.e = MODE == kModeOuter ? reinterpret_cast<const TE*>(S->e[epar]) : nullptr;
  src.apply = MODE == kModeOuter && S->apply_e;
  double* __restrict__ xd = S->x[par ^ 1];
  const double* __restrict__ f = S->f;
  TR* __restrict__ rout = STORE_R ? reinterpret_cast<TR*>(S->r) : nullptr;

  const int y = it.y0;  // 3D: the fixed row
  const Geo<DIM> G(B, y);
  const int bx = B.bx;
  const int xs = it.seg * kSegF64;
  const int x = xs + 2 * lane;
  const bool v0 = x < bx, v1 = x + 1 < bx;
  const bool last0 = x == bx - 1, last1 = x + 1 == bx - 1;
  const bool east_inner = x + 2 < bx;
  const int64_t gW = B.xoff;
  const int64_t gE = B.xoff + (int64_t)B.by * B.bz;
  // halo push: the W / E neighbours' ghost columns are kept by the lanes
  // holding the block's first and last points; the march-axis faces and (3D)
  // the side rows are looked up on the lines that write them
  int64_t w_col = -1, e_col = -1;
  if constexpr (PUSH && WRITE) {
    if (x == 0 && B.nbr[0] >= 0) {
      const BlockDev& N = blocks[B.nbr[0]];
      w_col = N.xoff + (int64_t)N.by * N.bz;  // the west neighbour's east ghost column
    }
    if ((last0 || last1) && B.nbr[1] >= 0) e_col = blocks[B.nbr[1]].xoff;  // the east neighbour's west column
  }

  const int m0 = DIM == 2 ? it.y0 : it.z0;
  const int mend = m0 + it.n;

  // Values of line m gathered by one lane: the edge scalars it needs (east of
  // point 1 for lane 31 / the lane holding the block's last point, west of
  // point 0 for lane 0, the ghost east of point 0 for the lane whose point 0
  // is last), the source, and in 3D the side rows.
  // A lane needs at most two edge values: `wv` (lane 0) and one of `eg`
  // (lane 31 or the lane whose point 1 is last: east of point 1; the lane
  // whose point 0 is last: its east ghost).  fetch_aux only issues loads;
  // fin_aux forms the values where the next line starts.
  using Src = F64Src<MODE, TE, COH>;
  struct LineAux {
    typename Src::Raw1 egr, wvr;
    typename Src::Raw2 sr, qr;  // 3D: rows y-1 and y+1
    double eg;   // x[m][x+2], or the east ghost of point 1 or of point 0
    double wv;   // lane 0: x[m][xs-1] or the west ghost
    double f0, f1;
    double sn0, sn1;
  };
  const bool has_eg = (lane == 31 && east_inner) || last1 || last0;
  constexpr bool COL = COLP && !MARCH && EMU < 3;  // first-column pairs from `colp`
  const bool has_wv = lane == 0 && !(MARCH && xs > 0) && !(COL && xs == 0);
  auto fetch_aux = [&](int m, LineAux& a) {
    const int64_t lc = G.line(m);
    const int col = G.col(m);
    if (lane == 31 && east_inner) src.fetch1(lc + x + 2, a.egr);
    if (last1 || last0) src.fetch1(gE + col, a.egr);
    if (has_wv) {
      if (xs > 0) src.fetch1(lc + xs - 1, a.wvr);
      else src.fetch1(gW + col, a.wvr);
    }
    a.f0 = 0.0;
    a.f1 = 0.0;
    if (v0) {
      const double2 fv = ldd2<false>(f + lc + x);
      a.f0 = fv.x;
      a.f1 = fv.y;
    }
    if constexpr (DIM == 3) {
      src.fetch2(lc - G.side + x, v0, a.sr);
      src.fetch2(lc + G.side + x, v0, a.qr);
    }
  };
  auto fin_aux = [&](LineAux& a) {
    a.eg = 0.0;
    a.wv = 0.0;
    if (has_eg) a.eg = src.fin1(a.egr);
    if (has_wv) a.wv = src.fin1(a.wvr);
    a.sn0 = 0.0;
    a.sn1 = 0.0;
    if constexpr (DIM == 3) {
      double s0, s1, q0, q1;
      src.fin2(a.sr, s0, s1);
      src.fin2(a.qr, q0, q1);
      a.sn0 = add(s0, q0);
      a.sn1 = add(s1, q1);
    }
  };

  // lines m-1 (p), m (c), m+1 (n) and the aux values of line m
  double p0, p1, c0, c1, n0, n1;
  src.two(G.line(m0 - 1) + x, v0, p0, p1);
  src.two(G.line(m0) + x, v0, c0, c1);
  src.two(G.line(m0 + 1) + x, v0, n0, n1);
  LineAux a;
  fetch_aux(m0, a);
  fin_aux(a);
  // prologue pairs of line m-1: A0p = P(m-1, x) = p[x+1] + c[x]; A1p = P(m-1, x+1)
  double pE = __shfl_down_sync(FULL_MASK, p0, 1);
  if (lane == 31 && east_inner) pE = src.one(G.line(m0 - 1) + x + 2);
  if (last0) c1 = a.eg;
  double qacc = 0.0;  // residual: this lane's sum of r^2 over the current group
  double A0p = add(p1, c0);
  double A1p = add(pE, c1);
  // first-column pairs of lines mc .. mc + kMarchLines - 1 (COL, first segment)
  auto fill_col = [&](int mc) {
    __syncwarp();
    for (int j = lane; j < kMarchLines && mc + j < mend; j += 32) {
      const int mm = mc + j;
      colp[j] = add(src.one(gW + G.col(mm)), src.one(G.line(mm - 1)));
    }
    __syncwarp();
  };
  if constexpr (COL) {
    if (xs == 0) fill_col(m0);
  }

  for (int m = m0; m < mend; ++m) {
    const int64_t lc = G.line(m);
    const int col = G.col(m);
    // lines pf steps ahead of the register loads into L2 (march items; within
    // this item's lines and the ghost line after them)
    if constexpr (MARCH) {
      if (pf > 0 && lane == 0) {
        const uint32_t bytes = (uint32_t)min(kSegF64, B.pitch - xs) * 8u;
        if (m + 2 + pf <= mend) l2_prefetch(src.x + G.line(m + 2 + pf) + xs, bytes);
        if (m + 1 + pf < mend) l2_prefetch(f + G.line(m + 1 + pf) + xs, bytes);
      }
    }
    // prefetch line m+2 and the aux values of line m+1
    typename Src::Raw2 nnr;
    LineAux an;
    const bool more = m + 1 < mend;
    if (more) {
      src.fetch2(G.line(m + 2) + x, v0, nnr);
      fetch_aux(m + 1, an);
    }
    // east neighbour of point x+1 on line m
    double e1 = __shfl_down_sync(FULL_MASK, c0, 1);
    if ((lane == 31 && east_inner) || last1) e1 = a.eg;
    // (W + S) pair of point x: from the left lane, or formed here on lane 0
    double bw = __shfl_up_sync(FULL_MASK, A1p, 1);
    if constexpr (MARCH) {
      if (lane == 31) wr[m - m0] = A1p;
      if (xs > 0) {
        if (lane == 0) bw = rd[m - m0];
      } else if (lane == 0) {
        bw = add(a.wv, p0);
      }
    } else if constexpr (EMU >= 3) {
      const double be = dadd_int(a.wv, p0);
      if (lane == 0) bw = be;
    } else if constexpr (COL) {
      if (xs == 0) {
        if (m > m0 && ((m - m0) & (kMarchLines - 1)) == 0) fill_col(m);
        if (lane == 0) bw = colp[(m - m0) & (kMarchLines - 1)];
      } else if (lane == 0) {
        bw = add(a.wv, p0);
      }
    } else {
      if (lane == 0) bw = add(a.wv, p0);
    }
    const double A0 = add(c1, n0);  // P(m, x)   = c[x+1] + n[x]
    const double A1 = add(e1, n1);  // P(m, x+1) = c[x+2] + n[x+1]
    double t0 = add(bw, A0), t1 = add(A0p, A1);
    if constexpr (DIM == 3) {
      t0 = add(t0, a.sn0);
      t1 = add(t1, a.sn1);
    }
    if constexpr (EMU >= 2) {
      t0 = dadd_int(t0, a.f0);
      t1 = dadd_int(t1, a.f1);
    } else {
      t0 = add(t0, a.f0);
      t1 = add(t1, a.f1);
    }

    if constexpr (WRITE) {
      double o0, o1;
      if constexpr (MODE == kModeSweep) {
        o0 = jdiv<DIM>(t0, v0);
        o1 = jdiv<DIM>(t1, v1);
      } else {
        o0 = c0;  // outer step: the updated iterate itself
        o1 = c1;
      }
      double* d = xd + lc + x;
      if (v1) *reinterpret_cast<double2*>(d) = make_double2(o0, o1);
      else if (v0) *d = o0;
      if constexpr (PUSH) {
        auto put2 = [&](double* q) {
          if (v1) *reinterpret_cast<double2*>(q) = make_double2(o0, o1);
          else if (v0) *q = o0;
        };
        constexpr int lo = DIM == 2 ? 2 : 4;  // the march-axis faces
        if (m == 0) {
          const int nb = __ldg(&blocks[it.block].nbr[lo]);
          if (nb >= 0) {
            const Geo<DIM> GN(blocks[nb], y);
            put2(xd + GN.line(GN.extent) + x);
          }
        }
        if (m == G.extent - 1) {
          const int nb = __ldg(&blocks[it.block].nbr[lo + 1]);
          if (nb >= 0) {
            const Geo<DIM> GN(blocks[nb], y);
            put2(xd + GN.line(-1) + x);
          }
        }
        if constexpr (DIM == 3) {
          if (y == 0) {  // the S neighbour's north ghost row of plane m
            const int nb = __ldg(&blocks[it.block].nbr[2]);
            if (nb >= 0) {
              const BlockDev& N = blocks[nb];
              put2(xd + N.off + (int64_t)(N.by + 1) * N.pitch + (int64_t)(m + 1) * N.plane + x);
            }
          }
          if (y == B.by - 1) {  // the N neighbour's south ghost row of plane m
            const int nb = __ldg(&blocks[it.block].nbr[3]);
            if (nb >= 0) {
              const BlockDev& N = blocks[nb];
              put2(xd + N.off + (int64_t)(m + 1) * N.plane + x);
            }
          }
        }
        if (w_col >= 0) xd[w_col + col] = o0;
        if (e_col >= 0) {
          if (last0) xd[e_col + col] = o0;
          if (last1) xd[e_col + col] = o1;
        }
      }
    }
    if constexpr (RESID || STORE_R) {
      // t - (2d) x rounded once: in 2D fma(x, -4, t) (4 x is exact); in 3D
      // fma(6 x, -1, t) with 6 x rounded first, as the subtraction does
      double r0, r1;
      if constexpr (DIM == 2) {
        r0 = dfma1(c0, mfour, t0);
        r1 = dfma1(c1, mfour, t1);
      } else {
        r0 = dfma1(twod_x<DIM>(c0), mone, t0);
        r1 = dfma1(twod_x<DIM>(c1), mone, t1);
      }
      if constexpr (STORE_R) {
        const float rf0 = d2f(r0), rf1 = d2f(r1);
        if (v1) {
          store_r<TR>(rout + lc + x, rf0);
          store_r<TR>(rout + lc + x + 1, rf1);
        } else if (v0) {
          store_r<TR>(rout + lc + x, rf0);
        }
      }
      if constexpr (RESID) {
        // r^2 summed per lane over a group of kResGroup lines (line order,
        // point order), then across the warp by a fixed butterfly: one
        // partial per (group, 64-point segment), the same for any work split
        if (v0) qacc = __fma_rn(r0, r0, qacc);
        if (v1) qacc = __fma_rn(r1, r1, qacc);
        if ((m + 1) % kResGroup == 0 || m + 1 == G.extent) {
          double q = qacc;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) q = add(q, __shfl_xor_sync(FULL_MASK, q, o));
          if (lane == 0) {
            const int64_t grp = (int64_t)B.pg + m / kResGroup;
            const int64_t row = DIM == 2 ? grp : grp * S->ny + (B.oy + y);
            S->part[B.part + row * S->part_row + it.seg] = q;
          }
          qacc = 0.0;
        }
      }
    }
    if (!more) break;
    double nn0, nn1;
    src.fin2(nnr, nn0, nn1);
    fin_aux(an);
    A0p = A0;
    A1p = A1;
    p0 = c0;
    p1 = c1;
    c0 = n0;
    c1 = last0 ? an.eg : n1;
    n0 = nn0;
    n1 = nn1;
    a = an;
  }
}

template <int DIM, int MODE, bool PUSH, bool RESID, typename TE, typename TR, int EMU = 0>
__global__ void __launch_bounds__(kThreads, DIM == 2 && (MODE == kModeSweep || MODE == kModeOuter) ? 3
                                            : (MODE == kModeOuter ? 2 : 1))
k_f64(const WorkItem* __restrict__ items, int nitems, int kpar, const BlockDev* __restrict__ blocks,
      const SolveDev* __restrict__ solves, int epar) {
  __shared__ double colp[kWarps][kMarchLines];
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (w >= nitems) return;
  const WorkItem it = items[w];
  if (!solves[blocks[it.block].solve].active) return;
  f64_item<DIM, MODE, PUSH, RESID, TE, TR, false, EMU, false, true>(it, blocks, solves, kpar, epar, nullptr, nullptr,
                                                                   0, colp[threadIdx.x >> 5]);
}

// 2D FP64 sweep over march items: one warp per (block, range of lines),
// computing every 64-point segment of the block in turn.  The pairs
// lane 31 leaves in shared memory for the next segment alternate between two
// buffers, so a segment never overwrites what it is still reading.
template <int DIM, bool PUSH>
__global__ void __launch_bounds__(kThreads, 3)
k_f64_march(const WorkItem* __restrict__ items, int nitems, int kpar, const BlockDev* __restrict__ blocks,
            const SolveDev* __restrict__ solves, int pf) {
  __shared__ double pairs[kWarps][2][kMarchLines];
  const int wi = threadIdx.x >> 5;
  const int w = blockIdx.x * kWarps + wi;
  if (w >= nitems) return;
  WorkItem it = items[w];
  if (!solves[blocks[it.block].solve].active) return;
  const int nseg = (blocks[it.block].bx + kSegF64 - 1) / kSegF64;
  for (int sg = 0; sg < nseg; ++sg) {
    it.seg = (int16_t)sg;
    f64_item<DIM, kModeSweep, PUSH, false, float, float, false, 0, true>(it, blocks, solves, kpar, 0,
                                                                         pairs[wi][(sg + 1) & 1], pairs[wi][sg & 1], pf);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// 2D FP64 sweep over march items, four points per lane (128-point segments).
//
// The same canonical arithmetic as f64_item, with the per-line work that is
// not FP64 arithmetic (addresses, loads, shuffles, the edge lanes, the warp
// vote of the exact division, the loop) spread over four points instead of
// two: on GB300 that overhead, not the FP64 pipe, limited the two-point
// march.  Lines are loaded with 32-byte vector loads.  The (W + S) pair of a
// segment's first point comes from shared memory: for the block's first
// segment the warp forms these edge pairs gW[m] + x[m-1][0] for all of its
// lines up front, one line per lane (a handful of FP64 instructions per item
// instead of a one-lane instruction per line); for later segments lane 31 of
// the previous segment left its pair Q(m-1, xs-1) there.
constexpr int kSegF64x4 = 128;


__device__ __forceinline__ void ldg4d(const double* p, double (&v)[4]) {
  asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
}
__device__ __forceinline__ void stg4d(double* p, const double (&v)[4]) {
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
               : "memory");
}
// the valid leading elements of a 4-vector (all four in one store when valid)
__device__ __forceinline__ void st4d_valid(double* p, const double (&v)[4], int nv) {
  if (nv >= 4) {
    stg4d(p, v);
  } else {
    if (nv > 0) p[0] = v[0];
    if (nv > 1) p[1] = v[1];
    if (nv > 2) p[2] = v[2];
  }
}

// One 128-point segment of a march item: lines it.y0 .. it.y0 + it.n - 1.
// STG > 0: x and f of the lines ahead are staged in shared memory by per-lane
// 16-byte asynchronous copies, STG lines ahead (ring `stage`: STG slots of
// 128 x then 128 f values per warp); each lane reads back only the bytes it
// copied itself, so no warp barrier is needed.  STG = 0: register prefetch of
// one line.
__device__ __forceinline__ void cp_async16_g2s(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// V values of a lane from shared memory as float (float: 16-byte aligned
// vector reads; bfloat16: 8- or 16-byte aligned)
template <int V>
__device__ __forceinline__ void unpack_smem(const float* p, float (&o)[V]) {
#pragma unroll
  for (int q = 0; q < V / 4; ++q) {
    const float4 a = *reinterpret_cast<const float4*>(p + 4 * q);
    o[4 * q] = a.x; o[4 * q + 1] = a.y; o[4 * q + 2] = a.z; o[4 * q + 3] = a.w;
  }
}
template <int V>
__device__ __forceinline__ void unpack_smem(const __nv_bfloat16* p, float (&o)[V]) {
  if constexpr (V == 4) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    o[0] = __uint_as_float(u.x << 16); o[1] = __uint_as_float(u.x & 0xFFFF0000u);
    o[2] = __uint_as_float(u.y << 16); o[3] = __uint_as_float(u.y & 0xFFFF0000u);
  } else {
#pragma unroll
    for (int q = 0; q < V / 8; ++q) {
      const uint4 u = *reinterpret_cast<const uint4*>(p + 8 * q);
      const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        o[8 * q + 2 * j] = __uint_as_float(w4[j] << 16);
        o[8 * q + 2 * j + 1] = __uint_as_float(w4[j] & 0xFFFF0000u);
      }
    }
  }
}

// cp.async of 4 or 8 bytes (cache in L1 and L2) or 16 bytes (L2 only)
template <int BYTES>
__device__ __forceinline__ void cp_async_g2s(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (BYTES == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}

// Extra arrays of the 4-point march for the fused-residual sweep (RESID) and
// the refinement's outer step (MODE kModeOuter).  In the outer step the field
// the stencil reads is x_new = x + e, e (type TE) laid out like x, ghost ring
// and columns included, and added only when `apply`; x_new is written and
// r = t - 4 x_new is stored as TR.  RESID: r^2 is summed into the residual
// partials, one per (group of kResGroup lines, 64-point segment), in the
// order and through the butterfly that f64_item uses, so every partial is bit
// for bit the one the per-segment items write.
template <typename TE, typename TR>
struct March4Ext {
  const TE* __restrict__ e;
  TR* __restrict__ r;
  double* __restrict__ part;
  int64_t part_off;  // B.part + B.pg * part_row
  int part_row;
  bool apply;
};

// doubles per staged line group of a warp: 128 x and 128 f values, and in the
// outer step 128 e values
template <int MODE, typename TE>
__host__ __device__ constexpr int march4_slot_doubles() {
  return MODE == kModeOuter ? 256 + 128 * (int)sizeof(TE) / 8 : 256;
}

// four low-precision values as float (16- or 8-byte vector load)
template <typename TE>
__device__ __forceinline__ void ld4_low(const TE* p, float (&v)[4]) {
  const float4 a = ldf4<false>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}

// the valid leading values of four r values (one vector store when all four are)
__device__ __forceinline__ void st4r_valid(float* p, const float (&v)[4], int nv) {
  if (nv >= 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    if (nv > 0) p[0] = v[0];
    if (nv > 1) p[1] = v[1];
    if (nv > 2) p[2] = v[2];
  }
}
__device__ __forceinline__ void st4r_valid(__nv_bfloat16* p, const float (&v)[4], int nv) {
  if (nv >= 4) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 u;
    memcpy(&u.x, &a, 4);
    memcpy(&u.y, &b, 4);
    *reinterpret_cast<uint2*>(p) = u;
  } else {
    if (nv > 0) p[0] = __float2bfloat16_rn(v[0]);
    if (nv > 1) p[1] = __float2bfloat16_rn(v[1]);
    if (nv > 2) p[2] = __float2bfloat16_rn(v[2]);
  }
}

template <bool PUSH, int STG, int MODE = kModeSweep, bool RESID = false, typename TE = float, typename TR = float>
__device__ __forceinline__ void f64_march4_seg(const WorkItem& it, int sg, const BlockDev& B,
                                               const BlockDev* __restrict__ blocks, const double* __restrict__ xsrc,
                                               double* __restrict__ xd, const double* __restrict__ f,
                                               const double* rd, double* wr, double one, int pf,
                                               double* stage = nullptr, const March4Ext<TE, TR>* ex = nullptr) {
  constexpr bool OUTER = MODE == kModeOuter;
  constexpr int SLOT = march4_slot_doubles<MODE, TE>();
  constexpr int NST = STG > 0 ? STG : 1;
  auto add = [one](double u, double v) { return dadd1(u, v, one); };
  const int lane = threadIdx.x & 31;
  const Geo<2> G(B, 0);
  const int bx = B.bx;
  const int xs = sg * kSegF64x4;
  const int x = xs + 4 * lane;
  const int nv = bx - x;                         // points of this lane: min(nv, 4) when nv > 0
  const bool valid = nv > 0;
  const bool holds_last = nv >= 1 && nv <= 4;    // the block's last point is x + nv - 1
  const bool east_in = lane == 31 && nv > 4;     // east of point 3 is the next segment's first point
  const int64_t gE = B.xoff + (int64_t)B.by;     // 2D: the east ghost column, one value per line
  bool apply = false;                            // outer step: x_new = x + e
  if constexpr (OUTER) apply = ex->apply;
  // the W / E neighbours' ghost columns, written every line by the lanes
  // holding the block's first and last points (the S / N neighbours' ghost
  // lines are looked up on the block's first and last line only)
  int64_t w_col = -1, e_col = -1;
  if constexpr (PUSH) {
    if (x == 0 && B.nbr[0] >= 0) {
      const BlockDev& N = blocks[B.nbr[0]];
      w_col = N.xoff + (int64_t)N.by * N.bz;
    }
    if (holds_last && B.nbr[1] >= 0) e_col = blocks[B.nbr[1]].xoff;
  }
  const int m0 = it.y0, mend = m0 + it.n;

  auto load4 = [&](int64_t o, double (&v)[4]) {
    v[0] = v[1] = v[2] = v[3] = 0.0;
    if (valid) ldg4d(xsrc + o, v);
  };
  auto loadf = [&](int64_t o, double (&v)[4]) {
    v[0] = v[1] = v[2] = v[3] = 0.0;
    if (valid) ldg4d(f + o, v);
  };
  // e at a lane's four points (outer step, once a correction exists)
  auto load4e = [&](int64_t o, float (&v)[4]) {
    v[0] = v[1] = v[2] = v[3] = 0.f;
    if constexpr (OUTER) {
      if (apply && valid) ld4_low(ex->e + o, v);
    }
  };
  auto load1e = [&](int64_t o) -> float {
    if constexpr (OUTER) {
      if (apply) return ldf<false>(ex->e + o);
    }
    return 0.f;
  };
  // x_new = x + e at a lane's four points; called by every lane (one warp
  // vote for the four integer-pipe conversions)
  auto fin4 = [&](double (&v)[4], const float (&ev)[4]) {
    if constexpr (OUTER) {
      if (apply) {
        double d[4];
        bool ok[4], all = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          d[k] = f64_from_bits(f32_to_f64_bits(__float_as_uint(ev[k]), ok[k]));
          all = all && ok[k];
        }
        if (!__all_sync(FULL_MASK, all)) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (!ok[k]) d[k] = slow_f2d(ev[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = add(v[k], d[k]);
      }
    }
  };
  // x + e of one value (edge lanes only: the plain conversion)
  auto fin1 = [&](double v, float e1) {
    if constexpr (OUTER) {
      if (apply) return add(v, (double)e1);
    }
    return v;
  };
  // the same called by every lane (the integer-pipe conversion with a warp vote)
  auto fin1w = [&](double v, float e1) {
    if constexpr (OUTER) {
      if (apply) return add(v, f2d(e1));
    }
    return v;
  };
  // staged form: group j holds x of line j + 1 and f of line j (and in the
  // outer step e of line j + 1)
  auto issue = [&](int j) {
    if constexpr (STG > 0) {
      if (j < mend && valid) {
        double* d = stage + ((unsigned)(j - m0) % (unsigned)NST) * SLOT + 4 * lane;
        const double* sx = xsrc + G.line(j + 1) + x;
        const double* sf = f + G.line(j) + x;
        cp_async16_g2s(d, sx);
        cp_async16_g2s(d + 2, sx + 2);
        cp_async16_g2s(d + 128, sf);
        cp_async16_g2s(d + 130, sf + 2);
        if constexpr (OUTER) {
          if (apply)
            cp_async_g2s<4 * (int)sizeof(TE)>(reinterpret_cast<TE*>(stage + ((unsigned)(j - m0) % (unsigned)NST) * SLOT + 256) + 4 * lane,
                                              ex->e + G.line(j + 1) + x);
        }
      }
      cp_async_commit_group();
    }
  };
  // x (and e) of line j + 1 from group j; f of line j is read where the line
  // is computed (staged_f), just before group j's slot is reissued
  auto staged = [&](int j, double (&xv)[4], float (&ev)[4]) {
    const double* d = stage + ((unsigned)(j - m0) % (unsigned)NST) * SLOT + 4 * lane;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xv[k] = valid ? d[k] : 0.0;
      ev[k] = 0.f;
    }
    if constexpr (OUTER) {
      if (apply && valid)
        unpack_smem<4>(reinterpret_cast<const TE*>(stage + ((unsigned)(j - m0) % (unsigned)NST) * SLOT + 256) + 4 * lane, ev);
    }
  };
  auto staged_f = [&](int j, double (&fv)[4]) {
    const double* d = stage + ((unsigned)(j - m0) % (unsigned)NST) * SLOT + 128 + 4 * lane;
#pragma unroll
    for (int k = 0; k < 4; ++k) fv[k] = valid ? d[k] : 0.0;
  };
  // prologue: lines m0 - 1 (p), m0 (c), m0 + 1 (n); pairs Q(m0 - 1, x_k);
  // fc: f of line m0 (register form only)
  double p[4], c[4], n[4], fc[4], Qp[4];
  {
    float ep[4], ec[4], en0[4];
    load4(G.line(m0 - 1) + x, p);
    load4(G.line(m0) + x, c);
    load4e(G.line(m0 - 1) + x, ep);
    load4e(G.line(m0) + x, ec);
    if constexpr (STG > 0) {
#pragma unroll
      for (int j = 0; j < STG; ++j) issue(m0 + j);
      cp_async_wait_group<NST - 1>();
      staged(m0, n, en0);
    } else {
      load4(G.line(m0 + 1) + x, n);
      loadf(G.line(m0) + x, fc);
      load4e(G.line(m0 + 1) + x, en0);
    }
    fin4(p, ep);
    fin4(c, ec);
    fin4(n, en0);
  }
  double ce = 0.0, ge = 0.0, pe = 0.0;
  if (east_in) {
    ce = fin1(__ldg(xsrc + G.line(m0) + x + 4), load1e(G.line(m0) + x + 4));
    pe = fin1(__ldg(xsrc + G.line(m0 - 1) + x + 4), load1e(G.line(m0 - 1) + x + 4));
  }
  if (holds_last) ge = fin1(__ldg(xsrc + gE + m0), load1e(gE + m0));
  {
    double pn = __shfl_down_sync(FULL_MASK, p[0], 1);
    if (east_in) pn = pe;
    Qp[0] = add(p[1], c[0]);
    Qp[1] = add(p[2], c[1]);
    Qp[2] = add(p[3], c[2]);
    Qp[3] = add(pn, c[3]);
  }
  double mfour = 0.0;  // -4 in a register (residual)
  if constexpr (RESID || OUTER) mfour = __dmul_rn(one, -4.0);
  double qa0 = 0.0, qa1 = 0.0;  // RESID: this lane's r^2 of points 0-1 and of points 2-3 over the current group
#pragma unroll 1
  for (int m = m0; m < mend; ++m) {
    const bool more = m + 1 < mend;
    // lines pf steps ahead of the register loads into L2 (within this item's
    // lines and the ghost line after them)
    if (pf > 0 && lane == 0) {
      const uint32_t bytes = (uint32_t)min(kSegF64x4, B.pitch - xs) * 8u;
      if (m + 2 + pf <= mend) l2_prefetch(xsrc + G.line(m + 2 + pf) + xs, bytes);
      if (m + 1 + pf < mend) l2_prefetch(f + G.line(m + 1 + pf) + xs, bytes);
    }
    // loads for the next line: x of line m + 2, f and the edge values of line m + 1
    double nn[4], fn[4];
    float en[4];
    double cen = 0.0, gen = 0.0;
    float cee = 0.f, gee = 0.f;
    if (more) {
      if constexpr (STG == 0) {
        load4(G.line(m + 2) + x, nn);
        loadf(G.line(m + 1) + x, fn);
        load4e(G.line(m + 2) + x, en);
      }
      if (east_in) {
        cen = __ldg(xsrc + G.line(m + 1) + x + 4);
        cee = load1e(G.line(m + 1) + x + 4);
      }
      if (holds_last) {
        gen = __ldg(xsrc + gE + m + 1);
        gee = load1e(gE + m + 1);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        nn[k] = fn[k] = 0.0;
        en[k] = 0.f;
      }
    }
    // Q(m, x_k) = x[m][x_k + 1] + x[m + 1][x_k]; the block's last point takes the ghost
    double ceast = __shfl_down_sync(FULL_MASK, c[0], 1);
    if (east_in) ceast = ce;
    double ck[4] = {c[1], c[2], c[3], ceast};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (holds_last && k == nv - 1) ck[k] = ge;
    double Q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) Q[k] = add(ck[k], n[k]);
    // (W + S) of point 0: the left lane's pair, or for lane 0 the pair in shared memory
    double w0 = __shfl_up_sync(FULL_MASK, Qp[3], 1);
    if (lane == 31) wr[m - m0] = Qp[3];
    if (lane == 0) w0 = rd[m - m0];
    double fm[4];  // f of line m
    if constexpr (STG > 0) {
      staged_f(m, fm);
      issue(m + STG);  // group m + STG into the slot group m leaves now
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) fm[k] = fc[k];
    }
    double t[4];
    t[0] = add(add(w0, Q[0]), fm[0]);
    t[1] = add(add(Qp[0], Q[1]), fm[1]);
    t[2] = add(add(Qp[1], Q[2]), fm[2]);
    t[3] = add(add(Qp[2], Q[3]), fm[3]);
    double o[4];
    if constexpr (MODE == kModeSweep) {
      // t / 4 on the integer pipe; one warp vote for the four points
      bool fast = true;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint64_t b = f64_bits(t[k]);
        o[k] = quarter_bits(b);
        fast = fast && (quarter_fast(b) || k >= nv);
      }
      if (!__all_sync(FULL_MASK, fast)) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < nv && !quarter_fast(f64_bits(t[k]))) o[k] = slow_quarter(t[k]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) o[k] = c[k];  // outer step: the updated iterate itself
    }
    if (valid) {
      st4d_valid(xd + G.line(m) + x, o, nv);
      if constexpr (PUSH) {
        if (m == 0) {  // the S neighbour's north ghost line
          const int nb = __ldg(&blocks[it.block].nbr[2]);
          if (nb >= 0) {
            const BlockDev& N = blocks[nb];
            st4d_valid(xd + N.off + (int64_t)(N.by + 1) * N.pitch + x, o, nv);
          }
        }
        if (m == G.extent - 1) {  // the N neighbour's south ghost line
          const int nb = __ldg(&blocks[it.block].nbr[3]);
          if (nb >= 0) st4d_valid(xd + blocks[nb].off + x, o, nv);
        }
        if (w_col >= 0) xd[w_col + m] = o[0];
        if (e_col >= 0) {
          double last = o[0];
#pragma unroll
          for (int k = 1; k < 4; ++k)
            if (k == nv - 1) last = o[k];
          xd[e_col + m] = last;
        }
      }
    }
    if constexpr (RESID || OUTER) {
      // r = t - 4 c rounded once, as fma(c, -4, t) (4 c is exact)
      double r[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = dfma1(c[k], mfour, t[k]);
      if constexpr (OUTER) {
        float rf[4];
        bool okf[4], allf = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          rf[k] = __uint_as_float(f64_to_f32_bits(f64_bits(r[k]), okf[k]));
          allf = allf && (okf[k] || k >= nv);
        }
        if (!__all_sync(FULL_MASK, allf)) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (k < nv && !okf[k]) rf[k] = slow_d2f(r[k]);
        }
        if (valid) st4r_valid(ex->r + G.line(m) + x, rf, nv);
      }
      if constexpr (RESID) {
        // points 0-1 and 2-3 of this lane are the two points of lanes
        // 2l and 2l + 1 of f64_item's 64-point segment (lanes 0-15 form
        // segment 2 sg, lanes 16-31 segment 2 sg + 1)
        if (nv > 0) qa0 = __fma_rn(r[0], r[0], qa0);
        if (nv > 1) qa0 = __fma_rn(r[1], r[1], qa0);
        if (nv > 2) qa1 = __fma_rn(r[2], r[2], qa1);
        if (nv > 3) qa1 = __fma_rn(r[3], r[3], qa1);
        if ((m + 1) % kResGroup == 0 || m + 1 == G.extent) {
          // f64_item's butterfly over 32 lanes (xor 16, 8, 4, 2, 1) is, on
          // these lanes, xor 8, 4, 2, 1 then the lane's own two sums
#pragma unroll
          for (int s = 8; s > 0; s >>= 1) {
            qa0 = add(qa0, __shfl_xor_sync(FULL_MASK, qa0, s));
            qa1 = add(qa1, __shfl_xor_sync(FULL_MASK, qa1, s));
          }
          const double q = add(qa0, qa1);
          const int half = lane >> 4;
          if ((lane & 15) == 0 && xs + 64 * half < bx)
            ex->part[ex->part_off + (int64_t)(m / kResGroup) * ex->part_row + 2 * sg + half] = q;
          qa0 = 0.0;
          qa1 = 0.0;
        }
      }
    }
    if constexpr (STG > 0) {
      if (more) {
        cp_async_wait_group<NST - 1>();  // group m + 1 has landed
        staged(m + 1, nn, en);
      }
    }
    if constexpr (OUTER) {
      if (more) fin4(nn, en);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Qp[k] = Q[k];
      c[k] = n[k];
      n[k] = nn[k];
      fc[k] = fn[k];
    }
    if constexpr (OUTER) {
      // lane 31's east value and the last point's ghost: one instruction
      const double v = fin1w(east_in ? cen : gen, east_in ? cee : gee);
      ce = v;
      ge = v;
    } else {
      ce = cen;
      ge = gen;
    }
  }
  if constexpr (STG > 0) cp_async_wait_group<0>();  // nothing may still target this warp's ring
}

constexpr int kMarchStages = 4;  // lines staged ahead by the shared-memory form of the 4-point march

// MODE kModeSweep without RESID: the plain sweep; with RESID: the sweep that
// also writes the residual partials of its input.  MODE kModeOuter (RESID):
// the refinement's outer step, e from buffer epar.
//
// wstart == nullptr: warp w computes item w (nwarps = the item count).
// Otherwise warp w computes items wstart[w] .. wstart[w + 1] - 1 in turn: the
// lines of all blocks are dealt out in equal runs, one per resident warp, and
// a run that crosses a block boundary is two items, so every warp (and every
// SM) gets the same share of the sweep.
template <bool PUSH, int STG, int MODE = kModeSweep, bool RESID = false, typename TE = float, typename TR = float>
__global__ void __launch_bounds__(kThreads, 2)
k_f64_march4(const WorkItem* __restrict__ items, int nwarps, const int* __restrict__ wstart, int kpar,
             const BlockDev* __restrict__ blocks, const SolveDev* __restrict__ solves, int pf, int epar) {
  constexpr bool OUTER = MODE == kModeOuter;
  constexpr int SLOT = march4_slot_doubles<MODE, TE>();
  __shared__ double pairs[kWarps][2][kMarchLines];
  extern __shared__ __align__(16) double march_stage[];  // STG * SLOT doubles per warp when STG > 0
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.x * kWarps + wi;
  if (w >= nwarps) return;
  int k0 = w, k1 = w + 1;
  if (wstart) {
    k0 = wstart[w];
    k1 = wstart[w + 1];
  }
  const double one = load_one();
  for (int k = k0; k < k1; ++k) {
    const WorkItem it = items[k];
    const BlockDev B = blocks[it.block];
    const SolveDev* S = solves + B.solve;
    if (!S->active) continue;
    const int par = (S->phase + kpar) & 1;
    const double* __restrict__ xsrc = S->x[par];
    double* __restrict__ xd = S->x[par ^ 1];
    March4Ext<TE, TR> ex{};
    if constexpr (OUTER || RESID) {
      if constexpr (OUTER) {
        ex.e = reinterpret_cast<const TE*>(S->e[epar]);
        ex.r = reinterpret_cast<TR*>(S->r);
        ex.apply = S->apply_e != 0;
      }
      ex.part = S->part;
      ex.part_off = B.part + (int64_t)B.pg * S->part_row;
      ex.part_row = S->part_row;
    }
    // (W + S) pairs of the block's first column, x[m][-1] + x[m - 1][0], one
    // line per lane, into the buffer lane 0 of segment 0 reads
    const Geo<2> G(B, 0);
    for (int j = lane; j < it.n; j += 32) {
      const int m = it.y0 + j;
      double wv = __ldg(xsrc + B.xoff + m), sv = __ldg(xsrc + G.line(m - 1));
      if constexpr (OUTER) {
        if (ex.apply) {
          wv = dadd1(wv, (double)ldf<false>(ex.e + B.xoff + m), one);
          sv = dadd1(sv, (double)ldf<false>(ex.e + G.line(m - 1)), one);
        }
      }
      pairs[wi][1][j] = dadd1(wv, sv, one);
    }
    __syncwarp();
    const int nseg = (B.bx + kSegF64x4 - 1) / kSegF64x4;
    for (int sg = 0; sg < nseg; ++sg) {
      f64_march4_seg<PUSH, STG, MODE, RESID, TE, TR>(it, sg, B, blocks, xsrc, xd, S->f, pairs[wi][(sg + 1) & 1],
                                                     pairs[wi][sg & 1], one, pf,
                                                     STG > 0 ? march_stage + wi * STG * SLOT : nullptr, &ex);
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// Low-precision inner sweep of the refinement: A e = r with zero Dirichlet
// ghosts, FP32 arithmetic, e stored as TE (float or bfloat16, RNE), r read as
// TR.  Four points per lane, 128 per warp row.  FIRST: the input e is zero,
// so only r is read (e' = (0 + r) / 2d).

// Vector access of V consecutive low-precision values (V = 4 or 8): 16-byte
// loads for bfloat16 and for float with V = 4, two for float with V = 8.
template <bool COH, int V>
__device__ __forceinline__ void ldv(const float* p, float (&o)[V]) {
  const float4 a = ldf4<COH>(p);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  if constexpr (V == 8) {
    const float4 b = ldf4<COH>(p + 4);
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
}
template <bool COH, int V>
__device__ __forceinline__ void ldv(const __nv_bfloat16* p, float (&o)[V]) {
  if constexpr (V == 4) {
    const float4 a = ldf4<COH>(p);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  } else {
    uint4 u;
    if constexpr (COH) u = __ldcg(reinterpret_cast<const uint4*>(p));
    else u = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[2 * k] = __uint_as_float(w[k] << 16);
      o[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
    }
  }
}
template <int V>
__device__ __forceinline__ void stv(float* p, const float (&v)[V], int nvalid) {
  if (nvalid >= V) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    if constexpr (V == 8) *reinterpret_cast<float4*>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k)
      if (k < nvalid) p[k] = v[k];
  }
}
template <int V>
__device__ __forceinline__ void stv(__nv_bfloat16* p, const float (&v)[V], int nvalid) {
  if (nvalid >= V) {
    uint32_t w[V / 2];
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
      memcpy(&w[k], &h, 4);
    }
    if constexpr (V == 8) *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    else *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k)
      if (k < nvalid) p[k] = __float2bfloat16_rn(v[k]);
  }
}

// Points per lane of the low-precision sweeps: 4 float or 8 bfloat16 (16-byte
// loads of e).
template <typename TE>
__host__ __device__ constexpr int low_vpl() {
  return sizeof(TE) == 2 ? 8 : 4;
}

template <int DIM, bool FIRST, bool PUSH, typename TE, typename TR, bool COH>
__device__ __forceinline__ void low_item(const WorkItem& it, const BlockDev* __restrict__ blocks,
                                         const SolveDev* __restrict__ solves, int epar) {
  constexpr int V = low_vpl<TE>();
  const int lane = threadIdx.x & 31;
  const BlockDev B = blocks[it.block];
  const SolveDev* S = solves + B.solve;
  const TE* __restrict__ es = reinterpret_cast<const TE*>(S->e[epar ^ 1]);
  TE* __restrict__ ed = reinterpret_cast<TE*>(S->e[epar]);
  const TR* __restrict__ rr = reinterpret_cast<const TR*>(S->r);

  // 3D: a block row narrower than a warp row takes L = 2^lgL lanes and the
  // warp computes 32 / L adjacent rows y0, y0+1, ... (lanes of rows past the
  // block's last row stay idle); 2D: one row of 32 lanes
  const int lgL = DIM == 3 ? low_lanes_log2(B.bx, V) : 5;
  const int L = 1 << lgL;
  const int l = lane & (L - 1);
  const int y = DIM == 3 ? it.y0 + (lane >> lgL) : it.y0;
  const bool row_ok = DIM == 2 || y < B.by;
  const Geo<DIM> G(B, DIM == 2 ? y : (row_ok ? y : B.by - 1));
  const int bx = B.bx;
  const int xs = it.seg * (L * V);
  const int x = xs + V * l;
  const int nvalid = DIM == 2 ? bx - x : (row_ok ? bx - x : 0);  // > 0 when the lane holds points
  const bool any = nvalid > 0;
  const int64_t gW = B.xoff;
  const int64_t gE = B.xoff + (int64_t)B.by * B.bz;
  // halo push: the W / E ghost columns are kept by the lanes holding the
  // block's first and last points; the march-axis faces and (3D) the side
  // rows are looked up on the lines that write them
  const int yrow = DIM == 2 ? y : (row_ok ? y : B.by - 1);
  int64_t w_col = -1, e_col = -1;
  if constexpr (PUSH) {
    if (x == 0 && any && B.nbr[0] >= 0) {
      const BlockDev& N = blocks[B.nbr[0]];
      w_col = N.xoff + (int64_t)N.by * N.bz;  // the west neighbour's east ghost column
    }
    if (any && nvalid <= V && B.nbr[1] >= 0) e_col = blocks[B.nbr[1]].xoff;  // the east neighbour's west column
  }
  // the halo push of line m (values o of this lane's points)
  auto push = [&](int m, int col, const float (&o)[V]) {
    constexpr int lo = DIM == 2 ? 2 : 4;  // the march-axis faces
    if (m == 0) {
      const int nb = __ldg(&blocks[it.block].nbr[lo]);
      if (nb >= 0) {
        const Geo<DIM> GN(blocks[nb], yrow);
        stv<V>(ed + GN.line(GN.extent) + x, o, nvalid);
      }
    }
    if (m == G.extent - 1) {
      const int nb = __ldg(&blocks[it.block].nbr[lo + 1]);
      if (nb >= 0) {
        const Geo<DIM> GN(blocks[nb], yrow);
        stv<V>(ed + GN.line(-1) + x, o, nvalid);
      }
    }
    if constexpr (DIM == 3) {
      if (yrow == 0) {  // the S neighbour's north ghost row of plane m
        const int nb = __ldg(&blocks[it.block].nbr[2]);
        if (nb >= 0) {
          const BlockDev& N = blocks[nb];
          stv<V>(ed + N.off + (int64_t)(N.by + 1) * N.pitch + (int64_t)(m + 1) * N.plane + x, o, nvalid);
        }
      }
      if (yrow == B.by - 1) {  // the N neighbour's south ghost row of plane m
        const int nb = __ldg(&blocks[it.block].nbr[3]);
        if (nb >= 0) {
          const BlockDev& N = blocks[nb];
          stv<V>(ed + N.off + (int64_t)(m + 1) * N.plane + x, o, nvalid);
        }
      }
    }
    if (w_col >= 0) ed[w_col + col] = from_f<TE>(o[0]);
    if (e_col >= 0) {
      float last = o[0];
#pragma unroll
      for (int k = 1; k < V; ++k)
        if (k == nvalid - 1) last = o[k];
      ed[e_col + col] = from_f<TE>(last);
    }
  };

  const int m0 = DIM == 2 ? it.y0 : it.z0;
  const int mend = m0 + it.n;
  float p[V], c[V];
#pragma unroll
  for (int k = 0; k < V; ++k) p[k] = c[k] = 0.f;
  if constexpr (!FIRST) {
    if (any) {
      ldv<COH, V>(es + G.line(m0 - 1) + x, p);
      ldv<COH, V>(es + G.line(m0) + x, c);
    }
  }
  if constexpr (DIM == 3 && !FIRST && V == 4) {
    // Float in 3D: every load line m + 1 needs (r, e of line m + 2, the rows
    // y - 1 and y + 1, the edge scalars) is issued before line m is computed,
    // so a warp keeps two lines of loads in flight (measured 1.24x at 512^3;
    // with 8 bfloat16 per lane the second line's registers cost more
    // occupancy than the prefetch gains, and 4 per lane is slower still).
    struct Ln {
      float r[V], n[V], sa[V], sb[V];
      float wv, ev, ge;
    };
    auto fetch = [&](int m, Ln& q) {
      const int64_t lc = G.line(m);
      const int col = G.col(m);
#pragma unroll
      for (int k = 0; k < V; ++k) q.r[k] = q.n[k] = q.sa[k] = q.sb[k] = 0.f;
      q.wv = q.ev = q.ge = 0.f;
      if (any) {
        ldv<false, V>(rr + lc + x, q.r);
        ldv<COH, V>(es + G.line(m + 1) + x, q.n);
        ldv<COH, V>(es + lc - G.side + x, q.sa);
        ldv<COH, V>(es + lc + G.side + x, q.sb);
        if (l == 0) q.wv = xs > 0 ? ldf<COH>(es + lc + xs - 1) : ldf<COH>(es + gW + col);
        if (l == L - 1 && x + V < bx) q.ev = ldf<COH>(es + lc + x + V);
        if (nvalid <= V) q.ge = ldf<COH>(es + gE + col);
      }
    };
    Ln cur;
    fetch(m0, cur);
    for (int m = m0; m < mend; ++m) {
      const int64_t lc = G.line(m);
      const int col = G.col(m);
      Ln nx;
      const bool more = m + 1 < mend;
      if (more) fetch(m + 1, nx);
      float wv = __shfl_up_sync(FULL_MASK, c[V - 1], 1, L);
      if (l == 0) wv = cur.wv;
      float ev = __shfl_down_sync(FULL_MASK, c[0], 1, L);
      if (l == L - 1 && x + V < bx) ev = cur.ev;
      float o[V];
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const float west = k == 0 ? wv : c[k - 1];
        float east = k == V - 1 ? ev : c[k + 1];
        if (k + 1 == nvalid) east = cur.ge;  // the block's last point takes the ghost
        float t = __fadd_rn(__fadd_rn(west, p[k]), __fadd_rn(east, cur.n[k]));
        t = __fadd_rn(t, __fadd_rn(cur.sa[k], cur.sb[k]));
        t = __fadd_rn(t, cur.r[k]);
        o[k] = jdivf<DIM>(t);
      }
      if (any) {
        stv<V>(ed + lc + x, o, nvalid);
        if constexpr (PUSH) push(m, col, o);
      }
      if (!more) break;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        p[k] = c[k];
        c[k] = cur.n[k];
      }
      cur = nx;
    }
  } else {
    for (int m = m0; m < mend; ++m) {
      const int64_t lc = G.line(m);
      const int col = G.col(m);
      float rv[V], o[V];
#pragma unroll
      for (int k = 0; k < V; ++k) rv[k] = 0.f;
      if (any) ldv<false, V>(rr + lc + x, rv);  // r is read-only during every sweep
      float n[V];
#pragma unroll
      for (int k = 0; k < V; ++k) n[k] = 0.f;
      if constexpr (FIRST) {
#pragma unroll
        for (int k = 0; k < V; ++k) o[k] = jdivf<DIM>(__fadd_rn(0.0f, rv[k]));
      } else {
        if (any) ldv<COH, V>(es + G.line(m + 1) + x, n);
        float sa[V], sb[V];
#pragma unroll
        for (int k = 0; k < V; ++k) sa[k] = sb[k] = 0.f;
        if constexpr (DIM == 3) {
          if (any) {
            ldv<COH, V>(es + lc - G.side + x, sa);
            ldv<COH, V>(es + lc + G.side + x, sb);
          }
        }
        // west of point 0, east of point V-1 (in 3D the shuffles stay inside
        // the row's L lanes; the 2D forms are written apart, as the compiler
        // schedules the plain ones measurably better)
        float wv, ev;
        if constexpr (DIM == 2) {
          wv = __shfl_up_sync(FULL_MASK, c[V - 1], 1);
          if (lane == 0) wv = xs > 0 ? ldf<COH>(es + lc + xs - 1) : ldf<COH>(es + gW + col);
          ev = __shfl_down_sync(FULL_MASK, c[0], 1);
          if (lane == 31 && x + V < bx) ev = ldf<COH>(es + lc + x + V);
        } else {
          wv = __shfl_up_sync(FULL_MASK, c[V - 1], 1, L);
          if (l == 0 && any) wv = xs > 0 ? ldf<COH>(es + lc + xs - 1) : ldf<COH>(es + gW + col);
          ev = __shfl_down_sync(FULL_MASK, c[0], 1, L);
          if (l == L - 1 && any && x + V < bx) ev = ldf<COH>(es + lc + x + V);
        }
        float ge = 0.f;
        if (any && nvalid <= V) ge = ldf<COH>(es + gE + col);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const float west = k == 0 ? wv : c[k - 1];
          float east = k == V - 1 ? ev : c[k + 1];
          if (k + 1 == nvalid) east = ge;  // the block's last point takes the ghost
          float t = __fadd_rn(__fadd_rn(west, p[k]), __fadd_rn(east, n[k]));
          if constexpr (DIM == 3) t = __fadd_rn(t, __fadd_rn(sa[k], sb[k]));
          t = __fadd_rn(t, rv[k]);
          o[k] = jdivf<DIM>(t);
        }
      }
      if (any) {
        stv<V>(ed + lc + x, o, nvalid);
        if constexpr (PUSH) push(m, col, o);
      }
      if constexpr (!FIRST) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
          p[k] = c[k];
          c[k] = n[k];
        }
      }
  }
}
}

// Launch bounds measured per form: bfloat16 in 2D runs best held to 4 CTAs
// per SM, float in 2D best with no occupancy hint at all (k_low_free).
template <int DIM, bool FIRST, bool PUSH, typename TE, typename TR>
__global__ void __launch_bounds__(kThreads, DIM == 2 && sizeof(TE) == 2 ? 4 : 1)
k_low(const WorkItem* __restrict__ items, int nitems, const BlockDev* __restrict__ blocks,
      const SolveDev* __restrict__ solves, int epar) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (w >= nitems) return;
  const WorkItem it = items[w];
  if (!solves[blocks[it.block].solve].active) return;
  low_item<DIM, FIRST, PUSH, TE, TR, false>(it, blocks, solves, epar);
}
template <int DIM, bool FIRST, bool PUSH, typename TE, typename TR>
__global__ void __launch_bounds__(kThreads)
k_low_free(const WorkItem* __restrict__ items, int nitems, const BlockDev* __restrict__ blocks,
           const SolveDev* __restrict__ solves, int epar) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (w >= nitems) return;
  const WorkItem it = items[w];
  if (!solves[blocks[it.block].solve].active) return;
  low_item<DIM, FIRST, PUSH, TE, TR, false>(it, blocks, solves, epar);
}

// ---------------------------------------------------------------------------
// 3D inner sweep (not the first of a refinement step) with each lane's lines
// staged ahead in shared memory.  For line m a lane needs, at its own V
// points, e of line m + 1, e of the rows y - 1 and y + 1 on line m, and r of
// line m.  It copies exactly those bytes with 16-byte asynchronous copies,
// low_s3_stages lines ahead, into its own slots of a per-warp ring, and reads
// back only what it copied, so no barrier is needed, and the bytes in flight
// hold no registers (the register form of low_item keeps one line ahead in
// registers, which caps it at 2 CTAs per SM).  Items, arithmetic and halo
// push are low_item's: bit-identical results.
// lines staged ahead (measured at 512^3: float 305.7 us per sweep with 3,
// 350.8 with 4, 382.5 with 6; bfloat16 351.4 with 3, 342.5 with 4)
template <typename TE>
__host__ __device__ constexpr int low_s3_stages() {
  return sizeof(TE) == 4 ? 3 : 4;
}

// bytes of one line group of a warp: e of line m + 1, e of the rows y - 1 and
// y + 1 (16 bytes per lane each), r (V values per lane)
template <typename TE, typename TR>
__host__ __device__ constexpr int low_s3_slot_bytes() {
  return 32 * (3 * 16 + low_vpl<TE>() * (int)sizeof(TR));
}

template <bool PUSH, typename TE, typename TR>
__global__ void __launch_bounds__(kThreads, sizeof(TE) == 4 ? 3 : 2)
k_low_s3(const WorkItem* __restrict__ items, int nitems, const BlockDev* __restrict__ blocks,
         const SolveDev* __restrict__ solves, int epar) {
  extern __shared__ __align__(16) unsigned char s3_smem[];
  constexpr int V = low_vpl<TE>();
  constexpr int RB = V * (int)sizeof(TR);  // bytes of r per lane and line
  constexpr int SLOT = low_s3_slot_bytes<TE, TR>();
  constexpr int NST = low_s3_stages<TE>();
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.x * kWarps + wi;
  if (w >= nitems) return;
  const WorkItem it = items[w];
  const BlockDev B = blocks[it.block];
  const SolveDev* S = solves + B.solve;
  if (!S->active) return;
  unsigned char* ring = s3_smem + wi * NST * SLOT;
  const TE* __restrict__ es = reinterpret_cast<const TE*>(S->e[epar ^ 1]);
  TE* __restrict__ ed = reinterpret_cast<TE*>(S->e[epar]);
  const TR* __restrict__ rr = reinterpret_cast<const TR*>(S->r);

  // a block row narrower than a warp row takes L = 2^lgL lanes and the warp
  // computes 32 / L adjacent rows (as in low_item)
  const int lgL = low_lanes_log2(B.bx, V);
  const int L = 1 << lgL;
  const int l = lane & (L - 1);
  const int y = it.y0 + (lane >> lgL);
  const bool row_ok = y < B.by;
  const int yrow = row_ok ? y : B.by - 1;
  const Geo<3> G(B, yrow);
  const int bx = B.bx;
  const int xs = it.seg * (L * V);
  const int x = xs + V * l;
  const int nvalid = row_ok ? bx - x : 0;  // > 0 when the lane holds points
  const bool any = nvalid > 0;
  const int64_t gW = B.xoff;
  const int64_t gE = B.xoff + (int64_t)B.by * B.bz;
  int64_t w_col = -1, e_col = -1;
  if constexpr (PUSH) {
    if (x == 0 && any && B.nbr[0] >= 0) {
      const BlockDev& N = blocks[B.nbr[0]];
      w_col = N.xoff + (int64_t)N.by * N.bz;  // the west neighbour's east ghost column
    }
    if (any && nvalid <= V && B.nbr[1] >= 0) e_col = blocks[B.nbr[1]].xoff;  // the east neighbour's west column
  }
  const int m0 = it.z0, mend = m0 + it.n;

  auto slot = [&](int j) { return ring + ((unsigned)(j - m0) % (unsigned)NST) * SLOT; };
  auto issue = [&](int j) {
    if (j < mend && any) {
      unsigned char* d = slot(j);
      const int64_t lc = G.line(j);
      cp_async_g2s<16>(d + lane * 16, es + G.line(j + 1) + x);
      cp_async_g2s<16>(d + 512 + lane * 16, es + lc - G.side + x);
      cp_async_g2s<16>(d + 1024 + lane * 16, es + lc + G.side + x);
      cp_async_g2s<16>(d + 1536 + lane * RB, rr + lc + x);
      if constexpr (RB == 32) cp_async_g2s<16>(d + 1536 + lane * RB + 16, rr + lc + x + 16 / (int)sizeof(TR));
    }
    cp_async_commit_group();
  };
  // the edge scalars of line m: west of point 0 (lane 0 of the row), east of
  // point V - 1 (the row's last lane, when the row goes on), the east ghost
  struct Edge {
    float wv, ev, ge;
  };
  auto fetch_edge = [&](int m, Edge& q) {
    q.wv = q.ev = q.ge = 0.f;
    if (any) {
      const int64_t lc = G.line(m);
      const int col = G.col(m);
      if (l == 0) q.wv = xs > 0 ? ldf<false>(es + lc + xs - 1) : ldf<false>(es + gW + col);
      if (l == L - 1 && x + V < bx) q.ev = ldf<false>(es + lc + x + V);
      if (nvalid <= V) q.ge = ldf<false>(es + gE + col);
    }
  };

  float p[V], c[V];
#pragma unroll
  for (int k = 0; k < V; ++k) p[k] = c[k] = 0.f;
  if (any) {
    ldv<false, V>(es + G.line(m0 - 1) + x, p);
    ldv<false, V>(es + G.line(m0) + x, c);
  }
#pragma unroll
  for (int j = 0; j < NST; ++j) issue(m0 + j);
  Edge cur;
  fetch_edge(m0, cur);
#pragma unroll 1
  for (int m = m0; m < mend; ++m) {
    const int64_t lc = G.line(m);
    const int col = G.col(m);
    const bool more = m + 1 < mend;
    Edge nx;
    nx.wv = nx.ev = nx.ge = 0.f;
    if (more) fetch_edge(m + 1, nx);
    cp_async_wait_group<NST - 1>();  // group m has landed
    float n[V], sa[V], sb[V], rv[V];
#pragma unroll
    for (int k = 0; k < V; ++k) n[k] = sa[k] = sb[k] = rv[k] = 0.f;
    if (any) {
      const unsigned char* d = slot(m);
      unpack_smem<V>(reinterpret_cast<const TE*>(d + lane * 16), n);
      unpack_smem<V>(reinterpret_cast<const TE*>(d + 512 + lane * 16), sa);
      unpack_smem<V>(reinterpret_cast<const TE*>(d + 1024 + lane * 16), sb);
      unpack_smem<V>(reinterpret_cast<const TR*>(d + 1536 + lane * RB), rv);
    }
    issue(m + NST);  // group m + NST into the slot group m leaves
    float wv = __shfl_up_sync(FULL_MASK, c[V - 1], 1, L);
    if (l == 0) wv = cur.wv;
    float ev = __shfl_down_sync(FULL_MASK, c[0], 1, L);
    if (l == L - 1 && x + V < bx) ev = cur.ev;
    float o[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float west = k == 0 ? wv : c[k - 1];
      float east = k == V - 1 ? ev : c[k + 1];
      if (k + 1 == nvalid) east = cur.ge;  // the block's last point takes the ghost
      float t = __fadd_rn(__fadd_rn(west, p[k]), __fadd_rn(east, n[k]));
      t = __fadd_rn(t, __fadd_rn(sa[k], sb[k]));
      t = __fadd_rn(t, rv[k]);
      o[k] = jdivf<3>(t);
    }
    if (any) {
      stv<V>(ed + lc + x, o, nvalid);
      if constexpr (PUSH) {
        if (m == 0) {  // the D neighbour's upper ghost plane
          const int nb = __ldg(&blocks[it.block].nbr[4]);
          if (nb >= 0) {
            const Geo<3> GN(blocks[nb], yrow);
            stv<V>(ed + GN.line(GN.extent) + x, o, nvalid);
          }
        }
        if (m == G.extent - 1) {  // the U neighbour's lower ghost plane
          const int nb = __ldg(&blocks[it.block].nbr[5]);
          if (nb >= 0) {
            const Geo<3> GN(blocks[nb], yrow);
            stv<V>(ed + GN.line(-1) + x, o, nvalid);
          }
        }
        if (yrow == 0) {  // the S neighbour's north ghost row of plane m
          const int nb = __ldg(&blocks[it.block].nbr[2]);
          if (nb >= 0) {
            const BlockDev& N = blocks[nb];
            stv<V>(ed + N.off + (int64_t)(N.by + 1) * N.pitch + (int64_t)(m + 1) * N.plane + x, o, nvalid);
          }
        }
        if (yrow == B.by - 1) {  // the N neighbour's south ghost row of plane m
          const int nb = __ldg(&blocks[it.block].nbr[3]);
          if (nb >= 0) {
            const BlockDev& N = blocks[nb];
            stv<V>(ed + N.off + (int64_t)(m + 1) * N.plane + x, o, nvalid);
          }
        }
        if (w_col >= 0) ed[w_col + col] = from_f<TE>(o[0]);
        if (e_col >= 0) {
          float last = o[0];
#pragma unroll
          for (int k = 1; k < V; ++k)
            if (k == nvalid - 1) last = o[k];
          ed[e_col + col] = from_f<TE>(last);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      p[k] = c[k];
      c[k] = n[k];
    }
    cur = nx;
  }
  cp_async_wait_group<0>();  // nothing may still target this warp's ring
}

// ---------------------------------------------------------------------------
// Two inner sweeps in one pass (temporal blocking, 2D): e2 = J(J(e0)) with
// J(e)_p = (((W + S) + (E + N)) + r_p) / 4, the arithmetic of low_item.  The
// intermediate e1 never leaves shared memory and is rounded to the storage
// type TE exactly as a stored e1 would be, so the result is bit-identical to
// two separate sweeps; e0 and r are read once and e2 written once, against
// twice each for two sweeps.
//
// One CTA per tile of kTbTH lines x kTbTW points of one block:
//   1. e0 on the tile and a two-point ring, r on the tile and a one-point
//      ring, into shared memory (as float).  Ring points outside the block
//      are read where they live: the neighbour block's second row or column,
//      its r, the corners of its ghost rows (so the layout needs no deeper
//      ghost ring).  Ring points no later step reads are left 0.
//   2. e1 on the tile and its one-point ring (0 on a domain face: the zero
//      Dirichlet values of the correction).
//   3. e2 on the tile, stored with the same halo push as low_item.
// FIRST: e0 = 0, so e1 = (0 + r) / 4 and e0 is not read.  The input buffer is
// never written: e2 and its push go to the other buffer.
constexpr int kTbTW = kTbTileW;       // points per tile along x (4 per lane)
constexpr int kTbTH = kTbTileH;       // lines per tile
constexpr int kTbSP = kTbTW + 8;      // shared row stride: x = xs - 4 .. xs + kTbTW + 3, xs at index 4

// one (or, persistent, two) buffers of e0 and r, one of e1
template <typename TE, typename TR, bool PERSIST>
__host__ __device__ constexpr int tb2_smem_bytes() {
  return ((PERSIST ? 2 : 1) * ((kTbTH + 4) * (int)sizeof(TE) + (kTbTH + 2) * (int)sizeof(TR)) + (kTbTH + 2) * 4) *
         kTbSP;
}

// e1 = RN_TE(v), as stored and read back by a separate sweep
template <typename TE>
__device__ __forceinline__ float round_store(float v) {
  if constexpr (sizeof(TE) == 2) return __bfloat162float(__float2bfloat16_rn(v));
  else return v;
}

// e0 at (x, y) of block B's neighbourhood, x in [-2, bx + 1], y in [-2, by + 1]
template <typename TE>
__device__ float tb_e0(const TE* __restrict__ es, const BlockDev* __restrict__ blocks, const BlockDev& B, int x,
                       int y) {
  const int bx = B.bx, by = B.by;
  if (x >= 0 && x < bx) {
    if (y >= -1 && y <= by) return ldf<false>(es + B.off + (int64_t)(y + 1) * B.pitch + x);
    if (y == -2 && B.nbr[2] >= 0) {
      const BlockDev& Sb = blocks[B.nbr[2]];
      return ldf<false>(es + Sb.off + (int64_t)(Sb.by - 1) * Sb.pitch + x);  // S's line by_S - 2
    }
    if (y == by + 1 && B.nbr[3] >= 0) {
      const BlockDev& Nb = blocks[B.nbr[3]];
      return ldf<false>(es + Nb.off + 2 * (int64_t)Nb.pitch + x);  // N's line 1
    }
    return 0.f;
  }
  if (y < -1 || y > by) return 0.f;
  if (x == -1) {
    if (y >= 0 && y < by) return ldf<false>(es + B.xoff + y);  // the west ghost column
    if (B.nbr[0] < 0) return 0.f;
    const BlockDev& W = blocks[B.nbr[0]];
    return ldf<false>(es + W.off + (int64_t)(y + 1) * W.pitch + W.bx - 1);  // corner of W's ghost row
  }
  if (x == bx) {
    if (y >= 0 && y < by) return ldf<false>(es + B.xoff + by + y);  // the east ghost column
    if (B.nbr[1] < 0) return 0.f;
    const BlockDev& E = blocks[B.nbr[1]];
    return ldf<false>(es + E.off + (int64_t)(y + 1) * E.pitch);  // corner of E's ghost row
  }
  if (y < 0 || y >= by) return 0.f;  // (x = -2 or bx + 1) beside a ghost row: never read
  if (x == -2 && B.nbr[0] >= 0) {
    const BlockDev& W = blocks[B.nbr[0]];
    return W.bx >= 2 ? ldf<false>(es + W.off + (int64_t)(y + 1) * W.pitch + W.bx - 2) : ldf<false>(es + W.xoff + y);
  }
  if (x == bx + 1 && B.nbr[1] >= 0) {
    const BlockDev& E = blocks[B.nbr[1]];
    return E.bx >= 2 ? ldf<false>(es + E.off + (int64_t)(y + 1) * E.pitch + 1)
                     : ldf<false>(es + E.xoff + E.by + y);
  }
  return 0.f;
}

// r at (x, y), x in [-1, bx], y in [-1, by] (0 at the ring's corners, never read)
template <typename TR>
__device__ float tb_r(const TR* __restrict__ rr, const BlockDev* __restrict__ blocks, const BlockDev& B, int x, int y) {
  const int bx = B.bx, by = B.by;
  if (x >= 0 && x < bx) {
    if (y >= 0 && y < by) return ldf<false>(rr + B.off + (int64_t)(y + 1) * B.pitch + x);
    if (y == -1 && B.nbr[2] >= 0) {
      const BlockDev& Sb = blocks[B.nbr[2]];
      return ldf<false>(rr + Sb.off + (int64_t)Sb.by * Sb.pitch + x);  // S's line by_S - 1
    }
    if (y == by && B.nbr[3] >= 0) {
      const BlockDev& Nb = blocks[B.nbr[3]];
      return ldf<false>(rr + Nb.off + (int64_t)Nb.pitch + x);  // N's line 0
    }
    return 0.f;
  }
  if (y < 0 || y >= by) return 0.f;
  if (x == -1 && B.nbr[0] >= 0) {
    const BlockDev& W = blocks[B.nbr[0]];
    return ldf<false>(rr + W.off + (int64_t)(y + 1) * W.pitch + W.bx - 1);
  }
  if (x == bx && B.nbr[1] >= 0) {
    const BlockDev& E = blocks[B.nbr[1]];
    return ldf<false>(rr + E.off + (int64_t)(y + 1) * E.pitch);
  }
  return 0.f;
}

// 4 values of a line, x .. x + 3 (vector load; float or bfloat16)
template <typename T>
__device__ __forceinline__ void tb_ld4(const T* p, float (&v)[4]) {
  ldv<false, 4>(p, v);
}


// PERSIST = false (default): one CTA per tile, one buffer; the loads of a
// tile are all in flight at once and the resident CTAs of an SM overlap one
// another's phases.  PERSIST = true: CTAs walk the tile table (tile
// blockIdx.x, then every gridDim.x-th) and issue the next tile's loads into
// the other of two buffers before computing the current one (measured slower
// at 8192^2: fewer resident CTAs, and four barriers per tile serialise them).
template <bool PUSH, bool FIRST, typename TE, typename TR, bool PERSIST>
__global__ void __launch_bounds__(kThreads)
k_low_tb2(const WorkItem* __restrict__ tiles, int ntiles, const BlockDev* __restrict__ blocks,
          const SolveDev* __restrict__ solves, int in_par, int out_par) {
  extern __shared__ __align__(16) unsigned char tb_smem[];
  constexpr int E0B = (kTbTH + 4) * kTbSP * (int)sizeof(TE);  // bytes of one e0 buffer
  constexpr int RB = (kTbTH + 2) * kTbSP * (int)sizeof(TR);   // bytes of one r buffer
  float* E1 = reinterpret_cast<float*>(tb_smem + (PERSIST ? 2 : 1) * (E0B + RB));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int xi = 4 + 4 * lane;  // shared-memory index of a lane's 4 points

  // issue the loads of tile t into buffer b: line copies (asynchronous) and
  // this thread's ring point (a plain load into `hv`, stored later at `hidx`)
  auto issue = [&](int t, int b, float& hv, int& hidx, bool& h_is_r) {
    hidx = -1;
    h_is_r = false;
    if (t < ntiles) {
      const WorkItem tile = tiles[t];
      const BlockDev& B = blocks[tile.block];
      const SolveDev* S = solves + B.solve;
      if (S->active) {
        const TE* __restrict__ es = reinterpret_cast<const TE*>(S->e[in_par]);
        const TR* __restrict__ rr = reinterpret_cast<const TR*>(S->r);
        TE* E0 = reinterpret_cast<TE*>(tb_smem + b * (E0B + RB));
        TR* R = reinterpret_cast<TR*>(tb_smem + b * (E0B + RB) + E0B);
        const int bx = B.bx, by = B.by;
        const int64_t pitch = B.pitch;
        const int xs = tile.seg * kTbTW, tw = min(kTbTW, bx - xs);
        const int y0 = tile.y0, th = tile.n;
        const int nS = B.nbr[2], nN = B.nbr[3];
        const int x = xs + 4 * lane;
        if constexpr (!FIRST) {
          for (int j = warp; j < th + 4; j += kWarps) {
            const int y = y0 - 2 + j;
            int64_t base = -1;
            if (y >= -1 && y <= by) base = B.off + (int64_t)(y + 1) * pitch;
            else if (y == -2 && nS >= 0) base = blocks[nS].off + (int64_t)(blocks[nS].by - 1) * pitch;
            else if (y == by + 1 && nN >= 0) base = blocks[nN].off + 2 * pitch;
            TE* d = E0 + j * kTbSP + xi;
            if (base >= 0 && x < xs + tw) {
              cp_async_g2s<4 * (int)sizeof(TE)>(d, es + base + x);
            } else {
#pragma unroll
              for (int k = 0; k < 4; ++k) d[k] = from_f<TE>(0.f);
            }
          }
        }
        for (int j = warp; j < th + 2; j += kWarps) {
          const int y = y0 - 1 + j;
          int64_t base = -1;
          if (y >= 0 && y < by) base = B.off + (int64_t)(y + 1) * pitch;
          else if (y == -1 && nS >= 0) base = blocks[nS].off + (int64_t)blocks[nS].by * pitch;
          else if (y == by && nN >= 0) base = blocks[nN].off + pitch;
          TR* d = R + j * kTbSP + xi;
          if (base >= 0 && x < xs + tw) {
            cp_async_g2s<4 * (int)sizeof(TR)>(d, rr + base + x);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = from_f<TR>(0.f);
          }
        }
        // ring points: (th + 4) lines x 4 of e0, then (th + 2) lines x 2 of r
        const int ne = FIRST ? 0 : (th + 4) * 4, nr = (th + 2) * 2;
        const int q = threadIdx.x;
        if (q < ne) {
          const int j = q >> 2, h = q & 3;
          const int hx = h < 2 ? xs - 2 + h : xs + tw + h - 2;
          hv = tb_e0(es, blocks, B, hx, y0 - 2 + j);
          hidx = j * kTbSP + hx - xs + 4;
        } else if (q < ne + nr) {
          const int j = (q - ne) >> 1, h = (q - ne) & 1;
          const int hx = h == 0 ? xs - 1 : xs + tw;
          hv = tb_r(rr, blocks, B, hx, y0 - 1 + j);
          hidx = j * kTbSP + hx - xs + 4;
          h_is_r = true;
        }
      }
    }
    cp_async_commit_group();
  };

  int t = blockIdx.x;
  float hv = 0.f;
  int hidx = -1;
  bool h_is_r = false;
  issue(t, 0, hv, hidx, h_is_r);
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    const int b = PERSIST ? (it & 1) : 0;
    // loads of the next tile into the other buffer, then wait for this one's
    float hv_n = 0.f;
    int hidx_n = -1;
    bool h_is_r_n = false;
    if constexpr (PERSIST) {
      issue(t + gridDim.x, b ^ 1, hv_n, hidx_n, h_is_r_n);
      cp_async_wait_group<1>();
    } else {
      cp_async_wait_group<0>();
    }
    __syncthreads();  // this tile's line copies have landed: its ring points go on top
    const WorkItem tile = tiles[t];
    const BlockDev& B = blocks[tile.block];
    const SolveDev* S = solves + B.solve;
    const bool active = S->active != 0;
    TE* E0 = reinterpret_cast<TE*>(tb_smem + b * (E0B + RB));
    TR* R = reinterpret_cast<TR*>(tb_smem + b * (E0B + RB) + E0B);
    if (hidx >= 0) {
      if (h_is_r) R[hidx] = from_f<TR>(hv);
      else E0[hidx] = from_f<TE>(hv);
    }
    __syncthreads();
    const int bx = B.bx, by = B.by;
    const int64_t pitch = B.pitch;
    const int xs = tile.seg * kTbTW, tw = min(kTbTW, bx - xs);
    const int y0 = tile.y0, th = tile.n;
    const int nW = B.nbr[0], nE = B.nbr[1], nS = B.nbr[2], nN = B.nbr[3];
    const int x = xs + 4 * lane;
    if (active) {
      // 2. e1 on lines y0 - 1 .. y0 + th, points xs - 1 .. xs + tw
      for (int j = warp; j < th + 2; j += kWarps) {
        const int y = y0 - 1 + j;
        const bool ylive = (y >= 0 && y < by) || (y == -1 && nS >= 0) || (y == by && nN >= 0);
        const TE* c = E0 + (j + 1) * kTbSP;
        const TR* r = R + j * kTbSP;
        float* o = E1 + j * kTbSP;
        float e1v[4] = {0.f, 0.f, 0.f, 0.f};
        if (ylive) {
          float rk[4];
          unpack_smem<4>(r + xi, rk);
          if constexpr (FIRST) {
#pragma unroll
            for (int k = 0; k < 4; ++k) e1v[k] = round_store<TE>(jdivf<2>(__fadd_rn(0.0f, rk[k])));
          } else {
            float cv[4], sk[4], nk[4];
            unpack_smem<4>(c + xi, cv);
            unpack_smem<4>(c - kTbSP + xi, sk);
            unpack_smem<4>(c + kTbSP + xi, nk);
            const float ck[6] = {to_f(c[xi - 1]), cv[0], cv[1], cv[2], cv[3], to_f(c[xi + 4])};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float tt = __fadd_rn(__fadd_rn(__fadd_rn(ck[k], sk[k]), __fadd_rn(ck[k + 2], nk[k])), rk[k]);
              e1v[k] = round_store<TE>(jdivf<2>(tt));
            }
          }
        }
        *reinterpret_cast<float4*>(o + xi) = make_float4(e1v[0], e1v[1], e1v[2], e1v[3]);
        if (lane < 2) {  // the ring points x = xs - 1, xs + tw (after the vector store: they may overlap it)
          const int hx = lane == 0 ? xs - 1 : xs + tw;
          const int i = hx - xs + 4;
          const bool xlive = (hx >= 0 && hx < bx) || (hx == -1 && nW >= 0) || (hx == bx && nE >= 0);
          float v = 0.f;
          if (ylive && xlive) {
            float tt;
            if constexpr (FIRST) tt = __fadd_rn(0.0f, to_f(r[i]));
            else
              tt = __fadd_rn(__fadd_rn(__fadd_rn(to_f(c[i - 1]), to_f(c[i - kTbSP])),
                                       __fadd_rn(to_f(c[i + 1]), to_f(c[i + kTbSP]))),
                             to_f(r[i]));
            v = round_store<TE>(jdivf<2>(tt));
          }
          o[i] = v;
        }
      }
    }
    __syncthreads();
    if (active) {
      // 3. e2 on lines y0 .. y0 + th - 1
      TE* __restrict__ ed = reinterpret_cast<TE*>(S->e[out_par]);
      PushTargets T;
      if constexpr (PUSH) push_targets<2>(T, B, blocks, 0);
      const int nvalid = xs + tw - x;  // > 0 when this lane holds points
      for (int j = warp; j < th; j += kWarps) {
        const int y = y0 + j;
        const float* c = E1 + (j + 1) * kTbSP;
        const float4 cv = *reinterpret_cast<const float4*>(c + xi);
        const float4 sv = *reinterpret_cast<const float4*>(c - kTbSP + xi);
        const float4 nv = *reinterpret_cast<const float4*>(c + kTbSP + xi);
        float rk[4];
        unpack_smem<4>(R + (j + 1) * kTbSP + xi, rk);
        const float ck[6] = {c[xi - 1], cv.x, cv.y, cv.z, cv.w, c[xi + 4]};
        const float sk[4] = {sv.x, sv.y, sv.z, sv.w}, nk[4] = {nv.x, nv.y, nv.z, nv.w};
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          o[k] = jdivf<2>(__fadd_rn(__fadd_rn(__fadd_rn(ck[k], sk[k]), __fadd_rn(ck[k + 2], nk[k])), rk[k]));
        if (nvalid > 0) {
          const int64_t lc = B.off + (int64_t)(y + 1) * pitch;
          stv<4>(ed + lc + x, o, nvalid);
          if constexpr (PUSH) {
            if (y == 0 && T.lo_line >= 0) stv<4>(ed + T.lo_line + x, o, nvalid);
            if (y == by - 1 && T.hi_line >= 0) stv<4>(ed + T.hi_line + x, o, nvalid);
            if (x == 0 && T.w_col >= 0) ed[T.w_col + y] = from_f<TE>(o[0]);
            if (xs + tw == bx && nvalid <= 4 && T.e_col >= 0) {
              float last = o[0];
#pragma unroll
              for (int k = 1; k < 4; ++k)
                if (k == nvalid - 1) last = o[k];
              ed[T.e_col + y] = from_f<TE>(last);
            }
          }
        }
      }
    }
    if constexpr (!PERSIST) break;  // one tile per CTA
    __syncthreads();  // buffer b and E1 are free for the tile after next
    hv = hv_n;
    hidx = hidx_n;
    h_is_r = h_is_r_n;
  }
  cp_async_wait_group<0>();  // the last (empty) group: nothing may still target shared memory
}

// ---------------------------------------------------------------------------
// Two inner sweeps in one pass, 3D: e2 = J(J(e0)) with J(e)_p =
// ((((W + D) + (E + U)) + (S + N)) + r_p) / 6, the arithmetic of low_item,
// bit-identical to two separate sweeps.  One CTA per (x, y) tile of
// kT3W x kT3H points and kTb3TileZ planes of one block marches along z (one
// plane further on each side for e1, two for e0: the neighbours' boundary
// planes at the block's faces): at step z it forms e1 on plane z (the tile and
// a one-point ring) and e2 on plane z - 1.  e0 planes (two-point
// ring) and r planes (one-point ring) arrive kT3PD steps ahead: whole lines by
// asynchronous copies into rings of kT3NS planes in shared memory, ring points
// one per thread by plain loads kept in registers until their plane's copies
// have landed.  Points outside the block are read where they live
// (tblock3.cuh); e1 is 0 on domain faces.
}  // namespace jgb
#include "tblock3.cuh"
namespace jgb {

constexpr int kT3W = kTb3TileW;           // x points per tile (16 threads x 4)
constexpr int kT3H = kTb3TileH;           // y rows per tile
constexpr int kT3SP = kT3W + 8;           // shared row stride, x = xs - 4 .. xs + kT3W + 3, xs at index 4
constexpr int kT3NS = 5;                  // planes in the e0 and r rings
constexpr int kT3PD = 2;                  // planes loaded ahead
constexpr int kT3E0P = (kT3H + 4) * kT3SP;  // elements of one e0 plane (rows y0 - 2 ..)
constexpr int kT3RP = (kT3H + 2) * kT3SP;   // elements of one r or e1 plane (rows y0 - 1 ..)

template <typename TE, typename TR>
__host__ __device__ constexpr int tb3_smem_bytes() {
  return kT3NS * kT3E0P * (int)sizeof(TE) + kT3NS * kT3RP * (int)sizeof(TR) + 3 * kT3RP * 4;
}

template <bool PUSH, bool FIRST, typename TE, typename TR>
__global__ void __launch_bounds__(kThreads)
k_low_tb3(const WorkItem* __restrict__ tiles, int ntiles, const BlockDev* __restrict__ blocks,
          const SolveDev* __restrict__ solves, int in_par, int out_par) {
  extern __shared__ __align__(16) unsigned char tb_smem[];
  if ((int)blockIdx.x >= ntiles) return;
  const WorkItem tile = tiles[blockIdx.x];
  const BlockDev& B = blocks[tile.block];
  const SolveDev* S = solves + B.solve;
  if (!S->active) return;
  const TE* __restrict__ es = reinterpret_cast<const TE*>(S->e[in_par]);
  TE* __restrict__ ed = reinterpret_cast<TE*>(S->e[out_par]);
  const TR* __restrict__ rr = reinterpret_cast<const TR*>(S->r);
  TE* E0 = reinterpret_cast<TE*>(tb_smem);
  TR* R = reinterpret_cast<TR*>(tb_smem + kT3NS * kT3E0P * sizeof(TE));
  float* E1 = reinterpret_cast<float*>(tb_smem + kT3NS * kT3E0P * sizeof(TE) + kT3NS * kT3RP * sizeof(TR));
  const int t = threadIdx.x;
  const int bx = B.bx, by = B.by, bz = B.bz;
  const int xs = tile.seg * kT3W, tw = min(kT3W, bx - xs);
  const int y0 = tile.y0, th = tile.n;
  // this tile's planes: e2 on z0 .. z1 - 1, e1 on z0 - 1 .. z1, e0 on z0 - 2 .. z1 + 1
  const int z0 = tile.z0, z1 = min(z0 + kTb3TileZ, bz);
  const int c4 = t & 15, x = xs + 4 * c4, xi = 4 + 4 * c4;  // this thread's 4-point chunk of a row

  // group q (q = z0 - 2 .. z1 + 1): e0 plane q (rows y0 - 2 .. y0 + th + 1) and
  // r plane q (rows y0 - 1 .. y0 + th, q in [-1, bz]) into ring slot (q + 2) % kT3NS
  auto issue = [&](int q) {
    if (q <= z1 + 1) {
      const int slot = (q + 2) % kT3NS;
      if constexpr (!FIRST) {
        for (int w = t; w < (th + 4) * 16; w += kThreads) {
          const int j = w >> 4, xc = xs + 4 * (w & 15);
          TE* d = E0 + slot * kT3E0P + j * kT3SP + 4 + 4 * (w & 15);
          const int64_t base = tb3_eline(blocks, B, y0 - 2 + j, q);
          if (base >= 0 && xc < xs + tw) {
            cp_async_g2s<4 * (int)sizeof(TE)>(d, es + base + xc);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = from_f<TE>(0.f);
          }
        }
      }
      if (q >= -1 && q <= bz) {
        for (int w = t; w < (th + 2) * 16; w += kThreads) {
          const int j = w >> 4, xc = xs + 4 * (w & 15);
          TR* d = R + slot * kT3RP + j * kT3SP + 4 + 4 * (w & 15);
          const int64_t base = tb3_rline(blocks, B, y0 - 1 + j, q);
          if (base >= 0 && xc < xs + tw) {
            cp_async_g2s<4 * (int)sizeof(TR)>(d, rr + base + xc);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = from_f<TR>(0.f);
          }
        }
      }
    }
    cp_async_commit_group();
  };
  // this thread's ring point of group q: e0 at x = xs - 2, xs - 1, xs + tw,
  // xs + tw + 1 of each row, then r at x = xs - 1, xs + tw
  struct Ring {
    float v;
    int idx;  // element index in the e0 ring, or in the r ring (is_r), or -1
    bool is_r;
  };
  auto ring_load = [&](int q) {
    Ring g{0.f, -1, false};
    if (q > z1 + 1) return g;
    const int slot = (q + 2) % kT3NS;
    const int ne = FIRST ? 0 : (th + 4) * 4, nr = (q >= -1 && q <= bz) ? (th + 2) * 2 : 0;
    if (t < ne) {
      const int j = t >> 2, h = t & 3;
      const int hx = h < 2 ? xs - 2 + h : xs + tw + h - 2;
      const int y = y0 - 2 + j;
      if (hx >= 0 && hx < bx) {
        const int64_t base = tb3_eline(blocks, B, y, q);
        g.v = base >= 0 ? ldf<false>(es + base + hx) : 0.f;
      } else {
        g.v = tb3_e0_xring(es, blocks, B, hx, y, q);
      }
      g.idx = slot * kT3E0P + j * kT3SP + hx - xs + 4;
    } else if (t < ne + nr) {
      const int j = (t - ne) >> 1, h = (t - ne) & 1;
      const int hx = h == 0 ? xs - 1 : xs + tw;
      const int y = y0 - 1 + j;
      if (hx >= 0 && hx < bx) {
        const int64_t base = tb3_rline(blocks, B, y, q);
        g.v = base >= 0 ? ldf<false>(rr + base + hx) : 0.f;
      } else {
        g.v = tb3_r_xring(rr, blocks, B, hx, y, q);
      }
      g.idx = slot * kT3RP + j * kT3SP + hx - xs + 4;
      g.is_r = true;
    }
    return g;
  };
  auto ring_store = [&](const Ring& g) {
    if (g.idx < 0) return;
    if (g.is_r) R[g.idx] = from_f<TR>(g.v);
    else E0[g.idx] = from_f<TE>(g.v);
  };
  // e1 is computed at (x, y, z): inside the block, or one cell outside along
  // one axis where that neighbour exists
  auto live = [&](int px, int py, int pz) {
    const int ox = px < 0 ? 0 : (px >= bx ? 1 : -1);
    const int oy = py < 0 ? 2 : (py >= by ? 3 : -1);
    const int oz = pz < 0 ? 4 : (pz >= bz ? 5 : -1);
    const int nout = (ox >= 0) + (oy >= 0) + (oz >= 0);
    if (nout == 0) return true;
    if (nout > 1) return false;
    const int f = ox >= 0 ? ox : (oy >= 0 ? oy : oz);
    return B.nbr[f] >= 0;
  };
  // prologue: groups -2 .. kT3PD - 1; the ring points of groups -2 and -1 go
  // on top once their copies have landed, those of the next kT3PD groups wait
  // in registers (g0: group z + 1 at step z, g1: group z + 2)
  static_assert(kT3PD == 2, "the ring-point register pipeline holds two groups");
  for (int q = z0 - 2; q < z0 + kT3PD; ++q) issue(q);
  const Ring gm2 = ring_load(z0 - 2), gm1 = ring_load(z0 - 1);
  Ring g0 = ring_load(z0), g1 = ring_load(z0 + 1);
  cp_async_wait_group<kT3PD>();
  __syncthreads();
  ring_store(gm2);
  ring_store(gm1);
  for (int z = z0 - 1; z <= z1; ++z) {
    cp_async_wait_group<kT3PD - 1>();  // this thread's copies of group z + 1 have landed
    __syncthreads();                    // everyone's, and step z - 1 is over
    ring_store(g0);                     // ring points of group z + 1 on top of its lines
    g0 = g1;
    issue(z + 1 + kT3PD);               // into the slot of plane z - 2, free since step z - 1
    g1 = ring_load(z + 1 + kT3PD);
    __syncthreads();
    // e1 on plane z: the tile's rows y0 - 1 .. y0 + th, points xs - 1 .. xs + tw
    {
      const TE* pc = E0 + ((z + 2) % kT3NS) * kT3E0P;
      const TE* pd = E0 + ((z + 1) % kT3NS) * kT3E0P;
      const TE* pu = E0 + ((z + 3) % kT3NS) * kT3E0P;
      const TR* pr = R + ((z + 2) % kT3NS) * kT3RP;
      float* o = E1 + ((z + 3) % 3) * kT3RP;
      const int nmain = (th + 2) * 16, nring = (th + 2) * 2;
      for (int w = t; w < nmain + nring; w += kThreads) {
        if (w < nmain) {
          const int j = w >> 4, c = w & 15, xc = xs + 4 * c, ii = 4 + 4 * c;
          const int y = y0 - 1 + j;
          const int nv = xs + tw - xc;  // valid points of this chunk
          if (nv <= 0) continue;
          float e1v[4] = {0.f, 0.f, 0.f, 0.f};
          if (live(xc, y, z)) {  // x inside the block: only y and z decide
            float rk[4];
            unpack_smem<4>(pr + j * kT3SP + ii, rk);
            if constexpr (FIRST) {
#pragma unroll
              for (int k = 0; k < 4; ++k) e1v[k] = round_store<TE>(jdivf<3>(__fadd_rn(0.0f, rk[k])));
            } else {
              const TE* rowc = pc + (j + 1) * kT3SP;
              float cv[4], sv[4], nk[4], dv[4], uv[4];
              unpack_smem<4>(rowc + ii, cv);
              unpack_smem<4>(rowc - kT3SP + ii, sv);
              unpack_smem<4>(rowc + kT3SP + ii, nk);
              unpack_smem<4>(pd + (j + 1) * kT3SP + ii, dv);
              unpack_smem<4>(pu + (j + 1) * kT3SP + ii, uv);
              const float ck[6] = {to_f(rowc[ii - 1]), cv[0], cv[1], cv[2], cv[3], to_f(rowc[ii + 4])};
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float tt = __fadd_rn(
                    __fadd_rn(__fadd_rn(__fadd_rn(ck[k], dv[k]), __fadd_rn(ck[k + 2], uv[k])), __fadd_rn(sv[k], nk[k])),
                    rk[k]);
                e1v[k] = round_store<TE>(jdivf<3>(tt));
              }
            }
          }
          float* d = o + j * kT3SP + ii;
          if (nv >= 4) {
            *reinterpret_cast<float4*>(d) = make_float4(e1v[0], e1v[1], e1v[2], e1v[3]);
          } else {  // only the valid points: x = xs + tw is the ring's (another thread)
#pragma unroll
            for (int k = 0; k < 3; ++k)
              if (k < nv) d[k] = e1v[k];
          }
        } else {
          const int q2 = w - nmain, j = q2 >> 1;
          const int hx = (q2 & 1) ? xs + tw : xs - 1;
          const int y = y0 - 1 + j, i = hx - xs + 4;
          float v = 0.f;
          if (live(hx, y, z)) {
            const float rv = to_f(pr[j * kT3SP + i]);
            float tt;
            if constexpr (FIRST) {
              tt = __fadd_rn(0.0f, rv);
            } else {
              const TE* rowc = pc + (j + 1) * kT3SP;
              tt = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(to_f(rowc[i - 1]), to_f(pd[(j + 1) * kT3SP + i])),
                                                 __fadd_rn(to_f(rowc[i + 1]), to_f(pu[(j + 1) * kT3SP + i]))),
                                       __fadd_rn(to_f(rowc[i - kT3SP]), to_f(rowc[i + kT3SP]))),
                             rv);
            }
            v = round_store<TE>(jdivf<3>(tt));
          }
          o[j * kT3SP + i] = v;
        }
      }
    }
    __syncthreads();
    // e2 on plane m = z - 1
    const int m = z - 1;
    if (m < z0 || m >= z1) continue;
    const float* qd = E1 + ((z + 1) % 3) * kT3RP;  // e1 plane m - 1
    const float* qc = E1 + ((z + 2) % 3) * kT3RP;  // e1 plane m
    const float* qu = E1 + (z % 3) * kT3RP;        // e1 plane m + 1
    const TR* pr = R + ((z + 1) % kT3NS) * kT3RP;  // r plane m
    for (int w = t; w < th * 16; w += kThreads) {
      const int jj = w >> 4, c = w & 15, xc = xs + 4 * c, ii = 4 + 4 * c;
      const int y = y0 + jj;
      const int nv = xs + tw - xc;
      if (nv <= 0) continue;
      const float* rowc = qc + (jj + 1) * kT3SP;
      const float4 cv = *reinterpret_cast<const float4*>(rowc + ii);
      const float4 sv = *reinterpret_cast<const float4*>(rowc - kT3SP + ii);
      const float4 nv4 = *reinterpret_cast<const float4*>(rowc + kT3SP + ii);
      const float4 dv = *reinterpret_cast<const float4*>(qd + (jj + 1) * kT3SP + ii);
      const float4 uv = *reinterpret_cast<const float4*>(qu + (jj + 1) * kT3SP + ii);
      float rk[4];
      unpack_smem<4>(pr + (jj + 1) * kT3SP + ii, rk);
      const float ck[6] = {rowc[ii - 1], cv.x, cv.y, cv.z, cv.w, rowc[ii + 4]};
      const float sk[4] = {sv.x, sv.y, sv.z, sv.w}, nk[4] = {nv4.x, nv4.y, nv4.z, nv4.w};
      const float dk[4] = {dv.x, dv.y, dv.z, dv.w}, uk[4] = {uv.x, uv.y, uv.z, uv.w};
      float o2[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        o2[k] = jdivf<3>(__fadd_rn(
            __fadd_rn(__fadd_rn(__fadd_rn(ck[k], dk[k]), __fadd_rn(ck[k + 2], uk[k])), __fadd_rn(sk[k], nk[k])), rk[k]));
      stv<4>(ed + b3_at(B, xc, y, m), o2, nv);
      if constexpr (PUSH) {
        if (m == 0 && B.nbr[4] >= 0) {
          const BlockDev& N = blocks[B.nbr[4]];
          stv<4>(ed + b3_at(N, xc, y, N.bz), o2, nv);
        }
        if (m == bz - 1 && B.nbr[5] >= 0) stv<4>(ed + b3_at(blocks[B.nbr[5]], xc, y, -1), o2, nv);
        if (y == 0 && B.nbr[2] >= 0) {
          const BlockDev& N = blocks[B.nbr[2]];
          stv<4>(ed + b3_at(N, xc, N.by, m), o2, nv);
        }
        if (y == by - 1 && B.nbr[3] >= 0) stv<4>(ed + b3_at(blocks[B.nbr[3]], xc, -1, m), o2, nv);
        if (xc == 0 && B.nbr[0] >= 0) {
          const BlockDev& N = blocks[B.nbr[0]];
          ed[N.xoff + (int64_t)N.by * N.bz + (int64_t)m * N.by + y] = from_f<TE>(o2[0]);
        }
        if (xs + tw == bx && nv <= 4 && B.nbr[1] >= 0) {  // this chunk holds the block's last point
          float last = o2[0];
#pragma unroll
          for (int k = 1; k < 4; ++k)
            if (k == nv - 1) last = o2[k];
          ed[blocks[B.nbr[1]].xoff + (int64_t)m * by + y] = from_f<TE>(last);
        }
      }
    }
  }
  cp_async_wait_group<0>();  // only empty groups can be pending; none may outlive the CTA
}

// ---------------------------------------------------------------------------
// Inner sweep with shared-memory staging by bulk asynchronous copies (2D).
//
// The same arithmetic as low_item, but the lines of e and r a warp needs are
// brought into shared memory by 1D bulk copies (cp.async.bulk, completion on
// an mbarrier) up to kTmaStages - 2 lines ahead of the line being computed,
// so the bytes in flight do not cost registers.  Lane 0 of each warp owns its
// warp's ring; every wait is bounded.  A wait that runs out sets bit 1 of
// *status (JACOBI_ERR_TIMEOUT on the host; the outputs of that launch are then
// invalid): the warp stops computing and issuing, waits (bounded) for the
// copies it has in flight, and leaves.

constexpr int kTmaStages = 6;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

template <typename TE, typename TR>
__host__ __device__ constexpr int tma_warp_bytes() {
  return kTmaStages * 32 * low_vpl<TE>() * (int)(sizeof(TE) + sizeof(TR)) + kTmaStages * 8;
}

template <bool PUSH, typename TE, typename TR>
__global__ void __launch_bounds__(kThreads)
k_low_tma(const WorkItem* __restrict__ items, int nitems, const BlockDev* __restrict__ blocks,
          const SolveDev* __restrict__ solves, int epar, uint32_t* status, uint32_t spin_limit) {
  constexpr int V = low_vpl<TE>();
  constexpr int SEGW = 32 * V;
  constexpr int EB = SEGW * (int)sizeof(TE), RB = SEGW * (int)sizeof(TR);
  constexpr int NS = kTmaStages;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = blockIdx.x * kWarps + warp;
  if (w >= nitems) return;  // whole warp; warps never synchronise with each other here
  const WorkItem it = items[w];
  const BlockDev B = blocks[it.block];
  const SolveDev* S = solves + B.solve;
  if (!S->active) return;
  unsigned char* wb = tma_smem + warp * tma_warp_bytes<TE, TR>();
  TE* se = reinterpret_cast<TE*>(wb);                     // NS lines of e
  TR* sr = reinterpret_cast<TR*>(wb + NS * EB);           // NS lines of r
  uint64_t* bars = reinterpret_cast<uint64_t*>(wb + NS * (EB + RB));
  const TE* __restrict__ es = reinterpret_cast<const TE*>(S->e[epar ^ 1]);
  TE* __restrict__ ed = reinterpret_cast<TE*>(S->e[epar]);
  const TR* __restrict__ rr = reinterpret_cast<const TR*>(S->r);

  const Geo<2> G(B, it.y0);
  const int bx = B.bx;
  const int xs = it.seg * SEGW;
  const int x = xs + V * lane;
  const int nvalid = bx - x;
  const bool any = nvalid > 0;
  const int64_t gW = B.xoff;
  const int64_t gE = B.xoff + (int64_t)B.by * B.bz;
  // elements of this segment's lines that exist in the array (a multiple of
  // 16 elements, so every copy is a multiple of 16 bytes)
  const int cnt = min(SEGW, B.pitch - xs);
  PushTargets T;
  if constexpr (PUSH) push_targets<2>(T, B, blocks, it.y0);
  const int m0 = it.y0, mend = m0 + it.n;
  const int L0 = m0 - 1, L1 = mend;  // lines of e needed: L0..L1; lines of r: m0..mend-1

  if (lane == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bars[k]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  auto issue = [&](int L) {  // lane 0: bring line L into stage (L - L0) % NS
    const int st = (L - L0) % NS;
    const bool with_r = L >= m0 && L < mend;
    const uint32_t eb = (uint32_t)(cnt * (int)sizeof(TE)), rb = with_r ? (uint32_t)(cnt * (int)sizeof(TR)) : 0u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bars[st], eb + rb);
    bulk_copy_g2s(se + st * SEGW, es + G.line(L) + xs, eb, &bars[st]);
    if (with_r) bulk_copy_g2s(sr + st * SEGW, rr + G.line(L) + xs, rb, &bars[st]);
  };
  if (lane == 0)
    for (int L = L0; L <= L1 && L < L0 + NS; ++L) issue(L);
  int issued = min(L1, L0 + NS - 1);  // last line whose copies were issued (warp-uniform)
  bool failed = false;
  auto wait_line = [&](int L) {
    const int st = (L - L0) % NS;
    const uint32_t par = (uint32_t)(((L - L0) / NS) & 1);
    uint32_t iters = 0;
    while (!mbar_try_wait(&bars[st], par)) {
      if (++iters > spin_limit) {
        failed = true;
        break;
      }
    }
  };
  auto ld_stage = [&](const TE* p, float (&o)[V]) {  // V values of one line from shared memory
    if constexpr (sizeof(TE) == 4) {
      const float4 a = *reinterpret_cast<const float4*>(p);
      o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else {
      const uint4 u = *reinterpret_cast<const uint4*>(p);
      const uint32_t wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        o[2 * k] = __uint_as_float(wv[k] << 16);
        o[2 * k + 1] = __uint_as_float(wv[k] & 0xFFFF0000u);
      }
    }
  };
  auto ld_stage_r = [&](const TR* p, float (&o)[V]) {
    if constexpr (sizeof(TR) == 4) {
      const float4 a = *reinterpret_cast<const float4*>(p);
      o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
      if constexpr (V == 8) {
        const float4 b = *reinterpret_cast<const float4*>(p + 4);
        o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
      }
    } else {
      const uint4 u = *reinterpret_cast<const uint4*>(p);
      const uint32_t wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        o[2 * k] = __uint_as_float(wv[k] << 16);
        o[2 * k + 1] = __uint_as_float(wv[k] & 0xFFFF0000u);
      }
    }
  };
  // edge scalars of line m, fetched one line ahead
  auto edges = [&](int m, float& wv, float& ev, float& ge) {
    const int64_t lc = G.line(m);
    const int col = G.col(m);
    wv = ev = ge = 0.f;
    if (lane == 0) wv = xs > 0 ? ldf<false>(es + lc + xs - 1) : ldf<false>(es + gW + col);
    if (lane == 31 && x + V < bx) ev = ldf<false>(es + lc + x + V);
    if (any && nvalid <= V) ge = ldf<false>(es + gE + col);
  };
  float p[V], c[V], n[V];
  wait_line(L0);
  wait_line(m0);
  failed = __any_sync(FULL_MASK, failed);
  if (any) {
    ld_stage(se + ((L0 - L0) % NS) * SEGW + V * lane, p);
    ld_stage(se + ((m0 - L0) % NS) * SEGW + V * lane, c);
  }
  float wv, ev, ge;
  edges(m0, wv, ev, ge);
  for (int m = m0; m < mend && !failed; ++m) {
    const int64_t lc = G.line(m);
    const int col = G.col(m);
    float wn = 0.f, en = 0.f, gn = 0.f;
    if (m + 1 < mend) edges(m + 1, wn, en, gn);
    wait_line(m + 1);
    failed = __any_sync(FULL_MASK, failed);
    if (failed) break;  // no new copies: only the ones in flight are drained below
    const int stc = (m - L0) % NS, stn = (m + 1 - L0) % NS;
    float rv[V], o[V];
#pragma unroll
    for (int k = 0; k < V; ++k) n[k] = rv[k] = 0.f;
    if (any) {
      ld_stage(se + stn * SEGW + V * lane, n);
      ld_stage_r(sr + stc * SEGW + V * lane, rv);
    }
    float wl = __shfl_up_sync(FULL_MASK, c[V - 1], 1);
    if (lane == 0) wl = wv;
    float el = __shfl_down_sync(FULL_MASK, c[0], 1);
    if (lane == 31 && x + V < bx) el = ev;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float west = k == 0 ? wl : c[k - 1];
      float east = k == V - 1 ? el : c[k + 1];
      if (k + 1 == nvalid) east = ge;  // the block's last point takes the ghost
      float t = __fadd_rn(__fadd_rn(west, p[k]), __fadd_rn(east, n[k]));
      t = __fadd_rn(t, rv[k]);
      o[k] = jdivf<2>(t);
    }
    // line m-1's stage is free once every lane has read it: refill it
    __syncwarp();
    if (m - 1 + NS <= L1) {
      if (lane == 0) issue(m - 1 + NS);
      issued = m - 1 + NS;
    }
    if (any) {
      stv<V>(ed + lc + x, o, nvalid);
      if constexpr (PUSH) {
        if (m == 0 && T.lo_line >= 0) stv<V>(ed + T.lo_line + x, o, nvalid);
        if (m == G.extent - 1 && T.hi_line >= 0) stv<V>(ed + T.hi_line + x, o, nvalid);
        if (x == 0 && T.w_col >= 0) ed[T.w_col + col] = from_f<TE>(o[0]);
        if (nvalid <= V && T.e_col >= 0) {
          float last = o[0];
#pragma unroll
          for (int k = 1; k < V; ++k)
            if (k == nvalid - 1) last = o[k];
          ed[T.e_col + col] = from_f<TE>(last);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      p[k] = c[k];
      c[k] = n[k];
    }
    wv = wn;
    ev = en;
    ge = gn;
  }
  if (failed) {
    if (lane == 0) atomicOr(status, 2u);
    // let the copies still in flight (at most the last NS lines issued, each
    // stage's latest phase) land before the warp's shared memory is released
    for (int L = max(L0, issued - NS + 1); L <= issued; ++L) {
      const int st = (L - L0) % NS;
      const uint32_t par = (uint32_t)(((L - L0) / NS) & 1);
      uint32_t iters = 0;
      while (!mbar_try_wait(&bars[st], par) && ++iters <= spin_limit) {
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 3D inner sweep with shared-memory staging (non-first sweeps).
//
// Same items and arithmetic as low_item in 3D: a warp computes R = 32 / L
// adjacent block rows y0 .. y0+R-1 (L lanes per row) of one segment, marching
// along z.  For every z-line the warp needs, its lanes copy into a ring of
// kStages3 stages in shared memory, by 16-byte asynchronous copies
// (cp.async, one commit group per line): e of rows y0-1 .. y0+R (its own rows
// and the rows above and below) and r of its own rows.  The march keeps e of
// lines z-1 and z of its own points in registers; e of line z+1 and of rows
// y-1 and y+1, and r, come from shared memory, so each row of e crosses from
// L2 once per warp instead of three times, and the copies in flight (up to
// kStages3 - 1 lines ahead) cost no registers.  Edge scalars (the x-ghost
// columns, the neighbouring segment's points) are plain loads one line ahead.

constexpr int kStages3 = 5;

// Shared-memory bytes of one warp's ring (NS stages of e and r), rounded up to
// 128 bytes so every warp's copies land 16-byte aligned.
template <typename TE, typename TR>
__host__ __device__ constexpr int stage3_warp_bytes(int estage) {
  return (kStages3 * (estage * (int)sizeof(TE) + 32 * low_vpl<TE>() * (int)sizeof(TR)) + 127) / 128 * 128;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <bool PUSH, typename TE, typename TR>
__global__ void __launch_bounds__(kThreads, 2)
k_low_stage3(const WorkItem* __restrict__ items, int nitems, const BlockDev* __restrict__ blocks,
             const SolveDev* __restrict__ solves, int epar, int estage) {
  constexpr int V = low_vpl<TE>();
  constexpr int NS = kStages3;
  constexpr int RST = 32 * V;  // r elements per stage: R rows of L * V points
  extern __shared__ __align__(128) unsigned char st3_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = blockIdx.x * kWarps + warp;
  if (w >= nitems) return;  // whole warp; warps never synchronise with each other here
  const WorkItem it = items[w];
  const BlockDev B = blocks[it.block];
  const SolveDev* S = solves + B.solve;
  if (!S->active) return;
  unsigned char* wb = st3_smem + warp * stage3_warp_bytes<TE, TR>(estage);
  TE* se = reinterpret_cast<TE*>(wb);                                  // NS stages of (R+2) rows of e
  TR* sr = reinterpret_cast<TR*>(wb + NS * estage * (int)sizeof(TE));  // NS stages of R rows of r
  const TE* __restrict__ es = reinterpret_cast<const TE*>(S->e[epar ^ 1]);
  TE* __restrict__ ed = reinterpret_cast<TE*>(S->e[epar]);
  const TR* __restrict__ rr = reinterpret_cast<const TR*>(S->r);

  const int lgL = low_lanes_log2(B.bx, V);
  const int L = 1 << lgL, R = 32 >> lgL;
  const int SEGW = L * V;
  const int rg = lane >> lgL, l = lane & (L - 1);
  const int y = it.y0 + rg;
  const bool row_ok = y < B.by;
  const int bx = B.bx;
  const int xs = it.seg * SEGW;
  const int x = xs + V * l;
  const int nvalid = row_ok ? bx - x : 0;
  const bool any = nvalid > 0;
  const int64_t gW = B.xoff;
  const int64_t gE = B.xoff + (int64_t)B.by * B.bz;
  const Geo<3> G(B, row_ok ? y : B.by - 1);
  PushTargets T;
  if constexpr (PUSH) push_targets<3>(T, B, blocks, row_ok ? y : B.by - 1);
  // rows of e staged per line: y0-1 .. ylast+1 (ylast the warp's last row in
  // the block; row by is the ghost row); elements per row: cnt, a multiple of
  // 16 bytes inside the row pitch
  const int ylast = min(it.y0 + R - 1, B.by - 1);
  const int nrows_e = ylast - it.y0 + 3, nrows_r = ylast - it.y0 + 1;
  const int cnt = min(SEGW, B.pitch - xs);
  const int ecpr = cnt * (int)sizeof(TE) / 16, rcpr = cnt * (int)sizeof(TR) / 16;  // 16-byte chunks per row
  const int m0 = it.z0, mend = m0 + it.n;
  const int L0 = m0 - 1, L1 = mend;  // e lines L0..L1; r lines m0..mend-1
  auto row_off = [&](int yy, int m) {  // element offset of (x = xs, row yy, line m)
    return B.off + (int64_t)(m + 1) * B.plane + (int64_t)(yy + 1) * B.pitch + xs;
  };
  // every lane: copy its share of line Ln into stage (Ln - L0) % NS, then
  // commit one group (empty past the last line, so the group count per
  // step stays constant)
  auto issue = [&](int Ln) {
    if (Ln <= L1) {
      const int st = (Ln - L0) % NS;
      for (int c = lane; c < nrows_e * ecpr; c += 32) {
        const int j = c / ecpr, k = c - j * ecpr;
        cp_async16(reinterpret_cast<unsigned char*>(se + st * estage + j * SEGW) + 16 * k,
                   reinterpret_cast<const unsigned char*>(es + row_off(it.y0 - 1 + j, Ln)) + 16 * k);
      }
      if (Ln >= m0 && Ln < mend)
        for (int c = lane; c < nrows_r * rcpr; c += 32) {
          const int j = c / rcpr, k = c - j * rcpr;
          cp_async16(reinterpret_cast<unsigned char*>(sr + st * RST + j * SEGW) + 16 * k,
                     reinterpret_cast<const unsigned char*>(rr + row_off(it.y0 + j, Ln)) + 16 * k);
        }
    }
    cp_async_commit();
  };
  auto ld_e = [&](int st, int j, float (&o)[V]) {  // this lane's V values of staged row j
    const TE* q = se + st * estage + j * SEGW + V * l;
    if constexpr (sizeof(TE) == 4) {
      const float4 a = *reinterpret_cast<const float4*>(q);
      o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else {
      const uint4 u = *reinterpret_cast<const uint4*>(q);
      const uint32_t wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        o[2 * k] = __uint_as_float(wv[k] << 16);
        o[2 * k + 1] = __uint_as_float(wv[k] & 0xFFFF0000u);
      }
    }
  };
  auto ld_r = [&](int st, float (&o)[V]) {
    const TR* q = sr + st * RST + rg * SEGW + V * l;
    if constexpr (sizeof(TR) == 4) {
      const float4 a = *reinterpret_cast<const float4*>(q);
      o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
      if constexpr (V == 8) {
        const float4 b = *reinterpret_cast<const float4*>(q + 4);
        o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
      }
    } else {
      const uint4 u = *reinterpret_cast<const uint4*>(q);
      const uint32_t wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        o[2 * k] = __uint_as_float(wv[k] << 16);
        o[2 * k + 1] = __uint_as_float(wv[k] & 0xFFFF0000u);
      }
    }
  };
  // edge scalars of line m (west of point 0, east of point V-1, the east
  // ghost of the block's last point), fetched one line ahead
  auto edges = [&](int m, float& wv, float& ev, float& ge) {
    const int64_t lc = G.line(m);
    const int col = G.col(m);
    wv = ev = ge = 0.f;
    if (any) {
      if (l == 0) wv = xs > 0 ? ldf<false>(es + lc + xs - 1) : ldf<false>(es + gW + col);
      if (l == L - 1 && x + V < bx) ev = ldf<false>(es + lc + x + V);
      if (nvalid <= V) ge = ldf<false>(es + gE + col);
    }
  };
  for (int i = 0; i < NS; ++i) issue(L0 + i);
  cp_async_wait<NS - 2>();  // lines L0 and L0 + 1 = m0 have landed
  __syncwarp();
  float p[V], c[V];
#pragma unroll
  for (int k = 0; k < V; ++k) p[k] = c[k] = 0.f;
  if (any) {
    ld_e(0, rg + 1, p);
    ld_e(1 % NS, rg + 1, c);
  }
  float wv, ev, ge;
  edges(m0, wv, ev, ge);
  __syncwarp();   // line L0's stage is free once every lane has read p
  issue(L0 + NS);
  for (int m = m0; m < mend; ++m) {
    const int64_t lc = G.line(m);
    const int col = G.col(m);
    float wn = 0.f, en = 0.f, gn = 0.f;
    if (m + 1 < mend) edges(m + 1, wn, en, gn);
    cp_async_wait<NS - 2>();  // line m + 1 (the oldest pending group) has landed
    __syncwarp();
    const int stc = (m - L0) % NS, stn = (m + 1 - L0) % NS;
    float n[V], sa[V], sb[V], rv[V], o[V];
#pragma unroll
    for (int k = 0; k < V; ++k) n[k] = sa[k] = sb[k] = rv[k] = 0.f;
    if (any) {
      ld_e(stn, rg + 1, n);
      ld_e(stc, rg, sa);
      ld_e(stc, rg + 2, sb);
      ld_r(stc, rv);
    }
    float wl = __shfl_up_sync(FULL_MASK, c[V - 1], 1, L);
    if (l == 0) wl = wv;
    float el = __shfl_down_sync(FULL_MASK, c[0], 1, L);
    if (l == L - 1 && x + V < bx) el = ev;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const float west = k == 0 ? wl : c[k - 1];
      float east = k == V - 1 ? el : c[k + 1];
      if (k + 1 == nvalid) east = ge;  // the block's last point takes the ghost
      float t = __fadd_rn(__fadd_rn(west, p[k]), __fadd_rn(east, n[k]));
      t = __fadd_rn(t, __fadd_rn(sa[k], sb[k]));
      t = __fadd_rn(t, rv[k]);
      o[k] = jdivf<3>(t);
    }
    // line m's stage is free once every lane has read it: refill it
    __syncwarp();
    issue(m + NS);
    if (any) {
      stv<V>(ed + lc + x, o, nvalid);
      if constexpr (PUSH) {
        if (m == 0 && T.lo_line >= 0) stv<V>(ed + T.lo_line + x, o, nvalid);
        if (m == G.extent - 1 && T.hi_line >= 0) stv<V>(ed + T.hi_line + x, o, nvalid);
        if (T.lo_side >= 0) stv<V>(ed + T.lo_side + (int64_t)(m + 1) * T.lo_side_step + x, o, nvalid);
        if (T.hi_side >= 0) stv<V>(ed + T.hi_side + (int64_t)(m + 1) * T.hi_side_step + x, o, nvalid);
        if (x == 0 && T.w_col >= 0) ed[T.w_col + col] = from_f<TE>(o[0]);
        if (nvalid <= V && T.e_col >= 0) {
          float last = o[0];
#pragma unroll
          for (int k = 1; k < V; ++k)
            if (k == nvalid - 1) last = o[k];
          ed[T.e_col + col] = from_f<TE>(last);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
      p[k] = c[k];
      c[k] = n[k];
    }
    wv = wn;
    ev = en;
    ge = gn;
  }
  cp_async_wait<0>();  // no copy may still target this warp's shared memory on exit
}

// ---------------------------------------------------------------------------
// Persistent block scheduler (section 3.1.4's push/pop scheduler and the
// implicit dependencies of section 3.1.2, moved onto the device).  A task is
// one CTA's worth of warp items of one block; (sweep j, task t) pairs are
// handed out in sweep order by an atomic counter.  Before sweep j of block b
// runs, b and its neighbours must have finished sweep j-1: that covers both
// the data b reads (its interior and the ghosts its neighbours pushed) and the
// buffer it overwrites (read by b and its neighbours during sweep j-1).  A task
// only ever waits for tasks with smaller indices, which were taken earlier by
// CTAs that are running, so the scheme needs no co-residency guarantee.  Every
// wait is bounded: when it runs out the task records JACOBI_ERR_TIMEOUT in the
// control word and every CTA leaves.

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Called by the 32 lanes of one warp: lane 0 watches block b, lanes 1..6 its
// neighbours, all at once (one L2 round trip instead of seven in a row).
template <bool LOW>
__device__ bool wait_deps(const BlockDev& B, int b, const BlockDev* __restrict__ blocks, const uint32_t* done, int j,
                          SchedCtl* ctl, uint32_t spin_limit, int poison) {
  const int lane = threadIdx.x & 31;
  const int q = lane == 0 ? b : (lane < 7 ? B.nbr[lane - 1] : -1);
  bool ok = true;
  if (q >= 0) {
    const int nt = lane == 0 ? (LOW ? B.ntlo : B.nt64) : (LOW ? blocks[q].ntlo : blocks[q].nt64);
    const uint32_t need = poison ? 0xffffffffu : (uint32_t)j * (uint32_t)nt;
    uint32_t iters = 0;
    while (ld_acquire_u32(done + q) < need) {
      if (++iters > spin_limit || *(volatile uint32_t*)&ctl->status != 0u) {
        ok = false;
        break;
      }
      __nanosleep(64);
    }
  }
  return __all_sync(FULL_MASK, ok);
}

template <bool LOW, typename Body>
__device__ __forceinline__ void persist_loop(const CtaTask* __restrict__ tasks, int ntasks, int nsweeps,
                                             const BlockDev* __restrict__ blocks, const SolveDev* __restrict__ solves,
                                             uint32_t* done, SchedCtl* ctl, uint32_t spin_limit, int poison,
                                             Body body) {
  __shared__ int s_idx;
  __shared__ int s_stop;
  const int warp = threadIdx.x >> 5;
  const long long total = (long long)ntasks * nsweeps;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned idx = atomicAdd(&ctl->head, 1u);
      s_idx = (int)idx;
      s_stop = ((long long)idx >= total) || (*(volatile uint32_t*)&ctl->status != 0u);
    }
    __syncthreads();
    if (s_stop) break;
    const int idx = s_idx;
    const int j = idx / ntasks;
    const CtaTask T = tasks[idx - j * ntasks];
    const BlockDev& B = blocks[T.block];
    const bool act = solves[B.solve].active != 0;
    if (warp == 0 && act && j > 0) {
      const bool ok = wait_deps<LOW>(B, T.block, blocks, done, j, ctl, spin_limit, poison);
      if (threadIdx.x == 0) {
        if (!ok) {
          if (atomicExch(&ctl->status, 1u) == 0u) ctl->fail_task = (uint32_t)idx;
          s_stop = 1;
        }
        __threadfence();
      }
    }
    __syncthreads();
    if (s_stop) break;
    if (act && warp < T.nw) body(T.w0 + warp, j);
    __syncthreads();
    if (threadIdx.x == 0 && act) {
      __threadfence();
      atomicAdd(done + T.block, 1u);
    }
  }
}

template <int DIM, typename TE, typename TR>
__global__ void __launch_bounds__(kThreads)
k_persist_low(const CtaTask* __restrict__ tasks, int ntasks, int nsweeps, const WorkItem* __restrict__ items,
              const BlockDev* __restrict__ blocks, const SolveDev* __restrict__ solves, uint32_t* done, SchedCtl* ctl,
              uint32_t spin_limit, int poison) {
  persist_loop<true>(tasks, ntasks, nsweeps, blocks, solves, done, ctl, spin_limit, poison, [&](int wi, int j) {
    const WorkItem it = items[wi];
    if (j == 0) low_item<DIM, true, true, TE, TR, true>(it, blocks, solves, 0);
    else low_item<DIM, false, true, TE, TR, true>(it, blocks, solves, j & 1);
  });
}

template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_persist_f64(const CtaTask* __restrict__ tasks, int ntasks, int nsweeps, int resid_last,
              const WorkItem* __restrict__ items, const BlockDev* __restrict__ blocks,
              const SolveDev* __restrict__ solves, uint32_t* done, SchedCtl* ctl, uint32_t spin_limit, int poison) {
  persist_loop<false>(tasks, ntasks, nsweeps, blocks, solves, done, ctl, spin_limit, poison, [&](int wi, int j) {
    const WorkItem it = items[wi];
    if (resid_last && j == nsweeps - 1)
      f64_item<DIM, kModeSweep, true, true, float, float, true>(it, blocks, solves, j & 1, 0);
    else
      f64_item<DIM, kModeSweep, true, false, float, float, true>(it, blocks, solves, j & 1, 0);
  });
}

__global__ void k_solve_ctl(SolveDev* solves, const int32_t* __restrict__ ctl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t c = ctl[i];
  if (c & 8) return;
  SolveDev* S = solves + i;
  if (c & 2) S->phase ^= 1;
  if (c & 4) S->apply_e = 0;
  S->active = c & 1;
}

// ---------------------------------------------------------------------------
// Standalone halo exchange (section 4.3: pack the GPU faces, move them, unpack
// them into the halo).  One CTA per (block, face); domain faces are skipped.
// Face element order: x faces (z, y), y faces (z, x), z faces (y, x), lowest
// axis fastest.

__device__ __forceinline__ int64_t face_elem(const BlockDev& B, int face, int i, bool ghost) {
  // offset of element i of face `face` of block B: its boundary layer
  // (ghost = false) or its ghost layer (ghost = true)
  const int axis = face >> 1, hi = face & 1;
  if (axis == 0) {
    const int y = i % B.by, z = i / B.by;
    if (ghost) return (hi ? B.xoff + (int64_t)B.by * B.bz : B.xoff) + (int64_t)z * B.by + y;
    const int x = hi ? B.bx - 1 : 0;
    return B.off + (int64_t)(z + B.gz) * B.plane + (int64_t)(y + 1) * B.pitch + x;
  }
  if (axis == 1) {
    const int x = i % B.bx, z = i / B.bx;
    const int y = ghost ? (hi ? B.by : -1) : (hi ? B.by - 1 : 0);
    return B.off + (int64_t)(z + B.gz) * B.plane + (int64_t)(y + 1) * B.pitch + x;
  }
  const int x = i % B.bx, y = i / B.bx;
  const int z = ghost ? (hi ? B.bz : -1) : (hi ? B.bz - 1 : 0);
  return B.off + (int64_t)(z + 1) * B.plane + (int64_t)(y + 1) * B.pitch + x;
}

__device__ __forceinline__ int64_t face_send_off(const BlockDev& B, int face) {
  int64_t o = B.foff;
  for (int k = 0; k < face; ++k) o += B.fsz[k];
  return o;
}

template <typename T>
__global__ void k_halo_pack(const FaceItem* __restrict__ items, const BlockDev* __restrict__ blocks,
                            const SolveDev* __restrict__ solves, int which, int par) {
  const FaceItem it = items[blockIdx.x];
  const BlockDev B = blocks[it.block];
  const SolveDev* S = solves + B.solve;
  if (!S->active || B.nbr[it.face] < 0) return;
  // which = 0: the FP64 iterate x[(phase + par) & 1]; which = 1: e[par]
  const T* a = which == 0 ? reinterpret_cast<const T*>(S->x[(S->phase + par) & 1])
                          : reinterpret_cast<const T*>(S->e[par]);
  T* send = which == 0 ? reinterpret_cast<T*>(S->send64) : reinterpret_cast<T*>(S->sendlo);
  const int64_t so = face_send_off(B, it.face);
  const int n = B.fsz[it.face];
  for (int i = threadIdx.x; i < n; i += blockDim.x) send[so + i] = a[face_elem(B, it.face, i, false)];
}

template <typename T>
__global__ void k_halo_unpack(const FaceItem* __restrict__ items, const BlockDev* __restrict__ blocks,
                              const SolveDev* __restrict__ solves, int which, int par) {
  const FaceItem it = items[blockIdx.x];
  const BlockDev B = blocks[it.block];
  const SolveDev* S = solves + B.solve;
  const int nb = B.nbr[it.face];
  if (!S->active || nb < 0) return;
  const BlockDev N = blocks[nb];
  T* a = which == 0 ? reinterpret_cast<T*>(S->x[(S->phase + par) & 1]) : reinterpret_cast<T*>(S->e[par]);
  const T* send = which == 0 ? reinterpret_cast<const T*>(S->send64) : reinterpret_cast<const T*>(S->sendlo);
  const int64_t so = face_send_off(N, it.face ^ 1);  // the neighbour's opposite face
  const int n = B.fsz[it.face];
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[face_elem(B, it.face, i, true)] = send[so + i];
}

// ---------------------------------------------------------------------------
// Deterministic residual reduction: CTA c of a solve sums its chunk of
// partials in a fixed order (thread-strided, then a shared-memory tree); the
// last CTA of the solve to finish sums the chunk results in a fixed order.
// The result depends only on the partials, never on scheduling.

__global__ void __launch_bounds__(kRedThreads)
k_reduce(const RedItem* __restrict__ items, SolveDev* __restrict__ solves) {
  __shared__ double sm[kRedThreads];
  __shared__ int is_last;
  const RedItem it = items[blockIdx.x];
  SolveDev* S = solves + it.solve;
  if (!S->active) return;
  const int t = threadIdx.x;
  double acc = 0.0;
  const double* part = S->part + it.start;
  for (int i = t; i < it.len; i += kRedThreads) acc = dadd(acc, part[i]);
  sm[t] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (t < s) sm[t] = dadd(sm[t], sm[t + s]);
    __syncthreads();
  }
  if (t == 0) {
    S->lvl1[it.chunk] = sm[0];
    __threadfence();
    const unsigned tk = atomicAdd(S->ticket, 1u);
    is_last = tk == (unsigned)(it.nchunks - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  acc = 0.0;
  for (int i = t; i < it.nchunks; i += kRedThreads) acc = dadd(acc, __ldcg(S->lvl1 + i));
  sm[t] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (t < s) sm[t] = dadd(sm[t], sm[t + s]);
    __syncthreads();
  }
  if (t == 0) {
    S->rss[0] = sm[0];
    *S->ticket = 0u;
  }
}

// ---------------------------------------------------------------------------
// Dense (interior, x fastest) <-> blocked copies; one warp per block row.

__global__ void k_scatter(const RowItem* __restrict__ items, int n, const BlockDev* __restrict__ blocks,
                          SolveDev* __restrict__ solves, const double* __restrict__ dense, int which, int par,
                          int64_t nx, int64_t ny) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (w >= n) return;
  const RowItem it = items[w];
  const BlockDev B = blocks[it.block];
  SolveDev* S = solves + B.solve;
  double* a = which == 0 ? S->x[(S->phase + par) & 1] : S->f;
  const int64_t o = B.off + (int64_t)(it.z + B.gz) * B.plane + (int64_t)(it.y + 1) * B.pitch;
  const int64_t d = ((int64_t)(B.oz + it.z) * ny + (B.oy + it.y)) * nx + B.ox;
  for (int x = threadIdx.x & 31; x < B.bx; x += 32) a[o + x] = dense[d + x];
}

__global__ void k_gather(const RowItem* __restrict__ items, int n, const BlockDev* __restrict__ blocks,
                         const SolveDev* __restrict__ solves, double* __restrict__ dense, int par, int64_t nx,
                         int64_t ny) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (w >= n) return;
  const RowItem it = items[w];
  const BlockDev B = blocks[it.block];
  const SolveDev* S = solves + B.solve;
  const double* a = S->x[(S->phase + par) & 1];
  const int64_t o = B.off + (int64_t)(it.z + B.gz) * B.plane + (int64_t)(it.y + 1) * B.pitch;
  const int64_t d = ((int64_t)(B.oz + it.z) * ny + (B.oy + it.y)) * nx + B.ox;
  for (int x = threadIdx.x & 31; x < B.bx; x += 32) dense[d + x] = a[o + x];
}

// Dirichlet values g into the domain-boundary ghosts of x[par].
struct FacePtrs {
  const double* f[6];
};

__global__ void k_ghost_fill(const FaceItem* __restrict__ items, const BlockDev* __restrict__ blocks,
                             SolveDev* __restrict__ solves, FacePtrs faces, int par, int64_t nx, int64_t ny,
                             int64_t nz) {
  const FaceItem it = items[blockIdx.x];
  const BlockDev B = blocks[it.block];
  if (B.nbr[it.face] >= 0) return;
  SolveDev* S = solves + B.solve;
  double* a = S->x[par];
  const double* g = faces.f[it.face];
  const int axis = it.face >> 1;
  const int n = B.fsz[it.face];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int64_t gi;
    if (axis == 0) {
      const int y = i % B.by, z = i / B.by;
      gi = (int64_t)(B.oy + y) + ny * (B.oz + z);
    } else if (axis == 1) {
      const int x = i % B.bx, z = i / B.bx;
      gi = (int64_t)(B.ox + x) + nx * (B.oz + z);
    } else {
      const int x = i % B.bx, y = i / B.bx;
      gi = (int64_t)(B.ox + x) + nx * (B.oy + y);
    }
    a[face_elem(B, it.face, i, true)] = g ? g[gi] : 0.0;
  }
  (void)nz;
}

__global__ void k_phase_advance(SolveDev* solves, int n, int dphase, int set_apply_e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  SolveDev* S = solves + i;
  if (!S->active) return;
  S->phase = (S->phase + dphase) & 1;
  if (set_apply_e >= 0) S->apply_e = set_apply_e;
}

// ---------------------------------------------------------------------------
// launch wrappers

static inline int grid_of(int items, int per) { return (items + per - 1) / per; }

template <int DIM>
static int sweep_f64_dim(const Tables& t, int kpar, bool push, bool resid, bool write, int emu, cudaStream_t s) {
  const dim3 g(grid_of(t.n64, kWarps)), b(kThreads);
  if (t.n64 == 0) return 0;
  if (!write) {
    k_f64<DIM, kModeResid, false, true, float, float><<<g, b, 0, s>>>(t.w64, t.n64, kpar, t.blocks, t.solves, 0);
  } else if (push) {
    if (resid) k_f64<DIM, kModeSweep, true, true, float, float><<<g, b, 0, s>>>(t.w64, t.n64, kpar, t.blocks, t.solves, 0);
    else if (emu >= 3)
      k_f64<DIM, kModeSweep, true, false, float, float, 3><<<g, b, 0, s>>>(t.w64, t.n64, kpar, t.blocks, t.solves, 0);
    else if (emu == 2)
      k_f64<DIM, kModeSweep, true, false, float, float, 2><<<g, b, 0, s>>>(t.w64, t.n64, kpar, t.blocks, t.solves, 0);
    else k_f64<DIM, kModeSweep, true, false, float, float><<<g, b, 0, s>>>(t.w64, t.n64, kpar, t.blocks, t.solves, 0);
  } else {
    if (resid) k_f64<DIM, kModeSweep, false, true, float, float><<<g, b, 0, s>>>(t.w64, t.n64, kpar, t.blocks, t.solves, 0);
    else k_f64<DIM, kModeSweep, false, false, float, float><<<g, b, 0, s>>>(t.w64, t.n64, kpar, t.blocks, t.solves, 0);
  }
  return (int)cudaGetLastError();
}

template <int MODE = kModeSweep, typename TE = float>
static constexpr int march_stage_bytes() {
  return kWarps * kMarchStages * march4_slot_doubles<MODE, TE>() * (int)sizeof(double);
}

// width: 2 (64-point segments), 4 (128-point segments, register prefetch),
// 5 (128-point segments, lines staged in shared memory)
int launch_sweep_f64_march(const Tables& t, int kpar, bool push, int width, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.nm == 0) return 0;
  const dim3 g(grid_of(t.nm, kWarps)), b(kThreads);
  if (t.ndim != 2) return (int)cudaErrorInvalidValue;
  if (width == 5) {
    const int sm = march_stage_bytes();
    auto k = push ? k_f64_march4<true, kMarchStages> : k_f64_march4<false, kMarchStages>;
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return (int)e;
    if (t.nmw == 0) return 0;
    k<<<grid_of(t.nmw, kWarps), b, sm, s>>>(t.wm, t.nmw, t.wms, kpar, t.blocks, t.solves, t.l2pf, 0);
  } else if (width == 4) {
    if (push) k_f64_march4<true, 0><<<g, b, 0, s>>>(t.wm, t.nm, nullptr, kpar, t.blocks, t.solves, t.l2pf, 0);
    else k_f64_march4<false, 0><<<g, b, 0, s>>>(t.wm, t.nm, nullptr, kpar, t.blocks, t.solves, t.l2pf, 0);
  } else {
    if (push) k_f64_march<2, true><<<g, b, 0, s>>>(t.wm, t.nm, kpar, t.blocks, t.solves, t.l2pf);
    else k_f64_march<2, false><<<g, b, 0, s>>>(t.wm, t.nm, kpar, t.blocks, t.solves, t.l2pf);
  }
  return (int)cudaGetLastError();
}

int march_f64_resident_warps(int ndim, bool push, int width) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (ndim != 2) return 0;
  cudaError_t e;
  if (width == 5) {
    const int sm = march_stage_bytes();
    auto k = push ? k_f64_march4<true, kMarchStages> : k_f64_march4<false, kMarchStages>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, sm);
  } else if (width == 4)
    e = push ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_f64_march4<true, 0>, kThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_f64_march4<false, 0>, kThreads, 0);
  else
    e = push ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_f64_march<2, true>, kThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_f64_march<2, false>, kThreads, 0);
  if (e != cudaSuccess) return 0;
  return per_sm * sms * kWarps;
}

// The fused-residual sweep and the outer step over the residual-aligned march
// items (t.wmr), four points per lane, lines staged in shared memory.
template <bool PUSH, int MODE, typename TE, typename TR>
static cudaError_t march4r_launch(const Tables& t, int kpar, int epar, cudaStream_t s) {
  if (t.nmrw == 0) return cudaSuccess;
  constexpr int sm = march_stage_bytes<MODE, TE>();
  auto k = k_f64_march4<PUSH, kMarchStages, MODE, true, TE, TR>;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  k<<<grid_of(t.nmrw, kWarps), kThreads, sm, s>>>(t.wmr, t.nmrw, t.wmrs, kpar, t.blocks, t.solves, t.l2pf, epar);
  return cudaGetLastError();
}

template <bool PUSH, int MODE, typename TE, typename TR>
static int march4r_per_sm() {
  constexpr int sm = march_stage_bytes<MODE, TE>();
  auto k = k_f64_march4<PUSH, kMarchStages, MODE, true, TE, TR>;
  int per_sm = 0;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, sm);
  return e == cudaSuccess ? per_sm : 0;
}

int launch_sweep_f64_march_resid(const Tables& t, int kpar, bool push, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.ndim != 2) return (int)cudaErrorInvalidValue;
  return (int)(push ? march4r_launch<true, kModeSweep, float, float>(t, kpar, 0, s)
                    : march4r_launch<false, kModeSweep, float, float>(t, kpar, 0, s));
}

int launch_refine_outer_march(const Tables& t, int epar_last, bool push, int low, bool r_bf16, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.ndim != 2) return (int)cudaErrorInvalidValue;
  cudaError_t e;
  if (low == kLowF32)
    e = push ? march4r_launch<true, kModeOuter, float, float>(t, 0, epar_last, s)
             : march4r_launch<false, kModeOuter, float, float>(t, 0, epar_last, s);
  else if (r_bf16)
    e = push ? march4r_launch<true, kModeOuter, __nv_bfloat16, __nv_bfloat16>(t, 0, epar_last, s)
             : march4r_launch<false, kModeOuter, __nv_bfloat16, __nv_bfloat16>(t, 0, epar_last, s);
  else
    e = push ? march4r_launch<true, kModeOuter, __nv_bfloat16, float>(t, 0, epar_last, s)
             : march4r_launch<false, kModeOuter, __nv_bfloat16, float>(t, 0, epar_last, s);
  return (int)e;
}

int march_f64r_resident_warps(int ndim, bool push) {
  int dev = 0, sms = 0;
  if (ndim != 2) return 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  // the fewest resident CTAs of the kernels that run over these items
  int per_sm = push ? march4r_per_sm<true, kModeSweep, float, float>() : march4r_per_sm<false, kModeSweep, float, float>();
  per_sm = std::min(per_sm, push ? march4r_per_sm<true, kModeOuter, float, float>()
                                 : march4r_per_sm<false, kModeOuter, float, float>());
  return per_sm * sms * kWarps;
}

int launch_sweep_f64(const Tables& t, int kpar, bool push, bool resid, bool write, int emu, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return t.ndim == 2 ? sweep_f64_dim<2>(t, kpar, push, resid, write, emu, s)
                     : sweep_f64_dim<3>(t, kpar, push, resid, write, emu, s);
}

template <int DIM, typename TE, typename TR>
static int low_typed(const Tables& t, int epar, bool first, bool push, cudaStream_t s) {
  const dim3 g(grid_of(t.nlo, kWarps)), b(kThreads);
  if (t.nlo == 0) return 0;
  if constexpr (DIM == 2 && sizeof(TE) == 4) {
    if (first) {
      if (push) k_low_free<DIM, true, true, TE, TR><<<g, b, 0, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
      else k_low_free<DIM, true, false, TE, TR><<<g, b, 0, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
    } else {
      if (push) k_low_free<DIM, false, true, TE, TR><<<g, b, 0, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
      else k_low_free<DIM, false, false, TE, TR><<<g, b, 0, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
    }
  } else if (first) {
    if (push) k_low<DIM, true, true, TE, TR><<<g, b, 0, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
    else k_low<DIM, true, false, TE, TR><<<g, b, 0, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
  } else {
    if (push) k_low<DIM, false, true, TE, TR><<<g, b, 0, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
    else k_low<DIM, false, false, TE, TR><<<g, b, 0, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
  }
  return (int)cudaGetLastError();
}

template <int DIM>
static int low_dim(const Tables& t, int epar, bool first, bool push, int low, bool r_bf16, cudaStream_t s) {
  if (low == kLowF32) return low_typed<DIM, float, float>(t, epar, first, push, s);
  if (r_bf16) return low_typed<DIM, __nv_bfloat16, __nv_bfloat16>(t, epar, first, push, s);
  return low_typed<DIM, __nv_bfloat16, float>(t, epar, first, push, s);
}

int launch_sweep_low(const Tables& t, int epar, bool first, bool push, int low, bool r_bf16, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return t.ndim == 2 ? low_dim<2>(t, epar, first, push, low, r_bf16, s)
                     : low_dim<3>(t, epar, first, push, low, r_bf16, s);
}

template <typename TE, typename TR>
static int low_s3_typed(const Tables& t, int epar, bool push, cudaStream_t s) {
  if (t.nlo == 0) return 0;
  constexpr int sm = kWarps * low_s3_stages<TE>() * low_s3_slot_bytes<TE, TR>();
  auto k = push ? k_low_s3<true, TE, TR> : k_low_s3<false, TE, TR>;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return (int)e;
  k<<<grid_of(t.nlo, kWarps), kThreads, sm, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar);
  return (int)cudaGetLastError();
}

int launch_sweep_low_s3(const Tables& t, int epar, bool push, int low, bool r_bf16, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.ndim != 3) return (int)cudaErrorInvalidValue;
  if (low == kLowF32) return low_s3_typed<float, float>(t, epar, push, s);
  if (r_bf16) return low_s3_typed<__nv_bfloat16, __nv_bfloat16>(t, epar, push, s);
  return low_s3_typed<__nv_bfloat16, float>(t, epar, push, s);
}

template <int DIM, typename TE, typename TR>
static int outer_typed(const Tables& t, int epar_last, bool push, cudaStream_t s) {
  const dim3 g(grid_of(t.n64, kWarps)), b(kThreads);
  if (t.n64 == 0) return 0;
  if (push) k_f64<DIM, kModeOuter, true, true, TE, TR><<<g, b, 0, s>>>(t.w64, t.n64, 0, t.blocks, t.solves, epar_last);
  else k_f64<DIM, kModeOuter, false, true, TE, TR><<<g, b, 0, s>>>(t.w64, t.n64, 0, t.blocks, t.solves, epar_last);
  return (int)cudaGetLastError();
}

// x[phase^1] = x[phase] + e (or a copy while the solve has no correction
// yet) over every element of each active solve's layout; blockIdx.y = slot.
template <typename TE>
__global__ void __launch_bounds__(kThreads)
k_apply_e(SolveDev* __restrict__ solves, int epar) {
  const SolveDev* S = solves + blockIdx.y;
  if (!S->active) return;
  const int lane = threadIdx.x & 31;
  const double* __restrict__ xs = S->x[S->phase & 1];
  double* __restrict__ xd = S->x[(S->phase & 1) ^ 1];
  const TE* __restrict__ e = reinterpret_cast<const TE*>(S->e[epar]);
  const bool apply = S->apply_e != 0;
  const int64_t n = S->elems;  // a multiple of 32
  const int64_t wstride = (int64_t)gridDim.x * kWarps * 64;
  for (int64_t w0 = ((int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5)) * 64; w0 < n; w0 += wstride) {
    const int64_t i = w0 + 2 * lane;
    const bool valid = i < n;
    double2 v = make_double2(0.0, 0.0);
    float ea = 0.f, eb = 0.f;
    if (valid) {
      v = *reinterpret_cast<const double2*>(xs + i);
      if (apply) {
        ea = ldf<false>(e + i);
        eb = ldf<false>(e + i + 1);
      }
    }
    if (apply) {  // uniform
      v.x = dadd(v.x, f2d(ea));
      v.y = dadd(v.y, f2d(eb));
    }
    if (valid) *reinterpret_cast<double2*>(xd + i) = v;
  }
}

template <typename TE, typename TR>
static int outer_split_typed(const Tables& t, int nslots, int64_t max_elems, int epar_last, cudaStream_t s) {
  if (t.n64 == 0 || nslots <= 0 || max_elems <= 0) return 0;
  const int64_t per_cta = (int64_t)kWarps * 64;
  const unsigned gx = (unsigned)std::min<int64_t>((max_elems + per_cta - 1) / per_cta, 4096);
  k_apply_e<TE><<<dim3(gx, (unsigned)nslots), kThreads, 0, s>>>(t.solves, epar_last);
  k_f64<3, kModeOuterR, false, true, float, TR><<<grid_of(t.n64, kWarps), kThreads, 0, s>>>(t.w64, t.n64, 1, t.blocks,
                                                                                          t.solves, 0);
  return (int)cudaGetLastError();
}

int launch_refine_outer_split(const Tables& t, int nslots, int64_t max_elems, int epar_last, int low, bool r_bf16,
                              void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.ndim != 3 || nslots > 65535) return (int)cudaErrorInvalidValue;
  if (low == kLowF32) return outer_split_typed<float, float>(t, nslots, max_elems, epar_last, s);
  if (r_bf16) return outer_split_typed<__nv_bfloat16, __nv_bfloat16>(t, nslots, max_elems, epar_last, s);
  return outer_split_typed<__nv_bfloat16, float>(t, nslots, max_elems, epar_last, s);
}

template <int DIM>
static int outer_dim(const Tables& t, int epar_last, bool push, int low, bool r_bf16, cudaStream_t s) {
  if (low == kLowF32) return outer_typed<DIM, float, float>(t, epar_last, push, s);
  if (r_bf16) return outer_typed<DIM, __nv_bfloat16, __nv_bfloat16>(t, epar_last, push, s);
  return outer_typed<DIM, __nv_bfloat16, float>(t, epar_last, push, s);
}

int launch_refine_outer(const Tables& t, int epar_last, bool push, int low, bool r_bf16, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return t.ndim == 2 ? outer_dim<2>(t, epar_last, push, low, r_bf16, s)
                     : outer_dim<3>(t, epar_last, push, low, r_bf16, s);
}

int launch_halo_pack(const Tables& t, int which, int par, int low, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.nfaces == 0) return 0;
  if (which == 0) k_halo_pack<double><<<t.nfaces, 256, 0, s>>>(t.faces, t.blocks, t.solves, 0, par);
  else if (low == kLowF32) k_halo_pack<float><<<t.nfaces, 256, 0, s>>>(t.faces, t.blocks, t.solves, 1, par);
  else k_halo_pack<__nv_bfloat16><<<t.nfaces, 256, 0, s>>>(t.faces, t.blocks, t.solves, 1, par);
  return (int)cudaGetLastError();
}

int launch_halo_unpack(const Tables& t, int which, int par, int low, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.nfaces == 0) return 0;
  if (which == 0) k_halo_unpack<double><<<t.nfaces, 256, 0, s>>>(t.faces, t.blocks, t.solves, 0, par);
  else if (low == kLowF32) k_halo_unpack<float><<<t.nfaces, 256, 0, s>>>(t.faces, t.blocks, t.solves, 1, par);
  else k_halo_unpack<__nv_bfloat16><<<t.nfaces, 256, 0, s>>>(t.faces, t.blocks, t.solves, 1, par);
  return (int)cudaGetLastError();
}

int launch_reduce(const Tables& t, void* stream) {
  if (t.nred == 0) return 0;
  k_reduce<<<t.nred, kRedThreads, 0, (cudaStream_t)stream>>>(t.red, t.solves);
  return (int)cudaGetLastError();
}

int launch_scatter(const Tables& t, const double* dense, int which, int par, int64_t nx, int64_t ny, void* stream) {
  if (t.nrows == 0) return 0;
  k_scatter<<<grid_of(t.nrows, kWarps), kThreads, 0, (cudaStream_t)stream>>>(t.rows, t.nrows, t.blocks, t.solves,
                                                                                dense, which, par, nx, ny);
  return (int)cudaGetLastError();
}

int launch_gather(const Tables& t, double* dense, int par, int64_t nx, int64_t ny, void* stream) {
  if (t.nrows == 0) return 0;
  k_gather<<<grid_of(t.nrows, kWarps), kThreads, 0, (cudaStream_t)stream>>>(t.rows, t.nrows, t.blocks, t.solves,
                                                                               dense, par, nx, ny);
  return (int)cudaGetLastError();
}

int launch_ghost_fill(const Tables& t, const double* const* faces_dev, int par, int64_t nx, int64_t ny, int64_t nz,
                      void* stream) {
  if (t.nfaces == 0) return 0;
  FacePtrs fp;
  for (int i = 0; i < 6; ++i) fp.f[i] = faces_dev[i];
  k_ghost_fill<<<t.nfaces, 256, 0, (cudaStream_t)stream>>>(t.faces, t.blocks, t.solves, fp, par, nx, ny, nz);
  return (int)cudaGetLastError();
}

int launch_phase_advance(SolveDev* solves, int nsolves, int dphase, int set_apply_e, void* stream) {
  if (nsolves == 0) return 0;
  k_phase_advance<<<grid_of(nsolves, 256), 256, 0, (cudaStream_t)stream>>>(solves, nsolves, dphase, set_apply_e);
  return (int)cudaGetLastError();
}

template <typename K>
static int persist_grid(K kernel, int total_tasks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0);
  const int g = std::max(1, sms * std::max(1, per_sm));
  return std::min(g, std::max(1, total_tasks));
}

template <int DIM, typename TE, typename TR>
static int persist_low_typed(const Tables& t, int nsweeps, cudaStream_t s) {
  if (t.ntlo == 0 || nsweeps <= 0) return 0;
  auto k = k_persist_low<DIM, TE, TR>;
  const int g = persist_grid(k, t.ntlo * nsweeps);
  k<<<g, kThreads, 0, s>>>(t.tlo, t.ntlo, nsweeps, t.wlo, t.blocks, t.solves, t.done, t.ctl, t.spin_limit, t.poison);
  return (int)cudaGetLastError();
}

template <int DIM>
static int persist_low_dim(const Tables& t, int nsweeps, int low, bool r_bf16, cudaStream_t s) {
  if (low == kLowF32) return persist_low_typed<DIM, float, float>(t, nsweeps, s);
  if (r_bf16) return persist_low_typed<DIM, __nv_bfloat16, __nv_bfloat16>(t, nsweeps, s);
  return persist_low_typed<DIM, __nv_bfloat16, float>(t, nsweeps, s);
}

int launch_persist_low(const Tables& t, int nsweeps, int low, bool r_bf16, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return t.ndim == 2 ? persist_low_dim<2>(t, nsweeps, low, r_bf16, s) : persist_low_dim<3>(t, nsweeps, low, r_bf16, s);
}

template <int DIM>
static int persist_f64_dim(const Tables& t, int nsweeps, bool resid_last, cudaStream_t s) {
  if (t.nt64 == 0 || nsweeps <= 0) return 0;
  auto k = k_persist_f64<DIM>;
  const int g = persist_grid(k, t.nt64 * nsweeps);
  k<<<g, kThreads, 0, s>>>(t.t64, t.nt64, nsweeps, resid_last ? 1 : 0, t.w64, t.blocks, t.solves, t.done, t.ctl,
                           t.spin_limit, t.poison);
  return (int)cudaGetLastError();
}

int launch_persist_f64(const Tables& t, int nsweeps, bool resid_last, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return t.ndim == 2 ? persist_f64_dim<2>(t, nsweeps, resid_last, s) : persist_f64_dim<3>(t, nsweeps, resid_last, s);
}

template <typename TE, typename TR>
static int low_tma_typed(const Tables& t, int epar, bool push, cudaStream_t s) {
  const int smem = kWarps * tma_warp_bytes<TE, TR>();
  auto k = push ? k_low_tma<true, TE, TR> : k_low_tma<false, TE, TR>;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  k<<<grid_of(t.nlo, kWarps), kThreads, smem, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar, &t.ctl->status,
                                                   t.spin_limit);
  return (int)cudaGetLastError();
}

template <typename TE, typename TR>
static int low_stage3_typed(const Tables& t, int epar, bool push, int estage, cudaStream_t s) {
  const int smem = kWarps * stage3_warp_bytes<TE, TR>(estage);
  auto k = push ? k_low_stage3<true, TE, TR> : k_low_stage3<false, TE, TR>;
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  k<<<grid_of(t.nlo, kWarps), kThreads, smem, s>>>(t.wlo, t.nlo, t.blocks, t.solves, epar, estage);
  return (int)cudaGetLastError();
}

int launch_sweep_low_stage3(const Tables& t, int epar, bool push, int low, bool r_bf16, int estage, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.nlo == 0) return 0;
  if (t.ndim != 3 || estage <= 0) return (int)cudaErrorInvalidValue;
  if (low == kLowF32) return low_stage3_typed<float, float>(t, epar, push, estage, s);
  if (r_bf16) return low_stage3_typed<__nv_bfloat16, __nv_bfloat16>(t, epar, push, estage, s);
  return low_stage3_typed<__nv_bfloat16, float>(t, epar, push, estage, s);
}

int launch_sweep_low_tma(const Tables& t, int epar, bool push, int low, bool r_bf16, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.nlo == 0) return 0;
  if (t.ndim != 2) return (int)cudaErrorInvalidValue;
  if (low == kLowF32) return low_tma_typed<float, float>(t, epar, push, s);
  if (r_bf16) return low_tma_typed<__nv_bfloat16, __nv_bfloat16>(t, epar, push, s);
  return low_tma_typed<__nv_bfloat16, float>(t, epar, push, s);
}

template <typename TE, typename TR, bool PERSIST>
static int low_tb2_typed(const Tables& t, int in_par, int out_par, bool first, bool push, cudaStream_t s) {
  const int sm = tb2_smem_bytes<TE, TR, PERSIST>();
  auto k = first ? (push ? k_low_tb2<true, true, TE, TR, PERSIST> : k_low_tb2<false, true, TE, TR, PERSIST>)
                 : (push ? k_low_tb2<true, false, TE, TR, PERSIST> : k_low_tb2<false, false, TE, TR, PERSIST>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return (int)e;
  int g = t.ntb;  // one CTA per tile
  if (PERSIST) {  // as many CTAs as are resident at once
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, sm)) != cudaSuccess) return (int)e;
    g = std::max(1, std::min(t.ntb, sms * std::max(1, per_sm)));
  }
  k<<<g, kThreads, sm, s>>>(t.wtb, t.ntb, t.blocks, t.solves, in_par, out_par);
  return (int)cudaGetLastError();
}

template <typename TE, typename TR>
static int low_tb3_typed(const Tables& t, int in_par, int out_par, bool first, bool push, cudaStream_t s) {
  const int sm = tb3_smem_bytes<TE, TR>();
  auto k = first ? (push ? k_low_tb3<true, true, TE, TR> : k_low_tb3<false, true, TE, TR>)
                 : (push ? k_low_tb3<true, false, TE, TR> : k_low_tb3<false, false, TE, TR>);
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return (int)e;
  k<<<t.ntb, kThreads, sm, s>>>(t.wtb, t.ntb, t.blocks, t.solves, in_par, out_par);
  return (int)cudaGetLastError();
}

int launch_sweep_low_tb2(const Tables& t, int in_par, int out_par, bool first, bool push, int low, bool r_bf16,
                         void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (t.ntb == 0) return 0;
  if (in_par == out_par) return (int)cudaErrorInvalidValue;
  if (t.ndim == 3) {
    if (low == kLowF32) return low_tb3_typed<float, float>(t, in_par, out_par, first, push, s);
    if (r_bf16) return low_tb3_typed<__nv_bfloat16, __nv_bfloat16>(t, in_par, out_par, first, push, s);
    return low_tb3_typed<__nv_bfloat16, float>(t, in_par, out_par, first, push, s);
  }
  if (t.ndim != 2) return (int)cudaErrorInvalidValue;
  if (low == kLowF32) return low_tb2_typed<float, float, false>(t, in_par, out_par, first, push, s);
  if (r_bf16) return low_tb2_typed<__nv_bfloat16, __nv_bfloat16, false>(t, in_par, out_par, first, push, s);
  return low_tb2_typed<__nv_bfloat16, float, false>(t, in_par, out_par, first, push, s);
}

int launch_solve_ctl(SolveDev* solves, const int32_t* ctl, int nsolves, void* stream) {
  if (nsolves == 0) return 0;
  k_solve_ctl<<<grid_of(nsolves, 256), 256, 0, (cudaStream_t)stream>>>(solves, ctl, nsolves);
  return (int)cudaGetLastError();
}

}  // namespace jgb
