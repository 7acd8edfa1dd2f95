/*
 * Jacobi oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of the Jacobi
 * relaxation that the Jacobi3D proxy application runs (section 4.3: Jacobi
 * iterations, a set count of them, on a 3D domain cut into cuboid pieces), on
 * ONE monolithic grid with a one-cell ghost ring.  The
 * over-decomposition of section 4.4 changes how the work is split, not what
 * is computed, so the oracle has no blocks at all.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It shares no code, header or constant with the CUDA
 * path and never calls it.
 *
 * The paper never writes the equation out.  The readings adopted here:
 *   - Poisson -Lap(u) = f with Dirichlet values g on the ghost ring, unit grid
 *     spacing (f is supplied already scaled by h^2), the 3-point (1D),
 *     5-point (2D) or 7-point (3D) stencil, and the textbook Jacobi splitting
 *     with D = 2d I:  x'_p = (sum of the 2d neighbours of p + f_p) / (2d).
 *   - Two buffers, never in place (Jacobi, not Gauss-Seidel).
 *   - Summation order of one update (the "canonical" order; W/E, S/N, D/U
 *     are the -/+ neighbours along x, y, z):
 *         1D:    s = x_W + x_E
 *         2D:    s = (x_W + x_S) + (x_E + x_N)
 *         3D:    s = ((x_W + x_D) + (x_E + x_U)) + (x_S + x_N)
 *         t = s + f_p;      x'_p = t / (2d)   (IEEE division, round to nearest)
 *     i.e. the x pair is interleaved with the pair along the last axis.  Any
 *     fixed order gives a valid Jacobi iterate; this one is fixed so that two
 *     implementations can agree bit for bit.
 *   - Residual r_p = t_p - (2d) * x_p with the same t_p; it equals
 *     (b - A x)_p where A is the grid negative Laplacian and b holds f plus
 *     the Dirichlet values of ghost neighbours.
 *   - ||b||^2 is taken straight from its definition: b_p = f_p + (sum of the
 *     ghost neighbours of p).
 *   - Sums of squares use Neumaier's compensated summation, row by row, rows
 *     combined in index order, so the value does not depend on threads.
 *   - Mixed precision (iterative refinement): r is rounded to float (and
 *     optionally on to bfloat16, round-to-nearest-even), the correction e is
 *     swept in float arithmetic from e = 0 with zero Dirichlet ghosts, stored
 *     as float or as bfloat16 (RNE), and x += (double)e closes the step.
 *
 * Build: cc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * no fast-math), so every operation is one IEEE binary64 / binary32 rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { JO_OK = 0, JO_INVALID = 1, JO_OOM = 2, JO_NOT_CONVERGED = 4, JO_DIVERGED = 5 };

/* Grid with a one-cell ghost ring along each of its ndim axes. */
typedef struct {
  int ndim;
  int64_t n[3];   /* interior points along x, y, z (1 for missing axes)   */
  int64_t g[3];   /* ghost width along each axis (1 if axis used, else 0) */
  int64_t s[3];   /* strides of the ghost-ring array                       */
  int64_t total;  /* elements of the ghost-ring array                      */
} grid_t;

static int grid_init(grid_t* G, int ndim, const int64_t* n) {
  if (ndim < 1 || ndim > 3) return JO_INVALID;
  G->ndim = ndim;
  for (int a = 0; a < 3; a++) {
    G->n[a] = a < ndim ? n[a] : 1;
    G->g[a] = a < ndim ? 1 : 0;
    if (G->n[a] < 1) return JO_INVALID;
  }
  G->s[0] = 1;
  G->s[1] = G->n[0] + 2 * G->g[0];
  G->s[2] = G->s[1] * (G->n[1] + 2 * G->g[1]);
  G->total = G->s[2] * (G->n[2] + 2 * G->g[2]);
  return JO_OK;
}

/* Index of interior point (i, j, k) in the ghost-ring array; i, j, k may be
 * -1 or n to address ghosts. */
static inline int64_t gidx(const grid_t* G, int64_t i, int64_t j, int64_t k) {
  return (i + G->g[0]) * G->s[0] + (j + G->g[1]) * G->s[1] + (k + G->g[2]) * G->s[2];
}

/* Interior-dense index (x fastest). */
static inline int64_t didx(const grid_t* G, int64_t i, int64_t j, int64_t k) {
  return i + G->n[0] * (j + G->n[1] * k);
}

/* Copy the 2*ndim Dirichlet faces into the ghost ring.  Face order
 * -x,+x,-y,+y,-z,+z; a face lists the face's points with the remaining axes
 * in order, lowest axis fastest.  A NULL face means g = 0 on it. */
static void set_ghosts(const grid_t* G, double* a, const double* const* faces) {
  const int64_t nx = G->n[0], ny = G->n[1], nz = G->n[2];
  for (int64_t k = 0; k < nz; k++)
    for (int64_t j = 0; j < ny; j++) {
      a[gidx(G, -1, j, k)] = faces && faces[0] ? faces[0][j + ny * k] : 0.0;
      a[gidx(G, nx, j, k)] = faces && faces[1] ? faces[1][j + ny * k] : 0.0;
    }
  if (G->ndim >= 2)
    for (int64_t k = 0; k < nz; k++)
      for (int64_t i = 0; i < nx; i++) {
        a[gidx(G, i, -1, k)] = faces && faces[2] ? faces[2][i + nx * k] : 0.0;
        a[gidx(G, i, ny, k)] = faces && faces[3] ? faces[3][i + nx * k] : 0.0;
      }
  if (G->ndim == 3)
    for (int64_t j = 0; j < ny; j++)
      for (int64_t i = 0; i < nx; i++) {
        a[gidx(G, i, j, -1)] = faces && faces[4] ? faces[4][i + nx * j] : 0.0;
        a[gidx(G, i, j, nz)] = faces && faces[5] ? faces[5][i + nx * j] : 0.0;
      }
}

static void load_interior(const grid_t* G, double* a, const double* dense) {
  for (int64_t k = 0; k < G->n[2]; k++)
    for (int64_t j = 0; j < G->n[1]; j++)
      for (int64_t i = 0; i < G->n[0]; i++)
        a[gidx(G, i, j, k)] = dense ? dense[didx(G, i, j, k)] : 0.0;
}

static void store_interior(const grid_t* G, const double* a, double* dense) {
  for (int64_t k = 0; k < G->n[2]; k++)
    for (int64_t j = 0; j < G->n[1]; j++)
      for (int64_t i = 0; i < G->n[0]; i++)
        dense[didx(G, i, j, k)] = a[gidx(G, i, j, k)];
}

/* t_p: neighbour sum plus source in the canonical order (see header). */
static inline double neighbour_sum_plus_f(const grid_t* G, const double* a, int64_t p, double fp) {
  double s;
  if (G->ndim == 1) {
    s = a[p - G->s[0]] + a[p + G->s[0]];
  } else {
    const int64_t sl = G->s[G->ndim - 1];   /* stride of the last axis */
    s = (a[p - G->s[0]] + a[p - sl]) + (a[p + G->s[0]] + a[p + sl]);
    if (G->ndim == 3) s = s + (a[p - G->s[1]] + a[p + G->s[1]]);
  }
  return s + fp;
}

/* One Jacobi sweep over every interior point: dst = D^-1 (N src + b). */
static void sweep(const grid_t* G, const double* src, const double* f, double* dst) {
  const double two_d = 2.0 * G->ndim;
  const int64_t nx = G->n[0], ny = G->n[1], nz = G->n[2];
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t k = 0; k < nz; k++)
    for (int64_t j = 0; j < ny; j++)
      for (int64_t i = 0; i < nx; i++) {
        const int64_t p = gidx(G, i, j, k);
        const double fp = f ? f[didx(G, i, j, k)] : 0.0;
        dst[p] = neighbour_sum_plus_f(G, src, p, fp) / two_d;
      }
}

/* Neumaier compensated accumulation. */
typedef struct { double sum, comp; } acc_t;
static inline void acc_add(acc_t* a, double v) {
  const double t = a->sum + v;
  if (fabs(a->sum) >= fabs(v)) a->comp += (a->sum - t) + v;
  else a->comp += (v - t) + a->sum;
  a->sum = t;
}
static inline double acc_value(const acc_t* a) { return a->sum + a->comp; }

/* Sum over the interior of r_p^2 with r_p = t_p - 2d x_p; optionally also
 * stores r_p (interior-dense) into r_out. */
static double residual_ss(const grid_t* G, const double* a, const double* f, double* r_out) {
  const double two_d = 2.0 * G->ndim;
  const int64_t nx = G->n[0], ny = G->n[1], nz = G->n[2], rows = ny * nz;
  double* row_sum = (double*)malloc(sizeof(double) * (size_t)rows);
  if (!row_sum) return NAN;
#pragma omp parallel for schedule(static)
  for (int64_t row = 0; row < rows; row++) {
    const int64_t j = row % ny, k = row / ny;
    acc_t acc = {0.0, 0.0};
    for (int64_t i = 0; i < nx; i++) {
      const int64_t p = gidx(G, i, j, k);
      const double fp = f ? f[didx(G, i, j, k)] : 0.0;
      const double r = neighbour_sum_plus_f(G, a, p, fp) - two_d * a[p];
      if (r_out) r_out[didx(G, i, j, k)] = r;
      acc_add(&acc, r * r);
    }
    row_sum[row] = acc_value(&acc);
  }
  acc_t tot = {0.0, 0.0};
  for (int64_t row = 0; row < rows; row++) acc_add(&tot, row_sum[row]);
  free(row_sum);
  return acc_value(&tot);
}

/* ||b||^2 from its definition b_p = f_p + sum of ghost neighbours of p. */
static double rhs_ss(const grid_t* G, const double* a, const double* f) {
  const int64_t nx = G->n[0], ny = G->n[1], nz = G->n[2];
  acc_t tot = {0.0, 0.0};
  for (int64_t k = 0; k < nz; k++)
    for (int64_t j = 0; j < ny; j++)
      for (int64_t i = 0; i < nx; i++) {
        const int64_t p = gidx(G, i, j, k);
        double b = f ? f[didx(G, i, j, k)] : 0.0;
        if (i == 0) b += a[p - G->s[0]];
        if (i == nx - 1) b += a[p + G->s[0]];
        if (G->ndim >= 2 && j == 0) b += a[p - G->s[1]];
        if (G->ndim >= 2 && j == ny - 1) b += a[p + G->s[1]];
        if (G->ndim == 3 && k == 0) b += a[p - G->s[2]];
        if (G->ndim == 3 && k == nz - 1) b += a[p + G->s[2]];
        acc_add(&tot, b * b);
      }
  return acc_value(&tot);
}

/* threads > 0: use that many OpenMP threads; 0: the runtime's default (all
 * host cores unless OMP_NUM_THREADS says otherwise), restored even after an
 * earlier call asked for fewer. */
static void set_threads(int threads) {
#ifdef _OPENMP
  static int default_threads = 0;
  if (default_threads == 0) default_threads = omp_get_max_threads();
  omp_set_num_threads(threads > 0 ? threads : default_threads);
#else
  (void)threads;
#endif
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int jo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* nsweeps Jacobi sweeps; x (interior-dense) is updated in place. */
int jo_sweeps(int ndim, const int64_t* n, const double* const* faces, const double* f,
              double* x, int64_t nsweeps, int threads) {
  grid_t G;
  if (grid_init(&G, ndim, n) != JO_OK || nsweeps < 0) return JO_INVALID;
  set_threads(threads);
  double* a = (double*)calloc((size_t)G.total, sizeof(double));
  double* b = (double*)calloc((size_t)G.total, sizeof(double));
  if (!a || !b) { free(a); free(b); return JO_OOM; }
  set_ghosts(&G, a, faces);
  set_ghosts(&G, b, faces);
  load_interior(&G, a, x);
  for (int64_t it = 0; it < nsweeps; it++) {
    sweep(&G, a, f, b);
    double* t = a; a = b; b = t;
  }
  store_interior(&G, a, x);
  free(a); free(b);
  return JO_OK;
}

/* Sum of squares of the residual of x (rss) and of b (bss); r_out may be NULL. */
int jo_residual(int ndim, const int64_t* n, const double* const* faces, const double* f,
                const double* x, double* rss, double* bss, double* r_out, int threads) {
  grid_t G;
  if (grid_init(&G, ndim, n) != JO_OK) return JO_INVALID;
  set_threads(threads);
  double* a = (double*)calloc((size_t)G.total, sizeof(double));
  if (!a) return JO_OOM;
  set_ghosts(&G, a, faces);
  load_interior(&G, a, x);
  if (rss) *rss = residual_ss(&G, a, f, r_out);
  if (bss) *bss = rhs_ss(&G, a, f);
  free(a);
  return JO_OK;
}

static double relative(double rss, double bss) {
  return bss > 0.0 ? sqrt(rss) / sqrt(bss) : sqrt(rss);
}

/* Plain FP64 solve: the residual is tested at iterates 0, c, 2c, ... (c =
 * check_every) and the solve stops at the first one with rel <= tol, or when
 * max_sweeps sweeps have been done. */
int jo_solve(int ndim, const int64_t* n, const double* const* faces, const double* f,
             double* x, double tol, int64_t max_sweeps, int64_t check_every,
             int64_t* sweeps_out, double* rel_out, int threads) {
  grid_t G;
  if (grid_init(&G, ndim, n) != JO_OK || !(tol > 0.0) || max_sweeps < 0 || check_every < 1)
    return JO_INVALID;
  set_threads(threads);
  double* a = (double*)calloc((size_t)G.total, sizeof(double));
  double* b = (double*)calloc((size_t)G.total, sizeof(double));
  if (!a || !b) { free(a); free(b); return JO_OOM; }
  set_ghosts(&G, a, faces);
  set_ghosts(&G, b, faces);
  load_interior(&G, a, x);
  const double bss = rhs_ss(&G, a, f);
  int64_t m = 0;
  int status;
  double rel;
  for (;;) {
    rel = relative(residual_ss(&G, a, f, NULL), bss);
    if (!isfinite(rel)) { status = JO_DIVERGED; break; }
    if (rel <= tol) { status = JO_OK; break; }
    if (m >= max_sweeps) { status = JO_NOT_CONVERGED; break; }
    const int64_t k = check_every < max_sweeps - m ? check_every : max_sweeps - m;
    for (int64_t it = 0; it < k; it++) {
      sweep(&G, a, f, b);
      double* t = a; a = b; b = t;
    }
    m += k;
  }
  store_interior(&G, a, x);
  if (sweeps_out) *sweeps_out = m;
  if (rel_out) *rel_out = rel;
  free(a); free(b);
  return status;
}

/* ---- mixed precision: bfloat16 storage and float inner sweeps ---------- */

/* float -> bfloat16 -> float, rounding to nearest, ties to even, done on the
 * bit pattern: add 0x7FFF plus the lowest kept bit, then clear the low half. */
static inline float round_bf16(float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) {
    u |= 0x00400000u;             /* NaN stays NaN (quiet) */
  } else {
    u += 0x7FFFu + ((u >> 16) & 1u);
  }
  u &= 0xFFFF0000u;
  memcpy(&v, &u, 4);
  return v;
}

/* Exposed so a test can pin the rounding against a library conversion. */
float jo_round_bf16(float v) { return round_bf16(v); }

/* One float Jacobi sweep of A e = r with zero Dirichlet ghosts. */
static void sweep_low(const grid_t* G, const float* src, const float* r, float* dst, int e_bf16) {
  const float two_d = (float)(2 * G->ndim);
  const int64_t nx = G->n[0], ny = G->n[1], nz = G->n[2];
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t k = 0; k < nz; k++)
    for (int64_t j = 0; j < ny; j++)
      for (int64_t i = 0; i < nx; i++) {
        const int64_t p = gidx(G, i, j, k);
        float s;
        if (G->ndim == 1) {
          s = src[p - G->s[0]] + src[p + G->s[0]];
        } else {
          const int64_t sl = G->s[G->ndim - 1];
          s = (src[p - G->s[0]] + src[p - sl]) + (src[p + G->s[0]] + src[p + sl]);
          if (G->ndim == 3) s = s + (src[p - G->s[1]] + src[p + G->s[1]]);
        }
        const float t = s + r[didx(G, i, j, k)];
        const float v = t / two_d;
        dst[p] = e_bf16 ? round_bf16(v) : v;
      }
}

/* Mixed-precision iterative refinement (FP64 outer, float inner):
 *   repeat: [x += e]; r = b - A x (FP64); stop if rel(r) <= tol;
 *           r_low = round(r); e = 0; k float sweeps of A e = r_low.
 * k = period (the last step is shortened so that at most max_sweeps inner
 * sweeps run).  sweeps_out counts inner sweeps. */
int jo_refine_solve(int ndim, const int64_t* n, const double* const* faces, const double* f,
                    double* x, int e_bf16, int r_bf16, int64_t period, double tol,
                    int64_t max_sweeps, int64_t* sweeps_out, double* rel_out, int threads) {
  grid_t G;
  if (grid_init(&G, ndim, n) != JO_OK || period < 1 || max_sweeps < 0 || !(tol > 0.0))
    return JO_INVALID;
  set_threads(threads);
  const int64_t N = G.n[0] * G.n[1] * G.n[2];
  double* a = (double*)calloc((size_t)G.total, sizeof(double));
  double* r = (double*)malloc(sizeof(double) * (size_t)N);
  float* rl = (float*)malloc(sizeof(float) * (size_t)N);
  float* e0 = (float*)calloc((size_t)G.total, sizeof(float));
  float* e1 = (float*)calloc((size_t)G.total, sizeof(float));
  if (!a || !r || !rl || !e0 || !e1) {
    free(a); free(r); free(rl); free(e0); free(e1);
    return JO_OOM;
  }
  set_ghosts(&G, a, faces);
  load_interior(&G, a, x);
  const double bss = rhs_ss(&G, a, f);
  int64_t m = 0;
  int first = 1, status;
  double rel;
  float* e = e0;
  for (;;) {
    if (!first) {
      for (int64_t k = 0; k < G.n[2]; k++)
        for (int64_t j = 0; j < G.n[1]; j++)
          for (int64_t i = 0; i < G.n[0]; i++) {
            const int64_t p = gidx(&G, i, j, k);
            a[p] = a[p] + (double)e[p];
          }
    }
    first = 0;
    rel = relative(residual_ss(&G, a, f, r), bss);
    if (!isfinite(rel)) { status = JO_DIVERGED; break; }
    if (rel <= tol) { status = JO_OK; break; }
    if (m >= max_sweeps) { status = JO_NOT_CONVERGED; break; }
    const int64_t ksw = period < max_sweeps - m ? period : max_sweeps - m;
    for (int64_t q = 0; q < N; q++) {
      const float v = (float)r[q];
      rl[q] = r_bf16 ? round_bf16(v) : v;
    }
    memset(e0, 0, sizeof(float) * (size_t)G.total);
    memset(e1, 0, sizeof(float) * (size_t)G.total);
    float* src = e0;
    float* dst = e1;
    for (int64_t it = 0; it < ksw; it++) {
      sweep_low(&G, src, rl, dst, e_bf16);
      float* t = src; src = dst; dst = t;
    }
    e = src;
    m += ksw;
  }
  store_interior(&G, a, x);
  if (sweeps_out) *sweeps_out = m;
  if (rel_out) *rel_out = rel;
  free(a); free(r); free(rl); free(e0); free(e1);
  return status;
}
