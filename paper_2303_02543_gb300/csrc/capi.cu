// extern "C" entry points declared in include/jacobi.h.  Every entry point
// catches internal errors and turns them into a jacobi_status plus a message.
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/jacobi.h"
#include "engine.h"

using namespace jgb;

struct jacobi_ctx {
  Workset* ws = nullptr;
  int slot = 0;
  std::string err;
};

static thread_local std::string t_err;

namespace jgb {
// Records the calling thread's last error for entry points without a context.
void set_thread_error(const std::string& msg) { t_err = msg; }
}  // namespace jgb

#define API_BEGIN try {
#define API_END(ctx)                                              \
  }                                                               \
  catch (const JErr& e) {                                         \
    if (ctx) (ctx)->err = e.msg;                                  \
    t_err = e.msg;                                                \
    return (jacobi_status)e.code;                                 \
  }                                                               \
  catch (const std::bad_alloc&) {                                 \
    if (ctx) (ctx)->err = "host allocation failed";               \
    t_err = "host allocation failed";                             \
    return JACOBI_ERR_OOM;                                        \
  }                                                               \
  catch (...) {                                                   \
    if (ctx) (ctx)->err = "unexpected internal error";            \
    t_err = "unexpected internal error";                          \
    return JACOBI_ERR_INVALID;                                    \
  }

static void require(bool ok, const std::string& msg) {
  if (!ok) throw JErr{JACOBI_ERR_INVALID, msg};
}

// ---------------------------------------------------------------------------
// solve loops shared by the single-grid context

static double rel_of(double rss, double bss) { return bss > 0.0 ? std::sqrt(rss) / std::sqrt(bss) : std::sqrt(rss); }

// Plain FP64: the residual of iterate m is reduced inside sweep m+1 (the
// last sweep of a chunk); when the test passes, the phase flips back so the
// field is iterate m again.  One extra sweep is run and discarded.
static jacobi_status solve_f64(Workset& ws, int slot, double tol, int64_t max_sweeps, int64_t* done, double* rel_out) {
  SolveHost* s = ws.solve(slot);
  const int64_t c = ws.opt.check_every;
  std::vector<double> rss;
  int64_t m = 0;
  ws.sweeps_f64(1, true);
  jacobi_status st;
  double rel;
  for (;;) {
    ws.read_rss(rss);
    rel = rel_of(rss[slot], s->bss);
    if (!std::isfinite(rel)) {
      st = JACOBI_ERR_DIVERGED;
      break;
    }
    if (rel <= tol) {
      st = JACOBI_OK;
      break;
    }
    if (m >= max_sweeps) {
      st = JACOBI_ERR_NOT_CONVERGED;
      break;
    }
    const int64_t n = std::min(c, max_sweeps - m);
    ws.sweeps_f64(n, true);
    m += n;
  }
  ws.phase_advance(1, -1);  // back to iterate m
  if (done) *done = m;
  if (rel_out) *rel_out = rel;
  return st;
}

// Refinement: outer step (x += e, r = b - A x in FP64, residual), then
// refine_period inner sweeps; the test follows every outer step.
static jacobi_status solve_refine(Workset& ws, int slot, double tol, int64_t max_sweeps, int64_t* done,
                                  double* rel_out) {
  SolveHost* s = ws.solve(slot);
  const int64_t k = ws.opt.refine_period;
  std::vector<double> rss;
  int64_t m = 0;
  jacobi_status st;
  double rel;
  for (;;) {
    ws.refine_outer();
    ws.read_rss(rss);
    rel = rel_of(rss[slot], s->bss);
    if (!std::isfinite(rel)) {
      st = JACOBI_ERR_DIVERGED;
      break;
    }
    if (rel <= tol) {
      st = JACOBI_OK;
      break;
    }
    if (m >= max_sweeps) {
      st = JACOBI_ERR_NOT_CONVERGED;
      break;
    }
    const int64_t n = std::min(k, max_sweeps - m);
    ws.refine_inner(n);
    m += n;
  }
  ws.phase_advance(0, 0);  // the correction has been applied
  if (done) *done = m;
  if (rel_out) *rel_out = rel;
  return st;
}

// ---------------------------------------------------------------------------

extern "C" {

void jacobi_set_allocator(void* (*alloc)(size_t, void*, void*), void (*free_fn)(void*, void*, void*), void* user) {
  AllocHooks h;
  h.alloc = alloc;
  h.free = free_fn;
  h.user = user;
  if (!alloc || !free_fn) h = AllocHooks();
  set_alloc_hooks(h);
}

int jacobi_version(void) { return 10000; }

static void fill_spec(ProblemSpec& p, int ndim, const int64_t dims[3], const int64_t block[3], const jacobi_boundary* bc,
                      const double* source, const double* x0) {
  require(ndim == 2 || ndim == 3, "ndim must be 2 or 3");
  require(dims != nullptr && block != nullptr, "dims and block are required");
  p.ndim = ndim;
  for (int a = 0; a < 3; ++a) {
    p.n[a] = a < ndim ? dims[a] : 1;
    p.blk[a] = a < ndim ? block[a] : 1;
    require(p.n[a] >= 1, "every dimension must be >= 1");
    require(p.blk[a] >= 1 && p.blk[a] <= p.n[a], "block extents must satisfy 1 <= block <= dims");
    require(p.n[a] < (1LL << 30), "dimension too large");
  }
  int64_t nblocks = 1;
  for (int a = 0; a < ndim; ++a) nblocks *= (p.n[a] + p.blk[a] - 1) / p.blk[a];
  require(nblocks < (1LL << 28), "too many blocks");
  if (bc) {
    require(bc->kind >= 0 && bc->kind <= 2, "unknown boundary kind");
    p.bc_kind = bc->kind;
    p.bc_value = bc->value;
    for (int q = 0; q < 6; ++q) p.faces[q] = bc->faces[q];
  }
  p.source = source;
  p.x0 = x0;
}

jacobi_status jacobi_create(jacobi_t* out, int ndim, const int64_t dims[3], const int64_t block[3], int dtype,
                            const jacobi_boundary* bc, const double* source, const double* x0, void* cuda_stream) {
  jacobi_ctx* ctx = nullptr;
  API_BEGIN
  require(out != nullptr, "out is NULL");
  *out = nullptr;
  require(dtype >= 0 && dtype <= 2, "unknown dtype");
  ProblemSpec p;
  fill_spec(p, ndim, dims, block, bc, source, x0);
  ctx = new jacobi_ctx();
  try {
    ctx->ws = new Workset(ndim, dtype, (cudaStream_t)cuda_stream, 1);
    ctx->slot = ctx->ws->add_solve(p);
  } catch (...) {
    delete ctx->ws;
    delete ctx;
    ctx = nullptr;
    throw;
  }
  *out = ctx;
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_sweep(jacobi_t ctx, int64_t n) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  require(n >= 0, "n must be >= 0");
  Workset& ws = *ctx->ws;
  if (!ws.refine()) {
    ws.sweeps_f64(n, false);
  } else if (n > 0) {
    int64_t doneq = 0;
    while (doneq < n) {
      const int64_t k = std::min<int64_t>(ws.opt.refine_period, n - doneq);
      ws.refine_outer();
      ws.refine_inner(k);
      doneq += k;
    }
    ws.refine_outer();       // apply the last correction
    ws.phase_advance(0, 0);  // nothing pending
  }
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_residual(jacobi_t ctx, double* rel, double* abs) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  Workset& ws = *ctx->ws;
  ws.residual_only();
  std::vector<double> rss;
  ws.read_rss(rss);
  const double r = rss[ctx->slot];
  if (rel) *rel = rel_of(r, ws.solve(ctx->slot)->bss);
  if (abs) *abs = std::sqrt(r);
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_solve(jacobi_t ctx, double tol, int64_t max_sweeps, int64_t* sweeps_done, double* final_rel) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  require(tol > 0.0, "tol must be > 0");
  require(max_sweeps >= 0, "max_sweeps must be >= 0");
  Workset& ws = *ctx->ws;
  return ws.refine() ? solve_refine(ws, ctx->slot, tol, max_sweeps, sweeps_done, final_rel)
                     : solve_f64(ws, ctx->slot, tol, max_sweeps, sweeps_done, final_rel);
  API_END(ctx)
}

jacobi_status jacobi_get_field(jacobi_t ctx, double* out, int on_device) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  require(out != nullptr, "out is NULL");
  ctx->ws->gather(ctx->slot, out, on_device);
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_set_field(jacobi_t ctx, const double* in, int on_device) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  require(in != nullptr, "in is NULL");
  Workset& ws = *ctx->ws;
  ws.scatter(ctx->slot, in, 0, on_device);
  ws.halo_exchange_x(0);
  ws.phase_advance(0, 0);
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_set_source(jacobi_t ctx, const double* in, int on_device) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  require(in != nullptr, "in is NULL");
  Workset& ws = *ctx->ws;
  SolveHost* s = ws.solve(ctx->slot);
  ws.scatter(ctx->slot, in, 1, on_device);
  // ||b|| changes with f: recompute it as the residual of the zero field
  std::vector<double> zero((size_t)s->points(), 0.0);
  std::vector<double> cur((size_t)s->points());
  ws.gather(ctx->slot, cur.data(), 0);
  ws.scatter(ctx->slot, zero.data(), 0, 0);
  ws.halo_exchange_x(0);
  ws.residual_only();
  std::vector<double> rss;
  ws.read_rss(rss);
  s->bss = rss[ctx->slot];
  ws.scatter(ctx->slot, cur.data(), 0, 0);
  ws.halo_exchange_x(0);
  ws.sync();
  return JACOBI_OK;
  API_END(ctx)
}

static int64_t* option_slot(Options& o, const char* key) {
  if (!key) return nullptr;
  if (!strcmp(key, "check_every")) return &o.check_every;
  if (!strcmp(key, "refine_period")) return &o.refine_period;
  if (!strcmp(key, "halo")) return &o.halo;
  if (!strcmp(key, "rows_f64")) return &o.rows_f64;
  if (!strcmp(key, "rows_low")) return &o.rows_low;
  if (!strcmp(key, "r_bf16")) return &o.r_bf16;
  if (!strcmp(key, "profile")) return &o.profile;
  return nullptr;
}

jacobi_status jacobi_set_option(jacobi_t ctx, const char* key, int64_t value) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  Workset& ws = *ctx->ws;
  int64_t* p = option_slot(ws.opt, key);
  require(p != nullptr, std::string("unknown option ") + (key ? key : "(null)"));
  if (!strcmp(key, "check_every") || !strcmp(key, "refine_period") || !strcmp(key, "rows_f64") ||
      !strcmp(key, "rows_low"))
    require(value >= 1, std::string(key) + " must be >= 1");
  if (!strcmp(key, "halo") || !strcmp(key, "profile")) require(value == 0 || value == 1, std::string(key) + " must be 0 or 1");
  if (!strcmp(key, "r_bf16")) require(false, "r_bf16 is fixed when the context is created");
  const bool retable = (!strcmp(key, "rows_f64") || !strcmp(key, "rows_low")) && *p != value;
  *p = value;
  if (retable) ws.rebuild_tables();
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_get_option(jacobi_t ctx, const char* key, int64_t* value) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  int64_t* p = option_slot(ctx->ws->opt, key);
  require(p != nullptr && value != nullptr, "unknown option or NULL value");
  *value = *p;
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_profile(jacobi_t ctx, const char* kernel, double* total_ms, int64_t* launches, int reset) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  require(kernel != nullptr, "kernel is NULL");
  int k = -1;
  if (!strcmp(kernel, "sweep_f64")) k = kProfSweepF64;
  else if (!strcmp(kernel, "sweep_low")) k = kProfSweepLow;
  else if (!strcmp(kernel, "refine_outer")) k = kProfOuter;
  else if (!strcmp(kernel, "reduce")) k = kProfReduce;
  else if (!strcmp(kernel, "halo")) k = kProfHalo;
  if (!strcmp(kernel, "all")) {  // every kernel launched by this context so far
    ctx->ws->sync();
    if (total_ms) *total_ms = 0.0;
    if (launches) *launches = ctx->ws->launches();
    return JACOBI_OK;
  }
  require(k >= 0, "unknown kernel class");
  ctx->ws->prof_collect(k, total_ms, launches, reset != 0);
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_device_bytes(jacobi_t ctx, int64_t* bytes) {
  if (!ctx || !bytes) return JACOBI_ERR_INVALID;
  *bytes = ctx->ws->device_bytes();
  return JACOBI_OK;
}

void jacobi_destroy(jacobi_t ctx) {
  if (!ctx) return;
  try {
    delete ctx->ws;
  } catch (...) {
  }
  delete ctx;
}

const char* jacobi_last_error(jacobi_t ctx) { return ctx ? ctx->err.c_str() : t_err.c_str(); }

}  // extern "C"
