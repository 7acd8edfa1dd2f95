// extern "C" entry points declared in include/jacobi.h.  Every entry point
// catches internal errors and turns them into a jacobi_status plus a message.
#include <cmath>
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/jacobi.h"
#include "engine.h"

using namespace jgb;

// NVTX range around one entry point (visible on profiler timelines; free
// when no profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

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

static double rel_of(double rss, double bss) { return bss > 0.0 ? std::sqrt(rss) / std::sqrt(bss) : std::sqrt(rss); }

static void require_single(jacobi_ctx* ctx) {
  require(ctx->ws->live() == 1, "this call needs a single-grid context; use the jacobi_batch_* calls");
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
  NvtxRange nvtx_range_("jacobi_create");
  API_BEGIN
  require(out != nullptr, "out is NULL");
  *out = nullptr;
  require(dtype >= 0 && dtype <= 3, "unknown dtype");
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
  NvtxRange nvtx_range_("jacobi_sweep");
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
  NvtxRange nvtx_range_("jacobi_residual");
  API_BEGIN
  require_single(ctx);
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
  NvtxRange nvtx_range_("jacobi_solve");
  API_BEGIN
  require(tol > 0.0, "tol must be > 0");
  require(max_sweeps >= 0, "max_sweeps must be >= 0");
  require_single(ctx);
  std::vector<SlotResult> res;
  ctx->ws->solve_all(tol, max_sweeps, res);
  const SlotResult& r = res[ctx->slot];
  if (sweeps_done) *sweeps_done = r.sweeps;
  if (final_rel) *final_rel = r.rel;
  if (r.status != JACOBI_OK) {
    const std::string what = r.status == JACOBI_ERR_DIVERGED        ? "diverged"
                             : r.status == JACOBI_ERR_NOT_CONVERGED ? "not converged"
                                                                    : "stopped (status " + std::to_string(r.status) + ")";
    ctx->err = what + " after " + std::to_string(r.sweeps) + " sweeps (relative residual " + std::to_string(r.rel) + ")";
    t_err = ctx->err;
  }
  return (jacobi_status)r.status;
  API_END(ctx)
}

jacobi_status jacobi_get_field(jacobi_t ctx, double* out, int on_device) {
  if (!ctx) return JACOBI_ERR_INVALID;
  NvtxRange nvtx_range_("jacobi_get_field");
  API_BEGIN
  require(out != nullptr, "out is NULL");
  require_single(ctx);
  ctx->ws->gather(ctx->slot, out, on_device);
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_set_field(jacobi_t ctx, const double* in, int on_device) {
  if (!ctx) return JACOBI_ERR_INVALID;
  NvtxRange nvtx_range_("jacobi_set_field");
  API_BEGIN
  require(in != nullptr, "in is NULL");
  require_single(ctx);
  Workset& ws = *ctx->ws;
  ws.scatter(ctx->slot, in, 0, on_device);
  ws.halo_exchange_x(0);
  ws.phase_advance(0, 0);
  return JACOBI_OK;
  API_END(ctx)
}

jacobi_status jacobi_set_source(jacobi_t ctx, const double* in, int on_device) {
  if (!ctx) return JACOBI_ERR_INVALID;
  NvtxRange nvtx_range_("jacobi_set_source");
  API_BEGIN
  require(in != nullptr, "in is NULL");
  require_single(ctx);
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
  if (!strcmp(key, "profile")) return &o.profile;
  if (!strcmp(key, "schedule")) return &o.schedule;
  if (!strcmp(key, "graph")) return &o.graph;
  if (!strcmp(key, "spin_limit")) return &o.spin_limit;
  if (!strcmp(key, "poison_wait")) return &o.poison_wait;
  if (!strcmp(key, "autotune")) return &o.autotune;
  if (!strcmp(key, "emu_adds")) return &o.emu_adds;
  if (!strcmp(key, "tma")) return &o.tma;
  if (!strcmp(key, "stage3")) return &o.stage3;
  if (!strcmp(key, "march")) return &o.march;
  if (!strcmp(key, "outer_split")) return &o.outer_split;
  if (!strcmp(key, "l2pf")) return &o.l2pf;
  if (!strcmp(key, "tb")) return &o.tb;
  return nullptr;
}

jacobi_status jacobi_set_option(jacobi_t ctx, const char* key, int64_t value) {
  if (!ctx) return JACOBI_ERR_INVALID;
  API_BEGIN
  Workset& ws = *ctx->ws;
  int64_t* p = option_slot(ws.opt, key);
  require(p != nullptr, std::string("unknown option ") + (key ? key : "(null)"));
  const std::string k(key);
  if (k == "check_every" || k == "rows_f64") require(value >= 1, k + " must be >= 1");
  if (k == "rows_low") require(value >= 0, "rows_low must be >= 0 (0: automatic)");
  if (k == "refine_period") require(value >= 1 && value <= 4096, "refine_period must be in [1, 4096]");
  if (k == "halo" || k == "profile" || k == "schedule" || k == "graph" || k == "poison_wait" || k == "autotune" ||
      k == "tma" || k == "outer_split" || k == "stage3")
    require(value == 0 || value == 1, k + " must be 0 or 1");
  if (k == "march") require(value >= 0 && value <= 3, "march must be in [0, 3]");
  if (k == "l2pf") require(value >= 0 && value <= 64, "l2pf must be in [0, 64]");
  if (k == "tb") require(value >= 0 && value <= 2, "tb must be 0, 1 or 2");
  const bool remarch = k == "march" && *p != value && ws.ndim() == 2;
  if (k == "spin_limit") require(value >= 0 && value <= 0x7fffffff, "spin_limit must be in [0, 2^31)");
  if (k == "emu_adds") require(value == 0 || value == 2 || value == 3, "emu_adds must be 0, 2 or 3");
  const bool retable = ((k == "rows_f64" || k == "rows_low" || k == "tb") && *p != value) || remarch;
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
  if (!strcmp(kernel, "graph")) {
    ctx->ws->sync();
    if (total_ms) *total_ms = 0.0;
    if (launches) *launches = ctx->ws->graph_replays();
    return JACOBI_OK;
  }
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

jacobi_status jacobi_batch_create(jacobi_t* out, int n, const jacobi_problem* probs, int dtype, void* cuda_stream) {
  jacobi_ctx* ctx = nullptr;
  NvtxRange nvtx_range_("jacobi_batch_create");
  API_BEGIN
  require(out != nullptr, "out is NULL");
  *out = nullptr;
  require(n >= 1 && n <= (1 << 20), "n must be in [1, 2^20]");
  require(probs != nullptr, "probs is NULL");
  require(dtype >= 0 && dtype <= 3, "unknown dtype");
  std::vector<ProblemSpec> specs((size_t)n);
  for (int i = 0; i < n; ++i) {
    fill_spec(specs[i], probs[i].ndim, probs[i].dims, probs[i].block, &probs[i].bc, probs[i].source, probs[i].x0);
    require(specs[i].ndim == specs[0].ndim, "every problem of a batch must have the same ndim");
  }
  ctx = new jacobi_ctx();
  try {
    ctx->ws = new Workset(specs[0].ndim, dtype, (cudaStream_t)cuda_stream, n);
    for (int i = 0; i < n; ++i) ctx->ws->add_solve(specs[i]);
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

jacobi_status jacobi_batch_solve(jacobi_t ctx, double tol, int64_t max_sweeps, jacobi_result* results) {
  if (!ctx) return JACOBI_ERR_INVALID;
  NvtxRange nvtx_range_("jacobi_batch_solve");
  API_BEGIN
  require(tol > 0.0, "tol must be > 0");
  require(max_sweeps >= 0, "max_sweeps must be >= 0");
  std::vector<SlotResult> res;
  ctx->ws->solve_all(tol, max_sweeps, res);
  jacobi_status worst = JACOBI_OK;
  for (int i = 0; i < ctx->ws->capacity(); ++i) {
    if (!ctx->ws->solve(i)) continue;
    if (results) {
      results[i].status = res[i].status;
      results[i].reserved = 0;
      results[i].sweeps = res[i].sweeps;
      results[i].rel = res[i].rel;
      results[i].seconds = res[i].seconds;
    }
    if (res[i].status != JACOBI_OK && worst == JACOBI_OK) worst = (jacobi_status)res[i].status;
  }
  return worst;
  API_END(ctx)
}

jacobi_status jacobi_batch_get_field(jacobi_t ctx, int i, double* out, int on_device) {
  if (!ctx) return JACOBI_ERR_INVALID;
  NvtxRange nvtx_range_("jacobi_batch_get_field");
  API_BEGIN
  require(out != nullptr, "out is NULL");
  require(ctx->ws->solve(i) != nullptr, "no such problem index");
  ctx->ws->gather(i, out, on_device);
  return JACOBI_OK;
  API_END(ctx)
}

}  // extern "C"
