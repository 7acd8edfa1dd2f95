// Serving loop: continuous batching of Jacobi solves under an HBM budget.
//
// Requests arrive through jacobi_server_submit from any thread.  One driver
// thread per server (the dedicated per-device thread of section 4.1.6) owns
// the GPU work: between refinement steps it retires finished solves (copying
// their fields to host memory and freeing their state) and admits queued
// requests while their device memory fits in the budget.  Every admitted
// solve's state stays resident until it finishes; all active solves of one
// dimensionality advance together in the same launches.
//
// Device memory comes from one arena allocated at creation (the custom
// device memory pool of section 4.1.2): the driver thread never calls an
// allocator outside the library, and admission is exact.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <cmath>
#include <thread>

#include <nvtx3/nvToolsExt.h>

#include "../../include/jacobi.h"
#include "engine.h"
#include "first_fit.h"

using namespace jgb;

namespace jgb {
void set_thread_error(const std::string& msg);
}

namespace {

// First-fit arena over one device allocation (placement in first_fit.h).
class Arena {
 public:
  bool init(size_t bytes, const AllocHooks& hooks, cudaStream_t s) {
    hooks_ = hooks;
    stream_ = s;
    const size_t size = FirstFit::round_up(bytes);
    if (hooks_.alloc) base_ = (char*)hooks_.alloc(size, (void*)s, hooks_.user);
    else if (cudaMalloc((void**)&base_, size) != cudaSuccess) base_ = nullptr;
    if (!base_) {
      cudaGetLastError();
      return false;
    }
    fit_.reset(size);
    return true;
  }
  ~Arena() {
    if (!base_) return;
    cudaStreamSynchronize(stream_);
    if (hooks_.free) hooks_.free(base_, (void*)stream_, hooks_.user);
    else cudaFree(base_);
  }
  void* alloc(size_t n) {
    std::lock_guard<std::mutex> lk(mu_);
    const size_t off = fit_.alloc(n);
    return off == FirstFit::npos ? nullptr : base_ + off;
  }
  void release(void* p) {
    std::lock_guard<std::mutex> lk(mu_);
    fit_.release((size_t)((char*)p - base_));
  }
  size_t in_use() {
    std::lock_guard<std::mutex> lk(mu_);
    return fit_.in_use();
  }
  size_t size() const { return fit_.size(); }

  static void* hook_alloc(size_t n, void*, void* user) { return ((Arena*)user)->alloc(n); }
  static void hook_free(void* p, void*, void* user) { ((Arena*)user)->release(p); }

 private:
  AllocHooks hooks_;
  cudaStream_t stream_ = nullptr;
  char* base_ = nullptr;
  FirstFit fit_;
  std::mutex mu_;
};

// Page-locked host staging for the dense fields of admitted and retired
// solves.  The layout kernels read and write it directly over the host link,
// so neither admission nor retirement takes a device temporary from the arena
// (a retirement must not fail for want of arena space).  It only grows: every
// admission sizes it for its solve, so a retirement never allocates.
class PinnedStage {
 public:
  ~PinnedStage() {
    if (p_) cudaFreeHost(p_);
  }
  double* get(size_t n) {
    if (n > n_) {
      if (p_) cudaFreeHost(p_);
      p_ = nullptr;
      n_ = 0;
      if (cudaMallocHost((void**)&p_, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        p_ = nullptr;
        throw JErr{JACOBI_ERR_OOM, "page-locked host staging of " + std::to_string(n * sizeof(double)) +
                                       " bytes failed"};
      }
      n_ = n;
    }
    return p_;
  }

 private:
  double* p_ = nullptr;
  size_t n_ = 0;
};

struct Request {
  uint64_t ticket = 0;
  ProblemSpec spec;
  std::vector<double> faces[6], source, x0;
  double tol = 1e-8;
  int64_t max_sweeps = 0;
  int64_t bytes = 0;
  std::chrono::steady_clock::time_point t_submit;
  // a solve that was evicted and waits to resume: inner sweeps done so far
  // (x0 holds its iterate) and how often it has been evicted
  int64_t resume_sweeps = 0;
  int evictions = 0;
  int64_t waited_steps = 0;  // driver steps spent at the head of the queue
};

struct Active {
  uint64_t ticket = 0;
  int64_t sweeps = 0;
  bool had_outer = false;
  double tol = 1e-8;
  int64_t max_sweeps = 0;
  int64_t points = 0;
  std::chrono::steady_clock::time_point t_submit;
  int64_t steps_resident = 0;  // driver steps since this admission
  Request req;                 // the inputs, kept on the host for a resume after an eviction
};

struct Done {
  jacobi_result res;
  std::vector<double> field;
};

}  // namespace

struct jacobi_server {
  int dtype = 1;
  int device = 0;
  int max_slots = 64;
  cudaStream_t stream = nullptr;
  Options opt;
  Arena arena;
  PinnedStage stage;                    // driver thread only
  Workset* ws[2] = {nullptr, nullptr};  // 2D, 3D
  std::map<int, Active> active[2];      // slot -> solve
  std::deque<Request> queue;
  std::map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::thread driver;
  bool stop = false;
  bool started = false;                 // a request was submitted: options are fixed
  std::string fatal;                    // set when the driver thread fails
  jacobi_server_stats stats;
  std::string err;
  // eviction under HBM pressure (options "evict", "evict_min_steps",
  // "evict_wait_steps", "max_evictions")
  bool evict = false;
  int64_t evict_min_steps = 20;
  int64_t evict_wait_steps = 2;
  int64_t max_evictions = 2;

  ~jacobi_server() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_all();
    if (driver.joinable()) driver.join();
    delete ws[0];
    delete ws[1];
  }

  Workset* workset(int ndim) {
    Workset*& w = ws[ndim - 2];
    if (!w) {
      AllocHooks h;
      h.alloc = &Arena::hook_alloc;
      h.free = &Arena::hook_free;
      h.user = &arena;
      w = new Workset(ndim, dtype, stream, max_slots, dtype == 3, &h);
      w->opt = opt;
    }
    return w;
  }

  void loop();
  bool step_once();
  bool maybe_evict();
};

// Eviction (the memory monitor with offload of section 3.1.1, between
// refinement steps).  For the oldest queued request that has waited
// evict_wait_steps driver steps for room in the arena or a slot and still
// does not fit, the resident solve that has run longest since its admission
// (at least evict_min_steps steps; evicted fewer than max_evictions times; at
// least twice the waiting request's points; of the waiting request's
// dimensionality when it lacks a slot) is evicted: its iterate is copied to host memory
// through the page-locked stage, its device state is freed, and it joins the
// back of the queue with its inputs and its inner-sweep count.  When it is
// admitted again it is a new solve whose initial field is that iterate: its
// first step computes r of that field (the r it had when it left, bit for
// bit) and is not counted, so its later steps, its field and its sweep count
// equal those of a solve that never left.
bool jacobi_server::maybe_evict() {
  if (!evict) return false;
  struct Waiting {
    int d;
    int64_t need, points, waited;
  };
  std::vector<Waiting> waiting;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (Request& h : queue) {
      h.waited_steps += 1;
      const int d = h.spec.ndim - 2;
      waiting.push_back(Waiting{d, h.bytes + h.bytes / 16 + (ws[d] ? 0 : (int64_t)(1 << 20)),
                                h.spec.n[0] * h.spec.n[1] * h.spec.n[2], h.waited_steps});
    }
  }
  const int64_t room = (int64_t)arena.size() - (int64_t)arena.in_use();
  // the oldest request that has waited long enough and does not fit, and a
  // resident solve to give way for it
  for (const Waiting& h : waiting) {
    if (h.waited < evict_wait_steps) continue;
    const bool slot_free = (int)active[h.d].size() < max_slots;
    if (h.need <= room && slot_free) continue;  // it fits: admission will take it
    int vd = -1, vslot = -1;
    int64_t best = -1;
    for (int dd = 0; dd < 2; ++dd) {
      if (!slot_free && dd != h.d) continue;
      for (auto& kv : active[dd]) {
        const Active& a = kv.second;
        // only a solve at least twice the waiting one's size gives way (two
        // solves of similar size never evict each other)
        if (a.steps_resident < evict_min_steps || a.req.evictions >= max_evictions || a.points < 2 * h.points)
          continue;
        if (a.steps_resident > best) {
          best = a.steps_resident;
          vd = dd;
          vslot = kv.first;
        }
      }
    }
    if (vd < 0) continue;
    Workset* w = ws[vd];
    Active& a = active[vd][vslot];
    double* staged = stage.get((size_t)a.points);  // sized at its admission: no allocation
    w->gather(vslot, staged, 0);
    Request r = std::move(a.req);
    r.x0.assign(staged, staged + a.points);
    r.spec.x0 = r.x0.data();
    r.resume_sweeps = a.sweeps;
    r.evictions += 1;
    r.waited_steps = 0;
    w->remove_solve(vslot);
    active[vd].erase(vslot);
    std::lock_guard<std::mutex> lk(mu);
    queue.push_back(std::move(r));
    stats.evictions += 1;
    return true;  // one eviction per driver pass
  }
  return false;
}

// One pass of the driver: admit, step every workset once, retire.
bool jacobi_server::step_once() {
  nvtxRangePushA("jacobi_server_step");
  struct PopOnExit {
    ~PopOnExit() { nvtxRangePop(); }
  } pop_on_exit;
  maybe_evict();
  // admission: first fit, in arrival order, within the arena
  std::vector<Request> admit;
  const bool fresh = !ws[0] && !ws[1];  // the arena holds no workset state yet
  {
    std::lock_guard<std::mutex> lk(mu);
    int free_slots[2] = {max_slots - (int)active[0].size(), max_slots - (int)active[1].size()};
    int64_t room = (int64_t)arena.size() - (int64_t)arena.in_use();
    for (auto it = queue.begin(); it != queue.end();) {
      const int d = it->spec.ndim - 2;
      // a workset not yet created also needs its tables; keep 1/16 of the request as margin
      const int64_t need = it->bytes + it->bytes / 16 + (ws[d] ? 0 : (int64_t)(1 << 20));
      if (free_slots[d] > 0 && need <= room) {
        room -= need;
        --free_slots[d];
        admit.push_back(std::move(*it));
        it = queue.erase(it);
      } else {
        ++it;
      }
    }
  }
  for (size_t ai = 0; ai < admit.size(); ++ai) {
    Request& r = admit[ai];
    const int d = r.spec.ndim - 2;
    try {
      Workset* w = workset(r.spec.ndim);
      // source and initial field go in through the page-locked stage; the
      // request keeps its own copies in case it has to wait and retry
      ProblemSpec spec = r.spec;
      const size_t npts = (size_t)(spec.n[0] * spec.n[1] * spec.n[2]);
      const size_t x0_at = spec.source ? (npts + 1) & ~(size_t)1 : 0;  // 16-byte aligned
      double* st = stage.get(x0_at + npts);
      if (spec.source) {
        memcpy(st, spec.source, npts * sizeof(double));
        spec.source = st;
      }
      if (spec.x0) {
        memcpy(st + x0_at, spec.x0, npts * sizeof(double));
        spec.x0 = st + x0_at;
      }
      const int slot = w->add_solve(spec);
      Active a;
      a.ticket = r.ticket;
      a.tol = r.tol;
      a.max_sweeps = r.max_sweeps;
      a.points = r.spec.n[0] * r.spec.n[1] * r.spec.n[2];
      a.t_submit = r.t_submit;
      a.sweeps = r.resume_sweeps;  // a resumed solve continues its count
      const bool resumed = r.evictions > 0;
      if (evict) {
        // keep the inputs on the host for a later resume (not the initial field)
        a.req = std::move(r);
        a.req.x0.clear();
        a.req.x0.shrink_to_fit();
        a.req.spec.x0 = nullptr;
      }
      active[d][slot] = std::move(a);
      std::lock_guard<std::mutex> lk(mu);
      stats.admitted += 1;
      if (resumed) stats.resumed += 1;
    } catch (const JErr& e) {
      if (e.code != JACOBI_ERR_OOM && e.code != JACOBI_ERR_BUSY) throw;
      // Out of arena (fragmentation, or workset tables larger than the margin).
      // While some solve is resident, this request and the ones after it go
      // back to the head of the queue, in order, and wait for a retirement.
      // With nothing resident no retirement will come: empty worksets are
      // freed and the request retried once from a clean arena; if it fails
      // there too it can never fit, and it completes with JACOBI_ERR_OOM.
      size_t from = ai;
      if (active[0].empty() && active[1].empty()) {
        if (!fresh) {
          delete ws[0];
          delete ws[1];
          ws[0] = ws[1] = nullptr;
        } else {
          Done dn;
          dn.res.status = JACOBI_ERR_OOM;
          dn.res.reserved = 0;
          dn.res.sweeps = 0;
          dn.res.rel = std::nan("");
          dn.res.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t_submit).count();
          std::lock_guard<std::mutex> lk(mu);
          stats.rejected += 1;
          done[r.ticket] = std::move(dn);
          from = ai + 1;
        }
      }
      std::lock_guard<std::mutex> lk(mu);
      for (size_t bi = admit.size(); bi-- > from;) queue.push_front(std::move(admit[bi]));
      break;
    }
  }
  bool worked = false;
  for (int d = 0; d < 2; ++d) {
    if (active[d].empty()) continue;
    Workset* w = ws[d];
    worked = true;
    const int64_t k = w->opt.refine_period;
    w->serve_step(k);
    std::vector<double> rss;
    w->read_rss(rss);
    const auto now = std::chrono::steady_clock::now();
    std::vector<int> finished;
    for (auto& kv : active[d]) {
      Active& a = kv.second;
      if (a.had_outer) a.sweeps += k;
      a.had_outer = true;
      a.steps_resident += 1;
      const SolveHost* s = w->solve(kv.first);
      const double rel = s->bss > 0.0 ? std::sqrt(rss[kv.first]) / std::sqrt(s->bss) : std::sqrt(rss[kv.first]);
      int st = -1;
      if (!std::isfinite(rel)) st = JACOBI_ERR_DIVERGED;
      else if (rel <= a.tol) st = JACOBI_OK;
      else if (a.sweeps >= a.max_sweeps) st = JACOBI_ERR_NOT_CONVERGED;
      if (st < 0) continue;
      Done dn;
      dn.res.status = st;
      dn.res.reserved = 0;
      dn.res.sweeps = a.sweeps;
      dn.res.rel = rel;
      dn.res.seconds = std::chrono::duration<double>(now - a.t_submit).count();
      dn.field.resize((size_t)a.points);
      double* staged = stage.get((size_t)a.points);  // sized at admission: no allocation
      w->gather(kv.first, staged, 0);
      memcpy(dn.field.data(), staged, (size_t)a.points * sizeof(double));
      {
        std::lock_guard<std::mutex> lk(mu);
        stats.completed += 1;
        stats.lups += (double)a.points * (double)a.sweeps;
        done[a.ticket] = std::move(dn);
      }
      finished.push_back(kv.first);
    }
    for (int slot : finished) {
      w->remove_solve(slot);
      active[d].erase(slot);
    }
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    stats.active = (int64_t)(active[0].size() + active[1].size());
    stats.queued = (int64_t)queue.size();
    stats.bytes_in_use = (int64_t)arena.in_use();
    if (worked) stats.steps += 1;
  }
  cv.notify_all();
  return worked || !admit.empty();
}

void jacobi_server::loop() {
  cudaSetDevice(device);
  try {
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop) break;
      }
      const bool worked = step_once();
      if (!worked) {
        std::unique_lock<std::mutex> lk(mu);
        if (stop) break;
        cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return stop || !queue.empty(); });
      }
    }
  } catch (const JErr& e) {
    std::lock_guard<std::mutex> lk(mu);
    fatal = e.msg;
  } catch (...) {
    std::lock_guard<std::mutex> lk(mu);
    fatal = "unexpected internal error in the driver thread";
  }
  cv.notify_all();
}

// Workset::serve_step lives here to keep the serving logic in one file.
namespace jgb {
void Workset::serve_step(int64_t k) {
  if (live() == 0) return;
  step_refine(k);
}
}  // namespace jgb

#define SRV_BEGIN try {
#define SRV_END(srv)                                   \
  }                                                    \
  catch (const JErr& e) {                              \
    if (srv) (srv)->err = e.msg;                       \
    set_thread_error(e.msg);                           \
    return (jacobi_status)e.code;                      \
  }                                                    \
  catch (const std::bad_alloc&) {                      \
    set_thread_error("host allocation failed");        \
    return JACOBI_ERR_OOM;                             \
  }                                                    \
  catch (...) {                                        \
    set_thread_error("unexpected internal error");     \
    return JACOBI_ERR_INVALID;                         \
  }

extern "C" {

jacobi_status jacobi_server_create(jacobi_server_t* out, int dtype, int64_t hbm_budget_bytes, int max_slots,
                                   void* cuda_stream) {
  jacobi_server* srv = nullptr;
  SRV_BEGIN
  if (!out) throw JErr{JACOBI_ERR_INVALID, "out is NULL"};
  *out = nullptr;
  if (dtype < 1 || dtype > 3) throw JErr{JACOBI_ERR_INVALID, "the server runs the refinement dtypes (1..3)"};
  if (hbm_budget_bytes < (1 << 20)) throw JErr{JACOBI_ERR_INVALID, "hbm_budget_bytes must be >= 1 MiB"};
  if (max_slots < 1 || max_slots > 4096) throw JErr{JACOBI_ERR_INVALID, "max_slots must be in [1, 4096]"};
  srv = new jacobi_server();
  srv->dtype = dtype;
  srv->max_slots = max_slots;
  srv->stream = (cudaStream_t)cuda_stream;
  // one launch per sweep, each refinement step replayed from a CUDA graph:
  // on a stream of small solves this steps faster than the persistent
  // scheduler (whose per-block waits dominate small grids)
  srv->opt.schedule = 0;
  srv->opt.graph = 1;
  memset(&srv->stats, 0, sizeof(srv->stats));
  cudaGetDevice(&srv->device);
  if (!srv->arena.init((size_t)hbm_budget_bytes, current_alloc_hooks(), srv->stream)) {
    delete srv;
    srv = nullptr;
    throw JErr{JACOBI_ERR_OOM, "could not allocate the HBM budget"};
  }
  srv->driver = std::thread([srv] { srv->loop(); });
  *out = srv;
  return JACOBI_OK;
  SRV_END(srv)
}

jacobi_status jacobi_server_set_option(jacobi_server_t srv, const char* key, int64_t value) {
  if (!srv || !key) return JACOBI_ERR_INVALID;
  SRV_BEGIN
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->started) throw JErr{JACOBI_ERR_BUSY, "options are fixed once the first request is submitted"};
  const std::string k(key);
  if (k == "refine_period") {
    if (value < 1 || value > 4096) throw JErr{JACOBI_ERR_INVALID, "refine_period must be in [1, 4096]"};
    srv->opt.refine_period = value;
  } else if (k == "schedule" || k == "graph" || k == "halo") {
    if (value != 0 && value != 1) throw JErr{JACOBI_ERR_INVALID, k + " must be 0 or 1"};
    (k == "schedule" ? srv->opt.schedule : k == "graph" ? srv->opt.graph : srv->opt.halo) = value;
  } else if (k == "evict") {
    if (value != 0 && value != 1) throw JErr{JACOBI_ERR_INVALID, "evict must be 0 or 1"};
    srv->evict = value != 0;
  } else if (k == "evict_min_steps" || k == "evict_wait_steps" || k == "max_evictions") {
    if (value < (k == "evict_wait_steps" ? 0 : 1) || value > (1LL << 40))
      throw JErr{JACOBI_ERR_INVALID, k + " out of range"};
    (k == "evict_min_steps" ? srv->evict_min_steps : k == "evict_wait_steps" ? srv->evict_wait_steps
                                                                              : srv->max_evictions) = value;
  } else if (k == "rows_low" || k == "rows_f64") {
    if (value < (k == "rows_low" ? 0 : 1))
      throw JErr{JACOBI_ERR_INVALID, k == "rows_low" ? "rows_low must be >= 0 (0: automatic)" : "rows_f64 must be >= 1"};
    (k == "rows_low" ? srv->opt.rows_low : srv->opt.rows_f64) = value;
  } else {
    throw JErr{JACOBI_ERR_INVALID, "unknown server option " + k};
  }
  return JACOBI_OK;
  SRV_END(srv)
}

jacobi_status jacobi_server_submit(jacobi_server_t srv, const jacobi_problem* p, double tol, int64_t max_sweeps,
                                   uint64_t* ticket) {
  if (!srv || !p || !ticket) return JACOBI_ERR_INVALID;
  SRV_BEGIN
  if (!(tol > 0.0)) throw JErr{JACOBI_ERR_INVALID, "tol must be > 0"};
  if (max_sweeps < 0) throw JErr{JACOBI_ERR_INVALID, "max_sweeps must be >= 0"};
  if (p->ndim != 2 && p->ndim != 3) throw JErr{JACOBI_ERR_INVALID, "ndim must be 2 or 3"};
  Request r;
  ProblemSpec& s = r.spec;
  s.ndim = p->ndim;
  int64_t pts = 1;
  for (int a = 0; a < 3; ++a) {
    s.n[a] = a < p->ndim ? p->dims[a] : 1;
    s.blk[a] = a < p->ndim ? p->block[a] : 1;
    if (s.n[a] < 1 || s.blk[a] < 1 || s.blk[a] > s.n[a] || s.n[a] >= (1LL << 30))
      throw JErr{JACOBI_ERR_INVALID, "bad dims/block"};
    pts *= s.n[a];
  }
  s.bc_kind = p->bc.kind;
  s.bc_value = p->bc.value;
  if (s.bc_kind < 0 || s.bc_kind > 2) throw JErr{JACOBI_ERR_INVALID, "unknown boundary kind"};
  // copy the inputs: the caller keeps ownership of its arrays
  const int64_t fc[6] = {s.n[1] * s.n[2], s.n[1] * s.n[2], s.n[0] * s.n[2],
                         s.n[0] * s.n[2], s.n[0] * s.n[1], s.n[0] * s.n[1]};
  if (s.bc_kind == 2)
    for (int q = 0; q < 2 * p->ndim; ++q)
      if (p->bc.faces[q]) {
        r.faces[q].assign(p->bc.faces[q], p->bc.faces[q] + fc[q]);
        s.faces[q] = r.faces[q].data();
      }
  if (p->source) {
    r.source.assign(p->source, p->source + pts);
    s.source = r.source.data();
  }
  if (p->x0) {
    r.x0.assign(p->x0, p->x0 + pts);
    s.x0 = r.x0.data();
  }
  r.tol = tol;
  r.max_sweeps = max_sweeps;
  r.bytes = solve_device_bytes(s, srv->dtype, srv->dtype == 3);
  r.t_submit = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(srv->mu);
  if (!srv->fatal.empty()) throw JErr{JACOBI_ERR_CUDA, "server stopped: " + srv->fatal};
  if (r.bytes + r.bytes / 16 + (1 << 20) > (int64_t)srv->arena.size()) {
    srv->stats.rejected += 1;
    throw JErr{JACOBI_ERR_BUSY, "the request needs " + std::to_string(r.bytes) +
                                    " bytes of device memory, more than the whole budget"};
  }
  r.ticket = srv->next_ticket++;
  *ticket = r.ticket;
  srv->stats.submitted += 1;
  srv->started = true;
  srv->queue.push_back(std::move(r));
  srv->cv.notify_all();
  return JACOBI_OK;
  SRV_END(srv)
}

jacobi_status jacobi_server_poll(jacobi_server_t srv, uint64_t ticket, jacobi_result* out, double* field_out) {
  if (!srv) return JACOBI_ERR_INVALID;
  SRV_BEGIN
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->done.find(ticket);
  if (it == srv->done.end()) {
    if (!srv->fatal.empty()) throw JErr{JACOBI_ERR_CUDA, "server stopped: " + srv->fatal};
    if (ticket == 0 || ticket >= srv->next_ticket) throw JErr{JACOBI_ERR_INVALID, "unknown ticket"};
    return JACOBI_ERR_BUSY;
  }
  if (out) *out = it->second.res;
  if (field_out) memcpy(field_out, it->second.field.data(), it->second.field.size() * sizeof(double));
  srv->done.erase(it);
  return JACOBI_OK;
  SRV_END(srv)
}

jacobi_status jacobi_server_wait(jacobi_server_t srv, uint64_t ticket, double timeout_s) {
  if (!srv) return JACOBI_ERR_INVALID;
  std::unique_lock<std::mutex> lk(srv->mu);
  const bool ok = srv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return srv->done.count(ticket) > 0 || !srv->fatal.empty();
  });
  if (!srv->fatal.empty()) return JACOBI_ERR_CUDA;
  return ok ? JACOBI_OK : JACOBI_ERR_BUSY;
}

jacobi_status jacobi_server_get_stats(jacobi_server_t srv, jacobi_server_stats* out) {
  if (!srv || !out) return JACOBI_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  *out = srv->stats;
  out->budget_bytes = (int64_t)srv->arena.size();
  return srv->fatal.empty() ? JACOBI_OK : JACOBI_ERR_CUDA;
}

void jacobi_server_destroy(jacobi_server_t srv) { delete srv; }

}  // extern "C"
