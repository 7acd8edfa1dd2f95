// Host engine of the GB300 Jacobi library: block layout, work tables, launch
// sequences.  See engine.h.
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace jgb {

// ---------------------------------------------------------------------------
// allocation

static std::mutex g_hooks_mu;
static AllocHooks g_hooks;

AllocHooks current_alloc_hooks() {
  std::lock_guard<std::mutex> lk(g_hooks_mu);
  return g_hooks;
}

void set_alloc_hooks(const AllocHooks& h) {
  std::lock_guard<std::mutex> lk(g_hooks_mu);
  g_hooks = h;
}

static void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw JErr{3, std::string(what) + ": " + cudaGetErrorString(e)};
}

static void launch_check(int e, const char* what) {
  if (e != 0) throw JErr{3, std::string(what) + ": " + cudaGetErrorString((cudaError_t)e)};
}

#define LAUNCH(call, what)      \
  do {                          \
    launch_check((call), what); \
    ++launches_;                \
  } while (0)

DevPool::~DevPool() {
  cudaStreamSynchronize(stream_);
  for (auto& r : recs_) {
    if (hooks_.free) hooks_.free(r.p, (void*)stream_, hooks_.user);
    else cudaFree(r.p);
  }
}

void* DevPool::alloc(size_t bytes) {
  if (bytes == 0) return nullptr;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (hooks_.alloc) {
    p = hooks_.alloc(bytes, (void*)stream_, hooks_.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) throw JErr{2, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  recs_.push_back({p, bytes});
  bytes_ += (int64_t)bytes;
  cuda_check(cudaMemsetAsync(p, 0, bytes, stream_), "cudaMemsetAsync");
  return p;
}

void DevPool::release(void* p) {
  if (!p) return;
  for (size_t i = 0; i < recs_.size(); ++i) {
    if (recs_[i].p == p) {
      if (hooks_.free) hooks_.free(p, (void*)stream_, hooks_.user);
      else cudaFree(p);
      bytes_ -= (int64_t)recs_[i].n;
      recs_.erase(recs_.begin() + i);
      return;
    }
  }
}

// ---------------------------------------------------------------------------
// workset

static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

Workset::Workset(int ndim, int dtype, cudaStream_t stream, int capacity)
    : ndim_(ndim), dtype_(dtype), capacity_(capacity), stream_(stream), pool_(current_alloc_hooks(), stream) {
  solves_.assign(capacity, nullptr);
  d_solves_ = (SolveDev*)pool_.alloc(sizeof(SolveDev) * capacity);
  d_rss_ = (double*)pool_.alloc(sizeof(double) * capacity);
  d_ticket_ = (uint32_t*)pool_.alloc(sizeof(uint32_t) * capacity);
  cuda_check(cudaMallocHost((void**)&h_rss_, sizeof(double) * capacity), "cudaMallocHost");
}

Workset::~Workset() {
  cudaStreamSynchronize(stream_);
  for (auto* s : solves_) delete s;
  for (int k = 0; k < kProfCount; ++k)
    for (auto& p : ev_pending_[k]) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
  for (auto e : ev_free_) cudaEventDestroy(e);
  if (ev_open_) cudaEventDestroy(ev_open_);
  if (h_rss_) cudaFreeHost(h_rss_);
}

void Workset::layout_solve(SolveHost& s) {
  const ProblemSpec& p = s.spec;
  const int nd = p.ndim;
  for (int a = 0; a < 3; ++a) s.nb[a] = a < nd ? (int)((p.n[a] + p.blk[a] - 1) / p.blk[a]) : 1;
  const int gz = nd == 3 ? 1 : 0;
  int64_t cursor = 0, fcursor = 0;
  // residual partial layout: segments of every block column, row by row
  std::vector<int64_t> seg_base(s.nb[0] + 1, 0);
  for (int i = 0; i < s.nb[0]; ++i) {
    const int64_t bx = i < s.nb[0] - 1 ? p.blk[0] : p.n[0] - (int64_t)(s.nb[0] - 1) * p.blk[0];
    seg_base[i + 1] = seg_base[i] + (bx + kResSeg - 1) / kResSeg;
  }
  s.part_row = (int)seg_base[s.nb[0]];
  s.nparts = (int64_t)s.part_row * p.n[1] * p.n[2];
  s.nchunks = (int)((s.nparts + kRedChunk - 1) / kRedChunk);
  s.blocks.clear();
  auto idx = [&](int i, int j, int k) { return (k * s.nb[1] + j) * s.nb[0] + i; };
  for (int k = 0; k < s.nb[2]; ++k)
    for (int j = 0; j < s.nb[1]; ++j)
      for (int i = 0; i < s.nb[0]; ++i) {
        BlockDev B;
        memset(&B, 0, sizeof(B));
        auto ext = [&](int a, int t) {
          return (int32_t)(t < s.nb[a] - 1 ? p.blk[a] : p.n[a] - (int64_t)(s.nb[a] - 1) * p.blk[a]);
        };
        B.bx = ext(0, i);
        B.by = ext(1, j);
        B.bz = nd == 3 ? ext(2, k) : 1;
        B.ox = (int32_t)(i * p.blk[0]);
        B.oy = (int32_t)(j * p.blk[1]);
        B.oz = nd == 3 ? (int32_t)(k * p.blk[2]) : 0;
        B.gz = gz;
        B.pitch = (int32_t)round_up(B.bx, 16);
        B.plane = (B.by + 2) * B.pitch;
        B.off = round_up(cursor, 32);
        cursor = B.off + (int64_t)(B.bz + 2 * gz) * B.plane;
        B.xoff = round_up(cursor, 32);
        cursor = B.xoff + 2 * (int64_t)B.by * B.bz;
        B.nbr[0] = i > 0 ? idx(i - 1, j, k) : -1;
        B.nbr[1] = i < s.nb[0] - 1 ? idx(i + 1, j, k) : -1;
        B.nbr[2] = j > 0 ? idx(i, j - 1, k) : -1;
        B.nbr[3] = j < s.nb[1] - 1 ? idx(i, j + 1, k) : -1;
        B.nbr[4] = nd == 3 && k > 0 ? idx(i, j, k - 1) : -1;
        B.nbr[5] = nd == 3 && k < s.nb[2] - 1 ? idx(i, j, k + 1) : -1;
        B.fsz[0] = B.fsz[1] = B.by * B.bz;
        B.fsz[2] = B.fsz[3] = B.bx * B.bz;
        B.fsz[4] = B.fsz[5] = nd == 3 ? B.bx * B.by : 0;
        B.foff = round_up(fcursor, 32);
        int64_t fs = 0;
        for (int q = 0; q < 6; ++q) fs += B.fsz[q];
        fcursor = B.foff + fs;
        B.part = seg_base[i];
        s.blocks.push_back(B);
      }
  s.elems = round_up(cursor, 32);
  s.face_elems = round_up(std::max<int64_t>(fcursor, 1), 32);
}

void Workset::alloc_solve(SolveHost& s) {
  auto a = [&](size_t bytes) {
    void* p = pool_.alloc(bytes);
    s.allocs.push_back(p);
    return p;
  };
  const size_t E = (size_t)s.elems;
  s.x[0] = (double*)a(E * 8);
  s.x[1] = (double*)a(E * 8);
  s.f = (double*)a(E * 8);
  if (refine()) {
    const size_t le = dtype_ == 2 ? 2 : 4;
    const size_t re = (dtype_ == 2 && opt.r_bf16) ? 2 : 4;
    s.e[0] = a(E * le);
    s.e[1] = a(E * le);
    s.r = a(E * re);
    s.sendlo = a((size_t)s.face_elems * le);
  }
  s.send64 = (double*)a((size_t)s.face_elems * 8);
  s.part = (double*)a((size_t)s.nparts * 8);
  s.lvl1 = (double*)a((size_t)std::max(1, s.nchunks) * 8);
}

void Workset::push_solve_dev(SolveHost& s) {
  SolveDev d;
  memset(&d, 0, sizeof(d));
  d.x[0] = s.x[0];
  d.x[1] = s.x[1];
  d.f = s.f;
  d.e[0] = s.e[0];
  d.e[1] = s.e[1];
  d.r = s.r;
  d.send64 = s.send64;
  d.sendlo = s.sendlo;
  d.part = s.part;
  d.lvl1 = s.lvl1;
  d.rss = d_rss_ + s.slot;
  d.ticket = d_ticket_ + s.slot;
  d.nparts = s.nparts;
  d.part_row = s.part_row;
  d.ny = (int32_t)s.spec.n[1];
  d.ndim = s.spec.ndim;
  d.phase = s.phase;
  d.active = s.active;
  d.apply_e = s.apply_e;
  d.low = low();
  d.r_bf16 = (dtype_ == 2 && opt.r_bf16) ? 1 : 0;
  cuda_check(cudaMemcpyAsync(d_solves_ + s.slot, &d, sizeof(d), cudaMemcpyHostToDevice, stream_), "upload solve");
  cuda_check(cudaStreamSynchronize(stream_), "sync");
}

void Workset::set_active(int slot, int active) {
  SolveHost* s = solve(slot);
  if (!s || s->active == active) return;
  s->active = active;
  const int32_t v = active;
  cuda_check(cudaMemcpyAsync((char*)(d_solves_ + slot) + offsetof(SolveDev, active), &v, sizeof(v),
                             cudaMemcpyHostToDevice, stream_),
             "set active");
  cuda_check(cudaStreamSynchronize(stream_), "sync");
}

void Workset::rebuild_tables() {
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  for (void* p : table_allocs_) pool_.release(p);
  table_allocs_.clear();
  std::vector<BlockDev> blocks;
  std::vector<WorkItem> w64, wlo;
  std::vector<FaceItem> faces;
  std::vector<RedItem> red;
  std::vector<RowItem> rows;
  block_base_.assign(capacity_, 0);
  face_base_.assign(capacity_, 0);
  face_cnt_.assign(capacity_, 0);
  row_base_.assign(capacity_, 0);
  row_cnt_.assign(capacity_, 0);
  const int r64 = (int)std::min<int64_t>(std::max<int64_t>(opt.rows_f64, 1), 32767);
  const int rlo = (int)std::min<int64_t>(std::max<int64_t>(opt.rows_low, 1), 32767);
  for (int slot = 0; slot < capacity_; ++slot) {
    SolveHost* s = solves_[slot];
    if (!s) continue;
    const int base = (int)blocks.size();
    block_base_[slot] = base;
    face_base_[slot] = (int)faces.size();
    row_base_[slot] = (int)rows.size();
    for (size_t b = 0; b < s->blocks.size(); ++b) {
      BlockDev B = s->blocks[b];
      B.solve = slot;
      for (int q = 0; q < 6; ++q)
        if (B.nbr[q] >= 0) B.nbr[q] += base;
      blocks.push_back(B);
      const int bi = base + (int)b;
      const int ext = ndim_ == 2 ? B.by : B.bz;
      auto items = [&](std::vector<WorkItem>& out, int seg_w, int R) {
        const int segs = (B.bx + seg_w - 1) / seg_w;
        for (int m0 = 0; m0 < ext; m0 += R) {
          const int n = std::min(R, ext - m0);
          for (int sg = 0; sg < segs; ++sg) {
            if (ndim_ == 2) {
              out.push_back(WorkItem{bi, (int16_t)sg, (int16_t)n, m0, 0});
            } else {
              for (int y = 0; y < B.by; ++y) out.push_back(WorkItem{bi, (int16_t)sg, (int16_t)n, y, m0});
            }
          }
        }
      };
      items(w64, kSegF64, r64);
      if (refine()) items(wlo, kSegLow, rlo);
      for (int q = 0; q < 2 * ndim_; ++q) faces.push_back(FaceItem{bi, q});
      for (int z = 0; z < B.bz; ++z)
        for (int y = 0; y < B.by; ++y) rows.push_back(RowItem{bi, y, z, 0});
    }
    face_cnt_[slot] = (int)faces.size() - face_base_[slot];
    row_cnt_[slot] = (int)rows.size() - row_base_[slot];
    for (int c = 0; c < s->nchunks; ++c) {
      const int64_t start = (int64_t)c * kRedChunk;
      red.push_back(RedItem{slot, c, s->nchunks, (int)std::min<int64_t>(kRedChunk, s->nparts - start), start});
    }
  }
  auto up = [&](const void* src, size_t bytes) -> void* {
    if (bytes == 0) return nullptr;
    void* p = pool_.alloc(bytes);
    table_allocs_.push_back(p);
    cuda_check(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, stream_), "upload table");
    return p;
  };
  d_blocks_ = (BlockDev*)up(blocks.data(), blocks.size() * sizeof(BlockDev));
  d_w64_ = (WorkItem*)up(w64.data(), w64.size() * sizeof(WorkItem));
  d_wlo_ = (WorkItem*)up(wlo.data(), wlo.size() * sizeof(WorkItem));
  d_faces_ = (FaceItem*)up(faces.data(), faces.size() * sizeof(FaceItem));
  d_red_ = (RedItem*)up(red.data(), red.size() * sizeof(RedItem));
  d_rows_ = (RowItem*)up(rows.data(), rows.size() * sizeof(RowItem));
  n64_ = (int)w64.size();
  nlo_ = (int)wlo.size();
  nfaces_ = (int)faces.size();
  nred_ = (int)red.size();
  nrows_ = (int)rows.size();
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  tables_dirty_ = false;
}

Tables Workset::tables() const {
  Tables t;
  t.w64 = d_w64_;
  t.n64 = n64_;
  t.wlo = d_wlo_;
  t.nlo = nlo_;
  t.faces = d_faces_;
  t.nfaces = nfaces_;
  t.red = d_red_;
  t.nred = nred_;
  t.rows = d_rows_;
  t.nrows = nrows_;
  t.blocks = d_blocks_;
  t.solves = d_solves_;
  t.ndim = ndim_;
  return t;
}

// Tables restricted to the rows / faces of one solve (copies, ghost fill).
Tables Workset::solve_tables(const SolveHost& s) const {
  Tables t = tables();
  t.rows = d_rows_ + row_base_[s.slot];
  t.nrows = row_cnt_[s.slot];
  t.faces = d_faces_ + face_base_[s.slot];
  t.nfaces = face_cnt_[s.slot];
  return t;
}

void Workset::scatter(int slot, const double* dense, int which, int on_device) {
  SolveHost* s = solve(slot);
  const int64_t npts = s->points();
  const double* src = dense;
  void* tmp = nullptr;
  if (!on_device) {
    tmp = pool_.alloc((size_t)npts * 8);
    cuda_check(cudaMemcpyAsync(tmp, dense, (size_t)npts * 8, cudaMemcpyHostToDevice, stream_), "H2D field");
    src = (const double*)tmp;
  }
  LAUNCH(launch_scatter(solve_tables(*s), src, which, 0, s->spec.n[0], s->spec.n[1], stream_), "scatter");
  if (tmp) {
    cuda_check(cudaStreamSynchronize(stream_), "sync");
    pool_.release(tmp);
  }
}

void Workset::gather(int slot, double* dense, int on_device) {
  SolveHost* s = solve(slot);
  const int64_t npts = s->points();
  double* dst = dense;
  void* tmp = nullptr;
  if (!on_device) {
    tmp = pool_.alloc((size_t)npts * 8);
    dst = (double*)tmp;
  }
  LAUNCH(launch_gather(solve_tables(*s), dst, 0, s->spec.n[0], s->spec.n[1], stream_), "gather");
  if (tmp) {
    cuda_check(cudaMemcpyAsync(dense, tmp, (size_t)npts * 8, cudaMemcpyDeviceToHost, stream_), "D2H field");
    cuda_check(cudaStreamSynchronize(stream_), "sync");
    pool_.release(tmp);
  }
}

// Standalone exchange of the FP64 iterate x[(phase + kpar) & 1] for every
// active solve: pack every interior face, then unpack into the neighbours.
void Workset::halo_exchange_x(int kpar) {
  const Tables t = tables();
  LAUNCH(launch_halo_pack(t, 0, kpar, low(), stream_), "halo pack");
  LAUNCH(launch_halo_unpack(t, 0, kpar, low(), stream_), "halo unpack");
}

void Workset::upload_inputs(SolveHost& s) {
  const ProblemSpec& p = s.spec;
  // source term
  if (p.source) scatter(s.slot, p.source, 1, p.inputs_on_device);
  // Dirichlet ghosts into both parities
  const int nfaces = 2 * p.ndim;
  int64_t fcount[6];
  fcount[0] = fcount[1] = p.n[1] * p.n[2];
  fcount[2] = fcount[3] = p.n[0] * p.n[2];
  fcount[4] = fcount[5] = p.n[0] * p.n[1];
  const double* dfaces[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<void*> tmps;
  if (p.bc_kind != 0) {
    for (int q = 0; q < nfaces; ++q) {
      std::vector<double> host;
      const double* src = nullptr;
      if (p.bc_kind == 1) {
        host.assign((size_t)fcount[q], p.bc_value);
        src = host.data();
      } else {
        src = p.faces[q];
      }
      if (!src) continue;
      void* d = pool_.alloc((size_t)fcount[q] * 8);
      tmps.push_back(d);
      cuda_check(cudaMemcpyAsync(d, src, (size_t)fcount[q] * 8,
                                 p.inputs_on_device && p.bc_kind == 2 ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyHostToDevice,
                                 stream_),
                 "H2D face");
      cuda_check(cudaStreamSynchronize(stream_), "sync");
      dfaces[q] = (const double*)d;
    }
  }
  const Tables st = solve_tables(s);
  for (int par = 0; par < 2; ++par)
    LAUNCH(launch_ghost_fill(st, dfaces, par, p.n[0], p.n[1], p.n[2], stream_), "ghost fill");
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  for (void* d : tmps) pool_.release(d);
  // ||b||^2 = residual of the zero field (interiors are still zero)
  {
    // only this solve is active during set-up work
    std::vector<int> was(capacity_, 0);
    for (int k = 0; k < capacity_; ++k)
      if (solves_[k] && k != s.slot) {
        was[k] = solves_[k]->active;
        set_active(k, 0);
      }
    residual_only();
    std::vector<double> rss;
    read_rss(rss);
    s.bss = rss[s.slot];
    // initial iterate
    if (p.x0) {
      scatter(s.slot, p.x0, 0, p.inputs_on_device);
      halo_exchange_x(0);
    }
    cuda_check(cudaStreamSynchronize(stream_), "sync");
    for (int k = 0; k < capacity_; ++k)
      if (solves_[k] && k != s.slot) set_active(k, was[k]);
  }
}

int Workset::add_solve(const ProblemSpec& p) {
  int slot = -1;
  for (int k = 0; k < capacity_; ++k)
    if (!solves_[k]) {
      slot = k;
      break;
    }
  if (slot < 0) throw JErr{7, "workset is full"};
  SolveHost* s = new SolveHost();
  s->spec = p;
  s->slot = slot;
  try {
    layout_solve(*s);
    alloc_solve(*s);
    solves_[slot] = s;
    push_solve_dev(*s);
    rebuild_tables();
    upload_inputs(*s);
  } catch (...) {
    solves_[slot] = nullptr;
    for (void* q : s->allocs) pool_.release(q);
    delete s;
    SolveDev z;
    memset(&z, 0, sizeof(z));
    cudaMemcpyAsync(d_solves_ + slot, &z, sizeof(z), cudaMemcpyHostToDevice, stream_);
    cudaStreamSynchronize(stream_);
    rebuild_tables();
    throw;
  }
  return slot;
}

void Workset::remove_solve(int slot) {
  SolveHost* s = solve(slot);
  if (!s) return;
  set_active(slot, 0);
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  for (void* q : s->allocs) pool_.release(q);
  delete s;
  solves_[slot] = nullptr;
  SolveDev z;
  memset(&z, 0, sizeof(z));
  cuda_check(cudaMemcpyAsync(d_solves_ + slot, &z, sizeof(z), cudaMemcpyHostToDevice, stream_), "clear solve");
  rebuild_tables();
}

void Workset::sync() { cuda_check(cudaStreamSynchronize(stream_), "cudaStreamSynchronize"); }

void Workset::reduce() {
  prof_begin(kProfReduce);
  LAUNCH(launch_reduce(tables(), stream_), "reduce");
  prof_end(kProfReduce);
}

void Workset::sweeps_f64(int64_t n, bool resid_last) {
  if (tables_dirty_) rebuild_tables();
  const Tables t = tables();
  const bool push = opt.halo == 0;
  for (int64_t k = 0; k < n; ++k) {
    const bool resid = resid_last && k == n - 1;
    const int kpar = (int)(k & 1);
    prof_begin(kProfSweepF64);
    LAUNCH(launch_sweep_f64(t, kpar, push, resid, true, stream_), "sweep f64");
    prof_end(kProfSweepF64);
    if (!push) {
      prof_begin(kProfHalo);
      halo_exchange_x(kpar ^ 1);
      prof_end(kProfHalo);
    }
  }
  if (resid_last && n > 0) reduce();
  if (n & 1) phase_advance(1, -1);
}

void Workset::phase_advance(int d, int set_apply_e) {
  LAUNCH(launch_phase_advance(d_solves_, capacity_, d, set_apply_e, stream_), "phase advance");
  for (auto* s : solves_)
    if (s && s->active) {
      s->phase = (s->phase + d) & 1;
      if (set_apply_e >= 0) s->apply_e = set_apply_e;
    }
}

void Workset::residual_only() {
  if (tables_dirty_) rebuild_tables();
  LAUNCH(launch_sweep_f64(tables(), 0, false, true, false, stream_), "residual");
  reduce();
}

void Workset::refine_outer() {
  if (tables_dirty_) rebuild_tables();
  const Tables t = tables();
  const bool push = opt.halo == 0;
  prof_begin(kProfOuter);
  LAUNCH(launch_refine_outer(t, epar_last_, push, low(), dtype_ == 2 && opt.r_bf16, stream_), "refine outer");
  prof_end(kProfOuter);
  if (!push) {
    prof_begin(kProfHalo);
    halo_exchange_x(1);
    prof_end(kProfHalo);
  }
  reduce();
  phase_advance(1, 1);
}

void Workset::refine_inner(int64_t k) {
  if (tables_dirty_) rebuild_tables();
  const Tables t = tables();
  const bool push = opt.halo == 0;
  const bool rb = dtype_ == 2 && opt.r_bf16;
  for (int64_t j = 0; j < k; ++j) {
    const int epar = (int)(j & 1);
    prof_begin(kProfSweepLow);
    LAUNCH(launch_sweep_low(t, epar, j == 0, push, low(), rb, stream_), "sweep low");
    prof_end(kProfSweepLow);
    if (!push) {
      prof_begin(kProfHalo);
      LAUNCH(launch_halo_pack(t, 1, epar, low(), stream_), "halo pack e");
      LAUNCH(launch_halo_unpack(t, 1, epar, low(), stream_), "halo unpack e");
      prof_end(kProfHalo);
    }
  }
  if (k > 0) epar_last_ = (int)((k - 1) & 1);
}

void Workset::read_rss(std::vector<double>& out) {
  cuda_check(cudaMemcpyAsync(h_rss_, d_rss_, sizeof(double) * capacity_, cudaMemcpyDeviceToHost, stream_), "D2H rss");
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  out.assign(h_rss_, h_rss_ + capacity_);
}

// ---------------------------------------------------------------------------
// profiling with CUDA events on the launching stream

void Workset::prof_begin(int kind) {
  (void)kind;
  if (!opt.profile) return;
  if (ev_free_.empty()) {
    cudaEvent_t e;
    cuda_check(cudaEventCreate(&e), "cudaEventCreate");
    ev_free_.push_back(e);
  }
  ev_open_ = ev_free_.back();
  ev_free_.pop_back();
  cuda_check(cudaEventRecord(ev_open_, stream_), "cudaEventRecord");
}

void Workset::prof_end(int kind) {
  if (!opt.profile || !ev_open_) return;
  if (ev_free_.empty()) {
    cudaEvent_t e;
    cuda_check(cudaEventCreate(&e), "cudaEventCreate");
    ev_free_.push_back(e);
  }
  cudaEvent_t b = ev_free_.back();
  ev_free_.pop_back();
  cuda_check(cudaEventRecord(b, stream_), "cudaEventRecord");
  ev_pending_[kind].push_back(EvPair{ev_open_, b});
  ev_open_ = nullptr;
}

void Workset::prof_collect(int kind, double* ms, int64_t* n, bool reset) {
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  for (int k = 0; k < kProfCount; ++k) {
    for (auto& p : ev_pending_[k]) {
      float v = 0.f;
      cuda_check(cudaEventElapsedTime(&v, p.a, p.b), "cudaEventElapsedTime");
      prof_ms_[k] += v;
      prof_n_[k] += 1;
      ev_free_.push_back(p.a);
      ev_free_.push_back(p.b);
    }
    ev_pending_[k].clear();
  }
  if (ms) *ms = prof_ms_[kind];
  if (n) *n = prof_n_[kind];
  if (reset) {
    prof_ms_[kind] = 0;
    prof_n_[kind] = 0;
  }
}

}  // namespace jgb
