// Host engine of the GB300 Jacobi library: block layout, work tables, launch
// sequences, solve loops, CUDA graphs and the autotuner.  See engine.h.
#include "engine.h"
#include "deal_runs.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>

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
// layout (section 4.4: the domain cut into blocks, each with a ghost ring)

static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// points per lane of the 2D FP64 march kernel for option "march" (1: two,
// 2: four, 3: four with the lines staged in shared memory; see
// launch_sweep_f64_march)
static int march_width(int64_t march) { return march == 3 ? 5 : march == 2 ? 4 : 2; }

static void layout(SolveHost& s) {
  const ProblemSpec& p = s.spec;
  const int nd = p.ndim;
  for (int a = 0; a < 3; ++a) s.nb[a] = a < nd ? (int)((p.n[a] + p.blk[a] - 1) / p.blk[a]) : 1;
  const int gz = nd == 3 ? 1 : 0;
  int64_t cursor = 0, fcursor = 0;
  // residual partials: segments of every block column, grid row by grid row
  std::vector<int64_t> seg_base(s.nb[0] + 1, 0);
  for (int i = 0; i < s.nb[0]; ++i) {
    const int64_t bx = i < s.nb[0] - 1 ? p.blk[0] : p.n[0] - (int64_t)(s.nb[0] - 1) * p.blk[0];
    seg_base[i + 1] = seg_base[i] + (bx + kResSeg - 1) / kResSeg;
  }
  s.part_row = (int)seg_base[s.nb[0]];
  // groups of kResGroup lines along the march axis (y in 2D, z in 3D),
  // counted block by block so that no group straddles two blocks
  const int ma = nd == 3 ? 2 : 1;
  std::vector<int64_t> grp_base(s.nb[ma] + 1, 0);
  for (int t = 0; t < s.nb[ma]; ++t) {
    const int64_t ext = t < s.nb[ma] - 1 ? p.blk[ma] : p.n[ma] - (int64_t)(s.nb[ma] - 1) * p.blk[ma];
    grp_base[t + 1] = grp_base[t] + (ext + kResGroup - 1) / kResGroup;
  }
  s.nparts = (int64_t)s.part_row * grp_base[s.nb[ma]] * (nd == 3 ? p.n[1] : 1);
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
        B.pg = (int32_t)grp_base[nd == 3 ? k : j];
        s.blocks.push_back(B);
      }
  s.elems = round_up(cursor, 32);
  s.face_elems = round_up(std::max<int64_t>(fcursor, 1), 32);
}

int64_t solve_device_bytes(const ProblemSpec& p, int dtype, bool r_bf16) {
  SolveHost s;
  s.spec = p;
  layout(s);
  const int64_t le = dtype >= 2 ? 2 : 4, re = (dtype == 3 || (dtype == 2 && r_bf16)) ? 2 : 4;
  int64_t b = s.elems * 24 + s.face_elems * 8 + s.nparts * 8 + std::max(1, s.nchunks) * 8;
  if (dtype != 0) b += s.elems * (2 * le + re) + s.face_elems * le;
  // work tables: about one 16-byte item per 32 points, plus block descriptors
  b += (s.points() / 32 + 1) * 16 * (dtype != 0 ? 2 : 1) + (int64_t)s.blocks.size() * 256;
  return b;
}

// ---------------------------------------------------------------------------
// workset

Workset::Workset(int ndim, int dtype, cudaStream_t stream, int capacity, bool r_bf16, const AllocHooks* hooks)
    : ndim_(ndim), dtype_(dtype), capacity_(capacity), r_bf16_(r_bf16 || dtype == 3), stream_(stream),
      cur_(stream), pool_(hooks ? *hooks : current_alloc_hooks(), stream) {
  solves_.assign(capacity, nullptr);
  // device arrays belong to pool_, which frees them if a later step throws
  d_solves_ = (SolveDev*)pool_.alloc(sizeof(SolveDev) * capacity);
  d_rss_ = (double*)pool_.alloc(sizeof(double) * capacity);
  d_ticket_ = (uint32_t*)pool_.alloc(sizeof(uint32_t) * capacity);
  d_ctl_ = (SchedCtl*)pool_.alloc(sizeof(SchedCtl));
  d_slotctl_ = (int32_t*)pool_.alloc(sizeof(int32_t) * capacity);
  try {
    cuda_check(cudaMallocHost((void**)&h_rss_, sizeof(double) * capacity), "cudaMallocHost");
    cuda_check(cudaMallocHost((void**)&h_ctl_, sizeof(SchedCtl)), "cudaMallocHost");
    cuda_check(cudaMallocHost((void**)&h_slotctl_, sizeof(int32_t) * capacity), "cudaMallocHost");
    cuda_check(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking), "cudaStreamCreate");
  } catch (...) {
    free_host_side();  // the destructor does not run for a throwing constructor
    throw;
  }
}

void Workset::free_host_side() {
  if (h_rss_) cudaFreeHost(h_rss_);
  if (h_ctl_) cudaFreeHost(h_ctl_);
  if (h_slotctl_) cudaFreeHost(h_slotctl_);
  if (cap_stream_) cudaStreamDestroy(cap_stream_);
  h_rss_ = nullptr;
  h_ctl_ = nullptr;
  h_slotctl_ = nullptr;
  cap_stream_ = nullptr;
}

Workset::~Workset() {
  cudaStreamSynchronize(stream_);
  drop_graphs();
  for (auto* s : solves_) delete s;
  for (int k = 0; k < kProfCount; ++k)
    for (auto& p : ev_pending_[k]) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
  for (auto e : ev_free_) cudaEventDestroy(e);
  if (ev_open_) cudaEventDestroy(ev_open_);
  free_host_side();
}

int Workset::live() const {
  int n = 0;
  for (auto* s : solves_) n += s != nullptr;
  return n;
}

void Workset::layout_solve(SolveHost& s) { layout(s); }

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
    const size_t le = dtype_ >= 2 ? 2 : 4;
    const size_t re = r_bf16_ ? 2 : 4;
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
  d.elems = s.elems;
  d.part_row = s.part_row;
  d.ny = (int32_t)s.spec.n[1];
  d.ndim = s.spec.ndim;
  d.phase = s.phase;
  d.active = s.active;
  d.apply_e = s.apply_e;
  d.low = low();
  d.r_bf16 = r_bf16_ ? 1 : 0;
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

// Per-slot control through one small kernel (see launch_solve_ctl); the
// host mirrors are updated here.
void Workset::apply_slot_ctl(const std::vector<int32_t>& ctl) {
  bool any = false;
  for (int i = 0; i < capacity_; ++i) {
    const int32_t c = i < (int)ctl.size() ? ctl[i] : 8;
    h_slotctl_[i] = c;
    if (c & 8) continue;
    any = true;
    SolveHost* s = solves_[i];
    if (!s) continue;
    if (c & 2) s->phase ^= 1;
    if (c & 4) s->apply_e = 0;
    s->active = c & 1;
  }
  if (!any) return;
  cuda_check(cudaMemcpyAsync(d_slotctl_, h_slotctl_, sizeof(int32_t) * capacity_, cudaMemcpyHostToDevice, stream_),
             "slot ctl");
  LAUNCH(launch_solve_ctl(d_solves_, d_slotctl_, capacity_, stream_), "solve ctl");
  cuda_check(cudaStreamSynchronize(stream_), "sync");
}

void Workset::drop_graphs() {
  for (auto& kv : graphs_)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  graphs_.clear();
}

void Workset::rebuild_tables() {
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  drop_graphs();
  for (void* p : table_allocs_) pool_.release(p);
  table_allocs_.clear();
  std::vector<BlockDev> blocks;
  std::vector<WorkItem> w64, wlo, wm, wmr, wtb;
  int estage = 0;
  std::vector<CtaTask> t64, tlo;
  std::vector<FaceItem> faces;
  std::vector<RedItem> red;
  std::vector<RowItem> rows;
  face_base_.assign(capacity_, 0);
  face_cnt_.assign(capacity_, 0);
  row_base_.assign(capacity_, 0);
  row_cnt_.assign(capacity_, 0);
  // FP64 items hold whole residual groups (a group is reduced by one warp)
  const int r64 = (int)std::min<int64_t>((std::max<int64_t>(opt.rows_f64, 1) + kResGroup - 1) / kResGroup * kResGroup,
                                         32760);
  // rows_low = 0: lines per low-precision item by form (measured at 8192^2 /
  // 512^3): 2D 16 (float) or 8 (bfloat16), 3D 32
  const int64_t rows_low_auto = ndim_ == 2 ? (low() == kLowBF16 ? 8 : 16) : 32;
  const int rlo = (int)std::min<int64_t>(std::max<int64_t>(opt.rows_low > 0 ? opt.rows_low : rows_low_auto, 1), 32767);
  // 2D FP64 march items: as many as the march kernel keeps resident (one
  // wave), each at least 8 and at most kMarchLines lines long, the lines of a
  // block split evenly
  int64_t mlines = 0;
  if (ndim_ == 2)
    for (auto* s : solves_)
      if (s)
        for (const BlockDev& B : s->blocks) mlines += B.by;
  int mlen = 8;
  if (mlines > 0 && opt.march != 3) {
    const int64_t target = std::max(march_f64_resident_warps(ndim_, opt.halo == 0, march_width(opt.march)), 1);
    auto count = [&](int len) {
      int64_t c = 0;
      for (auto* s : solves_)
        if (s)
          for (const BlockDev& B : s->blocks) c += (B.by + len - 1) / len;
      return c;
    };
    mlen = (int)std::min<int64_t>(std::max<int64_t>((mlines + target - 1) / target, 8), kMarchLines);
    while (mlen < kMarchLines && count(mlen) > target) ++mlen;
  }
  // option march 3: the blocks whose lines the march kernels deal out
  std::vector<std::pair<int, int>> mblk;  // (block index, lines)
  tabled_points_ = 0;
  for (int slot = 0; slot < capacity_; ++slot) {
    SolveHost* s = solves_[slot];
    if (!s) continue;
    const int base = (int)blocks.size();
    face_base_[slot] = (int)faces.size();
    row_base_[slot] = (int)rows.size();
    if (compact_ && !s->active) continue;  // retired inside solve_all: no work items
    tabled_points_ += s->points();
    for (size_t b = 0; b < s->blocks.size(); ++b) {
      BlockDev B = s->blocks[b];
      B.solve = slot;
      for (int q = 0; q < 6; ++q)
        if (B.nbr[q] >= 0) B.nbr[q] += base;
      const int bi = base + (int)b;
      const int ext = ndim_ == 2 ? B.by : B.bz;
      // warp items of this block, then its CTA tasks (groups of kWarps items)
      // seg_w: points per warp row; ystep (3D): block rows per warp item
      auto items = [&](std::vector<WorkItem>& out, std::vector<CtaTask>& tasks, int seg_w, int R, int ystep) {
        const int first = (int)out.size();
        const int segs = (B.bx + seg_w - 1) / seg_w;
        for (int m0 = 0; m0 < ext; m0 += R) {
          const int n = std::min(R, ext - m0);
          for (int sg = 0; sg < segs; ++sg) {
            if (ndim_ == 2) {
              out.push_back(WorkItem{bi, (int16_t)sg, (int16_t)n, m0, 0});
            } else {
              for (int y = 0; y < B.by; y += ystep) out.push_back(WorkItem{bi, (int16_t)sg, (int16_t)n, y, m0});
            }
          }
        }
        const int last = (int)out.size();
        int nt = 0;
        for (int w = first; w < last; w += kWarps, ++nt) tasks.push_back(CtaTask{bi, w, std::min(kWarps, last - w), 0});
        return nt;
      };
      B.nt64 = items(w64, t64, kSegF64, r64, 1);
      if (ndim_ == 2 && opt.march == 3) {
        mblk.emplace_back(bi, ext);  // dealt out in runs below
      } else if (ndim_ == 2) {
        const int pieces = (ext + mlen - 1) / mlen;
        for (int q = 0; q < pieces; ++q) {
          const int a = (int)((int64_t)ext * q / pieces), e = (int)((int64_t)ext * (q + 1) / pieces);
          wm.push_back(WorkItem{bi, 0, (int16_t)(e - a), a, 0});
        }
      }
      if (refine()) {  // tiles of the two-sweep inner kernel (option tb); in 3D a tile spans kTb3TileZ planes
        const int tw = ndim_ == 2 ? kTbTileW : kTb3TileW, th = ndim_ == 2 ? kTbTileH : kTb3TileH;
        const int tz = ndim_ == 2 ? 1 : kTb3TileZ;
        for (int z0 = 0; z0 < B.bz; z0 += tz)
          for (int y0 = 0; y0 < B.by; y0 += th)
            for (int xt = 0; xt * tw < B.bx; ++xt)
              wtb.push_back(WorkItem{bi, (int16_t)xt, (int16_t)std::min(th, B.by - y0), y0, ndim_ == 2 ? 0 : z0});
      }
      if (refine()) {
        // 3D rows narrower than a warp row share a warp (see low_item)
        const int v = low() == kLowBF16 ? kSegLow16 / 32 : kSegLow / 32;
        const int lg = ndim_ == 3 ? low_lanes_log2(B.bx, v) : 5;
        B.ntlo = items(wlo, tlo, v << lg, rlo, 32 >> lg);
        // staged 3D sweep: e elements per stage = (rows + 2) x points per row
        estage = std::max(estage, ((32 >> lg) + 2) * (v << lg));
      } else {
        B.ntlo = 0;
      }
      blocks.push_back(B);
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
  // option march 3: the lines of all blocks, in block order, dealt out in
  // equal runs, one per warp (deal_runs.h: as many warps as the kernel keeps
  // resident, but runs of at least 8 lines, and more warps only where a run
  // would exceed kMarchLines); a run crossing a block boundary becomes two
  // items.  `unit` lines per step: 1 for the plain sweep, kResGroup for the
  // fused-residual sweep and the outer step, whose items must hold whole
  // residual groups.
  std::vector<int> wms, wmrs;
  auto deal = [&](int64_t target, int unit, std::vector<WorkItem>& out, std::vector<int>& start) {
    std::vector<RunPiece> pieces;
    std::vector<int> st;
    deal_runs(mblk, target, unit, 8, kMarchLines, pieces, st);
    const int base = (int)out.size();
    for (const RunPiece& q : pieces) out.push_back(WorkItem{q.block, 0, (int16_t)q.n, q.y0, 0});
    for (int v : st) start.push_back(base + v);
  };
  if (!mblk.empty()) {
    deal(march_f64_resident_warps(ndim_, opt.halo == 0, march_width(3)), 1, wm, wms);
    deal(march_f64r_resident_warps(ndim_, opt.halo == 0), kResGroup, wmr, wmrs);
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
  d_wm_ = (WorkItem*)up(wm.data(), wm.size() * sizeof(WorkItem));
  d_wmr_ = (WorkItem*)up(wmr.data(), wmr.size() * sizeof(WorkItem));
  d_wms_ = (int*)up(wms.data(), wms.size() * sizeof(int));
  d_wmrs_ = (int*)up(wmrs.data(), wmrs.size() * sizeof(int));
  d_wtb_ = (WorkItem*)up(wtb.data(), wtb.size() * sizeof(WorkItem));
  d_t64_ = (CtaTask*)up(t64.data(), t64.size() * sizeof(CtaTask));
  d_tlo_ = (CtaTask*)up(tlo.data(), tlo.size() * sizeof(CtaTask));
  d_faces_ = (FaceItem*)up(faces.data(), faces.size() * sizeof(FaceItem));
  d_red_ = (RedItem*)up(red.data(), red.size() * sizeof(RedItem));
  d_rows_ = (RowItem*)up(rows.data(), rows.size() * sizeof(RowItem));
  d_done_ = nullptr;
  if (!blocks.empty()) {
    d_done_ = (uint32_t*)pool_.alloc(blocks.size() * sizeof(uint32_t));
    table_allocs_.push_back(d_done_);
  }
  n64_ = (int)w64.size();
  nm_ = (int)wm.size();
  nmr_ = (int)wmr.size();
  nmw_ = wms.empty() ? 0 : (int)wms.size() - 1;
  nmrw_ = wmrs.empty() ? 0 : (int)wmrs.size() - 1;
  ntb_ = (int)wtb.size();
  estage_ = estage;
  nlo_ = (int)wlo.size();
  nt64_ = (int)t64.size();
  ntlo_ = (int)tlo.size();
  nfaces_ = (int)faces.size();
  nred_ = (int)red.size();
  nrows_ = (int)rows.size();
  nblocks_ = (int)blocks.size();
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  tables_dirty_ = false;
}

Tables Workset::tables() const {
  Tables t;
  t.w64 = d_w64_;
  t.n64 = n64_;
  t.wm = d_wm_;
  t.nm = nm_;
  t.wmr = d_wmr_;
  t.nmr = nmr_;
  t.wms = d_wms_;
  t.nmw = nmw_;
  t.wmrs = d_wmrs_;
  t.nmrw = nmrw_;
  t.wtb = d_wtb_;
  t.ntb = ntb_;
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
  t.t64 = d_t64_;
  t.nt64 = nt64_;
  t.tlo = d_tlo_;
  t.ntlo = ntlo_;
  t.done = d_done_;
  t.ctl = d_ctl_;
  t.spin_limit = (uint32_t)std::min<int64_t>(std::max<int64_t>(opt.spin_limit, 0), 0x7fffffff);
  t.poison = opt.poison_wait ? 1 : 0;
  t.l2pf = (int)std::min<int64_t>(std::max<int64_t>(opt.l2pf, 0), 64);
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

// Device address of a page-locked host buffer (pinned or registered), which
// kernels can read and write directly over the host link; nullptr for any
// other host memory, which then goes through a device staging buffer.
static const void* locked_host_device_ptr(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

void Workset::scatter(int slot, const double* dense, int which, int on_device) {
  if (tables_dirty_) rebuild_tables();
  SolveHost* s = solve(slot);
  const int64_t npts = s->points();
  const double* src = dense;
  void* tmp = nullptr;
  bool host_direct = false;
  if (!on_device) {
    if (const void* dp = locked_host_device_ptr(dense)) {
      src = (const double*)dp;
      host_direct = true;
    } else {
      tmp = pool_.alloc((size_t)npts * 8);
      cuda_check(cudaMemcpyAsync(tmp, dense, (size_t)npts * 8, cudaMemcpyHostToDevice, stream_), "H2D field");
      src = (const double*)tmp;
    }
  }
  LAUNCH(launch_scatter(solve_tables(*s), src, which, 0, s->spec.n[0], s->spec.n[1], stream_), "scatter");
  // a host buffer is the caller's again when the call returns
  if (tmp || host_direct) cuda_check(cudaStreamSynchronize(stream_), "sync");
  if (tmp) pool_.release(tmp);
}

void Workset::gather(int slot, double* dense, int on_device) {
  if (tables_dirty_) rebuild_tables();
  SolveHost* s = solve(slot);
  const int64_t npts = s->points();
  double* dst = dense;
  void* tmp = nullptr;
  bool host_direct = false;
  if (!on_device) {
    if (const void* dp = locked_host_device_ptr(dense)) {
      dst = (double*)dp;
      host_direct = true;
    } else {
      tmp = pool_.alloc((size_t)npts * 8);
      dst = (double*)tmp;
    }
  }
  LAUNCH(launch_gather(solve_tables(*s), dst, 0, s->spec.n[0], s->spec.n[1], stream_), "gather");
  if (tmp) cuda_check(cudaMemcpyAsync(dense, tmp, (size_t)npts * 8, cudaMemcpyDeviceToHost, stream_), "D2H field");
  if (tmp || host_direct) cuda_check(cudaStreamSynchronize(stream_), "sync");
  if (tmp) pool_.release(tmp);
}

// Standalone exchange of the FP64 iterate x[(phase + kpar) & 1] for every
// active solve: pack every interior face, then unpack into the neighbours.
void Workset::halo_exchange_x(int kpar) {
  const Tables t = tables();
  LAUNCH(launch_halo_pack(t, 0, kpar, low(), cur_), "halo pack");
  LAUNCH(launch_halo_unpack(t, 0, kpar, low(), cur_), "halo unpack");
}

void Workset::upload_inputs(SolveHost& s) {
  const ProblemSpec& p = s.spec;
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
  // ||b||^2 = residual of the zero field (interiors are still zero); every
  // other solve is masked off meanwhile
  std::vector<int32_t> ctl(capacity_, 8), back(capacity_, 8);
  for (int k = 0; k < capacity_; ++k)
    if (solves_[k] && k != s.slot && solves_[k]->active) {
      ctl[k] = 0;
      back[k] = 1;
    }
  apply_slot_ctl(ctl);
  residual_only();
  std::vector<double> rss;
  read_rss(rss);
  s.bss = rss[s.slot];
  if (p.x0) {
    scatter(s.slot, p.x0, 0, p.inputs_on_device);
    halo_exchange_x(0);
  }
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  apply_slot_ctl(back);
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
    tables_dirty_ = true;
    throw;
  }
  return slot;
}

void Workset::remove_solve(int slot) {
  SolveHost* s = solve(slot);
  if (!s) return;
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  SolveDev z;
  memset(&z, 0, sizeof(z));
  cuda_check(cudaMemcpyAsync(d_solves_ + slot, &z, sizeof(z), cudaMemcpyHostToDevice, stream_), "clear solve");
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  for (void* q : s->allocs) pool_.release(q);
  delete s;
  solves_[slot] = nullptr;
  tables_dirty_ = true;
}

void Workset::sync() { cuda_check(cudaStreamSynchronize(stream_), "cudaStreamSynchronize"); }

void Workset::reduce() {
  prof_begin(kProfReduce);
  LAUNCH(launch_reduce(tables(), cur_), "reduce");
  prof_end(kProfReduce);
}

void Workset::sched_reset() {
  cuda_check(cudaMemsetAsync(d_ctl_, 0, sizeof(SchedCtl), cur_), "memset ctl");
  if (d_done_) cuda_check(cudaMemsetAsync(d_done_, 0, sizeof(uint32_t) * nblocks_, cur_), "memset done");
}

void Workset::sweeps_f64(int64_t n, bool resid_last) {
  if (tables_dirty_) rebuild_tables();
  if (n <= 0) return;
  const Tables t = tables();
  const bool push = opt.halo == 0;
  if (opt.schedule == 1 && push) {
    // persistent block scheduler, in launches of at most 4096 sweeps
    for (int64_t done = 0; done < n;) {
      const int64_t k = std::min<int64_t>(4096, n - done);
      const bool last = done + k == n;
      sched_reset();
      prof_begin(kProfSweepF64);
      LAUNCH(launch_persist_f64(t, (int)k, resid_last && last, cur_), "persistent sweep f64");
      prof_end(kProfSweepF64);
      if (k & 1) phase_advance(1, -1);
      done += k;
    }
    if (resid_last) reduce();
    return;
  }
  for (int64_t k = 0; k < n; ++k) {
    const bool resid = resid_last && k == n - 1;
    const int kpar = (int)(k & 1);
    prof_begin(kProfSweepF64);
    if (opt.march && ndim_ == 2 && !resid && opt.emu_adds == 0)
      LAUNCH(launch_sweep_f64_march(t, kpar, push, march_width(opt.march), cur_), "sweep f64");
    else if (opt.march == 3 && ndim_ == 2 && opt.emu_adds == 0)
      LAUNCH(launch_sweep_f64_march_resid(t, kpar, push, cur_), "sweep f64 + residual");
    else LAUNCH(launch_sweep_f64(t, kpar, push, resid, true, (int)opt.emu_adds, cur_), "sweep f64");
    prof_end(kProfSweepF64);
    if (!push) {
      prof_begin(kProfHalo);
      halo_exchange_x(kpar ^ 1);
      prof_end(kProfHalo);
    }
  }
  if (resid_last) reduce();
  if (n & 1) phase_advance(1, -1);
}

void Workset::phase_advance(int d, int set_apply_e) {
  LAUNCH(launch_phase_advance(d_solves_, capacity_, d, set_apply_e, cur_), "phase advance");
  for (auto* s : solves_)
    if (s && s->active) {
      s->phase = (s->phase + d) & 1;
      if (set_apply_e >= 0) s->apply_e = set_apply_e;
    }
}

void Workset::residual_only() {
  if (tables_dirty_) rebuild_tables();
  LAUNCH(launch_sweep_f64(tables(), 0, false, true, false, 0, cur_), "residual");
  reduce();
}

void Workset::refine_outer() {
  if (tables_dirty_) rebuild_tables();
  const Tables t = tables();
  const bool push = opt.halo == 0;
  prof_begin(kProfOuter);
  if (ndim_ == 3 && opt.outer_split) {
    int64_t max_elems = 0;
    for (auto* s : solves_)
      if (s) max_elems = std::max<int64_t>(max_elems, s->elems);
    LAUNCH(launch_refine_outer_split(t, capacity_, max_elems, epar_last_, low(), r_bf16_, cur_),
           "refine outer (split)");
  } else if (ndim_ == 2 && opt.march == 3) {
    LAUNCH(launch_refine_outer_march(t, epar_last_, push, low(), r_bf16_, cur_), "refine outer");
  } else {
    LAUNCH(launch_refine_outer(t, epar_last_, push, low(), r_bf16_, cur_), "refine outer");
  }
  prof_end(kProfOuter);
  if (!push) {
    prof_begin(kProfHalo);
    halo_exchange_x(1);
    prof_end(kProfHalo);
  }
  reduce();
  phase_advance(1, 1);
}

bool Workset::use_tb2() const {
  const bool want = opt.tb == 2 || (opt.tb == 1 && low() == kLowF32 && ndim_ == 2);
  return want && opt.halo == 0 && opt.schedule == 0 && !opt.tma;
}

int Workset::inner_final_par(int64_t k) const {
  if (k <= 0) return epar_last_;
  if (!use_tb2()) return (int)((k - 1) & 1);
  // an odd k starts with one sweep into e[0]; the pairs then alternate from
  // the other buffer, and an even k starts with a pair into e[0]
  const int64_t pairs = k / 2;
  return (k & 1) ? (int)(pairs & 1) : (int)((pairs - 1) & 1);
}

void Workset::refine_inner(int64_t k) {
  if (tables_dirty_) rebuild_tables();
  if (k <= 0) return;
  const Tables t = tables();
  const bool push = opt.halo == 0;
  if (use_tb2()) {
    // two sweeps per launch: bit-identical to k single sweeps
    int cur = -1;  // buffer holding the current correction (none: e = 0)
    int64_t j = 0;
    if (k & 1) {
      prof_begin(kProfSweepLow);
      LAUNCH(launch_sweep_low(t, 0, true, push, low(), r_bf16_, cur_), "sweep low");
      prof_end(kProfSweepLow);
      cur = 0;
      j = 1;
    }
    for (; j < k; j += 2) {
      const int out = cur < 0 ? 0 : cur ^ 1;
      prof_begin(kProfSweepLow);
      LAUNCH(launch_sweep_low_tb2(t, out ^ 1, out, cur < 0, push, low(), r_bf16_, cur_), "sweep low (two per launch)");
      prof_end(kProfSweepLow);
      cur = out;
    }
    epar_last_ = cur;
    return;
  }
  if (opt.schedule == 1 && push) {
    if (k > 4096) throw JErr{1, "refine_period above 4096 with the persistent scheduler"};
    sched_reset();
    prof_begin(kProfSweepLow);
    LAUNCH(launch_persist_low(t, (int)k, low(), r_bf16_, cur_), "persistent sweep low");
    prof_end(kProfSweepLow);
  } else {
    const bool tma = opt.tma != 0;
    for (int64_t j = 0; j < k; ++j) {
      const int epar = (int)(j & 1);
      prof_begin(kProfSweepLow);
      if (tma && j > 0 && ndim_ == 2)
        LAUNCH(launch_sweep_low_tma(t, epar, push, low(), r_bf16_, cur_), "sweep low (staged)");
      else if (tma && j > 0)
        LAUNCH(launch_sweep_low_stage3(t, epar, push, low(), r_bf16_, estage_, cur_), "sweep low (staged, 3D)");
      else if (ndim_ == 3 && opt.stage3 && j > 0)
        LAUNCH(launch_sweep_low_s3(t, epar, push, low(), r_bf16_, cur_), "sweep low (lane-staged, 3D)");
      else LAUNCH(launch_sweep_low(t, epar, j == 0, push, low(), r_bf16_, cur_), "sweep low");
      prof_end(kProfSweepLow);
      if (!push) {
        prof_begin(kProfHalo);
        LAUNCH(launch_halo_pack(t, 1, epar, low(), cur_), "halo pack e");
        LAUNCH(launch_halo_unpack(t, 1, epar, low(), cur_), "halo unpack e");
        prof_end(kProfHalo);
      }
    }
  }
  epar_last_ = (int)((k - 1) & 1);
}

void Workset::read_rss(std::vector<double>& out) {
  cuda_check(cudaMemcpyAsync(h_rss_, d_rss_, sizeof(double) * capacity_, cudaMemcpyDeviceToHost, stream_), "D2H rss");
  cuda_check(cudaMemcpyAsync(h_ctl_, d_ctl_, sizeof(SchedCtl), cudaMemcpyDeviceToHost, stream_), "D2H ctl");
  cuda_check(cudaStreamSynchronize(stream_), "sync");
  out.assign(h_rss_, h_rss_ + capacity_);
  if (h_ctl_->status != 0) {
    const uint32_t task = h_ctl_->fail_task;
    cuda_check(cudaMemsetAsync(d_ctl_, 0, sizeof(SchedCtl), stream_), "memset ctl");
    cuda_check(cudaStreamSynchronize(stream_), "sync");
    throw JErr{6, "persistent scheduler: a dependency wait ran out (task " + std::to_string(task) +
                      "); the field is no longer consistent"};
  }
}

// ---------------------------------------------------------------------------
// CUDA graphs: one solve step is captured once (on a private stream) and then
// replayed on the caller's stream.

template <typename F>
bool Workset::run_graph(int64_t key, F body) {
  if (tables_dirty_) rebuild_tables();
  auto it = graphs_.find(key);
  const bool captured = it == graphs_.end();
  if (captured) {
    GraphRec rec;
    const int64_t l0 = launches_;
    cudaGraph_t g = nullptr;
    cuda_check(cudaStreamSynchronize(stream_), "sync");
    cuda_check(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cur_ = cap_stream_;
    capturing_ = true;
    try {
      body();
    } catch (...) {
      capturing_ = false;
      cur_ = stream_;
      cudaStreamEndCapture(cap_stream_, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    capturing_ = false;
    cur_ = stream_;
    cuda_check(cudaStreamEndCapture(cap_stream_, &g), "cudaStreamEndCapture");
    const cudaError_t e = cudaGraphInstantiate(&rec.exec, g, 0);
    cudaGraphDestroy(g);
    cuda_check(e, "cudaGraphInstantiate");
    rec.nodes = launches_ - l0;
    launches_ = l0;
    it = graphs_.emplace(key, rec).first;
  }
  cuda_check(cudaGraphLaunch(it->second.exec, stream_), "cudaGraphLaunch");
  launches_ += it->second.nodes;
  ++graph_replays_;
  return captured;  // the body ran on the host (and updated the host mirrors)
}

// k inner sweeps, then the outer step (x += e, r, residual).
void Workset::step_refine(int64_t k) {
  auto body = [&]() {
    refine_inner(k);
    refine_outer();
  };
  if (opt.graph && !opt.profile) {
    if (!run_graph(2 * k, body)) {
      epar_last_ = inner_final_par(k);
      for (auto* s : solves_)
        if (s && s->active) {
          s->phase ^= 1;
          s->apply_e = 1;
        }
    }
  } else {
    body();
  }
}

// n FP64 sweeps, the last one reducing the residual of its input.
void Workset::chunk_f64(int64_t n) {
  auto body = [&]() { sweeps_f64(n, true); };
  if (opt.graph && !opt.profile) {
    if (!run_graph(2 * n + 1, body))
      for (auto* s : solves_)
        if (s && s->active) s->phase = (s->phase + (int)(n & 1)) & 1;
  } else {
    body();
  }
}

// ---------------------------------------------------------------------------
// solve loop over every active slot

void Workset::solve_all(double tol, int64_t max_sweeps, std::vector<SlotResult>& res) {
  if (tables_dirty_) rebuild_tables();
  if (opt.autotune && !tuned_) autotune();
  // however the loop ends (also by an exception), tables compacted to the
  // active solves are marked for a full rebuild, and a work shape re-tuned
  // for the last solves is not kept for the next call
  struct CompactGuard {
    Workset* w;
    bool retuned = false;
    ~CompactGuard() {
      if (w->compact_) {
        w->compact_ = false;
        w->tables_dirty_ = true;
      }
      if (retuned) w->tuned_ = false;
    }
  } guard{this};
  res.assign(capacity_, SlotResult());
  std::vector<int> slots;
  for (int k = 0; k < capacity_; ++k)
    if (solves_[k] && solves_[k]->active) slots.push_back(k);
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<double> rss;
  int64_t m = 0;
  int left = (int)slots.size();
  const bool ref = refine();
  if (ref) refine_outer();
  else chunk_f64(1);
  std::vector<int32_t> ctl(capacity_, 8);
  while (left > 0) {
    read_rss(rss);
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    std::fill(ctl.begin(), ctl.end(), 8);
    bool retire = false;
    for (int k : slots) {
      SlotResult& r = res[k];
      if (r.done) continue;
      SolveHost* s = solves_[k];
      const double rel = s->bss > 0.0 ? std::sqrt(rss[k]) / std::sqrt(s->bss) : std::sqrt(rss[k]);
      int st = -1;
      if (!std::isfinite(rel)) st = 5;
      else if (rel <= tol) st = 0;
      else if (m >= max_sweeps) st = 4;
      if (st < 0) continue;
      r = SlotResult{st, m, rel, secs, true};
      --left;
      // retire the slot; plain FP64 also steps back to iterate m (the checked
      // one: the last sweep only reduced its residual)
      ctl[k] = ref ? 4 : 2;
      retire = true;
    }
    if (retire) {
      apply_slot_ctl(ctl);
      // once the retired solves hold most of the tabled points, launch only
      // the active ones (the tables and graphs are rebuilt at the next step)
      int64_t live_pts = 0;
      for (int k : slots)
        if (!res[k].done) live_pts += solves_[k]->points();
      if (left > 0 && 2 * live_pts < tabled_points_) {
        compact_ = true;
        tables_dirty_ = true;
        // the work shape tuned for the whole batch may leave the GPU idle
        // once only the largest grids remain: tune again for the active ones
        if (opt.autotune) {
          tuned_ = false;
          autotune();
          guard.retuned = true;
        }
      }
    }
    if (left == 0) break;
    const int64_t n = std::min<int64_t>(ref ? opt.refine_period : opt.check_every, max_sweeps - m);
    if (ref) step_refine(n);
    else chunk_f64(n);
    m += n;
  }
  // every slot that took part is active again; a refinement's correction is consumed
  std::fill(ctl.begin(), ctl.end(), 8);
  for (int k : slots) ctl[k] = ref ? (1 | 4) : 1;
  apply_slot_ctl(ctl);
}

// ---------------------------------------------------------------------------
// autotuner: time a few sweeps of each candidate (rows per work item, launch
// schedule) and keep the fastest.  Every candidate computes the same bits, so
// the choice never changes a result.  Choices are cached in the JSON-lines
// file named by JACOBI_TUNE_CACHE (when set).

static std::string tune_key(const Workset& w, const std::vector<SolveHost*>& solves, int dtype) {
  std::ostringstream k;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  int64_t pts = 0, nb = 0, bx = 0, by = 0, bz = 0;
  for (auto* s : solves)
    if (s && s->active) {
      pts += s->points();
      nb += (int64_t)s->blocks.size();
      bx = s->spec.blk[0];
      by = s->spec.blk[1];
      bz = s->spec.blk[2];
    }
  // points rounded to a power of two so that similar worksets share an entry
  const int lg = pts > 0 ? (int)std::lround(std::log2((double)pts)) : 0;
  k << prop.name << "|d" << w.ndim() << "|t" << dtype << "|b" << bx << "x" << by << "x" << bz << "|p2^" << lg
    << "|nb" << (nb > 1 ? (int)std::lround(std::log2((double)nb)) : 0);
  std::string s = k.str();
  for (auto& c : s)
    if (c == '"') c = '\'';
  return s;
}

static bool tune_cache_lookup(const std::string& key, int64_t& rows, int64_t& sched, int64_t& march, int64_t& tb) {
  const char* path = std::getenv("JACOBI_TUNE_CACHE");
  if (!path) return false;
  std::ifstream in(path);
  std::string line;
  bool found = false;
  while (std::getline(in, line)) {
    const std::string kk = "\"key\": \"" + key + "\"";
    if (line.find(kk) == std::string::npos) continue;
    long long r = 0, s = 0;
    const size_t pr = line.find("\"rows\": "), ps = line.find("\"schedule\": ");
    if (pr == std::string::npos || ps == std::string::npos) continue;
    r = std::atoll(line.c_str() + pr + 8);
    s = std::atoll(line.c_str() + ps + 12);
    const size_t pm = line.find("\"march\": ");
    if (r >= 1 && (s == 0 || s == 1)) {
      rows = r;
      sched = s;
      if (pm != std::string::npos) march = std::min<long long>(std::max<long long>(std::atoll(line.c_str() + pm + 9), 0), 3);
      const size_t pt = line.find("\"tb\": ");
      if (pt != std::string::npos) tb = std::min<long long>(std::max<long long>(std::atoll(line.c_str() + pt + 6), 0), 2);
      found = true;
    }
  }
  return found;
}

static void tune_cache_store(const std::string& key, int64_t rows, int64_t sched, int64_t march, int64_t tb,
                             double us) {
  const char* path = std::getenv("JACOBI_TUNE_CACHE");
  if (!path) return;
  std::ofstream out(path, std::ios::app);
  out << "{\"key\": \"" << key << "\", \"rows\": " << rows << ", \"schedule\": " << sched
      << ", \"march\": " << march << ", \"tb\": " << tb << ", \"us_per_sweep\": " << us << "}\n";
}

void Workset::autotune() {
  tuned_ = true;
  if (live() == 0) return;
  const bool ref = refine();
  const std::string key = tune_key(*this, solves_, dtype_);
  int64_t rows = 0, sched = 0, march = opt.march, tb = opt.tb;
  int64_t& opt_rows = ref ? opt.rows_low : opt.rows_f64;
  if (tune_cache_lookup(key, rows, sched, march, tb)) {
    opt_rows = rows;
    opt.schedule = sched;
    opt.march = march;
    opt.tb = tb;
    rebuild_tables();
    tune_summary_ = "cache: rows " + std::to_string(rows) + ", schedule " + std::to_string(sched) + ", march " +
                    std::to_string(march) + ", tb " + std::to_string(tb);
    return;
  }
  // snapshot of every FP64 iterate so the timing sweeps leave no trace
  std::vector<std::pair<double*, void*>> saved;
  if (!ref) {
    for (auto* s : solves_)
      if (s) {
        void* tmp = pool_.alloc((size_t)s->elems * 16);
        cuda_check(cudaMemcpyAsync(tmp, s->x[0], (size_t)s->elems * 8, cudaMemcpyDeviceToDevice, stream_), "save");
        cuda_check(cudaMemcpyAsync((char*)tmp + s->elems * 8, s->x[1], (size_t)s->elems * 8, cudaMemcpyDeviceToDevice,
                                   stream_),
                   "save");
        saved.push_back({(double*)tmp, s});
      }
  }
  std::vector<int> phases;
  for (auto* s : solves_) phases.push_back(s ? s->phase : 0);
  const int64_t prof = opt.profile, graph = opt.graph;
  opt.profile = 0;
  opt.graph = 0;
  cudaEvent_t a, b;
  cuda_check(cudaEventCreate(&a), "event");
  cuda_check(cudaEventCreate(&b), "event");
  double best = 1e300;
  int64_t best_rows = opt_rows, best_sched = opt.schedule, best_march = opt.march, best_tb = opt.tb;
  // FP64 items hold whole residual groups of 8 lines; the low-precision
  // items may be shorter (small grids need many short items to fill the GPU)
  std::vector<int64_t> cand_rows = {8, 16, 32, 64, 128};
  if (ref) cand_rows.insert(cand_rows.begin(), {1, 2, 4});
  struct Cand {
    int64_t rows, sched, march, tb;
  };
  std::vector<Cand> cands;
  for (int64_t sc = 0; sc <= 1; ++sc)
    for (int64_t r : cand_rows) cands.push_back(Cand{r, sc, ref ? opt.march : 0, 0});
  // FP64 march items are sized by the workset itself; rows only shapes the
  // residual sweeps then
  if (!ref && ndim_ == 2) {
    cands.push_back(Cand{32, 0, 1, 0});
    cands.push_back(Cand{32, 0, 2, 0});
    cands.push_back(Cand{32, 0, 3, 0});
  }
  // 2D inner sweeps two per launch (even sweep counts time the pairs)
  if (ref && opt.halo == 0) {
    for (auto& c : cands) c.tb = 0;  // the candidates above: one sweep per launch
    cands.push_back(Cand{ndim_ == 2 ? 16 : 32, 0, opt.march, 2});
  }
  const int sweeps = 8;
  {
    bool first = true;
    for (const Cand& cd : cands) {
      const int64_t r = cd.rows, sc = cd.sched;
      opt_rows = r;
      opt.schedule = sc;
      opt.march = cd.march;
      opt.tb = cd.tb;
      rebuild_tables();
      auto run = [&]() {
        if (ref) refine_inner(sweeps);
        else sweeps_f64(sweeps, false);
      };
      // warm-up (the first candidate longer, so that clocks and caches have
      // settled before anything is timed), then the best of three timings
      for (int w = 0; w < (first ? 8 : 1); ++w) run();
      first = false;
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cuda_check(cudaEventRecord(a, stream_), "event");
        run();
        cuda_check(cudaEventRecord(b, stream_), "event");
        cuda_check(cudaEventSynchronize(b), "event");
        float t = 0.f;
        cuda_check(cudaEventElapsedTime(&t, a, b), "event");
        ms = std::min(ms, t);
      }
      if (ms < best) {
        best = ms;
        best_rows = r;
        best_sched = sc;
        best_march = cd.march;
        best_tb = cd.tb;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  opt.profile = prof;
  opt.graph = graph;
  opt_rows = best_rows;
  opt.schedule = best_sched;
  opt.march = best_march;
  opt.tb = best_tb;
  rebuild_tables();
  // restore the iterates and phases the timing sweeps changed
  if (!ref) {
    size_t i = 0;
    for (auto* s : solves_)
      if (s) {
        double* tmp = saved[i++].first;
        cuda_check(cudaMemcpyAsync(s->x[0], tmp, (size_t)s->elems * 8, cudaMemcpyDeviceToDevice, stream_), "restore");
        cuda_check(cudaMemcpyAsync(s->x[1], (char*)tmp + s->elems * 8, (size_t)s->elems * 8, cudaMemcpyDeviceToDevice,
                                   stream_),
                   "restore");
      }
    sync();
    for (auto& sv : saved) pool_.release(sv.first);
  }
  std::vector<int32_t> ctl(capacity_, 8);
  for (int k = 0; k < capacity_; ++k)
    if (solves_[k] && solves_[k]->phase != phases[k]) ctl[k] = (solves_[k]->active ? 1 : 0) | 2;
  apply_slot_ctl(ctl);
  const double us = best * 1e3 / sweeps;
  tune_cache_store(key, best_rows, best_sched, best_march, best_tb, us);
  tune_summary_ = "measured: rows " + std::to_string(best_rows) + ", schedule " + std::to_string(best_sched) +
                  ", march " + std::to_string(best_march) + ", tb " + std::to_string(best_tb) + ", " +
                  std::to_string(us) + " us per sweep";
}

// ---------------------------------------------------------------------------
// profiling with CUDA events on the launching stream

void Workset::prof_begin(int kind) {
  (void)kind;
  if (!opt.profile || capturing_) return;
  if (ev_free_.empty()) {
    cudaEvent_t e;
    cuda_check(cudaEventCreate(&e), "cudaEventCreate");
    ev_free_.push_back(e);
  }
  ev_open_ = ev_free_.back();
  ev_free_.pop_back();
  cuda_check(cudaEventRecord(ev_open_, cur_), "cudaEventRecord");
}

void Workset::prof_end(int kind) {
  if (!opt.profile || capturing_ || !ev_open_) return;
  if (ev_free_.empty()) {
    cudaEvent_t e;
    cuda_check(cudaEventCreate(&e), "cudaEventCreate");
    ev_free_.push_back(e);
  }
  cudaEvent_t b = ev_free_.back();
  ev_free_.pop_back();
  cuda_check(cudaEventRecord(b, cur_), "cudaEventRecord");
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
