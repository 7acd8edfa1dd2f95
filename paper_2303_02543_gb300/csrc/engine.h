// Host-side engine: a "workset" is a set of independent Jacobi solves whose
// blocks are processed together by every kernel launch.  A single-grid
// context is a workset of one solve; the batch and server interfaces add and
// retire solves.  Over-decomposition (section 4.4) is the block table: every
// block of every solve becomes warp work items in one table, so one launch
// covers all blocks and all solves.
#pragma once
#include <cuda_runtime.h>

#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "jacobi_internal.h"

namespace jgb {

struct JErr {
  int code;
  std::string msg;
};

struct AllocHooks {
  void* (*alloc)(size_t, void*, void*) = nullptr;
  void (*free)(void*, void*, void*) = nullptr;
  void* user = nullptr;
};

AllocHooks current_alloc_hooks();
void set_alloc_hooks(const AllocHooks& h);

// Owns device allocations made through the hooks captured at construction.
class DevPool {
 public:
  DevPool(const AllocHooks& h, cudaStream_t s) : hooks_(h), stream_(s) {}
  ~DevPool();
  void* alloc(size_t bytes);  // zero bytes -> nullptr; failure throws JErr(OOM)
  void release(void* p);      // frees one allocation
  int64_t bytes() const { return bytes_; }

 private:
  struct Rec {
    void* p;
    size_t n;
  };
  AllocHooks hooks_;
  cudaStream_t stream_;
  std::vector<Rec> recs_;
  int64_t bytes_ = 0;
};

// Problem description of one solve (host memory unless inputs_on_device).
struct ProblemSpec {
  int ndim = 2;
  int64_t n[3] = {1, 1, 1};
  int64_t blk[3] = {1, 1, 1};
  int bc_kind = 0;
  double bc_value = 0.0;
  const double* faces[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const double* source = nullptr;
  const double* x0 = nullptr;
  int inputs_on_device = 0;
};

struct SolveHost {
  ProblemSpec spec;
  int nb[3] = {1, 1, 1};
  int slot = -1;                 // index in the solve table
  int64_t elems = 0;             // elements per array in the layout
  int64_t face_elems = 0;        // elements of the face send buffers
  int64_t nparts = 0;
  int part_row = 0;
  int nchunks = 0;
  double bss = 0.0;              // ||b||^2
  std::vector<BlockDev> blocks;  // nbr indices are local (0-based within the solve)
  // device memory (owned by the workset pool)
  double* x[2] = {nullptr, nullptr};
  double* f = nullptr;
  void* e[2] = {nullptr, nullptr};
  void* r = nullptr;
  double* send64 = nullptr;
  void* sendlo = nullptr;
  double* part = nullptr;
  double* lvl1 = nullptr;
  std::vector<void*> allocs;
  // host mirrors of device state
  int phase = 0;
  int apply_e = 0;
  int active = 1;
  int64_t points() const { return spec.n[0] * spec.n[1] * spec.n[2]; }
};

// Bytes of device memory one solve needs (layout arrays, face buffers,
// partial sums): the admission test of the server.
int64_t solve_device_bytes(const ProblemSpec& p, int dtype, bool r_bf16);

enum ProfKind { kProfSweepF64 = 0, kProfSweepLow, kProfOuter, kProfReduce, kProfHalo, kProfCount };

struct Options {
  int64_t check_every = 50;
  int64_t refine_period = 20;
  int64_t halo = 0;          // 0 fused, 1 standalone pack/unpack
  int64_t rows_f64 = 32;
  int64_t rows_low = 0;      // 0: chosen by dimensionality and type (see rebuild_tables)
  int64_t profile = 0;
  int64_t schedule = 0;      // 0 one launch per sweep, 1 persistent block scheduler
  int64_t graph = 0;         // 1: replay each solve step from a captured CUDA graph
  int64_t spin_limit = 1 << 22;
  int64_t poison_wait = 0;   // test hook: every dependency wait of the persistent kernel runs out
  int64_t autotune = 0;      // 1: pick rows/schedule by timing before the first solve
  int64_t emu_adds = 0;      // FP64 sweep: additions per warp step done on the integer pipe (0, 2, 3)
  int64_t tma = 0;           // inner sweeps (2D and 3D): stage lines in shared memory with bulk async copies
  int64_t stage3 = 1;        // 3D inner sweeps after the first: each lane's lines staged ahead in shared memory
  int64_t march = 3;         // FP64 sweeps without a residual: one warp computes all segments of a line range
  int64_t outer_split = 1;   // 3D outer step as x += e over the layout, then the residual pass
  int64_t l2pf = 0;          // FP64 sweeps: lines ahead brought into L2 by bulk prefetches (0: none)
  int64_t tb = 1;            // inner sweeps two per launch (temporal blocking; 2D, fused halo, launch schedule):
                             // 2 always, 0 never, 1 (default) for FP32 corrections (measured faster) only
};

// Outcome of one solve inside solve_all.
struct SlotResult {
  int status = 0;
  int64_t sweeps = 0;
  double rel = 0.0;
  double seconds = 0.0;
  bool done = false;
};

class Workset {
 public:
  Workset(int ndim, int dtype, cudaStream_t stream, int capacity, bool r_bf16 = false,
          const AllocHooks* hooks = nullptr);
  ~Workset();
  Workset(const Workset&) = delete;
  Workset& operator=(const Workset&) = delete;

  // Adds a solve, uploads its inputs, computes ||b||; returns its slot.
  int add_solve(const ProblemSpec& p);
  void remove_solve(int slot);
  void rebuild_tables();

  // Plain FP64 sweeps of every active solve; with resid_last the last sweep
  // also reduces the residual of its input iterate.
  void sweeps_f64(int64_t n, bool resid_last);
  void phase_advance(int d, int set_apply_e);
  // Residual of the current iterate of every active solve (no sweep).
  void residual_only();
  // Refinement: outer step (x += e if pending; r; reduction), then k inner sweeps.
  void refine_outer();
  void refine_inner(int64_t k);
  // Read the sums of squares of every slot (synchronises; throws on a timed
  // out dependency wait of the persistent scheduler).
  void read_rss(std::vector<double>& out);
  void set_active(int slot, int active);
  void sync();

  // Solve every active slot to tol (the test of section 8's solve rule):
  // plain FP64 with checks every check_every sweeps, or refinement with a
  // check after every outer step.  Slots stay active afterwards.
  void solve_all(double tol, int64_t max_sweeps, std::vector<SlotResult>& res);
  // Pick rows_f64 / rows_low / schedule by timing (restores the state).
  void autotune();
  // Serving: k inner sweeps then the outer step for every active solve (a
  // newly added solve's first inner sweeps see r = 0 and leave e = 0, so its
  // first outer step only computes r of its initial iterate).
  void serve_step(int64_t k);

  void scatter(int slot, const double* dense, int which, int on_device);
  void gather(int slot, double* dense, int on_device);
  void halo_exchange_x(int kpar);

  // profiling
  void prof_begin(int kind);
  void prof_end(int kind);
  void prof_collect(int kind, double* ms, int64_t* n, bool reset);

  bool refine() const { return dtype_ != 0; }
  int ndim() const { return ndim_; }
  int dtype() const { return dtype_; }
  int low() const { return dtype_ >= 2 ? kLowBF16 : kLowF32; }
  bool r_bf16() const { return r_bf16_; }
  cudaStream_t stream() const { return stream_; }
  SolveHost* solve(int slot) { return slot >= 0 && slot < (int)solves_.size() ? solves_[slot] : nullptr; }
  int capacity() const { return capacity_; }
  int live() const;
  int64_t device_bytes() const { return pool_.bytes(); }
  int64_t launches() const { return launches_; }
  int64_t graph_replays() const { return graph_replays_; }
  std::string tune_summary() const { return tune_summary_; }

  Options opt;

 private:
  void layout_solve(SolveHost& s);
  void alloc_solve(SolveHost& s);
  void upload_inputs(SolveHost& s);
  void push_solve_dev(SolveHost& s);
  Tables tables() const;
  Tables solve_tables(const SolveHost& s) const;
  void reduce();
  void sched_reset();
  void apply_slot_ctl(const std::vector<int32_t>& ctl);
  // one solve step, captured in a CUDA graph when opt.graph is set
  void step_refine(int64_t k);
  // buffer e[.] that holds the correction after refine_inner(k)
  int inner_final_par(int64_t k) const;
  bool use_tb2() const;
  void chunk_f64(int64_t n);
  template <typename F>
  bool run_graph(int64_t key, F body);
  void drop_graphs();

  int ndim_, dtype_, capacity_;
  bool r_bf16_;
  cudaStream_t stream_;   // the caller's stream: everything ends up here
  cudaStream_t cur_;      // where launches are issued (stream_, or the capture stream)
  cudaStream_t cap_stream_ = nullptr;
  void free_host_side();  // page-locked mirrors and the capture stream
  bool capturing_ = false;
  DevPool pool_;
  std::vector<SolveHost*> solves_;   // slot -> solve (nullptr when free)
  // device tables
  SolveDev* d_solves_ = nullptr;
  double* d_rss_ = nullptr;
  uint32_t* d_ticket_ = nullptr;
  double* h_rss_ = nullptr;          // pinned
  SchedCtl* d_ctl_ = nullptr;
  SchedCtl* h_ctl_ = nullptr;        // pinned
  int32_t* d_slotctl_ = nullptr;
  int32_t* h_slotctl_ = nullptr;     // pinned
  BlockDev* d_blocks_ = nullptr;
  WorkItem* d_w64_ = nullptr;
  WorkItem* d_wlo_ = nullptr;
  WorkItem* d_wm_ = nullptr;
  int nm_ = 0;
  WorkItem* d_wmr_ = nullptr;  // march items on residual-group boundaries (option march 3)
  int nmr_ = 0;
  int* d_wms_ = nullptr;   // option march 3: first item of each warp's run (wm), then the end
  int* d_wmrs_ = nullptr;  // the same for wmr
  int nmw_ = 0, nmrw_ = 0; // warps of the two runs tables
  WorkItem* d_wtb_ = nullptr;  // tiles of the two-sweep inner kernel
  int ntb_ = 0;
  int estage_ = 0;  // staged 3D inner sweep: e elements per stage per warp
  // solve_all: tables hold only the active solves (retired ones dropped once
  // they are most of the tabled points); restored before solve_all returns
  bool compact_ = false;
  int64_t tabled_points_ = 0;
  CtaTask* d_t64_ = nullptr;
  CtaTask* d_tlo_ = nullptr;
  uint32_t* d_done_ = nullptr;
  FaceItem* d_faces_ = nullptr;
  RedItem* d_red_ = nullptr;
  RowItem* d_rows_ = nullptr;
  int n64_ = 0, nlo_ = 0, nt64_ = 0, ntlo_ = 0, nfaces_ = 0, nred_ = 0, nrows_ = 0, nblocks_ = 0;
  std::vector<void*> table_allocs_;
  std::vector<int> face_base_, face_cnt_, row_base_, row_cnt_;
  int epar_last_ = 0;
  int64_t launches_ = 0;           // kernel launches issued so far
  int64_t graph_replays_ = 0;
  bool tables_dirty_ = true;
  bool tuned_ = false;
  std::string tune_summary_;
  struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
  };
  std::map<int64_t, GraphRec> graphs_;
  // profiling events
  struct EvPair {
    cudaEvent_t a, b;
  };
  std::vector<EvPair> ev_pending_[kProfCount];
  std::vector<cudaEvent_t> ev_free_;
  double prof_ms_[kProfCount] = {0, 0, 0, 0, 0};
  int64_t prof_n_[kProfCount] = {0, 0, 0, 0, 0};
  cudaEvent_t ev_open_ = nullptr;
};

}  // namespace jgb
