// Internal data structures shared by the host engine and the CUDA kernels.
//
// Layout of one solve in HBM (the over-decomposed domain of section 4.4: the
// grid is cut into blocks, each block a task with its own storage):
//
//   * Every array of a solve (x[0], x[1], f in FP64; e[0], e[1], r in the
//     low-precision type) uses the SAME element layout, so one element offset
//     addresses a point in all of them.
//   * Block main array: planes z = -gz .. bz-1+gz (gz = 1 in 3D, 0 in 2D),
//     rows y = -1 .. by, each row `pitch` elements holding x = 0 .. bx-1.
//     Rows -1 and by (and planes -1 and bz in 3D) are the ghost ring along
//     y (and z); element (x, y, z) sits at off + (z+gz)*plane + (y+1)*pitch + x.
//     pitch is a multiple of 16 elements and off a multiple of 32, so rows are
//     128-byte aligned for FP64 and 64-byte aligned for FP32.
//   * The ghost ring along x is stored apart, as two contiguous columns
//     (gW then gE, bz*by elements each, y fastest) at xoff, so that reading a
//     block's west/east ghosts costs a contiguous stream, not one sector per
//     row.
//   * Ghosts on the domain boundary hold the Dirichlet values g (x) or 0 (e)
//     and are written once; ghosts on block boundaries are rewritten after
//     every sweep by the halo exchange (section 4.3: pack, transfer, unpack).
#pragma once
#include <stdint.h>

namespace jgb {

constexpr int kWarps = 8;            // warps per CTA of the sweep kernels
constexpr int kThreads = 32 * kWarps;
constexpr int kSegF64 = 64;          // points per warp row, FP64 kernels (2 per lane)
constexpr int kSegLow = 128;         // points per warp row, FP32 inner sweeps (4 per lane)
constexpr int kSegLow16 = 256;       // points per warp row, bfloat16 inner sweeps (8 per lane)
constexpr int kResSeg = 64;          // points per residual partial along x (fixed: decomposition independent)
constexpr int kResGroup = 8;         // lines of the march axis summed into one residual partial
// log2 of the lanes one block row takes in a 3D low-precision warp item:
// enough for bx points at v per lane, a power of two, at most 32
__host__ __device__ inline int low_lanes_log2(int bx, int v) {
  const int need = (bx + v - 1) / v;
  int lg = 0;
  while (lg < 5 && (1 << lg) < need) ++lg;
  return lg;
}
constexpr int kMarchLines = 64;      // most lines in one FP64 march item (its shared-memory pair buffer)
constexpr int kTbTileW = 128;        // two-sweep inner kernel: tile width (points) ...
constexpr int kTbTileH = 32;         // ... and height (lines; measured faster than 30 or 62)
constexpr int kTb3TileW = 64;        // 3D two-sweep inner kernel: tile width (x points) ...
constexpr int kTb3TileH = 16;        // ... height (y rows) ...
constexpr int kTb3TileZ = 16;        // ... and depth (z planes it marches through)
constexpr int kRedThreads = 256;     // threads of the reduction kernel
constexpr int kRedChunk = 4096;      // partials summed by one reduction CTA

enum LowType { kLowF32 = 0, kLowBF16 = 1 };

// Neighbour order: -x, +x, -y, +y, -z, +z.
struct BlockDev {
  int64_t off;        // element offset of the main array (plane -gz, row -1)
  int64_t xoff;       // element offset of the x ghost columns
  int64_t part;       // first residual slot of this block column (solve-relative)
  int64_t foff;       // element offset of this block's 6 face send buffers (standalone halo)
  int32_t bx, by, bz;
  int32_t pitch;      // elements per row
  int32_t plane;      // elements per plane = (by + 2) * pitch
  int32_t gz;         // 1 in 3D, 0 in 2D
  int32_t oy, oz;     // origin of the block in the solve grid (y, z)
  int32_t solve;      // index into the solve table
  int32_t nbr[6];     // neighbour block index (table-wide) or -1 on the domain boundary
  int32_t fsz[6];     // elements of each face send buffer
  int32_t ox;         // origin of the block in the solve grid (x)
  int32_t nt64;       // CTA tasks of this block in the FP64 task table
  int32_t ntlo;       // CTA tasks of this block in the low-precision task table
  int32_t pg;         // first residual group of this block along the march axis (solve-wide)
};

struct SolveDev {
  double* x[2];       // FP64 iterate, ping-pong
  double* f;          // FP64 source (interior points only are read)
  void* e[2];         // low-precision correction, ping-pong
  void* r;            // low-precision residual
  double* send64;     // face send buffers (FP64 arrays)
  void* sendlo;       // face send buffers (low arrays)
  double* part;       // residual partials
  double* lvl1;       // first-level reduction results
  double* rss;        // [0] = sum of squares written by the reduction
  uint32_t* ticket;   // reduction ticket
  int64_t nparts;     // residual partial slots
  int64_t elems;      // elements of each layout array (x, f, e, r)
  int32_t part_row;   // partial slots per grid row
  int32_t ny;         // grid rows along y (for the partial row index)
  int32_t ndim;
  int32_t phase;      // x[phase] holds the current iterate
  int32_t active;     // 0: every kernel skips this solve
  int32_t apply_e;    // refinement: 1 once a correction e exists
  int32_t low;        // LowType of e and r
  int32_t r_bf16;     // 1: r stored as bfloat16 (else FP32)
};

// One warp's work: `n` consecutive rows (2D: along y) or planes (3D: along z)
// of one segment of one block.  In 3D the row y is fixed.
struct WorkItem {
  int32_t block;
  int16_t seg;
  int16_t n;
  int32_t y0;
  int32_t z0;
};

// One task of the persistent scheduler: up to kWarps consecutive warp items,
// all of one block (a task in the sense of section 3.1.2: a unit of work with
// known inputs; its dependencies are the block and its neighbours).
struct CtaTask {
  int32_t block;
  int32_t w0;  // first warp item
  int32_t nw;  // warp items (1 .. kWarps)
  int32_t pad;
};

// Control word of one persistent launch (zeroed before it).
struct SchedCtl {
  uint32_t head;       // next task index handed out
  uint32_t status;     // 0 ok, 1 a dependency wait ran out (JACOBI_ERR_TIMEOUT)
  uint32_t fail_task;  // task index whose wait ran out
  uint32_t pad;
};

// One face of one block for the standalone pack / unpack kernels.
struct FaceItem {
  int32_t block;
  int32_t face;
};

// One CTA of the reduction: `len` partials of solve `solve` from `start`.
struct RedItem {
  int32_t solve;
  int32_t chunk;      // chunk index within the solve
  int32_t nchunks;    // chunks of this solve
  int32_t len;
  int64_t start;
};

// One CTA-row job of the dense <-> blocked copies: one row of one block.
struct RowItem {
  int32_t block;
  int32_t y;
  int32_t z;
  int32_t pad;
};

// Kernel launch wrappers (kernels.cu).  All return cudaError_t as int.
struct Tables {
  const WorkItem* w64;  int n64;     // FP64 sweep / residual / refine-outer items
  const WorkItem* wlo;  int nlo;     // low-precision sweep items
  const WorkItem* wm;   int nm;      // FP64 march items (all segments of a line range)
  const int* wms;       int nmw;     // option march 3: warp w computes items wms[w] .. wms[w+1]-1 of wm
  const WorkItem* wmr;  int nmr;     // march items of whole residual groups (kResGroup lines)
  const int* wmrs;      int nmrw;    // warp w computes items wmrs[w] .. wmrs[w+1]-1 of wmr
  const WorkItem* wtb;  int ntb;     // tiles of the two-sweep inner kernel (seg = tile column, n = lines)
  const FaceItem* faces; int nfaces; // interior faces
  const RedItem* red;   int nred;    // reduction CTAs
  const RowItem* rows;  int nrows;   // block rows
  const BlockDev* blocks;
  SolveDev* solves;
  int ndim;
  const CtaTask* t64;   int nt64;    // persistent tasks over w64
  const CtaTask* tlo;   int ntlo;    // persistent tasks over wlo
  uint32_t* done;                    // per block: tasks completed in this launch
  SchedCtl* ctl;
  uint32_t spin_limit;               // bounded dependency waits
  int poison;                        // test hook: every dependency wait runs out
  int l2pf;                          // FP64 sweeps: lines ahead prefetched into L2 (0: none)
};

int launch_sweep_f64(const Tables& t, int kpar, bool push, bool resid, bool write, int emu, void* stream);
// 2D FP64 sweep (no residual) over the march items; width = points per lane
// (2: 64-point segments, 4: 128-point segments)
int launch_sweep_f64_march(const Tables& t, int kpar, bool push, int width, void* stream);
// warps of the 2D march sweep resident at once on the current device (0 on
// error or in 3D)
int march_f64_resident_warps(int ndim, bool push, int width);
// 2D fused-residual FP64 sweep over t.wmr (four points per lane, lines
// staged in shared memory): bit-identical to launch_sweep_f64 with resid,
// partials included
int launch_sweep_f64_march_resid(const Tables& t, int kpar, bool push, void* stream);
// 2D refinement outer step over t.wmr: bit-identical to launch_refine_outer
int launch_refine_outer_march(const Tables& t, int epar_last, bool push, int low, bool r_bf16, void* stream);
// warps of the two kernels above resident at once (the smaller count; 0 on
// error or in 3D)
int march_f64r_resident_warps(int ndim, bool push);
int launch_sweep_low(const Tables& t, int epar, bool first, bool push, int low, bool r_bf16, void* stream);
// 3D inner sweep (not the first of a refinement step) with each lane's lines
// staged ahead in shared memory by per-lane asynchronous copies (option stage3)
int launch_sweep_low_s3(const Tables& t, int epar, bool push, int low, bool r_bf16, void* stream);
// 2D inner sweep (not the first of a step) with rows staged in shared memory
// by bulk asynchronous copies; a timed-out wait sets ctl->status bit 1.
int launch_sweep_low_tma(const Tables& t, int epar, bool push, int low, bool r_bf16, void* stream);
// 3D inner sweep (not the first of a step) with the rows of e and r a warp
// needs staged in shared memory by 16-byte asynchronous copies; estage =
// elements of e per stage per warp (the largest (R + 2) * L * V over the
// workset's blocks).
int launch_sweep_low_stage3(const Tables& t, int epar, bool push, int low, bool r_bf16, int estage, void* stream);
// Two inner sweeps in one launch (2D), one CTA per tile of t.wtb:
// e[out_par] = J(J(e[in_par])), or J(J(0)) when first; bit-identical to two
// launch_sweep_low calls.  The input buffer is not written (in_par != out_par).
int launch_sweep_low_tb2(const Tables& t, int in_par, int out_par, bool first, bool push, int low, bool r_bf16,
                         void* stream);
int launch_refine_outer(const Tables& t, int epar_last, bool push, int low, bool r_bf16, void* stream);
// The outer step in two passes: x[phase^1] = x[phase] + e over every element
// of the layout (ghosts included: e's ghosts hold the neighbours' values and
// zero on the domain faces), then r = b - A x[phase^1] with no x write.
// max_elems: the largest `elems` of the solves.
int launch_refine_outer_split(const Tables& t, int nslots, int64_t max_elems, int epar_last, int low, bool r_bf16,
                              void* stream);
int launch_halo_pack(const Tables& t, int which, int par, int low, void* stream);
int launch_halo_unpack(const Tables& t, int which, int par, int low, void* stream);
int launch_reduce(const Tables& t, void* stream);
int launch_scatter(const Tables& t, const double* dense, int which, int par, int64_t nx, int64_t ny, void* stream);
int launch_gather(const Tables& t, double* dense, int par, int64_t nx, int64_t ny, void* stream);
int launch_ghost_fill(const Tables& t, const double* const* faces_dev, int par, int64_t nx, int64_t ny,
                      int64_t nz, void* stream);
int launch_phase_advance(SolveDev* solves, int nsolves, int dphase, int set_apply_e, void* stream);
// Persistent block scheduler: one launch runs nsweeps sweeps of every active
// solve; CTAs pull (sweep, task) pairs in sweep order and wait (bounded) for
// the block's and its neighbours' previous sweep.
int launch_persist_f64(const Tables& t, int nsweeps, bool resid_last, void* stream);
int launch_persist_low(const Tables& t, int nsweeps, int low, bool r_bf16, void* stream);
// Per-slot control from the host: ctl[i] bit 0 = new active flag, bit 1 = flip the phase,
// bit 2 = clear apply_e, bit 3 = leave the slot unchanged.
int launch_solve_ctl(SolveDev* solves, const int32_t* ctl, int nsolves, void* stream);

}  // namespace jgb
