// jacobi_residual_noalloc: the residual norm of an interior-dense field with
// no device allocation at all.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned
// in full by another runtime's pool, or a latency-bound loop that must never
// stall, since cudaMalloc and cudaFree may synchronise the whole device.  This
// entry point serves them.  It allocates nothing; its scratch memory (the
// partial sums, the first-level sums and the reduction ticket) lives
// in one file-scope __device__ array of fixed size that every GPU loading the
// library holds until the process exits.
//
// The arithmetic is that of the library's fused residual: r = t - (2d) x with
// t the neighbour sum plus source in the canonical order, r^2 summed per lane
// over groups of 8 lines of the last axis and then across a 64-point segment
// by the same warp tree, then the same two-level reduction.  Its result is
// bit-identical to jacobi_residual on a monolithic context (and on any context
// whose block extents are multiples of 64 along x and of 8 along the last axis).
#include <cuda.h>  // CUcontext / CUresult types only: the driver is reached through the runtime
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/jacobi.h"

namespace jgb {
void set_thread_error(const std::string& msg);  // capi.cu
}

namespace {

constexpr int64_t kNaMaxParts = 1 << 20;  // partial sums: 8 MiB of doubles
constexpr int kNaChunk = 4096;            // partials per reduction CTA
constexpr int kNaMaxChunks = (int)(kNaMaxParts / kNaChunk);
constexpr int kNaThreads = 256;
constexpr int kNaWarps = 8;
constexpr int kNaGroup = 8;               // lines per partial along the last axis (as the context kernels)

struct NaScratch {
  double part[kNaMaxParts];
  double lvl1[kNaMaxChunks];
  unsigned int ticket;
};

static __device__ __align__(256) NaScratch g_na_scratch;

// Device address of g_na_scratch per CUDA context.  A __device__ variable
// has one instance per context that loads the module, so the address belongs
// to the context, not to the device: a context made current through the
// driver API, or the primary context re-created after a reset, has its own.
// The cache is keyed by the context's unique ID (cuCtxGetId: never reused
// within a process, unlike a context handle).  The host symbol itself is only
// a stand-in and must never be handed to a kernel.
struct NaAddr {
  unsigned long long ctx_id;
  NaScratch* addr;
};
std::mutex g_na_mu;
std::vector<NaAddr> g_na_addr;
constexpr size_t kNaMaxContexts = 256;  // entries of contexts long gone are dropped beyond this

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// ID of the current context through driver entry points fetched by the
// runtime (the library does not link the driver library itself).  False when
// the driver offers no such call; the caller then looks the address up on
// every call.
bool current_context_id(unsigned long long* id) {
  static PfnCtxGetCurrent get_cur = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = (PfnCtxGetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (PfnCtxGetId)f;
    (void)cudaGetLastError();
  });
  if (!get_cur || !get_id) return false;
  CUcontext c = nullptr;
  if (get_cur(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

struct NaFaces {
  const double* f[6];
};

__device__ __forceinline__ double na_add(double a, double b) { return __dadd_rn(a, b); }

template <int DIM>
__global__ void __launch_bounds__(kNaThreads)
k_na_residual(const double* __restrict__ x, const double* __restrict__ f, NaFaces g, int nx, int ny, int nz,
              int segs, NaScratch* __restrict__ S) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kNaWarps + (threadIdx.x >> 5);
  // one warp per (group of kNaGroup lines along the last axis, [row y in 3D], segment)
  const int ext = DIM == 2 ? ny : nz;
  const int64_t ngroups = (ext + kNaGroup - 1) / kNaGroup;
  const int64_t nwarps = ngroups * (DIM == 3 ? ny : 1) * segs;
  if (w >= nwarps) return;
  const int seg = (int)(w % segs);
  const int64_t rest = w / segs;
  const int grp = DIM == 2 ? (int)rest : (int)(rest / ny);
  const int yfix = DIM == 2 ? 0 : (int)(rest % ny);
  const int xi = seg * 64 + 2 * lane;
  const bool v0 = xi < nx, v1 = xi + 1 < nx;
  auto X = [&](int64_t o) { return __ldg(x + o); };
  auto face = [&](int q, int64_t i) { return g.f[q] ? __ldg(g.f[q] + i) : 0.0; };
  double qacc = 0.0;
  const int m0 = grp * kNaGroup, m1 = min(m0 + kNaGroup, ext);
  for (int m = m0; m < m1; ++m) {
    const int y = DIM == 2 ? m : yfix, z = DIM == 2 ? 0 : m;
    const int64_t rb = ((int64_t)z * ny + y) * nx;  // dense offset of (0, y, z)
    if (!v0) continue;
    const double c0 = X(rb + xi);
    const double c1 = v1 ? X(rb + xi + 1) : 0.0;
    const double w0 = xi > 0 ? X(rb + xi - 1) : face(0, y + (int64_t)ny * z);
    const double e0 = v1 ? c1 : face(1, y + (int64_t)ny * z);
    const double w1 = c0;
    const double e1 = v1 ? (xi + 2 < nx ? X(rb + xi + 2) : face(1, y + (int64_t)ny * z)) : 0.0;
    auto ynb = [&](int dy, int k) {
      const int yy = y + dy;
      if (yy >= 0 && yy < ny) return X(rb + (int64_t)dy * nx + xi + k);
      return face(dy < 0 ? 2 : 3, xi + k + (int64_t)nx * z);
    };
    const double fv0 = f ? __ldg(f + rb + xi) : 0.0;
    const double fv1 = (f && v1) ? __ldg(f + rb + xi + 1) : 0.0;
    double t0, t1;
    if constexpr (DIM == 2) {
      t0 = na_add(na_add(na_add(w0, ynb(-1, 0)), na_add(e0, ynb(1, 0))), fv0);
      t1 = v1 ? na_add(na_add(na_add(w1, ynb(-1, 1)), na_add(e1, ynb(1, 1))), fv1) : 0.0;
    } else {
      const int64_t pl = (int64_t)nx * ny;
      auto znb = [&](int dz, int k) {
        const int zz = z + dz;
        if (zz >= 0 && zz < nz) return X(rb + (int64_t)dz * pl + xi + k);
        return face(dz < 0 ? 4 : 5, xi + k + (int64_t)nx * y);
      };
      t0 = na_add(na_add(na_add(na_add(w0, znb(-1, 0)), na_add(e0, znb(1, 0))), na_add(ynb(-1, 0), ynb(1, 0))), fv0);
      t1 = v1 ? na_add(na_add(na_add(na_add(w1, znb(-1, 1)), na_add(e1, znb(1, 1))), na_add(ynb(-1, 1), ynb(1, 1))),
                       fv1)
              : 0.0;
    }
    const double twod = DIM == 2 ? 4.0 : 6.0;
    const double r0 = __dsub_rn(t0, __dmul_rn(twod, c0));
    qacc = __fma_rn(r0, r0, qacc);
    if (v1) {
      const double r1 = __dsub_rn(t1, __dmul_rn(twod, c1));
      qacc = __fma_rn(r1, r1, qacc);
    }
  }
  double q = qacc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q = na_add(q, __shfl_xor_sync(0xffffffffu, q, o));
  if (lane == 0) S->part[w] = q;
}

// Two-level deterministic reduction of S->part[0, nparts) into *out; the last
// CTA to finish sums the first-level results and resets the ticket.
__global__ void __launch_bounds__(kNaThreads)
k_na_reduce(NaScratch* __restrict__ S, int64_t nparts, int nchunks, double* __restrict__ out) {
  __shared__ double sm[kNaThreads];
  __shared__ int is_last;
  const int t = threadIdx.x;
  const int64_t start = (int64_t)blockIdx.x * kNaChunk;
  const int len = (int)((nparts - start) < kNaChunk ? (nparts - start) : kNaChunk);
  double acc = 0.0;
  for (int i = t; i < len; i += kNaThreads) acc = na_add(acc, S->part[start + i]);
  sm[t] = acc;
  __syncthreads();
  for (int s = kNaThreads / 2; s > 0; s >>= 1) {
    if (t < s) sm[t] = na_add(sm[t], sm[t + s]);
    __syncthreads();
  }
  if (t == 0) {
    S->lvl1[blockIdx.x] = sm[0];
    __threadfence();
    const unsigned tk = atomicAdd(&S->ticket, 1u);
    is_last = tk == (unsigned)(nchunks - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  acc = 0.0;
  for (int i = t; i < nchunks; i += kNaThreads) acc = na_add(acc, __ldcg(S->lvl1 + i));
  sm[t] = acc;
  __syncthreads();
  for (int s = kNaThreads / 2; s > 0; s >>= 1) {
    if (t < s) sm[t] = na_add(sm[t], sm[t + s]);
    __syncthreads();
  }
  if (t == 0) {
    *out = sm[0];
    S->ticket = 0u;
  }
}

jacobi_status na_fail(jacobi_status st, const std::string& msg) {
  jgb::set_thread_error(msg);
  return st;
}

}  // namespace

extern "C" jacobi_status jacobi_residual_noalloc(int ndim, const int64_t dims[3], const double* x, const double* f,
                                                 const double* const faces[6], double* rss_out, void* cuda_stream) {
  if (ndim != 2 && ndim != 3) return na_fail(JACOBI_ERR_INVALID, "ndim must be 2 or 3");
  if (!dims || !x || !rss_out) return na_fail(JACOBI_ERR_INVALID, "dims, x and rss_out are required");
  const int64_t nx = dims[0], ny = dims[1], nz = ndim == 3 ? dims[2] : 1;
  if (nx < 1 || ny < 1 || nz < 1 || nx >= (1LL << 30) || ny >= (1LL << 30) || nz >= (1LL << 30))
    return na_fail(JACOBI_ERR_INVALID, "every dimension must be in [1, 2^30)");
  const int64_t segs = (nx + 63) / 64;
  const int64_t ext = ndim == 2 ? ny : nz;
  const int64_t groups = (ext + kNaGroup - 1) / kNaGroup;
  // the count of partials, each factor checked before it multiplies (in 3D
  // the plain product of three dimensions below 2^30 can pass 2^63)
  const std::string too_big =
      "grid too large for the fixed scratch: ceil(nx / 64) * ceil(n_last / 8) * (3D: ny) must be <= " +
      std::to_string(kNaMaxParts);
  if (segs > kNaMaxParts / groups) return na_fail(JACOBI_ERR_INVALID, too_big);
  int64_t nparts = segs * groups;
  if (ndim == 3) {
    if (nparts > kNaMaxParts / ny) return na_fail(JACOBI_ERR_INVALID, too_big);
    nparts *= ny;
  }
  if (nparts > kNaMaxParts) return na_fail(JACOBI_ERR_INVALID, too_big);
  cudaError_t e = cudaSuccess;
  NaScratch* S = nullptr;
  {
    // set-up once per CUDA context, with that context current: the device
    // address of the scratch array in this context
    std::lock_guard<std::mutex> lk(g_na_mu);
    unsigned long long id = 0;
    const bool keyed = current_context_id(&id);
    if (keyed)
      for (const NaAddr& a : g_na_addr)
        if (a.ctx_id == id) S = a.addr;
    if (!S) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess)
        return na_fail(JACOBI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      S = (NaScratch*)p;
      if (keyed) {
        if (g_na_addr.size() >= kNaMaxContexts) g_na_addr.clear();
        g_na_addr.push_back(NaAddr{id, S});
      }
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  NaFaces g;
  for (int q = 0; q < 6; ++q) g.f[q] = (faces && q < 2 * ndim) ? faces[q] : nullptr;
  // the ticket is shared by every call and must start at zero
  e = cudaMemsetAsync(&S->ticket, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return na_fail(JACOBI_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const int64_t nwarps = nparts;
  const unsigned grid1 = (unsigned)((nwarps + kNaWarps - 1) / kNaWarps);
  if (ndim == 2)
    k_na_residual<2><<<grid1, kNaThreads, 0, st>>>(x, f, g, (int)nx, (int)ny, (int)nz, (int)segs, S);
  else
    k_na_residual<3><<<grid1, kNaThreads, 0, st>>>(x, f, g, (int)nx, (int)ny, (int)nz, (int)segs, S);
  const int nchunks = (int)((nparts + kNaChunk - 1) / kNaChunk);
  k_na_reduce<<<nchunks, kNaThreads, 0, st>>>(S, nparts, nchunks, rss_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(JACOBI_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return JACOBI_OK;
}
