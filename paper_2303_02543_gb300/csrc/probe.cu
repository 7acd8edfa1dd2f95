// Measurement helper: the issue rate of the FP64 pipe on the current device.
//
// The plain FP64 Jacobi sweep is bound by its FP64 additions on GB300, not by
// HBM (the FP64 pipe runs at a small fraction of the FP32 rate), so its
// roofline is the FP64 pipe's measured throughput.  Every FP64 addition of
// the sweep kernels is issued as fma.rn.f64 d, a, 1.0, b; this probe times
// that same instruction form in `chains` independent dependency chains per
// thread, with `ctas_per_sm` CTAs of 256 threads resident per SM.  With
// enough independent chains the rate is the pipe's throughput; with one chain
// it shows the dependent-issue latency that the sweeps must hide.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "../../include/jacobi.h"

namespace jgb {
void set_thread_error(const std::string& msg);  // capi.cu
}

namespace {

constexpr int kProbeThreads = 256;

// Sink for the chains' results (never read by the host: it only keeps the
// arithmetic from being removed).
__device__ double g_probe_sink;

template <int CH>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma_rate(int iters, double seed) {
  double a[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) a[c] = seed * (double)(threadIdx.x + 1 + c);
  const double b = seed * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int c = 0; c < CH; ++c)
        asm volatile("fma.rn.f64 %0, %0, 0d3FF0000000000000, %1;" : "+d"(a[c]) : "d"(b));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += a[c];
  if (s == 12345.678) g_probe_sink = s;  // practically never true
}

template <int CH>
cudaError_t run(int iters, int ctas, cudaStream_t st) {
  k_fp64_fma_rate<CH><<<ctas, kProbeThreads, 0, st>>>(iters, 1e-300);
  return cudaGetLastError();
}

jacobi_status fail(jacobi_status s, const std::string& msg) {
  jgb::set_thread_error(msg);
  return s;
}

}  // namespace

extern "C" jacobi_status jacobi_probe_fp64_rate(int chains, int ctas_per_sm, int64_t iters, double* lane_ops_per_s,
                                                void* cuda_stream) {
  if (!lane_ops_per_s) return fail(JACOBI_ERR_INVALID, "lane_ops_per_s is NULL");
  if (chains != 1 && chains != 2 && chains != 4 && chains != 8)
    return fail(JACOBI_ERR_INVALID, "chains must be 1, 2, 4 or 8");
  if (ctas_per_sm < 1 || ctas_per_sm > 8) return fail(JACOBI_ERR_INVALID, "ctas_per_sm must be in [1, 8]");
  if (iters < 1 || iters > (1 << 24)) return fail(JACOBI_ERR_INVALID, "iters must be in [1, 2^24]");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(JACOBI_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
  const int ctas = sms * ctas_per_sm;
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return fail(JACOBI_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
  }
  auto launch = [&](int it) {
    switch (chains) {
      case 1: return run<1>(it, ctas, st);
      case 2: return run<2>(it, ctas, st);
      case 4: return run<4>(it, ctas, st);
      default: return run<8>(it, ctas, st);
    }
  };
  float ms = 0.f;
  e = launch((int)std::min<int64_t>(iters, 64));  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) e = launch((int)iters);
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return fail(JACOBI_ERR_CUDA, std::string("probe: ") + cudaGetErrorString(e));
  const double ops = (double)ctas * kProbeThreads * chains * 8.0 * (double)iters;
  *lane_ops_per_s = ms > 0.f ? ops / (ms * 1e-3) : 0.0;
  return JACOBI_OK;
}
