// Measurement helper: the issue rate of the FP64 pipe on the current device.
//
// The plain FP64 Jacobi sweep is bound by its FP64 additions on GB300, not by
// HBM (the FP64 pipe runs at a small fraction of the FP32 rate), so its
// roofline is the FP64 pipe's measured throughput.  Every FP64 addition of
// the sweep kernels is issued as fma.rn.f64 d, a, one, b with `one` = 1.0 in
// a register (form 1 below, the fastest form on GB300); this probe times that
// instruction form and the others in `chains` independent dependency chains
// per thread, with `ctas_per_sm` CTAs of 256 threads resident per SM.  With
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
// arithmetic from being removed) and the multiplier 1.0 read at run time (so
// the compiler cannot see its value and fold it into an immediate).
__device__ double g_probe_sink;
__device__ double g_probe_one = 1.0;
__constant__ double c_probe_one = 1.0;

// FORM 0: fma.rn.f64 with the immediate multiplier 1.0; 1: fma.rn.f64 with
// the multiplier 1.0 in a register; 2: add.f64; 3: mul.f64 by a register;
// 4: fma.rn.f64 with the multiplier 1.0 read from constant memory; 5 and 6:
// form 1 with 2 or 4 independent 32-bit integer additions after each FMA (to
// see whether integer work competes with the FP64 pipe).
template <int CH, int FORM>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_rate(int iters, double seed) {
  double a[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) a[c] = seed * (double)(threadIdx.x + 1 + c);
  const double b = seed * 1e-3;
  const double one = __ldg(&g_probe_one);
  uint32_t ic[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) ic[c] = threadIdx.x + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        if constexpr (FORM == 0)
          asm volatile("fma.rn.f64 %0, %0, 0d3FF0000000000000, %1;" : "+d"(a[c]) : "d"(b));
        else if constexpr (FORM == 1)
          asm volatile("fma.rn.f64 %0, %0, %2, %1;" : "+d"(a[c]) : "d"(b), "d"(one));
        else if constexpr (FORM == 5 || FORM == 6) {
          asm volatile("fma.rn.f64 %0, %0, %2, %1;" : "+d"(a[c]) : "d"(b), "d"(one));
#pragma unroll
          for (int q = 0; q < (FORM == 5 ? 2 : 4); ++q)
            asm volatile("add.u32 %0, %0, %1;" : "+r"(ic[c]) : "r"(q + 1));
        } else if constexpr (FORM == 4)
          asm volatile("fma.rn.f64 %0, %0, %2, %1;" : "+d"(a[c]) : "d"(b), "d"(c_probe_one));
        else if constexpr (FORM == 2)
          asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(a[c]) : "d"(b));
        else
          asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(a[c]) : "d"(one));
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += a[c];
  uint32_t is = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) is += ic[c];
  if (s == 12345.678 || is == 0xFFFFFFFFu) g_probe_sink = s;  // practically never true
}

template <int CH>
cudaError_t run(int form, int iters, int ctas, cudaStream_t st) {
  switch (form) {
    case 0: k_fp64_rate<CH, 0><<<ctas, kProbeThreads, 0, st>>>(iters, 1e-300); break;
    case 1: k_fp64_rate<CH, 1><<<ctas, kProbeThreads, 0, st>>>(iters, 1e-300); break;
    case 2: k_fp64_rate<CH, 2><<<ctas, kProbeThreads, 0, st>>>(iters, 1e-300); break;
    case 4: k_fp64_rate<CH, 4><<<ctas, kProbeThreads, 0, st>>>(iters, 1e-300); break;
    case 5: k_fp64_rate<CH, 5><<<ctas, kProbeThreads, 0, st>>>(iters, 1e-300); break;
    case 6: k_fp64_rate<CH, 6><<<ctas, kProbeThreads, 0, st>>>(iters, 1e-300); break;
    default: k_fp64_rate<CH, 3><<<ctas, kProbeThreads, 0, st>>>(iters, 1e-300); break;
  }
  return cudaGetLastError();
}

jacobi_status fail(jacobi_status s, const std::string& msg) {
  jgb::set_thread_error(msg);
  return s;
}

}  // namespace

extern "C" jacobi_status jacobi_probe_fp64_rate(int form, int chains, int ctas_per_sm, int64_t iters,
                                                double* lane_ops_per_s, void* cuda_stream) {
  if (!lane_ops_per_s) return fail(JACOBI_ERR_INVALID, "lane_ops_per_s is NULL");
  if (form < 0 || form > 6) return fail(JACOBI_ERR_INVALID, "form must be in [0, 6]");
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
      case 1: return run<1>(form, it, ctas, st);
      case 2: return run<2>(form, it, ctas, st);
      case 4: return run<4>(form, it, ctas, st);
      default: return run<8>(form, it, ctas, st);
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
