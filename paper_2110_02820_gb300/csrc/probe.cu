// Measured throughput of the execution units that bound the library's
// ALU-limited kernels (no counterpart in the paper): the FP64 FMA pipe (the
// dense FP64 matvec), the FP32 FMA pipe (the double-FP32 residual products)
// and the MUFU ex2 unit (one exponential per Gaussian kernel entry).  Each
// kernel runs independent dependency chains in registers on every SM, long
// enough that launch overhead is negligible, and is timed with CUDA events on
// the caller's stream after one untimed launch.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace nys {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) fma64_probe_kernel(double* sink, int iters, double a,
                                                                 double b) {
  double x[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) x[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += x[k];
  if (s == -1.0) sink[0] = s;  // never true: keeps the chains live
}

__global__ void __launch_bounds__(PK_THREADS) fma32_probe_kernel(float* sink, int iters, float a,
                                                                 float b) {
  float x[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) x[k] = 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += x[k];
  if (s == -1.f) sink[0] = s;
}

// x <- 2^(-x) stays in (1/2, 1): one MUFU op (and one FP32 negation) per step
__global__ void __launch_bounds__(PK_THREADS) ex2_probe_kernel(float* sink, int iters) {
  float x[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) x[k] = 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[k]));
      x[k] = y;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += x[k];
  if (s == -1.f) sink[0] = s;
}

}  // namespace nys

using namespace nys;

extern "C" int32_t nys_unit_peak(int32_t unit, double* ops_per_s, void* stream) {
  if (!ops_per_s || unit < 0 || unit > 2) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double* sink;
  NYS_TRY(sc.get(&sink, 1));
  // blocks: 8 per SM (2048 threads, full occupancy at <= 32 registers)
  const int blocks = 8 * num_sms();
  const int iters = unit == 0 ? 1 << 14 : unit == 1 ? 1 << 17 : 1 << 15;
  cudaEvent_t e0, e1;
  NYS_CUDA_TRY(cudaEventCreate(&e0));
  NYS_CUDA_TRY(cudaEventCreate(&e1));
  auto launch = [&]() {
    if (unit == 0)
      fma64_probe_kernel<<<blocks, PK_THREADS, 0, s>>>(sink, iters, 0.999999, 1e-7);
    else if (unit == 1)
      fma32_probe_kernel<<<blocks, PK_THREADS, 0, s>>>((float*)sink, iters, 0.9999f, 1e-4f);
    else
      ex2_probe_kernel<<<blocks, PK_THREADS, 0, s>>>((float*)sink, iters);
    count_launch();
  };
  launch();  // untimed
  NYS_CUDA_TRY(cudaEventRecord(e0, s));
  launch();
  NYS_CUDA_TRY(cudaEventRecord(e1, s));
  NYS_CUDA_TRY(cudaGetLastError());
  NYS_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  NYS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double ops = (double)blocks * PK_THREADS * PK_CHAINS * (double)iters *
                     (unit == 2 ? 1.0 : 2.0);  // FMA = 2 FLOP
  *ops_per_s = ops / (ms * 1e-3);
  return NYS_OK;
}
