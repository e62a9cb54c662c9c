// Shared device/host utilities of the Nystrom PCG library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/nyspcg.h"

namespace nys {

constexpr int kWarp = 32;

// ---------------------------------------------------------------- host checks

#define NYS_CUDA_TRY(expr)                                                  \
  do {                                                                      \
    cudaError_t _e = (expr);                                                \
    if (_e != cudaSuccess) {                                                \
      nys::set_last_cuda_error(_e, #expr, __FILE__, __LINE__);              \
      return (_e == cudaErrorMemoryAllocation) ? NYS_ERR_OOM : NYS_ERR_CUDA; \
    }                                                                       \
  } while (0)

#define NYS_TRY(expr)                 \
  do {                                \
    int32_t _s = (expr);              \
    if (_s != NYS_OK) return _s;      \
  } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Number of SMs of the current device (cached per device).
int num_sms();

// Process-wide count of kernel launches made by this library (every launch
// site calls this right after its launch).
void count_launch();

// ---------------------------------------------------------------- device helpers

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum in a fixed order (warp tree, then warp 0 over the warp
// partials).  `red` must hold blockDim.x/32 elements.  Result valid in all threads.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}

// "Last block" election for two-phase deterministic reductions: every block
// of a group (by default the blocks along x) writes its partials, then calls
// this; exactly one block (the last to arrive) gets true and may read all
// partials.  The counter is reset by the elected block so the kernel can be
// relaunched (also inside a CUDA graph).
__device__ __forceinline__ bool last_block_arrived(unsigned int* counter,
                                                   unsigned int expected = 0) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    unsigned int total = expected ? expected : gridDim.x;
    is_last = (prev == total - 1);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return is_last;
}

template <typename T>
struct TypeName;

// Bounded grid barrier for a cooperative launch.  Returns false (and sets
// *status = NYS_ERR_TIMEOUT) if the wait did not end within the spin limit
// or another block already failed; the caller then returns.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, unsigned int* gen, int* status) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = gen;
    volatile int* vstat = status;
    unsigned int g = *vgen;
    __threadfence();
    unsigned int nb = gridDim.x;
    if (atomicAdd(count, 1u) == nb - 1) {
      *count = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (*vstat != 0) { ok = 0; break; }
        if (++spins > (1ll << 26)) {  // ~ seconds: far beyond any legal wait
          atomicCAS(status, 0, (int)NYS_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace nys
