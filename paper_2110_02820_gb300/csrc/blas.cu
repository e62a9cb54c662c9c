// BLAS-like building blocks: a tiled SIMT GEMM (FP32 and FP64) with a
// deterministic split-K reduction, elementwise conversions, fixed-order sums
// of squares, the shift of Algorithm 1 (steps 4-5) and the Philox4x32-10 +
// Box-Muller Gaussian generator of step 1.

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace nys {

// ---------------------------------------------------------------- host utilities

static thread_local char g_last_err[512];

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_err, sizeof(g_last_err), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file,
           line);
}

static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void count_launches(long long k) {
  g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed);
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

static void raise_pool_threshold() {
  static bool done[64] = {false};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && !done[dev]) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
  }
}

int32_t dmalloc(void** p, size_t bytes, cudaStream_t s) {
  raise_pool_threshold();
  if (bytes == 0) bytes = 256;
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? NYS_ERR_OOM : NYS_ERR_CUDA;
  }
  return NYS_OK;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------- SIMT GEMM

// C_z = opA(A) * B over the K-range of split z, written to Cp + z * split_stride.
// Block tile BM x BN, K-slab BK, thread tile TM x TN; (BM/TM)*(BN/TN) threads.
template <typename T, typename TOut, bool TA, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(int64_t M, int64_t N, int64_t K, const T* __restrict__ A, int64_t lda,
            const T* __restrict__ B, int64_t ldb, TOut* __restrict__ Cp, int64_t ldc,
            int64_t kchunk, int64_t split_stride) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ T As[2][BK][BM + 4];
  __shared__ T Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  TOut* C = Cp + (int64_t)blockIdx.z * split_stride;

  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = T(0);

  constexpr int A_PER = (BM * BK + NT - 1) / NT;
  constexpr int B_PER = (BN * BK + NT - 1) / NT;
  T ra[A_PER], rb[B_PER];

  auto load_regs = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < A_PER; ++r) {
      int e = tid + r * NT;
      T v = T(0);
      if (e < BM * BK) {
        int i, k;
        if (TA) { k = e / BM; i = e % BM; } else { i = e / BK; k = e % BK; }
        int64_t gi = i0 + i, gk = k0 + k;
        if (gi < M && gk < kend) v = TA ? A[gk * lda + gi] : A[gi * lda + gk];
      }
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < B_PER; ++r) {
      int e = tid + r * NT;
      T v = T(0);
      if (e < BN * BK) {
        int k = e / BN, j = e % BN;
        int64_t gk = k0 + k, gj = j0 + j;
        if (gk < kend && gj < N) v = B[gk * ldb + gj];
      }
      rb[r] = v;
    }
  };
  auto store_regs = [&](int buf) {
#pragma unroll
    for (int r = 0; r < A_PER; ++r) {
      int e = tid + r * NT;
      if (e < BM * BK) {
        int i, k;
        if (TA) { k = e / BM; i = e % BM; } else { i = e / BK; k = e % BK; }
        As[buf][k][i] = ra[r];
      }
    }
#pragma unroll
    for (int r = 0; r < B_PER; ++r) {
      int e = tid + r * NT;
      if (e < BN * BK) {
        int k = e / BN, j = e % BN;
        Bs[buf][k][j] = rb[r];
      }
    }
  };

  int buf = 0;
  if (kbeg < kend) {
    load_regs(kbeg);
    store_regs(0);
  }
  __syncthreads();
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = (k0 + BK < kend);
    if (more) load_regs(k0 + BK);  // prefetch next slab into registers
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int t = 0; t < TM; ++t) a[t] = As[buf][kk][ty * TM + t];
#pragma unroll
      for (int t = 0; t < TN; ++t) b[t] = Bs[buf][kk][tx * TN + t];
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TN; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    if (more) store_regs(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int x = 0; x < TM; ++x) {
    int64_t gi = i0 + ty * TM + x;
    if (gi >= M) continue;
#pragma unroll
    for (int y = 0; y < TN; ++y) {
      int64_t gj = j0 + tx * TN + y;
      if (gj < N) C[gi * ldc + gj] = (TOut)acc[x][y];
    }
  }
}

// Out[i][j] = sum_z P[z][i][j] (fixed order), P dense M x N per split.
template <typename TAcc, typename TOut>
__global__ void split_reduce_kernel(const TAcc* __restrict__ P, int64_t splits, int64_t M,
                                    int64_t N, TOut* __restrict__ C, int64_t ldc) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  int64_t i = e / N, j = e % N;
  TAcc acc = 0;
  for (int64_t z = 0; z < splits; ++z) acc += P[z * M * N + e];
  C[i * ldc + j] = (TOut)acc;
}

template <typename T, typename TOut, int BM, int BN, int BK, int TM, int TN>
static int32_t gemm_launch(bool trans_a, int64_t M, int64_t N, int64_t K, const T* A, int64_t lda,
                           const T* B, int64_t ldb, TOut* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return NYS_OK;
  constexpr int NT = (BM / TM) * (BN / TN);
  int64_t tiles = cdiv(M, BM) * cdiv(N, BN);
  int64_t target = 2 * (int64_t)num_sms();
  int64_t splits = 1;
  if (tiles < target && K > 4 * BK) {
    splits = cdiv(target, tiles);
    // at least 256 K per split, 32 for FP64: an SM does ~2 FP64 FMA per
    // clock, so a small FP64 product (an ell x ell Gram of a tall block)
    // needs every SM, and the partial sums it adds are small
    constexpr int64_t kMinK = sizeof(T) == 8 ? 32 : 256;
    constexpr int64_t kMaxSplits = sizeof(T) == 8 ? 128 : 64;
    int64_t max_splits = cdiv(K, kMinK);
    if (splits > max_splits) splits = max_splits;
    if (splits > kMaxSplits) splits = kMaxSplits;
    if (splits < 1) splits = 1;
  }
  int64_t kchunk = cdiv(cdiv(K, splits), BK) * BK;
  splits = cdiv(K, kchunk);
  if (K == 0) { splits = 1; kchunk = 0; }
  dim3 grid((unsigned)cdiv(N, BN), (unsigned)cdiv(M, BM), (unsigned)splits);
  if (splits == 1) {
    if (trans_a)
      gemm_kernel<T, TOut, true, BM, BN, BK, TM, TN><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, C,
                                                                         ldc, kchunk > 0 ? kchunk : 1, 0);
    else
      gemm_kernel<T, TOut, false, BM, BN, BK, TM, TN><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb,
                                                                          C, ldc, kchunk > 0 ? kchunk : 1, 0);
    count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return NYS_OK;
  }
  T* P = nullptr;
  NYS_TRY(dmalloc((void**)&P, (size_t)splits * M * N * sizeof(T), s));
  if (trans_a)
    gemm_kernel<T, T, true, BM, BN, BK, TM, TN><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, P, N,
                                                                    kchunk, M * N);
  else
    gemm_kernel<T, T, false, BM, BN, BK, TM, TN><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, P, N,
                                                                     kchunk, M * N);
  count_launch();
  split_reduce_kernel<T, TOut><<<(unsigned)cdiv(M * N, 256), 256, 0, s>>>(P, splits, M, N, C, ldc); count_launch();
  cudaError_t e = cudaGetLastError();
  dfree(P, s);
  NYS_CUDA_TRY(e);
  return NYS_OK;
}

int32_t gemm_f32(bool ta, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                 const float* B, int64_t ldb, float* C, int64_t ldc, cudaStream_t s) {
  return gemm_launch<float, float, 128, 128, 8, 8, 8>(ta, M, N, K, A, lda, B, ldb, C, ldc, s);
}

int32_t gemm_f32_out64(bool ta, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                       const float* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  return gemm_launch<float, double, 128, 128, 8, 8, 8>(ta, M, N, K, A, lda, B, ldb, C, ldc, s);
}

int32_t gemm_f64(bool ta, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  return gemm_launch<double, double, 64, 64, 8, 4, 4>(ta, M, N, K, A, lda, B, ldb, C, ldc, s);
}

// ---------------------------------------------------------------- double-FP32 GEMM

// C = opA(A) B for FP64 matrices computed on the FP32 pipes in double-float
// arithmetic (Dekker 1971): each FP64 operand is split into an FP32 pair
// (hi, lo) as it is staged in shared memory; a term a b is the exact product
// hi_a hi_b (FMA two-product) plus hi_a lo_b + lo_a hi_b (lo_a lo_b, below
// 2^-48 |a b|, is dropped), and the terms are summed into a (hi, lo) pair
// with Knuth's TwoSum on the high parts.  Result within a few units of
// 2^-48 of sum |a| |b| (FP64 products would give 2^-53), at a fraction of
// the time of FP64 products on GB300.  sym: C is symmetric (A^T A-type
// products): only the tiles on or above the diagonal are computed, and
// the caller mirrors them.
constexpr int DG_BM = 64, DG_BN = 64, DG_BK = 8, DG_TM = 4, DG_TN = 4;
constexpr int DG_NT = (DG_BM / DG_TM) * (DG_BN / DG_TN);

__device__ __forceinline__ float2 dg_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

template <bool TA>
__global__ void __launch_bounds__(DG_NT)
gemm_dfl_kernel(int64_t M, int64_t N, int64_t K, const double* __restrict__ A, int64_t lda,
                const double* __restrict__ B, int64_t ldb, double* __restrict__ Cp, int64_t ldc,
                int64_t kchunk, int64_t split_stride, int sym) {
  const int64_t i0 = (int64_t)blockIdx.y * DG_BM, j0 = (int64_t)blockIdx.x * DG_BN;
  if (sym && i0 > j0 + DG_BN - 1) return;  // tile strictly below the diagonal
  __shared__ float2 As[DG_BK][DG_BM + 1];
  __shared__ float2 Bs[DG_BK][DG_BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % (DG_BN / DG_TN), ty = tid / (DG_BN / DG_TN);
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  double* C = Cp + (int64_t)blockIdx.z * split_stride;
  float sh[DG_TM][DG_TN], sl[DG_TM][DG_TN];
#pragma unroll
  for (int a = 0; a < DG_TM; ++a)
#pragma unroll
    for (int b = 0; b < DG_TN; ++b) sh[a][b] = sl[a][b] = 0.f;
  for (int64_t k0 = kbeg; k0 < kend; k0 += DG_BK) {
    __syncthreads();
    for (int e = tid; e < DG_BM * DG_BK; e += DG_NT) {
      int i, k;
      if (TA) { k = e / DG_BM; i = e % DG_BM; } else { i = e / DG_BK; k = e % DG_BK; }
      const int64_t gi = i0 + i, gk = k0 + k;
      double v = 0.0;
      if (gi < M && gk < kend) v = TA ? A[gk * lda + gi] : A[gi * lda + gk];
      As[k][i] = dg_split(v);
    }
    for (int e = tid; e < DG_BN * DG_BK; e += DG_NT) {
      const int k = e / DG_BN, j = e % DG_BN;
      const int64_t gk = k0 + k, gj = j0 + j;
      Bs[k][j] = dg_split((gk < kend && gj < N) ? B[gk * ldb + gj] : 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DG_BK; ++kk) {
      float2 a[DG_TM], b[DG_TN];
#pragma unroll
      for (int t = 0; t < DG_TM; ++t) a[t] = As[kk][ty * DG_TM + t];
#pragma unroll
      for (int t = 0; t < DG_TN; ++t) b[t] = Bs[kk][tx * DG_TN + t];
#pragma unroll
      for (int x = 0; x < DG_TM; ++x)
#pragma unroll
        for (int y = 0; y < DG_TN; ++y) {
          const float p = __fmul_rn(a[x].x, b[y].x);
          float e = __fmaf_rn(a[x].x, b[y].x, -p);
          e = __fmaf_rn(a[x].x, b[y].y, e);
          e = __fmaf_rn(a[x].y, b[y].x, e);
          const float s0 = __fadd_rn(sh[x][y], p);
          const float bb = __fsub_rn(s0, sh[x][y]);
          const float err = __fadd_rn(__fsub_rn(sh[x][y], __fsub_rn(s0, bb)), __fsub_rn(p, bb));
          sl[x][y] = __fadd_rn(sl[x][y], __fadd_rn(err, e));
          sh[x][y] = s0;
        }
    }
  }
#pragma unroll
  for (int x = 0; x < DG_TM; ++x) {
    const int64_t gi = i0 + ty * DG_TM + x;
    if (gi >= M) continue;
#pragma unroll
    for (int y = 0; y < DG_TN; ++y) {
      const int64_t gj = j0 + tx * DG_TN + y;
      if (gj < N) C[gi * ldc + gj] = (double)sh[x][y] + (double)sl[x][y];
    }
  }
}

// C[j][i] = C[i][j] for i < j (upper triangle mirrored down)
__global__ void mirror_upper_kernel(double* C, int64_t n, int64_t ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int64_t i = e / n, j = e - i * n;
  if (j < i) C[i * ldc + j] = C[j * ldc + i];
}

int32_t gemm_dfl(bool ta, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double* C, int64_t ldc, bool sym,
                 cudaStream_t s) {
  if (M <= 0 || N <= 0) return NYS_OK;
  if (sym && M != N) return NYS_ERR_ARG;
  const int64_t tiles = cdiv(M, DG_BM) * cdiv(N, DG_BN);
  const int64_t target = 2 * (int64_t)num_sms();
  int64_t splits = 1;
  if (tiles < target && K > 16 * DG_BK) {
    splits = std::min<int64_t>(cdiv(target, tiles), std::max<int64_t>(1, K / 64));
    splits = std::min<int64_t>(splits, 32);
  }
  int64_t kchunk = cdiv(cdiv(K, splits), DG_BK) * DG_BK;
  if (kchunk < 1) kchunk = DG_BK;
  splits = K > 0 ? cdiv(K, kchunk) : 1;
  const dim3 grid((unsigned)cdiv(N, DG_BN), (unsigned)cdiv(M, DG_BM), (unsigned)splits);
  double* P = C;
  int64_t ldp = ldc;
  Scratch sc(s);
  if (splits > 1) {
    NYS_TRY(sc.get(&P, (size_t)splits * M * N));
    ldp = N;
  }
  if (ta)
    gemm_dfl_kernel<true><<<grid, DG_NT, 0, s>>>(M, N, K, A, lda, B, ldb, P, ldp, kchunk,
                                                 splits > 1 ? M * N : 0, sym ? 1 : 0);
  else
    gemm_dfl_kernel<false><<<grid, DG_NT, 0, s>>>(M, N, K, A, lda, B, ldb, P, ldp, kchunk,
                                                  splits > 1 ? M * N : 0, sym ? 1 : 0);
  count_launch();
  if (splits > 1) {
    split_reduce_kernel<double, double><<<(unsigned)cdiv(M * N, 256), 256, 0, s>>>(
        P, splits, M, N, C, ldc);
    count_launch();
  }
  if (sym) {
    mirror_upper_kernel<<<(unsigned)cdiv(M * N, 256), 256, 0, s>>>(C, M, ldc);
    count_launch();
  }
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// ---------------------------------------------------------------- elementwise

template <typename A, typename B>
__global__ void convert_kernel(const A* in, B* out, int64_t count) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += stride)
    out[e] = (B)in[e];
}

static unsigned grid_for(int64_t count, int threads = 256) {
  int64_t b = cdiv(count, threads);
  int64_t cap = 8LL * num_sms();
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

int32_t convert_f64_to_f32(const double* in, float* out, int64_t count, cudaStream_t s) {
  convert_kernel<double, float><<<grid_for(count), 256, 0, s>>>(in, out, count); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

int32_t convert_f32_to_f64(const float* in, double* out, int64_t count, cudaStream_t s) {
  convert_kernel<float, double><<<grid_for(count), 256, 0, s>>>(in, out, count); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

__global__ void add_inplace_kernel(double* y, const double* x, int64_t count) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += stride)
    y[e] += x[e];
}

int32_t add_inplace_f64(double* y, const double* x, int64_t count, cudaStream_t s) {
  add_inplace_kernel<<<grid_for(count), 256, 0, s>>>(y, x, count); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// Fixed-order sum of squares: per-block partials, the last block sums them.
template <typename T>
__global__ void sumsq_kernel(const T* __restrict__ x, int64_t count, double* partial,
                             unsigned int* counter, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += stride) {
    double v = (double)x[e];
    acc += v * v;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  if (last_block_arrived(counter)) {
    double t = 0.0;
    if (threadIdx.x == 0) {
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(partial + b);
      *out = t;
    }
  }
}

template <typename T>
static int32_t sumsq_impl(const T* x, int64_t count, double* d_out, cudaStream_t s) {
  unsigned blocks = grid_for(count);
  unsigned char* aux = nullptr;
  NYS_TRY(dmalloc((void**)&aux, blocks * sizeof(double) + 16, s));
  double* partial = reinterpret_cast<double*>(aux + 16);
  unsigned int* counter = reinterpret_cast<unsigned int*>(aux);
  cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  sumsq_kernel<T><<<blocks, 256, 0, s>>>(x, count, partial, counter, d_out); count_launch();
  cudaError_t e = cudaGetLastError();
  dfree(aux, s);
  NYS_CUDA_TRY(e);
  return NYS_OK;
}

int32_t sumsq_f32(const float* x, int64_t count, double* d_out, cudaStream_t s) {
  return sumsq_impl(x, count, d_out, s);
}
int32_t sumsq_f64(const double* x, int64_t count, double* d_out, cudaStream_t s) {
  return sumsq_impl(x, count, d_out, s);
}

template <typename T>
__global__ void shift_add_kernel(const T* Y, const T* Q, T* Ynu, int64_t count, const double* d_nu,
                                 double factor) {
  const T nu = (T)(d_nu[0] * factor);
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += stride)
    Ynu[e] = Y[e] + nu * Q[e];
}

int32_t shift_add_f32(const float* Y, const float* Q, float* Ynu, int64_t count, const double* d_nu,
                      double factor, cudaStream_t s) {
  shift_add_kernel<float><<<grid_for(count), 256, 0, s>>>(Y, Q, Ynu, count, d_nu, factor); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}
int32_t shift_add_f64(const double* Y, const double* Q, double* Ynu, int64_t count,
                      const double* d_nu, double factor, cudaStream_t s) {
  shift_add_kernel<double><<<grid_for(count), 256, 0, s>>>(Y, Q, Ynu, count, d_nu, factor); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// eps(x) in MATLAB's sense at the given mantissa width: the spacing of
// floating-point numbers at |x|, 2^(floor(log2|x|) - p).
__global__ void compute_nu_kernel(const double* sumsq, double scale, int mantissa_bits,
                                  double* nu) {
  double x = sqrt(sumsq[0]);
  double pre = 1.0;
  if (x > 0.0 && isfinite(x)) {
    int e2;
    frexp(x, &e2);  // x = f 2^e2, f in [0.5, 1)
    pre = ldexp(1.0, (e2 - 1) - mantissa_bits);
  } else {
    pre = ldexp(1.0, -1074);
  }
  nu[0] = scale * pre;
}

int32_t compute_nu(const double* d_sumsq, double scale, int mantissa_bits, double* d_nu,
                   cudaStream_t s) {
  compute_nu_kernel<<<1, 1, 0, s>>>(d_sumsq, scale, mantissa_bits, d_nu); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

__global__ void lambda_kernel(const double* sigma, const double* d_nu, double* lam, int64_t ell) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ell) return;
  double v = sigma[j] * sigma[j] - d_nu[0];
  lam[j] = v > 0.0 ? v : 0.0;
}

int32_t lambda_from_sigma(const double* sigma, const double* d_nu, double* lam, int64_t ell,
                          cudaStream_t s) {
  lambda_kernel<<<(unsigned)cdiv(ell, 256), 256, 0, s>>>(sigma, d_nu, lam, ell); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// ---------------------------------------------------------------- Philox4x32-10

// Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds
// of the Philox S-box on a 128-bit counter under a 64-bit key, the key bumped
// by the Weyl constants between rounds.
struct Philox4 {
  uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(Philox4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c.v[0]), lo0 = M0 * c.v[0];
    uint32_t hi1 = __umulhi(M1, c.v[2]), lo1 = M1 * c.v[2];
    Philox4 n;
    n.v[0] = hi1 ^ c.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ c.v[3] ^ k1;
    n.v[3] = lo0;
    c = n;
    k0 += W0;
    k1 += W1;
  }
  return c;
}

// Element e of stream (seed, stream_id) is word e mod 4 of the block of
// counter (g, (g >> 32) ^ stream lo, stream hi, 0x6e79), g = e / 4, under key
// (seed lo, seed hi).  Uniforms u = ((w >> 9) + 1/2) 2^-23 take 23 bits of a
// word, so they are exact in FP32 (and equal to the FP64 value); Box-Muller
// pairs elements (0, 1) and (2, 3) of a block: sqrt(-2 ln u_even) times
// cos (even element) and sin (odd element) of 2 pi u_odd, the angle through
// sincospif so that 2 u is exact.  Elements [first, first + count) go to
// words[e - first] and gauss[e - first] (either may be NULL).
__global__ void philox_stream_kernel(uint32_t* words, double* gauss, int64_t first, int64_t count,
                                     uint64_t seed, uint64_t stream_id) {
  const int64_t g0 = first / 4, g1 = (first + count - 1) / 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = g0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= g1; g += stride) {
    Philox4 c;
    c.v[0] = (uint32_t)g;
    c.v[1] = (uint32_t)((uint64_t)g >> 32) ^ (uint32_t)stream_id;
    c.v[2] = (uint32_t)(stream_id >> 32);
    c.v[3] = 0x6e79u;  // fixed tag
    const Philox4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    float z[4];
    if (gauss) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float u1 = ((float)(r.v[2 * h] >> 9) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
        const float u2 = ((float)(r.v[2 * h + 1] >> 9) + 0.5f) * 1.1920928955078125e-07f;
        const float rad = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        z[2 * h] = rad * cs;
        z[2 * h + 1] = rad * sn;
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t e = g * 4 + t;
      if (e < first || e >= first + count) continue;
      if (words) words[e - first] = r.v[t];
      if (gauss) gauss[e - first] = (double)z[t];
    }
  }
}

int32_t philox_stream(uint32_t* words, double* gauss, int64_t first, int64_t count, uint64_t seed,
                      uint64_t stream_id, cudaStream_t s) {
  if (count <= 0) return NYS_OK;
  const int64_t blocks = (first + count - 1) / 4 - first / 4 + 1;
  philox_stream_kernel<<<grid_for(blocks), 256, 0, s>>>(words, gauss, first, count, seed,
                                                        stream_id);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

int32_t philox_gaussian_f64(double* out, int64_t count, uint64_t seed, uint64_t stream_id,
                            cudaStream_t s) {
  return philox_stream(nullptr, out, 0, count, seed, stream_id, s);
}

// The bare bijection on caller-given counters and keys (known-answer checks).
__global__ void philox_blocks_kernel(const uint32_t* __restrict__ ctr,
                                     const uint32_t* __restrict__ key, int64_t count,
                                     uint32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  Philox4 c;
#pragma unroll
  for (int t = 0; t < 4; ++t) c.v[t] = ctr[4 * i + t];
  const Philox4 r = philox4x32_10(c, key[2 * i], key[2 * i + 1]);
#pragma unroll
  for (int t = 0; t < 4; ++t) out[4 * i + t] = r.v[t];
}

int32_t philox_blocks(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out,
                      cudaStream_t s) {
  if (count <= 0) return NYS_OK;
  philox_blocks_kernel<<<(unsigned)cdiv(count, 256), 256, 0, s>>>(ctr, key, count, out);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

}  // namespace nys

namespace nys {

int32_t split_reduce_f32(const float* P, int64_t splits, int64_t M, int64_t N, float* D,
                         int64_t ldd, cudaStream_t s) {
  split_reduce_kernel<float, float><<<(unsigned)cdiv(M * N, 256), 256, 0, s>>>(P, splits, M, N, D,
                                                                               ldd); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// out[j * ld_out + i] = in[i * ld_in + j] for a rows x cols array: 32 x 32
// tiles through shared memory (coalesced reads and writes).
__global__ void transpose_f32_kernel(const float* __restrict__ in, int64_t rows, int64_t cols,
                                     int64_t ld_in, float* __restrict__ out, int64_t ld_out) {
  __shared__ float tile[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    int64_t i = by + r, j = bx + threadIdx.x;
    if (i < rows && j < cols) tile[r][threadIdx.x] = in[i * ld_in + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    int64_t j = bx + r, i = by + threadIdx.x;
    if (i < rows && j < cols) out[j * ld_out + i] = tile[threadIdx.x][r];
  }
}

// 64 x 64 tiles with 16-byte global accesses on both sides (rows, cols and
// ld_in multiples of 4, 16-byte aligned bases): 256 threads, each moving four
// float4 in and four out through a padded shared tile.
__global__ void __launch_bounds__(256)
transpose_f32_v4_kernel(const float* __restrict__ in, int64_t rows, int64_t cols, int64_t ld_in,
                        float* __restrict__ out, int64_t ld_out) {
  __shared__ float tile[64][65];
  const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
  const int t4 = threadIdx.x & 15, tr = threadIdx.x >> 4;  // 16 float4 per row, 16 rows per pass
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int r = tr + 16 * p;
    const int64_t i = r0 + r, j = c0 + 4 * t4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < rows && j < cols) v = *reinterpret_cast<const float4*>(in + i * ld_in + j);
    tile[r][4 * t4 + 0] = v.x;
    tile[r][4 * t4 + 1] = v.y;
    tile[r][4 * t4 + 2] = v.z;
    tile[r][4 * t4 + 3] = v.w;
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int c = tr + 16 * p;                 // output row = input column
    const int64_t j = c0 + c, i = r0 + 4 * t4;
    if (j < cols && i < rows) {
      const float4 v = make_float4(tile[4 * t4 + 0][c], tile[4 * t4 + 1][c], tile[4 * t4 + 2][c],
                                   tile[4 * t4 + 3][c]);
      *reinterpret_cast<float4*>(out + j * ld_out + i) = v;
    }
  }
}

int32_t transpose_f32(const float* in, int64_t rows, int64_t cols, int64_t ld_in, float* out,
                      cudaStream_t s) {
  const bool v4 = (rows % 4 == 0) && (cols % 4 == 0) && (ld_in % 4 == 0) &&
                  (((uintptr_t)in & 15u) == 0) && (((uintptr_t)out & 15u) == 0);
  // rows are processed in bands so that grid.y stays below 65536
  const int64_t tile = v4 ? 64 : 32;
  const int64_t band = 32768ll * tile;
  for (int64_t r0 = 0; r0 < rows; r0 += band) {
    int64_t rb = (rows - r0 < band) ? rows - r0 : band;
    dim3 g((unsigned)cdiv(cols, tile), (unsigned)cdiv(rb, tile));
    if (v4)
      transpose_f32_v4_kernel<<<g, 256, 0, s>>>(in + r0 * ld_in, rb, cols, ld_in, out + r0, rows);
    else
      transpose_f32_kernel<<<g, dim3(32, 8), 0, s>>>(in + r0 * ld_in, rb, cols, ld_in, out + r0,
                                                     rows);
    count_launch();
  }
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

}  // namespace nys
