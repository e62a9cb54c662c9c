// Operator kernels: x -> A x for the three operators (Sec. 1.1 accesses A
// only through matvecs) and the sketch Y = A Omega of Algorithm 1, step 3.
//
//  dense : A n x n FP64.  Warp per row, FP64 FMA.
//  gram  : A = X^T X, X m x n FP32 (ridge, Eq. (1.7)).  One pass over X:
//          each CTA streams its rows through shared memory with bulk async
//          copies (TMA engine) into a 3-stage mbarrier pipeline, forms
//          t_i = x_i . p with a CTA-wide reduction and accumulates t_i x_i
//          into a per-CTA n-vector held in registers; a second kernel sums
//          the per-CTA partials in a fixed order.  X is read from HBM once.
//  rbf   : A = K, K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2)) (Sec. 6.5),
//          computed on the fly tile by tile and never stored.

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace nys {

// ============================================================ dense

// One warp per row; blocks of DM_WARPS rows so that every block of a 2048-row
// matrix is resident at once (no tail wave).  Eight 16-byte loads and eight
// independent accumulators per step keep the L2 loads in flight; the FP64
// FMA rate of the part, not bandwidth, is the bound (A is L2-resident).
constexpr int DM_WARPS = 4;
template <typename P, typename V>
__global__ void __launch_bounds__(32 * DM_WARPS)
dense_matvec_kernel(const double* __restrict__ A, int64_t n, int64_t ld,
                    const P* __restrict__ p, double mu, V* __restrict__ v,
                    const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * DM_WARPS + (threadIdx.x >> 5);
  if (row >= n) return;
  const double* a = A + row * ld;
  double acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.0;
  int64_t j0 = 0;
  if (((ld & 1) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0)) {
    const double2* a2 = reinterpret_cast<const double2*>(a);
    const int64_t n2 = n >> 1;
    int64_t c = lane;
    for (; c + 7 * 32 < n2; c += 8 * 32) {
      double2 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = a2[c + 32 * u];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t j = 2 * (c + 32 * u);
        acc[u] = fma(x[u].x, (double)p[j], fma(x[u].y, (double)p[j + 1], acc[u]));
      }
    }
    for (; c < n2; c += 32) {
      const double2 x0 = a2[c];
      acc[0] = fma(x0.x, (double)p[2 * c], fma(x0.y, (double)p[2 * c + 1], acc[0]));
    }
    j0 = n2 << 1;
  }
  for (int64_t j = j0 + lane; j < n; j += 32) acc[0] = fma(a[j], (double)p[j], acc[0]);
  double t = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  t = warp_sum(t);
  if (lane == 0) v[row] = (V)(t + mu * (double)p[row]);
}

// ============================================================ gram (fused single pass)

constexpr int GR_THREADS = 256;
constexpr int GR_ROWS = 4;  // rows per pipeline stage

// part[blockIdx.x][0..n) = sum over this CTA's rows i of (x_i . p) x_i.
// NG = float4 column groups per thread (n <= NG * 4 * 256).
template <typename P, typename Acc, int NG>
__global__ void __launch_bounds__(GR_THREADS, 1)
gram_fused_kernel(const float* __restrict__ X, int64_t m, int64_t n, const P* __restrict__ p,
                  Acc* __restrict__ part, int stages, int64_t rows_per_cta, int* err,
                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  float* stage_mem = reinterpret_cast<float*>(smem + 128);
  __shared__ Acc red[GR_THREADS / 32][GR_ROWS];
  __shared__ int s_fail;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n4 = n >> 2;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = (r0 + rows_per_cta < m) ? r0 + rows_per_cta : m;
  Acc* out = part + (int64_t)blockIdx.x * n;

  Acc pr[NG][4], acc[NG][4];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    int64_t c4 = tid + (int64_t)g * GR_THREADS;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      pr[g][q] = (c4 < n4) ? (Acc)p[4 * c4 + q] : Acc(0);
      acc[g][q] = Acc(0);
    }
  }
  if (r0 >= r1) {
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      int64_t c4 = tid + (int64_t)g * GR_THREADS;
      if (c4 < n4)
#pragma unroll
        for (int q = 0; q < 4; ++q) out[4 * c4 + q] = Acc(0);
    }
    return;
  }
  const int64_t nrows = r1 - r0;
  const int64_t nchunks = (nrows + GR_ROWS - 1) / GR_ROWS;
  const int64_t stage_elems = (int64_t)GR_ROWS * n;

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    s_fail = 0;
  }
  __syncthreads();

  auto issue = [&](int64_t c) {
    int s = (int)(c % stages);
    int64_t rows = nrows - c * GR_ROWS;
    if (rows > GR_ROWS) rows = GR_ROWS;
    uint32_t bytes = (uint32_t)(rows * n * sizeof(float));
    mbar_arrive_expect_tx(&bars[s], bytes);
    bulk_g2s(stage_mem + s * stage_elems, X + (r0 + c * GR_ROWS) * n, bytes, &bars[s]);
  };
  if (tid == 0) {
    int64_t pre = (stages - 1 < nchunks) ? stages - 1 : nchunks;
    for (int64_t c = 0; c < pre; ++c) issue(c);
  }

  int64_t issued = (stages - 1 < nchunks) ? stages - 1 : nchunks;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int s = (int)(c % stages);
    if (c + stages - 1 < nchunks) {
      if (tid == 0) issue(c + stages - 1);
      issued = c + stages;
    }
    bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((c / stages) & 1));
    if (!ok) atomicOr(&s_fail, 1);
    int64_t rows = nrows - c * GR_ROWS;
    if (rows > GR_ROWS) rows = GR_ROWS;
    const float* st = stage_mem + s * stage_elems;

    float xr[GR_ROWS][NG][4];
    Acc d[GR_ROWS];
#pragma unroll
    for (int r = 0; r < GR_ROWS; ++r) {
      d[r] = Acc(0);
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        int64_t c4 = tid + (int64_t)g * GR_THREADS;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rows && c4 < n4) v = reinterpret_cast<const float4*>(st + r * n)[c4];
        xr[r][g][0] = v.x; xr[r][g][1] = v.y; xr[r][g][2] = v.z; xr[r][g][3] = v.w;
#pragma unroll
        for (int q = 0; q < 4; ++q) d[r] = fma((Acc)xr[r][g][q], pr[g][q], d[r]);
      }
      d[r] = warp_sum(d[r]);
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < GR_ROWS; ++r) red[warp][r] = d[r];
    }
    __syncthreads();
    if (s_fail) break;
    Acc t[GR_ROWS];
#pragma unroll
    for (int r = 0; r < GR_ROWS; ++r) {
      Acc v = Acc(0);
#pragma unroll
      for (int w = 0; w < GR_THREADS / 32; ++w) v += red[w][r];
      t[r] = v;
    }
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < GR_ROWS; ++r) acc[g][q] = fma(t[r], (Acc)xr[r][g][q], acc[g][q]);
    __syncthreads();
  }
  if (s_fail) {
    // drain: wait (bounded) for every copy this CTA issued, then report.
    if (tid == 0) {
      atomicCAS(err, 0, (int)NYS_ERR_TIMEOUT);
      for (int64_t c = 0; c < issued; ++c)
        mbar_wait_bounded(&bars[c % stages], (uint32_t)((c / stages) & 1), 1ll << 20);
    }
    return;
  }
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    int64_t c4 = tid + (int64_t)g * GR_THREADS;
    if (c4 < n4)
#pragma unroll
      for (int q = 0; q < 4; ++q) out[4 * c4 + q] = acc[g][q];
  }
}

// ------------------------------------------------------------ double-FP32 variant
//
// FP64-accurate ridge matvec for the refinement residual, in pairs of FP32
// numbers ("float-float"): each product of an FP32 entry of X with an FP32
// part of p is made error-free with one FMA, and the running sums carry their
// rounding errors with Knuth's TwoSum.  Relative accuracy ~2^-44, on the FP32
// pipes (GB300 issues FP32 far faster than FP64).  The rounded intrinsics
// keep the compiler from contracting the error-free steps.

struct FF {
  float hi, lo;
};

__device__ __forceinline__ void ff_add_prod(float x, float y, float& hi, float& lo) {
  const float p = __fmul_rn(x, y);
  const float pe = __fmaf_rn(x, y, -p);          // x*y = p + pe exactly
  const float s = __fadd_rn(hi, p);              // TwoSum(hi, p)
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ FF ff_sum(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  FF r;
  r.hi = __fadd_rn(s, e);                        // QuickTwoSum(s, e)
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
  return r;
}

__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = ff_sum(v, w);
  }
  return v;
}

// part[blockIdx.x][0..n) (FP64) = sum over this CTA's rows i of (x_i . p) x_i,
// p given in FP64 and split into FP32 hi + lo parts.  Same streaming
// structure as gram_fused_kernel.
template <int NG>
__global__ void __launch_bounds__(GR_THREADS, 1)
gram_fused_ff_kernel(const float* __restrict__ X, int64_t m, int64_t n,
                     const double* __restrict__ p, double* __restrict__ part, int stages,
                     int64_t rows_per_cta, int* err, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  float* stage_mem = reinterpret_cast<float*>(smem + 128);
  __shared__ FF red[GR_THREADS / 32][GR_ROWS];
  __shared__ int s_fail;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n4 = n >> 2;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = (r0 + rows_per_cta < m) ? r0 + rows_per_cta : m;
  double* out = part + (int64_t)blockIdx.x * n;

  float ph[NG][4], pl[NG][4];
  FF acc[NG][4];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    int64_t c4 = tid + (int64_t)g * GR_THREADS;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double pv = (c4 < n4) ? p[4 * c4 + q] : 0.0;
      ph[g][q] = __double2float_rn(pv);
      pl[g][q] = __double2float_rn(pv - (double)ph[g][q]);
      acc[g][q].hi = 0.f;
      acc[g][q].lo = 0.f;
    }
  }
  if (r0 >= r1) {
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      int64_t c4 = tid + (int64_t)g * GR_THREADS;
      if (c4 < n4)
#pragma unroll
        for (int q = 0; q < 4; ++q) out[4 * c4 + q] = 0.0;
    }
    return;
  }
  const int64_t nrows = r1 - r0;
  const int64_t nchunks = (nrows + GR_ROWS - 1) / GR_ROWS;
  const int64_t stage_elems = (int64_t)GR_ROWS * n;
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    s_fail = 0;
  }
  __syncthreads();
  auto issue = [&](int64_t c) {
    int s = (int)(c % stages);
    int64_t rows = nrows - c * GR_ROWS;
    if (rows > GR_ROWS) rows = GR_ROWS;
    uint32_t bytes = (uint32_t)(rows * n * sizeof(float));
    mbar_arrive_expect_tx(&bars[s], bytes);
    bulk_g2s(stage_mem + s * stage_elems, X + (r0 + c * GR_ROWS) * n, bytes, &bars[s]);
  };
  if (tid == 0) {
    int64_t pre = (stages - 1 < nchunks) ? stages - 1 : nchunks;
    for (int64_t c = 0; c < pre; ++c) issue(c);
  }
  int64_t issued = (stages - 1 < nchunks) ? stages - 1 : nchunks;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int s = (int)(c % stages);
    if (c + stages - 1 < nchunks) {
      if (tid == 0) issue(c + stages - 1);
      issued = c + stages;
    }
    bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((c / stages) & 1));
    if (!ok) atomicOr(&s_fail, 1);
    int64_t rows = nrows - c * GR_ROWS;
    if (rows > GR_ROWS) rows = GR_ROWS;
    const float* st = stage_mem + s * stage_elems;
    float xr[GR_ROWS][NG][4];
    FF d[GR_ROWS];
#pragma unroll
    for (int r = 0; r < GR_ROWS; ++r) {
      d[r].hi = 0.f;
      d[r].lo = 0.f;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        int64_t c4 = tid + (int64_t)g * GR_THREADS;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < rows && c4 < n4) v = reinterpret_cast<const float4*>(st + r * n)[c4];
        xr[r][g][0] = v.x; xr[r][g][1] = v.y; xr[r][g][2] = v.z; xr[r][g][3] = v.w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ff_add_prod(xr[r][g][q], ph[g][q], d[r].hi, d[r].lo);
          d[r].lo = __fmaf_rn(xr[r][g][q], pl[g][q], d[r].lo);
        }
      }
      d[r] = ff_warp_sum(d[r]);
    }
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < GR_ROWS; ++r) red[warp][r] = d[r];
    }
    __syncthreads();
    if (s_fail) break;
    FF t[GR_ROWS];
#pragma unroll
    for (int r = 0; r < GR_ROWS; ++r) {
      FF v = red[0][r];
#pragma unroll
      for (int w = 1; w < GR_THREADS / 32; ++w) v = ff_sum(v, red[w][r]);
      t[r] = v;
    }
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < GR_ROWS; ++r) {
          ff_add_prod(xr[r][g][q], t[r].hi, acc[g][q].hi, acc[g][q].lo);
          acc[g][q].lo = __fmaf_rn(xr[r][g][q], t[r].lo, acc[g][q].lo);
        }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) {
      atomicCAS(err, 0, (int)NYS_ERR_TIMEOUT);
      for (int64_t c = 0; c < issued; ++c)
        mbar_wait_bounded(&bars[c % stages], (uint32_t)((c / stages) & 1), 1ll << 20);
    }
    return;
  }
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    int64_t c4 = tid + (int64_t)g * GR_THREADS;
    if (c4 < n4)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        out[4 * c4 + q] = (double)acc[g][q].hi + (double)acc[g][q].lo;
  }
}

// v_j = sum_c part[c][j] (fixed order) + mu p_j; optionally r_j = b_j - v_j.
// Block = 32 columns x 8 warps: warp w sums partials w, w+8, ... of its
// lane's column, then warp 0 adds the 8 warp sums in order.
template <typename Acc, typename P, typename V>
__global__ void __launch_bounds__(256)
gram_reduce_kernel(const Acc* __restrict__ part, int64_t nparts, int64_t n, double mu,
                   const P* __restrict__ p, V* __restrict__ v, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ Acc ws[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  Acc acc = Acc(0);
  if (j < n) {
#pragma unroll 4
    for (int64_t c = warp; c < nparts; c += 8) acc += part[c * n + j];
  }
  ws[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && j < n) {
    Acc t = Acc(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) t += ws[w][lane];
    v[j] = (V)((double)t + mu * (double)p[j]);
  }
}

// Generic two-pass path (any n, any ld): t = X p, then v = X^T t.
template <typename P, typename Acc>
__global__ void gram_xp_kernel(const float* __restrict__ X, int64_t m, int64_t n, int64_t ld,
                               const P* __restrict__ p, Acc* __restrict__ t,
                               const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= m) return;
  const float* x = X + row * ld;
  Acc acc = Acc(0);
  for (int64_t j = lane; j < n; j += 32) acc = fma((Acc)x[j], (Acc)p[j], acc);
  acc = warp_sum(acc);
  if (lane == 0) t[row] = acc;
}

template <typename Acc>
__global__ void gram_xtt_kernel(const float* __restrict__ X, int64_t m, int64_t n, int64_t ld,
                                const Acc* __restrict__ t, int64_t rows_per_chunk,
                                Acc* __restrict__ part, const int* __restrict__ skip) {
  if (skip && *skip) return;
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t c = blockIdx.y;
  if (j >= n) return;
  int64_t i0 = c * rows_per_chunk, i1 = i0 + rows_per_chunk < m ? i0 + rows_per_chunk : m;
  Acc acc = Acc(0);
  for (int64_t i = i0; i < i1; ++i) acc = fma((Acc)X[i * ld + j], t[i], acc);
  part[c * n + j] = acc;
}

struct GramPlan {
  bool fused;
  int ng;
  int stages;
  int grid;
  int64_t rows_per_cta;
  size_t smem;
};

static GramPlan gram_plan(const nys_operator* op) {
  GramPlan g{};
  const int64_t n = op->n, m = op->m;
  bool aligned = ((uintptr_t)op->data % 16 == 0) && (n % 4 == 0) && (op->ld == n);
  int64_t n4 = n / 4;
  int ng = (int)cdiv(n4, GR_THREADS);
  g.fused = aligned && n4 > 0 && ng <= 8;
  if (!g.fused) return g;
  g.ng = ng <= 1 ? 1 : ng <= 2 ? 2 : ng <= 4 ? 4 : 8;
  size_t stage_bytes = (size_t)GR_ROWS * n * sizeof(float);
  int stages = (int)((200 * 1024) / stage_bytes);
  if (stages > 4) stages = 4;
  if (stages < 2) {
    g.fused = false;
    return g;
  }
  g.stages = stages;
  g.smem = 128 + stages * stage_bytes;
  g.grid = num_sms();
  g.rows_per_cta = cdiv(m, g.grid);
  return g;
}

template <typename P, typename Acc, int NG>
static int32_t gram_fused_launch(const nys_operator* op, const GramPlan& g, const P* p, Acc* part,
                                 int* err, const int* skip, cudaStream_t s) {
  auto kern = gram_fused_kernel<P, Acc, NG>;
  NYS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem));
  kern<<<g.grid, GR_THREADS, g.smem, s>>>((const float*)op->data, op->m, op->n, p, part, g.stages,
                                           g.rows_per_cta, err, skip); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

static size_t gram_work_bytes(const nys_operator* op, size_t acc_size) {
  GramPlan g = gram_plan(op);
  if (g.fused) return 256 + (size_t)g.grid * op->n * acc_size;
  int64_t chunks = 4 * (int64_t)num_sms();
  int64_t rpc = cdiv(op->m, chunks);
  chunks = cdiv(op->m, rpc);
  return 256 + ((size_t)op->m + 64) * acc_size + (size_t)chunks * op->n * acc_size;
}

// v = (X^T X + mu I) p; Acc = accumulation type (float: PCG inner, double: accurate).
// `work` holds gram_work_bytes(op, sizeof(Acc)) bytes; its first 256 bytes
// hold the timeout word.
template <typename P, typename Acc, typename V>
static int32_t gram_matvec(const nys_operator* op, double mu, const P* p, V* v, const int* skip,
                           void* work, cudaStream_t s, bool double_fp32 = false) {
  const int64_t n = op->n, m = op->m;
  GramPlan g = gram_plan(op);
  int* err = reinterpret_cast<int*>(work);
  Acc* base = reinterpret_cast<Acc*>(reinterpret_cast<unsigned char*>(work) + 256);
  if constexpr (std::is_same<P, double>::value && std::is_same<Acc, double>::value) {
    if (g.fused && double_fp32) {
      // FP64-accurate product in double-FP32 arithmetic
      double* part = base;
      auto launch = [&](auto kern) -> int32_t {
        NYS_CUDA_TRY(
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem));
        kern<<<g.grid, GR_THREADS, g.smem, s>>>((const float*)op->data, op->m, op->n, p, part,
                                                 g.stages, g.rows_per_cta, err, skip);
        count_launch();
        NYS_CUDA_TRY(cudaGetLastError());
        return NYS_OK;
      };
      switch (g.ng) {
        case 1: NYS_TRY(launch(gram_fused_ff_kernel<1>)); break;
        case 2: NYS_TRY(launch(gram_fused_ff_kernel<2>)); break;
        case 4: NYS_TRY(launch(gram_fused_ff_kernel<4>)); break;
        default: NYS_TRY(launch(gram_fused_ff_kernel<8>)); break;
      }
      gram_reduce_kernel<double, P, V><<<(unsigned)cdiv(n, 32), 256, 0, s>>>(part, g.grid, n, mu,
                                                                             p, v, skip);
      count_launch();
      NYS_CUDA_TRY(cudaGetLastError());
      return NYS_OK;
    }
  }
  if (g.fused) {
    Acc* part = base;
    switch (g.ng) {
      case 1: NYS_TRY((gram_fused_launch<P, Acc, 1>(op, g, p, part, err, skip, s))); break;
      case 2: NYS_TRY((gram_fused_launch<P, Acc, 2>(op, g, p, part, err, skip, s))); break;
      case 4: NYS_TRY((gram_fused_launch<P, Acc, 4>(op, g, p, part, err, skip, s))); break;
      default: NYS_TRY((gram_fused_launch<P, Acc, 8>(op, g, p, part, err, skip, s))); break;
    }
    gram_reduce_kernel<Acc, P, V><<<(unsigned)cdiv(n, 32), 256, 0, s>>>(part, g.grid, n, mu, p, v,
                                                                         skip); count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return NYS_OK;
  }
  int64_t chunks = 4 * (int64_t)num_sms();
  int64_t rpc = cdiv(m, chunks);
  chunks = cdiv(m, rpc);
  Acc* t = base;
  Acc* part = base + m + 64;
  gram_xp_kernel<P, Acc><<<(unsigned)cdiv(m, 8), 256, 0, s>>>((const float*)op->data, m, n, op->ld,
                                                               p, t, skip); count_launch();
  dim3 grid((unsigned)cdiv(n, 128), (unsigned)chunks);
  gram_xtt_kernel<Acc><<<grid, 128, 0, s>>>((const float*)op->data, m, n, op->ld, t, rpc, part,
                                            skip); count_launch();
  gram_reduce_kernel<Acc, P, V><<<(unsigned)cdiv(n, 32), 256, 0, s>>>(part, chunks, n, mu, p, v,
                                                                       skip); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// ============================================================ rbf

constexpr int RBF_DMAX = 64;
constexpr int RBF_BI = 128;  // rows per CTA (one per thread)
constexpr int RBF_BJ = 128;  // points per smem tile

// v_i = sum_j exp(-||x_i - x_j||^2 / (2 sigma^2)) p_j + mu p_i.
// T = arithmetic type of the distances, the exponential and the sum.
template <typename T, typename P, typename V>
__global__ void __launch_bounds__(RBF_BI)
rbf_matvec_kernel(const float* __restrict__ pts, int64_t n, int64_t d, int64_t ld, double sigma,
                  const P* __restrict__ p, double mu, V* __restrict__ v,
                  const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ float xs[RBF_BJ][RBF_DMAX + 1];
  __shared__ T ps[RBF_BJ];
  const int64_t i = (int64_t)blockIdx.x * RBF_BI + threadIdx.x;
  float xi[RBF_DMAX];
#pragma unroll
  for (int k = 0; k < RBF_DMAX; ++k) xi[k] = (i < n && k < d) ? pts[i * ld + k] : 0.f;
  const T scale = (T)(-1.0 / (2.0 * sigma * sigma));
  T acc = T(0);
  for (int64_t j0 = 0; j0 < n; j0 += RBF_BJ) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)RBF_BJ * d; e += RBF_BI) {
      int64_t jj = e / d, k = e % d;
      xs[jj][k] = (j0 + jj < n) ? pts[(j0 + jj) * ld + k] : 0.f;
    }
    for (int jj = threadIdx.x; jj < RBF_BJ; jj += RBF_BI) ps[jj] = (j0 + jj < n) ? (T)p[j0 + jj] : T(0);
    __syncthreads();
    const int jn = (int)((n - j0 < RBF_BJ) ? n - j0 : RBF_BJ);
    for (int jj = 0; jj < jn; ++jj) {
      T dist = T(0);
#pragma unroll
      for (int k = 0; k < RBF_DMAX; ++k) {
        if (k < d) {
          T df = (T)xi[k] - (T)xs[jj][k];
          dist = fma(df, df, dist);
        }
      }
      acc = fma(exp(dist * scale), ps[jj], acc);
    }
  }
  if (i < n) v[i] = (V)((double)acc + mu * (double)p[i]);
}

// FP32 matvec (inner PCG): with c = -log2(e) / (2 sigma^2),
//   K_ij = 2^(c ||x_i||^2 + c ||x_j||^2 - 2c x_i . x_j),
// so a tile stores -2c x_j and c ||x_j||^2 once and each entry costs one
// d-long FP32 dot, two adds and one exp2.  The norm expansion loses at most
// ~u (||x_i||^2 + ||x_j||^2) / (2 sigma^2) in the exponent, a relative error
// of a few u in K_ij for points at the bandwidth scale.
__global__ void __launch_bounds__(RBF_BI)
rbf_matvec_f32_kernel(const float* __restrict__ pts, int64_t n, int64_t d, int64_t ld,
                      double sigma, const float* __restrict__ p, double mu, float* __restrict__ v,
                      const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ float xs[RBF_BJ][RBF_DMAX + 1];
  __shared__ float aj[RBF_BJ];
  __shared__ float ps[RBF_BJ];
  const int64_t i = (int64_t)blockIdx.x * RBF_BI + threadIdx.x;
  const float c = (float)(-1.4426950408889634 / (2.0 * sigma * sigma));
  float xi[RBF_DMAX];
  float ai = 0.f;
#pragma unroll
  for (int k = 0; k < RBF_DMAX; ++k) {
    xi[k] = (i < n && k < d) ? pts[i * ld + k] : 0.f;
    ai = fmaf(xi[k], xi[k], ai);
  }
  ai *= c;
  float acc = 0.f;
  for (int64_t j0 = 0; j0 < n; j0 += RBF_BJ) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)RBF_BJ * d; e += RBF_BI) {
      int64_t jj = e / d, k = e % d;
      xs[jj][k] = (j0 + jj < n) ? -2.f * c * pts[(j0 + jj) * ld + k] : 0.f;
    }
    for (int jj = threadIdx.x; jj < RBF_BJ; jj += RBF_BI) {
      float s = 0.f;
      if (j0 + jj < n)
        for (int64_t k = 0; k < d; ++k) {
          const float x = pts[(j0 + jj) * ld + k];
          s = fmaf(x, x, s);
        }
      aj[jj] = c * s;
      ps[jj] = (j0 + jj < n) ? p[j0 + jj] : 0.f;
    }
    __syncthreads();
    const int jn = (int)((n - j0 < RBF_BJ) ? n - j0 : RBF_BJ);
    for (int jj = 0; jj < jn; ++jj) {
      float e = ai + aj[jj];
#pragma unroll
      for (int k = 0; k < RBF_DMAX; ++k)
        if (k < d) e = fmaf(xi[k], xs[jj][k], e);
      acc = fmaf(exp2f(fminf(e, 0.f)), ps[jj], acc);
    }
  }
  if (i < n) v[i] = acc + (float)mu * p[i];
}

// Y[i][l] = sum_j K_ij Q[j][l] for a 64-row x 64-column output tile per CTA.
constexpr int RS_BI = 64, RS_BL = 64;
template <typename T, int RS_BJ = (sizeof(T) == 8 ? 16 : 32)>
__global__ void __launch_bounds__(256)
rbf_sketch_kernel(const float* __restrict__ pts, int64_t n, int64_t d, int64_t ld, double sigma,
                  const T* __restrict__ Q, int64_t ell, T* __restrict__ Y) {
  __shared__ float xi[RS_BI][RBF_DMAX + 1];
  __shared__ float xj[RS_BJ][RBF_DMAX + 1];
  __shared__ T Ks[RS_BJ][RS_BI + 1];
  __shared__ T Qs[RS_BJ][RS_BL + 1];
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * RS_BI, l0 = (int64_t)blockIdx.y * RS_BL;
  const T scale = (T)(-1.0 / (2.0 * sigma * sigma));
  for (int64_t e = tid; e < (int64_t)RS_BI * d; e += 256) {
    int64_t r = e / d, k = e % d;
    xi[r][k] = (i0 + r < n) ? pts[(i0 + r) * ld + k] : 0.f;
  }
  const int tr = tid / 16, tc = tid % 16;  // 16 x 16 threads, 4 x 4 outputs each
  T acc[4][4] = {};
  for (int64_t j0 = 0; j0 < n; j0 += RS_BJ) {
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)RS_BJ * d; e += 256) {
      int64_t r = e / d, k = e % d;
      xj[r][k] = (j0 + r < n) ? pts[(j0 + r) * ld + k] : 0.f;
    }
    for (int e = tid; e < RS_BJ * RS_BL; e += 256) {
      int r = e / RS_BL, c = e % RS_BL;
      Qs[r][c] = (j0 + r < n && l0 + c < ell) ? Q[(j0 + r) * ell + l0 + c] : T(0);
    }
    __syncthreads();
    for (int e = tid; e < RS_BI * RS_BJ; e += 256) {
      int r = e % RS_BI, jj = e / RS_BI;
      T dist = T(0);
      for (int k = 0; k < d; ++k) {
        T df = (T)xi[r][k] - (T)xj[jj][k];
        dist = fma(df, df, dist);
      }
      Ks[jj][r] = (j0 + jj < n) ? exp(dist * scale) : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < RS_BJ; ++jj) {
      T a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = Ks[jj][tr * 4 + x];
#pragma unroll
      for (int y = 0; y < 4; ++y) b[y] = Qs[jj][tc * 4 + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    int64_t i = i0 + tr * 4 + x;
    if (i >= n) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      int64_t l = l0 + tc * 4 + y;
      if (l < ell) Y[i * ell + l] = acc[x][y];
    }
  }
}

// ============================================================ dispatch

// Passes of the tensor-core kernel-times-test-matrix product in the
// mixed-precision sketch: 3 (3xTF32 distances and products, FP32-accurate
// kernel entries).  One TF32 pass puts ~1e-3 relative error into every kernel
// entry; the sketched matrix is then K + N with ||N|| ~ 1e-3 ||K||, and once
// mu is small against that the preconditioner built from it stalls PCG
// (measured at n = 50000, ell = 1024, mu = 5e-4: 832 iterations against 112
// with an FP64 sketch).
constexpr int kRbfSketchPasses = 3;

int32_t op_sketch(const nys_operator* op, bool f64, const void* Q, void* V, int64_t ell,
                  cudaStream_t s) {
  const int64_t n = op->n;
  if (op->kind == NYS_OP_DENSE) {
    // Y = A Omega in double-FP32 arithmetic (~2^-48 relative to sum |a| |omega|,
    // on the FP32 pipes): the sketch only shapes the preconditioner, and the
    // n x ell x n product is the one FP64 GEMM of the dense path that would
    // otherwise run at GB300's FP64 rate
    if (f64)
      return gemm_dfl(false, n, ell, n, (const double*)op->data, op->ld, (const double*)Q, ell,
                      (double*)V, ell, false, s);
    // mixed: FP64 matrix, FP32 block -> compute in double-FP32 and round
    Scratch sc(s);
    double *Qd, *Vd;
    NYS_TRY(sc.get(&Qd, n * ell));
    NYS_TRY(sc.get(&Vd, n * ell));
    NYS_TRY(convert_f32_to_f64((const float*)Q, Qd, n * ell, s));
    NYS_TRY(gemm_dfl(false, n, ell, n, (const double*)op->data, op->ld, Qd, ell, Vd, ell, false, s));
    return convert_f64_to_f32(Vd, (float*)V, n * ell, s);
  }
  if (op->kind == NYS_OP_GRAM) {
    const int64_t m = op->m;
    const float* X = (const float*)op->data;
    Scratch sc(s);
    if (f64) {
      // exact FP64 products of the FP32 data
      double *Xd, *Z;
      NYS_TRY(sc.get(&Z, m * ell));
      // Z = X Q computed from an FP64 copy of X in row blocks to bound memory
      const int64_t blk = 16384;
      NYS_TRY(sc.get(&Xd, (m < blk ? m : blk) * n));
      for (int64_t r0 = 0; r0 < m; r0 += blk) {
        int64_t rows = (m - r0 < blk) ? m - r0 : blk;
        if (op->ld == n) {
          NYS_TRY(convert_f32_to_f64(X + r0 * n, Xd, rows * n, s));
        } else {
          for (int64_t r = 0; r < rows; ++r)
            NYS_TRY(convert_f32_to_f64(X + (r0 + r) * op->ld, Xd + r * n, n, s));
        }
        NYS_TRY(gemm_f64(false, rows, ell, n, Xd, n, (const double*)Q, ell, Z + r0 * ell, ell, s));
      }
      // V = X^T Z = sum over row blocks of Xd_b^T Z_b
      double* acc;
      double* tmp;
      NYS_TRY(sc.get(&acc, n * ell));
      NYS_TRY(sc.get(&tmp, n * ell));
      NYS_CUDA_TRY(cudaMemsetAsync(acc, 0, n * ell * sizeof(double), s));
      for (int64_t r0 = 0; r0 < m; r0 += blk) {
        int64_t rows = (m - r0 < blk) ? m - r0 : blk;
        if (op->ld == n) {
          NYS_TRY(convert_f32_to_f64(X + r0 * n, Xd, rows * n, s));
        } else {
          for (int64_t r = 0; r < rows; ++r)
            NYS_TRY(convert_f32_to_f64(X + (r0 + r) * op->ld, Xd + r * n, n, s));
        }
        NYS_TRY(gemm_f64(true, n, ell, rows, Xd, n, Z + r0 * ell, ell, tmp, ell, s));
        NYS_TRY(add_inplace_f64(acc, tmp, n * ell, s));
      }
      NYS_CUDA_TRY(cudaMemcpyAsync(V, acc, n * ell * sizeof(double), cudaMemcpyDeviceToDevice, s));
      return NYS_OK;
    }
    if (tc_gemm_supported(ell, m, n, X, op->ld, X, op->ld) && (m % 4) == 0) {
      // Tensor cores, both operands K-major:  Z^T = Q^T X^T  (ell x m, K = n),
      // Y^T = Z^T (X^T)^T (ell x n, K = m) with X^T materialised once.
      float *Qt, *Xt, *Zt, *Yt;
      int* err;
      NYS_TRY(sc.get(&Qt, ell * n));
      NYS_TRY(sc.get(&Xt, n * m));
      NYS_TRY(sc.get(&Zt, ell * m));
      NYS_TRY(sc.get(&Yt, ell * n));
      NYS_TRY(sc.get(&err, 1));
      NYS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
      NYS_TRY(transpose_f32((const float*)Q, n, ell, ell, Qt, s));
      NYS_TRY(transpose_f32(X, m, n, op->ld, Xt, s));
      NYS_TRY(tc_gemm_tn_f32(ell, m, n, Qt, n, X, op->ld, Zt, m, err, s));
      NYS_TRY(tc_gemm_tn_f32(ell, n, m, Zt, m, Xt, m, Yt, n, err, s));
      NYS_TRY(transpose_f32(Yt, ell, n, n, (float*)V, s));
      int h_err = 0;
      NYS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      NYS_CUDA_TRY(cudaStreamSynchronize(s));
      return h_err ? NYS_ERR_TIMEOUT : NYS_OK;
    }
    float* Z;
    NYS_TRY(sc.get(&Z, m * ell));
    NYS_TRY(gemm_f32(false, m, ell, n, X, op->ld, (const float*)Q, ell, Z, ell, s));
    return gemm_f32(true, n, ell, m, X, op->ld, Z, ell, (float*)V, ell, s);
  }
  // RBF
  if (!f64 && rbf_tc_supported(op->d)) {
    // tensor cores: Y^T = K Q^T with the vectors of the sketch as rows
    Scratch sc(s);
    float *Qt, *Yt;
    int* err;
    NYS_TRY(sc.get(&Qt, ell * n));
    NYS_TRY(sc.get(&Yt, ell * n));
    NYS_TRY(sc.get(&err, 1));
    NYS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    NYS_TRY(transpose_f32((const float*)Q, n, ell, ell, Qt, s));
    NYS_TRY(rbf_tc_products((const float*)op->data, n, op->d, op->ld, op->sigma, ell, Qt, n, 0,
                            nullptr, 0.0, Yt, n, kRbfSketchPasses, nullptr, 0, nullptr, err, s));
    NYS_TRY(transpose_f32(Yt, ell, n, n, (float*)V, s));
    int h_err = 0;
    NYS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    return h_err ? NYS_ERR_TIMEOUT : NYS_OK;
  }
  dim3 grid((unsigned)cdiv(n, RS_BI), (unsigned)cdiv(ell, RS_BL));
  if (f64)
    rbf_sketch_kernel<double><<<grid, 256, 0, s>>>((const float*)op->data, n, op->d, op->ld,
                                                   op->sigma, (const double*)Q, ell, (double*)V);
  else
    rbf_sketch_kernel<float><<<grid, 256, 0, s>>>((const float*)op->data, n, op->d, op->ld,
                                                  op->sigma, (const float*)Q, ell, (float*)V); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// ============================================================ column sampling
//
// Q = I[:, S] (the selection matrix of the sampled columns S) and Y = A Q =
// A[:, S] for the column-sampling Nystrom sketch (Sec. 2.2, random projection
// versus column sampling): the Gaussian kernel evaluates its l columns directly
// (n l entries instead of n^2 l), dense A gathers them, the ridge operator
// forms X^T (X Q).

template <typename T>
__global__ void selection_kernel(const int64_t* __restrict__ cols, int64_t n, int64_t ell,
                                 T* __restrict__ Q) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * ell;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ell, c = e - i * ell;
    Q[e] = (cols[c] == i) ? T(1) : T(0);
  }
}

template <typename T>
__global__ void dense_columns_kernel(const double* __restrict__ A, int64_t n, int64_t ld,
                                     const int64_t* __restrict__ cols, int64_t ell,
                                     T* __restrict__ Y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * ell;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ell, c = e - i * ell;
    Y[e] = (T)A[i * ld + cols[c]];  // A symmetric: A[i][S_c]
  }
}

// Y[i][c] = exp(-||x_i - x_{S_c}||^2 / (2 sigma^2)); distances by direct
// differences (FP64 sums for T = double).  Block: 32 columns x 8 rows.
template <typename T>
__global__ void rbf_columns_kernel(const float* __restrict__ pts, int64_t n, int64_t d,
                                   int64_t ld, double sigma, const int64_t* __restrict__ cols,
                                   int64_t ell, T* __restrict__ Y) {
  __shared__ float xc[32][RBF_DMAX + 1];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  for (int e = threadIdx.y * 32 + threadIdx.x; e < 32 * d; e += 256) {
    const int cc = e / (int)d, k = e - cc * (int)d;
    xc[cc][k] = (c0 + cc < ell) ? pts[cols[c0 + cc] * ld + k] : 0.f;
  }
  __syncthreads();
  const int64_t c = c0 + threadIdx.x;
  const T scale = (T)(-1.0 / (2.0 * sigma * sigma));
  for (int64_t i = (int64_t)blockIdx.y * 8 + threadIdx.y; i < n; i += (int64_t)gridDim.y * 8) {
    T dist = T(0);
    for (int64_t k = 0; k < d; ++k) {
      const T df = (T)pts[i * ld + k] - (T)xc[threadIdx.x][k];
      dist = fma(df, df, dist);
    }
    if (c < ell) Y[i * ell + c] = exp(dist * scale);
  }
}

int32_t op_columns(const nys_operator* op, bool f64, const int64_t* cols, int64_t ell, void* Q,
                   void* Y, cudaStream_t s) {
  const int64_t n = op->n;
  const unsigned g = (unsigned)(cdiv(n * ell, 256) < 8192 ? cdiv(n * ell, 256) : 8192);
  if (f64)
    selection_kernel<double><<<g, 256, 0, s>>>(cols, n, ell, (double*)Q);
  else
    selection_kernel<float><<<g, 256, 0, s>>>(cols, n, ell, (float*)Q);
  count_launch();
  if (op->kind == NYS_OP_GRAM) return op_sketch(op, f64, Q, Y, ell, s);
  if (op->kind == NYS_OP_DENSE) {
    if (f64)
      dense_columns_kernel<double><<<g, 256, 0, s>>>((const double*)op->data, n, op->ld, cols,
                                                     ell, (double*)Y);
    else
      dense_columns_kernel<float><<<g, 256, 0, s>>>((const double*)op->data, n, op->ld, cols, ell,
                                                    (float*)Y);
    count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return NYS_OK;
  }
  if (op->d > RBF_DMAX) return NYS_ERR_ARG;
  const unsigned gy = (unsigned)(cdiv(n, 8) < 2048 ? cdiv(n, 8) : 2048);
  const dim3 grid((unsigned)cdiv(ell, 32), gy);
  if (f64)
    rbf_columns_kernel<double><<<grid, dim3(32, 8), 0, s>>>((const float*)op->data, n, op->d,
                                                            op->ld, op->sigma, cols, ell,
                                                            (double*)Y);
  else
    rbf_columns_kernel<float><<<grid, dim3(32, 8), 0, s>>>((const float*)op->data, n, op->d,
                                                           op->ld, op->sigma, cols, ell, (float*)Y);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

size_t op_matvec_work_bytes(const nys_operator* op, bool accurate) {
  if (op->kind == NYS_OP_GRAM) return gram_work_bytes(op, accurate ? sizeof(double) : sizeof(float));
  if (op->kind == NYS_OP_RBF && rbf_tc_supported(op->d)) return rbf_tc_work_bytes(op->n, 1, 3);
  return 256;
}

// ---------------------------------------------------------------- matvec timing
//
// Opt-in CUDA-event timing of the FP32 operator products (the inner PCG
// matvec) and of the dense products in either precision: a pool of event pairs recorded on the launching stream around each
// product while enabled, summed when timing stops.  Inside a stream capture
// the pair is recorded as two external event-record nodes of the graph on
// placeholder events; before each replay timing_graph_rebind() points those
// nodes at fresh pairs of the pool, so graph replays are timed product by
// product like plain launches.
namespace {
std::mutex g_tm_mutex;
bool g_tm_on = false;
std::vector<cudaEvent_t> g_tm_ev;   // 2 per product
size_t g_tm_used = 0;
std::vector<cudaEvent_t> g_tm_ph;   // placeholders of the capture in progress
size_t g_tm_ph_used = 0;

struct MatvecTimer {
  cudaStream_t s;
  int slot = -1;
  bool captured = false;
  explicit MatvecTimer(cudaStream_t st) : s(st) {
    std::lock_guard<std::mutex> lk(g_tm_mutex);
    if (!g_tm_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return;
    if (cs == cudaStreamCaptureStatusActive) {
      while (g_tm_ph.size() < g_tm_ph_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        g_tm_ph.push_back(e);
      }
      slot = (int)g_tm_ph_used;
      g_tm_ph_used += 2;
      captured = true;
      cudaEventRecordWithFlags(g_tm_ph[slot], s, cudaEventRecordExternal);
    } else if (g_tm_used + 2 <= g_tm_ev.size()) {
      slot = (int)g_tm_used;
      g_tm_used += 2;
      cudaEventRecord(g_tm_ev[slot], s);
    }
  }
  ~MatvecTimer() {
    if (slot < 0) return;
    if (captured)
      cudaEventRecordWithFlags(g_tm_ph[slot + 1], s, cudaEventRecordExternal);
    else
      cudaEventRecord(g_tm_ev[slot + 1], s);
  }
};
}  // namespace

bool timing_active() {
  std::lock_guard<std::mutex> lk(g_tm_mutex);
  return g_tm_on;
}

void timing_capture_begin() {
  std::lock_guard<std::mutex> lk(g_tm_mutex);
  g_tm_ph_used = 0;
}

int32_t timing_graph_nodes(cudaGraph_t g, GraphTiming* gt) {
  gt->nodes.clear();
  gt->index.clear();
  gt->products = 0;
  std::lock_guard<std::mutex> lk(g_tm_mutex);
  if (g_tm_ph_used == 0) return NYS_OK;
  size_t cnt = 0;
  NYS_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &cnt));
  std::vector<cudaGraphNode_t> nodes(cnt);
  NYS_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &cnt));
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    NYS_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t e;
    NYS_CUDA_TRY(cudaGraphEventRecordNodeGetEvent(nd, &e));
    for (size_t k = 0; k < g_tm_ph_used; ++k)
      if (g_tm_ph[k] == e) {
        gt->nodes.push_back(nd);
        gt->index.push_back((int)k);
      }
  }
  // both events of every pair must be present, else the graph is not timed
  if (gt->nodes.size() != g_tm_ph_used) {
    gt->nodes.clear();
    gt->index.clear();
    return NYS_OK;
  }
  gt->products = (int)(g_tm_ph_used / 2);
  gt->placeholders.assign(g_tm_ph.begin(), g_tm_ph.begin() + g_tm_ph_used);
  return NYS_OK;
}

int32_t timing_graph_rebind(cudaGraphExec_t ge, const GraphTiming& gt) {
  if (gt.products == 0) return NYS_OK;
  std::lock_guard<std::mutex> lk(g_tm_mutex);
  const size_t need = 2 * (size_t)gt.products;
  const bool pool = g_tm_on && g_tm_used + need <= g_tm_ev.size();
  const size_t base = g_tm_used;
  for (size_t k = 0; k < gt.nodes.size(); ++k) {
    const int i = gt.index[k];
    cudaEvent_t e = pool ? g_tm_ev[base + i] : gt.placeholders[i];
    NYS_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(ge, gt.nodes[k], e));
  }
  if (pool) g_tm_used += need;
  return NYS_OK;
}

int32_t timing_start(int32_t max_products) {
  std::lock_guard<std::mutex> lk(g_tm_mutex);
  for (cudaEvent_t e : g_tm_ev) cudaEventDestroy(e);
  g_tm_ev.clear();
  g_tm_used = 0;
  g_tm_on = false;
  if (max_products < 1) return NYS_ERR_ARG;
  g_tm_ev.resize(2 * (size_t)max_products);
  for (auto& e : g_tm_ev) NYS_CUDA_TRY(cudaEventCreate(&e));
  g_tm_on = true;
  return NYS_OK;
}

int32_t timing_stop(double* total_ms, int64_t* products) {
  std::lock_guard<std::mutex> lk(g_tm_mutex);
  g_tm_on = false;
  std::vector<float> dur;
  for (size_t i = 0; i + 1 < g_tm_used; i += 2) {
    NYS_CUDA_TRY(cudaEventSynchronize(g_tm_ev[i + 1]));
    float ms = 0.f;
    NYS_CUDA_TRY(cudaEventElapsedTime(&ms, g_tm_ev[i], g_tm_ev[i + 1]));
    dur.push_back(ms);
  }
  // A product launched for a system that has already converged (a graph
  // replay that runs past convergence) returns at once on the system's done
  // word: a few microseconds against the hundreds of a product that ran.
  // Products below a quarter of the median are such launches and are left
  // out of the total and the count.
  double tot = 0.0;
  int64_t cnt = 0;
  if (!dur.empty()) {
    std::vector<float> srt(dur);
    std::nth_element(srt.begin(), srt.begin() + srt.size() / 2, srt.end());
    const float cut = 0.25f * srt[srt.size() / 2];
    for (float ms : dur)
      if (ms >= cut) {
        tot += ms;
        ++cnt;
      }
  }
  if (total_ms) *total_ms = tot;
  if (products) *products = cnt;
  for (cudaEvent_t e : g_tm_ev) cudaEventDestroy(e);
  g_tm_ev.clear();
  g_tm_used = 0;
  return NYS_OK;
}

int32_t op_matvec_f32(const nys_operator* op, double mu, const float* p, float* v, const int* skip,
                      void* work, cudaStream_t s) {
  MatvecTimer timer(s);
  const int64_t n = op->n;
  if (op->kind == NYS_OP_DENSE) {
    dense_matvec_kernel<float, float><<<(unsigned)cdiv(n, DM_WARPS), 32 * DM_WARPS, 0, s>>>(
        (const double*)op->data, n, op->ld, p, mu, v, skip); count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return NYS_OK;
  }
  if (op->kind == NYS_OP_GRAM) {
    if (work) return gram_matvec<float, float, float>(op, mu, p, v, skip, work, s);
    Scratch sc(s);
    unsigned char* w;
    NYS_TRY(sc.get(&w, op_matvec_work_bytes(op, false)));
    NYS_CUDA_TRY(cudaMemsetAsync(w, 0, 256, s));
    return gram_matvec<float, float, float>(op, mu, p, v, skip, w, s);
  }
  if (rbf_tc_supported(op->d))
    return rbf_tc_products((const float*)op->data, n, op->d, op->ld, op->sigma, 1, p, n, 1, nullptr,
                           mu, v, n, 3, skip, 0, work, nullptr, s);
  rbf_matvec_f32_kernel<<<(unsigned)cdiv(n, RBF_BI), RBF_BI, 0, s>>>(
      (const float*)op->data, n, op->d, op->ld, op->sigma, p, mu, v, skip); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

int32_t op_matvec_f64(const nys_operator* op, double mu, const double* p, double* v,
                      const int* skip, void* work, cudaStream_t s) {
  const int64_t n = op->n;
  if (op->kind == NYS_OP_DENSE) {
    MatvecTimer timer(s);  // the dense products are timed in either precision
    dense_matvec_kernel<double, double><<<(unsigned)cdiv(n, DM_WARPS), 32 * DM_WARPS, 0, s>>>(
        (const double*)op->data, n, op->ld, p, mu, v, skip); count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return NYS_OK;
  }
  if (op->kind == NYS_OP_GRAM) {
    if (work) return gram_matvec<double, double, double>(op, mu, p, v, skip, work, s);
    Scratch sc(s);
    unsigned char* w;
    NYS_TRY(sc.get(&w, op_matvec_work_bytes(op, true)));
    NYS_CUDA_TRY(cudaMemsetAsync(w, 0, 256, s));
    return gram_matvec<double, double, double>(op, mu, p, v, skip, w, s);
  }
  if (op->d <= 64) {
    const float* pts = (const float*)op->data;
    return rbf_exact_products(pts, n, op->ld, pts, n, op->ld, op->d, op->sigma, 0, 1, nullptr, mu,
                              1, p, v, skip, s);
  }
  rbf_matvec_kernel<double, double, double><<<(unsigned)cdiv(n, RBF_BI), RBF_BI, 0, s>>>(
      (const float*)op->data, n, op->d, op->ld, op->sigma, p, mu, v, skip); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// ============================================================ batched rbf (FP32)
//
// V[s][i] = sum_j K_ij P[s][j] + mu_s P[s][i] for S systems sharing the kernel
// matrix: each 64 x 32 kernel tile is computed once per 64-system chunk and
// contracted against all of them (a 64 x 64 x 32 FP32 product per tile), so
// the exponentials are amortised over the batch.  A chunk whose systems have
// all converged returns at once.
constexpr int RB_BI = 64, RB_BJ = 32, RB_BS = 64;
__global__ void __launch_bounds__(256)
rbf_batched_kernel(const float* __restrict__ pts, int64_t n, int64_t d, int64_t ld, double sigma,
                   int64_t nsys, const double* __restrict__ mus, const float* __restrict__ P,
                   float* __restrict__ V, const int* __restrict__ done0, int64_t done_stride) {
  __shared__ float xi[RB_BI][RBF_DMAX + 1];
  __shared__ float xj[RB_BJ][RBF_DMAX + 1];
  __shared__ float Ks[RB_BJ][RB_BI + 4];
  __shared__ float Ps[RB_BJ][RB_BS + 4];
  __shared__ int any_active;
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * RB_BI, s0 = (int64_t)blockIdx.y * RB_BS;
  const int64_t ns = (nsys - s0 < RB_BS) ? nsys - s0 : RB_BS;
  if (tid == 0) {
    int act = 0;
    for (int64_t q = 0; q < ns; ++q)
      if (!done0 || !done0[(s0 + q) * done_stride]) act = 1;
    any_active = act;
  }
  __syncthreads();
  if (!any_active) return;
  const float scale = (float)(-1.0 / (2.0 * sigma * sigma));
  for (int64_t e = tid; e < (int64_t)RB_BI * d; e += 256) {
    int64_t r = e / d, k = e % d;
    xi[r][k] = (i0 + r < n) ? pts[(i0 + r) * ld + k] : 0.f;
  }
  const int tr = tid / 16, tc = tid % 16;  // 4 rows x 4 systems per thread
  float acc[4][4] = {};
  for (int64_t j0 = 0; j0 < n; j0 += RB_BJ) {
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)RB_BJ * d; e += 256) {
      int64_t r = e / d, k = e % d;
      xj[r][k] = (j0 + r < n) ? pts[(j0 + r) * ld + k] : 0.f;
    }
    for (int e = tid; e < RB_BJ * RB_BS; e += 256) {
      int q = e / RB_BJ, jj = e % RB_BJ;  // coalesced along j
      Ps[jj][q] = (q < ns && j0 + jj < n) ? P[(s0 + q) * n + j0 + jj] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < RB_BI * RB_BJ; e += 256) {
      int r = e % RB_BI, jj = e / RB_BI;
      float dist = 0.f;
      for (int k = 0; k < d; ++k) {
        float df = xi[r][k] - xj[jj][k];
        dist = fmaf(df, df, dist);
      }
      Ks[jj][r] = (j0 + jj < n) ? __expf(dist * scale) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < RB_BJ; ++jj) {
      float a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = Ks[jj][tr * 4 + x];
#pragma unroll
      for (int y = 0; y < 4; ++y) b[y] = Ps[jj][tc * 4 + y];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const int64_t q = s0 + tc * 4 + y;
    if (q >= nsys) continue;
    if (done0 && done0[q * done_stride]) continue;
    const float mu = (float)mus[q];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int64_t i = i0 + tr * 4 + x;
      if (i < n) V[q * n + i] = acc[x][y] + mu * P[q * n + i];
    }
  }
}

int32_t op_matvec_batched_f32(const nys_operator* op, const double* d_mu, int64_t nsys,
                              const float* P, float* V, const int* done0, int64_t done_stride,
                              int* err, void* work, cudaStream_t s) {
  if (op->kind != NYS_OP_RBF) return NYS_ERR_ARG;
  MatvecTimer timer(s);
  if (rbf_tc_supported(op->d))
    return rbf_tc_products((const float*)op->data, op->n, op->d, op->ld, op->sigma, nsys, P, op->n,
                           2, d_mu, 0.0, V, op->n, 3, done0, done_stride, work, err, s);
  dim3 grid((unsigned)cdiv(op->n, RB_BI), (unsigned)cdiv(nsys, RB_BS));
  rbf_batched_kernel<<<grid, 256, 0, s>>>((const float*)op->data, op->n, op->d, op->ld, op->sigma,
                                          nsys, d_mu, P, V, done0, done_stride);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// ============================================================ cross kernel (FP64)
//
// out[q][i] = sum_j k(t_i, x_j) v[q][j] with k the Gaussian kernel (kind 0)
// or its derivative in sigma, k(t, x) ||t - x||^2 / sigma^3 (kind 1).  Rows
// are the target points, columns the source points; FP64 arithmetic.  Used
// for predictions K_v alpha, their adjoint K_v^T g, and the sigma-derivative
// products of the KRR gradient.
constexpr int CX_BI = 128, CX_BJ = 64;
__global__ void __launch_bounds__(CX_BI)
rbf_cross_kernel(const float* __restrict__ tg, int64_t nt, int64_t ldt,
                 const float* __restrict__ pts, int64_t n, int64_t ldp, int64_t d, double sigma,
                 const double* __restrict__ v, double* __restrict__ out, int kind) {
  __shared__ float xs[CX_BJ][RBF_DMAX + 1];
  __shared__ double vs[CX_BJ];
  const int64_t q = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * CX_BI + threadIdx.x;
  float ti[RBF_DMAX];
#pragma unroll
  for (int k = 0; k < RBF_DMAX; ++k) ti[k] = (i < nt && k < d) ? tg[i * ldt + k] : 0.f;
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const double inv_s3 = 1.0 / (sigma * sigma * sigma);
  double acc = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += CX_BJ) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)CX_BJ * d; e += CX_BI) {
      int64_t jj = e / d, k = e % d;
      xs[jj][k] = (j0 + jj < n) ? pts[(j0 + jj) * ldp + k] : 0.f;
    }
    for (int jj = threadIdx.x; jj < CX_BJ; jj += CX_BI)
      vs[jj] = (j0 + jj < n) ? v[q * n + j0 + jj] : 0.0;
    __syncthreads();
    const int jn = (int)((n - j0 < CX_BJ) ? n - j0 : CX_BJ);
    for (int jj = 0; jj < jn; ++jj) {
      double dist = 0.0;
#pragma unroll
      for (int k = 0; k < RBF_DMAX; ++k) {
        if (k < d) {
          const double df = (double)ti[k] - (double)xs[jj][k];
          dist = fma(df, df, dist);
        }
      }
      double kv = exp(-dist * inv2s2);
      if (kind == 1) kv *= dist * inv_s3;
      acc = fma(kv, vs[jj], acc);
    }
  }
  if (i < nt) out[q * nt + i] = acc;
}

int32_t rbf_cross_matvec(const float* tg, int64_t nt, int64_t ldt, const float* pts, int64_t n,
                         int64_t ldp, int64_t d, double sigma, int64_t nvec, const double* v,
                         double* out, int kind, cudaStream_t s) {
  dim3 grid((unsigned)cdiv(nt, CX_BI), (unsigned)nvec);
  rbf_cross_kernel<<<grid, CX_BI, 0, s>>>(tg, nt, ldt, pts, n, ldp, d, sigma, v, out, kind);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

int32_t op_matvec_residual(const nys_operator* op, double mu, const double* p, double* v,
                           const int* skip, void* work, cudaStream_t s) {
  if (op->kind == NYS_OP_RBF && op->d <= 64) {
    Scratch sc(s);
    double* dm;
    NYS_TRY(sc.get(&dm, 1));
    NYS_CUDA_TRY(cudaMemcpyAsync(dm, &mu, sizeof(double), cudaMemcpyHostToDevice, s));
    NYS_TRY(rbf_residual_products(op, dm, 1, p, v, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    return NYS_OK;
  }
  if (op->kind != NYS_OP_GRAM) return op_matvec_f64(op, mu, p, v, skip, work, s);
  if (work) return gram_matvec<double, double, double>(op, mu, p, v, skip, work, s, true);
  Scratch sc(s);
  unsigned char* w;
  NYS_TRY(sc.get(&w, op_matvec_work_bytes(op, true)));
  NYS_CUDA_TRY(cudaMemsetAsync(w, 0, 256, s));
  return gram_matvec<double, double, double>(op, mu, p, v, skip, w, s, true);
}

}  // namespace nys

// ============================================================ allocation-free ridge matvec
//
// nys_gram_matvec_f32_noalloc: the fused ridge matvec above for callers that
// cannot allocate device memory.  Its scratch (the per-CTA partial n-vectors
// and the timeout word) lives in one file-scope device array, so the call
// needs no cudaMalloc.  The array is shared by every call on a device and
// keeps the last call's contents.

namespace {

// 256-byte header (timeout word) + up to 2^20 partial floats (4 MiB).
constexpr size_t kNoAllocHeaderFloats = 64;
constexpr size_t kNoAllocPartialFloats = size_t(1) << 20;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocHeaderFloats + kNoAllocPartialFloats];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[128] = {nullptr};

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol itself is only a host-side stand-in, so the address is looked
// up once per device (with that device current) and cached.  The cache is
// valid for the life of the device's primary context: cudaDeviceReset
// destroys the array with the context, and this entry point must not be
// called after it.
int32_t noalloc_scratch_address(void** out) {
  int dev = 0;
  NYS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return NYS_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    NYS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return NYS_OK;
}

}  // namespace

extern "C" int32_t nys_gram_matvec_f32_noalloc(const nys_operator* op, double mu, const float* x,
                                               float* y, void* stream) {
  using namespace nys;
  if (!op || !x || !y || x == y) return NYS_ERR_ARG;
  if (op->kind != NYS_OP_GRAM || op->dtype != NYS_F32 || !op->data || op->m <= 0 || op->n <= 0)
    return NYS_ERR_ARG;
  if (!(mu >= 0.0) || !std::isfinite(mu)) return NYS_ERR_ARG;
  if (((uintptr_t)x & 15u) || ((uintptr_t)y & 15u)) return NYS_ERR_ARG;
  GramPlan g = gram_plan(op);  // needs ld == n, n % 4 == 0, 16-byte aligned X
  if (!g.fused) return NYS_ERR_ARG;
  if ((size_t)g.grid * (size_t)op->n > kNoAllocPartialFloats) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  NYS_TRY(noalloc_scratch_address(&base));
  int* err = reinterpret_cast<int*>(base);
  float* part = reinterpret_cast<float*>(base) + kNoAllocHeaderFloats;
  NYS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  switch (g.ng) {
    case 1: NYS_TRY((gram_fused_launch<float, float, 1>(op, g, x, part, err, nullptr, s))); break;
    case 2: NYS_TRY((gram_fused_launch<float, float, 2>(op, g, x, part, err, nullptr, s))); break;
    case 4: NYS_TRY((gram_fused_launch<float, float, 4>(op, g, x, part, err, nullptr, s))); break;
    default: NYS_TRY((gram_fused_launch<float, float, 8>(op, g, x, part, err, nullptr, s))); break;
  }
  // the timeout word doubles as the reduction's skip word: after an expired
  // wait y is left as it was instead of summing incomplete partials
  gram_reduce_kernel<float, float, float><<<(unsigned)cdiv(op->n, 32), 256, 0, s>>>(
      part, g.grid, op->n, mu, x, y, err); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  int h_err = 0;
  NYS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return h_err ? NYS_ERR_TIMEOUT : NYS_OK;
}

