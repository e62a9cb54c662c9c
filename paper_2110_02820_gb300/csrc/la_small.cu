// Small dense FP64 linear algebra on ell x ell matrices (ell <= 4096):
// Cholesky and triangular inverse.  These carry the ell x ell core of
// Algorithm 1 (Sec. 2.2): chol(Omega^T Y_nu) and the triangular factors of
// the CholeskyQR passes; the SVD of the small factor R is in svd_small.cu.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so these kernels
// keep the ell x ell working set in L2/shared memory and spread each step
// over many SMs; the work is O(ell^3), tiny next to the n x ell passes.

#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace nys {

// ============================================================ Cholesky (upper)

constexpr int CH_NB = 32;

// 1/sqrt(d) for finite d > 0 in FP64 without a division or a square root:
// d = m 4^e with m in [1, 4) (exact exponent arithmetic), a single-precision
// estimate of 1/sqrt(m) (about 2^-22 relative), then two Newton-Raphson steps
// for f(y) = y^-2 - m, y <- y + y (1 - m y^2) / 2, each of which squares the
// relative error (2^-44, then below the FP64 rounding), and the scale 2^-e.
__device__ __forceinline__ double rsqrt_newton(double d) {
  int ex;
  double m = frexp(d, &ex);  // d = m 2^ex, m in [0.5, 1)
  if (ex & 1) {
    m *= 2.0;  // m in [1, 2), ex even after the shift
    ex -= 1;
  } else {
    m *= 4.0;  // m in [2, 4)
    ex -= 2;
  }
  double y = (double)rsqrtf((float)m);
  double h = fma(-m * y, y, 1.0);
  y = fma(0.5 * y, h, y);
  h = fma(-m * y, y, 1.0);
  y = fma(0.5 * y, h, y);
  return ldexp(y, -ex / 2);
}

// 1/d for finite d > 0 in FP64 without a division: d = m 2^e with m in
// [0.5, 1) (exact exponent arithmetic), a single-precision estimate of 1/m
// (about 2^-23 relative), two Newton-Raphson steps y <- y + y (1 - m y), each
// squaring the relative error, and the scale 2^-e.
__device__ __forceinline__ double recip_newton(double d) {
  int ex;
  const double m = frexp(d, &ex);
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)m));
  double y = (double)yf;
  double h = fma(-m, y, 1.0);
  y = fma(y, h, y);
  h = fma(-m, y, 1.0);
  y = fma(y, h, y);
  return ldexp(y, -ex);
}

// Factor the diagonal block D = M[k:k+nb, k:k+nb] in place: D = C_kk^T C_kk.
// 32 warps: warp r owns row r of the block in shared memory, lane c column c
// (the upper triangle).  The elimination runs without square roots (D =
// L diag(d) L^T form): at step j the lanes of warp j form the pivot's
// reciprocal (recip_newton: GB300 runs FP64 division and square root as long
// dependent chains, and each FP64 warp instruction occupies the SM
// sub-partition's FP64 unit for many cycles) and the scaled row W_j = D_j / d_j;
// after one barrier every warp r > j updates its row, D_rc -= D_jr W_jc, one
// FMA per thread, so the FP64 work of a step spreads over the four sub-
// partitions.  Only the pivot chain is sequential.  At the end C_jc = D_jc /
// sqrt(d_j) (C_jj = sqrt(d_j)) for all entries at once.
__global__ void __launch_bounds__(32 * CH_NB) chol_diag_kernel(double* M, int64_t ell, int64_t k,
                                                               int nb, int* info) {
  if (*info != 0) return;
  __shared__ double D[CH_NB][CH_NB + 1];
  __shared__ double W[CH_NB][CH_NB + 1];
  __shared__ int s_bad;
  const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
  D[r][c] = (r < nb && c < nb) ? M[(k + r) * ell + k + c] : (r == c ? 1.0 : 0.0);
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (r == j) {
      const double d = D[j][j];  // final: row j took its last update at step j - 1
      if (!(d > 0.0) || !isfinite(d)) {
        if (c == 0) s_bad = (int)(k + j + 1);
      } else if (c > j) {
        W[j][c] = D[j][c] * recip_newton(d);
      }
    }
    __syncthreads();
    if (s_bad) break;
    if (r > j && c >= r) D[r][c] = fma(-D[j][r], W[j][c], D[r][c]);
  }
  if (s_bad) {
    if (threadIdx.x == 0) atomicCAS(info, 0, s_bad);
    return;
  }
  // row r is final once warp r has passed step r - 1 (its own updates)
  if (r < nb && c < nb) {
    double v = 0.0;
    if (c >= r) {
      const double dr = D[r][r];
      const double sr = rsqrt_newton(dr);
      v = (c == r) ? dr * sr : D[r][c] * sr;
    }
    M[(k + r) * ell + k + c] = v;
  }
}

// Row panel: C[k:k+nb, c] = C_kk^{-T} M[k:k+nb, c] for c >= k + nb (forward
// substitution with the lower-triangular C_kk^T).  One warp per column: lane
// r holds row r; at step r lane r finishes x_r, broadcasts it, and the lanes
// below subtract its contribution.
__global__ void chol_panel_kernel(double* M, int64_t ell, int64_t k, int nb, const int* info) {
  if (*info != 0) return;
  __shared__ double Ck[CH_NB][CH_NB + 1];
  __shared__ double dinv[CH_NB];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    Ck[r][c] = M[(k + r) * ell + k + c];
  }
  __syncthreads();
  // reciprocal pivots once per block: the substitution then multiplies
  if (threadIdx.x < nb) {
    const double dd = Ck[threadIdx.x][threadIdx.x];
    const double rs = rsqrt_newton(dd);
    dinv[threadIdx.x] = rs * rs;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t c = k + nb + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ell) return;
  double m = (lane < nb) ? M[(k + lane) * ell + c] : 0.0;
  for (int r = 0; r < nb; ++r) {
    double xr = (lane == r) ? m * dinv[r] : 0.0;
    xr = __shfl_sync(0xffffffffu, xr, r);
    if (lane == r) m = xr;
    else if (lane > r && lane < nb) m -= Ck[r][lane] * xr;
  }
  if (lane < nb) M[(k + lane) * ell + c] = m;
}

// Trailing update of the upper triangle: M[i, j] -= sum_t C[k+t, i] C[k+t, j]
// for k+nb <= i <= j.  32 x 32 output tiles, lower tiles skipped.
__global__ void chol_trail_kernel(double* M, int64_t ell, int64_t k, int nb, const int* info) {
  if (*info != 0) return;
  const int64_t base = k + nb;
  const int64_t ti = base + (int64_t)blockIdx.y * 32, tj = base + (int64_t)blockIdx.x * 32;
  if (tj + 31 < ti) return;  // tile strictly below the diagonal
  __shared__ double Pi[CH_NB][33], Pj[CH_NB][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < nb; r += 8) {
    Pi[r][tx] = (ti + tx < ell) ? M[(k + r) * ell + ti + tx] : 0.0;
    Pj[r][tx] = (tj + tx < ell) ? M[(k + r) * ell + tj + tx] : 0.0;
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    int64_t i = ti + rr, j = tj + tx;
    if (i < ell && j < ell && j >= i) {
      double acc = 0.0;
      for (int t = 0; t < nb; ++t) acc += Pi[t][rr] * Pj[t][tx];
      M[i * ell + j] -= acc;
    }
  }
}

__global__ void zero_lower_kernel(double* M, int64_t ell) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ell * ell) return;
  int64_t i = e / ell, j = e % ell;
  if (j < i) M[e] = 0.0;
}

int32_t chol_upper(double* M, int64_t ell, int* d_info, cudaStream_t s) {
  NYS_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  for (int64_t k = 0; k < ell; k += CH_NB) {
    int nb = (int)((ell - k < CH_NB) ? ell - k : CH_NB);
    chol_diag_kernel<<<1, 32 * CH_NB, 0, s>>>(M, ell, k, nb, d_info); count_launch();
    int64_t rest = ell - k - nb;
    if (rest > 0) {
      chol_panel_kernel<<<(unsigned)cdiv(rest, 8), 256, 0, s>>>(M, ell, k, nb, d_info); count_launch();
      unsigned t = (unsigned)cdiv(rest, 32);
      chol_trail_kernel<<<dim3(t, t), dim3(32, 8), 0, s>>>(M, ell, k, nb, d_info); count_launch();
    }
  }
  zero_lower_kernel<<<(unsigned)cdiv(ell * ell, 256), 256, 0, s>>>(M, ell); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// ============================================================ triangular inverse

__global__ void transpose_kernel(const double* in, double* out, int64_t rows, int64_t cols) {
  __shared__ double tile[32][33];
  int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    int64_t i = by + r, j = bx + threadIdx.x;
    if (i < rows && j < cols) tile[r][threadIdx.x] = in[i * cols + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    int64_t i = bx + r, j = by + threadIdx.x;  // out is cols x rows
    if (i < cols && j < rows) out[i * rows + j] = tile[threadIdx.x][r];
  }
}

// Column j of X = C^{-1} by column-oriented back substitution on CT = C^T
// (row t of CT = column t of C, contiguous): with r_i = sum_{t>i} C_it x_t,
// x_i = (delta_ij - r_i) / C_ii for i = j, j-1, ..., 0.  One warp per column;
// r lives in shared memory, and the part of row t-1 of CT that this lane
// needs (first TI_PF entries) is loaded while step t runs, so a step does not
// wait on an L2 round trip.  Writes XT[j][i] = X[i][j].
constexpr int TI_WARPS = 4;
constexpr int TI_PF = 16;
__global__ void __launch_bounds__(32 * TI_WARPS)
tri_inv_cols2_kernel(const double* __restrict__ CT, const double* __restrict__ C, double* XT,
                     int64_t ell) {
  extern __shared__ double rsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // 1 / C_ii for every i, once per block: each step of the chain below then
  // waits on shared memory only, not on an L2 load of the diagonal
  double* dinv = rsm + (int64_t)TI_WARPS * ell;
  for (int64_t i = threadIdx.x; i < ell; i += blockDim.x) dinv[i] = 1.0 / C[i * ell + i];
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * TI_WARPS + wib;
  if (j >= ell) return;
  double* r = rsm + (int64_t)wib * ell;
  double* x = XT + j * ell;
  for (int64_t i = lane; i < ell; i += 32) {
    r[i] = 0.0;
    x[i] = 0.0;
  }
  __syncwarp();
  double xt = dinv[j];
  if (lane == 0) x[j] = xt;
  double pf[TI_PF];
  {
    const double* row = CT + j * ell;
#pragma unroll
    for (int q = 0; q < TI_PF; ++q) {
      const int64_t i = lane + 32 * q;
      pf[q] = (i < j) ? row[i] : 0.0;
    }
  }
  for (int64_t t = j; t >= 1; --t) {
    // r_i -= C[i][t] x_t for i < t, using the prefetched part of row t of CT
    const double* row = CT + t * ell;
    double nxt[TI_PF];
    const double* nrow = CT + (t - 1) * ell;
#pragma unroll
    for (int q = 0; q < TI_PF; ++q) {
      const int64_t i = lane + 32 * q;
      nxt[q] = (i < t - 1) ? nrow[i] : 0.0;
      if (i < t) r[i] = fma(pf[q], xt, r[i]);
    }
    for (int64_t i = lane + 32 * TI_PF; i < t; i += 32) r[i] = fma(row[i], xt, r[i]);
    __syncwarp();
    const int64_t i1 = t - 1;
    xt = -r[i1] * dinv[i1];
    if (lane == 0) x[i1] = xt;
#pragma unroll
    for (int q = 0; q < TI_PF; ++q) pf[q] = nxt[q];
    __syncwarp();
  }
}

// ---- the same inverse in double-FP32 arithmetic (Dekker 1971) on the FP32
// pipes, for the mixed-precision path, whose products with C^{-1} run in FP32:
// a value is an unevaluated pair hi + lo of FP32 numbers (~2^-48 relative).
// The column chain is the same; a step's FP64 FMAs, each occupying the FP64
// unit of an SM sub-partition for many cycles on GB300, become ~11 FP32
// operations with short latencies.
struct Dfl {
  float hi, lo;
};

__device__ __forceinline__ Dfl dfl_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

// r + a b (a b formed exactly in its high part by an FMA two-product, the
// cross terms hi.lo added, lo.lo dropped; the sum by Knuth's TwoSum)
__device__ __forceinline__ Dfl dfl_fma(Dfl a, Dfl b, Dfl r) {
  const float ph = a.hi * b.hi;
  float pl = fmaf(a.hi, b.hi, -ph);
  pl = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pl));
  const float s = r.hi + ph;
  const float bb = s - r.hi;
  float e = (r.hi - (s - bb)) + (ph - bb);
  e += r.lo + pl;
  const float h = s + e;
  return {h, e - (h - s)};
}

__device__ __forceinline__ Dfl dfl_mul(Dfl a, Dfl b) {
  const float ph = a.hi * b.hi;
  float pl = fmaf(a.hi, b.hi, -ph);
  pl = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pl));
  const float h = ph + pl;
  return {h, pl - (h - ph)};
}

// CTf[t][i] = split(C[i][t]) (the transpose as double-FP32 pairs) and
// dinvf[i] = split(1 / C_ii)
__global__ void tri_split_kernel(const double* __restrict__ C, float2* __restrict__ CTf,
                                 float2* __restrict__ dinvf, int64_t ell) {
  __shared__ double tile[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = by + r, j = bx + threadIdx.x;
    if (i < ell && j < ell) tile[r][threadIdx.x] = C[i * ell + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t t = bx + r, i = by + threadIdx.x;  // CTf[t][i] = C[i][t]
    if (t < ell && i < ell) {
      const double v = tile[threadIdx.x][r];
      const Dfl d = dfl_from(v);
      CTf[t * ell + i] = make_float2(d.hi, d.lo);
      if (t == i) {
        const Dfl q = dfl_from(1.0 / v);
        dinvf[i] = make_float2(q.hi, q.lo);
      }
    }
  }
}

// Column j of X = C^{-1} by back substitution, as tri_inv_cols2_kernel, in
// double-FP32; writes X[i][j] (FP64) for i <= j and zero below.
constexpr int TD_WARPS = 4;
constexpr int TD_PF = 16;
__global__ void __launch_bounds__(32 * TD_WARPS)
tri_inv_dfl_kernel(const float2* __restrict__ CTf, const float2* __restrict__ dinvf, double* X,
                   int64_t ell) {
  extern __shared__ float2 rsf[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * TD_WARPS + wib;
  if (j >= ell) return;
  float2* r = rsf + (int64_t)wib * ell;
  for (int64_t i = lane; i < ell; i += 32) {
    r[i] = make_float2(0.f, 0.f);
    if (i > j) X[i * ell + j] = 0.0;
  }
  __syncwarp();
  const float2 d0 = dinvf[j];
  Dfl xt = {d0.x, d0.y};
  if (lane == 0) X[j * ell + j] = (double)xt.hi + (double)xt.lo;
  float2 pf[TD_PF];
  {
    const float2* row = CTf + j * ell;
#pragma unroll
    for (int q = 0; q < TD_PF; ++q) {
      const int64_t i = lane + 32 * q;
      pf[q] = (i < j) ? row[i] : make_float2(0.f, 0.f);
    }
  }
  for (int64_t t = j; t >= 1; --t) {
    // r_i += C[i][t] x_t for i < t (the sign is applied when x is formed)
    const float2* row = CTf + t * ell;
    const float2* nrow = CTf + (t - 1) * ell;
    float2 nxt[TD_PF];
#pragma unroll
    for (int q = 0; q < TD_PF; ++q) {
      const int64_t i = lane + 32 * q;
      nxt[q] = (i < t - 1) ? nrow[i] : make_float2(0.f, 0.f);
      if (i < t) {
        const float2 ri = r[i];
        const Dfl v = dfl_fma({pf[q].x, pf[q].y}, xt, {ri.x, ri.y});
        r[i] = make_float2(v.hi, v.lo);
      }
    }
    for (int64_t i = lane + 32 * TD_PF; i < t; i += 32) {
      const float2 ri = r[i], ci = row[i];
      const Dfl v = dfl_fma({ci.x, ci.y}, xt, {ri.x, ri.y});
      r[i] = make_float2(v.hi, v.lo);
    }
    __syncwarp();
    const int64_t i1 = t - 1;
    const float2 rr = r[i1], dd = dinvf[i1];
    xt = dfl_mul({-rr.x, -rr.y}, {dd.x, dd.y});
    if (lane == 0) X[i1 * ell + j] = (double)xt.hi + (double)xt.lo;
#pragma unroll
    for (int q = 0; q < TD_PF; ++q) pf[q] = nxt[q];
    __syncwarp();
  }
}

int32_t tri_inv_upper_dfl(const double* C, double* X, int64_t ell, cudaStream_t s) {
  Scratch sc(s);
  float2 *CTf, *dinvf;
  NYS_TRY(sc.get(&CTf, ell * ell));
  NYS_TRY(sc.get(&dinvf, ell));
  dim3 g((unsigned)cdiv(ell, 32), (unsigned)cdiv(ell, 32));
  tri_split_kernel<<<g, dim3(32, 8), 0, s>>>(C, CTf, dinvf, ell); count_launch();
  const size_t sh = (size_t)TD_WARPS * ell * sizeof(float2);
  if (sh > 48 * 1024)
    NYS_CUDA_TRY(cudaFuncSetAttribute(tri_inv_dfl_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  tri_inv_dfl_kernel<<<(unsigned)cdiv(ell, TD_WARPS), 32 * TD_WARPS, sh, s>>>(CTf, dinvf, X, ell);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// ---- blocked Cholesky in double-FP32 arithmetic, for the mixed-precision
// path (its shifted Grams are conditioned for FP32 data, far inside the
// ~2^-48 of double-FP32).  Same three launches per 32-column step as
// chol_upper; M stays FP64 in memory, each kernel splits what it reads into
// FP32 pairs and rounds what it writes back to FP64.

__device__ __forceinline__ Dfl dfl_neg(Dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ double dfl_to(Dfl a) { return (double)a.hi + (double)a.lo; }

// 1/d for d > 0: FP32 estimate, one Newton-Raphson step y + y (1 - d y)
// with the residual 1 - d y formed in double-FP32 (~2^-46 relative)
__device__ __forceinline__ Dfl dfl_recip(Dfl d) {
  float y0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(d.hi));
  const float ph = d.hi * y0;
  const float pl = fmaf(d.hi, y0, -ph);
  const float e = ((1.0f - ph) - pl) - d.lo * y0;
  const float yl = y0 * e;
  const float h = y0 + yl;
  return {h, yl - (h - y0)};
}

// Diagonal block, as chol_diag_kernel (32 warps, one element per thread, no
// square root on the pivot chain), in double-FP32.
__global__ void __launch_bounds__(32 * CH_NB) chol_diag_dfl_kernel(double* M, int64_t ell,
                                                                   int64_t k, int nb, int* info) {
  if (*info != 0) return;
  __shared__ float2 D[CH_NB][CH_NB + 1];
  __shared__ float2 W[CH_NB][CH_NB + 1];
  __shared__ int s_bad;
  const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
  {
    const double v = (r < nb && c < nb) ? M[(k + r) * ell + k + c] : (r == c ? 1.0 : 0.0);
    const Dfl d = dfl_from(v);
    D[r][c] = make_float2(d.hi, d.lo);
  }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (r == j) {
      const float2 dj = D[j][j];
      if (!(dj.x > 0.f) || !isfinite(dj.x)) {
        if (c == 0) s_bad = (int)(k + j + 1);
      } else if (c > j) {
        const Dfl y = dfl_recip({dj.x, dj.y});
        const float2 djc = D[j][c];
        const Dfl w = dfl_mul({djc.x, djc.y}, y);
        W[j][c] = make_float2(w.hi, w.lo);
      }
    }
    __syncthreads();
    if (s_bad) break;
    if (r > j && c >= r) {
      const float2 a = D[j][r], b = W[j][c], m = D[r][c];
      const Dfl v = dfl_fma(dfl_neg({a.x, a.y}), {b.x, b.y}, {m.x, m.y});
      D[r][c] = make_float2(v.hi, v.lo);
    }
  }
  if (s_bad) {
    if (threadIdx.x == 0) atomicCAS(info, 0, s_bad);
    return;
  }
  if (r < nb && c < nb) {
    double v = 0.0;
    if (c >= r) {
      const float2 drr = D[r][r];
      const double dr = dfl_to({drr.x, drr.y});
      const double sr = rsqrt_newton(dr);
      const float2 drc = D[r][c];
      v = (c == r) ? dr * sr : dfl_to({drc.x, drc.y}) * sr;
    }
    M[(k + r) * ell + k + c] = v;
  }
}

// Row panel, as chol_panel_kernel, in double-FP32.
__global__ void chol_panel_dfl_kernel(double* M, int64_t ell, int64_t k, int nb, const int* info) {
  if (*info != 0) return;
  __shared__ float2 Ck[CH_NB][CH_NB + 1];
  __shared__ float2 dinv[CH_NB];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    const Dfl d = dfl_from(M[(k + r) * ell + k + c]);
    Ck[r][c] = make_float2(d.hi, d.lo);
  }
  if (threadIdx.x < nb) {
    const Dfl q = dfl_from(1.0 / M[(k + threadIdx.x) * ell + k + threadIdx.x]);
    dinv[threadIdx.x] = make_float2(q.hi, q.lo);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t c = k + nb + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ell) return;
  Dfl m = dfl_from((lane < nb) ? M[(k + lane) * ell + c] : 0.0);
  for (int r = 0; r < nb; ++r) {
    Dfl xr = {0.f, 0.f};
    if (lane == r) xr = dfl_mul(m, {dinv[r].x, dinv[r].y});
    xr.hi = __shfl_sync(0xffffffffu, xr.hi, r);
    xr.lo = __shfl_sync(0xffffffffu, xr.lo, r);
    if (lane == r) {
      m = xr;
    } else if (lane > r && lane < nb) {
      const float2 ck = Ck[r][lane];
      m = dfl_fma(dfl_neg({ck.x, ck.y}), xr, m);
    }
  }
  if (lane < nb) M[(k + lane) * ell + c] = dfl_to(m);
}

// Trailing update of the upper triangle, as chol_trail_kernel, with the
// 32-term sums in double-FP32.
__global__ void chol_trail_dfl_kernel(double* M, int64_t ell, int64_t k, int nb, const int* info) {
  if (*info != 0) return;
  const int64_t base = k + nb;
  const int64_t ti = base + (int64_t)blockIdx.y * 32, tj = base + (int64_t)blockIdx.x * 32;
  if (tj + 31 < ti) return;  // tile strictly below the diagonal
  __shared__ float2 Pi[CH_NB][33], Pj[CH_NB][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < nb; r += 8) {
    const Dfl a = dfl_from((ti + tx < ell) ? M[(k + r) * ell + ti + tx] : 0.0);
    const Dfl b = dfl_from((tj + tx < ell) ? M[(k + r) * ell + tj + tx] : 0.0);
    Pi[r][tx] = make_float2(a.hi, a.lo);
    Pj[r][tx] = make_float2(b.hi, b.lo);
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t i = ti + rr, j = tj + tx;
    if (i < ell && j < ell && j >= i) {
      Dfl acc = {0.f, 0.f};
      for (int t = 0; t < nb; ++t) {
        const float2 a = Pi[t][rr], b = Pj[t][tx];
        acc = dfl_fma({a.x, a.y}, {b.x, b.y}, acc);
      }
      M[i * ell + j] -= dfl_to(acc);
    }
  }
}

int32_t chol_upper_dfl(double* M, int64_t ell, int* d_info, cudaStream_t s) {
  NYS_CUDA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  for (int64_t k = 0; k < ell; k += CH_NB) {
    int nb = (int)((ell - k < CH_NB) ? ell - k : CH_NB);
    chol_diag_dfl_kernel<<<1, 32 * CH_NB, 0, s>>>(M, ell, k, nb, d_info); count_launch();
    int64_t rest = ell - k - nb;
    if (rest > 0) {
      chol_panel_dfl_kernel<<<(unsigned)cdiv(rest, 8), 256, 0, s>>>(M, ell, k, nb, d_info);
      count_launch();
      unsigned t = (unsigned)cdiv(rest, 32);
      chol_trail_dfl_kernel<<<dim3(t, t), dim3(32, 8), 0, s>>>(M, ell, k, nb, d_info);
      count_launch();
    }
  }
  zero_lower_kernel<<<(unsigned)cdiv(ell * ell, 256), 256, 0, s>>>(M, ell); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

int32_t tri_inv_upper(const double* C, double* X, int64_t ell, cudaStream_t s) {
  Scratch sc(s);
  double *XT, *CT;
  NYS_TRY(sc.get(&XT, ell * ell));
  NYS_TRY(sc.get(&CT, ell * ell));
  dim3 g((unsigned)cdiv(ell, 32), (unsigned)cdiv(ell, 32));
  transpose_kernel<<<g, dim3(32, 8), 0, s>>>(C, CT, ell, ell); count_launch();
  const size_t sh = (size_t)(TI_WARPS + 1) * ell * sizeof(double);
  if (sh > 48 * 1024)
    NYS_CUDA_TRY(cudaFuncSetAttribute(tri_inv_cols2_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  tri_inv_cols2_kernel<<<(unsigned)cdiv(ell, TI_WARPS), 32 * TI_WARPS, sh, s>>>(CT, C, XT, ell);
  count_launch();
  transpose_kernel<<<g, dim3(32, 8), 0, s>>>(XT, X, ell, ell); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

__global__ void symmetrize_kernel(double* M, int64_t ell) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ell * ell) return;
  int64_t i = e / ell, j = e % ell;
  if (j <= i) return;
  double a = M[i * ell + j], b = M[j * ell + i];
  double v = 0.5 * (a + b);
  M[i * ell + j] = v;
  M[j * ell + i] = v;
}

int32_t symmetrize(double* M, int64_t ell, cudaStream_t s) {
  symmetrize_kernel<<<(unsigned)cdiv(ell * ell, 256), 256, 0, s>>>(M, ell); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

__global__ void add_diag_kernel(double* M, int64_t ell, double shift) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ell) M[i * ell + i] += shift;
}

int32_t add_diag(double* M, int64_t ell, double shift, cudaStream_t s) {
  add_diag_kernel<<<(unsigned)cdiv(ell, 256), 256, 0, s>>>(M, ell, shift); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

}  // namespace nys
