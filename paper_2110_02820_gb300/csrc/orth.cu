// Orthonormality defect of an FP32 factor and the corrected preconditioner
// coefficients.
//
// Eq. (5.3) applies P^{-1} = I + U (D - I) U^T with D = diag((lam_ell + mu) /
// (lam_i + mu)), which is the intended operator only when U^T U = I.  A U
// stored in FP32 has U^T U = I + E with ||E||_2 ~ 1e-7 sqrt(ell), and in a top
// eigen-direction u_1 the term U (D - I) U^T then leaves ~||E|| lambda_1 where
// the operator should leave lambda_ell + mu: once (lambda_ell + mu) / lambda_1
// falls below ||E||, PCG stalls.  The corrected apply uses the orthonormal
// basis V = U G^{-1/2} (G = I + E) of the same range:
//
//   P^{-1} = I + V (D - I) V^T = I + U M U^T,
//   M = G^{-1/2} (D - I) G^{-1/2} = C - (E C + C E) / 2 + O(E^2),   C = D - I,
//
// so the ell coefficients w = U^T r become w' = c.w - (c.(E w) + E (c.w)) / 2
// (c the diagonal of C); the dropped O(E^2) terms are ~1e-10.  E itself is
// formed once per factor in double-FP32 arithmetic (exact FP32 products,
// TwoSum accumulation per 32-row chunk merged into a renormalised running
// sum), accurate to ~1e-13 absolute.

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

constexpr int OT = 64;     // output tile (OT x OT entries of G per block)
constexpr int OK = 32;     // rows of U per chunk
constexpr int OTH = 256;   // threads: 16 x 16, each 4 x 4 outputs

__device__ __forceinline__ void ts(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// part[z][i][j] = sum over rows [z * rows_per, ...) of U[k][i] U[k][j] as
// (hi, lo) double-float pairs.
__global__ void __launch_bounds__(OTH)
syrk_dfl_kernel(const float* __restrict__ U, int64_t n, int64_t ell, int64_t rows_per,
                float2* __restrict__ part) {
  __shared__ __align__(16) float ua[OK][OT], ub[OK][OT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * OT, j0 = (int64_t)blockIdx.x * OT;
  const int64_t k_begin = (int64_t)blockIdx.z * rows_per;
  const int64_t k_end = (n < k_begin + rows_per) ? n : k_begin + rows_per;
  float gh[4][4], gl[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) gh[a][b] = gl[a][b] = 0.f;
  for (int64_t k0 = k_begin; k0 < k_end; k0 += OK) {
    __syncthreads();
    for (int e = threadIdx.x; e < OK * OT; e += OTH) {
      const int r = e / OT, c = e - r * OT;
      const int64_t k = k0 + r;
      const bool okr = k < k_end;
      ua[r][c] = (okr && i0 + c < ell) ? U[k * ell + i0 + c] : 0.f;
      ub[r][c] = (okr && j0 + c < ell) ? U[k * ell + j0 + c] : 0.f;
    }
    __syncthreads();
    float ah[4][4], al[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) ah[a][b] = al[a][b] = 0.f;
    for (int r = 0; r < OK; ++r) {
      const float4 x = *reinterpret_cast<const float4*>(&ua[r][ty * 4]);
      const float4 y = *reinterpret_cast<const float4*>(&ub[r][tx * 4]);
      const float xa[4] = {x.x, x.y, x.z, x.w}, yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float p = __fmul_rn(xa[a], yb[b]);
          const float pe = __fmaf_rn(xa[a], yb[b], -p);
          float s, e;
          ts(ah[a][b], p, s, e);
          ah[a][b] = s;
          al[a][b] = __fadd_rn(al[a][b], __fadd_rn(e, pe));
        }
    }
    // merge the chunk into the running sums, renormalised
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        float s, e;
        ts(gh[a][b], ah[a][b], s, e);
        const float t = __fadd_rn(gl[a][b], __fadd_rn(al[a][b], e));
        const float h = __fadd_rn(s, t);
        gl[a][b] = __fsub_rn(t, __fsub_rn(h, s));
        gh[a][b] = h;
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
      if (i < ell && j < ell)
        part[((int64_t)blockIdx.z * ell + i) * ell + j] = make_float2(gh[a][b], gl[a][b]);
    }
}

// E[i][j] = sum_z part[z][i][j] - delta_ij (FP64 sum of the pairs, fixed order)
__global__ void syrk_finish_kernel(const float2* __restrict__ part, int nz, int64_t ell,
                                   float* __restrict__ E) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ell * ell) return;
  double s = 0.0;
  for (int z = 0; z < nz; ++z) {
    const float2 v = part[(int64_t)z * ell * ell + e];
    s += (double)v.x + (double)v.y;
  }
  const int64_t i = e / ell, j = e - i * ell;
  if (i == j) s -= 1.0;
  E[e] = (float)s;
}

}  // namespace

int32_t orth_defect_f32(const float* U, int64_t n, int64_t ell, float* E, cudaStream_t s) {
  const int64_t tiles = cdiv(ell, OT);
  const int64_t want = 2 * (int64_t)num_sms();
  int64_t nz = std::max<int64_t>(1, want / (tiles * tiles));
  nz = std::min<int64_t>(nz, std::max<int64_t>(1, n / (4 * OK)));
  const int64_t rows_per = cdiv(cdiv(n, nz), OK) * OK;
  nz = cdiv(n, rows_per);
  Scratch sc(s);
  float2* part;
  NYS_TRY(sc.get(&part, (size_t)nz * ell * ell));
  syrk_dfl_kernel<<<dim3((unsigned)tiles, (unsigned)tiles, (unsigned)nz), OTH, 0, s>>>(
      U, n, ell, rows_per, part);
  count_launch();
  syrk_finish_kernel<<<(unsigned)cdiv(ell * ell, 256), 256, 0, s>>>(part, (int)nz, ell, E);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

}  // namespace nys
