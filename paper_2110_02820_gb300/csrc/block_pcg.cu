// Block Nystrom PCG (Sec. 5.2, "Block Nystrom PCG"): O'Leary's block
// conjugate gradient for k right-hand sides of one shifted system
// (A + mu I) X = B, preconditioned by Eq. (5.3), after the initial residual
// block is orthonormalised (the pre-processing of Feng, Owen & Peric, 1995):
//
//   R_0 = B - A_mu X_0 = Q S    Gram-Schmidt with one reorthogonalisation; a
//                               column with no new direction adds no row to S
//   Y = 0, R = Q, Z = P^{-1} R, P = Z, rho = Z^T R
//   repeat:  V = A_mu P;  alpha = (P^T V)^{-1} rho;  Y += P alpha;  R -= V alpha
//            stop when every column j has ||(R S) e_j|| <= tol ||b_j||
//            Z = P^{-1} R;  rho' = Z^T R;  beta = rho^{-1} rho';  P = Z + P beta
//   X = X_0 + Y S
//
// Block vectors are system-major ([k][n]).  The k x k factors come from
// fixed-order partial sums (deterministic) and are solved by Cholesky in FP64
// on the device, so the iterations run without host round trips between the
// status reads.  Mixed precision wraps the FP32 block solve in the
// FP64-residual refinement of the single-system path.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

constexpr int BK = 32;      // widest block
constexpr int BT = 256;     // threads of the streaming kernels
constexpr int GR_TR = 32;   // rows per tile of the Gram kernel
constexpr int UT_TR = 64;   // rows per tile of the U^T R kernel

struct BState {
  int done, status, it, maxit;
  int k1, k;                // directions (rows of S), active columns
  double thresh2[BK];       // (tol ||b_j||)^2
  double res2[BK];          // ||(R S) e_j||^2 after the last step
};

// part[blockIdx.x][a * kb + b] = sum over this block's rows of A[a][i] B[b][i]
template <typename T>
__global__ void __launch_bounds__(BT)
bgram_part_kernel(const T* __restrict__ A, int ka, const T* __restrict__ B, int kb, int64_t n,
                  double* __restrict__ part, const BState* st) {
  if (st && st->done) return;
  __shared__ double as[BK][GR_TR + 1], bs[BK][GR_TR + 1];
  double acc[(BK * BK) / BT] = {};
  const int np = ka * kb;
  for (int64_t r0 = (int64_t)blockIdx.x * GR_TR; r0 < n; r0 += (int64_t)gridDim.x * GR_TR) {
    __syncthreads();
    for (int e = threadIdx.x; e < ka * GR_TR; e += BT) {
      const int a = e / GR_TR, r = e - a * GR_TR;
      as[a][r] = r0 + r < n ? (double)A[a * n + r0 + r] : 0.0;
    }
    for (int e = threadIdx.x; e < kb * GR_TR; e += BT) {
      const int b = e / GR_TR, r = e - b * GR_TR;
      bs[b][r] = r0 + r < n ? (double)B[b * n + r0 + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < (BK * BK) / BT; ++t) {
      const int e = threadIdx.x + t * BT;
      if (e < np) {
        const int a = e / kb, b = e - a * kb;
        double sum = 0.0;
#pragma unroll 8
        for (int r = 0; r < GR_TR; ++r) sum = fma(as[a][r], bs[b][r], sum);
        acc[t] += sum;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < (BK * BK) / BT; ++t) {
    const int e = threadIdx.x + t * BT;
    if (e < np) part[(int64_t)blockIdx.x * np + e] = acc[t];
  }
}

// out[e] = sum_b part[b][e] in block order, e < cnt
__global__ void bsum_kernel(const double* __restrict__ part, int nb, int cnt,
                            double* __restrict__ out, const BState* st) {
  if (st && st->done) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cnt) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * cnt + e];
  out[e] = s;
}

// out[q][i] = cs C[q][i] + ms sum_j A[j][i] M[j][q] for q < ko (M is ka x ko,
// row-major FP64).  Each thread reads its A[.][i] before writing, so out may
// alias A or C.  Arithmetic in FP64 for FP64 data, FP32 otherwise.
template <typename T, typename TO, int KM>
__global__ void __launch_bounds__(BT)
bcomb_kernel(const T* A, int ka, const double* __restrict__ M, int ko, const TO* C, double cs,
             double ms, TO* out, int64_t n, const BState* st) {
  using Acc = typename std::conditional<sizeof(T) == 8 || sizeof(TO) == 8, double, float>::type;
  if (st && st->done) return;
  __shared__ Acc Ms[KM * KM];
  for (int e = threadIdx.x; e < ka * ko; e += BT) Ms[e] = (Acc)(ms * M[e]);
  __syncthreads();
  // the column loop is unrolled only for narrow blocks (a fully unrolled
  // 32 x 32 body costs minutes of compilation for no measurable gain)
  constexpr int QU = KM <= 16 ? KM : 1;
  for (int64_t i = (int64_t)blockIdx.x * BT + threadIdx.x; i < n; i += (int64_t)gridDim.x * BT) {
    Acc a[KM];
#pragma unroll
    for (int j = 0; j < KM; ++j) a[j] = j < ka ? (Acc)A[j * n + i] : (Acc)0;
    // every A[.][i] is in registers before the first store of row i
#pragma unroll QU
    for (int q = 0; q < ko; ++q) {
      Acc v = C ? (Acc)(cs * (double)C[q * n + i]) : (Acc)0;
#pragma unroll
      for (int j = 0; j < KM; ++j)
        if (j < ka) v += a[j] * Ms[j * ko + q];
      out[q * n + i] = (TO)v;
    }
  }
}

// wpart[bx][l][q] = sum over the block's row tiles of U[i][l] R[q][i]
template <typename T, typename TU, int KM>
__global__ void __launch_bounds__(BT)
butr_part_kernel(const TU* __restrict__ U, int64_t n, int64_t ell, const T* __restrict__ R, int k,
                 double* __restrict__ wpart, const BState* st) {
  if (st && st->done) return;
  __shared__ T rs[KM][UT_TR];
  const int64_t l = (int64_t)blockIdx.y * BT + threadIdx.x;
  T acc[KM];
#pragma unroll
  for (int q = 0; q < KM; ++q) acc[q] = (T)0;
  for (int64_t r0 = (int64_t)blockIdx.x * UT_TR; r0 < n; r0 += (int64_t)gridDim.x * UT_TR) {
    __syncthreads();
    for (int e = threadIdx.x; e < KM * UT_TR; e += BT) {
      const int q = e / UT_TR, r = e - q * UT_TR;
      rs[q][r] = (q < k && r0 + r < n) ? R[q * n + r0 + r] : (T)0;
    }
    __syncthreads();
    if (l < ell) {
      const int rows = (int)((n - r0 < UT_TR) ? n - r0 : UT_TR);
      for (int r = 0; r < rows; ++r) {
        const T u = (T)U[(r0 + r) * ell + l];
#pragma unroll
        for (int q = 0; q < KM; ++q) acc[q] += u * rs[q][r];
      }
    }
  }
  if (l < ell)
    for (int q = 0; q < k; ++q) wpart[((int64_t)blockIdx.x * ell + l) * k + q] = (double)acc[q];
}

// w[l][q] = ((lam_ell + mu) / (lam_l + mu) - 1) sum_b wpart[b][l][q]; with an
// orthonormality defect E the raw sums go to wraw and the corrected
// coefficients are formed by bwcorr_kernel.
__global__ void bw_reduce_kernel(const double* __restrict__ wpart, int nb, int64_t ell, int k,
                                 const double* __restrict__ lam, double lam_ell, double mu,
                                 double* __restrict__ w, double* __restrict__ wraw,
                                 const BState* st) {
  if (st && st->done) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ell * k) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += wpart[(int64_t)b * ell * k + e];
  const int64_t l = e / k;
  const double c = (lam_ell + mu) / (lam[l] + mu) - 1.0;
  if (wraw) {
    wraw[e] = s;            // raw U^T r
    wraw[ell * k + e] = c * s;  // c . (U^T r)
  } else {
    w[e] = c * s;
  }
}

// w[i][q] = c_i W_iq - (c_i (E W)_iq + (E (c.W))_iq) / 2, with W and c.W in
// wraw[0 .. ell k) and wraw[ell k .. 2 ell k) (the apply through the
// orthonormal basis U (I + E)^{-1/2}, first order in E): one warp per (i, q).
__global__ void bwcorr_kernel(const float* __restrict__ E, int64_t ell, int k,
                              const double* __restrict__ lam, double lam_ell, double mu,
                              const double* __restrict__ wraw, double* __restrict__ w,
                              const BState* st) {
  if (st && st->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (g >= ell * k) return;
  const int64_t i = g / k;
  const int q = (int)(g - i * k);
  const double* wcw = wraw + ell * k;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t j = lane; j < ell; j += 32) {
    const double e = (double)E[i * ell + j];
    s1 += e * wraw[j * k + q];
    s2 += e * wcw[j * k + q];
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    const double ci = (lam_ell + mu) / (lam[i] + mu) - 1.0;
    w[i * k + q] = ci * wraw[i * k + q] - 0.5 * (ci * s1 + s2);
  }
}

// Z[q][i] = R[q][i] + sum_l U[i][l] w[l][q]: one warp per row
template <typename T, typename TU, int KM>
__global__ void __launch_bounds__(BT)
bz_kernel(const TU* __restrict__ U, int64_t n, int64_t ell, const double* __restrict__ w,
          const T* __restrict__ R, T* __restrict__ Z, int k, const BState* st) {
  if (st && st->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (BT / 32);
  for (int64_t i = ((int64_t)blockIdx.x * BT + threadIdx.x) >> 5; i < n; i += warps) {
    T acc[KM];
#pragma unroll
    for (int q = 0; q < KM; ++q) acc[q] = (T)0;
    for (int64_t l = lane; l < ell; l += 32) {
      const T u = (T)U[i * ell + l];
      const double* wl = w + l * k;
#pragma unroll
      for (int q = 0; q < KM; ++q)
        if (q < k) acc[q] += u * (T)wl[q];
    }
#pragma unroll
    for (int q = 0; q < KM; ++q) {
      if (q < k) {
        const T v = warp_sum(acc[q]);
        if (lane == q) Z[q * n + i] = R[q * n + i] + v;
      }
    }
  }
}

// ---------------------------------------------------------------- k x k FP64 on one thread

// Upper Cholesky in place (row-major k x k, upper triangle read); false on a
// non-positive or non-finite pivot.
__device__ bool chol_small(double* M, int k) {
  for (int j = 0; j < k; ++j) {
    double d = M[j * k + j];
    for (int p = 0; p < j; ++p) d -= M[p * k + j] * M[p * k + j];
    if (!(d > 0.0) || !isfinite(d)) return false;
    d = sqrt(d);
    M[j * k + j] = d;
    for (int c = j + 1; c < k; ++c) {
      double v = M[j * k + c];
      for (int p = 0; p < j; ++p) v -= M[p * k + j] * M[p * k + c];
      M[j * k + c] = v / d;
    }
  }
  return true;
}

// B <- (C^T C)^{-1} B for the upper factor C (k x k) and B k x m (row-major)
__device__ void chol_solve_small(const double* C, int k, double* B, int m) {
  for (int c = 0; c < m; ++c) {
    for (int j = 0; j < k; ++j) {
      double v = B[j * m + c];
      for (int p = 0; p < j; ++p) v -= C[p * k + j] * B[p * m + c];
      B[j * m + c] = v / C[j * k + j];
    }
    for (int j = k - 1; j >= 0; --j) {
      double v = B[j * m + c];
      for (int p = j + 1; p < k; ++p) v -= C[j * k + p] * B[p * m + c];
      B[j * m + c] = v / C[j * k + j];
    }
  }
}

// alpha = (P^T V)^{-1} rho from the partial sums of P^T V.
__global__ void balpha_kernel(const double* __restrict__ part, int nb, const double* rho,
                              double* alpha, BState* st) {
  if (st->done) return;
  __shared__ double G[BK * BK], A[BK * BK];
  const int k1 = st->k1, np = k1 * k1;
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * np + e];
    G[e] = s;
    A[e] = rho[e];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int a = 0; a < k1; ++a)
    for (int b = a + 1; b < k1; ++b) G[a * k1 + b] = 0.5 * (G[a * k1 + b] + G[b * k1 + a]);
  if (!chol_small(G, k1)) {
    st->status = NYS_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  chol_solve_small(G, k1, A, k1);
  for (int e = 0; e < np; ++e) alpha[e] = A[e];
}

// After R -= V alpha: column residuals ||(R S) e_j||^2 from R^T R, the stop
// test, then beta = rho^{-1} rho' (rho' = Z^T R) and rho <- rho'.
__global__ void bbeta_kernel(const double* __restrict__ part_rr, const double* __restrict__ part_zr,
                             int nb, const double* __restrict__ S, double* rho, double* beta,
                             BState* st) {
  if (st->done) return;
  __shared__ double RR[BK * BK], ZR[BK * BK], C[BK * BK];
  const int k1 = st->k1, k = st->k, np = k1 * k1;
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    double s = 0.0, z = 0.0;
    for (int b = 0; b < nb; ++b) {
      s += part_rr[(int64_t)b * np + e];
      z += part_zr[(int64_t)b * np + e];
    }
    RR[e] = s;
    ZR[e] = z;
    C[e] = rho[e];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  st->it += 1;
  bool all = true, finite = true;
  for (int j = 0; j < k; ++j) {
    double v = 0.0;
    for (int a = 0; a < k1; ++a) {
      double t = 0.0;
      for (int b = 0; b < k1; ++b) t += RR[a * k1 + b] * S[b * k + j];
      v += S[a * k + j] * t;
    }
    v = fmax(v, 0.0);
    st->res2[j] = v;
    finite = finite && isfinite(v);
    all = all && v <= st->thresh2[j];
  }
  if (!finite) {
    st->status = NYS_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  if (all) {
    st->status = NYS_OK;
    st->done = 1;
    return;
  }
  if (st->it >= st->maxit) {
    st->status = NYS_ERR_MAXIT;
    st->done = 1;
    return;
  }
  for (int a = 0; a < k1; ++a)
    for (int b = a + 1; b < k1; ++b) C[a * k1 + b] = 0.5 * (C[a * k1 + b] + C[b * k1 + a]);
  if (!chol_small(C, k1)) {
    st->status = NYS_ERR_BREAKDOWN;
    st->done = 1;
    return;
  }
  for (int a = 0; a < k1; ++a)
    for (int b = 0; b < k1; ++b) {
      const double v = 0.5 * (ZR[a * k1 + b] + ZR[b * k1 + a]);
      beta[a * k1 + b] = v;
      rho[a * k1 + b] = v;
    }
  chol_solve_small(C, k1, beta, k1);
}

// ---------------------------------------------------------------- host side

// Partial-sum geometry of the Gram kernel for n rows.
inline int gram_blocks(int64_t n) {
  const int64_t t = cdiv(n, GR_TR * 8);
  const int64_t cap = 2 * num_sms();
  return (int)(t < 1 ? 1 : (t > cap ? cap : t));
}

template <typename T>
int32_t gram(const T* A, int ka, const T* B, int kb, int64_t n, double* part, double* out,
             const BState* st, cudaStream_t s) {
  const int nb = gram_blocks(n);
  bgram_part_kernel<T><<<nb, BT, 0, s>>>(A, ka, B, kb, n, part, st);
  count_launch();
  if (out) {
    bsum_kernel<<<(unsigned)cdiv(ka * kb, 256), 256, 0, s>>>(part, nb, ka * kb, out, st);
    count_launch();
  }
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

template <typename T, typename TO>
int32_t comb(const T* A, int ka, const double* M, int ko, const TO* C, double cs, double ms,
             TO* out, int64_t n, const BState* st, cudaStream_t s) {
  const unsigned g = (unsigned)std::min<int64_t>(cdiv(n, BT), 8 * (int64_t)num_sms());
  const int km = ka > ko ? ka : ko;
  if (km <= 4) bcomb_kernel<T, TO, 4><<<g, BT, 0, s>>>(A, ka, M, ko, C, cs, ms, out, n, st);
  else if (km <= 8) bcomb_kernel<T, TO, 8><<<g, BT, 0, s>>>(A, ka, M, ko, C, cs, ms, out, n, st);
  else if (km <= 16) bcomb_kernel<T, TO, 16><<<g, BT, 0, s>>>(A, ka, M, ko, C, cs, ms, out, n, st);
  else bcomb_kernel<T, TO, 32><<<g, BT, 0, s>>>(A, ka, M, ko, C, cs, ms, out, n, st);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// Z = P^{-1} R (Eq. 5.3) for k columns: two passes over U.
template <typename T, typename TU>
int32_t precond_block(const TU* U, const float* E, const double* lam, int64_t ell, double lam_ell,
                      double mu, int64_t n, int k, const T* R, T* Z, double* wpart, double* w,
                      double* wraw, const BState* st, cudaStream_t s) {
  if (!U || ell == 0) {
    NYS_CUDA_TRY(cudaMemcpyAsync(Z, R, (size_t)k * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return NYS_OK;
  }
  const int nbu = (int)std::min<int64_t>(cdiv(n, UT_TR), num_sms());
  dim3 g1((unsigned)nbu, (unsigned)cdiv(ell, BT));
  const unsigned gz = (unsigned)std::min<int64_t>(cdiv(n, BT / 32), 8 * (int64_t)num_sms());
#define NYS_BLOCK_PRECOND(KM)                                                                 \
  butr_part_kernel<T, TU, KM><<<g1, BT, 0, s>>>(U, n, ell, R, k, wpart, st);                   \
  count_launch();                                                                             \
  bw_reduce_kernel<<<(unsigned)cdiv(ell * k, 256), 256, 0, s>>>(wpart, nbu, ell, k, lam,      \
                                                                 lam_ell, mu, w,              \
                                                                 E ? wraw : nullptr, st);     \
  count_launch();                                                                             \
  if (E) {                                                                                    \
    bwcorr_kernel<<<(unsigned)cdiv(ell * k * 32, 256), 256, 0, s>>>(E, ell, k, lam, lam_ell,  \
                                                                    mu, wraw, w, st);         \
    count_launch();                                                                           \
  }                                                                                           \
  bz_kernel<T, TU, KM><<<gz, BT, 0, s>>>(U, n, ell, w, R, Z, k, st);                           \
  count_launch();
  if (k <= 4) {
    NYS_BLOCK_PRECOND(4)
  } else if (k <= 8) {
    NYS_BLOCK_PRECOND(8)
  } else if (k <= 16) {
    NYS_BLOCK_PRECOND(16)
  } else {
    NYS_BLOCK_PRECOND(32)
  }
#undef NYS_BLOCK_PRECOND
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

size_t precond_wpart_elems(int64_t n, int64_t ell, int k) {
  return (size_t)std::min<int64_t>(cdiv(n, UT_TR), num_sms()) * ell * k;
}

// V = (A + mu I) P for k columns; skipped when *skip != 0.
template <typename T>
int32_t block_matvec(const nys_operator* op, double mu, const double* d_mu, int k, const T* P,
                     T* V, const int* skip, void* work, int* err, cudaStream_t s);

template <>
int32_t block_matvec<float>(const nys_operator* op, double mu, const double* d_mu, int k,
                            const float* P, float* V, const int* skip, void* work, int* err,
                            cudaStream_t s) {
  const int64_t n = op->n;
  if (op->kind == NYS_OP_RBF)
    return op_matvec_batched_f32(op, d_mu, k, P, V, skip, 0, err, nullptr, s);
  for (int q = 0; q < k; ++q) NYS_TRY(op_matvec_f32(op, mu, P + q * n, V + q * n, skip, work, s));
  return NYS_OK;
}

template <>
int32_t block_matvec<double>(const nys_operator* op, double mu, const double* d_mu, int k,
                             const double* P, double* V, const int* skip, void* work, int* err,
                             cudaStream_t s) {
  const int64_t n = op->n;
  (void)d_mu;
  (void)err;
  if (op->kind == NYS_OP_RBF && op->d <= 64) {
    const float* pts = (const float*)op->data;
    return rbf_exact_products(pts, n, op->ld, pts, n, op->ld, op->d, op->sigma, 0, 1, nullptr,
                              mu, k, P, V, skip, s);
  }
  for (int q = 0; q < k; ++q) NYS_TRY(op_matvec_f64(op, mu, P + q * n, V + q * n, skip, work, s));
  return NYS_OK;
}

template <typename T>
double drop_tol();
template <>
double drop_tol<double>() { return 64.0 * 1.1102230246251565e-16; }
template <>
double drop_tol<float>() { return 64.0 * 5.9604644775390625e-08; }

// Block PCG on k columns of B (device [k][n], type T) from X (device [k][n],
// the initial guess when use_x0, else overwritten), to ||(R S) e_j|| <=
// tol ||b_j||.  On return X holds the iterate; it, status[j], rel[j]
// (recurrence residual / ||b_j||) are host outputs.
template <typename T, typename TU>
int32_t run_block(const nys_operator* op, const TU* U, const float* E, const double* lam,
                  int64_t ell, double lam_ell, double mu, int k, const T* B, T* X, bool use_x0,
                  double tol,
                  int maxit, int* it_out, int* status, double* rel, cudaStream_t s) {
  const int64_t n = op->n;
  Scratch sc(s);
  const size_t kn = (size_t)k * n;
  T *R0, *Q, *Y, *R, *Z, *P, *V;
  NYS_TRY(sc.get(&R0, kn));
  NYS_TRY(sc.get(&Q, kn));
  NYS_TRY(sc.get(&Y, kn));
  NYS_TRY(sc.get(&R, kn));
  NYS_TRY(sc.get(&Z, kn));
  NYS_TRY(sc.get(&P, kn));
  NYS_TRY(sc.get(&V, kn));
  const int nbg = gram_blocks(n);
  double *part, *part2, *small, *wpart = nullptr, *w = nullptr, *wraw = nullptr, *d_mu;
  NYS_TRY(sc.get(&part, (size_t)nbg * BK * BK));
  NYS_TRY(sc.get(&part2, (size_t)nbg * BK * BK));
  NYS_TRY(sc.get(&small, 8 * BK * BK));
  NYS_TRY(sc.get(&d_mu, BK));
  if (U && ell > 0) {
    NYS_TRY(sc.get(&wpart, precond_wpart_elems(n, ell, k)));
    NYS_TRY(sc.get(&w, (size_t)ell * k));
    if (E) NYS_TRY(sc.get(&wraw, 2 * (size_t)ell * k));
  }
  double* d_rho = small;
  double* d_alpha = small + BK * BK;
  double* d_beta = small + 2 * BK * BK;
  double* d_S = small + 3 * BK * BK;
  double* d_c = small + 4 * BK * BK;
  double* d_g = small + 5 * BK * BK;
  double* d_m = small + 6 * BK * BK;
  BState* st;
  NYS_TRY(sc.get(&st, 1));
  unsigned char* work;
  NYS_TRY(sc.get(&work, op_matvec_work_bytes(op, sizeof(T) == sizeof(double))));
  NYS_CUDA_TRY(cudaMemsetAsync(work, 0, 256, s));
  int* err = reinterpret_cast<int*>(work);
  {
    std::vector<double> mus(BK, mu);
    NYS_CUDA_TRY(cudaMemcpyAsync(d_mu, mus.data(), BK * sizeof(double), cudaMemcpyHostToDevice, s));
  }

  // ---- R_0 = B - A_mu X_0, column norms of B and R_0
  if (use_x0) {
    NYS_TRY(block_matvec<T>(op, mu, d_mu, k, X, V, nullptr, work, err, s));
    // R0 = B - V: comb with A = V, M = I
    std::vector<double> I((size_t)k * k, 0.0);
    for (int q = 0; q < k; ++q) I[(size_t)q * k + q] = 1.0;
    NYS_CUDA_TRY(cudaMemcpyAsync(d_m, I.data(), I.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    NYS_TRY((comb<T, T>(V, k, d_m, k, B, 1.0, -1.0, R0, n, nullptr, s)));
  } else {
    NYS_CUDA_TRY(cudaMemcpyAsync(R0, B, kn * sizeof(T), cudaMemcpyDeviceToDevice, s));
    NYS_CUDA_TRY(cudaMemsetAsync(X, 0, kn * sizeof(T), s));
  }
  std::vector<double> gb((size_t)k * k), gr((size_t)k * k);
  NYS_TRY(gram<T>(B, k, B, k, n, part, d_g, nullptr, s));
  NYS_CUDA_TRY(cudaMemcpyAsync(gb.data(), d_g, gb.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  NYS_TRY(gram<T>(R0, k, R0, k, n, part, d_c, nullptr, s));
  NYS_CUDA_TRY(cudaMemcpyAsync(gr.data(), d_c, gr.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> bn(k), thresh(k);
  std::vector<int> act;
  for (int j = 0; j < k; ++j) {
    bn[j] = sqrt(fmax(gb[(size_t)j * k + j], 0.0));
    thresh[j] = tol * bn[j];
    const double r = sqrt(fmax(gr[(size_t)j * k + j], 0.0));
    rel[j] = bn[j] > 0 ? r / bn[j] : r;
    status[j] = NYS_OK;
    if (r > thresh[j]) act.push_back(j);
  }
  *it_out = 0;
  const int ka = (int)act.size();
  if (ka == 0) return NYS_OK;
  if (maxit <= 0) {
    for (int j : act) status[j] = NYS_ERR_MAXIT;
    return NYS_OK;
  }
  // active columns gathered into R (contiguous)
  for (int a = 0; a < ka; ++a)
    NYS_CUDA_TRY(cudaMemcpyAsync(R + (size_t)a * n, R0 + (size_t)act[a] * n, n * sizeof(T),
                                 cudaMemcpyDeviceToDevice, s));

  // ---- pre-processing: R = Q S (Gram-Schmidt, one reorthogonalisation)
  std::vector<double> S((size_t)ka * ka, 0.0);  // rows: directions, cols: active columns
  int k1 = 0;
  const double dtol = drop_tol<T>();
  for (int j = 0; j < ka; ++j) {
    T* v = Q + (size_t)k1 * n;
    NYS_CUDA_TRY(cudaMemcpyAsync(v, R + (size_t)j * n, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    const double nrm0 = sqrt(fmax(gr[(size_t)act[j] * k + act[j]], 0.0));
    std::vector<double> c(k1 > 0 ? k1 : 1, 0.0), col(k1 > 0 ? k1 : 1, 0.0);
    for (int pass = 0; pass < 2 && k1 > 0; ++pass) {
      NYS_TRY(gram<T>(Q, k1, v, 1, n, part, d_c, nullptr, s));
      NYS_CUDA_TRY(cudaMemcpyAsync(c.data(), d_c, k1 * sizeof(double), cudaMemcpyDeviceToHost, s));
      NYS_TRY((comb<T, T>(Q, k1, d_c, 1, v, 1.0, -1.0, v, n, nullptr, s)));
      NYS_CUDA_TRY(cudaStreamSynchronize(s));
      for (int a = 0; a < k1; ++a) col[a] += c[a];
    }
    double g = 0.0;
    NYS_TRY(gram<T>(v, 1, v, 1, n, part, d_c, nullptr, s));
    NYS_CUDA_TRY(cudaMemcpyAsync(&g, d_c, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    for (int a = 0; a < k1; ++a) S[(size_t)a * ka + j] = col[a];
    const double nrm = sqrt(fmax(g, 0.0));
    if (nrm > dtol * nrm0) {
      const double inv = 1.0 / nrm;
      NYS_CUDA_TRY(cudaMemcpyAsync(d_c, &inv, sizeof(double), cudaMemcpyHostToDevice, s));
      NYS_TRY((comb<T, T>(v, 1, d_c, 1, nullptr, 0.0, 1.0, v, n, nullptr, s)));
      NYS_CUDA_TRY(cudaStreamSynchronize(s));
      S[(size_t)k1 * ka + j] = nrm;
      ++k1;
    }
  }
  // S as k1 x ka
  std::vector<double> Sk((size_t)k1 * ka);
  for (int a = 0; a < k1; ++a)
    for (int j = 0; j < ka; ++j) Sk[(size_t)a * ka + j] = S[(size_t)a * ka + j];
  NYS_CUDA_TRY(cudaMemcpyAsync(d_S, Sk.data(), Sk.size() * sizeof(double), cudaMemcpyHostToDevice, s));

  BState h;
  memset(&h, 0, sizeof(h));
  h.maxit = maxit;
  h.k1 = k1;
  h.k = ka;
  for (int a = 0; a < ka; ++a) h.thresh2[a] = thresh[act[a]] * thresh[act[a]];
  NYS_CUDA_TRY(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, s));

  // ---- Y = 0, R = Q, Z = P^{-1} R, P = Z, rho = Z^T R
  NYS_CUDA_TRY(cudaMemsetAsync(Y, 0, (size_t)k1 * n * sizeof(T), s));
  NYS_CUDA_TRY(cudaMemcpyAsync(R, Q, (size_t)k1 * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  NYS_TRY((precond_block<T, TU>(U, E, lam, ell, lam_ell, mu, n, k1, R, Z, wpart, w, wraw, st, s)));
  NYS_CUDA_TRY(cudaMemcpyAsync(P, Z, (size_t)k1 * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  NYS_TRY(gram<T>(Z, k1, R, k1, n, part, d_rho, st, s));

  // ---- iterations, status read every `chunk`
  int launched = 0, chunk = 4;
  while (true) {
    for (int c = 0; c < chunk && launched < maxit; ++c, ++launched) {
      NYS_TRY(block_matvec<T>(op, mu, d_mu, k1, P, V, &st->done, work, err, s));
      NYS_TRY(gram<T>(P, k1, V, k1, n, part, nullptr, st, s));
      balpha_kernel<<<1, 1024, 0, s>>>(part, nbg, d_rho, d_alpha, st); count_launch();
      NYS_TRY((comb<T, T>(P, k1, d_alpha, k1, Y, 1.0, 1.0, Y, n, st, s)));
      NYS_TRY((comb<T, T>(V, k1, d_alpha, k1, R, 1.0, -1.0, R, n, st, s)));
      NYS_TRY(gram<T>(R, k1, R, k1, n, part, nullptr, st, s));
      NYS_TRY((precond_block<T, TU>(U, E, lam, ell, lam_ell, mu, n, k1, R, Z, wpart, w, wraw, st, s)));
      NYS_TRY(gram<T>(Z, k1, R, k1, n, part2, nullptr, st, s));
      bbeta_kernel<<<1, 1024, 0, s>>>(part, part2, nbg, d_S, d_rho, d_beta, st); count_launch();
      NYS_TRY((comb<T, T>(P, k1, d_beta, k1, Z, 1.0, 1.0, P, n, st, s)));
    }
    NYS_CUDA_TRY(cudaGetLastError());
    NYS_CUDA_TRY(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.done || launched >= maxit) break;
    if (chunk < 16) chunk *= 2;
  }
  int e = 0;
  NYS_CUDA_TRY(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  if (e) return NYS_ERR_TIMEOUT;

  // ---- X_act += Y S
  T* Xa = R0;  // reuse: active columns of X
  for (int a = 0; a < ka; ++a)
    NYS_CUDA_TRY(cudaMemcpyAsync(Xa + (size_t)a * n, X + (size_t)act[a] * n, n * sizeof(T),
                                 cudaMemcpyDeviceToDevice, s));
  NYS_TRY((comb<T, T>(Y, k1, d_S, ka, Xa, 1.0, 1.0, Xa, n, nullptr, s)));
  for (int a = 0; a < ka; ++a)
    NYS_CUDA_TRY(cudaMemcpyAsync(X + (size_t)act[a] * n, Xa + (size_t)a * n, n * sizeof(T),
                                 cudaMemcpyDeviceToDevice, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  *it_out = h.it;
  const int fin = h.done ? h.status : NYS_ERR_MAXIT;
  for (int a = 0; a < ka; ++a) {
    const int j = act[a];
    const double r = sqrt(h.res2[a]);
    if (h.it > 0) rel[j] = bn[j] > 0 ? r / bn[j] : r;
    const bool ok = h.it > 0 && h.res2[a] <= h.thresh2[a];
    status[j] = ok ? NYS_OK : (fin == NYS_OK ? NYS_ERR_MAXIT : fin);
  }
  return NYS_OK;
}

__global__ void block_sub_kernel(const double* b, const double* v, double* r, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    r[e] = b[e] - v[e];
}

__global__ void block_add_f32_kernel(double* x, const float* d, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    x[e] += (double)d[e];
}

}  // namespace

int32_t block_pcg_f64(const nys_operator* op, const nys_factor* f, double mu, int64_t k,
                      const double* b, double* x, double tol, int maxit, int use_x0,
                      nys_pcg_result* res, cudaStream_t s) {
  Scratch sc(s);
  const double* U = nullptr;
  if (f) {
    if (f->u_dtype == NYS_F64) {
      U = (const double*)f->U;
    } else {
      double* Ud;
      NYS_TRY(sc.get(&Ud, f->n * f->ell));
      NYS_TRY(convert_f32_to_f64((const float*)f->U, Ud, f->n * f->ell, s));
      U = Ud;
    }
  }
  std::vector<int> stt(k);
  std::vector<double> rel(k);
  int it = 0;
  NYS_TRY((run_block<double, double>(op, U, f ? f->E : nullptr, f ? f->lam : nullptr,
                                     f ? f->ell : 0,
                                     f ? f->lam_ell : 0.0, mu, (int)k, b, x, use_x0 != 0, tol,
                                     maxit, &it, stt.data(), rel.data(), s)));
  for (int64_t q = 0; q < k; ++q) {
    res[q].status = stt[q];
    res[q].iterations = it;
    res[q].refinements = 0;
    res[q].escalated = 0;
    res[q].rel_residual = rel[q];
  }
  return NYS_OK;
}

// Mixed precision: FP64-accurate outer residual of the block, FP32 block PCG
// for the correction of the columns still above tol (one block per step).
int32_t block_pcg_mixed(const nys_operator* op, const nys_factor* f, double mu, int64_t k,
                        const double* b, double* x, double tol, double inner_tol, int maxit,
                        int max_refine, int use_x0, nys_pcg_result* res, cudaStream_t s) {
  const int64_t n = op->n;
  Scratch sc(s);
  const float* U = nullptr;
  const float* Edef = nullptr;
  if (f) {
    if (f->u_dtype == NYS_F32) {
      U = (const float*)f->U;
      Edef = f->E;
    } else {
      float *Uf, *Ef;
      NYS_TRY(sc.get(&Uf, f->n * f->ell));
      NYS_TRY(sc.get(&Ef, f->ell * f->ell));
      NYS_TRY(convert_f64_to_f32((const double*)f->U, Uf, f->n * f->ell, s));
      NYS_TRY(orth_defect_f32(Uf, f->n, f->ell, Ef, s));
      U = Uf;
      Edef = Ef;
    }
  }
  double *r, *v, *d_mu, *nrm;
  float *rf, *df;
  NYS_TRY(sc.get(&r, k * n));
  NYS_TRY(sc.get(&v, k * n));
  NYS_TRY(sc.get(&rf, k * n));
  NYS_TRY(sc.get(&df, k * n));
  NYS_TRY(sc.get(&d_mu, k));
  NYS_TRY(sc.get(&nrm, k * k + 1));
  double* part;
  NYS_TRY(sc.get(&part, (size_t)gram_blocks(n) * k * k));
  unsigned char* work;
  NYS_TRY(sc.get(&work, op_matvec_work_bytes(op, true)));
  NYS_CUDA_TRY(cudaMemsetAsync(work, 0, 256, s));
  {
    std::vector<double> mus(k, mu);
    NYS_CUDA_TRY(cudaMemcpyAsync(d_mu, mus.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  if (!use_x0) NYS_CUDA_TRY(cudaMemsetAsync(x, 0, k * n * sizeof(double), s));
  std::vector<double> g((size_t)k * k);
  NYS_TRY(gram<double>(b, (int)k, b, (int)k, n, part, nrm, nullptr, s));
  NYS_CUDA_TRY(cudaMemcpyAsync(g.data(), nrm, g.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> bn(k), rel(k, 1.0), prev(k, 0.0);
  for (int64_t q = 0; q < k; ++q) bn[q] = sqrt(fmax(g[(size_t)q * k + q], 0.0));
  std::vector<int> stt(k, NYS_ERR_MAXIT);
  const unsigned gb = (unsigned)std::min<int64_t>(cdiv(k * n, 256), 1024);
  // FP64-accurate residual products: double-FP32 first, FP64 once the
  // residual stalls (as in the single-system refinement)
  bool exact = op->kind == NYS_OP_DENSE;
  const bool may_escalate = !exact;
  int total_it = 0, outer = 0;
  for (int kr = 0; kr <= max_refine; ++kr) {
    if (kr == 0 && !use_x0) {
      NYS_CUDA_TRY(cudaMemsetAsync(v, 0, k * n * sizeof(double), s));
    } else if (op->kind == NYS_OP_RBF && op->d <= 64) {
      const float* pts = (const float*)op->data;
      if (exact)
        NYS_TRY(rbf_exact_products(pts, n, op->ld, pts, n, op->ld, op->d, op->sigma, 0, 1,
                                   nullptr, mu, k, x, v, nullptr, s));
      else
        NYS_TRY(rbf_residual_products(op, d_mu, k, x, v, s));
    } else {
      for (int64_t q = 0; q < k; ++q) {
        if (exact)
          NYS_TRY(op_matvec_f64(op, mu, x + q * n, v + q * n, nullptr, work, s));
        else
          NYS_TRY(op_matvec_residual(op, mu, x + q * n, v + q * n, nullptr, work, s));
      }
    }
    block_sub_kernel<<<gb, 256, 0, s>>>(b, v, r, k * n); count_launch();
    NYS_TRY(gram<double>(r, (int)k, r, (int)k, n, part, nrm, nullptr, s));
    NYS_CUDA_TRY(cudaMemcpyAsync(g.data(), nrm, g.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int64_t> todo;
    bool finite = true;
    for (int64_t q = 0; q < k; ++q) {
      const double rq = sqrt(fmax(g[(size_t)q * k + q], 0.0));
      rel[q] = bn[q] > 0 ? rq / bn[q] : rq;
      finite = finite && std::isfinite(rel[q]);
      if (rel[q] <= tol) stt[q] = NYS_OK;
      else todo.push_back(q);
    }
    if (!finite) {
      for (int64_t q = 0; q < k; ++q)
        if (!std::isfinite(rel[q])) stt[q] = NYS_ERR_BREAKDOWN;
      break;
    }
    if (todo.empty() || total_it >= maxit || kr == max_refine) break;
    bool stalled = false;
    for (int64_t q : todo) stalled |= kr > 0 && rel[q] > 0.5 * prev[q];
    for (int64_t q = 0; q < k; ++q) prev[q] = rel[q];
    if (stalled && may_escalate && !exact) {
      exact = true;
      continue;  // the same iterate, its residual retaken in FP64
    }
    // inner block solve for the columns still above tol
    const int na = (int)todo.size();
    for (int a = 0; a < na; ++a)
      NYS_CUDA_TRY(cudaMemcpyAsync(v + (size_t)a * n, r + todo[a] * n, n * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
    NYS_TRY(convert_f64_to_f32(v, rf, (int64_t)na * n, s));
    std::vector<int> ist(na);
    std::vector<double> irel(na);
    int its = 0;
    NYS_TRY((run_block<float, float>(op, U, Edef, f ? f->lam : nullptr, f ? f->ell : 0,
                                     f ? f->lam_ell : 0.0, mu, na, rf, df, false, inner_tol,
                                     maxit - total_it, &its, ist.data(), irel.data(), s)));
    for (int a = 0; a < na; ++a) {
      block_add_f32_kernel<<<gb, 256, 0, s>>>(x + todo[a] * n, df + (size_t)a * n, n);
      count_launch();
    }
    total_it += its;
    ++outer;
    if (its == 0) {
      // the inner solve could not take a step (breakdown at its start)
      for (int a = 0; a < na; ++a)
        if (ist[a] == NYS_ERR_BREAKDOWN) stt[todo[a]] = NYS_ERR_BREAKDOWN;
      break;
    }
  }
  for (int64_t q = 0; q < k; ++q) {
    res[q].status = stt[q];
    res[q].iterations = total_it;
    res[q].refinements = outer;
    res[q].escalated = 0;
    res[q].rel_residual = rel[q];
  }
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

}  // namespace nys
