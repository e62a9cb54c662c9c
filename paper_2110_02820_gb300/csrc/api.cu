// C-ABI entry points (include/nyspcg.h): argument checks, the sketch and the
// shifted core of Algorithm 1, the adaptive loop of Algorithm 5 with the
// power estimate of Algorithm 4, and the PCG dispatch.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nys {

int32_t pcg_f64(const nys_operator* op, const nys_factor* f, const double* mu, int64_t nsys,
                const double* b, double* x, double tol, int maxit, int use_x0, double* hist,
                nys_pcg_result* res, cudaStream_t s);
int32_t pcg_mixed(const nys_operator* op, const nys_factor* f, const double* mu, int64_t nsys,
                  const double* b, double* x, double tol, double inner_tol, int maxit,
                  int max_refine, int use_x0, double* hist, nys_pcg_result* res, cudaStream_t s);
int32_t block_pcg_f64(const nys_operator* op, const nys_factor* f, double mu, int64_t k,
                      const double* b, double* x, double tol, int maxit, int use_x0,
                      nys_pcg_result* res, cudaStream_t s);
int32_t block_pcg_mixed(const nys_operator* op, const nys_factor* f, double mu, int64_t k,
                        const double* b, double* x, double tol, double inner_tol, int maxit,
                        int max_refine, int use_x0, nys_pcg_result* res, cudaStream_t s);
int32_t precond_apply(const nys_factor* f, const double* mu, int64_t nrhs, const void* v, void* z,
                      int32_t dtype, cudaStream_t s);
int32_t sketch_solve(const nys_factor* f, const double* mu, int64_t nrhs, const void* b, void* x,
                     int32_t dtype, cudaStream_t s);

constexpr int64_t kMaxEll = 4096;
constexpr int kMaxEscalations = 6;

// ---------------------------------------------------------------- validation

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int32_t check_op(const nys_operator* op) {
  if (!op || !op->data || op->n <= 0) return NYS_ERR_ARG;
  if (!aligned16(op->data)) return NYS_ERR_ARG;
  switch (op->kind) {
    case NYS_OP_DENSE:
      if (op->dtype != NYS_F64 || op->ld < op->n) return NYS_ERR_ARG;
      return NYS_OK;
    case NYS_OP_GRAM:
      if (op->dtype != NYS_F32 || op->m <= 0 || op->ld < op->n) return NYS_ERR_ARG;
      return NYS_OK;
    case NYS_OP_RBF:
      if (op->dtype != NYS_F32 || op->d <= 0 || op->d > 64 || op->ld < op->d) return NYS_ERR_ARG;
      if (!(op->sigma > 0.0) || !std::isfinite(op->sigma)) return NYS_ERR_ARG;
      return NYS_OK;
    default:
      return NYS_ERR_ARG;
  }
}

// ---------------------------------------------------------------- typed helpers

template <typename T>
struct Ops;

template <>
struct Ops<double> {
  static constexpr bool f64 = true;
  static constexpr int mantissa = 52;
  static int32_t gram(const double* A, const double* B, int64_t n, int64_t p, int64_t q, double* C,
                      cudaStream_t s) {  // C = A^T B  (A n x p, B n x q)
    return gemm_f64(true, p, q, n, A, p, B, q, C, q, s);
  }
  // C = A S (A n x p, S p x q FP64)
  static int32_t mul_small(const double* A, const double* S, int64_t n, int64_t p, int64_t q,
                           double* C, cudaStream_t s) {
    return gemm_f64(false, n, q, p, A, p, S, q, C, q, s);
  }
  static int32_t sumsq(const double* x, int64_t c, double* out, cudaStream_t s) {
    return sumsq_f64(x, c, out, s);
  }
  static int32_t shift(const double* Y, const double* Q, double* Ynu, int64_t c, const double* nu,
                       cudaStream_t s) {
    return shift_add_f64(Y, Q, Ynu, c, nu, 1.0, s);
  }
  static int32_t from_f64(const double* in, double* out, int64_t c, cudaStream_t s) {
    if (in != out)
      NYS_CUDA_TRY(cudaMemcpyAsync(out, in, c * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return NYS_OK;
  }
};

template <>
struct Ops<float> {
  static constexpr bool f64 = false;
  static constexpr int mantissa = 23;
  static int32_t gram(const float* A, const float* B, int64_t n, int64_t p, int64_t q, double* C,
                      cudaStream_t s) {
    return gemm_f32_out64(true, p, q, n, A, p, B, q, C, q, s);
  }
  static int32_t mul_small(const float* A, const double* S, int64_t n, int64_t p, int64_t q,
                           float* C, cudaStream_t s) {
    Scratch sc(s);
    float* Sf;
    NYS_TRY(sc.get(&Sf, p * q));
    NYS_TRY(convert_f64_to_f32(S, Sf, p * q, s));
    return gemm_f32(false, n, q, p, A, p, Sf, q, C, q, s);
  }
  static int32_t sumsq(const float* x, int64_t c, double* out, cudaStream_t s) {
    return sumsq_f32(x, c, out, s);
  }
  static int32_t shift(const float* Y, const float* Q, float* Ynu, int64_t c, const double* nu,
                       cudaStream_t s) {
    return shift_add_f32(Y, Q, Ynu, c, nu, 1.0, s);
  }
  static int32_t from_f64(const double* in, float* out, int64_t c, cudaStream_t s) {
    return convert_f64_to_f32(in, out, c, s);
  }
};

__global__ void scale_scalar_kernel(double* x, double f) { x[0] *= f; }

__global__ void diag_max_kernel(const double* G, int64_t ell, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < ell; i += blockDim.x) m = fmax(m, G[i * ell + i]);
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    out[0] = t;
  }
}

static int32_t read_int(const int* d, int* h, cudaStream_t s) {
  NYS_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

static int32_t read_double(const double* d, double* h, cudaStream_t s) {
  NYS_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

// CholeskyQR passes: X (n x ell, T) <- X R^{-1}, Racc (ell x ell FP64) <- R Racc.
// The first pass adds the diagonal shift of shifted CholeskyQR (Fukaya et
// al., SISC 2020) if the plain factorisation fails; then a third pass runs.
template <typename T>
static int32_t cholqr(T* X, int64_t n, int64_t ell, T* tmp, double* Racc, bool racc_init,
                      int passes0, cudaStream_t s) {
  Scratch sc(s);
  double *G, *Gi, *Rn, *dmax;
  int* info;
  NYS_TRY(sc.get(&G, ell * ell));
  NYS_TRY(sc.get(&Gi, ell * ell));
  NYS_TRY(sc.get(&Rn, ell * ell));
  NYS_TRY(sc.get(&dmax, 1));
  NYS_TRY(sc.get(&info, 1));
  int passes = passes0;
  T* cur = X;
  T* other = tmp;
  for (int pass = 0; pass < passes; ++pass) {
    NYS_TRY(Ops<T>::gram(cur, cur, n, ell, ell, G, s));
    NYS_TRY(symmetrize(G, ell, s));
    NYS_TRY(Ops<T>::f64 ? chol_upper(G, ell, info, s) : chol_upper_dfl(G, ell, info, s));
    int h_info = 0;
    NYS_TRY(read_int(info, &h_info, s));
    if (h_info != 0) {
      if (pass > 0) return NYS_ERR_NOT_PSD;
      // shifted CholeskyQR: G + s I with s = 11 (n ell + ell (ell + 1)) u max_i G_ii
      NYS_TRY(Ops<T>::gram(cur, cur, n, ell, ell, G, s));
      NYS_TRY(symmetrize(G, ell, s));
      diag_max_kernel<<<1, 256, 0, s>>>(G, ell, dmax); count_launch();
      double h_dmax = 0.0;
      NYS_TRY(read_double(dmax, &h_dmax, s));
      const double u = Ops<T>::f64 ? ldexp(1.0, -53) : ldexp(1.0, -24);
      double shift = 11.0 * ((double)n * ell + (double)ell * (ell + 1)) * u * h_dmax;
      if (!(shift > 0.0)) return NYS_ERR_NOT_PSD;
      NYS_TRY(add_diag(G, ell, shift, s));
      NYS_TRY(Ops<T>::f64 ? chol_upper(G, ell, info, s) : chol_upper_dfl(G, ell, info, s));
      NYS_TRY(read_int(info, &h_info, s));
      if (h_info != 0) return NYS_ERR_NOT_PSD;
      passes = passes0 + 1;
    }
    NYS_TRY(Ops<T>::f64 ? tri_inv_upper(G, Gi, ell, s) : tri_inv_upper_dfl(G, Gi, ell, s));
    NYS_TRY(Ops<T>::mul_small(cur, Gi, n, ell, ell, other, s));
    // Racc <- R_pass Racc
    if (!Racc) {
      // R not wanted
    } else if (pass == 0 && racc_init) {
      NYS_CUDA_TRY(cudaMemcpyAsync(Racc, G, ell * ell * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      NYS_TRY(gemm_f64(false, ell, ell, ell, G, ell, Racc, ell, Rn, ell, s));
      NYS_CUDA_TRY(cudaMemcpyAsync(Racc, Rn, ell * ell * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    T* t = cur;
    cur = other;
    other = t;
  }
  if (cur != X) NYS_CUDA_TRY(cudaMemcpyAsync(X, cur, n * ell * sizeof(T), cudaMemcpyDeviceToDevice, s));
  return NYS_OK;
}

// Thin QR of a Gaussian block (Algorithm 1, step 2), in place.  A Gaussian
// n x ell block with n >> ell has condition number near 1, so one
// CholeskyQR pass already leaves orthogonality at rounding level.
template <typename T>
static int32_t orthonormalize(T* Om, int64_t n, int64_t ell, cudaStream_t s) {
  Scratch sc(s);
  T* tmp;
  NYS_TRY(sc.get(&tmp, n * ell));
  return cholqr<T>(Om, n, ell, tmp, nullptr, true, (n >= 4 * ell) ? 1 : 2, s);
}

// ||Y||_2 by power iteration on Y^T Y (30 steps); only its binary exponent
// enters nu = sqrt(n) eps(||Y||_2) of Algorithm 5.
template <typename T>
static int32_t spectral_norm_sq(const T* Y, int64_t n, int64_t ell, double* d_out, cudaStream_t s) {
  Scratch sc(s);
  double* H;
  NYS_TRY(sc.get(&H, ell * ell));
  NYS_TRY(Ops<T>::gram(Y, Y, n, ell, ell, H, s));
  double *v, *w, *nrm;
  NYS_TRY(sc.get(&v, ell));
  NYS_TRY(sc.get(&w, ell));
  NYS_TRY(sc.get(&nrm, 1));
  std::vector<double> ones(ell, 1.0);
  NYS_CUDA_TRY(cudaMemcpyAsync(v, ones.data(), ell * sizeof(double), cudaMemcpyHostToDevice, s));
  double lam = 0.0;
  for (int it = 0; it < 30; ++it) {
    NYS_TRY(gemm_f64(false, ell, 1, ell, H, ell, v, 1, w, 1, s));
    NYS_TRY(sumsq_f64(w, ell, nrm, s));
    double h = 0.0;
    NYS_TRY(read_double(nrm, &h, s));
    if (!(h > 0.0)) break;
    double hn = sqrt(h);
    std::vector<double> hw(ell);
    NYS_CUDA_TRY(cudaMemcpyAsync(hw.data(), w, ell * sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    // Rayleigh-quotient style estimate ||H v|| / ||v|| with ||v|| = 1 after the first step
    lam = hn;
    for (auto& e : hw) e /= hn;
    NYS_CUDA_TRY(cudaMemcpyAsync(v, hw.data(), ell * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  // first step used v = ones (norm sqrt(ell)); later steps are unit vectors, so lam = ||H v||
  NYS_CUDA_TRY(cudaMemcpyAsync(d_out, &lam, sizeof(double), cudaMemcpyHostToDevice, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

// Steps 4-9 of Algorithm 1 (and of Algorithm 5) given Q (n x ell, orthonormal
// columns) and Y = A Q.  nu = scale * eps(norm), norm = ||Y||_F (Alg. 1) or
// ||Y||_2 (Alg. 5).  Writes U (n x ell, T) and lam (ell, FP64) of `f`.
template <typename T>
static int32_t shifted_core(const T* Q, const T* Y, int64_t n, int64_t ell, bool spectral,
                            double scale, nys_factor* f, cudaStream_t s) {
  Scratch sc(s);
  T *Ynu, *Bb;
  double *M, *Ci, *R, *Ut, *sig, *nrm2, *nu;
  int *info, *jst;
  NYS_TRY(sc.get(&Ynu, n * ell));
  NYS_TRY(sc.get(&Bb, n * ell));
  NYS_TRY(sc.get(&M, ell * ell));
  NYS_TRY(sc.get(&Ci, ell * ell));
  NYS_TRY(sc.get(&R, ell * ell));
  NYS_TRY(sc.get(&Ut, ell * ell));
  NYS_TRY(sc.get(&sig, ell));
  NYS_TRY(sc.get(&nrm2, 1));
  NYS_TRY(sc.get(&nu, 1));
  NYS_TRY(sc.get(&info, 1));
  NYS_TRY(sc.get(&jst, 1));
  if (spectral)
    NYS_TRY(spectral_norm_sq<T>(Y, n, ell, nrm2, s));
  else
    NYS_TRY(Ops<T>::sumsq(Y, n * ell, nrm2, s));
  NYS_TRY(compute_nu(nrm2, scale, Ops<T>::mantissa, nu, s));
  int esc = 0;
  for (;; ++esc) {
    NYS_TRY(Ops<T>::shift(Y, Q, Ynu, n * ell, nu, s));  // Y_nu = Y + nu Q
    NYS_TRY(Ops<T>::gram(Q, Ynu, n, ell, ell, M, s));    // Q^T Y_nu
    NYS_TRY(symmetrize(M, ell, s));
    // C^T C = Q^T Y_nu
    NYS_TRY(Ops<T>::f64 ? chol_upper(M, ell, info, s) : chol_upper_dfl(M, ell, info, s));
    int h = 0;
    NYS_TRY(read_int(info, &h, s));
    if (h == 0) break;
    if (esc >= kMaxEscalations) return NYS_ERR_NOT_PSD;
    scale_scalar_kernel<<<1, 1, 0, s>>>(nu, 10.0); count_launch();
  }
  NYS_TRY(Ops<T>::f64 ? tri_inv_upper(M, Ci, ell, s) : tri_inv_upper_dfl(M, Ci, ell, s));
  NYS_TRY(Ops<T>::mul_small(Ynu, Ci, n, ell, ell, Bb, s));  // B = Y_nu C^{-1}
  // thin SVD of B: B = Qb R (CholeskyQR2), R = Ut Sigma V^T (one-sided Jacobi)
  NYS_TRY(cholqr<T>(Bb, n, ell, Ynu, R, true, 2, s));
  int sweeps = 0, refine = 0;
  // The FP64 refinement runs for both precisions: the preconditioner needs U
  // orthonormal far below (lambda_ell + mu) / lambda_1, beyond what the FP32
  // rotations leave (~1e-6).
  NYS_TRY(jacobi_svd(R, Ut, sig, ell, true, jst, &sweeps, &refine, s));
  int hj = 0;
  NYS_TRY(read_int(jst, &hj, s));
  if (hj != 0) return NYS_ERR_TIMEOUT;
  NYS_TRY(Ops<T>::mul_small(Bb, Ut, n, ell, ell, (T*)f->U, s));  // U = Qb Ut
  if (!Ops<T>::f64) {
    // an FP32 U is orthonormal only to its rounding: keep U^T U - I for the
    // corrected preconditioner apply
    if (!f->E) NYS_CUDA_TRY(cudaMalloc(&f->E, (size_t)ell * ell * sizeof(float)));
    NYS_TRY(orth_defect_f32(reinterpret_cast<const float*>(f->U), n, ell, f->E, s));
  }
  NYS_TRY(lambda_from_sigma(sig, nu, f->lam, ell, s));         // lam = max(0, sigma^2 - nu)
  NYS_TRY(read_double(nu, &f->nu, s));
  NYS_TRY(read_double(f->lam + (ell - 1), &f->lam_ell, s));
  f->escalations = esc;
  f->svd_sweeps = sweeps;
  f->svd_refine = refine;
  return NYS_OK;
}

static int32_t factor_alloc(nys_factor** out, int64_t n, int64_t ell, bool f64, int precision) {
  nys_factor* f = new (std::nothrow) nys_factor();
  if (!f) return NYS_ERR_OOM;
  f->n = n;
  f->ell = ell;
  f->precision = precision;
  f->u_dtype = f64 ? NYS_F64 : NYS_F32;
  cudaGetDevice(&f->device);
  cudaError_t e = cudaMalloc(&f->U, (size_t)n * ell * (f64 ? sizeof(double) : sizeof(float)));
  if (e == cudaSuccess) e = cudaMalloc(&f->lam, ell * sizeof(double));
  if (e != cudaSuccess) {
    if (f->U) cudaFree(f->U);
    delete f;
    return e == cudaErrorMemoryAllocation ? NYS_ERR_OOM : NYS_ERR_CUDA;
  }
  *out = f;
  return NYS_OK;
}

template <typename T>
static int32_t sketch_impl(const nys_operator* op, int64_t ell, uint64_t seed, const double* omega,
                           int precision, nys_factor** out, cudaStream_t s) {
  const int64_t n = op->n;
  nys_factor* f = nullptr;
  NYS_TRY(factor_alloc(&f, n, ell, Ops<T>::f64, precision));
  int32_t st;
  {
    Scratch sc(s);
    T *Q, *Y;
    double* raw = nullptr;
    st = sc.get(&Q, n * ell);
    if (st == NYS_OK) st = sc.get(&Y, n * ell);
    if (st == NYS_OK && !omega) {
      st = sc.get(&raw, n * ell);
      if (st == NYS_OK) st = philox_gaussian_f64(raw, n * ell, seed, NYS_STREAM_OMEGA, s);
    }
    if (st == NYS_OK) st = Ops<T>::from_f64(omega ? omega : raw, Q, n * ell, s);
    if (st == NYS_OK) st = orthonormalize<T>(Q, n, ell, s);
    if (st == NYS_OK) st = op_sketch(op, Ops<T>::f64, Q, Y, ell, s);
    if (st == NYS_OK) st = shifted_core<T>(Q, Y, n, ell, false, 1.0, f, s);
    if (st == NYS_OK) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = NYS_ERR_CUDA;
    }
  }
  if (st != NYS_OK) {
    nys_factor_free(f);
    return st;
  }
  *out = f;
  return NYS_OK;
}

// ell distinct indices of [0, n), uniformly without replacement: a partial
// Fisher-Yates shuffle (swaps kept in a map) driven by SplitMix64 from `seed`.
static void sample_columns(int64_t n, int64_t ell, uint64_t seed, std::vector<int64_t>& out) {
  uint64_t st = seed ^ 0x636f6c756d6e73ull;  // stream tag
  auto next = [&st]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  std::unordered_map<int64_t, int64_t> swapped;
  auto at = [&swapped](int64_t i) {
    auto it = swapped.find(i);
    return it == swapped.end() ? i : it->second;
  };
  out.resize(ell);
  for (int64_t c = 0; c < ell; ++c) {
    const int64_t r = c + (int64_t)(next() % (uint64_t)(n - c));
    const int64_t vc = at(c), vr = at(r);
    swapped[r] = vc;
    swapped[c] = vr;
    out[c] = vr;
  }
}

template <typename T>
static int32_t columns_impl(const nys_operator* op, int64_t ell, const int64_t* cols,
                            int precision, nys_factor** out, cudaStream_t s) {
  const int64_t n = op->n;
  nys_factor* f = nullptr;
  NYS_TRY(factor_alloc(&f, n, ell, Ops<T>::f64, precision));
  int32_t st;
  {
    Scratch sc(s);
    T *Q, *Y;
    st = sc.get(&Q, n * ell);
    if (st == NYS_OK) st = sc.get(&Y, n * ell);
    if (st == NYS_OK) st = op_columns(op, Ops<T>::f64, cols, ell, Q, Y, s);
    if (st == NYS_OK) st = shifted_core<T>(Q, Y, n, ell, false, 1.0, f, s);
    if (st == NYS_OK) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = NYS_ERR_CUDA;
    }
  }
  if (st != NYS_OK) {
    nys_factor_free(f);
    return st;
  }
  *out = f;
  return NYS_OK;
}

// ---------------------------------------------------------------- Algorithm 4

// y -= U diag(c) U^T x  (x, y FP64 n; U n x ell of type TU; c FP64 ell)
template <typename TU>
__global__ void utx_partial_kernel(const TU* U, int64_t n, int64_t ell, const double* x,
                                   int64_t rows, double* part) {
  int64_t j = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= ell) return;
  int64_t i0 = (int64_t)blockIdx.x * rows, i1 = i0 + rows < n ? i0 + rows : n;
  double acc = 0.0;
  for (int64_t i = i0; i < i1; ++i) acc += (double)U[i * ell + j] * x[i];
  part[blockIdx.x * ell + j] = acc;
}

__global__ void utx_reduce_kernel(const double* part, int64_t nb, int64_t ell, const double* c,
                                  double* w) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ell) return;
  double acc = 0.0;
  for (int64_t b = 0; b < nb; ++b) acc += part[b * ell + j];
  w[j] = c[j] * acc;
}

template <typename TU>
__global__ void uw_sub_kernel(const TU* U, int64_t n, int64_t ell, const double* w, double* y) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  double acc = 0.0;
  for (int64_t j = lane; j < ell; j += 32) acc += (double)U[i * ell + j] * w[j];
  acc = warp_sum(acc);
  if (lane == 0) y[i] -= acc;
}

__global__ void dot_kernel(const double* a, const double* b, int64_t n, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += a[i] * b[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[0] = acc;
}

__global__ void scale_by_inv_norm_kernel(const double* in, double* out, int64_t n,
                                         const double* sumsq) {
  double inv = 1.0 / sqrt(sumsq[0]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * inv;
}

template <typename TU>
static int32_t lowrank_sub(const TU* U, int64_t n, int64_t ell, const double* c, const double* x,
                           double* y, cudaStream_t s) {
  Scratch sc(s);
  int64_t nb = cdiv(n, 256);
  if (nb > 256) nb = 256;
  int64_t rows = cdiv(n, nb);
  nb = cdiv(n, rows);
  double *part, *w;
  NYS_TRY(sc.get(&part, nb * ell));
  NYS_TRY(sc.get(&w, ell));
  utx_partial_kernel<TU><<<dim3((unsigned)nb, (unsigned)cdiv(ell, 128)), 128, 0, s>>>(U, n, ell, x,
                                                                                      rows, part); count_launch();
  utx_reduce_kernel<<<(unsigned)cdiv(ell, 256), 256, 0, s>>>(part, nb, ell, c, w); count_launch();
  uw_sub_kernel<TU><<<(unsigned)cdiv(n, 8), 256, 0, s>>>(U, n, ell, w, y); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// Algorithm 4 with start g (device FP64 n); returns the estimate on the host.
static int32_t power_estimate(const nys_operator* op, const nys_factor* f, const double* g, int q,
                              double* est, cudaStream_t s) {
  const int64_t n = op->n;
  Scratch sc(s);
  double *v0, *v, *nrm, *e, *work;
  NYS_TRY(sc.get(&v0, n));
  NYS_TRY(sc.get(&v, n));
  NYS_TRY(sc.get(&nrm, 1));
  NYS_TRY(sc.get(&e, 1));
  NYS_TRY(sc.get(&work, op_matvec_work_bytes(op, true) / sizeof(double) + 1));
  NYS_CUDA_TRY(cudaMemsetAsync(work, 0, 256, s));
  const unsigned gb = (unsigned)(cdiv(n, 256) > 1024 ? 1024 : cdiv(n, 256));
  NYS_TRY(sumsq_f64(g, n, nrm, s));
  scale_by_inv_norm_kernel<<<gb, 256, 0, s>>>(g, v0, n, nrm); count_launch();  // v0 = g / ||g||
  double h = 0.0;
  NYS_CUDA_TRY(cudaMemsetAsync(e, 0, sizeof(double), s));
  for (int i = 0; i < q; ++i) {
    NYS_TRY(op_matvec_f64(op, 0.0, v0, v, nullptr, work, s));  // v = A v0
    if (f->u_dtype == NYS_F64)
      NYS_TRY(lowrank_sub<double>((const double*)f->U, n, f->ell, f->lam, v0, v, s));
    else
      NYS_TRY(lowrank_sub<float>((const float*)f->U, n, f->ell, f->lam, v0, v, s));
    dot_kernel<<<1, 1024, 0, s>>>(v0, v, n, e); count_launch();  // E = v0^T v
    NYS_TRY(sumsq_f64(v, n, nrm, s));
    scale_by_inv_norm_kernel<<<gb, 256, 0, s>>>(v, v0, n, nrm); count_launch();  // v0 = v / ||v||
  }
  NYS_CUDA_TRY(cudaGetLastError());
  NYS_TRY(read_double(e, &h, s));
  *est = h;
  return NYS_OK;
}

// ---------------------------------------------------------------- Algorithm 5

__global__ void copy_cols_kernel(const double* src, int64_t src_ld, int64_t col0, double* dst,
                                 int64_t n, int64_t m) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  int64_t i = e / m, j = e % m;
  dst[e] = src[i * src_ld + col0 + j];
}

template <typename T>
__global__ void place_cols_kernel(const T* src, int64_t m, T* dst, int64_t dst_ld, int64_t col0,
                                  int64_t n) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * m) return;
  int64_t i = e / m, j = e % m;
  dst[i * dst_ld + col0 + j] = src[e];
}

template <typename T>
__global__ void repack_kernel(const T* src, int64_t src_ld, T* dst, int64_t dst_ld, int64_t n,
                              int64_t cols) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * cols) return;
  int64_t i = e / cols, j = e % cols;
  dst[i * dst_ld + j] = src[i * src_ld + j];
}

template <typename T>
static int32_t adaptive_impl(const nys_operator* op, int64_t ell0, int64_t ell_max, int rule,
                             double tol, int q, double mu, uint64_t seed, const double* omega,
                             const double* g, int precision, nys_factor** out,
                             nys_adapt_info* info, cudaStream_t s) {
  const int64_t n = op->n;
  Scratch sc(s);
  // Qall, Yall: n x ell_max with row stride ell_max; blocks fill columns in order
  T *Qall, *Yall, *Qc, *Yc, *blk, *yblk;
  double *raw, *gk;
  NYS_TRY(sc.get(&Qall, n * ell_max));
  NYS_TRY(sc.get(&Yall, n * ell_max));
  NYS_TRY(sc.get(&Qc, n * ell_max));
  NYS_TRY(sc.get(&Yc, n * ell_max));
  NYS_TRY(sc.get(&blk, n * ell_max));
  NYS_TRY(sc.get(&yblk, n * ell_max));
  NYS_TRY(sc.get(&raw, n * ell_max));
  NYS_TRY(sc.get(&gk, n));
  int64_t ell_tot = 0;
  int64_t ell_next = ell0 < ell_max ? ell0 : ell_max;
  int64_t m = ell_next;
  int k_est = 0, doublings = 0;
  double E = std::nan("");
  nys_factor* f = nullptr;

  auto add_block = [&](int64_t mm) -> int32_t {
    // raw Gaussian block n x mm
    if (omega) {
      copy_cols_kernel<<<(unsigned)cdiv(n * mm, 256), 256, 0, s>>>(omega, ell_max, ell_tot, raw, n,
                                                                  mm); count_launch();
    } else {
      NYS_TRY(philox_gaussian_f64(raw, n * mm, seed, NYS_STREAM_ADAPTIVE + (uint64_t)ell_tot, s));
    }
    NYS_TRY(Ops<T>::from_f64(raw, blk, n * mm, s));
    NYS_TRY(orthonormalize<T>(blk, n, mm, s));
    NYS_TRY(op_sketch(op, Ops<T>::f64, blk, yblk, mm, s));
    place_cols_kernel<T><<<(unsigned)cdiv(n * mm, 256), 256, 0, s>>>(blk, mm, Qall, ell_max,
                                                                     ell_tot, n); count_launch();
    place_cols_kernel<T><<<(unsigned)cdiv(n * mm, 256), 256, 0, s>>>(yblk, mm, Yall, ell_max,
                                                                     ell_tot, n); count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    ell_tot += mm;
    return NYS_OK;
  };
  auto compute = [&]() -> int32_t {
    if (f) nys_factor_free(f);
    f = nullptr;
    NYS_TRY(factor_alloc(&f, n, ell_tot, Ops<T>::f64, precision));
    repack_kernel<T><<<(unsigned)cdiv(n * ell_tot, 256), 256, 0, s>>>(Qall, ell_max, Qc, ell_tot,
                                                                      n, ell_tot); count_launch();
    repack_kernel<T><<<(unsigned)cdiv(n * ell_tot, 256), 256, 0, s>>>(Yall, ell_max, Yc, ell_tot,
                                                                      n, ell_tot); count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return shifted_core<T>(Qc, Yc, n, ell_tot, true, sqrt((double)n), f, s);
  };
  int32_t st = NYS_OK;
  while (true) {
    st = add_block(m);
    if (st == NYS_OK) st = compute();
    if (st != NYS_OK) break;
    bool stop;
    if (rule == NYS_RULE_ERR) {
      const double* gp = g ? g + (int64_t)k_est * n : nullptr;
      if (!gp) {
        st = philox_gaussian_f64(gk, n, seed, NYS_STREAM_ESTIMATE + (uint64_t)k_est, s);
        if (st != NYS_OK) break;
        gp = gk;
      }
      st = power_estimate(op, f, gp, q, &E, s);
      if (st != NYS_OK) break;
      ++k_est;
      stop = E <= tol;
    } else {
      stop = f->lam_ell / mu <= tol;
    }
    if (stop) break;
    m = ell_next;
    ell_next = 2 * ell_next;
    ++doublings;
    if (ell_next > ell_max) {
      ell_next = ell_next - m;
      m = ell_max - ell_next;
      if (m > 0) {
        st = add_block(m);
        if (st == NYS_OK) st = compute();
        E = std::nan("");  // the enlarged factor has no estimate
      } else {
        --doublings;       // the sketch is already at ell_max: its estimate stands
      }
      break;
    }
  }
  if (st != NYS_OK) {
    if (f) nys_factor_free(f);
    return st;
  }
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->ell = f->ell;
    info->doublings = doublings;
    info->estimates = k_est;
    info->err_est = E;
    info->lambda_ell = f->lam_ell;
    info->kappa_est = (std::isnan(E) || !(mu > 0)) ? std::nan("") : (f->lam_ell + mu + E) / mu;
  }
  *out = f;
  return NYS_OK;
}

}  // namespace nys

using namespace nys;

// ==================================================================== C ABI

extern "C" {

uint64_t nys_kernel_launch_count(void) { return (uint64_t)nys::launch_count(); }

int32_t nys_pcg_graphs(int32_t on) { return nys::pcg_graphs(on); }

int32_t nys_pcg_reliable(int32_t on) { return nys::pcg_reliable(on); }

int32_t nys_pcg_loop(int32_t on) { return nys::pcg_loop(on); }

uint64_t nys_pcg_graph_replays(void) { return (uint64_t)nys::pcg_graph_replays(); }

int32_t nys_autotune(int32_t on) { return nys::tune_switch(on); }

int64_t nys_autotune_dump(char* buf, int64_t cap) { return nys::tune_dump(buf, cap); }

void nys_autotune_clear(void) { nys::tune_clear(); }

int32_t nys_autotune_set(const char* key, int32_t choice) { return nys::tune_set(key, choice); }

const char* nys_status_str(int32_t st) {
  switch (st) {
    case NYS_OK: return "ok";
    case NYS_ERR_ARG: return "invalid argument";
    case NYS_ERR_NOT_PSD: return "Cholesky of Omega^T Y_nu failed after shift escalation (not psd)";
    case NYS_ERR_BREAKDOWN: return "PCG breakdown (p^T A p <= 0 or non-finite)";
    case NYS_ERR_MAXIT: return "iteration cap reached";
    case NYS_ERR_TIMEOUT: return "bounded device wait expired";
    case NYS_ERR_CUDA: return "CUDA runtime error";
    case NYS_ERR_OOM: return "device out of memory";
    default: return "unknown status";
  }
}

int32_t nys_sketch(const nys_operator* op, int64_t ell, uint64_t seed, const double* omega,
                   int32_t precision, nys_factor** out, void* stream) {
  if (!out) return NYS_ERR_ARG;
  *out = nullptr;
  NYS_TRY(check_op(op));
  if (ell < 1 || ell > op->n || ell > kMaxEll) return NYS_ERR_ARG;
  if (precision != NYS_PREC_F64 && precision != NYS_PREC_MIXED) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == NYS_PREC_F64) return sketch_impl<double>(op, ell, seed, omega, precision, out, s);
  return sketch_impl<float>(op, ell, seed, omega, precision, out, s);
}

int32_t nys_sketch_columns(const nys_operator* op, int64_t ell, uint64_t seed, const int64_t* cols,
                           int32_t precision, nys_factor** out, void* stream) {
  if (!out) return NYS_ERR_ARG;
  *out = nullptr;
  NYS_TRY(check_op(op));
  if (ell < 1 || ell > op->n || ell > kMaxEll) return NYS_ERR_ARG;
  if (precision != NYS_PREC_F64 && precision != NYS_PREC_MIXED) return NYS_ERR_ARG;
  if (op->kind == NYS_OP_RBF && op->d > 64) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  const int64_t* dcols = cols;
  if (!dcols) {
    std::vector<int64_t> h;
    sample_columns(op->n, ell, seed, h);
    int64_t* d;
    NYS_TRY(sc.get(&d, ell));
    NYS_CUDA_TRY(cudaMemcpyAsync(d, h.data(), ell * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));  // h goes out of scope
    dcols = d;
  }
  if (precision == NYS_PREC_F64) return columns_impl<double>(op, ell, dcols, precision, out, s);
  return columns_impl<float>(op, ell, dcols, precision, out, s);
}

int32_t nys_sketch_adaptive(const nys_operator* op, int64_t ell0, int64_t ell_max, int32_t rule,
                            double tol, int32_t q, double mu, uint64_t seed, const double* omega,
                            const double* g, int32_t precision, nys_factor** out,
                            nys_adapt_info* info, void* stream) {
  if (!out) return NYS_ERR_ARG;
  *out = nullptr;
  NYS_TRY(check_op(op));
  if (ell0 < 1 || ell_max < 1 || ell_max > op->n || ell_max > kMaxEll) return NYS_ERR_ARG;
  if (rule != NYS_RULE_ERR && rule != NYS_RULE_RATIO) return NYS_ERR_ARG;
  if (rule == NYS_RULE_ERR && q < 1) return NYS_ERR_ARG;
  if (rule == NYS_RULE_RATIO && !(mu > 0.0)) return NYS_ERR_ARG;
  if (!(tol >= 0.0) || !std::isfinite(tol)) return NYS_ERR_ARG;
  if (precision != NYS_PREC_F64 && precision != NYS_PREC_MIXED) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == NYS_PREC_F64)
    return adaptive_impl<double>(op, ell0, ell_max, rule, tol, q, mu, seed, omega, g, precision,
                                 out, info, s);
  return adaptive_impl<float>(op, ell0, ell_max, rule, tol, q, mu, seed, omega, g, precision, out,
                              info, s);
}

static int32_t check_mu(const nys_factor* f, const double* mu, int64_t cnt) {
  if (!mu) return NYS_ERR_ARG;
  for (int64_t i = 0; i < cnt; ++i) {
    if (!(mu[i] >= 0.0) || !std::isfinite(mu[i])) return NYS_ERR_ARG;
    if (f && mu[i] == 0.0 && !(f->lam_ell > 0.0)) return NYS_ERR_ARG;
  }
  return NYS_OK;
}

int32_t nys_precond_apply(const nys_factor* f, const double* mu, int64_t nrhs, const void* v,
                          void* z, int32_t dtype, void* stream) {
  if (!f || !v || !z || nrhs < 1) return NYS_ERR_ARG;
  if (dtype != NYS_F64 && dtype != NYS_F32) return NYS_ERR_ARG;
  if (v == z) return NYS_ERR_ARG;
  NYS_TRY(check_mu(f, mu, nrhs));
  return precond_apply(f, mu, nrhs, v, z, dtype, (cudaStream_t)stream);
}

int32_t nys_sketch_solve(const nys_factor* f, const double* mu, int64_t nrhs, const void* b,
                         void* x, int32_t dtype, void* stream) {
  if (!f || !b || !x || nrhs < 1 || !mu) return NYS_ERR_ARG;
  if (dtype != NYS_F64 && dtype != NYS_F32) return NYS_ERR_ARG;
  if (b == x) return NYS_ERR_ARG;
  for (int64_t q = 0; q < nrhs; ++q)
    if (!(mu[q] > 0.0) || !std::isfinite(mu[q])) return NYS_ERR_ARG;
  return sketch_solve(f, mu, nrhs, b, x, dtype, (cudaStream_t)stream);
}

int32_t pcg_solve(const nys_operator* op, const nys_factor* f, const double* mu, int64_t nsys,
                  const double* b, double* x, const nys_pcg_opts* opts, nys_pcg_result* results,
                  void* stream) {
  NYS_TRY(check_op(op));
  if (nsys < 1 || !b || !x || !results) return NYS_ERR_ARG;
  if (f && f->n != op->n) return NYS_ERR_ARG;
  NYS_TRY(check_mu(f, mu, nsys));
  nys_pcg_opts o;
  o.tol = 1e-8;
  o.maxit = 500;
  o.precision = NYS_PREC_F64;
  o.inner_tol = 1e-4;
  o.max_refine = 20;
  o.use_x0 = 0;
  o.residual_history = nullptr;
  if (opts) o = *opts;
  if (!(o.tol >= 0.0) || o.maxit < 0 || o.max_refine < 0) return NYS_ERR_ARG;
  if (o.precision != NYS_PREC_F64 && o.precision != NYS_PREC_MIXED) return NYS_ERR_ARG;
  if (o.precision == NYS_PREC_MIXED && !(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t st;
  if (o.precision == NYS_PREC_F64)
    st = pcg_f64(op, f, mu, nsys, b, x, o.tol, o.maxit, o.use_x0, o.residual_history, results, s);
  else
    st = pcg_mixed(op, f, mu, nsys, b, x, o.tol, o.inner_tol, o.maxit, o.max_refine, o.use_x0,
                   o.residual_history, results, s);
  if (st != NYS_OK) return st;
  int32_t worst = NYS_OK;
  for (int64_t q = 0; q < nsys; ++q) {
    int32_t r = results[q].status;
    if (r == NYS_ERR_BREAKDOWN) worst = NYS_ERR_BREAKDOWN;
    else if (r == NYS_ERR_MAXIT && worst == NYS_OK) worst = NYS_ERR_MAXIT;
  }
  return worst;
}

int32_t nys_block_pcg(const nys_operator* op, const nys_factor* f, double mu, int64_t nrhs,
                      const double* b, double* x, const nys_pcg_opts* opts,
                      nys_pcg_result* results, void* stream) {
  NYS_TRY(check_op(op));
  if (nrhs < 1 || nrhs > 32 || !b || !x || !results) return NYS_ERR_ARG;
  if (f && f->n != op->n) return NYS_ERR_ARG;
  NYS_TRY(check_mu(f, &mu, 1));
  nys_pcg_opts o;
  o.tol = 1e-8;
  o.maxit = 500;
  o.precision = NYS_PREC_F64;
  o.inner_tol = 1e-4;
  o.max_refine = 20;
  o.use_x0 = 0;
  o.residual_history = nullptr;
  if (opts) o = *opts;
  if (!(o.tol >= 0.0) || o.maxit < 0 || o.max_refine < 0) return NYS_ERR_ARG;
  if (o.precision != NYS_PREC_F64 && o.precision != NYS_PREC_MIXED) return NYS_ERR_ARG;
  if (o.precision == NYS_PREC_MIXED && !(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t st;
  if (o.precision == NYS_PREC_F64)
    st = block_pcg_f64(op, f, mu, nrhs, b, x, o.tol, o.maxit, o.use_x0, results, s);
  else
    st = block_pcg_mixed(op, f, mu, nrhs, b, x, o.tol, o.inner_tol, o.maxit, o.max_refine,
                         o.use_x0, results, s);
  if (st != NYS_OK) return st;
  int32_t worst = NYS_OK;
  for (int64_t q = 0; q < nrhs; ++q) {
    int32_t r = results[q].status;
    if (r == NYS_ERR_BREAKDOWN) worst = NYS_ERR_BREAKDOWN;
    else if (r == NYS_ERR_MAXIT && worst == NYS_OK) worst = NYS_ERR_MAXIT;
  }
  return worst;
}

int32_t nys_reg_path(const nys_operator* op, int64_t count, const double* mus, const double* b,
                     double* x, int64_t ell0, int64_t ell_max, double err_factor, int32_t q,
                     uint64_t seed, const double* omegas, const double* gs,
                     const nys_pcg_opts* opts, nys_path_result* results, void* stream) {
  NYS_TRY(check_op(op));
  const int64_t n = op->n;
  if (count < 1 || !mus || !b || !x || !results) return NYS_ERR_ARG;
  for (int64_t i = 0; i < count; ++i)
    if (!(mus[i] > 0.0) || !std::isfinite(mus[i])) return NYS_ERR_ARG;
  if (ell0 < 1 || ell0 > ell_max || ell_max > n || ell_max > kMaxEll) return NYS_ERR_ARG;
  if (!(err_factor > 0.0) || !std::isfinite(err_factor) || q < 1) return NYS_ERR_ARG;
  nys_pcg_opts o;
  o.tol = 1e-8;
  o.maxit = 500;
  o.precision = NYS_PREC_F64;
  o.inner_tol = 1e-4;
  o.max_refine = 20;
  if (opts) o = *opts;
  o.residual_history = nullptr;
  if (o.precision != NYS_PREC_F64 && o.precision != NYS_PREC_MIXED) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int64_t> order(count);
  for (int64_t i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t a, int64_t c) { return mus[a] > mus[c]; });
  const int64_t kmax = (int64_t)std::ceil(std::log2((double)ell_max / (double)ell0)) + 1;
  nys_factor* f = nullptr;
  double E = INFINITY;
  bool capped = false;
  int64_t builds = 0;
  const double* xprev = nullptr;
  int32_t worst = NYS_OK;
  for (int64_t idx : order) {
    const double mu = mus[idx], tol_e = err_factor * mu;
    int resk = 0;
    if (!f || (!capped && !(E <= tol_e))) {
      const int64_t start = f ? std::min<int64_t>(2 * f->ell, ell_max) : ell0;
      const double* om = omegas ? omegas + builds * n * ell_max : nullptr;
      const double* g = gs ? gs + builds * kmax * n : nullptr;
      nys_factor* nf = nullptr;
      nys_adapt_info info;
      int32_t st = nys_sketch_adaptive(op, start, ell_max, NYS_RULE_ERR, tol_e, q, mu,
                                       seed + (uint64_t)builds, om, g, o.precision, &nf, &info,
                                       stream);
      if (st != NYS_OK) {
        if (f) nys_factor_free(f);
        return st;
      }
      if (f) nys_factor_free(f);
      f = nf;
      E = info.err_est;
      capped = f->ell >= ell_max;
      ++builds;
      resk = 1;
    }
    double* xi = x + idx * n;
    if (xprev) {
      cudaError_t ce = cudaMemcpyAsync(xi, xprev, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
      if (ce != cudaSuccess) {
        nys_factor_free(f);
        NYS_CUDA_TRY(ce);
      }
    }
    nys_pcg_opts oo = o;
    oo.use_x0 = xprev ? 1 : 0;
    nys_pcg_result r;
    int32_t st = pcg_solve(op, f, &mu, 1, b, xi, &oo, &r, stream);
    if (st != NYS_OK && st != NYS_ERR_MAXIT && st != NYS_ERR_BREAKDOWN) {
      nys_factor_free(f);
      return st;
    }
    nys_path_result& pr = results[idx];
    pr.status = r.status;
    pr.iterations = r.iterations;
    pr.resketched = resk;
    pr.refinements = r.refinements;
    pr.ell = f->ell;
    pr.err_est = E;
    pr.rel_residual = r.rel_residual;
    if (r.status == NYS_ERR_BREAKDOWN) worst = NYS_ERR_BREAKDOWN;
    else if (r.status == NYS_ERR_MAXIT && worst == NYS_OK) worst = NYS_ERR_MAXIT;
    xprev = xi;
  }
  nys_factor_free(f);
  return worst;
}

int32_t nys_factor_get(const nys_factor* f, const void** U, int32_t* u_dtype,
                       const double** lambda_hat, int64_t* n, int64_t* ell, double* nu) {
  if (!f) return NYS_ERR_ARG;
  if (U) *U = f->U;
  if (u_dtype) *u_dtype = f->u_dtype;
  if (lambda_hat) *lambda_hat = f->lam;
  if (n) *n = f->n;
  if (ell) *ell = f->ell;
  if (nu) *nu = f->nu;
  return NYS_OK;
}

int32_t nys_timing_start(int32_t max_products) { return timing_start(max_products); }

int32_t nys_timing_stop(double* total_ms, int64_t* products) {
  return timing_stop(total_ms, products);
}

int32_t nys_factor_stats(const nys_factor* f, int32_t* shift_escalations, int32_t* svd_sweeps,
                         int32_t* svd_refinements, double* lambda_ell) {
  if (!f) return NYS_ERR_ARG;
  if (shift_escalations) *shift_escalations = f->escalations;
  if (svd_sweeps) *svd_sweeps = f->svd_sweeps;
  if (svd_refinements) *svd_refinements = f->svd_refine;
  if (lambda_ell) *lambda_ell = f->lam_ell;
  return NYS_OK;
}

void nys_factor_free(nys_factor* f) {
  if (!f) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != f->device) cudaSetDevice(f->device);
  cudaDeviceSynchronize();
  if (f->U) cudaFree(f->U);
  if (f->lam) cudaFree(f->lam);
  if (f->E) cudaFree(f->E);
  if (cur != f->device) cudaSetDevice(cur);
  delete f;
}

int32_t nys_op_matvec(const nys_operator* op, double mu, int64_t nvec, const double* x, double* y,
                      int32_t mode, void* stream) {
  NYS_TRY(check_op(op));
  if (nvec < 1 || !x || !y || x == y) return NYS_ERR_ARG;
  if (!(mu >= 0.0) || !std::isfinite(mu)) return NYS_ERR_ARG;
  if (mode != 0 && mode != 1 && mode != 2) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = op->n;
  Scratch sc(s);
  unsigned char* work;
  NYS_TRY(sc.get(&work, op_matvec_work_bytes(op, mode != 1)));
  NYS_CUDA_TRY(cudaMemsetAsync(work, 0, 256, s));
  if (mode == 0) {
    for (int64_t q = 0; q < nvec; ++q)
      NYS_TRY(op_matvec_f64(op, mu, x + q * n, y + q * n, nullptr, work, s));
  } else if (mode == 2) {
    if (op->kind == NYS_OP_RBF && op->d <= 64) {
      // all vectors in one pass over the kernel
      std::vector<double> mus(nvec, mu);
      double* d_mu;
      NYS_TRY(sc.get(&d_mu, nvec));
      NYS_CUDA_TRY(cudaMemcpyAsync(d_mu, mus.data(), nvec * sizeof(double),
                                   cudaMemcpyHostToDevice, s));
      NYS_TRY(rbf_residual_products(op, d_mu, nvec, x, y, s));
    } else {
      for (int64_t q = 0; q < nvec; ++q)
        NYS_TRY(op_matvec_residual(op, mu, x + q * n, y + q * n, nullptr, work, s));
    }
  } else {
    float *xf, *yf;
    NYS_TRY(sc.get(&xf, nvec * n));
    NYS_TRY(sc.get(&yf, nvec * n));
    NYS_TRY(convert_f64_to_f32(x, xf, nvec * n, s));
    if (op->kind == NYS_OP_RBF && nvec > 1 && rbf_tc_supported(op->d)) {
      // all vectors in one pass over the kernel matrix
      NYS_TRY(rbf_tc_products((const float*)op->data, n, op->d, op->ld, op->sigma, nvec, xf, n, 1,
                              nullptr, mu, yf, n, 3, nullptr, 0, nullptr,
                              reinterpret_cast<int*>(work), s));
    } else {
      for (int64_t q = 0; q < nvec; ++q)
        NYS_TRY(op_matvec_f32(op, mu, xf + q * n, yf + q * n, nullptr, work, s));
    }
    NYS_TRY(convert_f32_to_f64(yf, y, nvec * n, s));
  }
  int err = 0;
  NYS_CUDA_TRY(cudaMemcpyAsync(&err, work, sizeof(int), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return err ? NYS_ERR_TIMEOUT : NYS_OK;
}

int32_t nys_rbf_cross_matvec(const float* targets, int64_t nt, int64_t ldt, const float* points,
                             int64_t n, int64_t ldp, int64_t d, double sigma, int64_t nvec,
                             const double* v, double* out, int32_t kind, void* stream) {
  if (!targets || !points || !v || !out || nt < 1 || n < 1 || nvec < 1) return NYS_ERR_ARG;
  if (d < 1 || d > 64 || ldt < d || ldp < d) return NYS_ERR_ARG;
  if (!(sigma > 0.0) || !std::isfinite(sigma) || (kind != 0 && kind != 1)) return NYS_ERR_ARG;
  if ((const void*)v == (const void*)out) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  NYS_TRY(rbf_dfl_products(targets, nt, ldt, points, n, ldp, d, sigma, kind, nullptr, nvec, v, out,
                           s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

int32_t nys_gemm_tf32_tn(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                         const float* B, int64_t ldb, float* D, int64_t ldd, void* stream) {
  if (!A || !B || !D || ldd < N) return NYS_ERR_ARG;
  if (!tc_gemm_supported(M, N, K, A, lda, B, ldb)) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  int* err;
  NYS_TRY(sc.get(&err, 1));
  NYS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  NYS_TRY(tc_gemm_tn_f32(M, N, K, A, lda, B, ldb, D, ldd, err, s));
  int h = 0;
  NYS_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return h ? NYS_ERR_TIMEOUT : NYS_OK;
}

int32_t nys_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out,
                          void* stream) {
  if (count < 0 || (count > 0 && (!ctr || !key || !out))) return NYS_ERR_ARG;
  if (count > ((int64_t)1 << 40)) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  NYS_TRY(philox_blocks(ctr, key, count, out, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

int32_t nys_random_stream(uint64_t seed, uint64_t stream_id, int64_t first, int64_t count,
                          uint32_t* words, double* gauss, void* stream) {
  if (first < 0 || count < 0 || (count > 0 && !words && !gauss)) return NYS_ERR_ARG;
  if (first > ((int64_t)1 << 60) || count > ((int64_t)1 << 40)) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  NYS_TRY(philox_stream(words, gauss, first, count, seed, stream_id, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

int32_t nys_power_err_est(const nys_operator* op, const nys_factor* f, const double* g, int32_t q,
                          double* est, void* stream) {
  NYS_TRY(check_op(op));
  if (!f || !g || !est || q < 1 || f->n != op->n) return NYS_ERR_ARG;
  return power_estimate(op, f, g, q, est, (cudaStream_t)stream);
}

}  // extern "C"
