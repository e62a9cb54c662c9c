// Kernel ridge regression objective and gradient scalars (Sec. 6.5, Eq. (6.3)
// trains KRR with the Gaussian kernel; the gradient is implicit
// differentiation of the training solve, which the paper does not state):
//
//   alpha = (K + mu I)^{-1} b,  pred = K_v alpha,  L = mean((pred - y_v)^2)
//   g     = (2/m)(pred - y_v),  lambda = (K + mu I)^{-1} K_v^T g
//   dL/db = lambda,  dL/dmu = -lambda^T alpha,
//   dL/dsigma = g^T (dK_v/dsigma) alpha - lambda^T (dK/dsigma) alpha
//
// The products with K, K_v and their sigma-derivatives are the double-FP32
// Gaussian products of rbf_residual.cu (FP64 inputs and outputs); the dot
// products here are FP64 with a fixed reduction order (one block, fixed
// thread count), so every scalar is bitwise reproducible.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace nys {

constexpr int KR_THREADS = 1024;

// out[k] = sum_i u_k[i] w_k[i] for the pairs k < npairs (one block per pair).
struct DotPairs {
  const double* u[3];
  const double* w[3];
};

__global__ void __launch_bounds__(KR_THREADS) dot_pairs_kernel(DotPairs dp, int64_t n,
                                                               double* out) {
  __shared__ double red[KR_THREADS / 32];
  const double* u = dp.u[blockIdx.x];
  const double* w = dp.w[blockIdx.x];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += KR_THREADS) acc = fma(u[i], w[i], acc);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// resid = pred - yv; g = (2/m) resid; one block: loss = mean(resid^2)
__global__ void __launch_bounds__(KR_THREADS) mse_kernel(const double* __restrict__ pred,
                                                         const double* __restrict__ yv, int64_t m,
                                                         double* __restrict__ g,
                                                         double* __restrict__ loss) {
  __shared__ double red[KR_THREADS / 32];
  const double c = 2.0 / (double)m;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += KR_THREADS) {
    const double r = pred[i] - yv[i];
    g[i] = c * r;
    acc = fma(r, r, acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) loss[0] = acc / (double)m;
}

static int32_t dots(const DotPairs& dp, int npairs, int64_t n, double* host_out, cudaStream_t s) {
  Scratch sc(s);
  double* d;
  NYS_TRY(sc.get(&d, 3));
  dot_pairs_kernel<<<npairs, KR_THREADS, 0, s>>>(dp, n, d);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  NYS_CUDA_TRY(cudaMemcpyAsync(host_out, d, npairs * sizeof(double), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

static bool rbf_args_ok(const float* p, int64_t n, int64_t ld, int64_t d) {
  return p && n >= 1 && d >= 1 && d <= 64 && ld >= d;
}

}  // namespace nys

using namespace nys;

extern "C" {

int32_t nys_krr_validation(const float* points, int64_t n, int64_t ldp, const float* vpoints,
                           int64_t m, int64_t ldv, int64_t d, double sigma, const double* alpha,
                           const double* yv, double* loss, double* g, double* ktg, void* stream) {
  if (!rbf_args_ok(points, n, ldp, d) || !rbf_args_ok(vpoints, m, ldv, d)) return NYS_ERR_ARG;
  if (!(sigma > 0.0) || !std::isfinite(sigma) || !alpha || !yv || !loss || !g || !ktg)
    return NYS_ERR_ARG;
  if ((const void*)g == (const void*)ktg || (const void*)ktg == (const void*)alpha)
    return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double *pred, *dl;
  NYS_TRY(sc.get(&pred, m));
  NYS_TRY(sc.get(&dl, 1));
  // pred = K_v alpha (targets: validation points)
  NYS_TRY(rbf_dfl_products(vpoints, m, ldv, points, n, ldp, d, sigma, 0, nullptr, 1, alpha, pred,
                           s));
  mse_kernel<<<1, KR_THREADS, 0, s>>>(pred, yv, m, g, dl);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  // K_v^T g: the kernel is symmetric in its arguments, so targets = training points
  NYS_TRY(rbf_dfl_products(points, n, ldp, vpoints, m, ldv, d, sigma, 0, nullptr, 1, g, ktg, s));
  NYS_CUDA_TRY(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

int32_t nys_krr_gradients(const float* points, int64_t n, int64_t ldp, const float* vpoints,
                          int64_t m, int64_t ldv, int64_t d, double sigma, const double* alpha,
                          const double* lam, const double* g, double* out, void* stream) {
  if (!rbf_args_ok(points, n, ldp, d) || !alpha || !lam || !out) return NYS_ERR_ARG;
  if (vpoints && (!rbf_args_ok(vpoints, m, ldv, d) || !g)) return NYS_ERR_ARG;
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return NYS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  double *dka, *dkva = nullptr;
  NYS_TRY(sc.get(&dka, n));
  // (dK/dsigma) alpha over the training points
  NYS_TRY(rbf_dfl_products(points, n, ldp, points, n, ldp, d, sigma, 1, nullptr, 1, alpha, dka,
                           s));
  DotPairs dp{};
  dp.u[0] = lam;
  dp.w[0] = alpha;
  dp.u[1] = lam;
  dp.w[1] = dka;
  double h[3] = {0.0, 0.0, 0.0};
  NYS_TRY(dots(dp, 2, n, h, s));
  double pred_term = 0.0;
  if (vpoints) {
    // (dK_v/dsigma) alpha on the validation points, then g^T of it
    NYS_TRY(sc.get(&dkva, m));
    NYS_TRY(rbf_dfl_products(vpoints, m, ldv, points, n, ldp, d, sigma, 1, nullptr, 1, alpha, dkva,
                             s));
    DotPairs dv{};
    dv.u[0] = g;
    dv.w[0] = dkva;
    double hv[3] = {0.0, 0.0, 0.0};
    NYS_TRY(dots(dv, 1, m, hv, s));
    pred_term = hv[0];
  }
  out[0] = -h[0];
  out[1] = pred_term - h[1];
  return NYS_OK;
}

}  // extern "C"
