// Nystrom PCG (Algorithm 3, Sec. 5.2) and the preconditioner apply of
// Eq. (5.3), for one or many independent systems (A + mu_s I) x_s = b_s that
// share the operator and the factor (U, lambda_hat).
//
// One iteration is five stream-ordered launches:
//   matvec       v = (A + mu I) p                         (operator kernels)
//   pv_alpha     alpha = (r^T z) / (p^T v)                 breakdown check
//   update       x += alpha p, r -= alpha v, ||r||^2, W = U^T r (partials);
//                the last block reduces W into w'_j = ((lam_ell+mu)/(lam_j+mu) - 1) w_j,
//                counts the iteration and sets `done` on convergence or cap
//   z            z = r + U w' = P^{-1} r (Eq. (5.3)),  r^T z -> beta
//   p            p = z + beta p
// Scalars live on the device in FP64; every dot product is a two-phase
// fixed-order reduction (per-block partials, summed by the last block to
// arrive), so results do not depend on scheduling.  Once a system's `done`
// word is set every kernel of that system returns at once, so the host can
// enqueue several iterations between convergence checks.

#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nys {

struct SysState {
  double mu;
  double lam_ell_mu;  // lambda_hat_ell + mu
  double rz, pv, alpha, beta, rr, thresh2;
  int it, done, status, maxit;
};

constexpr int PC_THREADS = 256;
constexpr int PC_JPT = 16;  // U columns per thread in the U^T r partials (ell <= 4096)

template <typename T, typename TU>
struct PcgArgs {
  int64_t n, ell, nsys;
  const TU* U;            // n x ell or NULL (plain CG)
  const double* lam;      // ell
  SysState* st;           // [nsys]
  T *x, *r, *z, *p, *v;   // [nsys][n]
  TU* wpart;              // [nsys][nblk_u][ell]
  T* w;                   // [nsys][ell]  (w' = coefficient * U^T r)
  double* dpart;          // [nsys][nblk] dot partials
  unsigned int* counters; // [nsys][4]
  int64_t nblk_u;         // blocks of the update kernel (row chunks)
  int64_t rows_u;         // rows per update block
  int64_t nblk_d;         // blocks of the dot kernels
  double* hist;           // [nsys][maxit+1] or NULL
};

// -------------------------------------------------------------- kernels

template <typename T, typename TU>
__global__ void __launch_bounds__(PC_THREADS)
pv_alpha_kernel(PcgArgs<T, TU> a) {
  const int64_t sidx = blockIdx.y;
  SysState* st = a.st + sidx;
  if (st->done) return;
  __shared__ double red[32];
  const T* p = a.p + sidx * a.n;
  const T* v = a.v + sidx * a.n;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * PC_THREADS + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * PC_THREADS)
    acc += (double)p[i] * (double)v[i];
  acc = block_sum(acc, red);
  double* part = a.dpart + sidx * a.nblk_d;
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
  if (last_block_arrived(a.counters + sidx * 4 + 0)) {
    double t = 0.0;
    for (int64_t b = threadIdx.x; b < gridDim.x; b += PC_THREADS) t += __ldcg(part + b);
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
      st->pv = t;
      if (!(t > 0.0) || !isfinite(t) || !isfinite(st->rz)) {
        st->status = NYS_ERR_BREAKDOWN;
        st->done = 1;
      } else {
        st->alpha = st->rz / t;
      }
    }
  }
}

// update (do_update) + ||r||^2 + U^T r partials; last block finishes w', the
// iteration count and the convergence test.
template <typename T, typename TU>
__global__ void __launch_bounds__(PC_THREADS)
update_kernel(PcgArgs<T, TU> a, int do_update) {
  const int64_t sidx = blockIdx.y;
  SysState* st = a.st + sidx;
  if (st->done) return;
  __shared__ double red[32];
  __shared__ T rs[PC_THREADS];
  T* x = a.x + sidx * a.n;
  T* r = a.r + sidx * a.n;
  const T* p = a.p + sidx * a.n;
  const T* v = a.v + sidx * a.n;
  const double alpha = st->alpha;
  const int64_t i0 = (int64_t)blockIdx.x * a.rows_u;
  const int64_t i1 = (i0 + a.rows_u < a.n) ? i0 + a.rows_u : a.n;
  TU acc[PC_JPT];
#pragma unroll
  for (int k = 0; k < PC_JPT; ++k) acc[k] = TU(0);
  double rr = 0.0;
  for (int64_t c0 = i0; c0 < i1; c0 += PC_THREADS) {
    int64_t i = c0 + threadIdx.x;
    T ri = T(0);
    if (i < i1) {
      ri = r[i];
      if (do_update) {
        x[i] = (T)((double)x[i] + alpha * (double)p[i]);
        ri = (T)((double)ri - alpha * (double)v[i]);
        r[i] = ri;
      }
      rr += (double)ri * (double)ri;
    }
    __syncthreads();
    rs[threadIdx.x] = ri;
    __syncthreads();
    if (a.U) {
      int64_t rows = (i1 - c0 < PC_THREADS) ? i1 - c0 : PC_THREADS;
      for (int64_t t = 0; t < rows; ++t) {
        const TU* urow = a.U + (c0 + t) * a.ell;
        const TU rt = (TU)rs[t];
#pragma unroll
        for (int k = 0; k < PC_JPT; ++k) {
          int64_t j = threadIdx.x + (int64_t)k * PC_THREADS;
          if (j < a.ell) acc[k] = fma(urow[j], rt, acc[k]);
        }
      }
    }
  }
  rr = block_sum(rr, red);
  double* part = a.dpart + sidx * a.nblk_d;
  if (threadIdx.x == 0) part[blockIdx.x] = rr;
  if (a.U) {
    TU* wp = a.wpart + (sidx * a.nblk_u + blockIdx.x) * a.ell;
#pragma unroll
    for (int k = 0; k < PC_JPT; ++k) {
      int64_t j = threadIdx.x + (int64_t)k * PC_THREADS;
      if (j < a.ell) wp[j] = acc[k];
    }
  }
  if (last_block_arrived(a.counters + sidx * 4 + 1)) {
    double t = 0.0;
    for (int64_t b = threadIdx.x; b < gridDim.x; b += PC_THREADS) t += __ldcg(part + b);
    t = block_sum(t, red);
    if (a.U) {
      const double lm = st->lam_ell_mu, mu = st->mu;
      const TU* wp = a.wpart + sidx * a.nblk_u * a.ell;
      T* w = a.w + sidx * a.ell;
      for (int64_t j = threadIdx.x; j < a.ell; j += PC_THREADS) {
        TU s = TU(0);
        for (int64_t b = 0; b < gridDim.x; ++b) s += __ldcg(wp + b * a.ell + j);
        double coef = lm / (a.lam[j] + mu) - 1.0;
        w[j] = (T)(coef * (double)s);
      }
    }
    if (threadIdx.x == 0) {
      st->rr = t;
      if (do_update) st->it += 1;
      if (a.hist) a.hist[sidx * (st->maxit + 1) + st->it] = sqrt(t);
      if (!isfinite(t)) {
        st->status = NYS_ERR_BREAKDOWN;
        st->done = 1;
      } else if (t <= st->thresh2) {
        st->done = 1;
      } else if (st->it >= st->maxit) {
        st->status = NYS_ERR_MAXIT;
        st->done = 1;
      }
    }
  }
}

// z = r + U w' (= P^{-1} r), r^T z; last block: beta (setup: rz only).
template <typename T, typename TU>
__global__ void __launch_bounds__(PC_THREADS)
z_kernel(PcgArgs<T, TU> a, int setup) {
  const int64_t sidx = blockIdx.y;
  SysState* st = a.st + sidx;
  if (st->done && !setup) return;
  extern __shared__ unsigned char zsm[];
  T* ws = reinterpret_cast<T*>(zsm);
  __shared__ double red[32];
  const T* r = a.r + sidx * a.n;
  T* z = a.z + sidx * a.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (a.U)
    for (int64_t j = threadIdx.x; j < a.ell; j += PC_THREADS) ws[j] = a.w[sidx * a.ell + j];
  __syncthreads();
  double rz = 0.0;
  const int64_t wstride = (int64_t)gridDim.x * (PC_THREADS / 32);
  for (int64_t i = (int64_t)blockIdx.x * (PC_THREADS / 32) + warp; i < a.n; i += wstride) {
    T zi = r[i];
    if (a.U) {
      const TU* urow = a.U + i * a.ell;
      T s = T(0);
      for (int64_t j = lane; j < a.ell; j += 32) s = fma((T)urow[j], ws[j], s);
      s = warp_sum(s);
      zi = zi + s;
    }
    if (lane == 0) {
      z[i] = zi;
      rz += (double)r[i] * (double)zi;
    }
  }
  rz = block_sum(rz, red);
  double* part = a.dpart + sidx * a.nblk_d;
  if (threadIdx.x == 0) part[blockIdx.x] = rz;
  if (last_block_arrived(a.counters + sidx * 4 + 2)) {
    double t = 0.0;
    for (int64_t b = threadIdx.x; b < gridDim.x; b += PC_THREADS) t += __ldcg(part + b);
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
      if (setup) {
        st->rz = t;
      } else {
        st->beta = t / st->rz;
        st->rz = t;
      }
    }
  }
}

template <typename T, typename TU>
__global__ void p_kernel(PcgArgs<T, TU> a, int setup) {
  const int64_t sidx = blockIdx.y;
  SysState* st = a.st + sidx;
  if (st->done && !setup) return;
  const double beta = setup ? 0.0 : st->beta;
  const T* z = a.z + sidx * a.n;
  T* p = a.p + sidx * a.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = setup ? z[i] : (T)((double)z[i] + beta * (double)p[i]);
}

// r = b - v (v = A_mu x0) or r = b; x = x0 or 0.
template <typename T>
__global__ void init_r_kernel(const double* __restrict__ b, const T* __restrict__ v, T* r, T* x,
                              int64_t n, int use_x0) {
  const int64_t sidx = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double bi = b[sidx * n + i];
    if (use_x0) {
      r[sidx * n + i] = (T)(bi - (double)v[sidx * n + i]);
    } else {
      r[sidx * n + i] = (T)bi;
      x[sidx * n + i] = T(0);
    }
  }
}

// ||b||^2 per system -> thresh2 = tol^2 ||b||^2 (fixed order; one block per system).
template <typename T>
__global__ void init_state_kernel(const T* __restrict__ b, int64_t n, SysState* st,
                                  const double* mus, double lam_ell, double tol, int maxit) {
  __shared__ double red[32];
  const int64_t sidx = blockIdx.x;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double v = (double)b[sidx * n + i];
    acc += v * v;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    SysState s;
    memset(&s, 0, sizeof(s));
    s.mu = mus[sidx];
    s.lam_ell_mu = lam_ell + mus[sidx];
    s.thresh2 = tol * tol * acc;
    s.maxit = maxit;
    st[sidx] = s;
  }
}

// -------------------------------------------------------------- host driver

template <typename T, typename TU>
struct PcgBuffers {
  PcgArgs<T, TU> a;
  SysState* st = nullptr;
  double* d_mu = nullptr;
  void* op_work = nullptr;
  std::vector<void*> allocs;
  cudaStream_t s;
  ~PcgBuffers() {
    for (void* p : allocs) dfree(p, s);
  }
  int32_t get(void** p, size_t bytes) {
    NYS_TRY(dmalloc(p, bytes + 256, s));
    allocs.push_back(*p);
    return NYS_OK;
  }
};

template <typename T>
static int32_t matvec_T(const nys_operator* op, double mu, const T* p, T* v, const int* skip,
                        void* work, cudaStream_t s);
template <>
int32_t matvec_T<float>(const nys_operator* op, double mu, const float* p, float* v,
                        const int* skip, void* work, cudaStream_t s) {
  return op_matvec_f32(op, mu, p, v, skip, work, s);
}
template <>
int32_t matvec_T<double>(const nys_operator* op, double mu, const double* p, double* v,
                         const int* skip, void* work, cudaStream_t s) {
  return op_matvec_f64(op, mu, p, v, skip, work, s);
}

// Runs Algorithm 3 on T vectors.  x (device, T, [nsys][n]) receives the
// solution; b_dev (device FP64 [nsys][n]) is the right-hand side; with
// use_x0 the incoming x is the initial guess.  Fills iterations/status.
template <typename T, typename TU>
static int32_t run_pcg(const nys_operator* op, const TU* U, const double* lam, int64_t ell,
                       double lam_ell, const double* mus_host, int64_t nsys, const double* b_dev,
                       const T* b_T, T* x, double tol, int maxit, int use_x0, double* hist,
                       int* iters_out, int* status_out, double* relres_out, cudaStream_t s) {
  const int64_t n = op->n;
  PcgBuffers<T, TU> B;
  B.s = s;
  PcgArgs<T, TU>& a = B.a;
  a.n = n;
  a.ell = U ? ell : 0;
  a.nsys = nsys;
  a.U = U;
  a.lam = lam;
  a.x = x;
  a.hist = hist;
  const int sms = num_sms();
  a.nblk_u = cdiv(n, 64);
  if (a.nblk_u > 2 * sms) a.nblk_u = 2 * sms;
  if (a.nblk_u < 1) a.nblk_u = 1;
  a.rows_u = cdiv(n, a.nblk_u);
  a.nblk_u = cdiv(n, a.rows_u);
  a.nblk_d = 2 * sms;
  if (a.nblk_d < a.nblk_u) a.nblk_d = a.nblk_u;
  const size_t vec = (size_t)nsys * n * sizeof(T);
  NYS_TRY(B.get((void**)&a.r, vec));
  NYS_TRY(B.get((void**)&a.z, vec));
  NYS_TRY(B.get((void**)&a.p, vec));
  NYS_TRY(B.get((void**)&a.v, vec));
  NYS_TRY(B.get((void**)&a.st, nsys * sizeof(SysState)));
  NYS_TRY(B.get((void**)&a.dpart, (size_t)nsys * a.nblk_d * sizeof(double)));
  NYS_TRY(B.get((void**)&a.counters, (size_t)nsys * 4 * sizeof(unsigned)));
  NYS_TRY(B.get((void**)&B.d_mu, nsys * sizeof(double)));
  if (U) {
    NYS_TRY(B.get((void**)&a.wpart, (size_t)nsys * a.nblk_u * ell * sizeof(TU)));
    NYS_TRY(B.get((void**)&a.w, (size_t)nsys * ell * sizeof(T)));
  }
  size_t wbytes = op_matvec_work_bytes(op, sizeof(T) == sizeof(double));
  NYS_TRY(B.get(&B.op_work, wbytes));
  NYS_CUDA_TRY(cudaMemsetAsync(B.op_work, 0, 256, s));
  NYS_CUDA_TRY(cudaMemsetAsync(a.counters, 0, (size_t)nsys * 4 * sizeof(unsigned), s));
  NYS_CUDA_TRY(cudaMemcpyAsync(B.d_mu, mus_host, nsys * sizeof(double), cudaMemcpyHostToDevice, s));
  if (hist) {
    // NaN padding
    std::vector<double> nanbuf((size_t)nsys * (maxit + 1), std::nan(""));
    NYS_CUDA_TRY(cudaMemcpyAsync(hist, nanbuf.data(), nanbuf.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  const unsigned gd = (unsigned)a.nblk_d;
  const dim3 g_d(gd, (unsigned)nsys), g_u((unsigned)a.nblk_u, (unsigned)nsys);
  const int64_t zblocks = a.nblk_d;
  const dim3 g_z((unsigned)zblocks, (unsigned)nsys);
  const size_t zsm = U ? ell * sizeof(T) : 0;
  if (zsm > 48 * 1024)
    NYS_CUDA_TRY(cudaFuncSetAttribute(z_kernel<T, TU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)zsm));

  // ---- setup: state, r0, z0 = P^{-1} r0, p0 = z0, r0^T z0
  init_state_kernel<T><<<(unsigned)nsys, 256, 0, s>>>(b_T, n, a.st, B.d_mu, lam_ell, tol, maxit); count_launch();
  if (use_x0) {
    for (int64_t q = 0; q < nsys; ++q)
      NYS_TRY(matvec_T<T>(op, mus_host[q], x + q * n, a.v + q * n, nullptr, B.op_work, s));
  }
  init_r_kernel<T><<<dim3(gd, (unsigned)nsys), 256, 0, s>>>(b_dev, a.v, a.r, x, n, use_x0); count_launch();
  update_kernel<T, TU><<<g_u, PC_THREADS, 0, s>>>(a, 0); count_launch();
  z_kernel<T, TU><<<g_z, PC_THREADS, zsm, s>>>(a, 1); count_launch();
  p_kernel<T, TU><<<g_d, 256, 0, s>>>(a, 1); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());

  // ---- iterations, checked every `chunk`
  std::vector<SysState> hst(nsys);
  int64_t launched = 0;
  int chunk = 4;
  while (true) {
    for (int c = 0; c < chunk && launched < maxit; ++c, ++launched) {
      for (int64_t q = 0; q < nsys; ++q)
        NYS_TRY(matvec_T<T>(op, mus_host[q], a.p + q * n, a.v + q * n, &a.st[q].done, B.op_work, s));
      pv_alpha_kernel<T, TU><<<g_d, PC_THREADS, 0, s>>>(a); count_launch();
      update_kernel<T, TU><<<g_u, PC_THREADS, 0, s>>>(a, 1); count_launch();
      z_kernel<T, TU><<<g_z, PC_THREADS, zsm, s>>>(a, 0); count_launch();
      p_kernel<T, TU><<<g_d, 256, 0, s>>>(a, 0); count_launch();
    }
    NYS_CUDA_TRY(cudaGetLastError());
    NYS_CUDA_TRY(cudaMemcpyAsync(hst.data(), a.st, nsys * sizeof(SysState), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    bool all = true;
    for (auto& h : hst) all = all && h.done;
    if (all || launched >= maxit) break;
    if (chunk < 16) chunk *= 2;
  }
  int err = 0;
  NYS_CUDA_TRY(cudaMemcpyAsync(&err, B.op_work, sizeof(int), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  if (err) return NYS_ERR_TIMEOUT;
  for (int64_t q = 0; q < nsys; ++q) {
    iters_out[q] = hst[q].it;
    int stq = hst[q].status;
    if (stq == NYS_OK && !hst[q].done) stq = NYS_ERR_MAXIT;
    status_out[q] = stq;
    relres_out[q] = hst[q].thresh2 > 0 ? sqrt(hst[q].rr * tol * tol / hst[q].thresh2)
                                        : sqrt(hst[q].rr);
  }
  return NYS_OK;
}

// -------------------------------------------------------------- entry helpers

template <typename T>
__global__ void axpy_to_f64_kernel(double* x, const T* d, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    x[e] += (double)d[e];
}

__global__ void sub_kernel(const double* b, const double* v, double* r, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    r[e] = b[e] - v[e];
}

// per-system sum of squares, one block per system (fixed order)
__global__ void sys_sumsq_kernel(const double* x, int64_t n, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double v = x[blockIdx.x * n + i];
    acc += v * v;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

int32_t pcg_f64(const nys_operator* op, const nys_factor* f, const double* mu, int64_t nsys,
                const double* b, double* x, double tol, int maxit, int use_x0, double* hist,
                nys_pcg_result* res, cudaStream_t s) {
  std::vector<int> it(nsys), stt(nsys);
  std::vector<double> rel(nsys);
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
  NYS_TRY((run_pcg<double, double>(op, U, f ? f->lam : nullptr, f ? f->ell : 0,
                                   f ? f->lam_ell : 0.0, mu, nsys, b, b, x, tol, maxit, use_x0,
                                   hist, it.data(), stt.data(), rel.data(), s)));
  for (int64_t q = 0; q < nsys; ++q) {
    res[q].status = stt[q];
    res[q].iterations = it[q];
    res[q].refinements = 0;
    res[q].reserved = 0;
    res[q].rel_residual = rel[q];
  }
  return NYS_OK;
}

// Mixed precision: FP64 outer loop r = b - (A + mu I) x (FP64-accurate
// matvec), inner Algorithm 3 on FP32 vectors for the correction.
int32_t pcg_mixed(const nys_operator* op, const nys_factor* f, const double* mu, int64_t nsys,
                  const double* b, double* x, double tol, double inner_tol, int maxit,
                  int max_refine, int use_x0, double* hist, nys_pcg_result* res, cudaStream_t s) {
  const int64_t n = op->n;
  Scratch sc(s);
  const float* U = nullptr;
  if (f) {
    if (f->u_dtype == NYS_F32) {
      U = (const float*)f->U;
    } else {
      float* Uf;
      NYS_TRY(sc.get(&Uf, f->n * f->ell));
      NYS_TRY(convert_f64_to_f32((const double*)f->U, Uf, f->n * f->ell, s));
      U = Uf;
    }
  }
  double *r, *v, *nrm;
  float *rf, *df;
  NYS_TRY(sc.get(&r, nsys * n));
  NYS_TRY(sc.get(&v, nsys * n));
  NYS_TRY(sc.get(&nrm, 2 * nsys));
  NYS_TRY(sc.get(&rf, nsys * n));
  NYS_TRY(sc.get(&df, nsys * n));
  unsigned char* work;
  size_t wbytes = op_matvec_work_bytes(op, true);
  NYS_TRY(sc.get(&work, wbytes));
  NYS_CUDA_TRY(cudaMemsetAsync(work, 0, 256, s));
  if (!use_x0) NYS_CUDA_TRY(cudaMemsetAsync(x, 0, nsys * n * sizeof(double), s));
  std::vector<double> bn2(nsys), rn2(nsys);
  sys_sumsq_kernel<<<(unsigned)nsys, 256, 0, s>>>(b, n, nrm); count_launch();
  NYS_CUDA_TRY(cudaMemcpyAsync(bn2.data(), nrm, nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
  std::vector<int> active(nsys, 1), total_it(nsys, 0), outer(nsys, 0), stt(nsys, NYS_ERR_MAXIT);
  std::vector<double> rel(nsys, 1.0);
  const unsigned gb = (unsigned)cdiv(n, 256) > 1024 ? 1024 : (unsigned)cdiv(n, 256);
  for (int k = 0; k <= max_refine; ++k) {
    // true residual in FP64 for every system
    for (int64_t q = 0; q < nsys; ++q)
      NYS_TRY(op_matvec_f64(op, mu[q], x + q * n, v + q * n, nullptr, work, s));
    sub_kernel<<<gb, 256, 0, s>>>(b, v, r, nsys * n); count_launch();
    sys_sumsq_kernel<<<(unsigned)nsys, 256, 0, s>>>(r, n, nrm); count_launch();
    NYS_CUDA_TRY(cudaMemcpyAsync(rn2.data(), nrm, nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int64_t> todo;
    for (int64_t q = 0; q < nsys; ++q) {
      rel[q] = bn2[q] > 0 ? sqrt(rn2[q] / bn2[q]) : sqrt(rn2[q]);
      if (!active[q]) continue;
      if (rel[q] <= tol) {
        active[q] = 0;
        stt[q] = NYS_OK;
      } else if (!std::isfinite(rel[q])) {
        active[q] = 0;
        stt[q] = NYS_ERR_BREAKDOWN;
      } else if (k < max_refine) {
        todo.push_back(q);
      }
    }
    if (todo.empty()) break;
    // inner solves for the systems still active (batched over them)
    int64_t na = (int64_t)todo.size();
    std::vector<double> mua(na);
    for (int64_t t = 0; t < na; ++t) {
      mua[t] = mu[todo[t]];
      // gather the residual of system todo[t] into slot t (FP64 -> FP32 rhs)
      NYS_CUDA_TRY(cudaMemcpyAsync(v + t * n, r + todo[t] * n, n * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
    }
    NYS_TRY(convert_f64_to_f32(v, rf, na * n, s));
    std::vector<int> it(na), st(na);
    std::vector<double> rr(na);
    NYS_TRY((run_pcg<float, float>(op, U, f ? f->lam : nullptr, f ? f->ell : 0,
                                   f ? f->lam_ell : 0.0, mua.data(), na, v, rf, df, inner_tol,
                                   maxit, 0, (k == 0) ? hist : nullptr, it.data(), st.data(),
                                   rr.data(), s)));
    for (int64_t t = 0; t < na; ++t) {
      int64_t q = todo[t];
      axpy_to_f64_kernel<float><<<gb, 256, 0, s>>>(x + q * n, df + t * n, n); count_launch();
      total_it[q] += it[t];
      outer[q] += 1;
      if (st[t] == NYS_ERR_BREAKDOWN) {
        active[q] = 0;
        stt[q] = NYS_ERR_BREAKDOWN;
      }
    }
    NYS_CUDA_TRY(cudaGetLastError());
  }
  for (int64_t q = 0; q < nsys; ++q) {
    res[q].status = stt[q];
    res[q].iterations = total_it[q];
    res[q].refinements = outer[q];
    res[q].reserved = 0;
    res[q].rel_residual = rel[q];
  }
  return NYS_OK;
}

// -------------------------------------------------------------- P^{-1} apply

template <typename T, typename TU>
static int32_t precond_apply_impl(const nys_factor* f, const TU* U, const double* mu,
                                  int64_t nrhs, const T* v, T* z, cudaStream_t s) {
  const int64_t n = f->n, ell = f->ell;
  PcgBuffers<T, TU> B;
  B.s = s;
  PcgArgs<T, TU>& a = B.a;
  a.n = n;
  a.ell = ell;
  a.nsys = nrhs;
  a.U = U;
  a.lam = f->lam;
  a.hist = nullptr;
  const int sms = num_sms();
  a.nblk_u = cdiv(n, 64);
  if (a.nblk_u > 2 * sms) a.nblk_u = 2 * sms;
  a.rows_u = cdiv(n, a.nblk_u);
  a.nblk_u = cdiv(n, a.rows_u);
  a.nblk_d = 2 * sms;
  if (a.nblk_d < a.nblk_u) a.nblk_d = a.nblk_u;
  a.r = const_cast<T*>(v);
  a.z = z;
  a.x = nullptr;
  a.p = nullptr;
  a.v = nullptr;
  NYS_TRY(B.get((void**)&a.st, nrhs * sizeof(SysState)));
  NYS_TRY(B.get((void**)&a.dpart, (size_t)nrhs * a.nblk_d * sizeof(double)));
  NYS_TRY(B.get((void**)&a.counters, (size_t)nrhs * 4 * sizeof(unsigned)));
  NYS_TRY(B.get((void**)&a.wpart, (size_t)nrhs * a.nblk_u * ell * sizeof(TU)));
  NYS_TRY(B.get((void**)&a.w, (size_t)nrhs * ell * sizeof(T)));
  NYS_TRY(B.get((void**)&B.d_mu, nrhs * sizeof(double)));
  NYS_CUDA_TRY(cudaMemsetAsync(a.counters, 0, (size_t)nrhs * 4 * sizeof(unsigned), s));
  NYS_CUDA_TRY(cudaMemcpyAsync(B.d_mu, mu, nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  // states: done = 0, thresh2 = -1 (never "converged"), maxit large
  init_state_kernel<T><<<(unsigned)nrhs, 256, 0, s>>>(v, n, a.st, B.d_mu, f->lam_ell, 0.0, 1 << 30); count_launch();
  const size_t zsm = ell * sizeof(T);
  if (zsm > 48 * 1024)
    NYS_CUDA_TRY(cudaFuncSetAttribute(z_kernel<T, TU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)zsm));
  update_kernel<T, TU><<<dim3((unsigned)a.nblk_u, (unsigned)nrhs), PC_THREADS, 0, s>>>(a, 0); count_launch();
  z_kernel<T, TU><<<dim3((unsigned)a.nblk_d, (unsigned)nrhs), PC_THREADS, zsm, s>>>(a, 1); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  // keep the buffers alive until the kernels have run
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

int32_t precond_apply(const nys_factor* f, const double* mu, int64_t nrhs, const void* v, void* z,
                      int32_t dtype, cudaStream_t s) {
  Scratch sc(s);
  if (dtype == NYS_F64) {
    const double* U = (const double*)f->U;
    if (f->u_dtype != NYS_F64) {
      double* Ud;
      NYS_TRY(sc.get(&Ud, f->n * f->ell));
      NYS_TRY(convert_f32_to_f64((const float*)f->U, Ud, f->n * f->ell, s));
      U = Ud;
    }
    return precond_apply_impl<double, double>(f, U, mu, nrhs, (const double*)v, (double*)z, s);
  }
  const float* U = (const float*)f->U;
  if (f->u_dtype != NYS_F32) {
    float* Uf;
    NYS_TRY(sc.get(&Uf, f->n * f->ell));
    NYS_TRY(convert_f64_to_f32((const double*)f->U, Uf, f->n * f->ell, s));
    U = Uf;
  }
  return precond_apply_impl<float, float>(f, U, mu, nrhs, (const float*)v, (float*)z, s);
}

}  // namespace nys
