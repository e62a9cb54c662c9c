// Nystrom PCG (Algorithm 3, Sec. 5.2) and the preconditioner apply of
// Eq. (5.3), for one or many independent systems (A + mu_s I) x_s = b_s that
// share the operator and the factor (U, lambda_hat).
//
// One iteration is six stream-ordered launches after the operator matvec:
//   matvec       v = (A + mu I) p                          (operator kernels)
//   pv_alpha     alpha = (r^T z) / (p^T v), breakdown check
//   update       x += alpha p, r -= alpha v; ||r||^2 and W = U^T r as
//                per-block partials (a warp walks 16-row groups of U with
//                16-byte loads; the row residuals are broadcast by shuffle)
//   wreduce      w'_j = ((lam_ell + mu)/(lam_j + mu) - 1) sum_b W_bj,
//                ||r||^2, iteration count, convergence / cap -> `done`
//   z            z = r + U w' = P^{-1} r,  r^T z -> beta
//   p            p = z + beta p
// Scalars live on the device in FP64.  Every reduction runs in a fixed order
// (per-block partials summed in index order), so results do not depend on
// scheduling.  Once a system's `done` word is set every kernel of that system
// returns at once, so the host enqueues several iterations between checks:
// by default it captures four iterations once per solve as a CUDA graph and
// replays that graph (IterGraph below).

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <algorithm>
#include <atomic>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nys {

struct SysState {
  double mu;
  double lam_ell_mu;  // lambda_hat_ell + mu
  double rz, pv, alpha, beta, rr, thresh2;
  int it, done, status, maxit;
  int conv;  // set by wreduce when the test passes; p_kernel promotes it to `done`
  int pad;
};

constexpr int PC_THREADS = 256;
constexpr int PC_WARPS = PC_THREADS / 32;
constexpr int PC_GROUP = 16;   // rows of U a warp handles per inner group
constexpr int PC_MAXRG = 4;    // 32-row register groups per warp (rows per warp <= 128)
constexpr int PC_CQ = 4;       // 16-byte vectors of U per lane per column chunk

template <typename T, typename TU>
struct PcgArgs {
  int64_t n, ell, nsys;
  const TU* U;            // n x ell or NULL (plain CG)
  const double* lam;      // ell
  SysState* st;           // [nsys]
  T *x, *r, *z, *p, *v;   // [nsys][n]
  TU* wpart;              // [nsys][nblk_u][ell]
  T* w;                   // [nsys][ell]  (w' = coefficient * U^T r)
  double* dpart;          // [nsys][npart] dot partials
  unsigned int* counters; // [nsys][4]
  int64_t nblk_u;         // blocks of the update / z kernels
  int64_t rows_w;         // rows per warp in the update / z kernels (multiple of 16, <= 128)
  int64_t nblk_d;         // blocks of the elementwise dot kernels
  int64_t npart;          // stride of dpart per system
  double* hist;           // [nsys][maxit+1] or NULL
  const float* E;         // U^T U - I (ell x ell) of an FP32 factor, or NULL
  T* wraw;                // [nsys][ell] U^T r (when E is set)
  T* wc;                  // [nsys][ell] coefficient * U^T r (when E is set)
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
  double* part = a.dpart + sidx * a.npart;
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

// 16-byte vector of U: VE elements of type TU.
template <typename TU, int VE>
struct UVec {
  TU e[VE];
};

template <typename TU, int VE>
__device__ __forceinline__ UVec<TU, VE> load_uvec(const TU* p) {
  UVec<TU, VE> v;
  if constexpr (VE == 4 && sizeof(TU) == 4) {
    float4 q = *reinterpret_cast<const float4*>(p);
    v.e[0] = q.x; v.e[1] = q.y; v.e[2] = q.z; v.e[3] = q.w;
  } else if constexpr (VE == 2 && sizeof(TU) == 8) {
    double2 q = *reinterpret_cast<const double2*>(p);
    v.e[0] = q.x; v.e[1] = q.y;
  } else {
#pragma unroll
    for (int k = 0; k < VE; ++k) v.e[k] = p[k];
  }
  return v;
}

// x += alpha p and r -= alpha v (do_update), ||r||^2 and W = U^T r partials.
// Warp w of block b owns rows [(b*PC_WARPS + w) * rows_w, +rows_w).  VE = U
// elements per vector load (16 bytes, or 1 when ell is not a multiple).
// Dynamic shared memory: PC_WARPS x (32 * PC_CQ * VE) values of TU.
template <typename T, typename TU, int VE>
__global__ void __launch_bounds__(PC_THREADS)
update_kernel(PcgArgs<T, TU> a, int do_update) {
  const int64_t sidx = blockIdx.y;
  SysState* st = a.st + sidx;
  if (st->done) return;
  extern __shared__ __align__(16) unsigned char usm[];
  TU* wsm = reinterpret_cast<TU*>(usm);
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* x = a.x + sidx * a.n;
  T* r = a.r + sidx * a.n;
  const T* p = a.p + sidx * a.n;
  const T* v = a.v + sidx * a.n;
  const double alpha = st->alpha;
  const int64_t row0 = ((int64_t)blockIdx.x * PC_WARPS + warp) * a.rows_w;
  const int nrg = (int)(a.rows_w / 32 + ((a.rows_w % 32) ? 1 : 0));

  // 1) residual update: lane owns rows row0 + 32 g + lane
  T rg[PC_MAXRG];
  double rr = 0.0;
#pragma unroll
  for (int g = 0; g < PC_MAXRG; ++g) {
    rg[g] = T(0);
    const int64_t i = row0 + 32 * g + lane;
    if (g < nrg && 32 * g + lane < a.rows_w && i < a.n) {
      T ri = r[i];
      if (do_update) {
        x[i] = (T)((double)x[i] + alpha * (double)p[i]);
        ri = (T)((double)ri - alpha * (double)v[i]);
        r[i] = ri;
      }
      rr += (double)ri * (double)ri;
      rg[g] = ri;
    }
  }
  rr = block_sum(rr, red);
  double* part = a.dpart + sidx * a.npart;
  if (threadIdx.x == 0) part[blockIdx.x] = rr;

  // 2) W = U^T r over this block's rows, one column chunk at a time
  if (a.U) {
    constexpr int CW = 32 * PC_CQ * VE;  // columns per chunk
    TU* wp = a.wpart + (sidx * a.nblk_u + blockIdx.x) * a.ell;
    const int64_t rows_here = (row0 < a.n) ? ((a.n - row0 < a.rows_w) ? a.n - row0 : a.rows_w) : 0;
    for (int64_t c0 = 0; c0 < a.ell; c0 += CW) {
      TU acc[PC_CQ][VE];
#pragma unroll
      for (int q = 0; q < PC_CQ; ++q)
#pragma unroll
        for (int k = 0; k < VE; ++k) acc[q][k] = TU(0);
      for (int64_t t0 = 0; t0 < rows_here; t0 += PC_GROUP) {
#pragma unroll 4
        for (int tt = 0; tt < PC_GROUP; ++tt) {
          const int64_t t = t0 + tt;
          const int g = (int)(t >> 5), src = (int)(t & 31);
          T rsel = rg[0];
#pragma unroll
          for (int gg = 1; gg < PC_MAXRG; ++gg)
            if (g == gg) rsel = rg[gg];
          const TU rt = (TU)__shfl_sync(0xffffffffu, rsel, src);
          if (t < rows_here) {
            const TU* urow = a.U + (row0 + t) * a.ell + c0;
#pragma unroll
            for (int q = 0; q < PC_CQ; ++q) {
              const int64_t col = (int64_t)(lane + 32 * q) * VE;
              if (c0 + col < a.ell) {
                UVec<TU, VE> u = load_uvec<TU, VE>(urow + col);
#pragma unroll
                for (int k = 0; k < VE; ++k) acc[q][k] = fma(u.e[k], rt, acc[q][k]);
              }
            }
          }
        }
      }
      // block combine over warps in a fixed order
#pragma unroll
      for (int q = 0; q < PC_CQ; ++q)
#pragma unroll
        for (int k = 0; k < VE; ++k) wsm[warp * CW + (lane + 32 * q) * VE + k] = acc[q][k];
      __syncthreads();
      for (int j = threadIdx.x; j < CW; j += PC_THREADS) {
        if (c0 + j < a.ell) {
          TU s = TU(0);
#pragma unroll
          for (int w = 0; w < PC_WARPS; ++w) s += wsm[w * CW + j];
          wp[c0 + j] = s;
        }
      }
      __syncthreads();
    }
  }
}

// w' = coefficient * sum over update blocks of W (fixed order); block 0 also
// finishes ||r||^2, counts the iteration and records convergence or the cap.  grid.x covers ell
// in chunks of 32 columns (at least one block).
template <typename T, typename TU>
__global__ void __launch_bounds__(PC_THREADS)
wreduce_kernel(PcgArgs<T, TU> a, int do_update) {
  const int64_t sidx = blockIdx.y;
  SysState* st = a.st + sidx;
  if (st->done) return;
  __shared__ double red[32];
  __shared__ TU ws[PC_WARPS][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (a.U) {
    const int64_t j = (int64_t)blockIdx.x * 32 + lane;
    const TU* wp = a.wpart + sidx * a.nblk_u * a.ell;
    TU s = TU(0);
    if (j < a.ell)
      for (int64_t b = warp; b < a.nblk_u; b += PC_WARPS) s += __ldcg(wp + b * a.ell + j);
    ws[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && j < a.ell) {
      TU tot = TU(0);
#pragma unroll
      for (int w = 0; w < PC_WARPS; ++w) tot += ws[w][lane];
      const double coef = st->lam_ell_mu / (a.lam[j] + st->mu) - 1.0;
      if (a.E) {
        a.wraw[sidx * a.ell + j] = (T)tot;
        a.wc[sidx * a.ell + j] = (T)(coef * (double)tot);
      } else {
        a.w[sidx * a.ell + j] = (T)(coef * (double)tot);
      }
    }
  }
  if (blockIdx.x == 0) {
    const double* part = a.dpart + sidx * a.npart;
    double t = 0.0;
    for (int64_t b = threadIdx.x; b < a.nblk_u; b += PC_THREADS) t += __ldcg(part + b);
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
      st->rr = t;
      if (do_update) st->it += 1;
      if (a.hist) a.hist[sidx * (st->maxit + 1) + st->it] = sqrt(t);
      // other blocks of this launch still read `done` at entry, so the
      // decision is recorded in `conv` and published by p_kernel
      if (!isfinite(t)) {
        st->status = NYS_ERR_BREAKDOWN;
        st->conv = 1;
      } else if (t <= st->thresh2) {
        st->conv = 1;
      } else if (st->it >= st->maxit) {
        st->status = NYS_ERR_MAXIT;
        st->conv = 1;
      }
    }
  }
}

// z = r + U w' (= P^{-1} r), r^T z; last block: beta (setup: rz only).  Same
// row ownership as update_kernel; w' is staged in shared memory.
template <typename T, typename TU, int VE>
__global__ void __launch_bounds__(PC_THREADS)
z_kernel(PcgArgs<T, TU> a, int setup) {
  const int64_t sidx = blockIdx.y;
  SysState* st = a.st + sidx;
  if (st->done && !setup) return;
  extern __shared__ __align__(16) unsigned char zsm[];
  TU* ws = reinterpret_cast<TU*>(zsm);
  __shared__ double red[32];
  const T* r = a.r + sidx * a.n;
  T* z = a.z + sidx * a.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (a.U)
    for (int64_t j = threadIdx.x; j < a.ell; j += PC_THREADS) ws[j] = (TU)a.w[sidx * a.ell + j];
  __syncthreads();
  const int64_t row0 = ((int64_t)blockIdx.x * PC_WARPS + warp) * a.rows_w;
  const int64_t rows_here = (row0 < a.n) ? ((a.n - row0 < a.rows_w) ? a.n - row0 : a.rows_w) : 0;
  double rz = 0.0;
  constexpr int ZB = 8;  // rows whose U loads are in flight together
  for (int64_t t0 = 0; t0 < rows_here; t0 += ZB) {
    TU sp[ZB];
#pragma unroll
    for (int b = 0; b < ZB; ++b) sp[b] = TU(0);
    if (a.U) {
      for (int64_t col = (int64_t)lane * VE; col < a.ell; col += 32 * VE) {
        const UVec<TU, VE> wv = load_uvec<TU, VE>(ws + col);
#pragma unroll
        for (int b = 0; b < ZB; ++b) {
          if (t0 + b < rows_here) {
            const UVec<TU, VE> u = load_uvec<TU, VE>(a.U + (row0 + t0 + b) * a.ell + col);
#pragma unroll
            for (int k = 0; k < VE; ++k) sp[b] = fma(u.e[k], wv.e[k], sp[b]);
          }
        }
      }
#pragma unroll
      for (int b = 0; b < ZB; ++b) sp[b] = warp_sum(sp[b]);
    }
    if (lane < ZB && t0 + lane < rows_here) {
      TU mine = sp[0];
#pragma unroll
      for (int b = 1; b < ZB; ++b)
        if (lane == b) mine = sp[b];
      const int64_t i = row0 + t0 + lane;
      const T ri = r[i];
      const T zi = a.U ? (T)((double)ri + (double)mine) : ri;
      z[i] = zi;
      rz += (double)ri * (double)zi;
    }
  }
  rz = block_sum(rz, red);
  double* part = a.dpart + sidx * a.npart;
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
  if (blockIdx.x == 0 && threadIdx.x == 0 && st->conv) st->done = 1;
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

// -------------------------------------------------------------- shared-U preconditioner
//
// For many systems sharing one factor, the two passes over U of Eq. (5.3)
// serve a group of MUKM systems at once (U read once per group, not once per
// system): W = U^T R for the group, w'_s = coefficient_s * W_s, and
// z_s = r_s + U w'_s with the r^T z partials.  The residual update, the
// ||r||^2 test and alpha / beta bookkeeping stay in the per-system kernels.
template <typename T>
struct MuGroup {
  static constexpr int KM = sizeof(T) == 4 ? 16 : 8;  // systems per group
};
constexpr int MU_TR = 64;    // rows per tile of the U^T R pass
constexpr int MU_LC = 256;   // columns of U per staged chunk of the z pass

// wpart[bx][l][q] = sum over this block's row tiles of U[i][l] r[s0 + q][i]
template <typename T, typename TU>
__global__ void __launch_bounds__(PC_THREADS)
mutr_kernel(PcgArgs<T, TU> a, T* __restrict__ wpart_all) {
  constexpr int KM = MuGroup<T>::KM;
  const int64_t s0 = (int64_t)blockIdx.z * KM;
  const int ks = (int)((a.nsys - s0 < KM) ? a.nsys - s0 : KM);
  T* wpart = wpart_all + (int64_t)blockIdx.z * gridDim.x * a.ell * KM;
  __shared__ __align__(16) T rs[MU_TR][KM];
  const int64_t l = (int64_t)blockIdx.y * PC_THREADS + threadIdx.x;
  T acc[KM];
#pragma unroll
  for (int q = 0; q < KM; ++q) acc[q] = T(0);
  for (int64_t r0 = (int64_t)blockIdx.x * MU_TR; r0 < a.n; r0 += (int64_t)gridDim.x * MU_TR) {
    __syncthreads();
    for (int e = threadIdx.x; e < KM * MU_TR; e += PC_THREADS) {
      const int q = e / MU_TR, r = e - q * MU_TR;
      rs[r][q] = (q < ks && r0 + r < a.n) ? a.r[(s0 + q) * a.n + r0 + r] : T(0);
    }
    __syncthreads();
    if (l < a.ell) {
      const int rows = (int)((a.n - r0 < MU_TR) ? a.n - r0 : MU_TR);
      for (int r = 0; r < rows; ++r) {
        const T u = (T)a.U[(r0 + r) * a.ell + l];
#pragma unroll
        for (int q = 0; q < KM; ++q) acc[q] = fma(u, rs[r][q], acc[q]);
      }
    }
  }
  if (l < a.ell)
#pragma unroll
    for (int q = 0; q < KM; ++q) wpart[((int64_t)blockIdx.x * a.ell + l) * KM + q] = acc[q];
}

// w'[s0 + q][l] = ((lam_ell + mu) / (lam_l + mu) - 1) sum_b wpart[b][l][q]
template <typename T, typename TU>
__global__ void mw_kernel(PcgArgs<T, TU> a, const T* __restrict__ wpart_all, int nb) {
  constexpr int KM = MuGroup<T>::KM;
  const int64_t s0 = (int64_t)blockIdx.y * KM;
  const int ks = (int)((a.nsys - s0 < KM) ? a.nsys - s0 : KM);
  const T* wpart = wpart_all + (int64_t)blockIdx.y * nb * a.ell * KM;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.ell * KM) return;
  const int64_t l = e / KM;
  const int q = (int)(e - l * KM);
  if (q >= ks) return;
  const SysState* st = a.st + s0 + q;
  if (st->done) return;
  double sum = 0.0;
  for (int b = 0; b < nb; ++b) sum += (double)wpart[((int64_t)b * a.ell + l) * KM + q];
  const double coef = st->lam_ell_mu / (a.lam[l] + st->mu) - 1.0;
  if (a.E) {
    a.wraw[(s0 + q) * a.ell + l] = (T)sum;
    a.wc[(s0 + q) * a.ell + l] = (T)(coef * sum);
  } else {
    a.w[(s0 + q) * a.ell + l] = (T)(coef * sum);
  }
}

// z[s0 + q] = r + U w'[s0 + q] (one thread per row, w' staged in chunks of
// MU_LC columns), r^T z partials into dpart[s][blockIdx.x].
template <typename T, typename TU, int VE>
__global__ void __launch_bounds__(PC_THREADS)
mz_kernel(PcgArgs<T, TU> a, int setup) {
  constexpr int KM = MuGroup<T>::KM;
  const int64_t s0 = (int64_t)blockIdx.y * KM;
  const int ks = (int)((a.nsys - s0 < KM) ? a.nsys - s0 : KM);
  __shared__ __align__(16) T ws[MU_LC][KM];
  __shared__ double red[PC_WARPS][KM];
  __shared__ int act[KM];
  if (threadIdx.x < KM)
    act[threadIdx.x] = threadIdx.x < ks && (setup || !a.st[s0 + threadIdx.x].done);
  double rzq[KM];
#pragma unroll
  for (int q = 0; q < KM; ++q) rzq[q] = 0.0;
  for (int64_t i0 = (int64_t)blockIdx.x * PC_THREADS; i0 < a.n;
       i0 += (int64_t)gridDim.x * PC_THREADS) {
    const int64_t i = i0 + threadIdx.x;
    T acc[KM];
#pragma unroll
    for (int q = 0; q < KM; ++q) acc[q] = T(0);
    for (int64_t c0 = 0; c0 < a.ell; c0 += MU_LC) {
      const int lc = (int)((a.ell - c0 < MU_LC) ? a.ell - c0 : MU_LC);
      __syncthreads();
      for (int e = threadIdx.x; e < KM * MU_LC; e += PC_THREADS) {
        const int q = e / MU_LC, c = e - q * MU_LC;
        ws[c][q] = (q < ks && c < lc) ? a.w[(s0 + q) * a.ell + c0 + c] : T(0);
      }
      __syncthreads();
      if (i < a.n) {
        const TU* urow = a.U + i * a.ell + c0;
        // VE consecutive U entries per load (16 bytes when the rows allow it)
        for (int c = 0; c < lc; c += VE) {
          const UVec<TU, VE> u = load_uvec<TU, VE>(urow + c);
#pragma unroll
          for (int k = 0; k < VE; ++k)
#pragma unroll
            for (int q = 0; q < KM; ++q) acc[q] = fma((T)u.e[k], ws[c + k][q], acc[q]);
        }
      }
    }
    if (i < a.n) {
#pragma unroll
      for (int q = 0; q < KM; ++q) {
        if (q < ks && act[q]) {
          const T ri = a.r[(s0 + q) * a.n + i];
          const T zi = (T)((double)ri + (double)acc[q]);
          a.z[(s0 + q) * a.n + i] = zi;
          rzq[q] += (double)ri * (double)zi;
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < KM; ++q) {
    const double v = warp_sum(rzq[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < ks && act[threadIdx.x]) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < PC_WARPS; ++w) t += red[w][threadIdx.x];
    a.dpart[(s0 + threadIdx.x) * a.npart + blockIdx.x] = t;
  }
}

// r^T z from the mz partials (fixed order); beta and rz as z_kernel's last block.
template <typename T, typename TU>
__global__ void __launch_bounds__(PC_THREADS)
mrz_kernel(PcgArgs<T, TU> a, int nbz, int setup) {
  const int64_t sidx = blockIdx.x;
  SysState* st = a.st + sidx;
  if (st->done && !setup) return;
  __shared__ double red[32];
  double t = 0.0;
  for (int b = threadIdx.x; b < nbz; b += PC_THREADS) t += a.dpart[sidx * a.npart + b];
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

// Corrected coefficients for an FP32 factor (U^T U = I + E): w' = c.w -
// (c.(E w) + E (c.w)) / 2, the apply through the orthonormal basis U (I+E)^{-1/2}
// to first order in E.  One warp per (coefficient i, system).
template <typename T, typename TU>
__global__ void __launch_bounds__(PC_THREADS)
wcorr_kernel(PcgArgs<T, TU> a) {
  const int64_t sidx = blockIdx.y;
  const SysState* st = a.st + sidx;
  if (st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * PC_WARPS + warp;
  if (i >= a.ell) return;
  const T* wr = a.wraw + sidx * a.ell;
  const T* wc = a.wc + sidx * a.ell;
  const float* Ei = a.E + i * a.ell;
  float s1 = 0.f, s2 = 0.f;
  for (int64_t j = lane; j < a.ell; j += 32) {
    const float e = Ei[j];
    s1 = fmaf(e, (float)wr[j], s1);
    s2 = fmaf(e, (float)wc[j], s2);
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    const double ci = st->lam_ell_mu / (a.lam[i] + st->mu) - 1.0;
    a.w[sidx * a.ell + i] = (T)((double)wc[i] - 0.5 * (ci * (double)s1 + (double)s2));
  }
}

// flag[g] = 1 when every system of group g (systems [g*gs, min((g+1)*gs, nsys)))
// is done: a product shared by the group is skipped once none of them needs it.
__global__ void group_done_kernel(const SysState* st, int64_t nsys, int gs, int* flag) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t q0 = (int64_t)g * gs;
  if (q0 >= nsys) return;
  int all = 1;
  for (int64_t q = q0; q < q0 + gs && q < nsys; ++q) all &= (st[q].done != 0);
  flag[g] = all;
}

// -------------------------------------------------------------- host driver

template <typename T, typename TU>
struct PcgBuffers {
  PcgArgs<T, TU> a;
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

// Launch geometry shared by PCG and the standalone preconditioner apply.
template <typename T, typename TU>
static void plan_geometry(PcgArgs<T, TU>& a) {
  const int64_t sms = num_sms();
  // rows per warp: enough blocks to cover the GPU twice
  int64_t rw = cdiv(a.n, 2 * sms * PC_WARPS);
  if (rw < 4) rw = 4;
  if (rw > 32 * PC_MAXRG) rw = 32 * PC_MAXRG;
  a.rows_w = rw;
  a.nblk_u = cdiv(a.n, rw * PC_WARPS);
  a.nblk_d = 2 * sms;
  a.npart = a.nblk_u > a.nblk_d ? a.nblk_u : a.nblk_d;
}

template <typename T, typename TU>
struct PcgLaunch {
  bool vec;
  size_t usm, zsm;
  dim3 g_u, g_w, g_d;
  // shared-U passes for many systems (multi): groups of MuGroup<T>::KM systems
  bool multi = false, vec_m = false;
  T* mwpart = nullptr;
  int nbu_m = 0, nbz_m = 0;
  int32_t setup(PcgArgs<T, TU>& a, int64_t nsys) {
    constexpr int VE = 16 / sizeof(TU);
    vec = a.U && (a.ell % VE == 0) && (((uintptr_t)a.U & 15u) == 0);
    const int ve = vec ? VE : 1;
    usm = (size_t)PC_WARPS * 32 * PC_CQ * ve * sizeof(TU);
    zsm = a.U ? (size_t)cdiv(a.ell, 4) * 4 * sizeof(TU) : 16;
    g_u = dim3((unsigned)a.nblk_u, (unsigned)nsys);
    g_w = dim3((unsigned)(a.U ? cdiv(a.ell, 32) : 1), (unsigned)nsys);
    g_d = dim3((unsigned)a.nblk_d, (unsigned)nsys);
    if (zsm > 48 * 1024) {
      NYS_CUDA_TRY(cudaFuncSetAttribute(z_kernel<T, TU, VE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm));
      NYS_CUDA_TRY(cudaFuncSetAttribute(z_kernel<T, TU, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm));
    }
    return NYS_OK;
  }
  // Multi-system mode: the U passes run per group of systems.  `wpart` must
  // hold multi_wpart_elems(a) values of T.
  static size_t multi_wpart_elems(const PcgArgs<T, TU>& a) {
    return (size_t)cdiv(a.nsys, MuGroup<T>::KM) * multi_nbu(a) * a.ell * MuGroup<T>::KM;
  }
  static int multi_nbu(const PcgArgs<T, TU>& a) {
    const int64_t t = cdiv(a.n, MU_TR);
    const int64_t cap = num_sms();
    return (int)(t < cap ? t : cap);
  }
  void enable_multi(const PcgArgs<T, TU>& a, T* wpart) {
    multi = true;
    mwpart = wpart;
    // 16-byte loads of U in the z pass: rows of whole vectors, aligned base
    constexpr int VE = 16 / sizeof(TU);
    vec_m = (a.ell % VE == 0) && (((uintptr_t)a.U & 15u) == 0);
    nbu_m = multi_nbu(a);
    const int64_t t = cdiv(a.n, PC_THREADS);
    nbz_m = (int)(t < a.npart ? t : a.npart);
  }
  void update(PcgArgs<T, TU>& a, int do_update, cudaStream_t s) {
    constexpr int VE = 16 / sizeof(TU);
    if (multi) {
      // x, r update and ||r||^2 per system (no U), then U^T R per group
      PcgArgs<T, TU> b = a;
      b.U = nullptr;
      update_kernel<T, TU, 1><<<g_u, PC_THREADS, usm, s>>>(b, do_update); count_launch();
      wreduce_kernel<T, TU><<<dim3(1, (unsigned)a.nsys), PC_THREADS, 0, s>>>(b, do_update);
      count_launch();
      constexpr int KM = MuGroup<T>::KM;
      const unsigned groups = (unsigned)cdiv(a.nsys, KM);
      mutr_kernel<T, TU><<<dim3((unsigned)nbu_m, (unsigned)cdiv(a.ell, PC_THREADS), groups),
                           PC_THREADS, 0, s>>>(a, mwpart);
      count_launch();
      mw_kernel<T, TU><<<dim3((unsigned)cdiv(a.ell * KM, 256), groups), 256, 0, s>>>(a, mwpart,
                                                                                    nbu_m);
      count_launch();
      if (a.E) {
        wcorr_kernel<T, TU><<<dim3((unsigned)cdiv(a.ell, PC_WARPS), (unsigned)a.nsys), PC_THREADS,
                              0, s>>>(a);
        count_launch();
      }
      return;
    }
    if (vec)
      update_kernel<T, TU, VE><<<g_u, PC_THREADS, usm, s>>>(a, do_update);
    else
      update_kernel<T, TU, 1><<<g_u, PC_THREADS, usm, s>>>(a, do_update);
    count_launch();
    wreduce_kernel<T, TU><<<g_w, PC_THREADS, 0, s>>>(a, do_update); count_launch();
    if (a.E) {
      wcorr_kernel<T, TU><<<dim3((unsigned)cdiv(a.ell, PC_WARPS), (unsigned)a.nsys), PC_THREADS,
                            0, s>>>(a);
      count_launch();
    }
  }
  void z(PcgArgs<T, TU>& a, int setup_flag, cudaStream_t s) {
    constexpr int VE = 16 / sizeof(TU);
    if (multi) {
      constexpr int KM = MuGroup<T>::KM;
      const dim3 gz((unsigned)nbz_m, (unsigned)cdiv(a.nsys, KM));
      if (vec_m)
        mz_kernel<T, TU, 16 / sizeof(TU)><<<gz, PC_THREADS, 0, s>>>(a, setup_flag);
      else
        mz_kernel<T, TU, 1><<<gz, PC_THREADS, 0, s>>>(a, setup_flag);
      count_launch();
      mrz_kernel<T, TU><<<(unsigned)a.nsys, PC_THREADS, 0, s>>>(a, nbz_m, setup_flag);
      count_launch();
      return;
    }
    if (vec)
      z_kernel<T, TU, VE><<<g_u, PC_THREADS, zsm, s>>>(a, setup_flag);
    else
      z_kernel<T, TU, 1><<<g_u, PC_THREADS, zsm, s>>>(a, setup_flag);
    count_launch();
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

// Iterations per captured graph; the host check interval (4, 8, then 16
// iterations) is a multiple of it.  Iterations past convergence or the cap
// return at once on the device `done` words, so a replay may overrun both.
constexpr int kGraphIters = 4;

// Graph mode: NYS_PCG_GRAPH=0 in the environment turns it off at start-up;
// nys_pcg_graphs() switches it at run time.
static std::atomic<int> g_pcg_graphs{-1};
static bool pcg_graphs_enabled() {
  int v = g_pcg_graphs.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("NYS_PCG_GRAPH");
    int want = (e && e[0] == '0') ? 0 : 1;
    g_pcg_graphs.compare_exchange_strong(v, want);
    v = g_pcg_graphs.load(std::memory_order_relaxed);
  }
  return v == 1;
}

// Device-side loop (a conditional WHILE node) instead of replayed chunks:
// NYS_PCG_LOOP=0 in the environment turns it off at start-up; nys_pcg_loop()
// switches it.
static std::atomic<int> g_pcg_loop{-1};
static bool pcg_loop_enabled() {
  int v = g_pcg_loop.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("NYS_PCG_LOOP");
    v = (e && e[0] == '0') ? 0 : 1;
    g_pcg_loop.store(v, std::memory_order_relaxed);
  }
  return v == 1;
}

int32_t pcg_loop(int32_t on) {
  const int32_t prev = pcg_loop_enabled() ? 1 : 0;
  if (on == 0 || on == 1) g_pcg_loop.store(on, std::memory_order_relaxed);
  return prev;
}

static std::atomic<unsigned long long> g_graph_replays{0};
unsigned long long pcg_graph_replays() { return g_graph_replays.load(std::memory_order_relaxed); }

int32_t pcg_graphs(int32_t on) {
  const int32_t prev = pcg_graphs_enabled() ? 1 : 0;
  if (on == 0 || on == 1) g_pcg_graphs.store(on, std::memory_order_relaxed);
  return prev;
}

// A CUDA graph of kGraphIters PCG iterations.  Captured on a private stream
// (the caller's may be the legacy default stream, which cannot be captured)
// and replayed on the caller's.  Kernel parameters are captured by value:
// the graph is valid while the buffers of its solve live.
struct IterGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  GraphTiming timing;
  long long launches = 0;  // kernels per replay
  ~IterGraph() {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
  }
  bool ok() const { return ge != nullptr; }
  template <typename F>
  void build(F& iteration) {
    // one capture stream per thread and device, kept for the process
    thread_local cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
      cudaGetLastError();
      return;
    }
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
      streams[dev] = nullptr;
      cudaGetLastError();
      return;
    }
    cudaStream_t cs = streams[dev];
    const unsigned long long c0 = launch_count();
    timing_capture_begin();
    int32_t st = NYS_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      for (int c = 0; c < kGraphIters && st == NYS_OK; ++c) st = iteration(cs);
      cudaGraph_t cg = nullptr;
      const cudaError_t e = cudaStreamEndCapture(cs, &cg);
      if (st == NYS_OK && e == cudaSuccess && cg) {
        g = cg;
        if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess ||
            timing_graph_nodes(g, &timing) != NYS_OK) {
          if (ge) cudaGraphExecDestroy(ge);
          ge = nullptr;
        }
      } else if (cg) {
        cudaGraphDestroy(cg);
      }
    }
    cudaGetLastError();  // a refused capture leaves no sticky error
    // the capture recorded these launches without running them
    launches = (long long)(launch_count() - c0);
    count_launches(-launches);
  }
  int32_t replay(cudaStream_t s) {
    NYS_TRY(timing_graph_rebind(ge, timing));
    NYS_CUDA_TRY(cudaGraphLaunch(ge, s));
    count_launches(launches);
    g_graph_replays.fetch_add(1, std::memory_order_relaxed);
    return NYS_OK;
  }
};

// The whole PCG loop as one CUDA graph: a conditional WHILE node whose body
// is one iteration (the product and the PCG kernels) followed by a one-block
// kernel that counts the iteration and keeps the loop going while a system
// is still running and fewer than `limit` iterations have run.  A solve is
// then a single launch with no host round trip.  Conditional bodies may hold
// kernels, memsets and copies only, so this is used when the products of the
// iteration allocate nothing and no timing events are recorded; otherwise
// IterGraph replays fixed chunks between host checks.
__global__ void loop_cond_kernel(const SysState* __restrict__ st, int64_t nsys,
                                 unsigned* __restrict__ count, unsigned limit,
                                 cudaGraphConditionalHandle h) {
  __shared__ int running;
  if (threadIdx.x == 0) running = 0;
  __syncthreads();
  int mine = 0;
  for (int64_t q = threadIdx.x; q < nsys; q += blockDim.x) mine |= (st[q].done == 0);
  if (mine) running = 1;  // benign race: every writer stores 1
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned c = *count + 1;
    *count = c;
    cudaGraphSetConditional(h, (running && c < limit) ? 1u : 0u);
  }
}

struct LoopGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  long long body_launches = 0;  // kernels per loop iteration
  ~LoopGraph() {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
  }
  bool ok() const { return ge != nullptr; }
  template <typename F>
  void build(F& iteration, const SysState* st, int64_t nsys, unsigned* count, unsigned limit) {
    thread_local cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
      cudaGetLastError();
      return;
    }
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
      streams[dev] = nullptr;
      cudaGetLastError();
      return;
    }
    cudaStream_t cs = streams[dev];
    cudaGraphConditionalHandle h;
    if (cudaGraphCreate(&g, 0) != cudaSuccess ||
        cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const unsigned long long c0 = launch_count();
    int32_t st_ok = NYS_ERR_CUDA;
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      st_ok = iteration(cs);
      loop_cond_kernel<<<1, 256, 0, cs>>>(st, nsys, count, limit, h);
      count_launch();
      cudaGraph_t out = nullptr;
      if (cudaStreamEndCapture(cs, &out) != cudaSuccess) st_ok = NYS_ERR_CUDA;
    }
    body_launches = (long long)(launch_count() - c0);
    count_launches(-body_launches);  // recorded, not run
    if (st_ok == NYS_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
    if (st_ok != NYS_OK) ge = nullptr;
    cudaGetLastError();  // a refused capture leaves no sticky error
  }
  int32_t launch(cudaStream_t s) {
    NYS_CUDA_TRY(cudaGraphLaunch(ge, s));
    g_graph_replays.fetch_add(1, std::memory_order_relaxed);
    return NYS_OK;
  }
};

// Runs Algorithm 3 on T vectors.  x (device, T, [nsys][n]) receives the
// solution; b_dev (device FP64 [nsys][n]) is the right-hand side; with
// use_x0 the incoming x is the initial guess.  Fills iterations/status.
template <typename T, typename TU>
static int32_t run_pcg(const nys_operator* op, const TU* U, const double* lam, int64_t ell,
                       double lam_ell, const float* E, const double* mus_host, int64_t nsys,
                       const double* b_dev,
                       const T* b_T, T* x, double tol, int maxit, int use_x0, double* hist,
                       int* iters_out, int* status_out, double* relres_out, cudaStream_t s,
                       bool accurate = false) {
  // accurate (FP64 vectors only): the operator products are the FP64-accurate
  // ones of the refinement residual (double-FP32 for the ridge and Gaussian
  // operators) instead of op_matvec_f64; Gaussian systems share one pass over
  // the kernel per group of up to 8
  if (accurate && !std::is_same<T, double>::value) return NYS_ERR_ARG;
  const int64_t n = op->n;
  PcgBuffers<T, TU> B;
  B.s = s;
  PcgArgs<T, TU>& a = B.a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.ell = U ? ell : 0;
  a.nsys = nsys;
  a.U = U;
  a.lam = lam;
  a.x = x;
  a.hist = hist;
  plan_geometry(a);
  const size_t vec = (size_t)nsys * n * sizeof(T);
  NYS_TRY(B.get((void**)&a.r, vec));
  NYS_TRY(B.get((void**)&a.z, vec));
  NYS_TRY(B.get((void**)&a.p, vec));
  NYS_TRY(B.get((void**)&a.v, vec));
  NYS_TRY(B.get((void**)&a.st, nsys * sizeof(SysState)));
  NYS_TRY(B.get((void**)&a.dpart, (size_t)nsys * a.npart * sizeof(double)));
  NYS_TRY(B.get((void**)&a.counters, (size_t)nsys * 4 * sizeof(unsigned)));
  NYS_TRY(B.get((void**)&B.d_mu, nsys * sizeof(double)));
  if (U) {
    NYS_TRY(B.get((void**)&a.wpart, (size_t)nsys * a.nblk_u * ell * sizeof(TU)));
    NYS_TRY(B.get((void**)&a.w, (size_t)nsys * ell * sizeof(T)));
    if (E) {
      a.E = E;
      NYS_TRY(B.get((void**)&a.wraw, (size_t)nsys * ell * sizeof(T)));
      NYS_TRY(B.get((void**)&a.wc, (size_t)nsys * ell * sizeof(T)));
    }
  }
  size_t wbytes = op_matvec_work_bytes(op, sizeof(T) == sizeof(double));
  const bool rbf_tc_batch = std::is_same<T, float>::value && !accurate && nsys > 1 &&
                            op->kind == NYS_OP_RBF && rbf_tc_supported(op->d);
  // the batched Gaussian product works in this buffer (no allocation per product)
  if (rbf_tc_batch) wbytes = std::max(wbytes, rbf_tc_work_bytes(n, nsys, 3));
  NYS_TRY(B.get(&B.op_work, wbytes));
  unsigned* loop_count;
  NYS_TRY(B.get((void**)&loop_count, sizeof(unsigned)));
  NYS_CUDA_TRY(cudaMemsetAsync(B.op_work, 0, 256, s));
  NYS_CUDA_TRY(cudaMemsetAsync(a.counters, 0, (size_t)nsys * 4 * sizeof(unsigned), s));
  NYS_CUDA_TRY(cudaMemcpyAsync(B.d_mu, mus_host, nsys * sizeof(double), cudaMemcpyHostToDevice, s));
  if (hist) {
    std::vector<double> nanbuf((size_t)nsys * (maxit + 1), std::nan(""));
    NYS_CUDA_TRY(cudaMemcpyAsync(hist, nanbuf.data(), nanbuf.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  PcgLaunch<T, TU> L;
  NYS_TRY(L.setup(a, nsys));
  if (U && nsys >= 4) {
    // many systems share U: read it once per group of systems, not per system
    T* mw;
    NYS_TRY(B.get((void**)&mw, PcgLaunch<T, TU>::multi_wpart_elems(a) * sizeof(T)));
    L.enable_multi(a, mw);
  }

  // ---- setup: state, r0, z0 = P^{-1} r0, p0 = z0, r0^T z0
  init_state_kernel<T><<<(unsigned)nsys, 256, 0, s>>>(b_T, n, a.st, B.d_mu, lam_ell, tol, maxit);
  count_launch();
  if (use_x0) {
    for (int64_t q = 0; q < nsys; ++q)
      NYS_TRY(matvec_T<T>(op, mus_host[q], x + q * n, a.v + q * n, nullptr, B.op_work, s));
  }
  init_r_kernel<T><<<L.g_d, 256, 0, s>>>(b_dev, a.v, a.r, x, n, use_x0); count_launch();
  L.update(a, 0, s);
  L.z(a, 1, s);
  p_kernel<T, TU><<<L.g_d, 256, 0, s>>>(a, 1); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());

  // ---- iterations, checked every `chunk`
  const bool batched_rbf = std::is_same<T, float>::value && nsys > 1 && op->kind == NYS_OP_RBF;
  constexpr int kAccGroup = 8;
  const bool acc_rbf = accurate && op->kind == NYS_OP_RBF;
  int* gflag = nullptr;
  if (acc_rbf) NYS_TRY(B.get((void**)&gflag, (size_t)cdiv(nsys, kAccGroup) * sizeof(int)));
  auto products = [&](cudaStream_t st) -> int32_t {
    if (accurate) {
      if (acc_rbf) {
        const int ng = (int)cdiv(nsys, kAccGroup);
        group_done_kernel<<<(unsigned)cdiv(ng, 128), 128, 0, st>>>(a.st, nsys, kAccGroup, gflag);
        count_launch();
        for (int g = 0; g < ng; ++g) {
          const int64_t q0 = (int64_t)g * kAccGroup;
          const int64_t cnt = std::min<int64_t>(kAccGroup, nsys - q0);
          NYS_TRY(rbf_residual_products(op, B.d_mu + q0, cnt, (const double*)(a.p + q0 * n),
                                        (double*)(a.v + q0 * n), st, gflag + g));
        }
        return NYS_OK;
      }
      for (int64_t q = 0; q < nsys; ++q)
        NYS_TRY(op_matvec_residual(op, mus_host[q], (const double*)(a.p + q * n),
                                   (double*)(a.v + q * n), &a.st[q].done, B.op_work, st));
      return NYS_OK;
    }
    if (batched_rbf) {
      // one pass over the kernel matrix for all systems
      return op_matvec_batched_f32(op, B.d_mu, nsys, (const float*)a.p, (float*)a.v,
                                   &a.st[0].done, (int64_t)(sizeof(SysState) / sizeof(int)),
                                   reinterpret_cast<int*>(B.op_work),
                                   rbf_tc_batch ? B.op_work : nullptr, st);
    }
    for (int64_t q = 0; q < nsys; ++q)
      NYS_TRY(matvec_T<T>(op, mus_host[q], a.p + q * n, a.v + q * n, &a.st[q].done, B.op_work,
                          st));
    return NYS_OK;
  };
  auto iteration = [&](cudaStream_t st) -> int32_t {
    NYS_TRY(products(st));
    pv_alpha_kernel<T, TU><<<L.g_d, PC_THREADS, 0, st>>>(a); count_launch();
    L.update(a, 1, st);
    L.z(a, 0, st);
    p_kernel<T, TU><<<L.g_d, 256, 0, st>>>(a, 0); count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return NYS_OK;
  };
  // The launches of kGraphIters iterations are captured once as a CUDA graph
  // and replayed between host checks (one launch instead of ~7 per
  // iteration).  Falls back to plain launches when capture is not possible.
  IterGraph graph;
  LoopGraph loop;
  // The device-side loop needs products that allocate nothing inside the
  // iteration (FP64 Gaussian products and the FP64-accurate ones do) and no
  // timing events.
  const bool alloc_free = !accurate && (op->kind != NYS_OP_RBF || std::is_same<T, float>::value);
  if (maxit > 0 && pcg_graphs_enabled()) {
    // the tuner times launch shapes on a live stream only: let it see this
    // solve's product once before the capture (v is recomputed by the first
    // iteration)
    if (!accurate && std::is_same<T, float>::value && op->kind == NYS_OP_RBF &&
        rbf_tc_tune_pending(n, op->d, batched_rbf ? nsys : 1, 3))
      NYS_TRY(products(s));
    if (alloc_free && pcg_loop_enabled() && !timing_active())
      loop.build(iteration, a.st, nsys, loop_count, (unsigned)maxit);
    if (!loop.ok()) graph.build(iteration);
  }
  std::vector<SysState> hst(nsys);
  int64_t launched = 0;
  int chunk = 4;
  if (loop.ok()) {
    // one launch runs the iterations until every system is done or maxit
    NYS_CUDA_TRY(cudaMemsetAsync(loop_count, 0, sizeof(unsigned), s));
    NYS_TRY(loop.launch(s));
    unsigned ran = 0;
    NYS_CUDA_TRY(cudaMemcpyAsync(&ran, loop_count, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaMemcpyAsync(hst.data(), a.st, nsys * sizeof(SysState), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    count_launches(loop.body_launches * (long long)ran);
    launched = ran;
  }
  while (!loop.ok()) {
    if (graph.ok()) {
      for (int c = 0; c < chunk && launched < maxit; c += kGraphIters, launched += kGraphIters)
        NYS_TRY(graph.replay(s));
    } else {
      for (int c = 0; c < chunk && launched < maxit; ++c, ++launched) NYS_TRY(iteration(s));
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
                                   f ? f->lam_ell : 0.0, f ? f->E : nullptr, mu, nsys, b, b, x, tol, maxit, use_x0,
                                   hist, it.data(), stt.data(), rel.data(), s)));
  for (int64_t q = 0; q < nsys; ++q) {
    res[q].status = stt[q];
    res[q].iterations = it[q];
    res[q].refinements = 0;
    res[q].escalated = 0;
    res[q].rel_residual = rel[q];
  }
  return NYS_OK;
}

// Reliable-update mode of single-system mixed solves: NYS_PCG_RELIABLE=0 in
// the environment turns it off at start-up; nys_pcg_reliable() switches it.
static std::atomic<int> g_pcg_reliable{-1};
static bool pcg_reliable_enabled() {
  int v = g_pcg_reliable.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("NYS_PCG_RELIABLE");
    v = (e && e[0] == '0') ? 0 : 1;
    g_pcg_reliable.store(v, std::memory_order_relaxed);
  }
  return v == 1;
}

int32_t pcg_reliable(int32_t on) {
  const int32_t prev = pcg_reliable_enabled() ? 1 : 0;
  if (on == 0 || on == 1) g_pcg_reliable.store(on, std::memory_order_relaxed);
  return prev;
}

// Reduction of the recurrence residual between two replacements.
static double reliable_delta() {
  static double d = [] {
    const char* e = getenv("NYS_PCG_RELIABLE_DELTA");
    const double v = e ? atof(e) : 0.0;
    return (v > 0.0 && v < 1.0) ? v : 1e-3;
  }();
  return d;
}

// Contraction of the true residual over one FP32 inner solve above which a
// system of the refinement loop takes FP64-accurate inner solves
// (NYS_PCG_ESCALATE in the environment overrides it).
static double escalation_ratio() {
  static double r = [] {
    const char* e = getenv("NYS_PCG_ESCALATE");
    const double v = e ? atof(e) : 0.0;
    return (v > 0.0 && v <= 1.0) ? v : 0.5;
  }();
  return r;
}

// Reopens a system after a residual replacement: its recurrence continues.
__global__ void reopen_state_kernel(SysState* st) {
  st->done = 0;
  st->conv = 0;
  st->status = NYS_OK;
}

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out,
                                  int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

// x += (double) xl; xl = 0
__global__ void fold_kernel(double* __restrict__ x, float* __restrict__ xl, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    x[e] += (double)xl[e];
    xl[e] = 0.f;
  }
}

// Mixed-precision Algorithm 3 for one system with reliable updates (residual
// replacement; van der Vorst and Ye, SIAM J. Sci. Comput. 22, 2000): one FP32
// recurrence runs on while the iterate is kept in FP64.  Each time the
// recurrence residual has fallen by `delta` since the last replacement (or
// has met the tolerance), the FP32 correction is folded into x, the true
// residual b - (A + mu I) x is formed with FP64-accurate products, and it
// replaces the recurrence residual (z and r^T z are recomputed; the search
// direction is kept while the two residuals agree to a factor of two; a
// larger gap means the FP32 products, not rounding, set it, and the
// recurrence restarts from p = z).  Unlike refinement with restarts, the
// Krylov space is not thrown away at each correction, so the FP32 solve takes
// about as many iterations as an FP64 one.  Returns *stalled = true (x holds the best
// iterate) when the true residual stops halving between replacements, so
// that the caller continues with its escalating refinement loop.
static int32_t pcg_reliable_one(const nys_operator* op, const float* U, const double* lam,
                                int64_t ell, double lam_ell, const float* E, double mu,
                                const double* b, double* x, double bn2, double tol, int maxit,
                                int use_x0, double delta, bool* exq_io, int* iters, int* updates,
                                double* rel_out, int* status_out, bool* stalled, double* hist,
                                cudaStream_t s) {
  const int64_t n = op->n;
  *stalled = false;
  PcgBuffers<float, float> B;
  B.s = s;
  PcgArgs<float, float>& a = B.a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.ell = U ? ell : 0;
  a.nsys = 1;
  a.U = U;
  a.lam = lam;
  plan_geometry(a);
  const size_t vec = (size_t)n * sizeof(float);
  NYS_TRY(B.get((void**)&a.x, vec));
  NYS_TRY(B.get((void**)&a.r, vec));
  NYS_TRY(B.get((void**)&a.z, vec));
  NYS_TRY(B.get((void**)&a.p, vec));
  NYS_TRY(B.get((void**)&a.v, vec));
  NYS_TRY(B.get((void**)&a.st, sizeof(SysState)));
  NYS_TRY(B.get((void**)&a.dpart, (size_t)a.npart * sizeof(double)));
  NYS_TRY(B.get((void**)&a.counters, 4 * sizeof(unsigned)));
  NYS_TRY(B.get((void**)&B.d_mu, sizeof(double)));
  if (U) {
    NYS_TRY(B.get((void**)&a.wpart, (size_t)a.nblk_u * ell * sizeof(float)));
    NYS_TRY(B.get((void**)&a.w, (size_t)ell * sizeof(float)));
    if (E) {
      a.E = E;
      NYS_TRY(B.get((void**)&a.wraw, (size_t)ell * sizeof(float)));
      NYS_TRY(B.get((void**)&a.wc, (size_t)ell * sizeof(float)));
    }
  }
  double *rt, *vt, *nrm;
  NYS_TRY(B.get((void**)&rt, (size_t)n * sizeof(double)));
  NYS_TRY(B.get((void**)&vt, (size_t)n * sizeof(double)));
  NYS_TRY(B.get((void**)&nrm, sizeof(double)));
  NYS_TRY(B.get(&B.op_work, op_matvec_work_bytes(op, false)));
  void* rwork = nullptr;
  NYS_TRY(B.get(&rwork, op_matvec_work_bytes(op, true)));
  NYS_CUDA_TRY(cudaMemsetAsync(B.op_work, 0, 256, s));
  NYS_CUDA_TRY(cudaMemsetAsync(rwork, 0, 256, s));
  NYS_CUDA_TRY(cudaMemsetAsync(a.counters, 0, 4 * sizeof(unsigned), s));
  NYS_CUDA_TRY(cudaMemcpyAsync(B.d_mu, &mu, sizeof(double), cudaMemcpyHostToDevice, s));
  if (hist) {
    std::vector<double> nanbuf((size_t)maxit + 1, std::nan(""));
    NYS_CUDA_TRY(cudaMemcpyAsync(hist, nanbuf.data(), nanbuf.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    a.hist = hist;
  }
  PcgLaunch<float, float> L;
  NYS_TRY(L.setup(a, 1));
  const unsigned gb = (unsigned)std::min<int64_t>(cdiv(n, 256), 1024);

  // true residual of x in FP64-accurate arithmetic; rel = ||rt|| / ||b||
  auto true_residual = [&](double* rel) -> int32_t {
    if (*exq_io) {
      if (op->kind == NYS_OP_RBF && op->d <= 64) {
        const float* pts = (const float*)op->data;
        NYS_TRY(rbf_exact_products(pts, n, op->ld, pts, n, op->ld, op->d, op->sigma, 0, 2,
                                   B.d_mu, 0.0, 1, x, vt, nullptr, s));
      } else {
        NYS_TRY(op_matvec_f64(op, mu, x, vt, nullptr, rwork, s));
      }
    } else {
      NYS_TRY(op_matvec_residual(op, mu, x, vt, nullptr, rwork, s));
    }
    sub_kernel<<<gb, 256, 0, s>>>(b, vt, rt, n); count_launch();
    sys_sumsq_kernel<<<1, 256, 0, s>>>(rt, n, nrm); count_launch();
    double h = 0.0;
    NYS_CUDA_TRY(cudaMemcpyAsync(&h, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    *rel = bn2 > 0.0 ? sqrt(h / bn2) : sqrt(h);
    return NYS_OK;
  };

  // state: thresh2 = tol^2 ||b||^2, the recurrence's own stopping test
  init_state_kernel<double><<<1, 256, 0, s>>>(b, n, a.st, B.d_mu, lam_ell, tol, maxit);
  count_launch();
  double rel = 1.0;
  if (use_x0) {
    NYS_TRY(true_residual(&rel));
  } else {
    NYS_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    NYS_CUDA_TRY(cudaMemcpyAsync(rt, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rel = bn2 > 0.0 ? 1.0 : 0.0;
  }
  *updates = 0;
  *iters = 0;
  *status_out = NYS_ERR_MAXIT;
  *rel_out = rel;
  if (rel <= tol) {
    *status_out = NYS_OK;
    return NYS_OK;
  }
  // first segment: r = fp32(rt), x_lo = 0, z = P^{-1} r, p = z
  f64_to_f32_kernel<<<gb, 256, 0, s>>>(rt, a.r, n); count_launch();
  NYS_CUDA_TRY(cudaMemsetAsync(a.x, 0, vec, s));
  L.update(a, 0, s);
  L.z(a, 1, s);
  p_kernel<float, float><<<L.g_d, 256, 0, s>>>(a, 1); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());

  auto iteration = [&](cudaStream_t st) -> int32_t {
    NYS_TRY(matvec_T<float>(op, mu, a.p, a.v, &a.st[0].done, B.op_work, st));
    pv_alpha_kernel<float, float><<<L.g_d, PC_THREADS, 0, st>>>(a); count_launch();
    L.update(a, 1, st);
    L.z(a, 0, st);
    p_kernel<float, float><<<L.g_d, 256, 0, st>>>(a, 0); count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return NYS_OK;
  };
  IterGraph graph;
  if (maxit > 0 && pcg_graphs_enabled()) {
    if (op->kind == NYS_OP_RBF && rbf_tc_tune_pending(n, op->d, 1, 3))
      NYS_TRY(matvec_T<float>(op, mu, a.p, a.v, nullptr, B.op_work, s));
    graph.build(iteration);
  }
  SysState h;
  NYS_CUDA_TRY(cudaMemcpyAsync(&h, a.st, sizeof(SysState), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  double rr_seg = h.rr;  // recurrence ||r||^2 at the start of the segment
  double rel_prev = rel;
  int stall = 0, slow = 0;
  int64_t launched = 0;
  int chunk = 4;
  while (true) {
    if (graph.ok()) {
      for (int c = 0; c < chunk && launched < maxit; c += kGraphIters, launched += kGraphIters)
        NYS_TRY(graph.replay(s));
    } else {
      for (int c = 0; c < chunk && launched < maxit; ++c, ++launched) NYS_TRY(iteration(s));
    }
    NYS_CUDA_TRY(cudaMemcpyAsync(&h, a.st, sizeof(SysState), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    *iters = h.it;
    if (h.status == NYS_ERR_BREAKDOWN) {
      // p^T A p <= 0 with FP32 products: at this shift their error can make
      // the FP32 operator indefinite; the escalating loop takes over (its
      // FP64-accurate inner solve reports a genuine breakdown)
      fold_kernel<<<gb, 256, 0, s>>>(x, a.x, n); count_launch();
      *stalled = true;
      break;
    }
    const bool end_seg = h.done || h.rr <= delta * delta * rr_seg || launched >= maxit;
    if (!end_seg) {
      if (chunk < 16) chunk *= 2;
      continue;
    }
    // fold the FP32 correction into x and replace the recurrence residual
    fold_kernel<<<gb, 256, 0, s>>>(x, a.x, n); count_launch();
    NYS_TRY(true_residual(&rel));
    *updates += 1;
    *rel_out = rel;
    if (rel <= tol) {
      *status_out = NYS_OK;
      break;
    }
    if (!std::isfinite(rel)) {
      *status_out = NYS_ERR_BREAKDOWN;
      break;
    }
    if (h.it >= maxit || launched >= maxit) {
      // budget spent above tol: the escalating loop continues (its
      // FP64-accurate inner solves have a budget of their own)
      *stalled = true;
      break;
    }
    // a segment that cut the true residual by less than 10 (the recurrence
    // promised 1/delta) twice in a row: the FP32 products' error, not the
    // recurrence, sets the pace; the escalating loop takes over
    slow = (rel > 0.1 * rel_prev) ? slow + 1 : 0;
    if (slow >= 2 && rel <= 0.5 * rel_prev) {
      *stalled = true;
      break;
    }
    if (rel > 0.5 * rel_prev) {
      // no progress since the last replacement: first take the residual in
      // native FP64 (the double-FP32 floor may sit above tol), then hand the
      // system to the escalating refinement loop
      if (!*exq_io) {
        *exq_io = true;
        NYS_TRY(true_residual(&rel));
        *rel_out = rel;
        if (rel <= tol) {
          *status_out = NYS_OK;
          break;
        }
      }
      if (++stall >= 2) {
        *stalled = true;
        break;
      }
    } else {
      stall = 0;
    }
    rel_prev = rel;
    // Keep the search direction only while the recurrence residual was a
    // faithful estimate of the true one: when they differ by more than a
    // factor of two (the FP32 products' error, not rounding, dominates), the
    // old direction is scaled for the wrong residual and the next step size
    // would be meaningless, so the recurrence restarts from p = z.
    const double rr_true = rel * rel * (bn2 > 0.0 ? bn2 : 1.0);
    const bool restart = !(rr_true <= 4.0 * h.rr);
    f64_to_f32_kernel<<<gb, 256, 0, s>>>(rt, a.r, n); count_launch();
    reopen_state_kernel<<<1, 1, 0, s>>>(a.st); count_launch();
    L.update(a, 0, s);
    L.z(a, 1, s);
    if (restart) {
      p_kernel<float, float><<<L.g_d, 256, 0, s>>>(a, 1); count_launch();
    }
    NYS_CUDA_TRY(cudaGetLastError());
    NYS_CUDA_TRY(cudaMemcpyAsync(&h, a.st, sizeof(SysState), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    rr_seg = h.rr;
    chunk = 4;
  }
  int err = 0;
  NYS_CUDA_TRY(cudaMemcpyAsync(&err, B.op_work, sizeof(int), cudaMemcpyDeviceToHost, s));
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  if (err) return NYS_ERR_TIMEOUT;
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
  const float* Edef = nullptr;  // U^T U - I of the FP32 U the inner solves use
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
  double* d_mus;
  NYS_TRY(sc.get(&d_mus, nsys));
  NYS_CUDA_TRY(cudaMemcpyAsync(d_mus, mu, nsys * sizeof(double), cudaMemcpyHostToDevice, s));
  std::vector<double> bn2(nsys), rn2(nsys);
  sys_sumsq_kernel<<<(unsigned)nsys, 256, 0, s>>>(b, n, nrm); count_launch();
  NYS_CUDA_TRY(cudaMemcpyAsync(bn2.data(), nrm, nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
  // One system: a single FP32 recurrence with reliable updates; the
  // escalating refinement loop below takes over only if that stalls.
  bool rel_exq = op->kind == NYS_OP_DENSE, rel_stalled = false;
  int rel_it = 0, rel_upd = 0;
  // (Gaussian-kernel systems keep the refinement loop: their FP32 products'
  // error, not rounding, usually sets the gap between the recurrence and the
  // true residual, and the recurrence would restart at every replacement.)
  if (nsys == 1 && maxit > 0 && op->kind != NYS_OP_RBF && pcg_reliable_enabled()) {
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    int st0 = NYS_ERR_MAXIT;
    double rel0 = 1.0;
    NYS_TRY(pcg_reliable_one(op, U, f ? f->lam : nullptr, f ? f->ell : 0, f ? f->lam_ell : 0.0,
                             Edef, mu[0], b, x, bn2[0], tol, maxit, use_x0, reliable_delta(),
                             &rel_exq, &rel_it, &rel_upd, &rel0, &st0, &rel_stalled, hist, s));
    if (!rel_stalled) {
      res[0].status = st0;
      res[0].iterations = rel_it;
      res[0].refinements = rel_upd;
      res[0].escalated = 0;
      res[0].rel_residual = rel0;
      return NYS_OK;
    }
    use_x0 = 1;  // the refinement loop continues from the stalled iterate
  }
  std::vector<int> active(nsys, 1), total_it(nsys, 0), outer(nsys, 0), stt(nsys, NYS_ERR_MAXIT);
  std::vector<double> rel(nsys, 1.0), prev(nsys, 0.0);
  // Escalation of the inner solve: with FP64-accurate residuals, a system
  // whose true residual fails to halve over one inner solve, or that has
  // spent its FP32 iteration budget, has reached what an FP32 inner solve can
  // refine (the FP32 products' error is then comparable to mu: refinement
  // contracts by about ||(A + mu I)^{-1} dA||).  Its later inner solves run on
  // FP64 vectors with the FP64-accurate products of the residual (double-FP32
  // for the ridge and Gaussian operators, error ~2^-46 relative), with a
  // budget of maxit iterations of their own.  A system whose true residual
  // then still fails to halve over two consecutive inner solves stops with
  // NYS_ERR_MAXIT.
  std::vector<int> stag(nsys, 0), acc_it(nsys, 0);
  std::vector<char> acc(nsys, 0);
  const double* U64 = nullptr;
  const float* E64 = nullptr;
  double *ra = nullptr, *dd = nullptr;
  if (rel_stalled) {
    // the reliable-update recurrence made no progress with FP64-accurate
    // residuals: FP64-accurate inner solves from the start
    total_it[0] = rel_it;
    outer[0] = rel_upd;
    acc[0] = 1;
  }
  std::vector<double> before(nsys, 0.0);
  std::vector<char> bex(nsys, 0);
  const unsigned gb = (unsigned)cdiv(n, 256) > 1024 ? 1024 : (unsigned)cdiv(n, 256);
  // The refinement residual starts in double-FP32 arithmetic (kernel and ridge
  // operators, a few units of 2^-46 relative per product).  Its floor relative
  // to ||b|| is about that times ||A|| ||x|| / ||b||, which for a nearly flat
  // kernel and a small shift can sit above tol.  So a system whose residual
  // stops halving while still above tol takes its remaining residuals in
  // native FP64 (slower on this part, exact to FP64 rounding); the others
  // keep the double-FP32 products.
  std::vector<char> exq(nsys, op->kind == NYS_OP_DENSE ? 1 : 0);
  if (rel_stalled && rel_exq) exq[0] = 1;
  const bool may_escalate = op->kind != NYS_OP_DENSE;
  // The Gaussian residual runs as one pass over the kernel for a set of
  // systems (gathered into contiguous buffers unless it is all of them).
  double *xa = nullptr, *va = nullptr, *d_musa = nullptr;
  std::vector<double> musa;
  auto residual_pass = [&](const std::vector<int64_t>& set, bool ex) -> int32_t {
    if (set.empty()) return NYS_OK;
    const int64_t na = (int64_t)set.size();
    if (op->kind == NYS_OP_RBF && op->d <= 64) {
      const double *xs = x, *ms = d_mus;
      double* vs = v;
      const bool gather = na < nsys;
      if (gather) {
        if (!xa) {
          NYS_TRY(sc.get(&xa, nsys * n));
          NYS_TRY(sc.get(&va, nsys * n));
          NYS_TRY(sc.get(&d_musa, nsys));
        }
        musa.resize(na);
        for (int64_t t = 0; t < na; ++t) {
          musa[t] = mu[set[t]];
          NYS_CUDA_TRY(cudaMemcpyAsync(xa + t * n, x + set[t] * n, n * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
        }
        NYS_CUDA_TRY(cudaMemcpyAsync(d_musa, musa.data(), na * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        xs = xa;
        ms = d_musa;
        vs = va;
      }
      const float* pts = (const float*)op->data;
      if (ex)
        NYS_TRY(rbf_exact_products(pts, n, op->ld, pts, n, op->ld, op->d, op->sigma, 0, 2, ms, 0.0,
                                   na, xs, vs, nullptr, s));
      else
        NYS_TRY(rbf_residual_products(op, ms, na, xs, vs, s));
      if (gather)
        for (int64_t t = 0; t < na; ++t)
          NYS_CUDA_TRY(cudaMemcpyAsync(v + set[t] * n, va + t * n, n * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
    } else {
      for (int64_t q : set) {
        if (ex) NYS_TRY(op_matvec_f64(op, mu[q], x + q * n, v + q * n, nullptr, work, s));
        else NYS_TRY(op_matvec_residual(op, mu[q], x + q * n, v + q * n, nullptr, work, s));
      }
    }
    return NYS_OK;
  };
  auto residual_norms = [&]() -> int32_t {
    sub_kernel<<<gb, 256, 0, s>>>(b, v, r, nsys * n); count_launch();
    sys_sumsq_kernel<<<(unsigned)nsys, 256, 0, s>>>(r, n, nrm); count_launch();
    NYS_CUDA_TRY(cudaMemcpyAsync(rn2.data(), nrm, nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
    return NYS_OK;
  };
  for (int k = 0; k <= max_refine; ++k) {
    if (k == 0 && !use_x0) {
      // x = 0: the residual is b itself, no product needed
      NYS_CUDA_TRY(cudaMemsetAsync(v, 0, nsys * n * sizeof(double), s));
    } else {
      std::vector<int64_t> set_dfl, set_ex;
      for (int64_t q = 0; q < nsys; ++q)
        if (active[q]) (exq[q] ? set_ex : set_dfl).push_back(q);
      NYS_TRY(residual_pass(set_dfl, false));
      NYS_TRY(residual_pass(set_ex, true));
    }
    NYS_TRY(residual_norms());
    std::vector<int64_t> todo;
    for (int64_t q = 0; q < nsys; ++q) {
      if (!active[q]) continue;  // its residual was not retaken
      rel[q] = bn2[q] > 0 ? sqrt(rn2[q] / bn2[q]) : sqrt(rn2[q]);
      if (rel[q] <= tol) {
        active[q] = 0;
        stt[q] = NYS_OK;
      } else if (!std::isfinite(rel[q])) {
        active[q] = 0;
        stt[q] = NYS_ERR_BREAKDOWN;
      } else {
        if (exq[q] && bex[q] && outer[q] > 0)
          stag[q] = (rel[q] > 0.5 * before[q]) ? stag[q] + 1 : 0;
        // a system whose true residual contracted by less than the escalation
        // ratio over its last FP32 inner solve (asked for a 1e-4 reduction) is
        // limited by the FP32 products: FP64-accurate inner solves from now on
        const bool slow = outer[q] >= 2 && rel[q] > escalation_ratio() * before[q];
        if (!acc[q] && ((exq[q] && stag[q] >= 1) || total_it[q] >= maxit || slow)) {
          acc[q] = 1;
          stag[q] = 0;
        }
        if (stag[q] >= 2 || (acc[q] ? acc_it[q] >= maxit : total_it[q] >= maxit)) {
          active[q] = 0;  // stagnated or budget spent: NYS_ERR_MAXIT
        } else if (k < max_refine) {
          // maxit bounds a system's inner iterations over all refinements
          todo.push_back(q);
        }
      }
    }
    if (todo.empty()) break;
    // systems whose residual stopped halving: the same iterate, its residual
    // retaken in FP64, and FP64 residuals from now on
    std::vector<int64_t> newly;
    if (may_escalate && k > 0)
      for (int64_t t : todo)
        if (!exq[t] && rel[t] > 0.5 * prev[t]) newly.push_back(t);
    for (int64_t q = 0; q < nsys; ++q) prev[q] = rel[q];
    if (!newly.empty()) {
      for (int64_t t : newly) exq[t] = 1;
      NYS_TRY(residual_pass(newly, true));
      NYS_TRY(residual_norms());
      std::vector<int64_t> keep;
      for (int64_t q : todo) {
        if (exq[q] && std::find(newly.begin(), newly.end(), q) != newly.end()) {
          rel[q] = bn2[q] > 0 ? sqrt(rn2[q] / bn2[q]) : sqrt(rn2[q]);
          prev[q] = rel[q];
          if (rel[q] <= tol) {
            active[q] = 0;
            stt[q] = NYS_OK;
            continue;
          }
        }
        keep.push_back(q);
      }
      todo.swap(keep);
      if (todo.empty()) break;
    }
    for (int64_t t : todo) {
      before[t] = rel[t];
      bex[t] = exq[t];
    }
    std::vector<int64_t> todo_acc, todo_f32;
    for (int64_t q : todo) (acc[q] ? todo_acc : todo_f32).push_back(q);
    if (!todo_acc.empty()) {
      const int64_t nb = (int64_t)todo_acc.size();
      if (!ra) {
        NYS_TRY(sc.get(&ra, nsys * n));
        NYS_TRY(sc.get(&dd, nsys * n));
        if (f) {
          if (f->u_dtype == NYS_F64) {
            U64 = (const double*)f->U;
          } else {
            double* Ud;
            NYS_TRY(sc.get(&Ud, f->n * f->ell));
            NYS_TRY(convert_f32_to_f64((const float*)f->U, Ud, f->n * f->ell, s));
            U64 = Ud;
            E64 = f->E;
          }
        }
      }
      std::vector<double> mub(nb);
      for (int64_t t = 0; t < nb; ++t) {
        mub[t] = mu[todo_acc[t]];
        NYS_CUDA_TRY(cudaMemcpyAsync(ra + t * n, r + todo_acc[t] * n, n * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
      }
      std::vector<int> it(nb), st(nb);
      std::vector<double> rr(nb);
      int budget = 1;
      for (int64_t q : todo_acc) budget = std::max(budget, maxit - acc_it[q]);
      NYS_TRY((run_pcg<double, double>(op, U64, f ? f->lam : nullptr, f ? f->ell : 0,
                                       f ? f->lam_ell : 0.0, E64, mub.data(), nb, ra, ra, dd,
                                       inner_tol, budget, 0, nullptr, it.data(), st.data(),
                                       rr.data(), s, true)));
      for (int64_t t = 0; t < nb; ++t) {
        const int64_t q = todo_acc[t];
        axpy_to_f64_kernel<double><<<gb, 256, 0, s>>>(x + q * n, dd + t * n, n); count_launch();
        acc_it[q] += it[t];
        outer[q] += 1;
        if (st[t] == NYS_ERR_BREAKDOWN) {
          active[q] = 0;
          stt[q] = NYS_ERR_BREAKDOWN;
        }
      }
      NYS_CUDA_TRY(cudaGetLastError());
    }
    todo.swap(todo_f32);
    if (todo.empty()) continue;
    // inner solves for the systems still active (batched over them)
    int64_t na = (int64_t)todo.size();
    std::vector<double> mua(na);
    for (int64_t t = 0; t < na; ++t) {
      mua[t] = mu[todo[t]];
      NYS_CUDA_TRY(cudaMemcpyAsync(v + t * n, r + todo[t] * n, n * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
    }
    NYS_TRY(convert_f64_to_f32(v, rf, na * n, s));
    std::vector<int> it(na), st(na);
    std::vector<double> rr(na);
    int budget = 1;
    for (int64_t q : todo) budget = std::max(budget, maxit - total_it[q]);
    NYS_TRY((run_pcg<float, float>(op, U, f ? f->lam : nullptr, f ? f->ell : 0,
                                   f ? f->lam_ell : 0.0, Edef, mua.data(), na, v, rf, df, inner_tol,
                                   budget, 0, (k == 0) ? hist : nullptr, it.data(), st.data(),
                                   rr.data(), s)));
    for (int64_t t = 0; t < na; ++t) {
      int64_t q = todo[t];
      axpy_to_f64_kernel<float><<<gb, 256, 0, s>>>(x + q * n, df + t * n, n); count_launch();
      total_it[q] += it[t];
      outer[q] += 1;
      // an FP32 inner solve that broke down (p^T A p <= 0 with FP32 products,
      // whose error can make the operator indefinite at a small shift): the
      // system takes FP64-accurate inner solves from now on
      if (st[t] == NYS_ERR_BREAKDOWN) acc[q] = 1;
    }
    NYS_CUDA_TRY(cudaGetLastError());
  }
  for (int64_t q = 0; q < nsys; ++q) {
    res[q].status = stt[q];
    res[q].iterations = total_it[q] + acc_it[q];
    res[q].refinements = outer[q];
    res[q].escalated = acc[q];
    res[q].rel_residual = rel[q];
  }
  return NYS_OK;
}

// -------------------------------------------------------------- P^{-1} apply

template <typename T, typename TU>
static int32_t precond_apply_impl(const nys_factor* f, const TU* U, const float* E,
                                  const double* mu, int64_t nrhs, const T* v, T* z,
                                  double lam_ell, cudaStream_t s) {
  const int64_t n = f->n, ell = f->ell;
  PcgBuffers<T, TU> B;
  B.s = s;
  PcgArgs<T, TU>& a = B.a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.ell = ell;
  a.nsys = nrhs;
  a.U = U;
  a.lam = f->lam;
  a.hist = nullptr;
  plan_geometry(a);
  a.r = const_cast<T*>(v);
  a.z = z;
  NYS_TRY(B.get((void**)&a.st, nrhs * sizeof(SysState)));
  NYS_TRY(B.get((void**)&a.dpart, (size_t)nrhs * a.npart * sizeof(double)));
  NYS_TRY(B.get((void**)&a.counters, (size_t)nrhs * 4 * sizeof(unsigned)));
  NYS_TRY(B.get((void**)&a.wpart, (size_t)nrhs * a.nblk_u * ell * sizeof(TU)));
  NYS_TRY(B.get((void**)&a.w, (size_t)nrhs * ell * sizeof(T)));
  if (E) {
    a.E = E;
    NYS_TRY(B.get((void**)&a.wraw, (size_t)nrhs * ell * sizeof(T)));
    NYS_TRY(B.get((void**)&a.wc, (size_t)nrhs * ell * sizeof(T)));
  }
  NYS_TRY(B.get((void**)&B.d_mu, nrhs * sizeof(double)));
  NYS_CUDA_TRY(cudaMemsetAsync(a.counters, 0, (size_t)nrhs * 4 * sizeof(unsigned), s));
  NYS_CUDA_TRY(cudaMemcpyAsync(B.d_mu, mu, nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  // states: tol = 0 (never "converged"), cap never reached
  init_state_kernel<T><<<(unsigned)nrhs, 256, 0, s>>>(v, n, a.st, B.d_mu, lam_ell, 0.0,
                                                       1 << 30);
  count_launch();
  PcgLaunch<T, TU> L;
  NYS_TRY(L.setup(a, nrhs));
  L.update(a, 0, s);
  L.z(a, 1, s);
  NYS_CUDA_TRY(cudaGetLastError());
  // keep the buffers alive until the kernels have run
  NYS_CUDA_TRY(cudaStreamSynchronize(s));
  return NYS_OK;
}

template <typename T>
__global__ void scale_rows_kernel(T* z, int64_t n, const double* __restrict__ scale) {
  const int64_t q = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    z[q * n + i] = (T)((double)z[q * n + i] * scale[q]);
}

// z_s = P_s^{-1} v_s with lam_ell as the top coefficient (f->lam_ell for Eq. (5.3),
// 0 for sketch-and-solve), then z_s /= mu_s when `solve`.
static int32_t apply_impl(const nys_factor* f, const double* mu, int64_t nrhs, const void* v,
                          void* z, int32_t dtype, double lam_ell, bool solve, cudaStream_t s) {
  Scratch sc(s);
  double* inv = nullptr;
  if (solve) {
    std::vector<double> h(nrhs);
    for (int64_t q = 0; q < nrhs; ++q) h[q] = 1.0 / mu[q];
    NYS_TRY(sc.get(&inv, nrhs));
    NYS_CUDA_TRY(cudaMemcpyAsync(inv, h.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  const dim3 gs((unsigned)std::min<int64_t>(cdiv(f->n, 256), 1024), (unsigned)nrhs);
  if (dtype == NYS_F64) {
    const double* U = (const double*)f->U;
    if (f->u_dtype != NYS_F64) {
      double* Ud;
      NYS_TRY(sc.get(&Ud, f->n * f->ell));
      NYS_TRY(convert_f32_to_f64((const float*)f->U, Ud, f->n * f->ell, s));
      U = Ud;
    }
    NYS_TRY((precond_apply_impl<double, double>(f, U, f->E, mu, nrhs, (const double*)v,
                                                (double*)z, lam_ell, s)));
    if (solve) {
      scale_rows_kernel<double><<<gs, 256, 0, s>>>((double*)z, f->n, inv); count_launch();
      NYS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return NYS_OK;
  }
  const float* U = (const float*)f->U;
  const float* E = f->E;
  if (f->u_dtype != NYS_F32) {
    float *Uf, *Ef;
    NYS_TRY(sc.get(&Uf, f->n * f->ell));
    NYS_TRY(sc.get(&Ef, f->ell * f->ell));
    NYS_TRY(convert_f64_to_f32((const double*)f->U, Uf, f->n * f->ell, s));
    NYS_TRY(orth_defect_f32(Uf, f->n, f->ell, Ef, s));
    U = Uf;
    E = Ef;
  }
  NYS_TRY((precond_apply_impl<float, float>(f, U, E, mu, nrhs, (const float*)v, (float*)z,
                                            lam_ell, s)));
  if (solve) {
    scale_rows_kernel<float><<<gs, 256, 0, s>>>((float*)z, f->n, inv); count_launch();
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return NYS_OK;
}

int32_t precond_apply(const nys_factor* f, const double* mu, int64_t nrhs, const void* v, void* z,
                      int32_t dtype, cudaStream_t s) {
  return apply_impl(f, mu, nrhs, v, z, dtype, f->lam_ell, false, s);
}

// Algorithm 2: x = U (Lam + mu I)^{-1} U^T b + (b - U U^T b) / mu
//             = (1/mu) [b + U (mu / (Lam + mu) - 1) U^T b],
// the Eq. (5.3) apply with lam_ell replaced by 0, scaled by 1/mu.
int32_t sketch_solve(const nys_factor* f, const double* mu, int64_t nrhs, const void* b, void* x,
                     int32_t dtype, cudaStream_t s) {
  return apply_impl(f, mu, nrhs, b, x, dtype, 0.0, true, s);
}

}  // namespace nys
