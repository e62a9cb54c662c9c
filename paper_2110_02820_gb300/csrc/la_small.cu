// Small dense FP64 linear algebra on ell x ell matrices (ell <= 4096):
// Cholesky, triangular inverse and one-sided Jacobi SVD.  These carry the
// ell x ell core of Algorithm 1 (Sec. 2.2): chol(Omega^T Y_nu), the
// CholeskyQR passes of the thin QR/SVD, and the SVD of the small factor R.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so these kernels
// keep the ell x ell working set in L2/shared memory and spread each step
// over many SMs; the work is O(ell^3), tiny next to the n x ell passes.

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace nys {

// ============================================================ Cholesky (upper)

constexpr int CH_NB = 32;

// Factor the diagonal block D = M[k:k+nb, k:k+nb] in place: D = C_kk^T C_kk.
__global__ void chol_diag_kernel(double* M, int64_t ell, int64_t k, int nb, int* info) {
  if (*info != 0) return;
  __shared__ double D[CH_NB][CH_NB + 1];
  __shared__ int bad;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 32
  if (tx == 0 && ty == 0) bad = 0;
  if (ty < nb && tx < nb) D[ty][tx] = M[(k + ty) * ell + k + tx];
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tx == 0 && ty == 0) {
      double d = D[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = (int)(k + j + 1);
      } else {
        D[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    // row j right of the diagonal
    if (ty == 0 && tx > j && tx < nb) D[j][tx] = D[j][tx] / D[j][j];
    __syncthreads();
    // trailing update of the upper triangle r <= c, r, c > j
    if (ty > j && tx >= ty && tx < nb) D[ty][tx] -= D[j][ty] * D[j][tx];
    __syncthreads();
  }
  if (bad) {
    if (tx == 0 && ty == 0) atomicCAS(info, 0, bad);
    return;
  }
  if (ty < nb && tx < nb) M[(k + ty) * ell + k + tx] = (tx >= ty) ? D[ty][tx] : 0.0;
}

// Row panel: C[k:k+nb, c] = C_kk^{-T} M[k:k+nb, c] for c >= k + nb (forward
// substitution with the lower-triangular C_kk^T).  One warp per column: lane
// r holds row r; at step r lane r finishes x_r, broadcasts it, and the lanes
// below subtract its contribution.
__global__ void chol_panel_kernel(double* M, int64_t ell, int64_t k, int nb, const int* info) {
  if (*info != 0) return;
  __shared__ double Ck[CH_NB][CH_NB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int r = e / nb, c = e % nb;
    Ck[r][c] = M[(k + r) * ell + k + c];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t c = k + nb + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ell) return;
  double m = (lane < nb) ? M[(k + lane) * ell + c] : 0.0;
  for (int r = 0; r < nb; ++r) {
    double xr = (lane == r) ? m / Ck[r][r] : 0.0;
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
    chol_diag_kernel<<<1, dim3(32, 32), 0, s>>>(M, ell, k, nb, d_info); count_launch();
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

// Row j of X^T (= column j of X = C^{-1} e_j) by back substitution; one warp
// per column.  XT[j][i] = X[i][j]; entries i > j are zero.
__global__ void tri_inv_cols_kernel(const double* C, double* XT, int64_t ell) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= ell) return;
  double* x = XT + j * ell;
  for (int64_t i = lane; i < ell; i += 32) x[i] = 0.0;
  __syncwarp();
  if (lane == 0) x[j] = 1.0 / C[j * ell + j];
  __syncwarp();
  for (int64_t i = j - 1; i >= 0; --i) {
    const double* Ci = C + i * ell;
    double acc = 0.0;
    for (int64_t t = i + 1 + lane; t <= j; t += 32) acc += Ci[t] * x[t];
    acc = warp_sum(acc);
    if (lane == 0) x[i] = -acc / Ci[i];
    __syncwarp();
  }
}

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
  const int64_t j = (int64_t)blockIdx.x * TI_WARPS + wib;
  if (j >= ell) return;
  double* r = rsm + (int64_t)wib * ell;
  double* x = XT + j * ell;
  for (int64_t i = lane; i < ell; i += 32) {
    r[i] = 0.0;
    x[i] = 0.0;
  }
  __syncwarp();
  double xt = 1.0 / C[j * ell + j];
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
    xt = -r[i1] / C[i1 * ell + i1];
    if (lane == 0) x[i1] = xt;
#pragma unroll
    for (int q = 0; q < TI_PF; ++q) pf[q] = nxt[q];
    __syncwarp();
  }
}

int32_t tri_inv_upper(const double* C, double* X, int64_t ell, cudaStream_t s) {
  Scratch sc(s);
  double *XT, *CT;
  NYS_TRY(sc.get(&XT, ell * ell));
  NYS_TRY(sc.get(&CT, ell * ell));
  dim3 g((unsigned)cdiv(ell, 32), (unsigned)cdiv(ell, 32));
  transpose_kernel<<<g, dim3(32, 8), 0, s>>>(C, CT, ell, ell); count_launch();
  const size_t sh = (size_t)TI_WARPS * ell * sizeof(double);
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

// ============================================================ one-sided Jacobi SVD

// Bounded grid barrier for a cooperative launch.  Returns false (and sets
// *status = NYS_ERR_TIMEOUT) if the wait did not end within the spin limit
// or another block already failed; the caller then returns.
__device__ bool grid_barrier(unsigned int* count, unsigned int* gen, int* status) {
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

struct JacobiArgs {
  double* W;          // ell rows of length ell: row j = column j of the matrix being rotated
  double* nrm;        // [ell] squared column norms, refreshed at every sweep start
  int64_t ell;        // true size (row length)
  int64_t npad;       // number of columns incl. padding (even)
  int max_sweeps;
  unsigned int* bar;  // [2] barrier count, generation
  int* rot_count;     // [max_sweeps]
  int* status;
  int* sweeps_done;
};

// Column pairs (p, q) of round r of the circle ordering on npad players.
__device__ __forceinline__ void round_pair(int64_t npad, int64_t r, int64_t k, int64_t* p,
                                           int64_t* q) {
  auto pos = [&](int64_t i) -> int64_t {
    if (i == 0) return 0;
    return 1 + ((i - 1 + r) % (npad - 1));
  };
  *p = pos(k);
  *q = pos(npad - 1 - k);
}

// One-sided (Hestenes) Jacobi: each warp orthogonalises column pairs of a
// round; blocks of JC_WARPS warps spread the FP64 work of a round over all
// SMs.  Column norms are carried from the 2x2 rotation
// (alpha' = alpha - t gamma, beta' = beta + t gamma) and recomputed exactly
// at the start of every sweep, so a pair costs one dot product plus the
// rotation.  Whether any pair rotated is recorded once per block per sweep
// (not per rotation), which keeps same-address atomics off the round's
// critical path.
constexpr int JC_WARPS = 2;

__device__ __forceinline__ double pair_dot(const double* wp, const double* wq, int64_t ell,
                                           int lane, bool vec2) {
  double ga = 0.0;
  if (vec2) {
    const double2* p2 = reinterpret_cast<const double2*>(wp);
    const double2* q2 = reinterpret_cast<const double2*>(wq);
    for (int64_t i = lane; i < ell / 2; i += 32) {
      const double2 x = p2[i], y = q2[i];
      ga = fma(x.x, y.x, ga);
      ga = fma(x.y, y.y, ga);
    }
  } else {
    for (int64_t i = lane; i < ell; i += 32) ga = fma(wp[i], wq[i], ga);
  }
  return warp_sum(ga);
}

__global__ void __launch_bounds__(32 * JC_WARPS) jacobi_kernel(JacobiArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * JC_WARPS + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * JC_WARPS;
  const int64_t npairs = a.npad / 2;
  const bool vec2 = (a.ell % 2) == 0;
  __shared__ int blk_rot;
  // Rotate only when the cosine of the angle between the two columns exceeds
  // ell * eps: below that the computed inner product is rounding noise
  // (~eps sqrt(ell)) and further sweeps would not terminate.
  const double tol = (double)(a.ell < 8 ? 8 : a.ell) * 2.220446049250313e-16;
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) blk_rot = 0;
    for (int64_t j = warp; j < a.ell; j += nwarps) {
      const double* wj = a.W + j * a.ell;
      const double acc = pair_dot(wj, wj, a.ell, lane, vec2);
      if (lane == 0) a.nrm[j] = acc;
    }
    if (!grid_barrier(a.bar, a.bar + 1, a.status)) return;
    int rotated = 0;
    for (int64_t r = 0; r < a.npad - 1; ++r) {
      for (int64_t k = warp; k < npairs; k += nwarps) {
        int64_t p, q;
        round_pair(a.npad, r, k, &p, &q);
        if (p >= a.ell || q >= a.ell) continue;  // padding column
        double* wp = a.W + p * a.ell;
        double* wq = a.W + q * a.ell;
        const double al = a.nrm[p], be = a.nrm[q];
        const double ga = pair_dot(wp, wq, a.ell, lane, vec2);
        if (fabs(ga) > tol * sqrt(al * be) && al * be > 0.0) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t);
          const double sn = c * t;
          if (vec2) {
            double2* p2 = reinterpret_cast<double2*>(wp);
            double2* q2 = reinterpret_cast<double2*>(wq);
            for (int64_t i = lane; i < a.ell / 2; i += 32) {
              const double2 x = p2[i], y = q2[i];
              p2[i] = make_double2(c * x.x - sn * y.x, c * x.y - sn * y.y);
              q2[i] = make_double2(sn * x.x + c * y.x, sn * x.y + c * y.y);
            }
          } else {
            for (int64_t i = lane; i < a.ell; i += 32) {
              const double x = wp[i], y = wq[i];
              wp[i] = c * x - sn * y;
              wq[i] = sn * x + c * y;
            }
          }
          if (lane == 0) {
            a.nrm[p] = al - t * ga;
            a.nrm[q] = be + t * ga;
          }
          rotated = 1;
        }
      }
      if (r == a.npad - 2) {
        // last round of the sweep: publish this block's rotation flag before
        // the barrier that ends the sweep
        if (lane == 0 && rotated) blk_rot = 1;
        __syncthreads();
        if (threadIdx.x == 0 && blk_rot) atomicAdd(&a.rot_count[sweep], 1);
      }
      if (!grid_barrier(a.bar, a.bar + 1, a.status)) return;
    }
    if (a.npad - 1 == 0) {
      if (threadIdx.x == 0 && blk_rot) atomicAdd(&a.rot_count[sweep], 1);
      if (!grid_barrier(a.bar, a.bar + 1, a.status)) return;
    }
    volatile int* rc = a.rot_count;
    if (rc[sweep] == 0) {
      ++sweep;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.sweeps_done = sweep;
}

// sigma_j = ||w_j|| (one warp per column).
__global__ void col_norm_kernel(const double* W, int64_t ell, double* sigma) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= ell) return;
  const double* w = W + j * ell;
  double acc = 0.0;
  for (int64_t i = lane; i < ell; i += 32) acc = fma(w[i], w[i], acc);
  acc = warp_sum(acc);
  if (lane == 0) sigma[j] = sqrt(acc);
}

// Sort sigma descending (bitonic in shared memory, one block; ties by index).
__global__ void sort_desc_kernel(double* sigma, int* perm, int64_t ell, int64_t pow2) {
  extern __shared__ unsigned char smem_raw[];
  double* key = reinterpret_cast<double*>(smem_raw);
  int* idx = reinterpret_cast<int*>(key + pow2);
  for (int64_t j = threadIdx.x; j < pow2; j += blockDim.x) {
    key[j] = (j < ell) ? sigma[j] : -1.0;
    idx[j] = (int)j;
  }
  __syncthreads();
  for (int64_t size = 2; size <= pow2; size <<= 1) {
    for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int64_t t = threadIdx.x; t < pow2; t += blockDim.x) {
        int64_t partner = t ^ stride;
        if (partner > t) {
          bool desc = ((t & size) == 0);
          double ka = key[t], kb = key[partner];
          int ia = idx[t], ib = idx[partner];
          bool a_before_b = (ka > kb) || (ka == kb && ia < ib);
          bool swap = desc ? !a_before_b : a_before_b;
          if (swap) {
            key[t] = kb; key[partner] = ka;
            idx[t] = ib; idx[partner] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int64_t j = threadIdx.x; j < ell; j += blockDim.x) {
    sigma[j] = key[j];
    perm[j] = idx[j];
  }
}

// UtT[j][i] = w_{perm[j]}[i] / sigma_j (row j = j-th left singular vector).
__global__ void gather_scale_kernel(const double* W, const int* perm, const double* sigma,
                                    int64_t ell, double* UtT) {
  const int64_t j = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ell) return;
  const double sg = sigma[j];
  UtT[j * ell + i] = (sg > 0.0) ? W[(int64_t)perm[j] * ell + i] / sg : (i == j ? 1.0 : 0.0);
}

int32_t jacobi_svd(const double* R, double* Ut, double* sigma, int64_t ell, int* d_status,
                   int* sweeps_out, cudaStream_t s) {
  const int max_sweeps = 40;
  int64_t npad = ell + (ell & 1);
  double *W = nullptr, *UtT = nullptr, *nrm = nullptr;
  unsigned char* aux = nullptr;
  Scratch sc(s);
  NYS_TRY(sc.get(&W, ell * ell));
  NYS_TRY(sc.get(&UtT, ell * ell));
  NYS_TRY(sc.get(&nrm, ell));
  size_t aux_bytes = 2 * sizeof(unsigned) + max_sweeps * sizeof(int) + 2 * sizeof(int) + ell * sizeof(int);
  NYS_TRY(sc.get(&aux, aux_bytes));
  int* perm = reinterpret_cast<int*>(aux + 2 * sizeof(unsigned) + (max_sweeps + 2) * sizeof(int));
  // W rows = columns of R
  dim3 g((unsigned)cdiv(ell, 32), (unsigned)cdiv(ell, 32));
  transpose_kernel<<<g, dim3(32, 8), 0, s>>>(R, W, ell, ell); count_launch();
  NYS_CUDA_TRY(cudaMemsetAsync(aux, 0, aux_bytes, s));
  NYS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), s));
  JacobiArgs a;
  a.W = W;
  a.nrm = nrm;
  a.ell = ell;
  a.npad = npad;
  a.max_sweeps = max_sweeps;
  a.bar = reinterpret_cast<unsigned int*>(aux);
  a.rot_count = reinterpret_cast<int*>(aux + 2 * sizeof(unsigned));
  a.sweeps_done = a.rot_count + max_sweeps;
  a.status = d_status;
  // one warp per block, as many blocks as pairs, limited to co-resident blocks
  int per_sm = 0;
  NYS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel,
                                                             32 * JC_WARPS, 0));
  if (per_sm > 2) per_sm = 2;
  int64_t want = cdiv(npad / 2, JC_WARPS);
  int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
  int blocks = (int)(want < cap ? want : cap);
  if (blocks < 1) blocks = 1;
  void* args[] = {&a};
  NYS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)jacobi_kernel, dim3(blocks), dim3(32 * JC_WARPS),
                                           args, 0, s));
  count_launch();
  col_norm_kernel<<<(unsigned)cdiv(ell, 8), 256, 0, s>>>(W, ell, sigma); count_launch();
  int64_t pow2 = 1;
  while (pow2 < ell) pow2 <<= 1;
  size_t sh = pow2 * (sizeof(double) + sizeof(int));
  if (sh > 48 * 1024)
    NYS_CUDA_TRY(cudaFuncSetAttribute(sort_desc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sh));
  sort_desc_kernel<<<1, 1024, sh, s>>>(sigma, perm, ell, pow2); count_launch();
  gather_scale_kernel<<<dim3((unsigned)cdiv(ell, 128), (unsigned)ell), 128, 0, s>>>(W, perm, sigma,
                                                                                  ell, UtT);
  count_launch();
  // Ut (columns = left singular vectors) = UtT^T
  transpose_kernel<<<g, dim3(32, 8), 0, s>>>(UtT, Ut, ell, ell); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  if (sweeps_out) {
    NYS_CUDA_TRY(cudaMemcpyAsync(sweeps_out, a.sweeps_done, sizeof(int), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return NYS_OK;
}


}  // namespace nys
