// Thin SVD of the small ell x ell factor R of Algorithm 1 (Sec. 2.2, the
// "[V, Sigma, ~] = svd(B)" step after the CholeskyQR of B): R = Ut Sigma V^T,
// of which the core needs Ut (left singular vectors) and Sigma.
//
// GB300 runs FP64 at roughly 2 FMA per clock per SM against 128 for FP32, and
// a scalar cyclic Jacobi needs ell - 1 grid-wide steps per sweep.  So:
//
//  1. Block one-sided Jacobi in FP32.  The columns of R (scaled by a power
//     of two) are split into blocks of w; a round of the circle ordering
//     pairs the blocks, and one CTA takes a pair of blocks (2w columns of
//     length ell) into shared memory and runs a full cyclic sweep over those
//     2w columns there (one warp per column pair, __syncthreads between local
//     rounds).  A sweep over all columns then needs nb - 1 grid barriers
//     (nb = ell / w blocks) instead of ell - 1; after the first round of a
//     sweep a task only rotates the w^2 pairs across its two blocks.  Column pairs whose cosine
//     is below tol (just above the FP32 rounding level of the dot product)
//     are skipped; a sweep with no rotation ends the iteration.
//  2. The FP32 vectors X seed the iterative refinement for symmetric
//     eigenproblems of Ogita and Aishima (Japan J. Indust. Appl. Math. 35,
//     2018), applied to R R^T = Ut Sigma^2 Ut^T without forming it:
//     with G = X^T X, S = X^T R R^T X = (R^T X)^T (R^T X),
//     lambda_i = S_ii / G_ii and E_ij = (S_ij + lambda_j (I - G)_ij) /
//     (lambda_j - lambda_i) for well separated pairs, (I - G)_ij / 2
//     otherwise, X <- X (I + E).  A pair counts as separated when its gap
//     exceeds the method's threshold delta and its first-order correction
//     is below 1e-2 (the second condition is ours).  Each step squares the
//     error and costs four ell^3 products, formed in double-FP32 arithmetic
//     (gemm_dfl: ~2^-48 relative, several times faster than FP64 products on
//     GB300; the two symmetric ones by their upper triangle); two or three
//     steps take the FP32 start to that accuracy.
//     Eigenvalues closer than the separation threshold stay mixed inside
//     their (orthonormal) subspace, which leaves U Lambda U^T unchanged to
//     that threshold.

#include <cooperative_groups.h>

#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

constexpr int kMaxSweeps = 30;
constexpr int kMaxRefine = 8;
constexpr double kOaCap = 1e-2;
constexpr size_t kBjSmemMax = 200 * 1024;

struct SvdAux {
  unsigned int bar[2];  // grid barrier count, generation
  int rot[kMaxSweeps];  // per sweep: number of CTAs that rotated
  int sweeps;
  int pad;
  unsigned long long maxbits;           // max |R_ij| (bit pattern of a non-negative double)
  unsigned long long emax[kMaxRefine];   // step size per refinement step
  unsigned long long e2max[kMaxRefine];  // max E_ij^2 per refinement step
};


// Pair k of round r of the circle ordering on np players (np even): player
// 0 stays, the others rotate; np - 1 rounds meet every pair once.
__device__ __forceinline__ void circle_pair(int np, int r, int k, int* p, int* q) {
  auto pos = [&](int i) -> int { return i == 0 ? 0 : 1 + ((i - 1 + r) % (np - 1)); };
  *p = pos(k);
  *q = pos(np - 1 - k);
}

__device__ __forceinline__ double scale_of(const unsigned long long* maxbits) {
  const double mx = __longlong_as_double((long long)*maxbits);
  if (!(mx > 0.0) || !isfinite(mx)) return 1.0;
  int e;
  frexp(mx, &e);
  return ldexp(1.0, -e);  // max |R_ij| * scale in [0.5, 1)
}

__global__ void absmax_bits_kernel(const double* __restrict__ R, int64_t count,
                                   unsigned long long* out) {
  double m = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = fabs(R[e]);
    m = fmax(m, v);
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// W[j][i] = scale * R[i][j] (FP32) for i, j < ell, zero in the padding
// (npad rows of ellp floats).
__global__ void rows_f32_kernel(const double* __restrict__ R, int64_t ell, float* __restrict__ W,
                                int64_t ellp, int64_t npad, const unsigned long long* maxbits) {
  __shared__ float tile[32][33];
  const double sc = scale_of(maxbits);
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t i = i0 + k, j = j0 + threadIdx.x;
    tile[k][threadIdx.x] = (i < ell && j < ell) ? (float)(R[i * ell + j] * sc) : 0.0f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t j = j0 + k, i = i0 + threadIdx.x;
    if (j < npad && i < ellp) W[j * ellp + i] = tile[threadIdx.x][k];
  }
}

struct BJArgs {
  float* W;       // npad rows of ellp floats: row j = column j of the matrix being rotated
  int ellp;       // row length (ell rounded up to a multiple of 4, zero padded)
  int nb;         // number of column blocks (even, >= 2); npad = nb * w
  float tol;      // rotate when |cos(angle)| > tol
  unsigned int* bar;
  int* rot;       // [kMaxSweeps]
  int* sweeps;
  int* status;
};

// Hestenes rotation of the column pair (x, y): one butterfly for the three
// lane sums of x . x, y . y, x . y, and the rotation (cs, sn) that zeroes
// x . y when |cos| exceeds tol.  Returns false when the pair is already
// orthogonal to tol.
__device__ __forceinline__ bool hestenes_angle(float al, float be, float ga, float tol, float* cs,
                                               float* sn) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  // |gamma| > tol sqrt(alpha beta), without the square roots
  if (!(ga * ga > tol * tol * (al * be))) return false;
  // 2 x 2 rotation that zeroes the inner product (Hestenes):
  // zeta = (beta - alpha) / (2 gamma), t = tan of the angle.
  const float zeta = (be - al) / (2.0f * ga);
  const float az = fabsf(zeta);
  const float t = az > 1e18f ? 0.5f / zeta : copysignf(1.0f, zeta) / (az + sqrtf(1.0f + zeta * zeta));
  *cs = rsqrtf(1.0f + t * t);
  *sn = *cs * t;
  return true;
}

// Block one-sided Jacobi; blockDim = 32 * WB (one warp per local column pair).
// PR > 0: in the rounds after the first of a sweep, warp w keeps its fixed
// column (w) in registers (PR float4 per lane) for all WB local rounds, so a
// round moves only the partner column through shared memory (the shared
// memory traffic of a round, not its arithmetic, set the pace).  PR = 0:
// every column goes through shared memory.
template <int WB, int PR>
__global__ void __launch_bounds__(32 * WB) bjacobi_kernel(BJArgs a) {
  extern __shared__ float4 sm4[];  // 2 WB rows of ellp / 4 float4
  __shared__ int blk_rot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rq = a.ellp >> 2;
  const int tasks = a.nb >> 1;
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) blk_rot = 0;
    for (int r = 0; r < a.nb - 1; ++r) {
      for (int t = blockIdx.x; t < tasks; t += gridDim.x) {
        int bp, bq;
        circle_pair(a.nb, r, t, &bp, &bq);
        for (int e = threadIdx.x; e < 2 * WB * rq; e += blockDim.x) {
          const int slot = e / rq, c = e - slot * rq;
          const int64_t row = slot < WB ? (int64_t)bp * WB + slot : (int64_t)bq * WB + slot - WB;
          sm4[e] = __ldcg(reinterpret_cast<const float4*>(a.W + row * a.ellp) + c);
        }
        __syncthreads();
        bool rot = false;
        if (r == 0 || PR == 0) {
          // Round 0 of a sweep meets every pair of the two blocks (a cyclic
          // sweep over their 2 WB columns); later rounds only the WB^2 pairs
          // across the blocks (WB shifts), the pairs inside a block having had
          // their turn in round 0.  Same sweep count, ~45 % fewer local rounds.
          const int nlr = (r == 0) ? 2 * WB - 1 : WB;
          for (int lr = 0; lr < nlr; ++lr) {
            int p, q;
            if (r == 0) {
              circle_pair(2 * WB, lr, warp, &p, &q);
            } else {
              p = warp;
              q = WB + (warp + lr) % WB;
            }
            float4* P = sm4 + p * rq;
            float4* Q = sm4 + q * rq;
            float al = 0.f, be = 0.f, ga = 0.f;
            for (int c = lane; c < rq; c += 32) {
              const float4 x = P[c], y = Q[c];
              al = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, al))));
              be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
              ga = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, ga))));
            }
            float cs, sn;
            if (hestenes_angle(al, be, ga, a.tol, &cs, &sn)) {
              for (int c = lane; c < rq; c += 32) {
                const float4 x = P[c], y = Q[c];
                P[c] = make_float4(cs * x.x - sn * y.x, cs * x.y - sn * y.y, cs * x.z - sn * y.z,
                                   cs * x.w - sn * y.w);
                Q[c] = make_float4(sn * x.x + cs * y.x, sn * x.y + cs * y.y, sn * x.z + cs * y.z,
                                   sn * x.w + cs * y.w);
              }
              rot = true;
            }
            __syncthreads();
          }
        } else {
          // cross rounds: column p = warp stays in registers; the partner
          // column q is read once per round, rotated with it and written back
          float4* P = sm4 + warp * rq;
          float4 pr[PR > 0 ? PR : 1];
#pragma unroll
          for (int k = 0; k < PR; ++k) {
            const int c = lane + 32 * k;
            pr[k] = c < rq ? P[c] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
          for (int lr = 0; lr < WB; ++lr) {
            float4* Q = sm4 + (WB + (warp + lr) % WB) * rq;
            float4 qr[PR > 0 ? PR : 1];
            float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
            for (int k = 0; k < PR; ++k) {
              const int c = lane + 32 * k;
              qr[k] = c < rq ? Q[c] : make_float4(0.f, 0.f, 0.f, 0.f);
              const float4 x = pr[k], y = qr[k];
              al = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, al))));
              be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
              ga = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, ga))));
            }
            float cs, sn;
            if (hestenes_angle(al, be, ga, a.tol, &cs, &sn)) {
#pragma unroll
              for (int k = 0; k < PR; ++k) {
                const int c = lane + 32 * k;
                const float4 x = pr[k], y = qr[k];
                pr[k] = make_float4(cs * x.x - sn * y.x, cs * x.y - sn * y.y, cs * x.z - sn * y.z,
                                    cs * x.w - sn * y.w);
                if (c < rq)
                  Q[c] = make_float4(sn * x.x + cs * y.x, sn * x.y + cs * y.y, sn * x.z + cs * y.z,
                                     sn * x.w + cs * y.w);
              }
              rot = true;
            }
            __syncthreads();
          }
#pragma unroll
          for (int k = 0; k < PR; ++k) {
            const int c = lane + 32 * k;
            if (c < rq) P[c] = pr[k];
          }
          __syncthreads();
        }
        if (rot && lane == 0) blk_rot = 1;
        for (int e = threadIdx.x; e < 2 * WB * rq; e += blockDim.x) {
          const int slot = e / rq, c = e - slot * rq;
          const int64_t row = slot < WB ? (int64_t)bp * WB + slot : (int64_t)bq * WB + slot - WB;
          __stcg(reinterpret_cast<float4*>(a.W + row * a.ellp) + c, sm4[e]);
        }
        __syncthreads();
      }
      if (r == a.nb - 2) {
        // last round of the sweep: publish this block's rotation flag before
        // the barrier that ends the sweep
        __syncthreads();
        if (threadIdx.x == 0 && blk_rot) atomicAdd(&a.rot[sweep], 1);
      }
      if (!grid_barrier(a.bar, a.bar + 1, a.status)) return;
    }
    volatile int* rc = a.rot;
    if (rc[sweep] == 0) {
      ++sweep;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.sweeps = sweep;
}

// rn[j] = ||W row j|| (FP64 sum of the FP32 entries), sigma[j] = rn[j] / scale.
__global__ void row_norm_kernel(const float* __restrict__ W, int64_t ellp, int64_t ell,
                                const unsigned long long* maxbits, double* rn, double* sigma) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= ell) return;
  const float* w = W + j * ellp;
  double acc = 0.0;
  for (int64_t i = lane; i < ellp; i += 32) acc = fma((double)w[i], (double)w[i], acc);
  acc = warp_sum(acc);
  if (lane == 0) {
    rn[j] = sqrt(acc);
    sigma[j] = sqrt(acc) / scale_of(maxbits);
  }
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
        const int64_t partner = t ^ stride;
        if (partner > t) {
          const bool desc = ((t & size) == 0);
          const double ka = key[t], kb = key[partner];
          const int ia = idx[t], ib = idx[partner];
          const bool a_before_b = (ka > kb) || (ka == kb && ia < ib);
          if (desc ? !a_before_b : a_before_b) {
            key[t] = kb;
            key[partner] = ka;
            idx[t] = ib;
            idx[partner] = ia;
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

// X[i][j] = W[p][i] / rn[p], p = perm[j] (or j when perm is NULL): the
// normalised rotated columns, as the columns of the ell x ell matrix X.
__global__ void rows_to_cols_kernel(const float* __restrict__ W, int64_t ellp,
                                    const int* __restrict__ perm, const double* __restrict__ rn,
                                    double* __restrict__ X, int64_t ell) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t j = j0 + k, i = i0 + threadIdx.x;
    double v = 0.0;
    if (j < ell && i < ell) {
      const int64_t p = perm ? perm[j] : j;
      const double nr = rn[p];
      v = nr > 0.0 ? (double)W[p * ellp + i] / nr : (i == j ? 1.0 : 0.0);
    }
    tile[k][threadIdx.x] = v;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t i = i0 + k, j = j0 + threadIdx.x;
    if (i < ell && j < ell) X[i * ell + j] = tile[threadIdx.x][k];
  }
}

// lambda_i = S_ii / G_ii and the separation threshold
// delta = 2 (||S - diag(lambda)||_F + max|lambda| ||I - G||_F) (Frobenius
// norms bound the spectral norms of the method from above).  Two passes with
// a fixed summation order: per-block partials over row ranges, then one block.
constexpr int OA_ROWS = 4;  // rows per block of the partial pass

__global__ void oa_partial_kernel(const double* __restrict__ G, const double* __restrict__ S,
                                  int64_t ell, double* lam, double* part) {
  __shared__ double red[32];
  const int64_t r0 = (int64_t)blockIdx.x * OA_ROWS;
  const int64_t r1 = (r0 + OA_ROWS < ell) ? r0 + OA_ROWS : ell;
  double off = 0.0, orth = 0.0, lmax = 0.0;
  for (int64_t i = r0; i < r1; ++i) {
    const double li = S[i * ell + i] / G[i * ell + i];
    if (threadIdx.x == 0) lam[i] = li;
    lmax = fmax(lmax, fabs(li));
    for (int64_t j = threadIdx.x; j < ell; j += blockDim.x) {
      const int64_t e = i * ell + j;
      const double d = S[e] - (i == j ? li : 0.0);
      const double o = (i == j ? 1.0 : 0.0) - G[e];
      off = fma(d, d, off);
      orth = fma(o, o, orth);
    }
  }
  off = block_sum(off, red);
  orth = block_sum(orth, red);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = off;
    part[3 * blockIdx.x + 1] = orth;
    part[3 * blockIdx.x + 2] = lmax;
  }
}

__global__ void oa_final_kernel(const double* __restrict__ part, int64_t nblk, double* delta) {
  __shared__ double red[32];
  double off = 0.0, orth = 0.0, lmax = 0.0;
  for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) {
    off += part[3 * b];
    orth += part[3 * b + 1];
    lmax = fmax(lmax, part[3 * b + 2]);
  }
  off = block_sum(off, red);
  orth = block_sum(orth, red);
  lmax = warp_max(lmax);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    delta[0] = 2.0 * (sqrt(off) + m * sqrt(orth));
    delta[1] = m;
  }
}

// F = I + E of the refinement step.  emax receives the size of the step as it
// matters for R R^T = U Sigma^2 U^T: max over pairs of the orthogonality defect
// |(I - G)_ij| and of |E_ij| |lambda_j - lambda_i| / max|lambda| (a rotation
// between nearly equal eigenvalues changes U Sigma^2 U^T by that much only);
// e2max receives max E_ij^2, the orthogonality defect the step itself leaves.
__global__ void oa_update_kernel(const double* __restrict__ G, const double* __restrict__ S,
                                 const double* __restrict__ lam, const double* __restrict__ delta,
                                 int64_t ell, double* __restrict__ F, unsigned long long* emax,
                                 unsigned long long* e2max) {
  const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t i = (int64_t)blockIdx.y * 8 + threadIdx.y;
  double ae = 0.0, e2 = 0.0;
  if (i < ell && j < ell) {
    const int64_t e = i * ell + j;
    const double rij = (i == j ? 1.0 : 0.0) - G[e];
    double eij = 0.5 * rij;
    ae = fabs(rij);
    if (i != j) {
      const double d = lam[j] - lam[i];
      if (fabs(d) > delta[0]) {
        // first-order correction, kept only while it is small: a pair barely
        // above the threshold would otherwise get a large step that costs
        // orthogonality in the next one
        const double lin = (S[e] + lam[j] * rij) / d;
        if (fabs(lin) <= kOaCap) eij = lin;
      }
      const double lm = delta[1] > 0.0 ? delta[1] : 1.0;
      ae = fmax(ae, fabs(eij) * fabs(d) / lm);
    }
    e2 = eij * eij;  // the orthogonality defect the step itself leaves
    F[e] = (i == j ? 1.0 : 0.0) + eij;
    if (ae != ae) ae = __longlong_as_double(0x7ff0000000000000ll);  // NaN -> +inf
    if (e2 != e2) e2 = __longlong_as_double(0x7ff0000000000000ll);
  }
  ae = warp_max(ae);
  e2 = warp_max(e2);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(emax, (unsigned long long)__double_as_longlong(ae));
    atomicMax(e2max, (unsigned long long)__double_as_longlong(e2));
  }
}

__global__ void sig_from_eig_kernel(const double* lam, int64_t ell, double* sigma) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ell) sigma[i] = sqrt(fmax(lam[i], 0.0));
}

// Ut[i][j] = X[i][perm[j]]
__global__ void permute_cols_kernel(const double* __restrict__ X, const int* __restrict__ perm,
                                    int64_t ell, double* __restrict__ Ut) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ell * ell;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ell, j = e - i * ell;
    Ut[e] = X[i * ell + perm[j]];
  }
}

template <int WB, int PR>
int32_t launch_bjacobi(BJArgs& a, size_t smem, cudaStream_t s) {
  auto kern = bjacobi_kernel<WB, PR>;
  NYS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  NYS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WB, smem));
  if (per_sm < 1) return NYS_ERR_ARG;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  const int64_t tasks = a.nb / 2;
  const int blocks = (int)(tasks < cap ? tasks : cap);
  void* args[] = {&a};
  NYS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(blocks), dim3(32 * WB), args, smem, s));
  count_launch();
  return NYS_OK;
}

int32_t sort_sigma(double* sigma, int* perm, int64_t ell, cudaStream_t s) {
  int64_t pow2 = 1;
  while (pow2 < ell) pow2 <<= 1;
  const size_t sh = pow2 * (sizeof(double) + sizeof(int));
  if (sh > 48 * 1024)
    NYS_CUDA_TRY(cudaFuncSetAttribute(sort_desc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sh));
  sort_desc_kernel<<<1, 1024, sh, s>>>(sigma, perm, ell, pow2); count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

}  // namespace

int32_t jacobi_svd(const double* R, double* Ut, double* sigma, int64_t ell, bool refine,
                   int* d_status, int* sweeps_out, int* refine_out, cudaStream_t s) {
  if (ell < 1 || ell > 4096) return NYS_ERR_ARG;
  const int64_t ellp = (ell + 3) & ~(int64_t)3;
  int wb = 16;
  while (wb > 2 && (size_t)(2 * wb) * ellp * sizeof(float) > kBjSmemMax) wb >>= 1;
  const size_t smem = (size_t)(2 * wb) * ellp * sizeof(float);
  if (smem > kBjSmemMax) return NYS_ERR_ARG;
  int64_t nb = cdiv(ell, wb);
  if (nb < 2) nb = 2;
  if (nb & 1) ++nb;
  const int64_t npad = nb * wb;

  Scratch sc(s);
  float* Wm;
  double* rn;
  int* perm;
  SvdAux* aux;
  NYS_TRY(sc.get(&Wm, npad * ellp));
  NYS_TRY(sc.get(&rn, ell));
  NYS_TRY(sc.get(&perm, ell));
  NYS_TRY(sc.get(&aux, 1));
  NYS_CUDA_TRY(cudaMemsetAsync(aux, 0, sizeof(SvdAux), s));
  NYS_CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), s));

  const int64_t cnt = ell * ell;
  unsigned gmax = (unsigned)(cdiv(cnt, 256) < 1024 ? cdiv(cnt, 256) : 1024);
  absmax_bits_kernel<<<gmax, 256, 0, s>>>(R, cnt, &aux->maxbits); count_launch();
  rows_f32_kernel<<<dim3((unsigned)cdiv(ellp, 32), (unsigned)cdiv(npad, 32)), dim3(32, 8), 0, s>>>(
      R, ell, Wm, ellp, npad, &aux->maxbits);
  count_launch();

  BJArgs a;
  a.W = Wm;
  a.ellp = (int)ellp;
  a.nb = (int)nb;
  // Worst-case FP32 rounding of a computed cosine is about (ellp/32 + 5)
  // units of 2^-24 for this summation order; tol sits above it so that the
  // last sweep sees no rotation, and low enough that the columns come out
  // orthogonal to ~1e-5 or better.
  const double ru = 5.960464477539063e-08;
  double tol = 2.0 * ru * (double)(ellp / 32 + 8);
  if (tol < 32.0 * ru) tol = 32.0 * ru;
  a.tol = (float)tol;
  a.bar = aux->bar;
  a.rot = aux->rot;
  a.sweeps = &aux->sweeps;
  a.status = d_status;
  // columns of up to 512 (4 float4 per lane) or 1024 (8) entries stay in
  // registers during the cross rounds
  const int64_t pr = cdiv(ellp / 4, 32);
  if (wb == 16 && pr <= 4) {
    NYS_TRY((launch_bjacobi<16, 4>(a, smem, s)));
  } else if (wb == 16 && pr <= 8) {
    NYS_TRY((launch_bjacobi<16, 8>(a, smem, s)));
  } else {
    switch (wb) {
      case 16: NYS_TRY((launch_bjacobi<16, 0>(a, smem, s))); break;
      case 8: NYS_TRY((launch_bjacobi<8, 0>(a, smem, s))); break;
      case 4: NYS_TRY((launch_bjacobi<4, 0>(a, smem, s))); break;
      default: NYS_TRY((launch_bjacobi<2, 0>(a, smem, s))); break;
    }
  }
  row_norm_kernel<<<(unsigned)cdiv(ell, 8), 256, 0, s>>>(Wm, ellp, ell, &aux->maxbits, rn, sigma);
  count_launch();
  const dim3 tg((unsigned)cdiv(ell, 32), (unsigned)cdiv(ell, 32));
  int steps = 0;
  if (!refine) {
    NYS_TRY(sort_sigma(sigma, perm, ell, s));
    rows_to_cols_kernel<<<tg, dim3(32, 8), 0, s>>>(Wm, ellp, perm, rn, Ut, ell); count_launch();
  } else {
    double *X, *Xn, *G, *T, *S, *F, *lam, *delta;
    NYS_TRY(sc.get(&X, cnt));
    NYS_TRY(sc.get(&Xn, cnt));
    NYS_TRY(sc.get(&G, cnt));
    NYS_TRY(sc.get(&T, cnt));
    NYS_TRY(sc.get(&S, cnt));
    NYS_TRY(sc.get(&F, cnt));
    NYS_TRY(sc.get(&lam, ell));
    NYS_TRY(sc.get(&delta, 2));
    const int64_t oa_blocks = cdiv(ell, OA_ROWS);
    double* part;
    NYS_TRY(sc.get(&part, 3 * oa_blocks));
    rows_to_cols_kernel<<<tg, dim3(32, 8), 0, s>>>(Wm, ellp, nullptr, rn, X, ell); count_launch();
    const dim3 ug((unsigned)cdiv(ell, 32), (unsigned)cdiv(ell, 8));
    double em_prev = 1.0;
    for (int k = 0; k < kMaxRefine; ++k) {
      NYS_TRY(gemm_dfl(true, ell, ell, ell, X, ell, X, ell, G, ell, true, s));   // G = X^T X
      NYS_TRY(gemm_dfl(true, ell, ell, ell, R, ell, X, ell, T, ell, false, s));  // T = R^T X
      NYS_TRY(gemm_dfl(true, ell, ell, ell, T, ell, T, ell, S, ell, true, s));   // S = T^T T
      oa_partial_kernel<<<(unsigned)oa_blocks, 256, 0, s>>>(G, S, ell, lam, part); count_launch();
      oa_final_kernel<<<1, 256, 0, s>>>(part, oa_blocks, delta); count_launch();
      oa_update_kernel<<<ug, dim3(32, 8), 0, s>>>(G, S, lam, delta, ell, F, &aux->emax[k],
                                                  &aux->e2max[k]);
      count_launch();
      NYS_TRY(gemm_dfl(false, ell, ell, ell, X, ell, F, ell, Xn, ell, false, s));  // X <- X (I + E)
      double* tmp = X;
      X = Xn;
      Xn = tmp;
      ++steps;
      unsigned long long eb[2] = {0, 0};
      NYS_CUDA_TRY(cudaMemcpyAsync(&eb[0], &aux->emax[k], sizeof(eb[0]), cudaMemcpyDeviceToHost, s));
      NYS_CUDA_TRY(cudaMemcpyAsync(&eb[1], &aux->e2max[k], sizeof(eb[1]), cudaMemcpyDeviceToHost, s));
      NYS_CUDA_TRY(cudaStreamSynchronize(s));
      double em, e2;
      memcpy(&em, &eb[0], sizeof(em));
      memcpy(&e2, &eb[1], sizeof(e2));
      if (!std::isfinite(em) || !std::isfinite(e2)) return NYS_ERR_BREAKDOWN;  // non-finite R
      // The step converges quadratically; once its size (relative to
      // max|lambda|) is below 1e-8 the error it leaves is at the FP64
      // rounding level of U Sigma^2 U^T.  A small step that no longer halves
      // has reached the rounding floor, and further steps change nothing.
      // A step that was itself large (E^2 above 1e-12) is always followed by
      // another, which restores the orthogonality it cost.
      if ((em < 1e-8 || (em < 1e-6 && em > 0.5 * em_prev)) && e2 < 1e-12) break;
      em_prev = em;
    }
    sig_from_eig_kernel<<<(unsigned)cdiv(ell, 256), 256, 0, s>>>(lam, ell, sigma); count_launch();
    NYS_TRY(sort_sigma(sigma, perm, ell, s));
    const unsigned pg = (unsigned)(cdiv(cnt, 256) < 4096 ? cdiv(cnt, 256) : 4096);
    permute_cols_kernel<<<pg, 256, 0, s>>>(X, perm, ell, Ut); count_launch();
  }
  NYS_CUDA_TRY(cudaGetLastError());
  if (sweeps_out) {
    NYS_CUDA_TRY(cudaMemcpyAsync(sweeps_out, &aux->sweeps, sizeof(int), cudaMemcpyDeviceToHost, s));
    NYS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (refine_out) *refine_out = steps;
  return NYS_OK;
}

}  // namespace nys
