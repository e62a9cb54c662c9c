// FP64-accurate Gaussian-kernel products in double-FP32 arithmetic, for the
// refinement residual r = b - (K + mu I) x of the kernel-ridge workloads
// (Sec. 6.5).  GB300 runs FP64 at a small fraction of its FP32 rate, so each
// kernel entry is built from pairs of FP32 numbers ("double-float", Dekker
// 1971) to a few units of 2^-48 relative accuracy, with no FP64 operation in
// the inner loop:
//
//   e_ij = c ||x_i||^2 + c ||x_j||^2 - 2c x_i . x_j   (c = -1/(2 sigma^2)): the
//          inner product from exact FP32 products (one FMA each) summed with
//          TwoSum; the two norm terms rounded to double-float once per row and
//          once per point tile;
//   K_ij = exp(e_ij)                                  own double-float exp:
//          e / ln2 = k/1024 + f (|f| <= 2^-11), 2^(k/1024) = 2^(k >> 10) T[k & 1023]
//          with T[j] = 2^(j/1024) in double-float (built per block), and
//          e^(f ln2) = 1 + g + g^2/2 + g^3/6 + g^4/24 (|g| <= ln2 2^-11, truncation
//          below 4e-20) with g^2 split exactly;
//   y_q[i] = sum_j K_ij x_q[j]                        double-float accumulation.
//
// One thread per row i (two for d <= 32 with few vectors), a tile of points
// (and their norm terms) in shared memory, up to RP_Q right-hand sides per
// launch in registers.

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace nys {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl dfl_make(float h, float l) {
  dfl r;
  r.hi = h;
  r.lo = l;
  return r;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ dfl dfl_norm(float s, float e) {
  dfl r;
  r.hi = __fadd_rn(s, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
  return r;
}

__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfl_norm(p, e);
}

// acc += a * b for FP32 a, b (exact product, TwoSum accumulation, lazy lo)
__device__ __forceinline__ void dfl_acc_prod(float a, float b, float& hi, float& lo) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ dfl dfl_from_double(double x) {
  const float h = __double2float_rn(x);
  return dfl_make(h, __double2float_rn(x - (double)h));
}

// log2(e) and ln 2 as double-float constants
constexpr double kLog2e = 1.44269504088896340736, kLn2 = 0.69314718055994530942;
constexpr float kLog2eHi = (float)kLog2e, kLog2eLo = (float)(kLog2e - (double)kLog2eHi);
constexpr float kLn2Hi = (float)kLn2, kLn2Lo = (float)(kLn2 - (double)kLn2Hi);
constexpr int DFL_TAB = 1024;

// exp(e) for e <= 0 in double-float (see the file comment); tab[j] = 2^(j/1024)
// as (hi, lo).  Zero below e = -126 ln 2, where K_ij < 2^-126.
__device__ __forceinline__ dfl dfl_exp_neg(dfl e, const float2* tab) {
  // t = e / ln 2
  const float th = __fmul_rn(e.hi, kLog2eHi);
  float tl = __fmaf_rn(e.hi, kLog2eHi, -th);
  tl = __fmaf_rn(e.hi, kLog2eLo, tl);
  tl = __fmaf_rn(e.lo, kLog2eHi, tl);
  if (th < -126.f) return dfl_make(0.f, 0.f);
  // k = round(1024 th) through the 1.5 2^23 shifter (exact on |1024 th| < 2^22)
  const float kf = __fadd_rn(__fmul_rn(th, 1024.f), 12582912.f);
  const int k = __float_as_int(kf) - 0x4B400000;
  const float kr = __fsub_rn(kf, 12582912.f);
  // f = (th - k/1024) + tl: the first difference is exact; tl (~2^-24 |t|) can be
  // as large as f itself, so the sum is kept as a double-float
  float fh, fl;
  two_sum(__fmaf_rn(-kr, 0.0009765625f, th), tl, fh, fl);
  // g = f ln 2
  const float gh = __fmul_rn(fh, kLn2Hi);
  float gl = __fmaf_rn(fh, kLn2Hi, -gh);
  gl = __fmaf_rn(fh, kLn2Lo, gl);
  gl = __fmaf_rn(fl, kLn2Hi, gl);
  // e^g = 1 + gh + [gl + gh^2/2 + gh gl + gh^3/6 + gh^4/24], gh^2 = sq + sqe exactly
  const float sq = __fmul_rn(gh, gh);
  const float sqe = __fmaf_rn(gh, gh, -sq);
  const float c6 = __fmaf_rn(gh, 1.f / 24.f, 1.f / 6.f);
  float small = __fmaf_rn(__fmul_rn(sq, gh), c6, __fmul_rn(0.5f, sqe));
  small = __fmaf_rn(gh, gl, small);
  const float ph = __fadd_rn(1.f, gh);
  const float ea = __fsub_rn(gh, __fsub_rn(ph, 1.f));  // exact: |gh| < 1
  const float pl = __fadd_rn(__fadd_rn(ea, __fmul_rn(0.5f, sq)), __fadd_rn(gl, small));
  // times 2^(j/1024) (double-float table) and 2^(k >> 10) (exponent field; k >> 10 >= -126)
  const float2 T = tab[k & (DFL_TAB - 1)];
  const float vh = __fmul_rn(T.x, ph);
  float vl = __fmaf_rn(T.x, ph, -vh);
  vl = __fmaf_rn(T.x, pl, vl);
  vl = __fmaf_rn(T.y, ph, vl);
  const float sc = __int_as_float(((k >> 10) + 127) << 23);
  const dfl v = dfl_norm(vh, vl);
  return dfl_make(__fmul_rn(v.hi, sc), __fmul_rn(v.lo, sc));
}

constexpr int RR_DMAX = 64;

// ---------------------------------------------------------------- FP64-accurate variant
//
// Same products with the kernel entries and the sums in FP64, for a residual
// whose floor must sit below the double-float one (a nearly flat kernel with
// ||K|| / mu ~ 1e6) and for the FP64 PCG path.  The inner products stay in
// double-float (exact FP32 products, ~2^-48 relative); the exponential is our
// own FP64 routine: k = round(e 1024 / ln 2), r = e - k (ln2/1024) with ln2/1024
// split into a 24-bit head and a tail (so k times the head is exact), 2^(k/1024)
// = 2^(k >> 10) T[k & 1023] with T[j] = 2^(j/1024) (built per block with exp2),
// and e^r by its Taylor polynomial to degree 4 (|r| <= ln2/2048, truncation
// < 4e-20).  Error ~3 units of 2^-53 in K_ij; ~13 FP64 operations per entry.

struct Exp64Consts {
  double l_hi, l_lo, inv_l;  // ln2 / 1024 (24-bit head and tail), 1024 / ln2
};

constexpr int EXP_TAB = 1024;

// exp(e) for -700 <= e <= 0 (0 below): k = round(e 1024 / ln2), r = e - k ln2/1024
// (|r| <= ln2/2048), e^r to degree 4 (truncation < 4e-20), times 2^(j/1024) for
// j = k mod 1024 from the table, scaled by 2^(k / 1024) through the exponent
// field (the result stays a normal number on this range).
__device__ __forceinline__ double exp64_neg(double e, const double* tab, double l_hi, double l_lo,
                                            double inv_l) {
  if (e < -700.0) return 0.0;
  const double kd = rint(e * inv_l);
  double r = fma(-kd, l_hi, e);
  r = fma(-kd, l_lo, r);
  double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  const int k = (int)kd;
  const double t = tab[k & (EXP_TAB - 1)] * p;
  return __longlong_as_double(__double_as_longlong(t) + ((long long)(k >> 10) << 52));
}

// ---------------------------------------------------------------- the products kernel
//
// y[q][i] = sum_j k(t_i, x_j) v[q][j] for RP_Q vectors per block (8, or 32 for
// many vectors, so that each entry's exponential serves more of them), ROWS
// target rows per thread (two for d <= 32 with 8 vectors, so that each point
// coordinate read from shared memory serves two rows), the point tile read as
// float4 broadcasts.
// kind 0: k = K(t, x); kind 1: k = dK/dsigma = K D / sigma^3.  EXACT: k and the
// sums in FP64 (own FP64 exponential); otherwise double-float throughout.
// shift: 0 none, 1 mu0 v[q][i], 2 mus[q] v[q][i] (targets are the points).
constexpr int RP_THREADS = 128, RP_BJ = 64;

template <int DMAX, int ROWS, int RP_Q, bool EXACT>
__global__ void __launch_bounds__(RP_THREADS)
rbf_products_kernel(const float* __restrict__ tg, int64_t nt, int64_t ldt,
                    const double* __restrict__ nrm_t, const float* __restrict__ pts, int64_t n,
                    int64_t d, int64_t ld, const double* __restrict__ nrm, double neg_inv_2s2,
                    double inv_s3, int kind, int64_t nvec, int shift,
                    const double* __restrict__ mus, double mu0, const double* __restrict__ v,
                    double* __restrict__ y, const int* __restrict__ skip,
                    const __grid_constant__ Exp64Consts ec, int64_t jchunk,
                    double* __restrict__ ypart) {
  if (skip && *skip) return;
  __shared__ __align__(16) float xs[RP_BJ][DMAX];
  __shared__ double njs[EXACT ? RP_BJ : 1];
  __shared__ float2 bjs[EXACT ? 1 : RP_BJ];
  __shared__ double vjd[EXACT ? RP_Q : 1][RP_BJ];
  __shared__ float2 vjf[EXACT ? 1 : RP_Q][RP_BJ];
  __shared__ double tab[EXACT ? EXP_TAB : 1];
  __shared__ float2 tab2[EXACT ? 1 : DFL_TAB];
  // double-float running sums (dynamic shared memory, [RP_Q * ROWS][RP_THREADS],
  // one column per thread): each point tile is summed locally in registers and
  // merged here with a renormalising add, so the low word never grows past half
  // an ulp of the high word
  extern __shared__ float2 gacc_dyn[];
  auto gacc = reinterpret_cast<float2(*)[RP_THREADS]>(gacc_dyn);
  if (EXACT) {
    for (int t = threadIdx.x; t < EXP_TAB; t += blockDim.x)
      tab[EXACT ? t : 0] = exp2((double)t / (double)EXP_TAB);
  } else {
    for (int t = threadIdx.x; t < DFL_TAB; t += blockDim.x) {
      const dfl T = dfl_from_double(exp2((double)t / (double)DFL_TAB));
      tab2[EXACT ? 0 : t] = make_float2(T.hi, T.lo);
    }
  }
  // -2c = 1/sigma^2 and D / sigma^3 = e (1 / (c sigma^3)) in double-float
  const dfl c2 = dfl_from_double(-2.0 * neg_inv_2s2);
  const dfl wd = dfl_from_double(inv_s3 / neg_inv_2s2);
  const int64_t ib = (int64_t)blockIdx.x * (RP_THREADS * ROWS) + threadIdx.x;
  const int64_t q0 = (int64_t)blockIdx.y * RP_Q;
  const int nq = (int)((nvec - q0 < RP_Q) ? nvec - q0 : RP_Q);
  float xi[ROWS][DMAX];
  double ni[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int64_t i = ib + (int64_t)r * RP_THREADS;
#pragma unroll
    for (int k = 0; k < DMAX; ++k) xi[r][k] = (i < nt && k < d) ? tg[i * ldt + k] : 0.f;
    ni[r] = i < nt ? nrm_t[i] : 0.0;
  }
  double ai[ROWS];
  dfl aid[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    ai[r] = neg_inv_2s2 * ni[r];
    aid[r] = dfl_from_double(ai[r]);
  }
  double acc[EXACT ? ROWS : 1][EXACT ? RP_Q : 1];
  float ah[EXACT ? 1 : ROWS][EXACT ? 1 : RP_Q], al[EXACT ? 1 : ROWS][EXACT ? 1 : RP_Q];
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
#pragma unroll
    for (int q = 0; q < RP_Q; ++q) {
      if (EXACT) acc[EXACT ? r : 0][EXACT ? q : 0] = 0.0;
    }
  if (!EXACT) {
#pragma unroll
    for (int t = 0; t < RP_Q * ROWS; ++t)
      gacc[t][threadIdx.x] = make_float2(0.f, 0.f);
  }
  // this block's slice of the points (grid.z splits them; partial sums go to ypart)
  const int64_t jb = (int64_t)blockIdx.z * jchunk;
  const int64_t je = (n < jb + jchunk) ? n : jb + jchunk;
  for (int64_t j0 = jb; j0 < je; j0 += RP_BJ) {
    if (!EXACT) {
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int q = 0; q < RP_Q; ++q) {
          ah[EXACT ? 0 : r][EXACT ? 0 : q] = 0.f;
          al[EXACT ? 0 : r][EXACT ? 0 : q] = 0.f;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < RP_BJ * DMAX; e += RP_THREADS) {
      const int jj = e / DMAX, k = e - jj * DMAX;
      xs[jj][k] = (j0 + jj < je && k < d) ? pts[(j0 + jj) * ld + k] : 0.f;
    }
    for (int jj = threadIdx.x; jj < RP_BJ; jj += RP_THREADS) {
      const double bj = j0 + jj < je ? neg_inv_2s2 * nrm[j0 + jj] : 0.0;
      if (EXACT) {
        njs[EXACT ? jj : 0] = bj;
      } else {
        const dfl t = dfl_from_double(bj);
        bjs[EXACT ? 0 : jj] = make_float2(t.hi, t.lo);
      }
#pragma unroll
      for (int q = 0; q < RP_Q; ++q) {
        const double vv = (q < nq && j0 + jj < je) ? v[(q0 + q) * n + j0 + jj] : 0.0;
        if (EXACT) {
          vjd[EXACT ? q : 0][jj] = vv;
        } else {
          const dfl t = dfl_from_double(vv);
          vjf[EXACT ? 0 : q][jj] = make_float2(t.hi, t.lo);
        }
      }
    }
    __syncthreads();
    const int jn = (int)((je - j0 < RP_BJ) ? je - j0 : RP_BJ);
    for (int jj = 0; jj < jn; ++jj) {
      // inner products <t_i, x_j> in double-float (exact FP32 products)
      float dh[ROWS], dl[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) dh[r] = dl[r] = 0.f;
      const float4* xr = reinterpret_cast<const float4*>(xs[jj]);
#pragma unroll
      for (int k4 = 0; k4 < DMAX / 4; ++k4) {
        const float4 xj = xr[k4];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          dfl_acc_prod(xi[r][4 * k4 + 0], xj.x, dh[r], dl[r]);
          dfl_acc_prod(xi[r][4 * k4 + 1], xj.y, dh[r], dl[r]);
          dfl_acc_prod(xi[r][4 * k4 + 2], xj.z, dh[r], dl[r]);
          dfl_acc_prod(xi[r][4 * k4 + 3], xj.w, dh[r], dl[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        if (EXACT) {
          // exponent = c ||t_i||^2 + c ||x_j||^2 - 2c <t_i, x_j>, c = -1/(2 sigma^2)
          const double dot = (double)dh[r] + (double)dl[r];
          const double ex = fmin(fma(-2.0 * neg_inv_2s2, dot, ai[r] + njs[EXACT ? jj : 0]), 0.0);
          double K = exp64_neg(ex, tab, ec.l_hi, ec.l_lo, ec.inv_l);
          if (kind == 1) K *= (ex / neg_inv_2s2) * inv_s3;  // D = exponent / c
#pragma unroll
          for (int q = 0; q < RP_Q; ++q)
            if (q < nq) acc[EXACT ? r : 0][EXACT ? q : 0] =
                fma(K, vjd[EXACT ? q : 0][jj], acc[EXACT ? r : 0][EXACT ? q : 0]);
        } else {
          // e = c ||t_i||^2 + c ||x_j||^2 + (-2c) <t_i, x_j> in double-float
          const dfl dot = dfl_norm(dh[r], dl[r]);
          const float mh = __fmul_rn(dot.hi, c2.hi);
          float ml = __fmaf_rn(dot.hi, c2.hi, -mh);
          ml = __fmaf_rn(dot.hi, c2.lo, ml);
          ml = __fmaf_rn(dot.lo, c2.hi, ml);
          const float2 bj = bjs[EXACT ? 0 : jj];
          float s1, e1, s2, e2;
          two_sum(aid[r].hi, bj.x, s1, e1);
          two_sum(s1, mh, s2, e2);
          const float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(aid[r].lo, bj.y), ml));
          dfl ex = dfl_norm(s2, lo);
          if (ex.hi > 0.f) ex = dfl_make(0.f, 0.f);  // D >= 0
          dfl Kij = dfl_exp_neg(ex, tab2);
          if (kind == 1) Kij = dfl_mul(Kij, dfl_mul(ex, wd));
#pragma unroll
          for (int q = 0; q < RP_Q; ++q) {
            if (q < nq) {
              const float2 vv = vjf[EXACT ? 0 : q][jj];
              const float p = __fmul_rn(Kij.hi, vv.x);
              float e = __fmaf_rn(Kij.hi, vv.x, -p);
              e = __fmaf_rn(Kij.hi, vv.y, e);
              e = __fmaf_rn(Kij.lo, vv.x, e);
              float sum, e2;
              two_sum(ah[EXACT ? 0 : r][EXACT ? 0 : q], p, sum, e2);
              ah[EXACT ? 0 : r][EXACT ? 0 : q] = sum;
              al[EXACT ? 0 : r][EXACT ? 0 : q] =
                  __fadd_rn(al[EXACT ? 0 : r][EXACT ? 0 : q], __fadd_rn(e2, e));
            }
          }
        }
      }
    }
    if (!EXACT) {
      // merge the tile's sums: (gh, gl) + (ah, al), renormalised
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int q = 0; q < RP_Q; ++q) {
          if (q < nq) {
            float2& g = gacc[q * ROWS + r][threadIdx.x];
            float sh, se;
            two_sum(g.x, ah[EXACT ? 0 : r][EXACT ? 0 : q], sh, se);
            const float t = __fadd_rn(g.y, __fadd_rn(al[EXACT ? 0 : r][EXACT ? 0 : q], se));
            const float hi = __fadd_rn(sh, t);
            g = make_float2(hi, __fsub_rn(t, __fsub_rn(hi, sh)));
          }
        }
    }
  }
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int64_t i = ib + (int64_t)r * RP_THREADS;
    if (i >= nt) continue;
#pragma unroll
    for (int q = 0; q < RP_Q; ++q)
      if (q < nq) {
        const int64_t g = q0 + q;
        double out;
        if (EXACT) {
          out = acc[EXACT ? r : 0][EXACT ? q : 0];
        } else {
          const float2 g = gacc[q * ROWS + r][threadIdx.x];
          out = (double)g.x + (double)g.y;
        }
        if (ypart) {
          ypart[((int64_t)blockIdx.z * nvec + g) * nt + i] = out;
        } else {
          if (shift) out = fma(shift == 2 ? mus[g] : mu0, v[g * n + i], out);
          y[g * nt + i] = out;
        }
      }
  }
}

// y[g][i] = sum_z ypart[z][g][i] (fixed order) + shift
__global__ void products_sum_kernel(const double* __restrict__ ypart, int nz, int64_t nt,
                                    int64_t nvec, int shift, const double* __restrict__ mus,
                                    double mu0, const double* __restrict__ v, int64_t n,
                                    double* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nvec * nt) return;
  const int64_t g = e / nt, i = e - g * nt;
  double out = 0.0;
  for (int z = 0; z < nz; ++z) out += ypart[(int64_t)z * nvec * nt + e];
  if (shift) out = fma(shift == 2 ? mus[g] : mu0, v[g * n + i], out);
  y[e] = out;
}

static Exp64Consts exp64_consts() {
  static Exp64Consts c;
  static bool init = false;
  if (!init) {
    const long double ln2 = logl(2.0L);
    const long double L = ln2 / (long double)EXP_TAB;
    c.l_hi = (double)(float)L;
    c.l_lo = (double)(L - (long double)c.l_hi);
    c.inv_l = (double)((long double)EXP_TAB / ln2);
    init = true;
  }
  return c;
}

__global__ void sq_norms_kernel(const float* __restrict__ pts, int64_t n, int64_t d, int64_t ld,
                                double* __restrict__ nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t k = 0; k < d; ++k) {
    const double x = (double)pts[i * ld + k];
    s = fma(x, x, s);
  }
  nrm[i] = s;
}

// ---------------------------------------------------------------- symmetric products
//
// y_q = (K + mu_q I) v_q for the points against themselves with every kernel
// entry computed once.  Row tiles I and column tiles J >= I of BR points form
// the units of the grid; a unit adds K_IJ v_J to the rows of I and, for
// J > I, K_IJ^T v_I to the rows of J (column sums reduced across the warp and
// then across the block's warps in a fixed order, in double-float).  Each
// contribution (tile t, row i) has a slot of its own, part[t][q][i], and the
// final sum over t runs in a fixed order: the result is reproducible.
template <int DMAX, int ROWS, int SQ>
__global__ void __launch_bounds__(RP_THREADS)
rbf_sym_products_kernel(const float* __restrict__ pts, int64_t n, int64_t d, int64_t ld,
                        const double* __restrict__ nrm, double neg_inv_2s2, int64_t nvec,
                        const double* __restrict__ v, double* __restrict__ part, int64_t nbr,
                        const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int BR = ROWS * RP_THREADS;
  constexpr int NW = RP_THREADS / 32;
  __shared__ __align__(16) float xs[RP_BJ][DMAX];
  __shared__ float2 bjs[RP_BJ];
  __shared__ float2 vjf[SQ][RP_BJ];
  __shared__ float2 tab2[DFL_TAB];
  __shared__ float2 cacc[NW][SQ][RP_BJ];
  // unit -> (I, J >= I): units before row tile a number a nbr - a (a - 1) / 2
  const int64_t u = blockIdx.x;
  const double tb = 2.0 * (double)nbr + 1.0;
  int64_t I = (int64_t)floor((tb - sqrt(fmax(tb * tb - 8.0 * (double)u, 0.0))) * 0.5);
  if (I < 0) I = 0;
  if (I > nbr - 1) I = nbr - 1;
  while (I > 0 && I * nbr - I * (I - 1) / 2 > u) --I;
  while (I + 1 < nbr && (I + 1) * nbr - (I + 1) * I / 2 <= u) ++I;
  const int64_t J = I + (u - (I * nbr - I * (I - 1) / 2));
  const bool diag = (I == J);
  const int64_t q0 = (int64_t)blockIdx.y * SQ;
  const int nq = (int)((nvec - q0 < SQ) ? nvec - q0 : SQ);
  for (int t = threadIdx.x; t < DFL_TAB; t += blockDim.x) {
    const dfl T = dfl_from_double(exp2((double)t / (double)DFL_TAB));
    tab2[t] = make_float2(T.hi, T.lo);
  }
  const dfl c2 = dfl_from_double(-2.0 * neg_inv_2s2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the rows of tile I (with v at those rows, for the column sums)
  float xi[ROWS][DMAX];
  dfl aid[ROWS];
  float2 vi[ROWS][SQ];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int64_t i = I * BR + (int64_t)r * RP_THREADS + threadIdx.x;
    const bool ok = i < n;
#pragma unroll
    for (int k = 0; k < DMAX; ++k) xi[r][k] = (ok && k < d) ? pts[i * ld + k] : 0.f;
    aid[r] = ok ? dfl_from_double(neg_inv_2s2 * nrm[i]) : dfl_make(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < SQ; ++q) {
      const dfl t = (ok && q < nq) ? dfl_from_double(v[(q0 + q) * n + i]) : dfl_make(0.f, 0.f);
      vi[r][q] = make_float2(t.hi, t.lo);
    }
  }
  float gh[ROWS][SQ], gl[ROWS][SQ];
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
#pragma unroll
    for (int q = 0; q < SQ; ++q) gh[r][q] = gl[r][q] = 0.f;
  const int64_t jt0 = J * BR, jt1 = (n < jt0 + BR) ? n : jt0 + BR;
  for (int64_t j0 = jt0; j0 < jt1; j0 += RP_BJ) {
    float ah[ROWS][SQ], al[ROWS][SQ];
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int q = 0; q < SQ; ++q) ah[r][q] = al[r][q] = 0.f;
    __syncthreads();
    for (int e = threadIdx.x; e < RP_BJ * DMAX; e += RP_THREADS) {
      const int jj = e / DMAX, k = e - jj * DMAX;
      xs[jj][k] = (j0 + jj < jt1 && k < d) ? pts[(j0 + jj) * ld + k] : 0.f;
    }
    for (int jj = threadIdx.x; jj < RP_BJ; jj += RP_THREADS) {
      const bool ok = j0 + jj < jt1;
      const dfl t = dfl_from_double(ok ? neg_inv_2s2 * nrm[j0 + jj] : 0.0);
      bjs[jj] = make_float2(t.hi, t.lo);
#pragma unroll
      for (int q = 0; q < SQ; ++q) {
        const dfl w = dfl_from_double((ok && q < nq) ? v[(q0 + q) * n + j0 + jj] : 0.0);
        vjf[q][jj] = make_float2(w.hi, w.lo);
      }
    }
    __syncthreads();
    const int jn = (int)((jt1 - j0 < RP_BJ) ? jt1 - j0 : RP_BJ);
    for (int jj = 0; jj < jn; ++jj) {
      float dh[ROWS], dl[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) dh[r] = dl[r] = 0.f;
      const float4* xr = reinterpret_cast<const float4*>(xs[jj]);
#pragma unroll
      for (int k4 = 0; k4 < DMAX / 4; ++k4) {
        const float4 xj = xr[k4];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          dfl_acc_prod(xi[r][4 * k4 + 0], xj.x, dh[r], dl[r]);
          dfl_acc_prod(xi[r][4 * k4 + 1], xj.y, dh[r], dl[r]);
          dfl_acc_prod(xi[r][4 * k4 + 2], xj.z, dh[r], dl[r]);
          dfl_acc_prod(xi[r][4 * k4 + 3], xj.w, dh[r], dl[r]);
        }
      }
      dfl Kr[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const dfl dot = dfl_norm(dh[r], dl[r]);
        const float mh = __fmul_rn(dot.hi, c2.hi);
        float ml = __fmaf_rn(dot.hi, c2.hi, -mh);
        ml = __fmaf_rn(dot.hi, c2.lo, ml);
        ml = __fmaf_rn(dot.lo, c2.hi, ml);
        const float2 bj = bjs[jj];
        float s1, e1, s2, e2;
        two_sum(aid[r].hi, bj.x, s1, e1);
        two_sum(s1, mh, s2, e2);
        const float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(aid[r].lo, bj.y), ml));
        dfl ex = dfl_norm(s2, lo);
        if (ex.hi > 0.f) ex = dfl_make(0.f, 0.f);
        Kr[r] = dfl_exp_neg(ex, tab2);
#pragma unroll
        for (int q = 0; q < SQ; ++q) {
          const float2 vv = vjf[q][jj];
          const float p = __fmul_rn(Kr[r].hi, vv.x);
          float e = __fmaf_rn(Kr[r].hi, vv.x, -p);
          e = __fmaf_rn(Kr[r].hi, vv.y, e);
          e = __fmaf_rn(Kr[r].lo, vv.x, e);
          float sum, e3;
          two_sum(ah[r][q], p, sum, e3);
          ah[r][q] = sum;
          al[r][q] = __fadd_rn(al[r][q], __fadd_rn(e3, e));
        }
      }
      if (!diag) {
        // column sums over the block's rows of tile I: K_ij v_i, this thread's
        // rows, then a butterfly across the warp (lane 0 keeps the total)
#pragma unroll
        for (int q = 0; q < SQ; ++q) {
          float sh = 0.f, sl = 0.f;
#pragma unroll
          for (int r = 0; r < ROWS; ++r) {
            const float2 vv = vi[r][q];
            const float p = __fmul_rn(Kr[r].hi, vv.x);
            float e = __fmaf_rn(Kr[r].hi, vv.x, -p);
            e = __fmaf_rn(Kr[r].hi, vv.y, e);
            e = __fmaf_rn(Kr[r].lo, vv.x, e);
            float sum, e3;
            two_sum(sh, p, sum, e3);
            sh = sum;
            sl = __fadd_rn(sl, __fadd_rn(e3, e));
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh, off);
            const float ol = __shfl_xor_sync(0xffffffffu, sl, off);
            float sum, e3;
            two_sum(sh, oh, sum, e3);
            sh = sum;
            sl = __fadd_rn(sl, __fadd_rn(ol, e3));
          }
          if (lane == 0) cacc[warp][q][jj] = make_float2(sh, sl);
        }
      }
    }
    // merge the chunk's row sums into the running sums, renormalised
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int q = 0; q < SQ; ++q) {
        float sh, se;
        two_sum(gh[r][q], ah[r][q], sh, se);
        const float t = __fadd_rn(gl[r][q], __fadd_rn(al[r][q], se));
        const float h = __fadd_rn(sh, t);
        gl[r][q] = __fsub_rn(t, __fsub_rn(h, sh));
        gh[r][q] = h;
      }
    if (!diag) {
      __syncthreads();
      // the chunk's column sums: warps added in a fixed order; slot I of the rows of J
      for (int e = threadIdx.x; e < SQ * RP_BJ; e += RP_THREADS) {
        const int q = e / RP_BJ, jj = e - q * RP_BJ;
        if (q < nq && jj < jn) {
          float2 a = cacc[0][q][jj];
#pragma unroll
          for (int w = 1; w < NW; ++w) {
            const float2 b = cacc[w][q][jj];
            float sum, e3;
            two_sum(a.x, b.x, sum, e3);
            a = make_float2(sum, __fadd_rn(a.y, __fadd_rn(b.y, e3)));
          }
          part[(I * nvec + q0 + q) * n + j0 + jj] = (double)a.x + (double)a.y;
        }
      }
    }
  }
  // row sums: slot J of the rows of I
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int64_t i = I * BR + (int64_t)r * RP_THREADS + threadIdx.x;
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < SQ; ++q)
      if (q < nq) part[(J * nvec + q0 + q) * n + i] = (double)gh[r][q] + (double)gl[r][q];
  }
}

namespace {

template <int DMAX, int ROWS, int SQ>
int32_t sym_go(const float* pts, int64_t n, int64_t ld, int64_t d, double sigma,
               const double* d_mu, int64_t nvec, const double* v, double* y, const int* skip,
               cudaStream_t s) {
  constexpr int BR = ROWS * RP_THREADS;
  const int64_t nbr = cdiv(n, BR);
  const int64_t units = nbr * (nbr + 1) / 2;
  if (units > 0x7fffffffll) return NYS_ERR_ARG;
  Scratch sc(s);
  double *nrm, *part;
  NYS_TRY(sc.get(&nrm, n));
  NYS_TRY(sc.get(&part, (size_t)nbr * nvec * n));
  sq_norms_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(pts, n, d, ld, nrm);
  count_launch();
  const double a = -1.0 / (2.0 * sigma * sigma);
  rbf_sym_products_kernel<DMAX, ROWS, SQ>
      <<<dim3((unsigned)units, (unsigned)cdiv(nvec, SQ)), RP_THREADS, 0, s>>>(
          pts, n, d, ld, nrm, a, nvec, v, part, nbr, skip);
  count_launch();
  products_sum_kernel<<<(unsigned)cdiv(nvec * n, 256), 256, 0, s>>>(
      part, (int)nbr, n, nvec, d_mu ? 2 : 0, d_mu, 0.0, v, n, y, skip);
  count_launch();
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

}  // namespace

namespace {

template <int DMAX, int ROWS, int Q, bool EXACT>
int32_t products_go(const float* tg, int64_t nt, int64_t ldt, const double* nrm_t,
                    const float* pts, int64_t n, int64_t ldp, const double* nrm, int64_t d,
                    double a, double b, int kind, int shift, const double* d_mu, double mu0,
                    int64_t nvec, const double* v, double* y, const int* skip,
                    const Exp64Consts& ec, cudaStream_t s) {
  // split the points over grid.z until the grid has ~4 blocks per SM, each
  // slice at least 4 point tiles; partial sums are added in a fixed order
  const int64_t bx = cdiv(nt, ROWS * RP_THREADS), by = cdiv(nvec, Q);
  const int64_t target = 4 * (int64_t)num_sms();
  int64_t nz = (bx * by >= target) ? 1 : cdiv(target, bx * by);
  nz = std::min<int64_t>(nz, std::max<int64_t>(1, n / (4 * RP_BJ)));
  const int64_t jchunk = cdiv(cdiv(n, nz), RP_BJ) * RP_BJ;
  nz = cdiv(n, jchunk);
  Scratch sc(s);
  double* ypart = nullptr;
  if (nz > 1) NYS_TRY(sc.get(&ypart, (size_t)nz * nvec * nt));
  const int dyn = EXACT ? 0 : Q * ROWS * RP_THREADS * (int)sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rbf_products_kernel<DMAX, ROWS, Q, EXACT>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    attr = true;
  }
  rbf_products_kernel<DMAX, ROWS, Q, EXACT>
      <<<dim3((unsigned)bx, (unsigned)by, (unsigned)nz), RP_THREADS, dyn, s>>>(
          tg, nt, ldt, nrm_t, pts, n, d, ldp, nrm, a, b, kind, nvec, shift, d_mu, mu0, v, y, skip,
          ec, jchunk, ypart);
  count_launch();
  if (ypart) {
    products_sum_kernel<<<(unsigned)cdiv(nvec * nt, 256), 256, 0, s>>>(
        ypart, (int)nz, nt, nvec, shift, d_mu, mu0, v, n, y, skip);
    count_launch();
  }
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

template <bool EXACT>
int32_t products_launch(const float* tg, int64_t nt, int64_t ldt, const double* nrm_t,
                        const float* pts, int64_t n, int64_t ldp, const double* nrm, int64_t d,
                        double sigma, int kind, int shift, const double* d_mu, double mu0,
                        int64_t nvec, const double* v, double* y, const int* skip,
                        cudaStream_t s) {
  const double a = -1.0 / (2.0 * sigma * sigma), b = 1.0 / (sigma * sigma * sigma);
  const Exp64Consts ec = exp64_consts();
#define NYS_PRODUCTS(DM, R, Q)                                                             \
  NYS_TRY((products_go<DM, R, Q, EXACT>(tg, nt, ldt, nrm_t, pts, n, ldp, nrm, d, a, b, kind, \
                                        shift, d_mu, mu0, nvec, v, y, skip, ec, s)))
  if (nvec <= 8) {
    if (d <= 16) NYS_PRODUCTS(16, 2, 8);
    else if (d <= 32) NYS_PRODUCTS(32, 2, 8);
    else NYS_PRODUCTS(64, 1, 8);
  } else {
    if (d <= 16) NYS_PRODUCTS(16, 1, 32);
    else if (d <= 32) NYS_PRODUCTS(32, 1, 32);
    else NYS_PRODUCTS(64, 1, 32);
  }
#undef NYS_PRODUCTS
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

int32_t products(bool exact, const float* tg, int64_t nt, int64_t ldt, const float* pts,
                 int64_t n, int64_t ldp, int64_t d, double sigma, int kind, int shift,
                 const double* d_mu, double mu0, int64_t nvec, const double* v, double* y,
                 const int* skip, cudaStream_t s) {
  if (d > RR_DMAX || d < 1 || nvec < 1 || (shift == 2 && !d_mu)) return NYS_ERR_ARG;
  Scratch sc(s);
  double *nrm, *nrm_t;
  NYS_TRY(sc.get(&nrm, n));
  NYS_TRY(sc.get(&nrm_t, nt));
  sq_norms_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(pts, n, d, ldp, nrm);
  count_launch();
  sq_norms_kernel<<<(unsigned)cdiv(nt, 256), 256, 0, s>>>(tg, nt, d, ldt, nrm_t);
  count_launch();
  return exact ? products_launch<true>(tg, nt, ldt, nrm_t, pts, n, ldp, nrm, d, sigma, kind, shift,
                                       d_mu, mu0, nvec, v, y, skip, s)
               : products_launch<false>(tg, nt, ldt, nrm_t, pts, n, ldp, nrm, d, sigma, kind,
                                        shift, d_mu, mu0, nvec, v, y, skip, s);
}

}  // namespace

int32_t rbf_dfl_products(const float* tg, int64_t nt, int64_t ldt, const float* pts, int64_t n,
                         int64_t ldp, int64_t d, double sigma, int kind, const double* d_mu,
                         int64_t nvec, const double* v, double* y, cudaStream_t s) {
  return products(false, tg, nt, ldt, pts, n, ldp, d, sigma, kind, d_mu ? 2 : 0, d_mu, 0.0, nvec,
                  v, y, nullptr, s);
}

int32_t rbf_exact_products(const float* tg, int64_t nt, int64_t ldt, const float* pts, int64_t n,
                           int64_t ldp, int64_t d, double sigma, int kind, int shift,
                           const double* d_mu, double mu0, int64_t nvec, const double* v, double* y,
                           const int* skip, cudaStream_t s) {
  return products(true, tg, nt, ldt, pts, n, ldp, d, sigma, kind, shift, d_mu, mu0, nvec, v, y,
                  skip, s);
}

// y_q = (K + mu_q I) v_q for q < nvec (device FP64 arrays), FP64-accurate.
// Up to 8 vectors take the symmetric products (each entry once, for 4 or 8
// vectors at a time); more take the row-block products (32 vectors per entry).  skip (device, may be NULL): nothing is computed
// while *skip is nonzero.
int32_t rbf_residual_products(const nys_operator* op, const double* d_mu, int64_t nvec,
                              const double* v, double* y, cudaStream_t s, const int* skip) {
  if (op->kind != NYS_OP_RBF || op->d > RR_DMAX) return NYS_ERR_ARG;
  const float* pts = (const float*)op->data;
  const int64_t n = op->n, d = op->d, ld = op->ld;
  if (nvec == 1) {
    if (d <= 16) return sym_go<16, 2, 1>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
    if (d <= 32) return sym_go<32, 2, 1>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
    return sym_go<64, 1, 1>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
  }
  if (nvec <= 4) {
    if (d <= 16) return sym_go<16, 2, 4>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
    if (d <= 32) return sym_go<32, 2, 4>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
    return sym_go<64, 1, 4>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
  }
  if (nvec <= 8) {
    // each kernel entry serves 8 vectors (fewer rows per thread above d = 16
    // keep the accumulators in registers)
    if (d <= 16) return sym_go<16, 2, 8>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
    if (d <= 32) return sym_go<32, 1, 8>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
    return sym_go<64, 1, 8>(pts, n, ld, d, op->sigma, d_mu, nvec, v, y, skip, s);
  }
  return products(false, pts, n, ld, pts, n, ld, d, op->sigma, 0, d_mu ? 2 : 0, d_mu, 0.0, nvec,
                  v, y, skip, s);
}

}  // namespace nys
