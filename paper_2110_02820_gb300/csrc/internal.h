// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/nyspcg.h"

struct nys_factor {
  int64_t n = 0, ell = 0;
  int32_t precision = NYS_PREC_F64;
  int32_t u_dtype = NYS_F64;  // NYS_F64 (double U) or NYS_F32 (float U)
  void* U = nullptr;          // n x ell row-major
  double* lam = nullptr;      // ell, descending
  double nu = 0.0;
  double lam_ell = 0.0;       // host copy of lam[ell-1]
  int32_t escalations = 0;
  int32_t svd_sweeps = 0;
  int32_t svd_refine = 0;
  float* E = nullptr;         // FP32 U only: U^T U - I (ell x ell), for the corrected P^{-1}
  int device = 0;
};

namespace nys {

// Kernel launches made by this library since the process started.
unsigned long long launch_count();
// Adds k (may be negative) to the launch count: a graph replay adds the
// launches it holds; a capture takes back the launches it only recorded.
void count_launches(long long k);
// Launch-shape autotuner (tune.cu).  tune_pick() returns in *choice the
// fastest of `cands` for `key` (cached per process and in the JSON file named
// by NYS_TUNE_CACHE); run(c) must launch the work with candidate c on `s`.
// With tuning off or `s` capturing, an uncached key gets `fallback`.
bool tune_enabled();
int32_t tune_switch(int32_t on);
bool tune_cached(const std::string& key, int* choice);
int32_t tune_pick(const std::string& key, const std::vector<int>& cands, int fallback,
                  const std::function<int32_t(int)>& run, cudaStream_t s, int* choice);
int64_t tune_dump(char* buf, int64_t cap);
void tune_clear();
int32_t tune_set(const char* key, int32_t choice);
unsigned long long tune_timed();

// PCG graph mode switch behind nys_pcg_graphs (pcg.cu).
int32_t pcg_graphs(int32_t on);
// Reliable-update mode of single-system mixed solves behind nys_pcg_reliable (pcg.cu).
int32_t pcg_reliable(int32_t on);
// Device-side PCG loop switch behind nys_pcg_loop (pcg.cu).
int32_t pcg_loop(int32_t on);
unsigned long long pcg_graph_replays();

// ---------------------------------------------------------------- workspace

// Stream-ordered device allocation (cudaMallocAsync from the device's
// default pool, whose release threshold is raised once so that repeated
// solves reuse memory instead of returning it to the driver).
int32_t dmalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

// RAII list of stream-ordered allocations freed at scope exit.
struct Scratch {
  cudaStream_t s;
  void* ptrs[64];
  int count = 0;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (int i = 0; i < count; ++i) dfree(ptrs[i], s);
  }
  template <typename T>
  int32_t get(T** p, size_t elems) {
    void* q = nullptr;
    int32_t st = dmalloc(&q, elems * sizeof(T) + 256, s);
    if (st != NYS_OK) return st;
    ptrs[count++] = q;
    *p = reinterpret_cast<T*>(q);
    return NYS_OK;
  }
};

// ---------------------------------------------------------------- dense ell x ell FP64 (la_small.cu)

// In-place upper Cholesky M = C^T C of a symmetric ell x ell matrix (upper
// triangle read); on return the strict lower triangle is zero.  *d_info
// (device int) is 0 on success, k+1 if the k-th pivot was not positive.
int32_t chol_upper(double* M, int64_t ell, int* d_info, cudaStream_t s);
// X = C^{-1} for upper-triangular C (ell x ell); X upper triangular.
int32_t tri_inv_upper(const double* C, double* X, int64_t ell, cudaStream_t s);
// The same inverse in double-FP32 arithmetic (~2^-48 relative; for the
// mixed-precision path, whose products with C^{-1} run in FP32).
int32_t tri_inv_upper_dfl(const double* C, double* X, int64_t ell, cudaStream_t s);
// Blocked Cholesky as chol_upper in double-FP32 arithmetic (mixed path).
int32_t chol_upper_dfl(double* M, int64_t ell, int* d_info, cudaStream_t s);
// M = (M + M^T) / 2.
int32_t symmetrize(double* M, int64_t ell, cudaStream_t s);
// M += shift * I (shift read from device scalar times factor).
int32_t add_diag(double* M, int64_t ell, double shift, cudaStream_t s);
// Thin SVD of the ell x ell matrix R (svd_small.cu): R = Ut Sigma V^T.
// Writes Ut (ell x ell row-major, columns = left singular vectors, sorted so
// that sigma is descending) and sigma (ell).  FP32 block Jacobi; with
// `refine`, FP64 eigen-refinement of R R^T to FP64 accuracy.  *d_status = 0
// ok, NYS_ERR_TIMEOUT if a grid barrier wait expired.  *sweeps_out /
// *refine_out (host, may be NULL): Jacobi sweeps and refinement steps.
int32_t jacobi_svd(const double* R, double* Ut, double* sigma, int64_t ell, bool refine,
                   int* d_status, int* sweeps_out, int* refine_out, cudaStream_t s);

// ---------------------------------------------------------------- BLAS-like (blas.cu)

// C (M x N, FP64 out) = op(A)^T... generic SIMT GEMM:
//   C = opA(A) * B,  opA(A) is M x K.  trans_a=false: A is M x K row-major
//   (lda); trans_a=true: A is K x M row-major (lda).  B is K x N row-major.
// T = element type (float/double); accumulation in T; the result is written
// as TOut (float/double) with leading dimension ldc.
int32_t gemm_f32(bool trans_a, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                 const float* B, int64_t ldb, float* C, int64_t ldc, cudaStream_t s);
int32_t gemm_f32_out64(bool trans_a, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                       const float* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s);
int32_t gemm_f64(bool trans_a, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double* C, int64_t ldc, cudaStream_t s);

// D = sum over z of P[z] (M x N each), fixed order.
// C = opA(A) B for FP64 matrices in double-FP32 arithmetic (~2^-48 relative
// to sum |a||b|); sym: C symmetric, only the upper tiles computed and mirrored.
int32_t gemm_dfl(bool trans_a, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double* C, int64_t ldc, bool sym, cudaStream_t s);
int32_t split_reduce_f32(const float* P, int64_t splits, int64_t M, int64_t N, float* D,
                         int64_t ldd, cudaStream_t s);
// out (cols x rows, row stride rows) = transpose of in (rows x cols, row stride ld_in).
int32_t transpose_f32(const float* in, int64_t rows, int64_t cols, int64_t ld_in, float* out,
                      cudaStream_t s);
// TF32 tensor-core GEMM D[M x N] = A[M x K] B[N x K]^T (tc_gemm.cu); *err
// (device) receives NYS_ERR_TIMEOUT if a bounded wait expired.  Returns
// NYS_ERR_ARG when the shapes or alignment are not supported.
bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                       const float* B, int64_t ldb);
int32_t tc_gemm_tn_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                       const float* B, int64_t ldb, float* D, int64_t ldd, int* err,
                       cudaStream_t s);
// y += x (elementwise)
int32_t add_inplace_f64(double* y, const double* x, int64_t count, cudaStream_t s);
int32_t convert_f64_to_f32(const double* in, float* out, int64_t count, cudaStream_t s);
// E = U^T U - I for an FP32 n x ell U, in double-FP32 arithmetic (orth.cu).
int32_t orth_defect_f32(const float* U, int64_t n, int64_t ell, float* E, cudaStream_t s);
int32_t convert_f32_to_f64(const float* in, double* out, int64_t count, cudaStream_t s);
// sum of squares of `count` values, written to d_out (FP64 accumulate, fixed order)
int32_t sumsq_f32(const float* x, int64_t count, double* d_out, cudaStream_t s);
int32_t sumsq_f64(const double* x, int64_t count, double* d_out, cudaStream_t s);
// Y_nu = Y + nu * Q where nu = d_nu[0] * factor
int32_t shift_add_f32(const float* Y, const float* Q, float* Ynu, int64_t count, const double* d_nu,
                      double factor, cudaStream_t s);
int32_t shift_add_f64(const double* Y, const double* Q, double* Ynu, int64_t count,
                      const double* d_nu, double factor, cudaStream_t s);
// Philox4x32-10 + Box-Muller N(0,1) draws; element e of the stream (seed, stream_id)
int32_t philox_gaussian_f64(double* out, int64_t count, uint64_t seed, uint64_t stream_id,
                            cudaStream_t s);
int32_t philox_stream(uint32_t* words, double* gauss, int64_t first, int64_t count, uint64_t seed,
                      uint64_t stream_id, cudaStream_t s);
int32_t philox_blocks(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out,
                      cudaStream_t s);
// nu = 2^(floor(log2(scale * sqrt(d_sumsq[0]))) - mantissa_bits), written to d_nu
int32_t compute_nu(const double* d_sumsq, double scale, int mantissa_bits, double* d_nu,
                   cudaStream_t s);
// Ut columns scaled: lam = max(0, sigma^2 - nu)
int32_t lambda_from_sigma(const double* sigma, const double* d_nu, double* lam, int64_t ell,
                          cudaStream_t s);

// ---------------------------------------------------------------- operators (operators.cu)

// V = A Q for an n x ell block (sketch).  Q, V: n x ell row-major, FP64 when
// f64 else FP32.
int32_t op_sketch(const nys_operator* op, bool f64, const void* Q, void* V, int64_t ell,
                  cudaStream_t s);

// Column sampling: Q = I[:, cols] and Y = A Q = A[:, cols] (n x ell, FP64 when
// f64 else FP32); cols device [ell], distinct indices in [0, n).
int32_t op_columns(const nys_operator* op, bool f64, const int64_t* cols, int64_t ell, void* Q,
                   void* Y, cudaStream_t s);

// Bytes of device workspace op_matvec_* needs (its first 256 bytes hold a
// device error word that must start at zero).
size_t op_matvec_work_bytes(const nys_operator* op, bool accurate);
// v = (A + mu I) p in FP32 arithmetic (inner PCG of the mixed path; dense:
// FP64 arithmetic on FP32 vectors).  `skip` (device int, may be NULL): when
// nonzero every kernel returns at once (a converged solve).  `work` may be
// NULL (allocated per call).
int32_t op_matvec_f32(const nys_operator* op, double mu, const float* p, float* v, const int* skip,
                      void* work, cudaStream_t s);
// Opt-in event timing of op_matvec_f32 (operators.cu).
int32_t timing_start(int32_t max_products);
// Event timing of products launched inside a stream capture (operators.cu):
// timing_capture_begin() before the capture, timing_graph_nodes() on the
// captured graph, timing_graph_rebind() before every replay of its
// executable.  A graph captured with timing off carries no timing nodes.
struct GraphTiming {
  std::vector<cudaGraphNode_t> nodes;
  std::vector<int> index;               // placeholder index of each node
  std::vector<cudaEvent_t> placeholders;
  int products = 0;
};
void timing_capture_begin();
// True while nys_timing_start's event timing is on.
bool timing_active();
int32_t timing_graph_nodes(cudaGraph_t g, GraphTiming* gt);
int32_t timing_graph_rebind(cudaGraphExec_t ge, const GraphTiming& gt);
int32_t timing_stop(double* total_ms, int64_t* products);
// v = (A + mu I) p in FP64 arithmetic (FP64 PCG).
int32_t op_matvec_f64(const nys_operator* op, double mu, const double* p, double* v,
                      const int* skip, void* work, cudaStream_t s);
// Batched FP32 matvec V[s] = (A + mu_s I) P[s] for nsys systems sharing the
// operator (RBF only; NYS_ERR_ARG otherwise, and the caller loops).  d_mu:
// device [nsys]; done0[s * done_stride] != 0 marks a converged system.
// work: NULL, or rbf_tc_work_bytes(n, nsys, 3) bytes (then nothing is
// allocated during the call).
int32_t op_matvec_batched_f32(const nys_operator* op, const double* d_mu, int64_t nsys,
                              const float* P, float* V, const int* done0, int64_t done_stride,
                              int* err, void* work, cudaStream_t s);
// y_q = (K + mu_q I) v_q, q < nvec, FP64-accurate in double-FP32 arithmetic
// (rbf_residual.cu).  d_mu: device [nvec].  NYS_ERR_ARG unless RBF, d <= 64.
// skip (device, may be NULL): nothing is computed while *skip is nonzero.
int32_t rbf_residual_products(const nys_operator* op, const double* d_mu, int64_t nvec,
                              const double* v, double* y, cudaStream_t s,
                              const int* skip = nullptr);
// Double-FP32 Gaussian products between targets (nt x d) and points (n x d):
// kind 0 y_q = K(t, x) v_q, kind 1 y_q = dK/dsigma v_q; d_mu (device [nvec],
// or NULL) adds mu_q v_q and requires targets == points.
int32_t rbf_dfl_products(const float* tg, int64_t nt, int64_t ldt, const float* pts, int64_t n,
                         int64_t ldp, int64_t d, double sigma, int kind, const double* d_mu,
                         int64_t nvec, const double* v, double* y, cudaStream_t s);
// The same products with FP64 kernel entries and FP64 sums (~4 units of
// 2^-53 per entry): shift 0 none, 1 mu0 v_q, 2 d_mu[q] v_q (targets ==
// points); skip (device, may be NULL) returns at once when nonzero.
int32_t rbf_exact_products(const float* tg, int64_t nt, int64_t ldt, const float* pts, int64_t n,
                           int64_t ldp, int64_t d, double sigma, int kind, int shift,
                           const double* d_mu, double mu0, int64_t nvec, const double* v, double* y,
                           const int* skip, cudaStream_t s);
// Gaussian cross-kernel products (FP64): kind 0 K(t, x) v, kind 1 dK/dsigma v.
int32_t rbf_cross_matvec(const float* tg, int64_t nt, int64_t ldt, const float* pts, int64_t n,
                         int64_t ldp, int64_t d, double sigma, int64_t nvec, const double* v,
                         double* out, int kind, cudaStream_t s);
// Gaussian-kernel products on the tensor cores (rbf_tc.cu), d <= 32:
// Y[q] = K V[q] (+ shift), q < nvec, V and Y vector-major FP32 (row strides
// ldv, ldy).  shift: 0 none, 1 mu0 V[q], 2 d_mu[q] V[q] (d_mu device).
// passes: 3 (3xTF32 products, FP32 accuracy) or 1 (TF32).  done0 (device,
// may be NULL): a block of vectors whose done0[q * done_stride] are all
// nonzero is skipped.  work: NULL, or rbf_tc_work_bytes() bytes whose first
// word is the device error word (err defaults to it; NYS_ERR_TIMEOUT is
// written there if a bounded wait expired).
bool rbf_tc_supported(int64_t d);
// True when the next product of this shape would time its launch shapes
// (the tuner is on and has no entry for it): a solve runs one product
// before it captures its iteration graph, where nothing can be timed.
bool rbf_tc_tune_pending(int64_t n, int64_t d, int64_t nvec, int passes);
// Work buffer of rbf_tc_products (input re-layouts and the partial sums of
// point slices), error word first.
size_t rbf_tc_work_bytes(int64_t n, int64_t nvec, int passes);
int32_t rbf_tc_products(const float* pts, int64_t n, int64_t d, int64_t ld, double sigma,
                        int64_t nvec, const float* V, int64_t ldv, int shift, const double* d_mu,
                        double mu0, float* Y, int64_t ldy, int passes, const int* done0,
                        int64_t done_stride, void* work, int* err, cudaStream_t s);
// FP64-accurate v = (A + mu I) p for the refinement residual: the ridge
// operator in double-FP32 arithmetic (~2^-44 relative), the others in FP64.
int32_t op_matvec_residual(const nys_operator* op, double mu, const double* p, double* v,
                           const int* skip, void* work, cudaStream_t s);

}  // namespace nys
