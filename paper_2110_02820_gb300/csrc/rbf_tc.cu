// Gaussian-kernel products on the 5th-generation tensor cores (sm_103a):
//
//   Y[s][i] = sum_j exp(-||x_i - x_j||^2 / (2 sigma^2)) V[s][j]  (+ mu_s V[s][i])
//
// for a block of vectors s, computed on the fly (the kernel matrix is never
// stored).  This is the matrix-free operator of kernel ridge regression
// (Sec. 6.2) applied inside PCG (one vector per system, Algorithm 3), to a
// batch of systems that share the kernel (a regularisation path), and to
// the n x ell test matrix of the sketch Y = K Omega (Algorithm 1).
//
// The exponent is formed by norm expansion,
//   -||x_i - x_j||^2 / (2 sigma^2) log2(e) = cn_i + cn_j + m2c <x_i, x_j>,
// with cn_i = -log2(e) ||x_i||^2 / (2 sigma^2) and m2c = log2(e) / sigma^2,
// so the inner products form a GEMM with K = d.  That GEMM cancels: for
// points far from the origin the inner product is much larger than the
// distance, so it runs as 3xTF32 (x = hi + lo, each TF32; hi.hi + hi.lo +
// lo.hi), which keeps it at FP32 accuracy.
//
// One CTA owns 128 rows i and sweeps all points j in tiles of 64:
//   warp 0, lane 0: TMA producer.  X_I (hi, lo) once; per tile a stage of
//                   X_J (hi, lo), cn_J and the tile's slice of the vectors,
//                   into an NS-deep ring.
//   warp 1, lane 0: MMA issuer.  GEMM1(t): P = X_I X_J^T (3 passes, K = 8
//                   per MMA, into one of two 128 x 64 TMEM buffers).  With
//                   several vectors, GEMM2(t-1): Yacc += K_{t-1} V_{t-1},
//                   the kernel tile K read from TMEM as the A operand (3
//                   passes, or 1 for the sketch).  Warp 1 also owns TMEM.
//   warps 2..9:     two exp groups of four warps that take alternate tiles
//                   (group g owns P / K buffer g), one thread per row i:
//                   tcgen05.ld of the 64 inner products, k = 2^(cn_i + cn_j +
//                   m2c p); then either (one vector) acc_i += k v_j on the
//                   FP32 pipe, or the TF32 hi / lo split of k stored into the
//                   tile's TMEM buffer for GEMM2.  Group 0 also promotes the
//                   Yacc chunks and writes the result (+ mu_s v_i).
// Tensor-core FP32 accumulation does not round to nearest; a long chain of
// accumulating MMAs drifts toward zero (~1e-8 relative per MMA, measured), so
// GEMM2 accumulates a chunk of two tiles at a time (48 chained TF32 MMAs, 24
// FP16 ones) and the exp groups add each chunk into FP32 sums with ordinary
// rounding.  Shorter chains leave less error on a product (3xTF32: 1.5e-6
// norm-wise with 48 MMAs against 2.6e-6 with 96; FP16: 7.3e-7 with 24, 1.2e-6
// with 48, 2.0e-6 with 96, measured at n = 5e4), and the regularisation
// path's refinement then contracts faster.  Every wait is bounded; on expiry the CTA records
// NYS_ERR_TIMEOUT in *err, lets its copies in flight land, frees its TMEM and
// returns.
//
// Many vectors run by default on FP16 splits (rbf_h16_kernel below: kind::f16
// at twice the TF32 rate, K tiles half the size in TMEM, a four-deep TMEM
// pipeline); the 3xTF32 kernel above it stays selectable (NYS_RBF_TF32=1).
// FP16 splits: the points scaled by a power of two (max |x| in [2^9, 2^10)),
// the kernel entries by 2^15 (k in (0, 2^15]) and each vector by its own
// power of two (max |v| in [2^14, 2^15)), each value split as hi = fp16(x),
// lo = fp16(x - hi), and the result scaled back by 2^-(15 + e_s).  An FP16
// hi + lo pair carries 22 significant bits like a TF32 pair; below the FP16
// normal range the split is absolute, at most 2^-39 of the largest entry of
// the operand.

#include <cuda_fp16.h>

#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "ptx.cuh"
#include "tmap.h"

namespace nys {

namespace {

constexpr int RT_BM = 128;   // rows i per CTA
constexpr int RT_BN = 64;    // points j per tile
constexpr int RT_DP = 32;    // padded point dimension (d <= 32)
constexpr int RT_EXP_WARPS = 8;
constexpr int RT_THREADS = 64 + 32 * RT_EXP_WARPS;
constexpr uint32_t RT_TMEM_COLS = 512;
constexpr int kMaxSlices = 4;  // point slices of a product (partial sums in the work buffer)

// The 3xTF32 kernel (kind::tf32, K = 8 per MMA): X_I, X_J and the vectors
// as TF32 hi and lo arrays.
template <int S, int P2>
struct RtCfg {
  static constexpr int NV = P2 == 3 ? 2 : 1;    // V arrays: hi, lo (or hi only)
  static constexpr int A_BYTES = RT_BM * 128;   // X_I: 128 rows x 128 bytes, per array
  static constexpr int A_ARR = 2;               // hi, lo
  static constexpr int XJ_BYTES = RT_BN * 128;  // X_J: 64 rows x 128 bytes, per array
  static constexpr int XJ_ARR = 2;
  static constexpr int VSLAB = S * 128;         // S vectors x 128 bytes of points
  static constexpr int VSLABS = 2;              // slabs of 32 points per V array per tile
  static constexpr int V_OFF = XJ_ARR * XJ_BYTES;
  static constexpr int CN_OFF = V_OFF + NV * VSLABS * VSLAB;
  static constexpr int TX = CN_OFF + RT_BN * 4;
  static constexpr int STAGE = (TX + 1023) / 1024 * 1024;
  static constexpr int NS = 3;
  // tiles per GEMM2 accumulation chunk (24 MMAs per tile at three passes);
  // exp group 0 takes the even tiles and promotes a chunk when it reaches
  // the next chunk's first tile, so a chunk spans an even number of tiles
  static constexpr int CH = 2;
  static constexpr bool CHUNKED = S <= 64;
  static constexpr int SUM_BYTES = CHUNKED ? S * RT_BM * 4 : 0;
  static constexpr int SMEM = 1024 + A_ARR * A_BYTES + NS * STAGE + SUM_BYTES + 256;
  // TMEM columns: P tiles at 0 / 64; K tiles (hi, lo) at TM_K, KCOLS columns
  // per part; Yacc (2 chunks) at TM_Y
  static constexpr uint32_t KCOLS = RT_BN;
  static constexpr uint32_t TM_K = 128;
  static constexpr uint32_t TM_Y = TM_K + 4 * KCOLS;
  static constexpr uint32_t YCOLS = CHUNKED ? 2 * S : S;
  static_assert(S % 32 == 0 && S <= 128, "S");
  static_assert(CH % 2 == 0 && CH >= 2, "CH");
  static_assert(TM_Y + YCOLS <= RT_TMEM_COLS, "tensor memory");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct RtArgs {
  const float* cn;     // [npad] cn_j (padding: -1e30, so that k = 0)
  float m2c;
  const float* m2c_dev;  // one vector: m2c for the scaled FP16 points (device)
  int64_t n;           // number of points
  int ntiles;          // npad / RT_BN
  int ksteps;          // ceil(d / 8): K-steps of GEMM1 (coordinates beyond d are zero)
  int64_t nvec;
  int64_t spad;        // rows of each V array in the stage map
  int64_t vec;         // one vector: its index q (the rest of the fields index all vectors)
  const float* vj;     // one vector: [npad] v_q (zero padded), loaded per tile
  const double* mus;   // [nvec] shifts (device), or NULL: mu0 for every vector
  float mu0;
  const float* v;      // [nvec][ldv] vectors for the shift term, or NULL: no shift
  int64_t ldv;
  float* y;            // [nvec][ldy]
  int64_t ldy;
  const int* done0;    // done0[s * done_stride] != 0: vector s needs no product (or NULL)
  int64_t done_stride;
  int* err;
  int tile_chunk;      // tiles of points per slice (0: all); slices are grid.y for one
                       // vector, grid.z for many
  float* ypart;        // partial sums (NULL: write y directly): one vector [slices][npad],
                       // many [slices][nvec][part_stride], no shift term
  int64_t part_stride;
  const float* vscale;  // [nvec] result scale per vector (FP16 products), or NULL
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// A operand from tensor memory (the kernel tile), B from shared memory.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Instruction descriptor: kind::f16 with FP16 A and B (both K-major), FP32 D.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
  return (1u << 4)                      // D format: F32
         | (0u << 7)                    // A format: F16
         | (0u << 10)                   // B format: F16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// A operand from tensor memory (the kernel tile, FP16 packed two to a
// column), B from shared memory.
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Two FP32 values rounded to FP16 (nearest even) in one word: x0 in the low
// half, x1 in the high half.
__device__ __forceinline__ uint32_t pack_f16x2(float x0, float x1) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
  return r;
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
      : "memory");
}


__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed FP32 pairs (sm_100 family): two lanes of FP32 arithmetic per
// instruction, each rounded as the scalar operation.
__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2unpack(uint64_t r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// The two FP16 halves of a word as FP32 values (exact).
__device__ __forceinline__ void unpack_f16x2(uint32_t w, float& lo, float& hi) {
  asm("{.reg .f16 a, b;\n\tmov.b32 {a, b}, %2;\n\tcvt.f32.f16 %0, a;\n\tcvt.f32.f16 %1, b;\n\t}"
      : "=f"(lo), "=f"(hi)
      : "r"(w));
}

// Round to the nearest TF32 value (ties away from zero), kept in an FP32
// container: add half a unit of the 13 dropped bits, then clear them.
// Integer ALU work (finite inputs below 2^127 only, which holds here).
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Ties the registers written by tcgen05.ld to a point after the wait, so
// that no use of them can be scheduled before tcgen05.wait::ld.
__device__ __forceinline__ void reg_fence16(uint32_t (&r)[16]) {
#pragma unroll
  for (int i = 0; i < 16; i += 8)
    asm volatile("" : "+r"(r[i]), "+r"(r[i + 1]), "+r"(r[i + 2]), "+r"(r[i + 3]), "+r"(r[i + 4]),
                 "+r"(r[i + 5]), "+r"(r[i + 6]), "+r"(r[i + 7])::"memory");
}

__device__ __forceinline__ void reg_fence32(uint32_t (&r)[32]) {
#pragma unroll
  for (int i = 0; i < 32; i += 8)
    asm volatile("" : "+r"(r[i]), "+r"(r[i + 1]), "+r"(r[i + 2]), "+r"(r[i + 3]), "+r"(r[i + 4]),
                 "+r"(r[i + 5]), "+r"(r[i + 6]), "+r"(r[i + 7])::"memory");
}


// Add Yacc chunk c (TMEM columns TMY + S (c & 1)) into the FP32 sums of
// row r (sY[s][r]) and release the buffer.  Called by each warp of group 0.
template <int S, uint32_t TMY>
__device__ __forceinline__ bool promote(uint32_t tmem, uint32_t lane_base, int c, uint64_t* ycf,
                                        uint64_t* ycfree, float* sY, int r, int lane) {
  if (!mbar_wait_bounded(&ycf[c & 1], (uint32_t)((c >> 1) & 1))) return false;
  tc_fence_after();
#pragma unroll 1
  for (int c0 = 0; c0 < S; c0 += 32) {
    uint32_t v[32];
    tmem_ld32_nw(tmem + lane_base + TMY + (uint32_t)((c & 1) * S + c0), v);
    tmem_wait_ld();
    reg_fence32(v);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float* p = &sY[(c0 + j) * RT_BM + r];
      *p = (c == 0) ? __uint_as_float(v[j]) : *p + __uint_as_float(v[j]);
    }
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&ycfree[c & 1]);
  return true;
}

// Many vectors: y[sv][row] = val (+ mu_sv v[sv][row]), or, with point
// slices, the slice's partial sum (the shift is added once, by rt_sum_kernel).
__device__ __forceinline__ void rt_store(const RtArgs& a, int64_t sv, int64_t row, float val) {
  if (a.vscale) val *= a.vscale[sv];
  if (a.ypart) {
    a.ypart[((int64_t)blockIdx.z * a.nvec + sv) * a.part_stride + row] = val;
    return;
  }
  if (a.v) val = fmaf(a.mus ? (float)a.mus[sv] : a.mu0, a.v[sv * a.ldv + row], val);
  a.y[sv * a.ldy + row] = val;
}

template <int S, int P2>
__global__ void __launch_bounds__(RT_THREADS, 1)
rbf_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV,
              RtArgs a) {
  using Cfg = RtCfg<S, P2>;
  constexpr int NS = Cfg::NS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sSt = sm + Cfg::A_ARR * Cfg::A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sSt + NS * Cfg::STAGE);
  uint64_t* empty = full + NS;
  uint64_t* afull = empty + NS;
  uint64_t* pfull = afull + 1;
  uint64_t* pfree = pfull + 2;
  uint64_t* kfull = pfree + 2;
  uint64_t* kfree = kfull + 2;
  uint64_t* yfull = kfree + 2;
  uint64_t* ycf = yfull + 1;    // [2] chunk of Yacc complete (MMA -> group 0)
  uint64_t* ycfree = ycf + 2;   // [2] chunk promoted, buffer free (group 0 -> MMA)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ycfree + 2);
  float* sY = reinterpret_cast<float*>(sSt + NS * Cfg::STAGE + 256);
  __shared__ int s_fail, s_skip;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * RT_BM;
  const int64_t s0 = (int64_t)blockIdx.y * S;
  // this CTA's slice of the point tiles, [t0, t0 + T) (grid.z; see ypart)
  const int t0 = a.tile_chunk > 0 ? (int)blockIdx.z * a.tile_chunk : 0;
  const int T = a.tile_chunk > 0 ? min(a.ntiles - t0, a.tile_chunk) : a.ntiles;

  if (threadIdx.x == 0) {
    int skip = 0;
    if (a.done0) {
      skip = 1;
      const int64_t s1 = (s0 + S < a.nvec) ? s0 + S : a.nvec;
      for (int64_t s = s0; s < s1; ++s)
        if (!a.done0[s * a.done_stride]) { skip = 0; break; }
    }
    s_skip = skip;
    s_fail = 0;
    if (!skip) {
      for (int i = 0; i < NS; ++i) {
        mbar_init(&full[i], 1);
        mbar_init(&empty[i], 1);
      }
      mbar_init(afull, 1);
      for (int i = 0; i < 2; ++i) {
        mbar_init(&pfull[i], 1);
        mbar_init(&pfree[i], 4);
        mbar_init(&kfull[i], 4);
        mbar_init(&kfree[i], 1);
        mbar_init(&ycf[i], 1);
        mbar_init(&ycfree[i], 4);
      }
      mbar_init(yfull, 1);
      fence_barrier_init();
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmX) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmV) : "memory");
    }
  }
  __syncthreads();
  if (s_skip) return;
  if (warp == 1) tmem_alloc(tmem_slot, RT_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // all 512 columns of lane 0 onward: anything else is recorded and the CTA
  // does no work (it frees what it was given and reports NYS_ERR_TIMEOUT)
  const bool tmem_ok = tmem == 0u;
  if (!tmem_ok) {
    if (threadIdx.x == 0) atomicCAS(a.err, 0, (int)NYS_ERR_TIMEOUT);
  } else if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      mbar_arrive_expect_tx(afull, (uint32_t)(Cfg::A_ARR * Cfg::A_BYTES));
#pragma unroll
      for (int arr = 0; arr < Cfg::A_ARR; ++arr) {
        tma_load_2d(sA + arr * Cfg::A_BYTES, &tmX, arr * RT_DP, (int)m0, afull);
        tma_load_2d(sA + arr * Cfg::A_BYTES + Cfg::A_BYTES / 2, &tmX, arr * RT_DP, (int)m0 + 64,
                    afull);
      }
      int issued = 0;
      for (int t = 0; t < T; ++t) {
        const int s = t % NS;
        if (t >= NS && !mbar_wait_bounded(&empty[s], (uint32_t)(((t / NS) - 1) & 1))) {
          atomicOr(&s_fail, 1);
          break;
        }
        if (*(volatile int*)&s_fail) break;
        unsigned char* st = sSt + s * Cfg::STAGE;
        const int j0 = (t0 + t) * RT_BN;
        mbar_arrive_expect_tx(&full[s], (uint32_t)Cfg::TX);
#pragma unroll
        for (int arr = 0; arr < Cfg::XJ_ARR; ++arr)
          tma_load_2d(st + arr * Cfg::XJ_BYTES, &tmX, arr * RT_DP, j0, &full[s]);
#pragma unroll
        for (int arr = 0; arr < Cfg::NV; ++arr)
#pragma unroll
          for (int slab = 0; slab < Cfg::VSLABS; ++slab)
            tma_load_2d(st + Cfg::V_OFF + (arr * Cfg::VSLABS + slab) * Cfg::VSLAB, &tmV,
                        j0 + 32 * slab, (int)(arr * a.spad + s0), &full[s]);
        bulk_g2s(st + Cfg::CN_OFF, a.cn + j0, RT_BN * 4, &full[s]);
        issued = t + 1;
      }
      if (*(volatile int*)&s_fail) {
        // let the copies still in flight land before the CTA exits
        mbar_wait_bounded(afull, 0u);
        for (int t = (issued > NS ? issued - NS : 0); t < issued; ++t)
          mbar_wait_bounded(&full[t % NS], (uint32_t)((t / NS) & 1));
      } else {
        // the last stages' releases include the tensor core's asynchronous
        // commit arrivals: they must land before the shared memory is freed
        for (int t = (T > NS ? T - NS : 0); t < T; ++t)
          if (!mbar_wait_bounded(&empty[t % NS], (uint32_t)((t / NS) & 1))) atomicOr(&s_fail, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc1 = tf32_idesc(RT_BM, RT_BN);
      constexpr uint32_t idesc2 = tf32_idesc(RT_BM, S);
      // one K-step (8 TF32) is 32 bytes of a 128-byte row: +2 in the
      // descriptor's 16-byte units
      constexpr int K1 = RT_DP / 8;  // K-steps of GEMM1 at d = 32
      bool ok = mbar_wait_bounded(afull, 0u);
      const uint64_t aHiD = sw128_kmajor_desc(smem_u32(sA));
      const uint64_t aLoD = sw128_kmajor_desc(smem_u32(sA + Cfg::A_BYTES));
      const int ks = a.ksteps;
      for (int t = 0; ok && t <= T; ++t) {
        if (t < T) {
          const int s = t % NS, b = t & 1;
          if (!mbar_wait_bounded(&full[s], (uint32_t)((t / NS) & 1))) { ok = false; break; }
          if (t >= 2 && !mbar_wait_bounded(&pfree[b], (uint32_t)(((t - 2) >> 1) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t bHiD = sw128_kmajor_desc(smem_u32(sSt + s * Cfg::STAGE));
          const uint64_t bLoD = bHiD + (uint64_t)(Cfg::XJ_BYTES >> 4);
          const uint32_t dP = tmem + (uint32_t)(b * RT_BN);
#pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const uint64_t ad = pass == 2 ? aLoD : aHiD;
            const uint64_t bd = pass == 1 ? bLoD : bHiD;
#pragma unroll
            for (int k = 0; k < K1; ++k)
              if (k < ks)
                mma_tf32(dP, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc1,
                         (pass > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(&pfull[b]);
        }
        if (t >= 1) {
          const int u = t - 1, bu = u & 1, su = u % NS;
          if (!mbar_wait_bounded(&kfull[bu], (uint32_t)((u >> 1) & 1))) { ok = false; break; }
          const int c = u / Cfg::CH;
          const bool first = Cfg::CHUNKED ? (u % Cfg::CH == 0) : (u == 0);
          if (Cfg::CHUNKED && first && c >= 2 &&
              !mbar_wait_bounded(&ycfree[c & 1], (uint32_t)(((c - 2) >> 1) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t kHi = tmem + Cfg::TM_K + (uint32_t)(bu * 2 * Cfg::KCOLS);
          const uint32_t kLo = kHi + Cfg::KCOLS;
          const uint64_t vD = sw128_kmajor_desc(smem_u32(sSt + su * Cfg::STAGE + Cfg::V_OFF));
          const uint32_t dY = tmem + Cfg::TM_Y + (Cfg::CHUNKED ? (uint32_t)((c & 1) * S) : 0u);
#pragma unroll
          for (int pass = 0; pass < P2; ++pass) {
            const uint32_t ka = (pass == 2) ? kLo : kHi;
            const int arr = (pass == 1) ? 1 : 0;
#pragma unroll
            for (int k = 0; k < RT_BN / 8; ++k) {
              const uint64_t vd = vD + (uint64_t)(((arr * 2 + (k >> 2)) * Cfg::VSLAB) >> 4) +
                                  (uint64_t)(2 * (k & 3));
              mma_tf32_ts(dY, ka + (uint32_t)(8 * k), vd, idesc2,
                          (!first || pass > 0 || k > 0) ? 1u : 0u);
            }
          }
          mma_commit(&kfree[bu]);
          mma_commit(&empty[su]);
          if (Cfg::CHUNKED && (u % Cfg::CH == Cfg::CH - 1 || u == T - 1)) mma_commit(&ycf[c & 1]);
        }
      }
      if (ok) {
        if (!Cfg::CHUNKED) mma_commit(yfull);
        // the kfree arrivals of the last two tiles are not awaited by the
        // exp groups: wait here so that none lands after the CTA exits
        for (int u = (T > 2 ? T - 2 : 0); u < T; ++u)
          if (!mbar_wait_bounded(&kfree[u & 1], (uint32_t)((u >> 1) & 1))) ok = false;
      }
      if (!ok) atomicOr(&s_fail, 1);
    }
  } else {
    // ---------------- exp groups (warps 2..9); TMEM lane quarter q = warp % 4
    const int g = (warp - 2) >> 2;
    const int q = warp & 3;
    const int r = 32 * q + lane;  // row within the CTA tile
    const int64_t row = m0 + r;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const float ai = a.cn[row];
    const float m2c = a.m2c;
    bool ok = true;
    for (int t = g; t < T; t += 2) {
      const int b = g, s = t % NS;
      if (!mbar_wait_bounded(&pfull[b], (uint32_t)((t >> 1) & 1))) { ok = false; break; }
      tc_fence_after();
      uint32_t r0[32], r1[32];
      tmem_ld32_nw(tmem + lane_base + (uint32_t)(b * RT_BN), r0);
      tmem_ld32_nw(tmem + lane_base + (uint32_t)(b * RT_BN) + 32, r1);
      tmem_wait_ld();
      reg_fence32(r0);
      reg_fence32(r1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&pfree[b]);
      // the stage (cn_J) is resident: GEMM1(t) consumed it
      if (!mbar_wait_bounded(&full[s], (uint32_t)((t / NS) & 1))) { ok = false; break; }
      const float4* cn4 = reinterpret_cast<const float4*>(sSt + s * Cfg::STAGE + Cfg::CN_OFF);
      if (t >= 2 && !mbar_wait_bounded(&kfree[b], (uint32_t)(((t - 2) >> 1) & 1))) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t kHi = tmem + lane_base + Cfg::TM_K + (uint32_t)(b * 2 * Cfg::KCOLS);
      const uint32_t kLo = kHi + Cfg::KCOLS;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t(&pr)[32] = h ? r1 : r0;
        uint32_t lo[32];
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          const float4 c4 = cn4[h * 8 + j4];
          const float cj[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int jj = j4 * 4 + e;
            const float kv = ex2_approx(fmaf(__uint_as_float(pr[jj]), m2c, ai + cj[e]));
            const uint32_t hi = tf32_rna(kv);
            // the low part rounded to TF32 as well: the tensor core would
            // otherwise truncate its last 13 bits (a bias toward zero)
            lo[jj] = tf32_rna(kv - __uint_as_float(hi));
            pr[jj] = hi;
          }
        }
        tmem_st32(kHi + (uint32_t)(32 * h), pr);
        if (P2 == 3) tmem_st32(kLo + (uint32_t)(32 * h), lo);
      }
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&kfull[b]);
      if (Cfg::CHUNKED && g == 0 && t % Cfg::CH == 0 && t >= Cfg::CH) {
        if (!promote<S, Cfg::TM_Y>(tmem, lane_base, t / Cfg::CH - 1, ycf, ycfree, sY, r, lane)) {
          ok = false;
          break;
        }
      }
    }
    if (!ok) atomicOr(&s_fail, 1);
    if (g == 0) {
      if (Cfg::CHUNKED) {
        if (ok) ok = promote<S, Cfg::TM_Y>(tmem, lane_base, (T - 1) / Cfg::CH, ycf, ycfree, sY, r, lane);
        if (!ok) atomicOr(&s_fail, 1);
        if (ok && row < a.n) {
          for (int sv = 0; sv < S && s0 + sv < a.nvec; ++sv)
            rt_store(a, s0 + sv, row, sY[sv * RT_BM + r]);
        }
      } else {
        if (ok) ok = mbar_wait_bounded(yfull, 0u, 1ll << 26);
        if (!ok) atomicOr(&s_fail, 1);
        tc_fence_after();
        if (ok) {
#pragma unroll 1
          for (int c0 = 0; c0 < S; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + lane_base + Cfg::TM_Y + (uint32_t)c0, v);
            if (row < a.n) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int64_t sv = s0 + c0 + jj;
                if (sv < a.nvec) rt_store(a, sv, row, __uint_as_float(v[jj]));
              }
            }
          }
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, RT_TMEM_COLS);
  if (threadIdx.x == 0 && s_fail) atomicCAS(a.err, 0, (int)NYS_ERR_TIMEOUT);
}

// ---------------------------------------------------------------- one vector
//
// y_i = sum_j k(x_i, x_j) v_j (+ mu v_i): GEMM1 on the tensor cores in 128-point
// tiles (3xTF32, N = 128), the exponentials and the products with v on the
// exp warps (FP32, Kahan-compensated across tiles).  Four exp groups take
// tiles round-robin, each with its own 128-column TMEM buffer, so that every
// SMSP holds four exp warps to cover the tensor-memory latency; within a tile
// the next 16 columns are loaded while the current ones are used.
//
// GEMM1 runs on FP16 splits: each point, scaled by a power of two so that its
// largest coordinate lies in [2^9, 2^10), is one 128-byte row [hi(32) | lo(32)]
// of FP16 values (hi = fp16(x), lo = fp16(x - hi)), and the inner products are
// hi.hi + hi.lo + lo.hi as kind::f16 MMAs (K = 16, FP32 accumulation): the
// 2^-22 relative accuracy of 3xTF32 at twice its tensor rate.
constexpr int GV_BN = 128;
constexpr int GV_G = 4;
constexpr int GV_THREADS = 64 + GV_G * 128;
constexpr int GV_NS = 6;
constexpr int GV_XJ = GV_BN * 128;            // X_J [hi | lo]: 128 rows x 64 FP16
constexpr int GV_CN = GV_XJ;                  // cn_J
constexpr int GV_VJ = GV_CN + GV_BN * 4;      // v_J
constexpr int GV_TX = GV_VJ + GV_BN * 4;
constexpr int GV_STAGE = (GV_TX + 1023) / 1024 * 1024;
constexpr int GV_A = RT_BM * 128;             // X_I [hi | lo]
constexpr int GV_SMEM = 1024 + GV_A + GV_NS * GV_STAGE + 256 + GV_G * RT_BM * 8;

static_assert(GV_SMEM <= 227 * 1024, "shared memory");

__device__ __forceinline__ void gv_bar_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(GV_G * 128) : "memory");
}

__global__ void __launch_bounds__(GV_THREADS, 1)
rbf_gemv_kernel(const __grid_constant__ CUtensorMap tmX, RtArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sSt = sm + GV_A;
  uint64_t* full = reinterpret_cast<uint64_t*>(sSt + GV_NS * GV_STAGE);
  uint64_t* empty = full + GV_NS;
  uint64_t* afull = empty + GV_NS;
  uint64_t* pfull = afull + 1;
  uint64_t* pfree = pfull + GV_G;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pfree + GV_G);
  double* sD = reinterpret_cast<double*>(sSt + GV_NS * GV_STAGE + 256);  // [G][128]
  __shared__ int s_fail, s_skip;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * RT_BM;
  const int64_t q0 = a.vec;
  // this CTA's slice of the point tiles (grid.y splits them; see ypart)
  const int t0 = a.tile_chunk > 0 ? (int)blockIdx.y * a.tile_chunk : 0;
  const int T = a.tile_chunk > 0 ? min(a.ntiles - t0, a.tile_chunk) : a.ntiles;

  if (threadIdx.x == 0) {
    s_skip = (a.done0 && a.done0[q0 * a.done_stride]) ? 1 : 0;
    s_fail = 0;
    if (!s_skip) {
      for (int i = 0; i < GV_NS; ++i) {
        mbar_init(&full[i], 1);
        mbar_init(&empty[i], 1 + 4);
      }
      mbar_init(afull, 1);
      for (int i = 0; i < GV_G; ++i) {
        mbar_init(&pfull[i], 1);
        mbar_init(&pfree[i], 4);
      }
      fence_barrier_init();
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmX) : "memory");
    }
  }
  __syncthreads();
  if (s_skip) return;
  if (warp == 1) tmem_alloc(tmem_slot, RT_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const bool tmem_ok = tmem == 0u;
  if (!tmem_ok) {
    if (threadIdx.x == 0) atomicCAS(a.err, 0, (int)NYS_ERR_TIMEOUT);
  } else if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      mbar_arrive_expect_tx(afull, (uint32_t)GV_A);
      tma_load_2d(sA, &tmX, 0, (int)m0, afull);
      tma_load_2d(sA + GV_A / 2, &tmX, 0, (int)m0 + 64, afull);
      int issued = 0;
      for (int t = 0; t < T; ++t) {
        const int s = t % GV_NS;
        if (t >= GV_NS && !mbar_wait_bounded(&empty[s], (uint32_t)(((t / GV_NS) - 1) & 1))) {
          atomicOr(&s_fail, 1);
          break;
        }
        if (*(volatile int*)&s_fail) break;
        unsigned char* st = sSt + s * GV_STAGE;
        const int j0 = (t0 + t) * GV_BN;
        mbar_arrive_expect_tx(&full[s], (uint32_t)GV_TX);
        tma_load_2d(st, &tmX, 0, j0, &full[s]);
        tma_load_2d(st + GV_XJ / 2, &tmX, 0, j0 + 64, &full[s]);
        bulk_g2s(st + GV_CN, a.cn + j0, GV_BN * 4, &full[s]);
        bulk_g2s(st + GV_VJ, a.vj + j0, GV_BN * 4, &full[s]);
        issued = t + 1;
      }
      if (*(volatile int*)&s_fail) {
        mbar_wait_bounded(afull, 0u);
        for (int t = (issued > GV_NS ? issued - GV_NS : 0); t < issued; ++t)
          mbar_wait_bounded(&full[t % GV_NS], (uint32_t)((t / GV_NS) & 1));
      } else {
        // the last stages' releases include the tensor core's asynchronous
        // commit arrivals: they must land before the shared memory is freed
        for (int t = (T > GV_NS ? T - GV_NS : 0); t < T; ++t)
          if (!mbar_wait_bounded(&empty[t % GV_NS], (uint32_t)((t / GV_NS) & 1)))
            atomicOr(&s_fail, 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer (GEMM1 only)
      constexpr uint32_t idesc = f16_idesc(RT_BM, GV_BN);
      bool ok = mbar_wait_bounded(afull, 0u);
      const uint64_t aHiD = sw128_kmajor_desc(smem_u32(sA));
      const uint64_t aLoD = aHiD + (uint64_t)(64 >> 4);  // lo half of each 128-byte row
      const int ks = a.ksteps;                             // ceil(d / 16)
      for (int t = 0; ok && t < T; ++t) {
        const int s = t % GV_NS, b = t % GV_G;
        if (!mbar_wait_bounded(&full[s], (uint32_t)((t / GV_NS) & 1))) { ok = false; break; }
        if (t >= GV_G && !mbar_wait_bounded(&pfree[b], (uint32_t)(((t - GV_G) / GV_G) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t bHiD = sw128_kmajor_desc(smem_u32(sSt + s * GV_STAGE));
        const uint64_t bLoD = bHiD + (uint64_t)(64 >> 4);
        const uint32_t dP = tmem + (uint32_t)(b * GV_BN);
#pragma unroll
        for (int pass = 0; pass < 3; ++pass) {
          const uint64_t ad = pass == 2 ? aLoD : aHiD;
          const uint64_t bd = pass == 1 ? bLoD : bHiD;
#pragma unroll
          for (int k = 0; k < 2; ++k)  // 16 FP16 (32 bytes) per K-step, d <= 32
            if (k < ks)
              mma_f16(dP, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                      (pass > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&pfull[b]);
        mma_commit(&empty[s]);
      }
      if (!ok) atomicOr(&s_fail, 1);
    }
  } else {
    // ---------------- exp groups (warps 2 .. 2 + 4G - 1); TMEM lane quarter q = warp % 4
    const int g = (warp - 2) >> 2;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const int64_t row = m0 + r;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const float ai = a.cn[row];
    const float m2c = *a.m2c_dev;  // log2(e) / (sigma^2 scale^2) for the scaled points
    bool ok = true;
    float acc = 0.f, comp = 0.f;
    for (int t = g; t < T; t += GV_G) {
      const int s = t % GV_NS;
      if (!mbar_wait_bounded(&pfull[g], (uint32_t)((t / GV_G) & 1))) { ok = false; break; }
      tc_fence_after();
      if (!mbar_wait_bounded(&full[s], (uint32_t)((t / GV_NS) & 1))) { ok = false; break; }
      const float4* cn4 = reinterpret_cast<const float4*>(sSt + s * GV_STAGE + GV_CN);
      const float4* v4 = reinterpret_cast<const float4*>(sSt + s * GV_STAGE + GV_VJ);
      const uint32_t P = tmem + lane_base + (uint32_t)(g * GV_BN);
      uint32_t ra[16], rb[16];
      tmem_ld16_nw(P, ra);
      tmem_wait_ld();
      reg_fence16(ra);
      // four partial sums (one per point of a float4): four short dependent
      // FMA chains per tile instead of one of 128
      float ts[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < GV_BN / 16; ++c) {
        uint32_t(&cur)[16] = (c & 1) ? rb : ra;
        uint32_t(&nxt)[16] = (c & 1) ? ra : rb;
        if (c + 1 < GV_BN / 16) tmem_ld16_nw(P + (uint32_t)(16 * (c + 1)), nxt);
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) {
          const float4 c4 = cn4[c * 4 + j4], w4 = v4[c * 4 + j4];
          const float cj[4] = {c4.x, c4.y, c4.z, c4.w};
          const float vj[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float kv = ex2_approx(fmaf(__uint_as_float(cur[j4 * 4 + e]), m2c, ai + cj[e]));
            ts[e] = fmaf(kv, vj[e], ts[e]);
          }
        }
        if (c + 1 < GV_BN / 16) {
          tmem_wait_ld();
          reg_fence16(nxt);
          if (c + 2 == GV_BN / 16) {
            // the whole tile is in registers: release the TMEM buffer
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&pfree[g]);
          }
        }
      }
      const float yk = ((ts[0] + ts[1]) + (ts[2] + ts[3])) - comp;
      const float tk = acc + yk;
      comp = (tk - acc) - yk;
      acc = tk;
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (!ok) atomicOr(&s_fail, 1);
    sD[g * RT_BM + r] = (double)acc - (double)comp;
    gv_bar_sync();
    if (g == 0 && !*(volatile int*)&s_fail && row < a.n) {
      double tot = 0.0;
#pragma unroll
      for (int h = 0; h < GV_G; ++h) tot += sD[h * RT_BM + r];
      if (a.ypart) {
        a.ypart[(int64_t)blockIdx.y * a.part_stride + row] = (float)tot;
      } else {
        float val = (float)tot;
        if (a.v) val = fmaf(a.mus ? (float)a.mus[q0] : a.mu0, a.v[q0 * a.ldv + row], val);
        a.y[q0 * a.ldy + row] = val;
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, RT_TMEM_COLS);
  if (threadIdx.x == 0 && s_fail) atomicCAS(a.err, 0, (int)NYS_ERR_TIMEOUT);
}

// y[q][row] = sum_z part[z][row] (fixed order) + shift, for the one-vector
// product split over point slices.
__global__ void gv_sum_kernel(const float* __restrict__ part, int nz, int64_t stride, RtArgs a) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t q0 = a.vec;
  if (row >= a.n) return;
  if (a.done0 && a.done0[q0 * a.done_stride]) return;
  float val = 0.f;
  for (int z = 0; z < nz; ++z) val += part[(int64_t)z * stride + row];
  if (a.v) val = fmaf(a.mus ? (float)a.mus[q0] : a.mu0, a.v[q0 * a.ldv + row], val);
  a.y[q0 * a.ldy + row] = val;
}

// y[sv][row] = sum_z part[z][sv][row] (fixed order) + shift, for the
// many-vector product split over point slices; vectors whose `done` word is
// set are left alone, as the product kernel leaves them.
__global__ void rt_sum_kernel(const float* __restrict__ part, int nz, RtArgs a) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= a.n) return;
  for (int64_t sv = blockIdx.y; sv < a.nvec; sv += gridDim.y) {
    if (a.done0 && a.done0[sv * a.done_stride]) continue;
    float val = 0.f;
    for (int z = 0; z < nz; ++z) val += part[((int64_t)z * a.nvec + sv) * a.part_stride + row];
    if (a.v) val = fmaf(a.mus ? (float)a.mus[sv] : a.mu0, a.v[sv * a.ldv + row], val);
    a.y[sv * a.ldy + row] = val;
  }
}

// max |x_jk| over the points (bit pattern of a non-negative float).
__global__ void rt_absmax_kernel(const float* __restrict__ pts, int64_t n, int64_t d, int64_t ld,
                                 unsigned int* out) {
  float m = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / d, k = e - j * d;
    m = fmaxf(m, fabsf(pts[j * ld + k]));
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// One-vector layout: XS16[j] = [fp16(s x_j) | fp16(s x_j - fp16(s x_j))] (32 + 32
// FP16, zero padded) with s = 2^(10 - e), max |x| in [2^(e-1), 2^e); cn as for
// the FP32 layout; *m2c_dev = m2c / s^2.
__global__ void rt_prep_points16_kernel(const float* __restrict__ pts, int64_t n, int64_t d,
                                        int64_t ld, int64_t npad, double c, double m2c,
                                        const unsigned int* absmax, __half* __restrict__ XS16,
                                        float* __restrict__ cn, float* m2c_dev) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const float mx = __uint_as_float(*absmax);
  int e = 0;
  if (mx > 0.f) frexpf(mx, &e);
  const float sc = mx > 0.f ? ldexpf(1.f, 10 - e) : 1.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) *m2c_dev = (float)(m2c / ((double)sc * (double)sc));
  if (j >= npad) return;
  const float x = (j < n && lane < d) ? pts[j * ld + lane] : 0.0f;
  const float xs = x * sc;
  const __half hi = __float2half_rn(xs);
  const __half lo = __float2half_rn(xs - __half2float(hi));
  XS16[j * 64 + lane] = hi;
  XS16[j * 64 + 32 + lane] = lo;
  const double s2 = warp_sum((double)x * (double)x);
  if (lane == 0) cn[j] = (j < n) ? (float)(c * s2) : -1e30f;
}

// XS[j] = [tf32(x_j) | tf32(x_j - tf32(x_j))] (32 + 32 FP32, zero padded),
// cn[j] = c ||x_j||^2 (FP64 sum of the FP32 coordinates), -1e30 for padding.
__global__ void rt_prep_points_kernel(const float* __restrict__ pts, int64_t n, int64_t d,
                                      int64_t ld, int64_t npad, double c, float* __restrict__ XS,
                                      float* __restrict__ cn) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= npad) return;
  const float x = (j < n && lane < d) ? pts[j * ld + lane] : 0.0f;
  const float hi = __uint_as_float(tf32_rna(x));
  const float lo = __uint_as_float(tf32_rna(x - hi));
  XS[j * 64 + lane] = hi;
  XS[j * 64 + 32 + lane] = lo;
  const double s2 = warp_sum((double)x * (double)x);
  if (lane == 0) cn[j] = (j < n) ? (float)(c * s2) : -1e30f;
}

// VS[arr][s][j] (spad x npad each): nv = 2: arr 0 = tf32(v), arr 1 = tf32(v - tf32(v));
// nv = 1: tf32(v); nv = 0: v itself (one vector, FP32 products).
__global__ void rt_prep_vecs_kernel(const float* __restrict__ V, int64_t nvec, int64_t n,
                                    int64_t ldv, int64_t spad, int64_t npad, int nv,
                                    float* __restrict__ VS) {
  const int64_t total = spad * npad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / npad, j = e - s * npad;
    const float v = (s < nvec && j < n) ? V[s * ldv + j] : 0.0f;
    if (nv == 0) {
      VS[e] = v;
      continue;
    }
    const float hi = __uint_as_float(tf32_rna(v));
    VS[e] = hi;
    if (nv > 1) VS[total + e] = __uint_as_float(tf32_rna(v - hi));
  }
}

// amax[s] = max_j |V[s][j]| (bit pattern of a non-negative float; the
// array is cleared first).
__global__ void rt_vec_absmax_kernel(const float* __restrict__ V, int64_t nvec, int64_t n,
                                     int64_t ldv, unsigned int* amax) {
  for (int64_t sv = blockIdx.y; sv < nvec; sv += gridDim.y) {
    float m = 0.f;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
      m = fmaxf(m, fabsf(V[sv * ldv + j]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(&amax[sv], __float_as_uint(m));
  }
}

// FP16 vector layout: VS16[arr][s][j] (spad x npad each), arr 0 = fp16(c_s v),
// arr 1 = fp16(c_s v - fp16(c_s v)) (nv = 2), with c_s = 2^(15 - e_s) and
// max |v_s| in [2^(e_s - 1), 2^e_s), so that max |c_s v_s| lies in
// [2^14, 2^15); vscale[s] = 2^-15 / c_s undoes it and the 2^15 of the kernel
// entries.  Zero padding.
__global__ void rt_prep_vecs16_kernel(const float* __restrict__ V, int64_t nvec, int64_t n,
                                      int64_t ldv, int64_t spad, int64_t npad, int nv,
                                      const unsigned int* __restrict__ amax,
                                      __half* __restrict__ VS, float* __restrict__ vscale) {
  const int64_t total = spad * npad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sv = e / npad, j = e - sv * npad;
    float c = 1.f;
    if (sv < nvec) {
      const float mx = __uint_as_float(amax[sv]);
      int ex = 0;
      if (mx > 0.f) frexpf(mx, &ex);
      ex = max(ex, -100);
      c = ldexpf(1.f, 15 - ex);
      if (j == 0) vscale[sv] = ldexpf(1.f, ex - 30);
    }
    const float v = (sv < nvec && j < n) ? V[sv * ldv + j] * c : 0.0f;
    const __half hi = __float2half_rn(v);
    VS[e] = hi;
    if (nv > 1) VS[total + e] = __float2half_rn(v - __half2float(hi));
  }
}

// ---------------------------------------------------------------- many vectors, FP16 splits
//
// The same product on FP16 splits (kind::f16) with a deeper pipeline: four
// 64-column TMEM tile buffers, each holding a P tile (FP32) and then, in the
// same columns, its kernel tile K (hi | lo, FP16 packed two to a column), so
// that GEMM1 runs up to three tiles ahead of GEMM2 and an exp group finds its
// next P tile ready.  X_J / cn_J and the vector slabs come through separate
// rings (each refilled by its own producer warp): GEMM1 and the exp groups
// need X_J / cn_J several tiles before GEMM2 needs V_J.
//
//   warp 0, lane 0:  X producer.  X_I once; X_J and cn_J per tile (ring HX_NS).
//   warp 10, lane 0: V producer.  The tile's slabs of the vectors (ring HV_NS).
//   warp 11, lane 0: GEMM1 issuer.  GEMM1(u) into buffer u % HB once
//                    GEMM2(u - HB) is done with it.
//   warp 1, lane 0:  GEMM2 issuer.  GEMM2(t) into the Yacc chunk once the exp
//                    group stored K_t; it never waits for an MMA to finish.
//   warps 2..9:      two exp groups (tiles of one parity each).  P_t from
//                    TMEM, k 2^15 split into FP16 hi + lo, stored over P_t;
//                    each group adds half of the Yacc columns of a chunk into
//                    FP32 sums held in its threads' registers (one row each).
// The two issuers are separate threads because a commit's completion takes
// longer to reach a waiting thread than a tile's MMAs take to run: one
// thread that waited for GEMM2(t - 1) before issuing GEMM1 kept the tensor
// pipe idle two thirds of the time (measured with clock64 stamps).  Each
// thread's commits track its own MMAs only.
constexpr int HB = 4;        // TMEM tile buffers (64 columns each)
constexpr int HX_NS = 5;     // X_J / cn_J ring
constexpr int HV_NS = 3;     // vector-slab ring
constexpr int H_THREADS = 64 + 32 * RT_EXP_WARPS + 64;  // + V producer and GEMM1 issuer warps
constexpr int H_XSLOT = 9 * 1024;                        // X_J (8 KB) + cn_J (256 B)

template <int S, int P2>
struct H16Cfg {
  static constexpr int NV = P2 == 3 ? 2 : 1;
  static constexpr int A_BYTES = RT_BM * 128;       // X_I [hi | lo]
  static constexpr int VSLOT = NV * S * 128;        // S vectors x 64 points x FP16, per array
  // tiles per GEMM2 chunk: 2 (24 chained MMAs) leave 7.3e-7 norm-wise error on
  // a 128-vector product at n = 5e4 against 1.2e-6 with 4 and 2.0e-6 with 8
  // (measured), and the regularisation path, whose refinement contracts
  // faster on the more accurate product, runs faster with 2
  static constexpr int CH = 2;
  static constexpr bool CHUNKED = P2 == 3;
  static constexpr int HALF = S / 2;                // Yacc columns promoted by each group
  static constexpr int BAR_BYTES = 512;
  static constexpr int SMEM = 1024 + A_BYTES + HX_NS * H_XSLOT + HV_NS * VSLOT + BAR_BYTES;
  static constexpr uint32_t TM_Y = 64 * HB;
  static constexpr uint32_t YCOLS = CHUNKED ? 2 * S : S;
  static_assert(S % 32 == 0 && S <= 128, "S");
  static_assert(TM_Y + YCOLS <= RT_TMEM_COLS, "tensor memory");
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(VSLOT % 1024 == 0 && H_XSLOT % 1024 == 0, "1024-byte aligned tiles");
};

// Add columns [c0, c0 + HALF) of Yacc chunk c into this thread's FP32 sums
// (its row's, in registers) and release the chunk (one arrival per warp).
template <int S, int HALF, uint32_t TMY>
__device__ __forceinline__ bool h_promote(uint32_t tmem, uint32_t lane_base, int c, int c0,
                                          uint64_t* ycf, uint64_t* ycfree, float (&ysum)[HALF],
                                          int lane) {
  if (!mbar_wait_bounded(&ycf[c & 1], (uint32_t)((c >> 1) & 1))) return false;
  tc_fence_after();
#pragma unroll
  for (int j0 = 0; j0 < HALF; j0 += 16) {
    uint32_t v[16];
    tmem_ld16(tmem + lane_base + TMY + (uint32_t)((c & 1) * S + c0 + j0), v);
#pragma unroll
    for (int j = 0; j < 16; ++j) ysum[j0 + j] += __uint_as_float(v[j]);
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&ycfree[c & 1]);
  return true;
}

template <int S, int P2>
__global__ void __launch_bounds__(H_THREADS, 1)
rbf_h16_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmV,
               RtArgs a) {
  using Cfg = H16Cfg<S, P2>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sX = sA + Cfg::A_BYTES;
  unsigned char* sV = sX + HX_NS * H_XSLOT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sV + HV_NS * Cfg::VSLOT);
  uint64_t* afull = bars;
  uint64_t* xfull = afull + 1;      // [HX_NS] X_J, cn_J landed
  uint64_t* xempty = xfull + HX_NS; // [HX_NS] exp group read cn_J (GEMM1 is done by then)
  uint64_t* vfull = xempty + HX_NS; // [HV_NS]
  uint64_t* vempty = vfull + HV_NS; // [HV_NS] GEMM2 done with the slab
  uint64_t* pfull = vempty + HV_NS; // [HB] GEMM1 wrote P
  uint64_t* kfull = pfull + HB;     // [HB] exp group wrote K over P
  uint64_t* bfree = kfull + HB;     // [HB] GEMM2 done with K: buffer free
  uint64_t* yfull = bfree + HB;
  uint64_t* ycf = yfull + 1;        // [2] Yacc chunk complete
  uint64_t* ycfree = ycf + 2;       // [2] chunk promoted by both groups
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ycfree + 2);
  __shared__ int s_fail, s_skip;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * RT_BM;
  const int64_t s0 = (int64_t)blockIdx.y * S;
  const int t0 = a.tile_chunk > 0 ? (int)blockIdx.z * a.tile_chunk : 0;
  const int T = a.tile_chunk > 0 ? min(a.ntiles - t0, a.tile_chunk) : a.ntiles;

  if (threadIdx.x == 0) {
    int skip = 0;
    if (a.done0) {
      skip = 1;
      const int64_t s1 = (s0 + S < a.nvec) ? s0 + S : a.nvec;
      for (int64_t s = s0; s < s1; ++s)
        if (!a.done0[s * a.done_stride]) { skip = 0; break; }
    }
    s_skip = skip;
    s_fail = 0;
    if (!skip) {
      mbar_init(afull, 1);
      for (int i = 0; i < HX_NS; ++i) {
        mbar_init(&xfull[i], 1);
        mbar_init(&xempty[i], 4);
      }
      for (int i = 0; i < HV_NS; ++i) {
        mbar_init(&vfull[i], 1);
        mbar_init(&vempty[i], 1);
      }
      for (int i = 0; i < HB; ++i) {
        mbar_init(&pfull[i], 1);
        mbar_init(&kfull[i], 4);
        mbar_init(&bfree[i], 1);
      }
      mbar_init(yfull, 1);
      for (int i = 0; i < 2; ++i) {
        mbar_init(&ycf[i], 1);
        mbar_init(&ycfree[i], 8);
      }
      fence_barrier_init();
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmX) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmV) : "memory");
    }
  }
  __syncthreads();
  if (s_skip) return;
  if (warp == 1) tmem_alloc(tmem_slot, RT_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const bool tmem_ok = tmem == 0u;
  if (!tmem_ok) {
    if (threadIdx.x == 0) atomicCAS(a.err, 0, (int)NYS_ERR_TIMEOUT);
  } else if (warp == 0) {
    if (lane == 0) {
      // ---------------- X producer
      mbar_arrive_expect_tx(afull, (uint32_t)Cfg::A_BYTES);
      tma_load_2d(sA, &tmX, 0, (int)m0, afull);
      tma_load_2d(sA + Cfg::A_BYTES / 2, &tmX, 0, (int)m0 + 64, afull);
      int issued = 0;
      for (int t = 0; t < T; ++t) {
        const int s = t % HX_NS;
        if (t >= HX_NS && !mbar_wait_bounded(&xempty[s], (uint32_t)(((t / HX_NS) - 1) & 1))) {
          atomicOr(&s_fail, 1);
          break;
        }
        if (*(volatile int*)&s_fail) break;
        unsigned char* st = sX + s * H_XSLOT;
        const int j0 = (t0 + t) * RT_BN;
        mbar_arrive_expect_tx(&xfull[s], (uint32_t)(RT_BN * 128 + RT_BN * 4));
        tma_load_2d(st, &tmX, 0, j0, &xfull[s]);
        bulk_g2s(st + RT_BN * 128, a.cn + j0, RT_BN * 4, &xfull[s]);
        issued = t + 1;
      }
      // every X copy is awaited by GEMM1 and the exp groups; after a failure,
      // let the copies still in flight land before the CTA exits
      if (*(volatile int*)&s_fail) {
        mbar_wait_bounded(afull, 0u);
        for (int t = (issued > HX_NS ? issued - HX_NS : 0); t < issued; ++t)
          mbar_wait_bounded(&xfull[t % HX_NS], (uint32_t)((t / HX_NS) & 1));
      }
    }
  } else if (warp == RT_EXP_WARPS + 2) {
    if (lane == 0) {
      // ---------------- V producer
      int issued = 0;
      for (int t = 0; t < T; ++t) {
        const int s = t % HV_NS;
        if (t >= HV_NS && !mbar_wait_bounded(&vempty[s], (uint32_t)(((t / HV_NS) - 1) & 1))) {
          atomicOr(&s_fail, 1);
          break;
        }
        if (*(volatile int*)&s_fail) break;
        unsigned char* st = sV + s * Cfg::VSLOT;
        const int j0 = (t0 + t) * RT_BN;
        mbar_arrive_expect_tx(&vfull[s], (uint32_t)Cfg::VSLOT);
#pragma unroll
        for (int arr = 0; arr < Cfg::NV; ++arr)
          tma_load_2d(st + arr * S * 128, &tmV, j0, (int)(arr * a.spad + s0), &vfull[s]);
        issued = t + 1;
      }
      if (*(volatile int*)&s_fail) {
        for (int t = (issued > HV_NS ? issued - HV_NS : 0); t < issued; ++t)
          mbar_wait_bounded(&vfull[t % HV_NS], (uint32_t)((t / HV_NS) & 1));
      } else {
        // the last slabs' releases are the tensor core's asynchronous commit
        // arrivals: they must land before the shared memory is freed
        for (int t = (T > HV_NS ? T - HV_NS : 0); t < T; ++t)
          if (!mbar_wait_bounded(&vempty[t % HV_NS], (uint32_t)((t / HV_NS) & 1)))
            atomicOr(&s_fail, 1);
      }
    }
  } else if (warp == RT_EXP_WARPS + 3) {
    if (lane == 0) {
      // ---------------- GEMM1 issuer: P_u = X_I X_J^T (hi.hi + hi.lo + lo.hi,
      // K = 16 per MMA) into buffer u % HB
      constexpr uint32_t idesc1 = f16_idesc(RT_BM, RT_BN);
      bool ok = mbar_wait_bounded(afull, 0u);
      const uint64_t aHiD = sw128_kmajor_desc(smem_u32(sA));
      const uint64_t aLoD = aHiD + (uint64_t)(64 >> 4);  // lo halves: 64 bytes into each row
      const int ks = a.ksteps;                             // ceil(d / 16)
      for (int u = 0; ok && u < T; ++u) {
        const int s = u % HX_NS, b = u % HB;
        if (u >= HB && !mbar_wait_bounded(&bfree[b], (uint32_t)(((u - HB) / HB) & 1))) {
          ok = false;
          break;
        }
        if (!mbar_wait_bounded(&xfull[s], (uint32_t)((u / HX_NS) & 1))) { ok = false; break; }
        tc_fence_after();
        const uint64_t bHiD = sw128_kmajor_desc(smem_u32(sX + s * H_XSLOT));
        const uint64_t bLoD = bHiD + (uint64_t)(64 >> 4);
        const uint32_t dP = tmem + (uint32_t)(b * 64);
#pragma unroll
        for (int pass = 0; pass < 3; ++pass) {
          const uint64_t ad = pass == 2 ? aLoD : aHiD;
          const uint64_t bd = pass == 1 ? bLoD : bHiD;
#pragma unroll
          for (int k = 0; k < 2; ++k)
            if (k < ks)
              mma_f16(dP, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc1,
                      (pass > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&pfull[b]);
      }
      if (!ok) atomicOr(&s_fail, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- GEMM2 issuer
      constexpr uint32_t idesc2 = f16_idesc(RT_BM, S);
      bool ok = true;
      for (int t = 0; ok && t < T; ++t) {
        const int b = t % HB, sv = t % HV_NS;
        if (!mbar_wait_bounded(&kfull[b], (uint32_t)((t / HB) & 1))) { ok = false; break; }
        const int c = t / Cfg::CH;
        const bool first = Cfg::CHUNKED ? (t % Cfg::CH == 0) : (t == 0);
        if (Cfg::CHUNKED && first && c >= 2 &&
            !mbar_wait_bounded(&ycfree[c & 1], (uint32_t)(((c - 2) >> 1) & 1))) {
          ok = false;
          break;
        }
        if (!mbar_wait_bounded(&vfull[sv], (uint32_t)((t / HV_NS) & 1))) { ok = false; break; }
        tc_fence_after();
        // GEMM2(t): Yacc += K_t V_t (Khi.Vhi + Khi.Vlo + Klo.Vhi); K_t in
        // TMEM, per 16 points (one K-step) 8 columns of hi then 8 of lo
        const uint32_t kHi = tmem + (uint32_t)(b * 64);
        const uint64_t vD = sw128_kmajor_desc(smem_u32(sV + sv * Cfg::VSLOT));
        const uint32_t dY = tmem + Cfg::TM_Y + (Cfg::CHUNKED ? (uint32_t)((c & 1) * S) : 0u);
#pragma unroll
        for (int pass = 0; pass < P2; ++pass) {
          const uint32_t ka = kHi + (pass == 2 ? 8u : 0u);
          const uint64_t vd0 = vD + (uint64_t)(((pass == 1 ? 1 : 0) * S * 128) >> 4);
#pragma unroll
          for (int k = 0; k < RT_BN / 16; ++k)
            mma_f16_ts(dY, ka + (uint32_t)(16 * k), vd0 + (uint64_t)(2 * k), idesc2,
                       (!first || pass > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&bfree[b]);
        mma_commit(&vempty[sv]);
        if (Cfg::CHUNKED && (t % Cfg::CH == Cfg::CH - 1 || t == T - 1)) mma_commit(&ycf[c & 1]);
      }
      if (ok) {
        if (!Cfg::CHUNKED) mma_commit(yfull);
        // the GEMM1 issuer awaits the bfree arrivals of tiles below T - HB:
        // wait for the others here so that none lands after the CTA exits
        for (int t = (T > HB ? T - HB : 0); t < T; ++t)
          if (!mbar_wait_bounded(&bfree[t % HB], (uint32_t)((t / HB) & 1))) ok = false;
      }
      if (!ok) atomicOr(&s_fail, 1);
    }
  } else {
    // ---------------- exp groups (warps 2..9); TMEM lane quarter q = warp % 4
    const int g = (warp - 2) >> 2;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const int64_t row = m0 + r;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const float ai = a.cn[row];
    const float m2c = *a.m2c_dev;
    const uint64_t m2c2 = f2pack(m2c, m2c), ai2 = f2pack(ai, ai),
                   scale2 = f2pack(32768.f, 32768.f);
    const int c0 = g * Cfg::HALF;  // this group's Yacc columns
    float ysum[Cfg::HALF];         // this row's sums of those columns
#pragma unroll
    for (int j = 0; j < Cfg::HALF; ++j) ysum[j] = 0.f;
    bool ok = true;
    int next_chunk = 0;            // next chunk this group promotes
    for (int t = g; t < T; t += 2) {
      const int b = t % HB, s = t % HX_NS;
      if (!mbar_wait_bounded(&pfull[b], (uint32_t)((t / HB) & 1))) { ok = false; break; }
      tc_fence_after();
      const uint32_t buf = tmem + lane_base + (uint32_t)(b * 64);
      // cn_J is resident (GEMM1(t) waited for it); this wait makes the
      // asynchronous copy visible to this thread
      if (!mbar_wait_bounded(&xfull[s], (uint32_t)((t / HX_NS) & 1))) { ok = false; break; }
      const float4* cn4 = reinterpret_cast<const float4*>(sX + s * H_XSLOT + RT_BN * 128);
      // P in four 16-column chunks (the next one loading while this one is
      // used); chunk q's K (hi: 8 columns, lo: 8) goes over chunk q's own
      // columns once they are read
      uint32_t pa[16], pb[16];
      tmem_ld16_nw(buf, pa);
      tmem_wait_ld();
      reg_fence16(pa);
#pragma unroll
      for (int qc = 0; qc < RT_BN / 16; ++qc) {
        uint32_t(&pr)[16] = (qc & 1) ? pb : pa;
        uint32_t(&pn)[16] = (qc & 1) ? pa : pb;
        if (qc + 1 < RT_BN / 16) tmem_ld16_nw(buf + (uint32_t)(16 * (qc + 1)), pn);
        // pairs of points in packed FP32 pairs (each half rounds as the
        // scalar operation): exponent, 2^15 scale, hi = fp16(k), lo =
        // fp16(k - hi) with k - hi exact in FP32; two points per TMEM column,
        // the lower point index in the lower half
        uint32_t hw[8], lw[8];
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) {
          const float4 c4 = cn4[qc * 4 + j4];
#pragma unroll
          for (int e = 0; e < 4; e += 2) {
            const uint64_t cj2 = e ? f2pack(c4.z, c4.w) : f2pack(c4.x, c4.y);
            const uint64_t p2 = f2pack(__uint_as_float(pr[j4 * 4 + e]),
                                       __uint_as_float(pr[j4 * 4 + e + 1]));
            float x0, x1;
            f2unpack(f2fma(p2, m2c2, f2add(ai2, cj2)), x0, x1);
            const uint64_t k2 = f2mul(f2pack(ex2_approx(x0), ex2_approx(x1)), scale2);
            float k0, k1;
            f2unpack(k2, k0, k1);
            const uint32_t hp = pack_f16x2(k0, k1);
            hw[2 * j4 + (e >> 1)] = hp;
            if (P2 == 3) {
              float h0, h1, l0, l1;
              unpack_f16x2(hp, h0, h1);
              f2unpack(f2sub(k2, f2pack(h0, h1)), l0, l1);
              lw[2 * j4 + (e >> 1)] = pack_f16x2(l0, l1);
            }
          }
        }
        tmem_st8(buf + (uint32_t)(16 * qc), hw);
        if (P2 == 3) tmem_st8(buf + (uint32_t)(16 * qc + 8), lw);
        if (qc + 1 < RT_BN / 16) {
          tmem_wait_ld();
          reg_fence16(pn);
        }
      }
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&kfull[b]);
        mbar_arrive(&xempty[s]);
      }
      // promote chunk c - 1 once this group reaches chunk c
      if (Cfg::CHUNKED && (t - g) % Cfg::CH == 0 && t >= Cfg::CH) {
        if (!h_promote<S, Cfg::HALF, Cfg::TM_Y>(tmem, lane_base, next_chunk, c0, ycf, ycfree,
                                                 ysum, lane)) {
          ok = false;
          break;
        }
        ++next_chunk;
      }
    }
    if (Cfg::CHUNKED) {
      const int last = (T - 1) / Cfg::CH;
      while (ok && next_chunk <= last) {
        ok = h_promote<S, Cfg::HALF, Cfg::TM_Y>(tmem, lane_base, next_chunk, c0, ycf, ycfree,
                                                 ysum, lane);
        ++next_chunk;
      }
      if (!ok) atomicOr(&s_fail, 1);
      if (ok && row < a.n) {
#pragma unroll
        for (int j = 0; j < Cfg::HALF; ++j)
          if (s0 + c0 + j < a.nvec) rt_store(a, s0 + c0 + j, row, ysum[j]);
      }
    } else {
      if (ok) ok = mbar_wait_bounded(yfull, 0u, 1ll << 26);
      if (!ok) atomicOr(&s_fail, 1);
      tc_fence_after();
      if (ok) {
#pragma unroll 1
        for (int j0 = 0; j0 < Cfg::HALF; j0 += 16) {
          uint32_t v[16];
          tmem_ld16(tmem + lane_base + Cfg::TM_Y + (uint32_t)(c0 + j0), v);
          if (row < a.n) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int64_t sv = s0 + c0 + j0 + j;
              if (sv < a.nvec) rt_store(a, sv, row, __uint_as_float(v[j]));
            }
          }
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, RT_TMEM_COLS);
  if (threadIdx.x == 0 && s_fail) atomicCAS(a.err, 0, (int)NYS_ERR_TIMEOUT);
}

template <int S, int P2>
int32_t h16_launch(const CUtensorMap& tx, const CUtensorMap& tv, const RtArgs& a0, int64_t npad,
                   int64_t nblk_y, int nz, float* part_ws, cudaStream_t s) {
  using Cfg = H16Cfg<S, P2>;
  auto kern = rbf_h16_kernel<S, P2>;
  NYS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
  RtArgs a = a0;
  if (nz > 1) {
    if (nz > kMaxSlices) return NYS_ERR_ARG;
    const int chunk = (int)cdiv(a.ntiles, nz);
    nz = (int)cdiv(a.ntiles, chunk);
    a.tile_chunk = chunk;
    a.part_stride = npad;
    a.ypart = part_ws;
  }
  kern<<<dim3((unsigned)(npad / RT_BM), (unsigned)nblk_y, (unsigned)nz), H_THREADS, Cfg::SMEM,
         s>>>(tx, tv, a);
  count_launch();
  if (a.ypart) {
    const unsigned gy = (unsigned)(a.nvec < 65535 ? a.nvec : 65535);
    rt_sum_kernel<<<dim3((unsigned)cdiv(a.n, 256), gy), 256, 0, s>>>(a.ypart, nz, a);
    count_launch();
  }
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// part_ws: room for kMaxSlices x nvec x npad partial sums (inside the work
// buffer, so that a product allocates nothing while a graph is captured)
template <int S, int P2>
int32_t rt_launch(const CUtensorMap& tx, const CUtensorMap& tv, const RtArgs& a0, int64_t npad,
                  int64_t nblk_y, int nz, float* part_ws, cudaStream_t s) {
  using Cfg = RtCfg<S, P2>;
  auto kern = rbf_tc_kernel<S, P2>;
  NYS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
  RtArgs a = a0;
  if (nz > 1) {
    if (nz > kMaxSlices) return NYS_ERR_ARG;
    const int chunk = (int)cdiv(a.ntiles, nz);
    nz = (int)cdiv(a.ntiles, chunk);
    a.tile_chunk = chunk;
    a.part_stride = npad;
    a.ypart = part_ws;
  }
  kern<<<dim3((unsigned)(npad / RT_BM), (unsigned)nblk_y, (unsigned)nz), RT_THREADS, Cfg::SMEM,
         s>>>(tx, tv, a);
  count_launch();
  if (a.ypart) {
    const unsigned gy = (unsigned)(a.nvec < 65535 ? a.nvec : 65535);
    rt_sum_kernel<<<dim3((unsigned)cdiv(a.n, 256), gy), 256, 0, s>>>(a.ypart, nz, a);
    count_launch();
  }
  NYS_CUDA_TRY(cudaGetLastError());
  return NYS_OK;
}

// One vector at a time (nvec <= 2), the points split into nz slices.
int32_t gv_run(const CUtensorMap& tx16, const RtArgs& a, const float* VS, const float* m2c_dev,
               int64_t npad, int64_t ntiles, int64_t d, int64_t nvec, int nz, float* part_ws,
               cudaStream_t s) {
  const int64_t ctas = npad / RT_BM;
  if (nz > kMaxSlices) return NYS_ERR_ARG;
  const int chunk = (int)cdiv(ntiles, nz);
  nz = (int)cdiv(ntiles, chunk);
  float* part = nz > 1 ? part_ws : nullptr;  // kMaxSlices x npad, reused vector by vector
  for (int64_t q = 0; q < nvec; ++q) {
    RtArgs aq = a;
    aq.vec = q;
    aq.vj = VS + q * npad;
    aq.ntiles = (int)ntiles;
    aq.ksteps = (int)cdiv(d, 16);
    aq.m2c_dev = m2c_dev;
    aq.tile_chunk = nz > 1 ? chunk : 0;
    aq.ypart = part;
    aq.part_stride = npad;
    rbf_gemv_kernel<<<dim3((unsigned)ctas, (unsigned)nz), GV_THREADS, GV_SMEM, s>>>(tx16, aq);
    count_launch();
    if (part) {
      gv_sum_kernel<<<(unsigned)cdiv(a.n, 256), 256, 0, s>>>(part, nz, npad, aq);
      count_launch();
    }
    NYS_CUDA_TRY(cudaGetLastError());
  }
  return NYS_OK;
}

// Slice counts worth timing.  One vector: 1..4 (the partial sums are a few
// n-vectors).  Many vectors: only while the grid is under 8 waves (beyond
// that the last wave costs little), each slice at least 4 tiles, and the
// partial sums (slices x nvec x npad floats) at most 256 MB.
std::vector<int> gv_slice_candidates(int64_t ntiles) {
  std::vector<int> c;
  for (int z = 1; z <= kMaxSlices; ++z)
    if (z == 1 || ntiles >= 2 * z) c.push_back(z);
  return c;
}

std::vector<int> rt_slice_candidates(int64_t npad, int64_t nvec, int64_t ctas, int64_t sms) {
  std::vector<int> c{1};
  if (ctas >= 8 * sms) return c;
  const int64_t ntiles = npad / RT_BN;
  for (int z = 2; z <= kMaxSlices; ++z)
    if (ntiles >= 4 * z && (double)z * nvec * npad * 4.0 <= 256.0 * (1 << 20)) c.push_back(z);
  return c;
}

// The untimed rule: the candidate whose last wave of CTAs (one per SM) is
// fullest, a smaller slice count unless a larger one fills 2 % more.
int wave_fill_rule(int64_t ctas, const std::vector<int>& cands, int64_t sms) {
  int pick = cands.empty() ? 1 : cands[0];
  double best = 0.0;
  for (int z : cands) {
    const double waves = (double)(ctas * z) / (double)sms;
    const double eff = waves / std::ceil(waves);
    if (eff > best + 0.02) {
      best = eff;
      pick = z;
    }
  }
  return pick;
}

std::string gv_tune_key(int64_t npad, int64_t d, int64_t nvec) {
  return "rbf_gemv npad=" + std::to_string(npad) + " d=" + std::to_string(d) +
         " nvec=" + std::to_string(nvec) + " sms=" + std::to_string(num_sms());
}

std::string rt_tune_key(int S, int passes, int64_t npad, int64_t d, int64_t nblk_y) {
  return "rbf_tc S=" + std::to_string(S) + " passes=" + std::to_string(passes) +
         " npad=" + std::to_string(npad) + " d=" + std::to_string(d) +
         " blocks=" + std::to_string(nblk_y) + " sms=" + std::to_string(num_sms());
}

std::string rt16_tune_key(int passes, int64_t npad, int64_t d, int64_t nvec) {
  return "rbf_tc16 passes=" + std::to_string(passes) + " npad=" + std::to_string(npad) +
         " d=" + std::to_string(d) + " nvec=" + std::to_string(nvec) +
         " sms=" + std::to_string(num_sms());
}

// Vectors per CTA of the 3xTF32 kernel: 1 (FP32 products on the exp warps)
// for one or two vectors, else 64 (three passes) or 128 (one pass).
int rt_block(int64_t nvec, int passes) {
  if (nvec <= 2) return 1;
  return passes == 3 ? 64 : 128;
}

// Many vectors on the FP16 kernel (the default; NYS_RBF_TF32=1 selects the
// 3xTF32 kernel).
bool rt_half() {
  static const bool h = [] {
    const char* e = getenv("NYS_RBF_TF32");
    return !(e && e[0] == '1' && e[1] == 0);
  }();
  return h;
}

// FP16 kernel shapes (vectors per CTA), tuned with the point-slice count:
// candidate = shape index * 8 + slices.  Three passes: 128, 64 or 32 vectors
// per CTA; one pass (the sketch): 128.
constexpr int kShapes3[3] = {128, 64, 32};
int rt16_nshapes(int passes) { return passes == 3 ? 3 : 1; }
int rt16_shape(int passes, int si) { return passes == 3 ? kShapes3[si] : 128; }

std::vector<int> rt16_candidates(int passes, int64_t npad, int64_t nvec, int64_t sms) {
  std::vector<int> c;
  for (int si = 0; si < rt16_nshapes(passes); ++si) {
    const int S = rt16_shape(passes, si);
    const int64_t ctas = (npad / RT_BM) * cdiv(nvec, S);
    for (int z : rt_slice_candidates(npad, nvec, ctas, sms)) c.push_back(si * 8 + z);
  }
  return c;
}

// The untimed rule: the narrowest shape that holds every vector in one CTA
// column (else the widest), with the fullest last wave of its slice counts.
int rt16_rule(int passes, int64_t npad, int64_t nvec, int64_t sms) {
  int si = 0;
  for (int k = rt16_nshapes(passes) - 1; k >= 0; --k)
    if (rt16_shape(passes, k) >= nvec) { si = k; break; }
  const int S = rt16_shape(passes, si);
  const int64_t ctas = (npad / RT_BM) * cdiv(nvec, S);
  const std::vector<int> z = rt_slice_candidates(npad, nvec, ctas, sms);
  return si * 8 + wave_fill_rule(ctas, z, sms);
}

}  // namespace

bool rbf_tc_supported(int64_t d) { return d >= 1 && d <= RT_DP; }

bool rbf_tc_tune_pending(int64_t n, int64_t d, int64_t nvec, int passes) {
  if (!tune_enabled() || !rbf_tc_supported(d) || n < 1 || nvec < 1) return false;
  const int64_t npad = cdiv(n, RT_BM) * RT_BM;
  const int S = rt_block(nvec, passes);
  if (S == 1) {
    const std::vector<int> c = gv_slice_candidates(npad / GV_BN);
    return c.size() > 1 && !tune_cached(gv_tune_key(npad, d, nvec), nullptr);
  }
  if (rt_half()) {
    const std::vector<int> c = rt16_candidates(passes, npad, nvec, num_sms());
    return c.size() > 1 && !tune_cached(rt16_tune_key(passes, npad, d, nvec), nullptr);
  }
  const int64_t nblk_y = cdiv(nvec, S);
  const std::vector<int> c = rt_slice_candidates(npad, nvec, (npad / RT_BM) * nblk_y, num_sms());
  return c.size() > 1 && !tune_cached(rt_tune_key(S, passes, npad, d, nblk_y), nullptr);
}

// Layout of the work buffer: [256: error word and one-vector scalars]
// [XS: npad x 64 FP32 (or FP16)] [cn: npad] [VS: the vectors' hi / lo
// copies] [partial sums of up to kMaxSlices point slices: kMaxSlices x
// (nvec or 1) x npad] [vscale: spad16] [amax: spad16].
static size_t rt_align(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t rt_vs_bytes(int64_t npad, int64_t nvec, int passes) {
  const int S = rt_block(nvec, passes);
  if (S == 1) return (size_t)nvec * npad * 4;
  const int nv = passes == 3 ? 2 : 1;
  const int64_t spad = cdiv(nvec, S) * S, spad16 = cdiv(nvec, 128) * 128;
  return std::max((size_t)nv * spad * npad * 4, (size_t)nv * spad16 * npad * 2);
}

size_t rbf_tc_work_bytes(int64_t n, int64_t nvec, int passes) {
  const int64_t npad = cdiv(n, RT_BM) * RT_BM;
  const int S = rt_block(nvec, passes);
  const int64_t spad16 = cdiv(nvec, 128) * 128;
  return 256 + rt_align((size_t)npad * 64 * 4) + rt_align((size_t)npad * 4) +
         rt_align(rt_vs_bytes(npad, nvec, passes)) +
         rt_align((size_t)kMaxSlices * (S == 1 ? 1 : nvec) * npad * 4) +
         2 * rt_align((size_t)spad16 * 4);
}

int32_t rbf_tc_products(const float* pts, int64_t n, int64_t d, int64_t ld, double sigma,
                        int64_t nvec, const float* V, int64_t ldv, int shift, const double* d_mu,
                        double mu0, float* Y, int64_t ldy, int passes, const int* done0,
                        int64_t done_stride, void* work, int* err, cudaStream_t s) {
  if (!rbf_tc_supported(d) || n < 1 || nvec < 1 || (passes != 1 && passes != 3)) return NYS_ERR_ARG;
  if (n > (1ll << 30) || (shift == 2 && !d_mu)) return NYS_ERR_ARG;
  const int64_t npad = cdiv(n, RT_BM) * RT_BM;
  const int S = rt_block(nvec, passes);
  const bool half = S > 1 && rt_half();
  const int64_t spad = half ? cdiv(nvec, 128) * 128 : cdiv(nvec, S) * S;
  const int nv = S == 1 ? 0 : (passes == 3 ? 2 : 1);
  if (spad * (nv ? nv : 1) > (1ll << 30)) return NYS_ERR_ARG;
  Scratch sc(s);
  unsigned char* w = (unsigned char*)work;
  if (!w) {
    NYS_TRY(sc.get(&w, rbf_tc_work_bytes(n, nvec, passes)));
    NYS_CUDA_TRY(cudaMemsetAsync(w, 0, 256, s));
  }
  if (!err) err = reinterpret_cast<int*>(w);
  float* XS = reinterpret_cast<float*>(w + 256);
  float* cn = reinterpret_cast<float*>(w + 256 + rt_align((size_t)npad * 64 * 4));
  float* VS = reinterpret_cast<float*>((unsigned char*)cn + rt_align((size_t)npad * 4));
  float* part_ws =
      reinterpret_cast<float*>((unsigned char*)VS + rt_align(rt_vs_bytes(npad, nvec, passes)));
  float* vscale = reinterpret_cast<float*>(
      (unsigned char*)part_ws + rt_align((size_t)kMaxSlices * (S == 1 ? 1 : nvec) * npad * 4));
  unsigned int* vamax = reinterpret_cast<unsigned int*>(
      (unsigned char*)vscale + rt_align((size_t)cdiv(nvec, 128) * 128 * 4));
  const double l2e = 1.4426950408889634;
  const double c = -l2e / (2.0 * sigma * sigma);
  unsigned int* absmax = reinterpret_cast<unsigned int*>(w + 64);
  float* m2c_dev = reinterpret_cast<float*>(w + 72);
  __half* XS16 = reinterpret_cast<__half*>(XS);
  if (S > 1 && !half) {
    rt_prep_points_kernel<<<(unsigned)cdiv(npad, 8), 256, 0, s>>>(pts, n, d, ld, npad, c, XS, cn);
    count_launch();
  } else {
    // FP16 split layout of the points (in the FP32 layout's space)
    NYS_CUDA_TRY(cudaMemsetAsync(absmax, 0, sizeof(unsigned int), s));
    const int64_t nd = n * d;
    rt_absmax_kernel<<<(unsigned)(cdiv(nd, 256) < 1024 ? cdiv(nd, 256) : 1024), 256, 0, s>>>(
        pts, n, d, ld, absmax);
    count_launch();
    rt_prep_points16_kernel<<<(unsigned)cdiv(npad, 8), 256, 0, s>>>(
        pts, n, d, ld, npad, c, l2e / (sigma * sigma), absmax, XS16, cn, m2c_dev);
    count_launch();
  }
  const int64_t tot = spad * npad;
  const unsigned gv = (unsigned)(cdiv(tot, 256) < 4096 ? cdiv(tot, 256) : 4096);
  if (half) {
    NYS_CUDA_TRY(cudaMemsetAsync(vamax, 0, (size_t)nvec * sizeof(unsigned int), s));
    const unsigned bx = (unsigned)std::min<int64_t>(cdiv(n, 4096), 16);
    rt_vec_absmax_kernel<<<dim3(bx, (unsigned)std::min<int64_t>(nvec, 65535)), 256, 0, s>>>(
        V, nvec, n, ldv, vamax);
    count_launch();
    rt_prep_vecs16_kernel<<<gv, 256, 0, s>>>(V, nvec, n, ldv, spad, npad, nv, vamax,
                                             reinterpret_cast<__half*>(VS), vscale);
  } else {
    rt_prep_vecs_kernel<<<gv, 256, 0, s>>>(V, nvec, n, ldv, spad, npad, nv, VS);
  }
  count_launch();
  RtArgs a;
  a.cn = cn;
  a.m2c = (float)(l2e / (sigma * sigma));
  a.m2c_dev = m2c_dev;
  a.n = n;
  a.ntiles = (int)(npad / RT_BN);
  a.ksteps = (int)cdiv(d, half ? 16 : 8);
  a.nvec = nvec;
  a.spad = spad;
  a.vec = 0;
  a.vj = VS;
  a.mus = shift == 2 ? d_mu : nullptr;
  a.mu0 = (float)mu0;
  a.v = shift ? V : nullptr;
  a.ldv = ldv;
  a.y = Y;
  a.ldy = ldy;
  a.done0 = done0;
  a.done_stride = done_stride;
  a.err = err;
  a.tile_chunk = 0;
  a.ypart = nullptr;
  a.part_stride = 0;
  a.vscale = half ? vscale : nullptr;
  const int64_t sms = num_sms();
  if (S == 1) {
    // one launch per vector (nvec <= 2), each reading its own padded copy
    CUtensorMap tx16;
    if (!tmap_f16_2d(&tx16, XS16, npad, 64, 64, 64, 64)) return NYS_ERR_CUDA;
    NYS_CUDA_TRY(
        cudaFuncSetAttribute(rbf_gemv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GV_SMEM));
    // One CTA per SM runs at a time; the points may be split into slices
    // (grid.y, fixed-order partial sums) so that the last wave of CTAs is
    // fuller.  The tuner times 1..4 slices; its fallback rule takes the
    // best last-wave fill.
    const int64_t ctas = npad / RT_BM, ntiles = npad / GV_BN;
    const std::vector<int> cands = gv_slice_candidates(ntiles);
    int nz = 1;
    NYS_TRY(tune_pick(gv_tune_key(npad, d, nvec), cands, wave_fill_rule(ctas, cands, sms),
                      [&](int z) -> int32_t {
                        return gv_run(tx16, a, VS, m2c_dev, npad, ntiles, d, nvec, z, part_ws,
                                      s);
                      },
                      s, &nz));
    return gv_run(tx16, a, VS, m2c_dev, npad, ntiles, d, nvec, nz, part_ws, s);
  }
  if (half) {
    CUtensorMap tx16;
    if (!tmap_f16_2d(&tx16, XS16, npad, 64, 64, 64, 64)) return NYS_ERR_CUDA;
    __half* VS16 = reinterpret_cast<__half*>(VS);
    auto run = [&](int code) -> int32_t {
      const int si = code / 8, z = code % 8;
      const int Sh = rt16_shape(passes, si);
      const int64_t nblk_y = cdiv(nvec, Sh);
      CUtensorMap tv16;
      if (!tmap_f16_2d(&tv16, VS16, nv * spad, npad, npad, Sh, 64)) return NYS_ERR_CUDA;
      if (passes == 1) return h16_launch<128, 1>(tx16, tv16, a, npad, nblk_y, z, part_ws, s);
      if (Sh == 128) return h16_launch<128, 3>(tx16, tv16, a, npad, nblk_y, z, part_ws, s);
      if (Sh == 64) return h16_launch<64, 3>(tx16, tv16, a, npad, nblk_y, z, part_ws, s);
      return h16_launch<32, 3>(tx16, tv16, a, npad, nblk_y, z, part_ws, s);
    };
    int code = 1;
    NYS_TRY(tune_pick(rt16_tune_key(passes, npad, d, nvec), rt16_candidates(passes, npad, nvec, sms),
                      rt16_rule(passes, npad, nvec, sms), run, s, &code));
    return run(code);
  }
  CUtensorMap tx, tv;
  if (!tmap_f32_2d(&tx, XS, npad, 64, 64, 64, 32)) return NYS_ERR_CUDA;
  if (!tmap_f32_2d(&tv, VS, nv * spad, npad, npad, S, 32)) return NYS_ERR_CUDA;
  // many vectors: point slices over grid.z where the grid is only a few waves
  const int64_t nblk_y = spad / S;
  const int64_t ctas = (npad / RT_BM) * nblk_y;
  const std::vector<int> cands = rt_slice_candidates(npad, nvec, ctas, sms);
  auto run = [&](int z) -> int32_t {
    return S == 64 ? rt_launch<64, 3>(tx, tv, a, npad, nblk_y, z, part_ws, s)
                   : rt_launch<128, 1>(tx, tv, a, npad, nblk_y, z, part_ws, s);
  };
  int nz = 1;
  NYS_TRY(tune_pick(rt_tune_key(S, passes, npad, d, nblk_y), cands,
                    wave_fill_rule(ctas, cands, sms), run, s, &nz));
  return run(nz);
}

}  // namespace nys
