// TF32 tensor-core GEMM for sm_103a (5th-generation tensor cores):
//   D[M x N] = A[M x K] . B[N x K]^T,   A and B FP32 row-major (K contiguous),
//   TF32 products, FP32 accumulation in tensor memory (TMEM).
//
// One CTA computes a 128 x BN output tile (BN = 256 or 128) over a K range
// (split-K along grid.z).  Four warps:
//   warp 0, lane 0 : TMA producer -- 2-D tiled bulk tensor copies of the A
//                    and B K-slabs (32 FP32 = 128 B wide, 128-byte swizzle)
//                    into a 4-stage shared-memory ring, completion counted
//                    on per-stage "full" mbarriers;
//   warp 1, lane 0 : MMA issuer -- four tcgen05.mma.kind::tf32 (K = 8 each)
//                    per slab into a 128 x BN FP32 accumulator in TMEM, then
//                    tcgen05.commit to the stage's "empty" mbarrier;
//   warp 2         : allocates / frees the TMEM columns;
//   all 4 warps    : epilogue -- tcgen05.ld of their 32 TMEM lanes, stores.
// Every mbarrier wait is bounded; on expiry the CTA records NYS_ERR_TIMEOUT,
// skips the epilogue, frees its TMEM and returns.
//
// Used for the sketch Y = X^T (X Omega) of the ridge operator (Algorithm 1,
// step 3), which is a genuinely dense contraction.

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "ptx.cuh"
#include "tmap.h"

namespace nys {

constexpr int TC_BM = 128;
constexpr int TC_BK = 32;  // FP32 elements per slab row = 128 bytes
constexpr int TC_STAGES = 4;

template <int BN>
struct TcCfg {
  static constexpr int A_BYTES = TC_BM * TC_BK * 4;
  static constexpr int B_BYTES = BN * TC_BK * 4;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM = 1024 + TC_STAGES * STAGE_BYTES + 256;
};

// ---------------------------------------------------------------- kernel

template <int BN>
__global__ void __launch_bounds__(128, 1)
tc_gemm_tn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  int M, int N, int64_t K, int64_t kchunk, float* __restrict__ D, int64_t ldd,
                  int64_t split_stride, int* err) {
  using Cfg = TcCfg<BN>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + TC_STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* done = empty + TC_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
  const int nkb = (kend > kbeg) ? (int)((kend - kbeg + TC_BK - 1) / TC_BK) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
    s_fail = 0;
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 2) tmem_alloc(tmem_slot, BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0 && nkb > 0) {
    // ---------------- TMA producer
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % TC_STAGES;
      if (kb >= TC_STAGES) {
        if (!mbar_wait_bounded(&empty[s], (uint32_t)(((kb / TC_STAGES) - 1) & 1))) {
          atomicOr(&s_fail, 1);
          break;
        }
      }
      unsigned char* st = sm + s * Cfg::STAGE_BYTES;
      const int kx = (int)(kbeg + (int64_t)kb * TC_BK);
      mbar_arrive_expect_tx(&full[s], (uint32_t)Cfg::STAGE_BYTES);
      tma_load_2d(st, &tmA, kx, m0, &full[s]);
      tma_load_2d(st + Cfg::A_BYTES, &tmB, kx, n0, &full[s]);
    }
  } else if (warp == 1 && lane == 0 && nkb > 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = tf32_idesc(TC_BM, BN);
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % TC_STAGES;
      if (!mbar_wait_bounded(&full[s], (uint32_t)((kb / TC_STAGES) & 1))) {
        atomicOr(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a_addr = smem_u32(sm + s * Cfg::STAGE_BYTES);
      const uint32_t b_addr = a_addr + Cfg::A_BYTES;
      const uint64_t adesc = sw128_kmajor_desc(a_addr);
      const uint64_t bdesc = sw128_kmajor_desc(b_addr);
#pragma unroll
      for (int k = 0; k < TC_BK / 8; ++k) {
        // advance 8 TF32 (32 bytes) along K inside the swizzled 128-byte rows
        mma_tf32(tmem, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), idesc,
                 (kb > 0 || k > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();

  // ---------------- epilogue
  bool ok = true;
  if (nkb > 0) ok = mbar_wait_bounded(done, 0u, 1ll << 26);
  if (!ok) atomicOr(&s_fail, 1);
  tc_fence_after();
  __syncthreads();
  float* Dz = D + (int64_t)blockIdx.z * split_stride;
  const int row = m0 + warp * 32 + lane;
  if (!s_fail) {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      if (nkb > 0) {
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = 0u;
      }
      if (row < M) {
        float* drow = Dz + (int64_t)row * ldd + n0 + c0;
        const int ncols = N - (n0 + c0);
        if (ncols >= 32 && ((((uintptr_t)drow) & 15u) == 0)) {
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4*>(drow + j) =
                make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                            __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < ncols) drow[j] = __uint_as_float(r[j]);
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicCAS(err, 0, (int)NYS_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tmem, BN);
}

// ---------------------------------------------------------------- host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool tmap_f32_2d(CUtensorMap* tm, const float* base, int64_t rows, int64_t cols, int64_t ld,
                 int box_rows, int box_cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstride,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tmap_f16_2d(CUtensorMap* tm, const void* base, int64_t rows, int64_t cols, int64_t ld,
                 int box_rows, int box_cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), gdim, gstride,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2-D FP32 tensor map over a row-major [rows x cols] array with row stride ld
// (elements); box = [box_rows x 32 cols], 128-byte swizzle, zero fill.
static bool make_map(CUtensorMap* tm, const float* base, int64_t rows, int64_t cols, int64_t ld,
                     int box_rows) {
  return tmap_f32_2d(tm, base, rows, cols, ld, box_rows, TC_BK);
}

bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                       const float* B, int64_t ldb) {
  if (M <= 0 || N <= 0 || K <= 0) return false;
  if (M > (1ll << 30) || N > (1ll << 30) || K > (1ll << 30)) return false;
  if (((uintptr_t)A & 15u) || ((uintptr_t)B & 15u)) return false;
  if ((lda * 4) % 16 || (ldb * 4) % 16) return false;
  if (lda < K || ldb < K) return false;
  return encode_fn() != nullptr;
}

template <int BN>
static int32_t tc_launch(int64_t M, int64_t N, int64_t K, const CUtensorMap& ta,
                         const CUtensorMap& tb, float* D, int64_t ldd, int* err, cudaStream_t s) {
  using Cfg = TcCfg<BN>;
  const int64_t mt = cdiv(M, TC_BM), nt = cdiv(N, BN);
  const int64_t tiles = mt * nt;
  const int64_t target = 2 * (int64_t)num_sms();
  int64_t splits = 1;
  const int64_t kblocks = cdiv(K, TC_BK);
  if (tiles < target) {
    splits = cdiv(target, tiles);
    int64_t max_splits = kblocks / 16;  // at least 16 slabs per split
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
  }
  int64_t kchunk = cdiv(kblocks, splits) * TC_BK;
  splits = cdiv(K, kchunk);
  auto kern = tc_gemm_tn_kernel<BN>;
  NYS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
  if (splits == 1) {
    kern<<<dim3((unsigned)mt, (unsigned)nt, 1), 128, Cfg::SMEM, s>>>(ta, tb, (int)M, (int)N, K,
                                                                      kchunk, D, ldd, 0, err); count_launch();
    NYS_CUDA_TRY(cudaGetLastError());
    return NYS_OK;
  }
  float* P = nullptr;
  NYS_TRY(dmalloc((void**)&P, (size_t)splits * M * N * sizeof(float), s));
  kern<<<dim3((unsigned)mt, (unsigned)nt, (unsigned)splits), 128, Cfg::SMEM, s>>>(
      ta, tb, (int)M, (int)N, K, kchunk, P, N, M * N, err); count_launch();
  cudaError_t e = cudaGetLastError();
  int32_t st = (e == cudaSuccess) ? split_reduce_f32(P, splits, M, N, D, ldd, s) : NYS_OK;
  dfree(P, s);
  NYS_CUDA_TRY(e);
  return st;
}

int32_t tc_gemm_tn_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                       const float* B, int64_t ldb, float* D, int64_t ldd, int* err,
                       cudaStream_t s) {
  if (!tc_gemm_supported(M, N, K, A, lda, B, ldb)) return NYS_ERR_ARG;
  const int bn = (N >= 256) ? 256 : 128;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, M, K, lda, TC_BM)) return NYS_ERR_CUDA;
  if (!make_map(&tb, B, N, K, ldb, bn)) return NYS_ERR_CUDA;
  if (bn == 256) return tc_launch<256>(M, N, K, ta, tb, D, ldd, err, s);
  return tc_launch<128>(M, N, K, ta, tb, D, ldd, err, s);
}

}  // namespace nys
