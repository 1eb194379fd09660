// tcgen05 BF16 GEMM with FP32 accumulation for the learned initialiser's MLP
// (forward and backward products).  D[m, n] = sum_k A[m, k] B[n, k], where
// each operand is stored either K-major (row-major with k contiguous) or
// MN-major (row-major with m, resp. n, contiguous), so that every product of
// the forward and backward pass reads its operands in place:
//   forward       Z = X W^T          A K-major,  B K-major
//   input grad    dX = dZ W          A K-major,  B MN-major
//   weight grad   dW = dZ^T X        A MN-major, B MN-major
// One CTA computes one 128 x 128 output tile: warp 0 issues TMA loads of
// 64-deep K slices (128-byte swizzle, 4-stage ring), warp 1 issues the MMAs
// into a TMEM accumulator, warps 2-5 run the fused epilogue (bias, GELU,
// GELU derivative, BF16 / FP32 stores).  Every wait is bounded.
// A product with few output tiles and a long K (the forward layers and the
// input gradients at batch <= 128: 8-10 tiles) is split over K: CTA z of the
// grid's third dimension sums its range of K slices into an FP32 partial
// tile, and a finishing kernel adds the partials in a fixed order and applies
// the same epilogue, so the weight stream is spread over the whole GPU.
#include <algorithm>

#include "mlp_internal.cuh"
#include "tc_common.cuh"

namespace tdk {
namespace {

using namespace tc;

constexpr int TM = 128, TN = 128, TK = 64, STAGES = 4;
constexpr uint32_t OP_BYTES = 16 * 1024;  // one 128 x 64 BF16 operand slice
constexpr uint32_t STAGE_BYTES = 2 * OP_BYTES;
constexpr int THREADS = 192;

struct GemmArgs {
  int M, N, K;
  int a_mn, b_mn;
  int mode;
  int kper;      // K slices per CTA along the grid's third dimension
  float* part;   // split over K: FP32 partial tiles [gridDim.z][M][N]; null: the epilogue itself
  const float* bias;
  const float* zin;
  int ldz;
  float* outf;
  int ldf;
  __nv_bfloat16* outb;
  int ldb;
  unsigned* status;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// operand slice of one K step (16 deep) inside a staged 128 x 64 slice
__device__ __forceinline__ uint64_t op_desc(uint32_t base, int kk, int mn) {
  // K-major: rows are m (or n), 128 B of k per row; a K step moves 32 B.
  // MN-major: rows are k, 128 B of m per row in two 64-wide boxes 8 KB apart;
  // a K step moves 16 rows (2 KB).
  return mn ? smem_desc(base + kk * 2048, 8192, 1024, SW128) : smem_desc(base + kk * 32, 16, 1024, SW128);
}

__global__ void __launch_bounds__(THREADS, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* dfull = bars + 2 * STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  const int KCT = (a.K + TK - 1) / TK;
  const int kc_lo = blockIdx.z * a.kper;
  const int KC = KCT - kc_lo < a.kper ? KCT - kc_lo : a.kper;  // this CTA's slices
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(dfull), 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TN);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&tmA);
      prefetch_tmap(&tmB);
      for (int kc = 0; kc < KC; ++kc) {
        const int s = kc % STAGES;
        const uint32_t n = kc / STAGES;
        if (!mbar_wait(smem_u32(&empty[s]), (n & 1) ^ 1, a.status)) break;
        const uint32_t dst = smem_u32(base + s * STAGE_BYTES);
        const uint32_t bar = smem_u32(&full[s]);
        mbar_expect_tx(bar, STAGE_BYTES);
        const int k0 = (kc_lo + kc) * TK;
        if (a.a_mn) {
          tma_load_2d(dst, &tmA, m0, k0, bar);
          tma_load_2d(dst + 8192, &tmA, m0 + 64, k0, bar);
        } else {
          tma_load_2d(dst, &tmA, k0, m0, bar);
        }
        if (a.b_mn) {
          tma_load_2d(dst + OP_BYTES, &tmB, n0, k0, bar);
          tma_load_2d(dst + OP_BYTES + 8192, &tmB, n0 + 64, k0, bar);
        } else {
          tma_load_2d(dst + OP_BYTES, &tmB, k0, n0, bar);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = idesc_bf16(TM, TN, a.a_mn, a.b_mn);
      bool ok = true;
      for (int kc = 0; kc < KC; ++kc) {
        const int s = kc % STAGES;
        const uint32_t n = kc / STAGES;
        if (!mbar_wait(smem_u32(&full[s]), n & 1, a.status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = smem_u32(base + s * STAGE_BYTES);
        const uint32_t sb = sa + OP_BYTES;
#pragma unroll
        for (int kk = 0; kk < TK / 16; ++kk)
          mma_bf16(tmem, op_desc(sa, kk, a.a_mn), op_desc(sb, kk, a.b_mn), id, (kc | kk) != 0);
        umma_commit(smem_u32(&empty[s]));
      }
      if (ok) umma_commit(smem_u32(dfull));
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 * (w % 4) .. + 31 (one output row per thread)
    const int q = warp & 3;
    const int row = m0 + 32 * q + lane;
    if (mbar_wait(smem_u32(dfull), 0, a.status)) {
      tc_fence_after();
#pragma unroll 1
      for (int c16 = 0; c16 < TN / 16; ++c16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + c16 * 16, v);
        tmem_wait_ld();
        if (row >= a.M) continue;
        const int nb = n0 + c16 * 16;
        if (a.part) {  // split over K: the raw partial tile
          float* pr = a.part + ((int64_t)blockIdx.z * a.M + row) * a.N;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (nb + j < a.N) pr[nb + j] = v[j];
          continue;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = nb + j;
          if (col >= a.N) break;
          // a column past a leading dimension would land in the next row
          if (!TDK_IN(col, (a.mode == GEMM_GELU_GRAD) ? a.ldb : a.ldf)) break;
          if (a.mode == GEMM_BIAS_GELU && !TDK_IN(col, a.ldb)) break;
          float x = v[j];
          switch (a.mode) {
            case GEMM_STORE_F32:
              a.outf[(int64_t)row * a.ldf + col] = x;
              break;
            case GEMM_BIAS_GELU:
              x += a.bias[col];
              a.outf[(int64_t)row * a.ldf + col] = x;
              a.outb[(int64_t)row * a.ldb + col] = __float2bfloat16_rn(gelu_f(x));
              break;
            case GEMM_BIAS_F32:
              a.outf[(int64_t)row * a.ldf + col] = x + a.bias[col];
              break;
            case GEMM_GELU_GRAD:
              a.outb[(int64_t)row * a.ldb + col] =
                  __float2bfloat16_rn(x * gelu_grad_f(a.zin[(int64_t)row * a.ldz + col]));
              break;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TN);
  }
}

// sum of the K-split partials in a fixed order, then the epilogue of the mode
__global__ void splitk_finish_kernel(const float* __restrict__ part, int ks, GemmArgs a) {
  const int64_t MN = (int64_t)a.M * a.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN; e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / a.N), col = (int)(e % a.N);
    float x = 0.f;
    for (int z = 0; z < ks; ++z) x += part[z * MN + e];
    if (!TDK_IN(col, (a.mode == GEMM_GELU_GRAD) ? a.ldb : a.ldf)) continue;
    if (a.mode == GEMM_BIAS_GELU && !TDK_IN(col, a.ldb)) continue;
    switch (a.mode) {
      case GEMM_STORE_F32:
        a.outf[(int64_t)row * a.ldf + col] = x;
        break;
      case GEMM_BIAS_GELU:
        x += a.bias[col];
        a.outf[(int64_t)row * a.ldf + col] = x;
        a.outb[(int64_t)row * a.ldb + col] = __float2bfloat16_rn(gelu_f(x));
        break;
      case GEMM_BIAS_F32:
        a.outf[(int64_t)row * a.ldf + col] = x + a.bias[col];
        break;
      case GEMM_GELU_GRAD:
        a.outb[(int64_t)row * a.ldb + col] = __float2bfloat16_rn(x * gelu_grad_f(a.zin[(int64_t)row * a.ldz + col]));
        break;
    }
  }
}

int make_map(CUtensorMap* map, const __nv_bfloat16* p, int inner, int outer, int ld, int mn) {
  uint64_t dims[2] = {(uint64_t)inner, (uint64_t)outer};
  uint64_t str[1] = {(uint64_t)ld * 2};
  uint32_t box[2] = {64u, mn ? 64u : 128u};
  return encode_tmap(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p, dims, str, box, true);
}

}  // namespace

int gemm_bf16(tdk_ctx* ctx, const GemmOp& op) {
  if (op.M < 1 || op.N < 1 || op.K < 1) return TDK_EINVAL;
  if ((op.lda & 7) || (op.ldb & 7)) return TDK_EINVAL;  // 16-byte TMA row pitch
  if (((uintptr_t)op.A & 15) || ((uintptr_t)op.B & 15)) return TDK_EINVAL;
  CUtensorMap tmA, tmB;
  int rc = op.a_mn ? make_map(&tmA, op.A, op.M, op.K, op.lda, 1) : make_map(&tmA, op.A, op.K, op.M, op.lda, 0);
  if (rc) return rc;
  rc = op.b_mn ? make_map(&tmB, op.B, op.N, op.K, op.ldb, 1) : make_map(&tmB, op.B, op.K, op.N, op.ldb, 0);
  if (rc) return rc;
  GemmArgs a{};
  a.M = op.M;
  a.N = op.N;
  a.K = op.K;
  a.a_mn = op.a_mn;
  a.b_mn = op.b_mn;
  a.mode = op.mode;
  a.bias = op.bias;
  a.zin = op.zin;
  a.ldz = op.ldz;
  a.outf = op.outf;
  a.ldf = op.ldf;
  a.outb = op.outb;
  a.ldb = op.ldob;
  a.status = ctx->d_status;
  const size_t smem = 1024 + (size_t)STAGES * STAGE_BYTES + 8 * (2 * STAGES + 2);
  TDK_CUDA_TRY(cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int gx = (op.M + TM - 1) / TM, gy = (op.N + TN - 1) / TN;
  const int KC = (op.K + TK - 1) / TK;
  // split over K when the tiles leave most SMs idle: at least 4 slices per
  // CTA, about one CTA per SM in all
  const int tiles = gx * gy;
  int ks = 1;
  if (2 * tiles <= ctx->num_sms && KC >= 8) ks = std::min((ctx->num_sms + tiles - 1) / tiles, KC / 4);
  a.kper = (KC + ks - 1) / ks;
  ks = (KC + a.kper - 1) / a.kper;
  if (ks > 1) {
    const size_t pbytes = sizeof(float) * (size_t)ks * op.M * op.N;
    const int rc2 = ws_reserve(ctx, pbytes);
    if (rc2) return rc2;
    a.part = reinterpret_cast<float*>(ctx->ws);
  }
  gemm_bf16_kernel<<<dim3(gx, gy, ks), THREADS, smem, ctx->stream>>>(tmA, tmB, a);
  TDK_LAUNCH_CHECK(ctx);
  if (ks > 1) {
    const int64_t MN = (int64_t)op.M * op.N;
    splitk_finish_kernel<<<(unsigned)std::min<int64_t>((MN + 255) / 256, 2048), 256, 0, ctx->stream>>>(a.part, ks, a);
    TDK_LAUNCH_CHECK(ctx);
  }
  return TDK_OK;
}

}  // namespace tdk

#ifdef TDK_TESTING
// test library only: one GEMM through the library (operands and outputs caller-owned)
extern "C" int tdk_test_gemm_bf16(tdk_ctx* ctx, int M, int N, int K, const void* A, int lda, int a_mn,
                                  const void* B, int ldb, int b_mn, int mode, const float* bias,
                                  const float* zin, int ldz, float* outf, int ldf, void* outb, int ldob) {
  using namespace tdk;
  if (!ctx || !A || !B) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  GemmOp op{};
  op.M = M;
  op.N = N;
  op.K = K;
  op.A = static_cast<const __nv_bfloat16*>(A);
  op.lda = lda;
  op.a_mn = a_mn;
  op.B = static_cast<const __nv_bfloat16*>(B);
  op.ldb = ldb;
  op.b_mn = b_mn;
  op.mode = mode;
  op.bias = bias;
  op.zin = zin;
  op.ldz = ldz;
  op.outf = outf;
  op.ldf = ldf;
  op.outb = static_cast<__nv_bfloat16*>(outb);
  op.ldob = ldob;
  if ((mode == GEMM_STORE_F32 || mode == GEMM_BIAS_F32 || mode == GEMM_BIAS_GELU) && !outf) return TDK_EINVAL;
  if ((mode == GEMM_BIAS_GELU || mode == GEMM_GELU_GRAD) && !outb) return TDK_EINVAL;
  if ((mode == GEMM_BIAS_GELU || mode == GEMM_BIAS_F32) && !bias) return TDK_EINVAL;
  if (mode == GEMM_GELU_GRAD && !zin) return TDK_EINVAL;
  if (mode < 0 || mode > 3) return TDK_EINVAL;
  return gemm_bf16(ctx, op);
}
#endif  // TDK_TESTING

namespace tdk {
TDK_CHECKED_UNIT(mlp_gemm)
}  // namespace tdk
