// Internal interface of the learned initialiser's kernels.
#pragma once

#include "tdk_internal.cuh"

namespace tdk {

// fused epilogues of gemm_bf16
enum {
  GEMM_STORE_F32 = 0,  // outf = D
  GEMM_BIAS_GELU = 1,  // outf = D + bias (pre-activation), outb = bf16(gelu(D + bias))
  GEMM_BIAS_F32 = 2,   // outf = D + bias
  GEMM_GELU_GRAD = 3   // outb = bf16(D * gelu'(zin))
};

// D[m, n] = sum_k A[m, k] B[n, k] in BF16 x BF16 -> FP32.
// a_mn = 0: A stored [M][lda] (k contiguous); a_mn = 1: A stored [K][lda]
// (m contiguous).  Likewise B with N.  Leading dimensions are multiples of
// 8 elements and the bases 16-byte aligned (TMA); elements outside M x K /
// N x K are never read.
struct GemmOp {
  int M, N, K;
  const __nv_bfloat16* A;
  int lda, a_mn;
  const __nv_bfloat16* B;
  int ldb, b_mn;
  int mode;
  const float* bias;
  const float* zin;
  int ldz;
  float* outf;
  int ldf;
  __nv_bfloat16* outb;
  int ldob;
};
int gemm_bf16(tdk_ctx* ctx, const GemmOp& op);

}  // namespace tdk
