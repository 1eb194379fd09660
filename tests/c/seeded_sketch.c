/* A C caller of libtdk.so that knows only the problem statement (I_n, R_n,
 * p) and a seed: it fills a tensor, runs tucker_sketch with W = NULL so that
 * the library draws the test matrices from the seed, and writes the sketches
 * and bases to a file for the test to compare with the oracle.
 *
 *   seeded_sketch OUT I1 I2 I3 R1 R2 R3 P SEED
 *
 * Y[i1, i2, i3] = sin(0.37 i1 + 0.11 i2 * i3) + 0.01 (i1 - i2 + 2 i3) / I3
 * in FP32.  OUT receives, in order, Z_1, Z_2, Z_3 then U_1, U_2, U_3 (FP64,
 * row-major [I_n x (R_n + P)]).  Exit code 0 on success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "tdk.h"

#define CHECK_CUDA(x)                                                     \
  do {                                                                    \
    cudaError_t e_ = (x);                                                 \
    if (e_ != cudaSuccess) {                                              \
      fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));            \
      return 2;                                                           \
    }                                                                     \
  } while (0)

int main(int argc, char** argv) {
  if (argc != 10) {
    fprintf(stderr, "usage: %s OUT I1 I2 I3 R1 R2 R3 P SEED\n", argv[0]);
    return 1;
  }
  tdk_tucker_desc d = {0};
  d.N = 3;
  d.dtype = TDK_F32;
  d.prec = TDK_PREC_SIMT;
  for (int n = 0; n < 3; ++n) {
    d.I[n] = atoll(argv[2 + n]);
    d.R[n] = atoi(argv[5 + n]);
  }
  d.p = atoi(argv[8]);
  d.seed = strtoull(argv[9], NULL, 0);
  if (tdk_tucker_check(&d) != TDK_OK) {
    fprintf(stderr, "bad problem\n");
    return 1;
  }
  const int64_t I1 = d.I[0], I2 = d.I[1], I3 = d.I[2];
  const size_t numel = (size_t)(I1 * I2 * I3);
  float* h = (float*)malloc(sizeof(float) * numel);
  for (int64_t a = 0; a < I1; ++a)
    for (int64_t b = 0; b < I2; ++b)
      for (int64_t c = 0; c < I3; ++c)
        h[(a * I2 + b) * I3 + c] =
            (float)(sin(0.37 * (double)a + 0.11 * (double)(b * c)) + 0.01 * (double)(a - b + 2 * c) / (double)I3);
  tdk_ctx* ctx = NULL;
  int rc = tdk_ctx_create(&ctx, 0, NULL);
  if (rc) {
    fprintf(stderr, "tdk_ctx_create: %s\n", tdk_strerror(rc));
    return 3;
  }
  void* Y = NULL;
  CHECK_CUDA(cudaMalloc(&Y, sizeof(float) * numel));
  rc = tdk_copy_in(ctx, Y, h, sizeof(float) * numel);
  double* Z[3];
  double* U[3];
  size_t bytes[3];
  for (int n = 0; n < 3; ++n) {
    bytes[n] = sizeof(double) * (size_t)d.I[n] * (size_t)(d.R[n] + d.p);
    CHECK_CUDA(cudaMalloc((void**)&Z[n], bytes[n]));
    CHECK_CUDA(cudaMalloc((void**)&U[n], bytes[n]));
  }
  if (!rc) rc = tucker_sketch(ctx, &d, Y, NULL, U, Z, NULL);
  int flags = 0;
  if (!rc) rc = tdk_ctx_sync_status(ctx, &flags);
  if (rc || flags) {
    fprintf(stderr, "tucker_sketch: %s (status %d)\n", tdk_strerror(rc), flags);
    return 4;
  }
  FILE* f = fopen(argv[1], "wb");
  if (!f) return 5;
  for (int pass = 0; pass < 2; ++pass)
    for (int n = 0; n < 3; ++n) {
      double* buf = (double*)malloc(bytes[n]);
      rc = tdk_copy_out(ctx, buf, pass == 0 ? Z[n] : U[n], bytes[n]);
      if (rc || fwrite(buf, 1, bytes[n], f) != bytes[n]) return 6;
      free(buf);
    }
  fclose(f);
  for (int n = 0; n < 3; ++n) {
    cudaFree(Z[n]);
    cudaFree(U[n]);
  }
  cudaFree(Y);
  tdk_ctx_destroy(ctx);
  free(h);
  return 0;
}
