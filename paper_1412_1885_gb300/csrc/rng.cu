// Seeded test matrices W_k^(n) of the all-mode sketch (Sec. IV-A draws a
// Gaussian test matrix; Sec. IV-B has the workers share the generator's seed
// rather than the matrices).  Every entry is a function of (seed, n, k, i, r)
// alone: one Philox4x32-10 block (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11) keyed by the seed, with the entry's
// indices as the counter; two 53-bit uniforms from its four words; one
// Box-Muller normal in FP64, rounded to the nearest BF16 value.  So any block
// of rows is drawn on its own with the same values, which is what a worker
// that owns a slab of mode 1 needs.
#include "tdk_internal.cuh"

namespace tdk {
namespace {

struct Philox4 {
  uint32_t v[4];
};

// Philox4x32 with 10 rounds: the round multiplies words 0 and 2 by the two
// round constants, swaps the halves and mixes in the key; the key is bumped
// by the Weyl constants between rounds
__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  return Philox4{{c0, c1, c2, c3}};
}

__device__ __forceinline__ double seeded_normal(uint64_t seed, int n, int k, int64_t i, int r) {
  const Philox4 x = philox4x32_10((uint32_t)r, (uint32_t)((uint64_t)i & 0xffffffffu), (uint32_t)((uint64_t)i >> 32),
                                  (uint32_t)(256 * n + k), (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  const uint64_t a = ((((uint64_t)x.v[0]) << 32) | x.v[1]) >> 11;
  const uint64_t b = ((((uint64_t)x.v[2]) << 32) | x.v[3]) >> 11;
  const double u1 = ((double)a + 0.5) * 0x1p-53;
  const double u2 = (double)b * 0x1p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// nearest BF16 value (8 significant bits, ties to even) of a finite FP64 value
// in BF16's normal range, as FP64: round the 52-bit fraction to its top 7
// bits on the bit pattern (a carry into the exponent is the correct result)
__device__ __forceinline__ double round_to_bf16(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long drop = 45;
  const unsigned long long half = (1ull << (drop - 1)) - 1ull + ((b >> drop) & 1ull);
  return __longlong_as_double((long long)((b + half) & ~((1ull << drop) - 1ull)));
}

struct DrawJob {
  double* out[TDK_MAX_MODES * TDK_MAX_MODES];  // [n*N + k] or null
  int64_t rows[TDK_MAX_MODES * TDK_MAX_MODES];
  int64_t row0[TDK_MAX_MODES * TDK_MAX_MODES];  // global index of the first row
  int cols[TDK_MAX_MODES * TDK_MAX_MODES];
  int N;
};

// grid.y = matrix (n*N + k); grid-stride over its entries
__global__ void draw_w_kernel(DrawJob j, uint64_t seed) {
  const int m = blockIdx.y;
  double* out = j.out[m];
  if (!out) return;
  const int n = m / j.N, k = m % j.N;
  const int cols = j.cols[m];
  const int64_t total = j.rows[m] * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols;
    const int r = (int)(e - i * cols);
    out[e] = round_to_bf16(seeded_normal(seed, n, k, j.row0[m] + i, r));
  }
}

}  // namespace

// W_out[n*N + k] (k != n, non-null) <- rows [row0_k, row0_k + rows_k) of the
// seeded W_k^(n), rows_k x Rt_n; rows and row0 per mode k
int draw_sketch_matrices(tdk_ctx* ctx, int N, const int64_t* rows, const int64_t* row0, const int* Rt,
                         uint64_t seed, double* const W_out[]) {
  DrawJob j{};
  j.N = N;
  int64_t biggest = 0;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) {
      const int m = n * N + k;
      if (k == n) continue;
      j.out[m] = W_out[m];
      j.rows[m] = rows[k];
      j.row0[m] = row0[k];
      j.cols[m] = Rt[n];
      if (W_out[m] && rows[k] * Rt[n] > biggest) biggest = rows[k] * Rt[n];
    }
  if (biggest == 0) return TDK_OK;
  const int blocks = (int)std::min<int64_t>((biggest + 255) / 256, 4 * (int64_t)ctx->num_sms);
  draw_w_kernel<<<dim3((unsigned)blocks, (unsigned)(N * N)), 256, 0, ctx->stream>>>(j, seed);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // namespace tdk

using namespace tdk;

extern "C" int tdk_sketch_matrices(tdk_ctx* ctx, const tdk_tucker_desc* desc, double* const W_out[]) {
  if (!ctx || !desc || !W_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n)
    for (int k = 0; k < g.N; ++k)
      if (k != n && !W_out[n * g.N + k]) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  int64_t rows[TDK_MAX_MODES], row0[TDK_MAX_MODES] = {};
  for (int n = 0; n < g.N; ++n) rows[n] = g.I[n];
  return draw_sketch_matrices(ctx, g.N, rows, row0, g.Rt, desc->seed, W_out);
}

namespace tdk {
TDK_CHECKED_UNIT(rng)
}  // namespace tdk
