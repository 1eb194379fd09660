// Orthonormal basis of every sketch Z_n (Sec. IV-A, range-finder step 3;
// Alg. 2, the basis of each mode's sketch).  The paper's distributed variant
// (Eq. 23) forms the Gram sum_s Z_s^T Z_s from row blocks and whitens it;
// here the same row-block Gram feeds a Cholesky factor instead of an EVD
// (CholQR), applied twice (CholQR2) so that the result is orthonormal to
// working precision.  All arithmetic is FP64.
//
// Breakdown (a Cholesky pivot not above Rt * eps * max diag, i.e. Z_n
// numerically rank deficient, which happens for noise-free tensors of exact
// multilinear rank with p > 0): that mode is redone by two-pass classical
// Gram-Schmidt, and a column whose projected norm falls below 1e-12 of its
// original norm is replaced by a fixed pseudo-random vector, itself
// orthogonalised twice.  The status bit TDK_STATUS_RANKDEF is raised.
#include <algorithm>

#include "tdk_internal.cuh"

namespace tdk {
namespace {

constexpr int GRAM_ROWS = 64;

struct QRArgs {
  int N;
  int64_t I[TDK_MAX_MODES];
  int Rt[TDK_MAX_MODES];
  int64_t zoff[TDK_MAX_MODES + 1];
  int nchunk[TDK_MAX_MODES];
  int64_t gp_off[TDK_MAX_MODES];  // offset of mode n's Gram partials
};

// partial Grams of row chunks: gp[n][chunk][a*Rt+b] for a <= b
__global__ void gram_partial_kernel(const double* __restrict__ Z, QRArgs q, double* __restrict__ gp,
                                    const int* __restrict__ fail) {
  const int n = blockIdx.y;
  if (n >= q.N || (int)blockIdx.x >= q.nchunk[n]) return;
  if (fail && fail[n]) return;
  const int Rt = q.Rt[n];
  const int64_t I = q.I[n];
  const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS;
  const int rows = (int)((I - r0) < GRAM_ROWS ? (I - r0) : GRAM_ROWS);
  __shared__ double Zs[GRAM_ROWS * TDK_MAX_RANK];  // 32 KB
  const double* Zn = Z + q.zoff[n];
  for (int e = threadIdx.x; e < rows * Rt; e += blockDim.x)
    Zs[e] = TDK_IN(r0 * Rt + e, I * Rt) ? Zn[r0 * Rt + e] : 0.0;
  __syncthreads();
  double* out = gp + q.gp_off[n] + (int64_t)blockIdx.x * Rt * Rt;
  for (int e = threadIdx.x; e < Rt * Rt; e += blockDim.x) {
    int a = e / Rt, b = e % Rt;
    if (a > b) continue;
    double s = 0.0;
    for (int i = 0; i < rows; ++i) s = fma(Zs[i * Rt + a], Zs[i * Rt + b], s);
    out[e] = s;
  }
}

// Gram = sum of the chunk partials, in chunk order (grid: entries x modes)
__global__ void gram_reduce_kernel(QRArgs q, const double* __restrict__ gp, const int* __restrict__ fail,
                                   double* __restrict__ gram) {
  const int n = blockIdx.y;
  if (n >= q.N || fail[n]) return;
  const int Rt = q.Rt[n];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Rt * Rt) return;
  const int a = e / Rt, b = e % Rt;
  double s = 0.0;
  if (a <= b) {
    const double* g = gp + q.gp_off[n] + e;
    for (int c = 0; c < q.nchunk[n]; ++c) s += g[(int64_t)c * Rt * Rt];
  }
  gram[(int64_t)n * TDK_MAX_RANK * TDK_MAX_RANK + e] = s;
}

// Cholesky of the Gram (upper R, Gram = R^T R) -> Rinv; one CTA per mode.
// FP64 arithmetic is scarce on this GPU (about two FMAs per clock per SM) and
// slow to return, so each step spreads its update over all threads (one
// element each, no serial chains) and every FP64 value is computed once: the
// pivot reciprocal and breakdown test by the thread that finalises the pivot,
// the pivot row scaled once per step.
__global__ void chol_kernel(QRArgs q, const double* __restrict__ gram, double* __restrict__ rinv,
                            int* __restrict__ fail) {
  const int n = blockIdx.x;
  const int Rt = q.Rt[n];
  __shared__ double A[TDK_MAX_RANK * TDK_MAX_RANK];
  __shared__ double Ri[TDK_MAX_RANK * TDK_MAX_RANK];
  __shared__ double inv_d[TDK_MAX_RANK], srow[TDK_MAX_RANK], idsq[TDK_MAX_RANK];
  __shared__ double tiny_s;
  __shared__ int bad;
  if (fail[n]) return;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int e = tid; e < Rt * Rt; e += nth) A[e] = gram[(int64_t)n * TDK_MAX_RANK * TDK_MAX_RANK + e];
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int j = 0; j < Rt; ++j) mx = fmax(mx, A[j * Rt + j]);
    tiny_s = Rt * 2.220446049250313e-16 * mx;
    bad = !(A[0] > tiny_s);
    inv_d[0] = 1.0 / A[0];
  }
  // right-looking Cholesky on the upper triangle, A = L D L^T (L unit lower):
  // step j scales the pivot row once (srow = A[j, :] / d_j, the multipliers
  // L[:, j]) and updates the trailing triangle A[a, b] -= srow[a] A[j, b]
  // (j < a <= b), one element per thread.  The same row operations, applied
  // to M = I (M[a, c] -= srow[a] M[j, c] for a > j >= c, row j being final),
  // leave M = L^{-1} when the loop ends, so R^{-1} = M^T D^{-1/2} needs no
  // second pass of back substitution: one element per thread per step, no
  // serial chains.
  for (int e = tid; e < Rt * Rt; e += nth) Ri[e] = (e / Rt == e % Rt) ? 1.0 : 0.0;
  for (int j = 0; j < Rt; ++j) {
    __syncthreads();
    if (bad) break;
    const int m = Rt - j - 1;
    for (int a = j + 1 + tid; a < Rt; a += nth) srow[a] = A[j * Rt + a] * inv_d[j];
    __syncthreads();
    for (int e = tid; e < m * m; e += nth) {
      const int a = j + 1 + e / m, b = j + 1 + e % m;
      if (b < a) continue;
      const double v = fma(-srow[a], A[j * Rt + b], A[a * Rt + b]);
      A[a * Rt + b] = v;
      if (b == a && a == j + 1) {  // the next pivot is final now
        bad = !(v > tiny_s);
        inv_d[a] = 1.0 / v;
      }
    }
    const int w = j + 1;
    for (int e = tid; e < m * w; e += nth) {
      const int a = j + 1 + e / w, cidx = e % w;
      Ri[a * Rt + cidx] = fma(-srow[a], Ri[j * Rt + cidx], Ri[a * Rt + cidx]);
    }
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) fail[n] = 1;
    return;
  }
  for (int j = tid; j < Rt; j += nth) idsq[j] = 1.0 / sqrt(A[j * Rt + j]);
  __syncthreads();
  double* out = rinv + (int64_t)n * TDK_MAX_RANK * TDK_MAX_RANK;
  for (int e = tid; e < Rt * Rt; e += nth) {
    const int i = e / Rt, j = e % Rt;
    out[e] = i <= j ? Ri[j * Rt + i] * idsq[j] : 0.0;  // R^{-1}[i, j] = M[j, i] / sqrt(d_j)
  }
}

// Q = Z Rinv, row-wise; Qdst packed by zoff (dst_ptrs null) or per-mode pointers
struct Dst {
  double* p[TDK_MAX_MODES];
};
__global__ void apply_rinv_kernel(const double* __restrict__ Z, QRArgs q, const double* __restrict__ rinv,
                                  const int* __restrict__ fail, Dst dst) {
  const int n = blockIdx.y;
  if (n >= q.N || fail[n]) return;
  const int Rt = q.Rt[n];
  const int64_t I = q.I[n];
  __shared__ double Ri[TDK_MAX_RANK * TDK_MAX_RANK];
  const double* rn = rinv + (int64_t)n * TDK_MAX_RANK * TDK_MAX_RANK;
  for (int e = threadIdx.x; e < Rt * Rt; e += blockDim.x) Ri[e] = rn[e];
  __syncthreads();
  const double* Zn = Z + q.zoff[n];
  double* Qn = dst.p[n];
  // (row, column) by 32-bit division where the mode fits (64-bit division is
  // a long instruction sequence next to the dot product)
  const bool small = I * Rt < 0x7fffffffLL;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < I * Rt;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i;
    int b;
    if (small) {
      i = (int)e / Rt;
      b = (int)e - (int)i * Rt;
    } else {
      i = e / Rt;
      b = (int)(e % Rt);
    }
    double s = 0.0;
    for (int a = 0; a <= b; ++a) s = fma(Zn[i * Rt + a], Ri[a * Rt + b], s);
    if (TDK_IN(i * Rt + b, I * Rt)) Qn[e] = s;
  }
}

__device__ __forceinline__ double refill_value(int64_t i, int j) {
  // splitmix64 of (i, j) mapped to [-1, 1): a fixed pseudo-random direction
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)(j + 1) * 0xD1B54A32D192ED03ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// block reduction of `cnt` values held per thread in vals[] (cnt <= 64)
__device__ void block_sum(double* vals, int cnt, double* red /* [32][64] */, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = 0; c < cnt; ++c) {
    double v = warp_sum(vals[c]);
    if (lane == 0) red[w * TDK_MAX_RANK + c] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += red[q * TDK_MAX_RANK + c];
    out[c] = s;
  }
  __syncthreads();
}

// two-pass classical Gram-Schmidt with deterministic completion; one CTA per mode
__global__ void __launch_bounds__(256) cgs2_kernel(const double* __restrict__ Z, QRArgs q,
                                                   const int* __restrict__ fail, Dst dst,
                                                   unsigned* __restrict__ status) {
  const int n = blockIdx.x;
  if (!fail[n]) return;
  const int Rt = q.Rt[n];
  const int64_t I = q.I[n];
  const double* Zn = Z + q.zoff[n];
  double* Qn = dst.p[n];
  __shared__ double red[8 * TDK_MAX_RANK];
  __shared__ double coef[TDK_MAX_RANK];
  __shared__ double nrm[2];
  extern __shared__ double v[];  // [I]
  double part[TDK_MAX_RANK];
  for (int j = 0; j < Rt; ++j) {
    for (int64_t i = threadIdx.x; i < I; i += blockDim.x) v[i] = Zn[i * Rt + j];
    __syncthreads();
    for (int attempt = 0; attempt < 2; ++attempt) {
      // original norm
      double s = 0.0;
      for (int64_t i = threadIdx.x; i < I; i += blockDim.x) s = fma(v[i], v[i], s);
      part[0] = s;
      block_sum(part, 1, red, nrm);
      const double n0 = sqrt(nrm[0]);
      for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < j; ++c) part[c] = 0.0;
        for (int64_t i = threadIdx.x; i < I; i += blockDim.x)
          for (int c = 0; c < j; ++c) part[c] = fma(Qn[i * Rt + c], v[i], part[c]);
        block_sum(part, j, red, coef);
        for (int64_t i = threadIdx.x; i < I; i += blockDim.x) {
          double x = v[i];
          for (int c = 0; c < j; ++c) x = fma(-Qn[i * Rt + c], coef[c], x);
          v[i] = x;
        }
        __syncthreads();
      }
      s = 0.0;
      for (int64_t i = threadIdx.x; i < I; i += blockDim.x) s = fma(v[i], v[i], s);
      part[0] = s;
      block_sum(part, 1, red, nrm + 1);
      const double n1 = sqrt(nrm[1]);
      if (n1 > 1e-12 * n0 && n1 > 0.0) break;
      // dependent column: replace by a fixed pseudo-random vector and retry
      for (int64_t i = threadIdx.x; i < I; i += blockDim.x) v[i] = refill_value(i, j);
      __syncthreads();
    }
    const double inv = 1.0 / sqrt(nrm[1]);
    for (int64_t i = threadIdx.x; i < I; i += blockDim.x) Qn[i * Rt + j] = v[i] * inv;
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicOr(status, TDK_STATUS_RANKDEF);
}

// a failed Cholesky of a standalone Gram shows in the context's status word
__global__ void fail_to_status_kernel(const int* __restrict__ fail, unsigned* __restrict__ status) {
  if (threadIdx.x == 0 && fail[0]) atomicOr(status, TDK_STATUS_RANKDEF);
}

QRArgs one_matrix(int64_t rows, int cols) {
  QRArgs q{};
  q.N = 1;
  q.I[0] = rows;
  q.Rt[0] = cols;
  q.zoff[0] = 0;
  q.zoff[1] = rows * cols;
  q.nchunk[0] = (int)((rows + GRAM_ROWS - 1) / GRAM_ROWS);
  q.gp_off[0] = 0;
  return q;
}

}  // namespace

int gram_one(tdk_ctx* ctx, const double* Z, int64_t rows, int cols, double* gram_out) {
  const QRArgs q = one_matrix(rows, cols);
  Planner pl;
  pl.take<double>((size_t)q.nchunk[0] * cols * cols);
  pl.take<int>(TDK_MAX_MODES);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  double* gpart = cv.take<double>((size_t)q.nchunk[0] * cols * cols);
  int* fail = cv.take<int>(TDK_MAX_MODES);
  TDK_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int) * TDK_MAX_MODES, ctx->stream));
  gram_partial_kernel<<<dim3((unsigned)q.nchunk[0], 1), 256, 0, ctx->stream>>>(Z, q, gpart, fail);
  TDK_LAUNCH_CHECK(ctx);
  gram_reduce_kernel<<<dim3((unsigned)((cols * cols + 255) / 256), 1), 256, 0, ctx->stream>>>(q, gpart, fail,
                                                                                               gram_out);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

int orth_apply_one(tdk_ctx* ctx, const double* gram, const double* Z, int64_t rows, int cols, double* Q_out) {
  const QRArgs q = one_matrix(rows, cols);
  Planner pl;
  pl.take<double>((size_t)TDK_MAX_RANK * TDK_MAX_RANK);
  pl.take<int>(TDK_MAX_MODES);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  double* rinv = cv.take<double>((size_t)TDK_MAX_RANK * TDK_MAX_RANK);
  int* fail = cv.take<int>(TDK_MAX_MODES);
  TDK_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int) * TDK_MAX_MODES, ctx->stream));
  chol_kernel<<<1, 256, 0, ctx->stream>>>(q, gram, rinv, fail);
  TDK_LAUNCH_CHECK(ctx);
  Dst d{};
  d.p[0] = Q_out;
  apply_rinv_kernel<<<dim3((unsigned)std::max(1, 2 * ctx->num_sms), 1), 256, 0, ctx->stream>>>(Z, q, rinv, fail, d);
  TDK_LAUNCH_CHECK(ctx);
  fail_to_status_kernel<<<1, 32, 0, ctx->stream>>>(fail, ctx->d_status);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

int cholqr2(tdk_ctx* ctx, const Geom& g, const double* Z, double* const U_out[]) {
  QRArgs q{};
  q.N = g.N;
  int maxchunk = 0;
  int64_t gp = 0, Imax = 0;
  for (int n = 0; n < g.N; ++n) {
    q.I[n] = g.I[n];
    q.Rt[n] = g.Rt[n];
    q.nchunk[n] = (int)((g.I[n] + GRAM_ROWS - 1) / GRAM_ROWS);
    q.gp_off[n] = gp;
    gp += (int64_t)q.nchunk[n] * g.Rt[n] * g.Rt[n];
    if (q.nchunk[n] > maxchunk) maxchunk = q.nchunk[n];
    if (g.I[n] > Imax) Imax = g.I[n];
  }
  for (int n = 0; n <= g.N; ++n) q.zoff[n] = g.zoff[n];
  Planner pl;
  pl.take<double>(gp);
  pl.take<double>((size_t)g.N * TDK_MAX_RANK * TDK_MAX_RANK);
  pl.take<double>((size_t)g.N * TDK_MAX_RANK * TDK_MAX_RANK);
  pl.take<double>(g.zoff[g.N]);
  pl.take<int>(TDK_MAX_MODES);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  double* gpart = cv.take<double>(gp);
  double* rinv = cv.take<double>((size_t)g.N * TDK_MAX_RANK * TDK_MAX_RANK);
  double* gram = cv.take<double>((size_t)g.N * TDK_MAX_RANK * TDK_MAX_RANK);
  double* Q1 = cv.take<double>(g.zoff[g.N]);
  int* fail = cv.take<int>(TDK_MAX_MODES);
  TDK_CUDA_TRY(cudaMemsetAsync(fail, 0, sizeof(int) * TDK_MAX_MODES, ctx->stream));
  Dst d1{}, d2{};
  for (int n = 0; n < g.N; ++n) {
    d1.p[n] = Q1 + g.zoff[n];
    d2.p[n] = U_out[n];
  }
  const dim3 ggrid(maxchunk, g.N);
  // the products are FP64-bound (about one FP64 FMA per clock per SM): the
  // same number of CTAs per mode, a multiple of the SM count in all
  const dim3 agrid((unsigned)std::max(1, 2 * ctx->num_sms), g.N);
  // first pass: Z -> Q1
  const dim3 rgrid((TDK_MAX_RANK * TDK_MAX_RANK + 255) / 256, g.N);
  const int cblk = 256;
  gram_partial_kernel<<<ggrid, 256, 0, ctx->stream>>>(Z, q, gpart, fail);
  TDK_LAUNCH_CHECK(ctx);
  gram_reduce_kernel<<<rgrid, 256, 0, ctx->stream>>>(q, gpart, fail, gram);
  TDK_LAUNCH_CHECK(ctx);
  chol_kernel<<<g.N, cblk, 0, ctx->stream>>>(q, gram, rinv, fail);
  TDK_LAUNCH_CHECK(ctx);
  apply_rinv_kernel<<<agrid, 256, 0, ctx->stream>>>(Z, q, rinv, fail, d1);
  TDK_LAUNCH_CHECK(ctx);
  // second pass: Q1 -> U
  gram_partial_kernel<<<ggrid, 256, 0, ctx->stream>>>(Q1, q, gpart, fail);
  TDK_LAUNCH_CHECK(ctx);
  gram_reduce_kernel<<<rgrid, 256, 0, ctx->stream>>>(q, gpart, fail, gram);
  TDK_LAUNCH_CHECK(ctx);
  chol_kernel<<<g.N, cblk, 0, ctx->stream>>>(q, gram, rinv, fail);
  TDK_LAUNCH_CHECK(ctx);
  apply_rinv_kernel<<<agrid, 256, 0, ctx->stream>>>(Q1, q, rinv, fail, d2);
  TDK_LAUNCH_CHECK(ctx);
  // fallback for modes whose Cholesky broke down (no-op otherwise)
  size_t vsm = sizeof(double) * (size_t)Imax;
  if (vsm > 200 * 1024) return TDK_EINVAL;
  TDK_CUDA_TRY(cudaFuncSetAttribute(cgs2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));
  cgs2_kernel<<<g.N, 256, vsm, ctx->stream>>>(Z, q, fail, d2, ctx->d_status);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // namespace tdk

namespace tdk {
TDK_CHECKED_UNIT(cholqr)
}  // namespace tdk
