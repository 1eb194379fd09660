// RandTucker2i refinement (Alg. 3): one pass of the loop body, every mode in
// order, each using the factors already refined in this pass:
//   X   = Y x_{p != n} U_p^T                       (Alg. 3 prints U_p: read U_p^T)
//   Z_n = X_(n) Omega_n,  Omega_n = KRP_{k != n} W_k^(n)   (W_k^(n): Rt_k x Rt_n)
//   U_n = orth(Z_n)                                  (CholQR2 in FP64)
// The contractions run on CUDA cores in the data's precision (FP64 or FP32),
// the shrinking tensor ping-ponging between two workspace buffers; the small
// sketch of X is one thread per entry of Z_n, accumulated in FP64.
#include <algorithm>

#include "tdk_internal.cuh"

namespace tdk {
namespace {

template <class T>
__global__ void cvt_factor(const double* __restrict__ s, T* __restrict__ d, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (T)s[e];
}

struct SmallSketch {
  int N, n;
  int64_t dim[TDK_MAX_MODES];     // dims of X (Rt_k for k != n, I_n at n)
  int64_t stride[TDK_MAX_MODES];  // row-major strides of X
  int Rn;                         // sketch width of mode n
  const double* W[TDK_MAX_MODES]; // W_k^(n) [dim_k x Rn] (k != n)
};

// Z[i, r] = sum over the other indices j of X[.., i, ..] prod_{k != n} W_k[j_k, r]
template <class T>
__global__ void small_sketch_kernel(const T* __restrict__ X, SmallSketch s, double* __restrict__ Z) {
  const int64_t In = s.dim[s.n];
  int64_t others = 1;
  for (int k = 0; k < s.N; ++k)
    if (k != s.n) others *= s.dim[k];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < In * s.Rn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / s.Rn;
    const int r = (int)(e % s.Rn);
    double acc = 0.0;
    for (int64_t j = 0; j < others; ++j) {
      int64_t rem = j, off = i * s.stride[s.n];
      double w = 1.0;
      for (int k = s.N - 1; k >= 0; --k) {
        if (k == s.n) continue;
        const int64_t jk = rem % s.dim[k];
        rem /= s.dim[k];
        off += jk * s.stride[k];
        w *= s.W[k][jk * s.Rn + r];
      }
      acc = fma((double)X[off], w, acc);
    }
    Z[e] = acc;
  }
}

inline unsigned grid_for(int64_t n, int per = 256) {
  const int64_t b = (n + per - 1) / per;
  return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

template <class T>
int refine_pass_t(tdk_ctx* ctx, const Geom& g, const T* Y, const double* const W[], double* const U_io[]) {
  const int N = g.N;
  // largest intermediate: the first contraction removes one full mode
  int64_t big = 0, Umax = 0;
  for (int p = 0; p < N; ++p) {
    big = std::max<int64_t>(big, g.numel / g.I[p] * g.Rt[p]);
    Umax += g.I[p] * g.Rt[p];
  }
  for (int n = 0; n < N; ++n) {
    // contraction order: the other modes from the last to the first
    int64_t dim[TDK_MAX_MODES];
    for (int k = 0; k < N; ++k) dim[k] = g.I[k];
    Planner pl;
    pl.take<T>((size_t)Umax);
    pl.take<T>((size_t)big);
    pl.take<T>((size_t)big);
    int rc = ws_reserve(ctx, pl.off);
    if (rc) return rc;
    Carver cv(ctx->ws);
    T* Ut[TDK_MAX_MODES];
    for (int p = 0; p < N; ++p) {
      Ut[p] = cv.take<T>((size_t)g.I[p] * g.Rt[p]);
      cvt_factor<T><<<grid_for(g.I[p] * g.Rt[p]), 256, 0, ctx->stream>>>(U_io[p], Ut[p], g.I[p] * g.Rt[p]);
      TDK_LAUNCH_CHECK(ctx);
    }
    T* buf[2] = {cv.take<T>((size_t)big), cv.take<T>((size_t)big)};
    const T* cur = Y;
    int pp = 0;
    for (int p = N - 1; p >= 0; --p) {
      if (p == n) continue;
      int64_t A = 1, Bd = 1;
      for (int k = 0; k < p; ++k) A *= dim[k];
      for (int k = p + 1; k < N; ++k) Bd *= dim[k];
      rc = launch_ttm_mid<T>(ctx, cur, A, dim[p], Bd, Ut[p], g.Rt[p], buf[pp], nullptr, 0);
      if (rc) return rc;
      dim[p] = g.Rt[p];
      cur = buf[pp];
      pp ^= 1;
    }
    // Z_n of the projected tensor, in its own allocation (CholQR2 carves the workspace)
    SmallSketch s{};
    s.N = N;
    s.n = n;
    s.Rn = g.Rt[n];
    int64_t st = 1;
    for (int k = N - 1; k >= 0; --k) {
      s.dim[k] = dim[k];
      s.stride[k] = st;
      st *= dim[k];
      s.W[k] = (k == n) ? nullptr : W[n * N + k];
    }
    double* Z = nullptr;
    if (cudaMallocAsync((void**)&Z, sizeof(double) * (size_t)g.I[n] * g.Rt[n], ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      return TDK_ENOMEM;
    }
    small_sketch_kernel<T><<<grid_for(g.I[n] * g.Rt[n], 128), 128, 0, ctx->stream>>>(cur, s, Z);
    rc = TDK_OK;
    if (cudaGetLastError() != cudaSuccess) rc = TDK_ECUDA;
    ctx->launches++;
    if (rc == TDK_OK) {
      Geom g1{};
      g1.N = 1;
      g1.I[0] = g.I[n];
      g1.Rt[0] = g.Rt[n];
      g1.numel = g.I[n];
      g1.M = 1;
      g1.L = g.I[n];
      g1.zoff[0] = 0;
      g1.zoff[1] = g.I[n] * g.Rt[n];
      g1.core_numel = g.Rt[n];
      double* dst[TDK_MAX_MODES] = {U_io[n]};
      rc = cholqr2(ctx, g1, Z, dst);
    }
    cudaFreeAsync(Z, ctx->stream);
    if (rc) return rc;
  }
  return TDK_OK;
}

}  // namespace

int refine_pass(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const W[],
                double* const U_io[]) {
  if (dtype == TDK_F64) return refine_pass_t<double>(ctx, g, reinterpret_cast<const double*>(Y), W, U_io);
  if (dtype == TDK_F32) return refine_pass_t<float>(ctx, g, reinterpret_cast<const float*>(Y), W, U_io);
  return TDK_ENOTSUP;
}

}  // namespace tdk
