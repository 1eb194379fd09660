// The two multi-pass compressions of Sec. IV-A.
//
// RandTucker2i (Alg. 3), one pass of its loop body, every mode in order and
// each using the factors already refined in this pass:
//   X   = Y x_{p != n} U_p^T                       (Alg. 3 prints U_p: read U_p^T)
//   Z_n = X_(n) Omega_n,  Omega_n = KRP_{k != n} W_k^(n)   (W_k^(n): Rt_k x Rt_n)
//   U_n = orth(Z_n)                                  (CholQR2 in FP64)
// Alg. 2 as printed (the sequential sketch), modes in order from X = Y:
//   Z_n = X_(n) Omega_n,  Omega_n = KRP_{k != n} W_k^(n)[0:d_k]
//   U_n = orth(Z_n),  X <- X x_n U_n^T                (mode n shrinks to Rt_n)
// with d_k the size of mode k at that point (Rt_k for k < n, I_k for k > n);
// the last X is the core.
//
// Both read the full tensor only through two kinds of pass: the core pass
// with mode 1 left open (Y x_{p >= 2} U_p^T; the fused tensor-core pass for
// BF16 data) and the leading-mode contraction Y x_1 U_1^T (tensor cores for
// BF16 data).  In a RandTucker2i pass the second one is shared by all modes
// n >= 2, which contract mode 1 with the U_1 refined at n = 1; so a pass reads
// Y twice whatever N is.  Everything after those passes works on tensors
// shrunk at least by I_1 / Rt_1: the contractions on CUDA cores, the sketches
// by the all-mode sketch of the shrunk tensor (its other modes are discarded).
#include <algorithm>

#include "tdk_internal.cuh"

namespace tdk {
namespace {

template <class T>
__global__ void cvt_factor(const double* __restrict__ s, T* __restrict__ d, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (T)s[e];
}

inline unsigned grid_for(int64_t n, int per = 256) {
  const int64_t b = (n + per - 1) / per;
  return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

// stream-ordered device buffer, freed on scope exit
struct DevBuf {
  tdk_ctx* ctx;
  void* p = nullptr;
  explicit DevBuf(tdk_ctx* c) : ctx(c) {}
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, ctx->stream);
  }
  int alloc(size_t bytes) {
    return pool_alloc(ctx, &p, bytes < 256 ? 256 : bytes);
  }
  template <class T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

// geometry of a partly contracted tensor with dims d and the sketch widths of g
Geom geom_of(const Geom& g, const int64_t* d) {
  Geom x{};
  x.N = g.N;
  x.numel = 1;
  x.core_numel = 1;
  x.zoff[0] = 0;
  for (int k = 0; k < g.N; ++k) {
    x.I[k] = d[k];
    x.Rt[k] = g.Rt[k];
    x.numel *= d[k];
    x.core_numel *= g.Rt[k];
    x.zoff[k + 1] = x.zoff[k] + d[k] * g.Rt[k];
  }
  x.L = d[g.N - 1];
  x.M = x.numel / x.L;
  return x;
}

// U_n = CholQR2 of Z_n (rows x cols, FP64)
int orth_one(tdk_ctx* ctx, const double* Z, int64_t rows, int cols, double* U) {
  Geom g1{};
  g1.N = 1;
  g1.I[0] = rows;
  g1.Rt[0] = cols;
  g1.numel = rows;
  g1.M = 1;
  g1.L = rows;
  g1.zoff[0] = 0;
  g1.zoff[1] = rows * cols;
  g1.core_numel = cols;
  double* const dst[TDK_MAX_MODES] = {U};
  return cholqr2(ctx, g1, Z, dst);
}

// Z_n of a (shrunk) tensor X in the compute type: the all-mode sketch of X
// (tensor-core form where it applies), mode n copied out, the rest dropped
template <class T>
int sketch_mode(tdk_ctx* ctx, const Geom& gx, int prec, const T* X, const double* const W[], int n, double* Zn) {
  const int dt = sizeof(T) == 8 ? TDK_F64 : TDK_F32;
  DevBuf Z(ctx);
  int rc = Z.alloc(sizeof(double) * (size_t)gx.zoff[gx.N]);
  if (rc) return rc;
  rc = TDK_ENOTSUP;
  if (prec == TDK_PREC_TC && dt == TDK_F32) rc = sketch_tc(ctx, gx, dt, X, W, Z.as<double>(), nullptr);
  if (rc == TDK_ENOTSUP) rc = sketch_simt(ctx, gx, dt, X, W, Z.as<double>());
  if (rc) return rc;
  TDK_CUDA_TRY(cudaMemcpyAsync(Zn, Z.as<double>() + gx.zoff[n], sizeof(double) * gx.I[n] * gx.Rt[n],
                               cudaMemcpyDeviceToDevice, ctx->stream));
  return TDK_OK;
}

// Xo = X x_p U_p^T for X with dims d (compute type); the contiguous mode by
// the row-tile kernel, the others by the slab kernel
template <class T>
int contract(tdk_ctx* ctx, const T* X, const int64_t* d, int N, int p, const T* Up, int Rtp, T* Xo,
             double* parts, int pgrid) {
  int64_t A = 1, Bd = 1;
  for (int k = 0; k < p; ++k) A *= d[k];
  for (int k = p + 1; k < N; ++k) Bd *= d[k];
  if (Bd == 1) {
    const int grid = (int)std::min<int64_t>(pgrid, (A + 63) / 64);
    return launch_ttm_last<T>(ctx, X, A, d[p], Up, Rtp, Xo, parts, grid);
  }
  return launch_ttm_mid<T>(ctx, X, A, d[p], Bd, Up, Rtp, Xo, nullptr, 0);
}

// W for the sketch of a shrunk tensor whose mode n is the one kept: the
// caller's W^(n); every other mode's matrices point at a zero block large
// enough for any of its factors (their sketches are discarded)
void w_for_mode(int N, int n, const double* const W[], const double* zero, const double** out) {
  for (int m = 0; m < N; ++m)
    for (int k = 0; k < N; ++k) out[m * N + k] = (k == m) ? nullptr : (m == n ? W[n * N + k] : zero);
}

template <class T>
int refine_pass_t(tdk_ctx* ctx, const Geom& g, int dtype, int prec, const void* Y, const double* const W[],
                  double* const U_io[]) {
  const int N = g.N;
  int64_t maxI = 0, maxRt = 0, Umax = 0;
  for (int p = 0; p < N; ++p) {
    maxI = std::max<int64_t>(maxI, g.I[p]);
    maxRt = std::max<int64_t>(maxRt, g.Rt[p]);
    Umax = std::max<int64_t>(Umax, g.I[p] * g.Rt[p]);
  }
  // Y x_{p >= 2} U_p^T (dims I_1, Rt_2, ...), Y x_1 U_1^T, and the largest
  // tensor shrunk from the latter for some mode n >= 2
  int64_t open0 = g.I[0];
  for (int p = 1; p < N; ++p) open0 *= g.Rt[p];
  const int64_t lead = g.numel / g.I[0] * g.Rt[0];
  int64_t shrunk = 1;
  for (int n = 1; n < N; ++n) {
    int64_t sz = lead;
    for (int p = N - 1; p >= 1; --p)
      if (p != n) {
        sz = sz / g.I[p] * g.Rt[p];
        shrunk = std::max<int64_t>(shrunk, sz);
      }
  }
  DevBuf Xs(ctx), Xl(ctx), Xa(ctx), Xb(ctx), Ut(ctx), Zn(ctx), zero(ctx), parts(ctx);
  int rc = Xs.alloc(sizeof(T) * (size_t)open0);
  if (!rc) rc = Xl.alloc(sizeof(T) * (size_t)lead);
  if (!rc) rc = Xa.alloc(sizeof(T) * (size_t)shrunk);
  if (!rc) rc = Xb.alloc(sizeof(T) * (size_t)shrunk);
  if (!rc) rc = Ut.alloc(sizeof(T) * (size_t)N * Umax);
  if (!rc) rc = Zn.alloc(sizeof(double) * (size_t)Umax);
  if (!rc) rc = zero.alloc(sizeof(double) * (size_t)maxI * maxRt);
  const int pgrid = 4 * ctx->num_sms;
  if (!rc) rc = parts.alloc(sizeof(double) * (size_t)pgrid);
  if (rc) return rc;
  TDK_CUDA_TRY(cudaMemsetAsync(zero.p, 0, sizeof(double) * (size_t)maxI * maxRt, ctx->stream));
  T* Uc[TDK_MAX_MODES];
  for (int p = 0; p < N; ++p) Uc[p] = Ut.as<T>() + (size_t)p * Umax;
  auto to_compute = [&](int p) -> int {
    cvt_factor<T><<<grid_for(g.I[p] * g.Rt[p]), 256, 0, ctx->stream>>>(U_io[p], Uc[p], g.I[p] * g.Rt[p]);
    TDK_LAUNCH_CHECK(ctx);
    return TDK_OK;
  };
  for (int p = 0; p < N; ++p)
    if ((rc = to_compute(p))) return rc;
  const double* wn[TDK_MAX_MODES * TDK_MAX_MODES];

  // n = 1: Y x_{p >= 2} U_p^T by the core pass with mode 1 open
  {
    rc = prec == TDK_PREC_TC ? core_tc(ctx, g, dtype, Y, U_io, Xs.p, nullptr, 1) : TDK_ENOTSUP;
    if (rc == TDK_ENOTSUP) rc = core_simt(ctx, g, dtype, Y, U_io, Xs.p, nullptr, 1);
    if (rc) return rc;
    int64_t d[TDK_MAX_MODES];
    for (int k = 0; k < N; ++k) d[k] = k == 0 ? g.I[0] : g.Rt[k];
    w_for_mode(N, 0, W, zero.as<double>(), wn);
    rc = sketch_mode<T>(ctx, geom_of(g, d), prec, Xs.as<T>(), wn, 0, Zn.as<double>());
    if (!rc) rc = orth_one(ctx, Zn.as<double>(), g.I[0], g.Rt[0], U_io[0]);
    if (!rc) rc = to_compute(0);
    if (rc) return rc;
  }
  // n >= 2: from Y x_1 U_1^T (the U_1 just refined), shared by all of them
  rc = ttm_lead(ctx, g, dtype, prec, Y, U_io[0], Xl.p);
  if (rc) return rc;
  for (int n = 1; n < N; ++n) {
    // contract the modes p != 0, n of the shared tensor, the last first
    int64_t d[TDK_MAX_MODES];
    for (int k = 0; k < N; ++k) d[k] = k == 0 ? g.Rt[0] : g.I[k];
    const T* cur = Xl.as<T>();
    T* bufs[2] = {Xa.as<T>(), Xb.as<T>()};
    int pp = 0;
    for (int p = N - 1; p >= 1; --p) {
      if (p == n) continue;
      rc = contract<T>(ctx, cur, d, N, p, Uc[p], g.Rt[p], bufs[pp], parts.as<double>(), pgrid);
      if (rc) return rc;
      d[p] = g.Rt[p];
      cur = bufs[pp];
      pp ^= 1;
    }
    w_for_mode(N, n, W, zero.as<double>(), wn);
    rc = sketch_mode<T>(ctx, geom_of(g, d), prec, cur, wn, n, Zn.as<double>());
    if (!rc) rc = orth_one(ctx, Zn.as<double>(), g.I[n], g.Rt[n], U_io[n]);
    if (!rc) rc = to_compute(n);
    if (rc) return rc;
  }
  return TDK_OK;
}

template <class T>
int seq_tucker_t(tdk_ctx* ctx, const Geom& g, int dtype, int prec, const void* Y, const double* const W[],
                 double* const U_out[], T* G, double* normY2) {
  const int N = g.N;
  int64_t Umax = 0;
  for (int p = 0; p < N; ++p) Umax = std::max<int64_t>(Umax, g.I[p] * g.Rt[p]);
  // Y x_1 U_1^T, and the same with mode 2 shrunk too (N >= 3; the core for N = 2)
  const int64_t lead = g.numel / g.I[0] * g.Rt[0];
  const int64_t second = N >= 3 ? lead / g.I[1] * g.Rt[1] : 1;
  DevBuf Xa(ctx), Xb(ctx), Uc(ctx), Zn(ctx), parts(ctx);
  int rc = Xa.alloc(sizeof(T) * (size_t)lead);
  if (!rc) rc = Xb.alloc(sizeof(T) * (size_t)second);
  if (!rc) rc = Uc.alloc(sizeof(T) * (size_t)Umax);
  if (!rc) rc = Zn.alloc(sizeof(double) * (size_t)Umax);
  const int pgrid = 4 * ctx->num_sms;
  if (!rc) rc = parts.alloc(sizeof(double) * (size_t)pgrid);
  if (rc) return rc;
  // mode 1 from Y: the sketch pass of Y (all modes, Z_1 kept) and ||Y||^2
  {
    DevBuf Z(ctx);
    rc = Z.alloc(sizeof(double) * (size_t)g.zoff[N]);
    if (rc) return rc;
    rc = (prec == TDK_PREC_TC && dtype != TDK_F64) ? sketch_tc(ctx, g, dtype, Y, W, Z.as<double>(), normY2)
                                                   : TDK_ENOTSUP;
    if (rc == TDK_ENOTSUP) {
      rc = sketch_simt(ctx, g, dtype, Y, W, Z.as<double>());
      if (!rc && normY2) rc = norm2_pass(ctx, g, dtype, Y, normY2);
    }
    if (!rc) rc = orth_one(ctx, Z.as<double>(), g.I[0], g.Rt[0], U_out[0]);
    if (rc) return rc;
  }
  rc = ttm_lead(ctx, g, dtype, prec, Y, U_out[0], Xa.p);
  if (rc) return rc;
  int64_t d[TDK_MAX_MODES];
  for (int k = 0; k < N; ++k) d[k] = k == 0 ? g.Rt[0] : g.I[k];
  T* cur = Xa.as<T>();
  T* nxt = Xb.as<T>();
  for (int n = 1; n < N; ++n) {
    // W_k^(n) has at least d_k rows (I_k >= Rt_k): the same arrays serve
    rc = sketch_mode<T>(ctx, geom_of(g, d), prec, cur, W, n, Zn.as<double>());
    if (!rc) rc = orth_one(ctx, Zn.as<double>(), g.I[n], g.Rt[n], U_out[n]);
    if (rc) return rc;
    cvt_factor<T><<<grid_for(g.I[n] * g.Rt[n]), 256, 0, ctx->stream>>>(U_out[n], Uc.as<T>(), g.I[n] * g.Rt[n]);
    TDK_LAUNCH_CHECK(ctx);
    T* out = (n == N - 1) ? G : nxt;
    rc = contract<T>(ctx, cur, d, N, n, Uc.as<T>(), g.Rt[n], out, parts.as<double>(), pgrid);
    if (rc) return rc;
    d[n] = g.Rt[n];
    nxt = cur;
    cur = out;
  }
  return TDK_OK;
}

}  // namespace

int ttm_lead(tdk_ctx* ctx, const Geom& g, int dtype, int prec, const void* Y, const double* U1, void* X) {
  if (dtype == TDK_BF16 && prec == TDK_PREC_TC) {
    const int rc = ttm_lead_tc(ctx, g, Y, U1, reinterpret_cast<float*>(X));
    if (rc != TDK_ENOTSUP) return rc;
  }
  const int64_t I0 = g.I[0], B = g.numel / I0;
  const int Rt = g.Rt[0];
  const size_t usz = (size_t)I0 * Rt;
  if (dtype == TDK_F64)
    return launch_ttm_mid<double>(ctx, reinterpret_cast<const double*>(Y), 1, I0, B, U1, Rt,
                                  reinterpret_cast<double*>(X), nullptr, 0);
  int rc = ws_reserve(ctx, usz * 4);
  if (rc) return rc;
  float* Uf = reinterpret_cast<float*>(ctx->ws);
  cvt_factor<float><<<grid_for((int64_t)usz), 256, 0, ctx->stream>>>(U1, Uf, (int64_t)usz);
  TDK_LAUNCH_CHECK(ctx);
  if (dtype == TDK_F32)
    return launch_ttm_mid<float>(ctx, reinterpret_cast<const float*>(Y), 1, I0, B, Uf, Rt,
                                 reinterpret_cast<float*>(X), nullptr, 0);
  return launch_ttm_mid_bf16(ctx, reinterpret_cast<const __nv_bfloat16*>(Y), 1, I0, B, Uf, Rt,
                             reinterpret_cast<float*>(X));
}

int refine_pass(tdk_ctx* ctx, const Geom& g, int dtype, int prec, const void* Y, const double* const W[],
                double* const U_io[]) {
  if (dtype == TDK_F64) return refine_pass_t<double>(ctx, g, dtype, prec, Y, W, U_io);
  return refine_pass_t<float>(ctx, g, dtype, prec, Y, W, U_io);
}

#ifdef TDK_TESTING
// test library only: the leading-mode contraction alone, X = Y x_1 U_1^T in
// the compute type (FP64 for FP64 data, else FP32), X [Rt_1 x numel / I_1]
extern "C" int tdk_test_ttm_lead(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* U1,
                                 void* X) {
  if (!ctx || !desc || !Y || !U1 || !X) return TDK_EINVAL;
  Geom g;
  const int rc = make_geom(desc, &g);
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  return ttm_lead(ctx, g, desc->dtype, desc->prec, Y, U1, X);
}
#endif

int seq_tucker(tdk_ctx* ctx, const Geom& g, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
               double* const U_out[], void* G_out, double* normY2) {
  if (desc->dtype == TDK_F64)
    return seq_tucker_t<double>(ctx, g, desc->dtype, desc->prec, Y, W, U_out, reinterpret_cast<double*>(G_out),
                                normY2);
  return seq_tucker_t<float>(ctx, g, desc->dtype, desc->prec, Y, W, U_out, reinterpret_cast<float*>(G_out), normY2);
}

}  // namespace tdk

namespace tdk {
TDK_CHECKED_UNIT(refine)
}  // namespace tdk
