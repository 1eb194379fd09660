// Internal declarations shared by the translation units of libtdk.so.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <vector>

#include "../../include/tdk.h"

#define TDK_STATUS_RANKDEF 1u
#define TDK_STATUS_TIMEOUT 256u
#define TDK_STATUS_OOB 512u  // checked build: a bounds check failed

// ---- bounds checks of the checked build ----------------------------------
// The test library is compiled with -DTDK_CHECKED.  TDK_IN(i, n) tests
// 0 <= i < n; a failure sets this translation unit's check word (and keeps
// the first failing source line) instead of faulting, and the caller skips
// the access.  tdk_ctx_sync_status collects the words of every unit into
// TDK_STATUS_OOB.  The product build compiles every check to `true`.
#ifdef TDK_CHECKED
namespace tdk_chk {
namespace {
__device__ unsigned word_;
__device__ unsigned line_;
__device__ __forceinline__ bool in_range(long long i, long long n, unsigned ln) {
  if (i >= 0 && i < n) return true;
  atomicOr(&word_, 1u);
  atomicCAS(&line_, 0u, ln);
  return false;
}
// host: this unit's word and first failing line, read and cleared on a stream
inline int take(cudaStream_t s, unsigned* w, unsigned* l) {
  unsigned v[2] = {0u, 0u};
  const unsigned z = 0u;
  if (cudaMemcpyFromSymbolAsync(&v[0], word_, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyFromSymbolAsync(&v[1], line_, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(word_, &z, sizeof(unsigned), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(line_, &z, sizeof(unsigned), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  *w = v[0];
  *l = v[1];
  return 0;
}
}  // namespace
}  // namespace tdk_chk
#define TDK_IN(i, n) tdk_chk::in_range((long long)(i), (long long)(n), (unsigned)__LINE__)
#define TDK_CHECKED_UNIT(name) \
  int tdk_chk_take_##name(cudaStream_t s, unsigned* w, unsigned* l) { return tdk_chk::take(s, w, l); }
#else
#define TDK_IN(i, n) true
#define TDK_CHECKED_UNIT(name)
#endif

// Host-side time marks of the test library: with TDK_HOST_MARKS set, each
// TDK_HMARK("name") prints the microseconds since the previous mark of the
// thread (where the host time of a call goes).  Nothing in other builds.
#ifdef TDK_TESTING
#include <chrono>
#include <cstdlib>
namespace tdk_chk {
inline void hmark(const char* name) {
  static const bool on = getenv("TDK_HOST_MARKS") != nullptr;
  if (!on) return;
  static thread_local std::chrono::steady_clock::time_point last = std::chrono::steady_clock::now();
  const auto now = std::chrono::steady_clock::now();
  fprintf(stderr, "tdk host: %s +%.1f us\n", name, std::chrono::duration<double, std::micro>(now - last).count());
  last = now;
}
}  // namespace tdk_chk
#define TDK_HMARK(name) tdk_chk::hmark(name)
#else
#define TDK_HMARK(name) ((void)0)
#endif

struct tdk_ctx {
  int device = 0;
  int num_sms = 0;
  int max_smem_optin = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;     // private non-blocking stream (graph capture)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  void* ws = nullptr;          // growable workspace
  size_t ws_size = 0;
  cudaMemPool_t pool = nullptr;  // the context's stream-ordered pool (keeps its memory between calls)
  unsigned* d_status = nullptr;  // device status word (TDK_STATUS_* bits)
  int64_t launches = 0;
  int fail_alloc_after = -1;   // set only by the test library's hook: fail the n-th workspace growth
  // event timing of the main kernels (regions 0: sketch pass, 1: core pass)
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev[2];
  double prof_ms[2] = {0.0, 0.0};
  int64_t prof_n[2] = {0, 0};
};

namespace tdk {

// record an event pair around the main kernel of a region (when profiling)
struct ProfScope {
  tdk_ctx* c;
  int region;
  cudaEvent_t e1 = nullptr;
  ProfScope(tdk_ctx* ctx, int r) : c(ctx), region(r) {
    if (!c->prof) return;
    cudaEvent_t e0;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    c->prof_ev[region].push_back(e0);
  }
  ~ProfScope() {
    if (!c->prof || !e1) return;
    cudaEventRecord(e1, c->stream);
    c->prof_ev[region].push_back(e1);
  }
};

// ---- host helpers -------------------------------------------------------
int ws_reserve(tdk_ctx* ctx, size_t bytes);
// stream-ordered allocation from the context's pool (freed with cudaFreeAsync)
int pool_alloc(tdk_ctx* ctx, void** p, size_t bytes);

struct Carver {  // carves 256-byte-aligned slices out of the workspace
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};
// size of a carve plan (same alignment rule)
struct Planner {
  size_t off = 0;
  template <class T>
  void take(size_t count) {
    off = (off + 255) & ~size_t(255);
    off += count * sizeof(T);
  }
};

#define TDK_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t e__ = (expr);                                                \
    if (e__ != cudaSuccess) {                                                \
      fprintf(stderr, "tdk: %s failed: %s (%s:%d)\n", #expr,                 \
              cudaGetErrorString(e__), __FILE__, __LINE__);                  \
      return TDK_ECUDA;                                                      \
    }                                                                        \
  } while (0)

#define TDK_LAUNCH_CHECK(ctx)                                                \
  do {                                                                       \
    (ctx)->launches++;                                                       \
    cudaError_t e__ = cudaGetLastError();                                    \
    if (e__ != cudaSuccess) {                                                \
      fprintf(stderr, "tdk: launch failed: %s (%s:%d)\n",                    \
              cudaGetErrorString(e__), __FILE__, __LINE__);                  \
      return TDK_ECUDA;                                                      \
    }                                                                        \
  } while (0)

// problem geometry derived from a descriptor
struct Geom {
  int N;
  int64_t I[TDK_MAX_MODES];
  int Rt[TDK_MAX_MODES];
  int64_t numel;
  int64_t M;      // rows of the last-mode unfolding: prod_{k<N-1} I_k
  int64_t L;      // I_{N-1} (contiguous mode)
  int64_t zoff[TDK_MAX_MODES + 1];  // offsets of Z_n in a packed buffer
  int64_t core_numel;
};
int make_geom(const tdk_tucker_desc* d, Geom* g);

// elements of the buffer for the partial outputs of split contractions in
// the core chain: eight copies of the largest contraction output that can
// be split (the core itself bounds the last ones)
inline int64_t chain_split_cap(const Geom& g) { return 8 * g.core_numel; }

// ---- entry points of the translation units --------------------------------
// sketch (SIMT): writes FP64 Z_n for all modes into Zdst (packed by zoff)
int sketch_simt(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const W[],
                double* Zdst);
// tensor-core sketch; returns TDK_ENOTSUP when the form does not apply.
// normY2 (null or an FP64 device scalar) receives ||Y||^2, summed while the
// tiles are staged where the form allows it, else by norm2_pass
int sketch_tc(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const W[],
              double* Zdst, double* normY2);
// ||Y||^2 by one streaming pass over Y (fixed-order sums)
int norm2_pass(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, double* normY2);
// CholQR2 of every Z_n (packed FP64) into U_out
int cholqr2(tdk_ctx* ctx, const Geom& g, const double* Z, double* const U_out[]);
// one matrix Z [rows x cols]: upper triangle of Z^T Z; Q = Z R^-1 from a Gram
int gram_one(tdk_ctx* ctx, const double* Z, int64_t rows, int cols, double* gram_out);
int orth_apply_one(tdk_ctx* ctx, const double* gram, const double* Z, int64_t rows, int cols, double* Q_out);
// seeded test matrices: W_out[n*N + k] <- rows [row0_k, row0_k + rows_k) of W_k^(n)
int draw_sketch_matrices(tdk_ctx* ctx, int N, const int64_t* rows, const int64_t* row0, const int* Rt,
                         uint64_t seed, double* const W_out[]);
// core: G (T) and ||Y||^2 (FP64 device scalar, may be null).  open0 = 1
// leaves mode 0 uncontracted: G receives Y x_2 U_2^T ... x_N U_N^T with dims
// (I_1, Rt_2, ..., Rt_N), and U[0] is not read
int core_simt(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const U[],
              void* G, double* normY2, int open0 = 0);
int core_tc(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const U[],
            void* G, double* normY2, int open0 = 0);
// the leading mode contracted: X[r, b] = sum_i U_1[i, r] Y[i, b], Y read as
// [I_1][B] with B = numel / I_1, X in the compute type (FP64 for FP64 data,
// FP32 otherwise); the tensor-core form for BF16 data when prec is TC and
// the shape allows it, else CUDA cores
int ttm_lead(tdk_ctx* ctx, const Geom& g, int dtype, int prec, const void* Y, const double* U1, void* X);
// tensor-core form of ttm_lead (BF16 data); TDK_ENOTSUP when it does not apply
int ttm_lead_tc(tdk_ctx* ctx, const Geom& g, const void* Y, const double* U1, float* X);
// one refinement pass of RandTucker2i
int refine_pass(tdk_ctx* ctx, const Geom& g, int dtype, int prec, const void* Y, const double* const W[],
                double* const U_io[]);
// Alg. 2 in its printed order (the sequential sketch)
int seq_tucker(tdk_ctx* ctx, const Geom& g, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
               double* const U_out[], void* G_out, double* normY2);
// X_out[a, r, b] = sum_i U[i, r] X[a, i, b] (T = float or double), with an
// optional buffer for split partial outputs (nullptr = no split)
template <class T>
int launch_ttm_mid(tdk_ctx* ctx, const T* X, int64_t A, int64_t Ic, int64_t Bd, const T* U, int Rt, T* Xo,
                   T* part, int64_t part_cap);
// the same with BF16 X and FP32 U and output (no split)
int launch_ttm_mid_bf16(tdk_ctx* ctx, const __nv_bfloat16* X, int64_t A, int64_t Ic, int64_t Bd, const float* U,
                        int Rt, float* Xo);
// Xo[row, r] = sum_col X[row, col] U[col, r] (the contiguous mode); parts
// receives grid FP64 partial sums of X's squares
template <class T>
int launch_ttm_last(tdk_ctx* ctx, const T* X, int64_t M, int64_t L, const T* U, int Rt, T* Xo, double* parts,
                    int grid);
int als_run(tdk_ctx* ctx, const Geom& g, int dtype, const void* G, const double* const U[],
            const double* normY2, const tdk_als_opts* o, double* const B_io[],
            double* const A_io[], double* lambda_out, tdk_als_report* rep);

}  // namespace tdk

// ---- device helpers -----------------------------------------------------------
template <class T>
__device__ __forceinline__ T tdk_load(const T* p) { return *p; }

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ double to_f(double x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

template <class T>
struct CvtIn {  // storage -> compute type
  template <class S>
  __device__ __forceinline__ static T cvt(S x) { return (T)to_f(x); }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
