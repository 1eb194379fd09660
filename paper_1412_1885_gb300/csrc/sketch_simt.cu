// All-mode randomized sketch on CUDA cores (the plain form), and the first
// contraction of the core chain in the same form.
//
// Sketch (Sec. IV-A step 2, Alg. 2, Eq. 22): for every mode n
//   Z_n[i_n, r] = sum_{i != i_n} y[i] * prod_{k != n} W_k^(n)[i_k, r].
// Y is viewed as M rows x L columns (row = (i_1..i_{N-1}), column = i_N, the
// contiguous mode).  One pass over Y computes, per row tile:
//   P[row, c]  = sum_col Y[row, col] * WN[col, c]   for the channels c of
//                every mode n < N (WN = [W_N^(1) | ... | W_N^(N-1)]), then
//                Z_n[i_n(row), r] += P[row, c] * prod_{k<N, k != n} W_k^(n)[i_k, r];
//   Z_N[col, r] += sum_row Y[row, col] * K[row, r],  K = KRP_{k<N} W_k^(N).
// Partial sums live per CTA (the CTA-level blocks play the role of the
// paper's sub-tensor workers, Eq. 22) and are reduced in a fixed order in
// FP64, so results are bitwise reproducible.
#include "tdk_internal.cuh"

namespace tdk {
namespace {

constexpr int BM = 64;   // rows per tile
constexpr int BL = 32;   // columns per chunk
constexpr int NT = 256;  // threads per CTA

struct SketchArgs {
  int N;
  int64_t I[TDK_MAX_MODES];
  int Rt[TDK_MAX_MODES];
  int64_t M, L;
  int C1, C1p;                   // channels of modes < N (padded to 16*TC)
  int off[TDK_MAX_MODES];        // channel offset of mode n (n < N-1)
  int RtL, RtLp;                 // sketch width of the last mode (padded to 8)
  int64_t zoff[TDK_MAX_MODES + 1];
  int64_t ztot;
  int64_t ntiles;
  int zlast_smem;                // 1: mode-N partial held in shared memory
  const void* WN;                // [L x C1] compute type
  const void* Wk[TDK_MAX_MODES][TDK_MAX_MODES];  // [n][k] : [I_k x Rt_n]
  void* part;                    // [gridDim.x][ztot] compute type
};

template <class T>
__device__ __forceinline__ void decode_row(int64_t row, const SketchArgs& a, int* idx) {
  // row-major over modes 0..N-2
  for (int k = a.N - 2; k >= 0; --k) {
    idx[k] = (int)(row % a.I[k]);
    row /= a.I[k];
  }
}

template <class TY, class T, int TC>
__global__ void __launch_bounds__(NT) sketch_simt_kernel(const TY* __restrict__ Y, SketchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ys = reinterpret_cast<T*>(smem_raw);                 // [BM][BL+1]
  T* WNs = Ys + BM * (BL + 1);                              // [BL][C1p]
  T* Ks = WNs + BL * a.C1p;                                 // [BM][RtLp]
  T* Pst = Ks + BM * a.RtLp;                                // [BM][C1p]
  T* zls = Pst + BM * a.C1p;                                // [L][RtL] if zlast_smem

  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int N = a.N;
  const int last = N - 1;
  T* part = reinterpret_cast<T*>(a.part) + (int64_t)blockIdx.x * a.ztot;
  const T* WN = reinterpret_cast<const T*>(a.WN);

  // zero this CTA's partials
  for (int64_t e = t; e < a.ztot; e += NT) part[e] = T(0);
  T* zlast = a.zlast_smem ? zls : part + a.zoff[last];
  if (a.zlast_smem)
    for (int64_t e = t; e < a.L * a.RtL; e += NT) zls[e] = T(0);
  __syncthreads();

  const int kk = t & 31, rg = t >> 5;  // mode-N mapping: column kk, channels rg + 8j
  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * BM;
    // K rows of this tile: K[row, r] = prod_{k<N-1} W_k^(N)[i_k, r]
    for (int e = t; e < BM * a.RtLp; e += NT) {
      int rr = e / a.RtLp, r = e % a.RtLp;
      T v = T(0);
      int64_t row = row0 + rr;
      if (row < a.M && r < a.RtL) {
        int idx[TDK_MAX_MODES];
        decode_row<T>(row, a, idx);
        v = T(1);
        for (int k = 0; k < N - 1; ++k)
          v *= TDK_IN(idx[k], a.I[k]) ? reinterpret_cast<const T*>(a.Wk[last][k])[(int64_t)idx[k] * a.RtL + r]
                                      : T(0);
      }
      Ks[e] = v;
    }
    T acc[4][TC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j) acc[i][j] = T(0);

    for (int64_t c0 = 0; c0 < a.L; c0 += BL) {
      __syncthreads();  // previous chunk consumed (and Ks written on first chunk)
      for (int e = t; e < BM * BL; e += NT) {
        int rr = e / BL, cc = e % BL;
        int64_t row = row0 + rr, col = c0 + cc;
        Ys[rr * (BL + 1) + cc] =
            (row < a.M && col < a.L) ? CvtIn<T>::cvt(Y[row * a.L + col]) : T(0);
      }
      for (int e = t; e < BL * a.C1p; e += NT) {
        int cc = e / a.C1p, c = e % a.C1p;
        int64_t col = c0 + cc;
        WNs[e] = (col < a.L && c < a.C1) ? WN[col * a.C1 + c] : T(0);
      }
      __syncthreads();
      // P[row, c] += Y[row, col] * WN[col, c]
#pragma unroll 4
      for (int k = 0; k < BL; ++k) {
        T y[4], w[TC];
#pragma unroll
        for (int i = 0; i < 4; ++i) y[i] = Ys[(ty + 16 * i) * (BL + 1) + k];
#pragma unroll
        for (int j = 0; j < TC; ++j) w[j] = WNs[k * a.C1p + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < TC; ++j) acc[i][j] = fma(y[i], w[j], acc[i][j]);
      }
      // Z_N[col, r] += sum_row Y[row, col] * K[row, r]
      {
        T accL[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) accL[j] = T(0);
        for (int rr = 0; rr < BM; ++rr) {
          T y = Ys[rr * (BL + 1) + kk];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            int r = rg + 8 * j;
            if (r < a.RtLp) accL[j] = fma(y, Ks[rr * a.RtLp + r], accL[j]);
          }
        }
        int64_t col = c0 + kk;
        if (col < a.L) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            int r = rg + 8 * j;
            if (r < a.RtL && TDK_IN(col * a.RtL + r, a.L * a.RtL)) zlast[col * a.RtL + r] += accL[j];
          }
        }
      }
    }
    // epilogue: P -> Z_n for n < N-1 ... N-2
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j) Pst[(ty + 16 * i) * a.C1p + tx + 16 * j] = acc[i][j];
    __syncthreads();
    for (int c = t; c < a.C1; c += NT) {
      int n = 0;
      while (n + 1 < N - 1 && c >= a.off[n + 1]) ++n;
      const int r = c - a.off[n];
      const int Rn = a.Rt[n];
      T* zn = part + a.zoff[n];
      int idx[TDK_MAX_MODES];
      decode_row<T>(row0, a, idx);
      T run = T(0);
      int cur = idx[n];
      const int rows = (int)((a.M - row0) < BM ? (a.M - row0) : BM);
      for (int rr = 0; rr < rows; ++rr) {
        T coef = T(1);
        for (int k = 0; k < N - 1; ++k)
          if (k != n)
            coef *= TDK_IN(idx[k], a.I[k]) ? reinterpret_cast<const T*>(a.Wk[n][k])[(int64_t)idx[k] * Rn + r] : T(0);
        T v = Pst[rr * a.C1p + c] * coef;
        if (n == N - 2) {
          // changes every row: update in place
          if (TDK_IN((int64_t)idx[n] * Rn + r, a.zoff[n + 1] - a.zoff[n])) zn[(int64_t)idx[n] * Rn + r] += v;
        } else {
          if (idx[n] != cur) {
            if (TDK_IN((int64_t)cur * Rn + r, a.zoff[n + 1] - a.zoff[n])) zn[(int64_t)cur * Rn + r] += run;
            run = T(0);
            cur = idx[n];
          }
          run += v;
        }
        // advance the row index (last row mode fastest)
        for (int k = N - 2; k >= 0; --k) {
          if (++idx[k] < a.I[k]) break;
          idx[k] = 0;
        }
      }
      if (n != N - 2 && TDK_IN((int64_t)cur * Rn + r, a.zoff[n + 1] - a.zoff[n])) zn[(int64_t)cur * Rn + r] += run;
    }
    __syncthreads();
  }
  if (a.zlast_smem) {
    __syncthreads();
    for (int64_t e = t; e < a.L * a.RtL; e += NT) part[a.zoff[last] + e] = zls[e];
  }
}

template <class T>
__global__ void z_reduce_kernel(const T* __restrict__ part, int64_t ztot, int nparts,
                                double* __restrict__ Z) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ztot;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += (double)part[(int64_t)q * ztot + e];
    Z[e] = s;
  }
}

template <class T>
__global__ void convert_w_kernel(const double* __restrict__ src, T* __restrict__ dst, int64_t rows,
                                 int cols, int ld_dst, int col0) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols;
    int c = (int)(e % cols);
    dst[i * ld_dst + col0 + c] = (T)src[e];
  }
}

template <class TY, class T, int TC>
int launch_sketch(tdk_ctx* ctx, SketchArgs& a, const void* Y, int grid, size_t smem) {
  auto kern = sketch_simt_kernel<TY, T, TC>;
  TDK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(ctx, 0);
  kern<<<grid, NT, smem, ctx->stream>>>(reinterpret_cast<const TY*>(Y), a);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

template <class TY, class T>
int sketch_simt_t(tdk_ctx* ctx, const Geom& g, const void* Y, const double* const W[], double* Zdst) {
  const int N = g.N, last = N - 1;
  SketchArgs a{};
  a.N = N;
  for (int n = 0; n < N; ++n) {
    a.I[n] = g.I[n];
    a.Rt[n] = g.Rt[n];
  }
  a.M = g.M;
  a.L = g.L;
  int C1 = 0;
  for (int n = 0; n < N - 1; ++n) {
    a.off[n] = C1;
    C1 += g.Rt[n];
  }
  a.C1 = C1;
  int TC = (C1 + 15) / 16;
  int tcs[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 28};
  int TCc = 0;
  for (int v : tcs)
    if (v >= TC) { TCc = v; break; }
  if (TCc == 0) return TDK_EINVAL;
  a.C1p = 16 * TCc;
  a.RtL = g.Rt[last];
  a.RtLp = ((a.RtL + 7) / 8) * 8;
  if (a.RtLp > 64) return TDK_EINVAL;
  for (int n = 0; n <= N; ++n) a.zoff[n] = g.zoff[n];
  a.ztot = g.zoff[N];
  a.ntiles = (g.M + BM - 1) / BM;

  size_t base_smem = sizeof(T) * ((size_t)BM * (BL + 1) + (size_t)BL * a.C1p + (size_t)BM * a.RtLp +
                                  (size_t)BM * a.C1p);
  size_t zl_bytes = sizeof(T) * (size_t)g.L * a.RtL;
  a.zlast_smem = (base_smem + zl_bytes <= 100 * 1024) ? 1 : 0;
  size_t smem = base_smem + (a.zlast_smem ? zl_bytes : 0);
  if (smem > (size_t)ctx->max_smem_optin) return TDK_EINVAL;
  int per_sm = a.zlast_smem ? 1 : 2;
  int64_t grid64 = (int64_t)ctx->num_sms * per_sm;
  if (grid64 > a.ntiles) grid64 = a.ntiles;
  int grid = (int)grid64;

  // workspace: converted W, WN, partials
  Planner pl;
  pl.take<T>((size_t)g.L * C1);
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k)
      if (k != n && k != last) pl.take<T>((size_t)g.I[k] * g.Rt[n]);
  pl.take<T>((size_t)grid * a.ztot);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  T* WN = cv.take<T>((size_t)g.L * C1);
  for (int n = 0; n < N - 1; ++n) {
    convert_w_kernel<T><<<64, 256, 0, ctx->stream>>>(W[n * N + last], WN, g.L, g.Rt[n], C1, a.off[n]);
    TDK_LAUNCH_CHECK(ctx);
  }
  a.WN = WN;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) {
      a.Wk[n][k] = nullptr;
      if (k == n || k == last) continue;
      T* d = cv.take<T>((size_t)g.I[k] * g.Rt[n]);
      convert_w_kernel<T><<<64, 256, 0, ctx->stream>>>(W[n * N + k], d, g.I[k], g.Rt[n], g.Rt[n], 0);
      TDK_LAUNCH_CHECK(ctx);
      a.Wk[n][k] = d;
    }
  T* part = cv.take<T>((size_t)grid * a.ztot);
  a.part = part;
  switch (TCc) {
    case 1: rc = launch_sketch<TY, T, 1>(ctx, a, Y, grid, smem); break;
    case 2: rc = launch_sketch<TY, T, 2>(ctx, a, Y, grid, smem); break;
    case 3: rc = launch_sketch<TY, T, 3>(ctx, a, Y, grid, smem); break;
    case 4: rc = launch_sketch<TY, T, 4>(ctx, a, Y, grid, smem); break;
    case 6: rc = launch_sketch<TY, T, 6>(ctx, a, Y, grid, smem); break;
    case 8: rc = launch_sketch<TY, T, 8>(ctx, a, Y, grid, smem); break;
    case 12: rc = launch_sketch<TY, T, 12>(ctx, a, Y, grid, smem); break;
    case 16: rc = launch_sketch<TY, T, 16>(ctx, a, Y, grid, smem); break;
    case 24: rc = launch_sketch<TY, T, 24>(ctx, a, Y, grid, smem); break;
    case 28: rc = launch_sketch<TY, T, 28>(ctx, a, Y, grid, smem); break;
    default: rc = TDK_EINVAL;
  }
  if (rc) return rc;
  z_reduce_kernel<T><<<256, 256, 0, ctx->stream>>>(part, a.ztot, grid, Zdst);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // namespace

int sketch_simt(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const W[],
                double* Zdst) {
  switch (dtype) {
    case TDK_F64: return sketch_simt_t<double, double>(ctx, g, Y, W, Zdst);
    case TDK_F32: return sketch_simt_t<float, float>(ctx, g, Y, W, Zdst);
    case TDK_BF16: return sketch_simt_t<__nv_bfloat16, float>(ctx, g, Y, W, Zdst);
  }
  return TDK_EINVAL;
}

namespace {
// ||Y||^2 over a grid-stride range per thread: FP64 sums of FP32 (Kahan) or
// FP64 chunk sums, then one FP64 partial per block in a fixed order
template <class TY>
__global__ void __launch_bounds__(256) norm2_pass_kernel(const TY* __restrict__ Y, int64_t n,
                                                         double* __restrict__ parts) {
  __shared__ double red[8];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  while (e < n) {
    // 64 elements at a time in the storage's natural precision
    double chunk = 0.0;
    float f = 0.f;
    for (int k = 0; k < 64 && e < n; ++k, e += stride) {
      if (sizeof(TY) == 8) {
        const double v = (double)to_f(Y[e]);
        chunk = fma(v, v, chunk);
      } else {
        const float v = to_f(Y[e]);
        f = fmaf(v, v, f);
      }
    }
    acc += sizeof(TY) == 8 ? chunk : (double)f;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    parts[blockIdx.x] = s;
  }
}
__global__ void norm2_sum_kernel(const double* __restrict__ parts, int n, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += parts[i];
    *out = s;
  }
}
}  // namespace

int norm2_pass(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, double* normY2) {
  const int blocks = 4 * ctx->num_sms;
  int rc = ws_reserve(ctx, sizeof(double) * blocks + 256);
  if (rc) return rc;
  double* parts = reinterpret_cast<double*>(ctx->ws);
  switch (dtype) {
    case TDK_F64: norm2_pass_kernel<double><<<blocks, 256, 0, ctx->stream>>>((const double*)Y, g.numel, parts); break;
    case TDK_F32: norm2_pass_kernel<float><<<blocks, 256, 0, ctx->stream>>>((const float*)Y, g.numel, parts); break;
    case TDK_BF16:
      norm2_pass_kernel<__nv_bfloat16><<<blocks, 256, 0, ctx->stream>>>((const __nv_bfloat16*)Y, g.numel, parts);
      break;
    default: return TDK_EINVAL;
  }
  TDK_LAUNCH_CHECK(ctx);
  norm2_sum_kernel<<<1, 32, 0, ctx->stream>>>(parts, blocks, normY2);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // namespace tdk

// ---- allocation-free variant of the sketch pass --------------------------------
// The whole scratch of tucker_sketch_static (converted W, the per-CTA partial
// sketches, the packed FP64 sum) lives in one file-scope device array, so the
// call allocates nothing.  Every call on a device shares it: calls that
// overlap on the GPU race.
#include <mutex>

namespace tdk {
namespace {

constexpr size_t SKETCH_STATIC_BYTES = TDK_SKETCH_STATIC_MAX_BYTES;  // 16 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_sketch_scratch[SKETCH_STATIC_BYTES];

std::mutex g_scratch_mu;
struct ScratchAddr {
  unsigned long long ctx_id;  // context the address was resolved in (0: unknown)
  void* addr;
};
ScratchAddr g_scratch_addr[MAX_DEVICES];

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// unique identity of the CUDA context current on this thread, 0 if the
// driver cannot tell (the caller then resolves the address on every call)
unsigned long long current_context_id() {
  static PfnCtxGetCurrent get_cur = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<PfnCtxGetCurrent>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PfnCtxGetId>(p);
    cudaGetLastError();
  }
  if (!get_cur || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// address of the array on the current device; resolved once per device and
// context (a context created after a device reset loads the module anew)
int static_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= MAX_DEVICES) return TDK_EINVAL;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  const unsigned long long id = current_context_id();
  ScratchAddr& s = g_scratch_addr[device];
  if (!s.addr || id == 0 || s.ctx_id != id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sketch_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      s.addr = nullptr;
      return TDK_ECUDA;
    }
    s.addr = p;
    s.ctx_id = id;
  }
  *out = static_cast<unsigned char*>(s.addr);
  return TDK_OK;
}

// byte carve of the static array with 256-byte aligned pieces
struct StaticCarve {
  size_t off = 0;
  template <class T>
  size_t take(size_t n) {
    size_t o = (off + 255) & ~(size_t)255;
    off = o + n * sizeof(T);
    return o;
  }
};

template <class TY, class T>
int sketch_static_t(tdk_ctx* ctx, const Geom& g, const void* Y, const double* const W[],
                    double* const Z_out[]) {
  const int N = g.N, last = N - 1;
  SketchArgs a{};
  a.N = N;
  for (int n = 0; n < N; ++n) {
    a.I[n] = g.I[n];
    a.Rt[n] = g.Rt[n];
  }
  a.M = g.M;
  a.L = g.L;
  int C1 = 0;
  for (int n = 0; n < N - 1; ++n) {
    a.off[n] = C1;
    C1 += g.Rt[n];
  }
  a.C1 = C1;
  int TC = (C1 + 15) / 16;
  int tcs[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 28};
  int TCc = 0;
  for (int v : tcs)
    if (v >= TC) { TCc = v; break; }
  if (TCc == 0) return TDK_EINVAL;
  a.C1p = 16 * TCc;
  a.RtL = g.Rt[last];
  a.RtLp = ((a.RtL + 7) / 8) * 8;
  if (a.RtLp > 64) return TDK_EINVAL;
  for (int n = 0; n <= N; ++n) a.zoff[n] = g.zoff[n];
  a.ztot = g.zoff[N];
  a.ntiles = (g.M + BM - 1) / BM;

  size_t base_smem = sizeof(T) * ((size_t)BM * (BL + 1) + (size_t)BL * a.C1p + (size_t)BM * a.RtLp +
                                  (size_t)BM * a.C1p);
  size_t zl_bytes = sizeof(T) * (size_t)g.L * a.RtL;
  a.zlast_smem = (base_smem + zl_bytes <= 100 * 1024) ? 1 : 0;
  size_t smem = base_smem + (a.zlast_smem ? zl_bytes : 0);
  if (smem > (size_t)ctx->max_smem_optin) return TDK_EINVAL;
  int per_sm = a.zlast_smem ? 1 : 2;
  int64_t grid64 = (int64_t)ctx->num_sms * per_sm;
  if (grid64 > a.ntiles) grid64 = a.ntiles;

  // fixed pieces first; the per-CTA partials take what is left, and the grid
  // shrinks to fit them (a different grid only changes the summation order)
  StaticCarve sc;
  const size_t o_wn = sc.take<T>((size_t)g.L * C1);
  size_t o_wk[TDK_MAX_MODES][TDK_MAX_MODES] = {};
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k)
      if (k != n && k != last) o_wk[n][k] = sc.take<T>((size_t)g.I[k] * g.Rt[n]);
  const size_t o_z = sc.take<double>((size_t)a.ztot);
  const size_t o_part = (sc.off + 255) & ~(size_t)255;
  if (o_part >= SKETCH_STATIC_BYTES) return TDK_ESCRATCH;
  const int64_t fit = (int64_t)((SKETCH_STATIC_BYTES - o_part) / (sizeof(T) * (size_t)a.ztot));
  if (fit < 1) return TDK_ESCRATCH;
  if (grid64 > fit) grid64 = fit;
  const int grid = (int)grid64;

  unsigned char* base = nullptr;
  int rc = static_scratch(ctx->device, &base);
  if (rc) return rc;
  T* WN = reinterpret_cast<T*>(base + o_wn);
  for (int n = 0; n < N - 1; ++n) {
    convert_w_kernel<T><<<64, 256, 0, ctx->stream>>>(W[n * N + last], WN, g.L, g.Rt[n], C1, a.off[n]);
    TDK_LAUNCH_CHECK(ctx);
  }
  a.WN = WN;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) {
      a.Wk[n][k] = nullptr;
      if (k == n || k == last) continue;
      T* d = reinterpret_cast<T*>(base + o_wk[n][k]);
      convert_w_kernel<T><<<64, 256, 0, ctx->stream>>>(W[n * N + k], d, g.I[k], g.Rt[n], g.Rt[n], 0);
      TDK_LAUNCH_CHECK(ctx);
      a.Wk[n][k] = d;
    }
  // the kernel zeroes its own partials before accumulating; the reduce
  // overwrites every element of the packed sum: nothing needs clearing here
  T* part = reinterpret_cast<T*>(base + o_part);
  a.part = part;
  switch (TCc) {
    case 1: rc = launch_sketch<TY, T, 1>(ctx, a, Y, grid, smem); break;
    case 2: rc = launch_sketch<TY, T, 2>(ctx, a, Y, grid, smem); break;
    case 3: rc = launch_sketch<TY, T, 3>(ctx, a, Y, grid, smem); break;
    case 4: rc = launch_sketch<TY, T, 4>(ctx, a, Y, grid, smem); break;
    case 6: rc = launch_sketch<TY, T, 6>(ctx, a, Y, grid, smem); break;
    case 8: rc = launch_sketch<TY, T, 8>(ctx, a, Y, grid, smem); break;
    case 12: rc = launch_sketch<TY, T, 12>(ctx, a, Y, grid, smem); break;
    case 16: rc = launch_sketch<TY, T, 16>(ctx, a, Y, grid, smem); break;
    case 24: rc = launch_sketch<TY, T, 24>(ctx, a, Y, grid, smem); break;
    case 28: rc = launch_sketch<TY, T, 28>(ctx, a, Y, grid, smem); break;
    default: rc = TDK_EINVAL;
  }
  if (rc) return rc;
  double* Z = reinterpret_cast<double*>(base + o_z);
  z_reduce_kernel<T><<<256, 256, 0, ctx->stream>>>(part, a.ztot, grid, Z);
  TDK_LAUNCH_CHECK(ctx);
  for (int n = 0; n < N; ++n)
    TDK_CUDA_TRY(cudaMemcpyAsync(Z_out[n], Z + g.zoff[n], sizeof(double) * (size_t)g.I[n] * g.Rt[n],
                                 cudaMemcpyDeviceToDevice, ctx->stream));
  return TDK_OK;
}

}  // namespace
}  // namespace tdk

extern "C" int tucker_sketch_static(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y,
                                    const double* const W[], double* const Z_out[]) {
  using namespace tdk;
  if (!ctx || !desc || !Y || !W || !Z_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  if (desc->prec != TDK_PREC_SIMT) return TDK_ENOTSUP;
  for (int n = 0; n < g.N; ++n) {
    if (!Z_out[n]) return TDK_EINVAL;
    for (int k = 0; k < g.N; ++k)
      if (k != n && !W[n * g.N + k]) return TDK_EINVAL;
  }
  TDK_CUDA_TRY(cudaSetDevice(ctx->device));
  switch (desc->dtype) {
    case TDK_F64: return sketch_static_t<double, double>(ctx, g, Y, W, Z_out);
    case TDK_F32: return sketch_static_t<float, float>(ctx, g, Y, W, Z_out);
    case TDK_BF16: return sketch_static_t<__nv_bfloat16, float>(ctx, g, Y, W, Z_out);
  }
  return TDK_EINVAL;
}

namespace tdk {
TDK_CHECKED_UNIT(sketch_simt)
}  // namespace tdk
