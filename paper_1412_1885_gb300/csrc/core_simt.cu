// Core G = Y x_1 U_1^T ... x_N U_N^T on CUDA cores (Alg. 2, the mode-n projection steps
// for every n; Eq. 1).  The contiguous mode N is contracted first:
//   X_1[row, r] = sum_col Y[row, col] U_N[col, r]        (row = (i_1..i_{N-1}))
// which is the only pass over the full tensor (it also accumulates ||Y||^2);
// the remaining modes are contracted on the shrunk tensors by
//   Xo[a, r, b] = sum_i U_m[i, r] X[a, i, b].
#include "tdk_internal.cuh"

namespace tdk {
namespace {

constexpr int BM = 64, BL = 32, NT = 256;

template <class T>
struct Acc2 {  // ||Y||^2 accumulator: Kahan-compensated in FP32, plain in FP64
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    T y = x * x - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <class TY, class T, int TC>
__global__ void __launch_bounds__(NT) ttm_last_kernel(const TY* __restrict__ Y, int64_t M, int64_t L,
                                                      const T* __restrict__ U, int Rt,
                                                      T* __restrict__ X, double* __restrict__ nrm_part) {
  __shared__ T Ys[BM * (BL + 1)];
  __shared__ T Us[BL * 16 * TC];
  __shared__ double red[NT / 32];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int ldu = 16 * TC;
  const int64_t ntiles = (M + BM - 1) / BM;
  Acc2<T> nrm;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * BM;
    T acc[4][TC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j) acc[i][j] = T(0);
    for (int64_t c0 = 0; c0 < L; c0 += BL) {
      __syncthreads();
      for (int e = t; e < BM * BL; e += NT) {
        int rr = e / BL, cc = e % BL;
        int64_t row = row0 + rr, col = c0 + cc;
        T y = (row < M && col < L) ? CvtIn<T>::cvt(Y[row * L + col]) : T(0);
        nrm.add(y);
        Ys[rr * (BL + 1) + cc] = y;
      }
      for (int e = t; e < BL * ldu; e += NT) {
        int cc = e / ldu, c = e % ldu;
        int64_t col = c0 + cc;
        Us[e] = (col < L && c < Rt) ? U[col * Rt + c] : T(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < BL; ++k) {
        T y[4], w[TC];
#pragma unroll
        for (int i = 0; i < 4; ++i) y[i] = Ys[(ty + 16 * i) * (BL + 1) + k];
#pragma unroll
        for (int j = 0; j < TC; ++j) w[j] = Us[k * ldu + tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < TC; ++j) acc[i][j] = fma(y[i], w[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t row = row0 + ty + 16 * i;
      if (row >= M) continue;
#pragma unroll
      for (int j = 0; j < TC; ++j) {
        int c = tx + 16 * j;
        if (c < Rt) X[row * Rt + c] = acc[i][j];
      }
    }
  }
  double v = warp_sum(nrm.value());
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    nrm_part[blockIdx.x] = s;
  }
}

// Xo[a, r, b] = sum_i U[i, r] X[a, i, b];  grid (A, min(ceil(Bd/64), 65535), KS),
// Rt <= 64; a CTA strides over the 64-column tiles of b.
// Split over the contracted index: CTA z sums i in [z kch, (z+1) kch) into
// the z-th copy of the output (KS = 1: the output itself).
// X may be stored in a narrower type TX (BF16 data), converted on load.
template <class T, class TX = T>
__global__ void __launch_bounds__(NT) ttm_mid_kernel(const TX* __restrict__ X, int64_t Ic, int64_t Bd,
                                                     const T* __restrict__ U, int Rt, T* __restrict__ Xo,
                                                     int64_t kch) {
  __shared__ T Xs[32 * 64];
  __shared__ T Us[32 * 64];
  const int t = threadIdx.x, tb = t & 15, tr = t >> 4;
  const int64_t a = blockIdx.x;
  const int64_t k0 = (int64_t)blockIdx.z * kch, k1 = k0 + kch < Ic ? k0 + kch : Ic;
  const TX* Xa = X + a * Ic * Bd;
  Xo += (int64_t)blockIdx.z * gridDim.x * (int64_t)Rt * Bd;
  const int64_t nbt = (Bd + 63) / 64;
  for (int64_t bt = blockIdx.y; bt < nbt; bt += gridDim.y) {
  const int64_t b0 = bt * 64;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int64_t i0 = k0; i0 < k1; i0 += 32) {
    __syncthreads();
    for (int e = t; e < 32 * 64; e += NT) {
      int ii = e / 64, c = e % 64;
      int64_t i = i0 + ii;
      Xs[e] = (i < k1 && b0 + c < Bd && TDK_IN(a * Ic * Bd + i * Bd + b0 + c, (int64_t)gridDim.x * Ic * Bd))
                  ? CvtIn<T>::cvt(Xa[i * Bd + b0 + c])
                  : T(0);
      Us[e] = (i < k1 && c < Rt) ? U[i * Rt + c] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int ii = 0; ii < 32; ++ii) {
      T u[4], x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        u[q] = Us[ii * 64 + tr + 16 * q];
        x[q] = Xs[ii * 64 + tb + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(u[p], x[q], acc[p][q]);
    }
  }
  T* Xoa = Xo + a * (int64_t)Rt * Bd;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int r = tr + 16 * p;
    if (r >= Rt) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int64_t b = b0 + tb + 16 * q;
      if (b < Bd && TDK_IN((a * Rt + r) * Bd + b, (int64_t)gridDim.x * Rt * Bd)) Xoa[(int64_t)r * Bd + b] = acc[p][q];
    }
  }
  }
}

// Same contraction for wide FP32 slabs (Rt and Bd above 32): a 64 x 64 output
// tile per CTA, 64 threads with 8 x 8 outputs each (two 4-wide groups 32 apart
// in each direction), K staged 32 deep through
// double-buffered shared memory with the next slice prefetched in registers.
// grid (A, min(ceil(Bd / 64), 65535), KS); a CTA strides over the column tiles
__global__ void __launch_bounds__(64) ttm_mid64_kernel(const float* __restrict__ X, int64_t Ic, int64_t Bd,
                                                       const float* __restrict__ U, int Rt, float* __restrict__ Xo,
                                                       int64_t kch) {
  constexpr int KC = 32;
  __shared__ __align__(16) float Xs[2][KC][64];
  __shared__ __align__(16) float Us[2][KC][64];
  const int t = threadIdx.x, tx = t & 7, ty = t >> 3;
  const int64_t a = blockIdx.x;
  const int64_t k0 = (int64_t)blockIdx.z * kch, k1 = k0 + kch < Ic ? k0 + kch : Ic;
  const float* Xa = X + a * Ic * Bd;
  Xo += (int64_t)blockIdx.z * gridDim.x * (int64_t)Rt * Bd;
  const int64_t nbt = (Bd + 63) / 64;
  for (int64_t bt = blockIdx.y; bt < nbt; bt += gridDim.y) {
  const int64_t b0 = bt * 64;
  const bool bok = b0 + t < Bd, rok = t < Rt;
  float rx[KC], ru[KC];
  // thread t loads column t of the slice: 32 rows of X (coalesced along b) and of U
  auto load = [&](int64_t i0) {
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      const int64_t i = i0 + j;
      rx[j] = (i < k1 && bok && TDK_IN(a * Ic * Bd + i * Bd + b0 + t, (int64_t)gridDim.x * Ic * Bd))
                  ? __ldg(Xa + i * Bd + b0 + t)
                  : 0.f;
      ru[j] = (i < k1 && rok) ? __ldg(U + i * Rt + t) : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      Xs[buf][j][t] = rx[j];
      Us[buf][j][t] = ru[j];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[p][q] = 0.f;
  load(k0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int64_t i0 = k0; i0 < k1; i0 += KC) {
    const bool more = i0 + KC < k1;
    if (more) load(i0 + KC);
#pragma unroll 4
    for (int k = 0; k < KC; ++k) {
      // rows ty*4 + {0..3} and 32 + ty*4 + {0..3}; columns likewise with tx:
      // a quarter-warp's float4 reads cover 32 distinct banks
      const float4 u0 = *reinterpret_cast<const float4*>(&Us[buf][k][ty * 4]);
      const float4 u1 = *reinterpret_cast<const float4*>(&Us[buf][k][32 + ty * 4]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Xs[buf][k][tx * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Xs[buf][k][32 + tx * 4]);
      const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
      const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(u[p], x[q], acc[p][q]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* Xoa = Xo + a * (int64_t)Rt * Bd;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int r = (p < 4) ? ty * 4 + p : 32 + ty * 4 + (p - 4);
    if (r >= Rt) continue;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t b = b0 + ((q < 4) ? tx * 4 + q : 32 + tx * 4 + (q - 4));
      if (b < Bd && TDK_IN((a * Rt + r) * Bd + b, (int64_t)gridDim.x * Rt * Bd)) Xoa[(int64_t)r * Bd + b] = acc[p][q];
    }
  }
  __syncthreads();  // the next tile refills the shared buffers
  }
}

// Same contraction for narrow FP32 slabs (Rt <= 32, Bd <= 32): the whole
// Rt x Bd output of one a per CTA.  Its 256 threads are 16 groups of the
// contracted index (k = kg mod 16 within each staged chunk of 64) times 16
// register tiles of T x T outputs (4 x 4 tiles cover Rt, Bd <= 4 T), so that
// every thread does T^2 FMAs per 2 T shared-memory loads and few threads
// idle on padding; the 16 partial outputs are then added in a fixed order
// (the two groups of a warp by a shuffle, the eight warps pairwise through
// the staging buffers).
template <int T>
__global__ void __launch_bounds__(256) ttm_mid32_kernel(const float* __restrict__ X, int64_t Ic, int Bd,
                                                        const float* __restrict__ U, int Rt, float* __restrict__ Xo,
                                                        int64_t kch) {
  constexpr int KC = 64;
  __shared__ __align__(16) float stage[2 * KC * 32];  // X chunk, U chunk; then the warps' partial outputs
  float* Xs = stage;
  float* Us = stage + KC * 32;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t a = blockIdx.x;
  const int64_t k0 = (int64_t)blockIdx.z * kch, k1 = k0 + kch < Ic ? k0 + kch : Ic;
  const float* Xa = X + a * Ic * Bd;
  Xo += (int64_t)blockIdx.z * gridDim.x * (int64_t)Rt * Bd;
  const int tile = t & 15, kg = t >> 4;  // two k groups per warp (lanes 0-15, 16-31)
  const int r0 = (tile >> 2) * T, b0 = (tile & 3) * T;
  float acc[T][T];
#pragma unroll
  for (int u = 0; u < T; ++u)
#pragma unroll
    for (int v = 0; v < T; ++v) acc[u][v] = 0.f;
  for (int64_t i0 = k0; i0 < k1; i0 += KC) {
    const int rows = (int)((k1 - i0) < KC ? (k1 - i0) : KC);
    __syncthreads();
    for (int e = t; e < rows * Bd; e += 256) Xs[(e / Bd) * 32 + e % Bd] = __ldg(Xa + i0 * Bd + e);
    for (int e = t; e < rows * Rt; e += 256) Us[(e / Rt) * 32 + e % Rt] = __ldg(U + i0 * Rt + e);
    __syncthreads();
    for (int k = kg; k < rows; k += 16) {
      float uv[T], xv[T];
#pragma unroll
      for (int u = 0; u < T; ++u) uv[u] = Us[k * 32 + ((r0 + u) & 31)];
#pragma unroll
      for (int v = 0; v < T; ++v) xv[v] = Xs[k * 32 + ((b0 + v) & 31)];
#pragma unroll
      for (int u = 0; u < T; ++u)
#pragma unroll
        for (int v = 0; v < T; ++v) acc[u][v] = fmaf(uv[u], xv[v], acc[u][v]);
    }
  }
  // the two k groups of the warp, then the warps pairwise (w + 4, w + 2,
  // w + 1 into w), through the staging buffers (32 x 32 outputs per warp)
#pragma unroll
  for (int u = 0; u < T; ++u)
#pragma unroll
    for (int v = 0; v < T; ++v) acc[u][v] += __shfl_xor_sync(0xffffffffu, acc[u][v], 16);
  float* red = stage;  // [4][32 * 32] floats
  for (int half = 4; half >= 1; half >>= 1) {
    __syncthreads();
    if (w >= half && w < 2 * half && lane < 16)
#pragma unroll
      for (int u = 0; u < T; ++u)
#pragma unroll
        for (int v = 0; v < T; ++v) red[(w - half) * 1024 + ((r0 + u) & 31) * 32 + ((b0 + v) & 31)] = acc[u][v];
    __syncthreads();
    if (w < half && lane < 16)
#pragma unroll
      for (int u = 0; u < T; ++u)
#pragma unroll
        for (int v = 0; v < T; ++v) acc[u][v] += red[w * 1024 + ((r0 + u) & 31) * 32 + ((b0 + v) & 31)];
  }
  float* Xoa = Xo + a * (int64_t)Rt * Bd;
  if (w == 0 && lane < 16)
#pragma unroll
    for (int u = 0; u < T; ++u)
#pragma unroll
      for (int v = 0; v < T; ++v) {
        const int r = r0 + u, b = b0 + v;
        if (r < Rt && b < Bd && TDK_IN((a * Rt + r) * Bd + b, (int64_t)gridDim.x * Rt * Bd))
          Xoa[(int64_t)r * Bd + b] = acc[u][v];
      }
}

// fixed-order sum of the KS partial outputs of a split contraction
template <class T>
__global__ void sum_split_kernel(const T* __restrict__ part, int ks, int64_t n, T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T v = part[e];
    for (int z = 1; z < ks; ++z) v += part[z * n + e];
    out[e] = v;
  }
}

// Number of slices of the contracted index: the contractions at the end of
// the chain have few output tiles (A = 1 at the last one), so their CTAs
// would leave most SMs idle; slices of at least 128 indices each, partials in
// `part` (capacity in elements), summed in a fixed order.
static int split_count(tdk_ctx* ctx, int64_t ctas, int per_sm, int64_t Ic, int64_t out_n, int64_t part_cap) {
  if (!part_cap) return 1;
  int64_t ks = (per_sm * (int64_t)ctx->num_sms + ctas - 1) / ctas;
  ks = std::min<int64_t>(ks, Ic / 128);
  ks = std::min<int64_t>(ks, part_cap / std::max<int64_t>(out_n, 1));
  return ks < 2 ? 1 : (int)std::min<int64_t>(ks, 64);
}

__global__ void sum_parts_kernel(const double* __restrict__ parts, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += parts[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    *out = v;
  }
}

template <class T>
__global__ void cvt_f64_kernel(const double* __restrict__ s, T* __restrict__ d, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (T)s[e];
}

template <class TY, class T, int TC>
int launch_last(tdk_ctx* ctx, const void* Y, int64_t M, int64_t L, const T* U, int Rt, T* X,
                double* parts, int grid) {
  ProfScope ps(ctx, 1);
  ttm_last_kernel<TY, T, TC><<<grid, NT, 0, ctx->stream>>>(reinterpret_cast<const TY*>(Y), M, L, U, Rt,
                                                          X, parts);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // namespace

template <class T>
int launch_ttm_mid(tdk_ctx* ctx, const T* X, int64_t A, int64_t Ic, int64_t Bd, const T* U, int Rt, T* Xo,
                   T* part, int64_t part_cap) {
  const int64_t nb = (Bd + 63) / 64, out_n = A * Rt * Bd;
  const int ks = split_count(ctx, A * nb, 2, Ic, out_n, part_cap);
  const int64_t kch = (Ic + ks - 1) / ks;
  dim3 grid((unsigned)A, (unsigned)std::min<int64_t>(nb, 65535), (unsigned)ks);
  ttm_mid_kernel<T><<<grid, NT, 0, ctx->stream>>>(X, Ic, Bd, U, Rt, ks > 1 ? part : Xo, kch);
  TDK_LAUNCH_CHECK(ctx);
  if (ks > 1) {
    sum_split_kernel<T><<<(unsigned)std::min<int64_t>((out_n + 255) / 256, 1024), 256, 0, ctx->stream>>>(
        part, ks, out_n, Xo);
    TDK_LAUNCH_CHECK(ctx);
  }
  return TDK_OK;
}
template <>
int launch_ttm_mid<float>(tdk_ctx* ctx, const float* X, int64_t A, int64_t Ic, int64_t Bd, const float* U, int Rt,
                          float* Xo, float* part, int64_t part_cap) {
  const int64_t nb = (Bd + 63) / 64, out_n = A * Rt * Bd;
  const bool wide = Rt > 32 && Bd > 32, narrow = Rt <= 32 && Bd <= 32;
  const int ks = wide ? split_count(ctx, A * nb, 6, Ic, out_n, part_cap)
                      : split_count(ctx, narrow ? A : A * nb, 2, Ic, out_n, part_cap);
  const int64_t kch = (Ic + ks - 1) / ks;
  float* dst = ks > 1 ? part : Xo;
  const unsigned gy = (unsigned)std::min<int64_t>(nb, 65535);
  if (wide)
    ttm_mid64_kernel<<<dim3((unsigned)A, gy, (unsigned)ks), 64, 0, ctx->stream>>>(X, Ic, Bd, U, Rt, dst, kch);
  else if (narrow) {
    // register tiles of T x T, 4 x 4 of them covering the output
    const int need = (int)std::max<int64_t>((Rt + 3) / 4, (Bd + 3) / 4);
    const dim3 g3((unsigned)A, 1, (unsigned)ks);
    if (need <= 2)
      ttm_mid32_kernel<2><<<g3, 256, 0, ctx->stream>>>(X, Ic, (int)Bd, U, Rt, dst, kch);
    else if (need <= 4)
      ttm_mid32_kernel<4><<<g3, 256, 0, ctx->stream>>>(X, Ic, (int)Bd, U, Rt, dst, kch);
    else if (need <= 5)
      ttm_mid32_kernel<5><<<g3, 256, 0, ctx->stream>>>(X, Ic, (int)Bd, U, Rt, dst, kch);
    else
      ttm_mid32_kernel<8><<<g3, 256, 0, ctx->stream>>>(X, Ic, (int)Bd, U, Rt, dst, kch);
  }
  else
    ttm_mid_kernel<float><<<dim3((unsigned)A, gy, (unsigned)ks), NT, 0, ctx->stream>>>(X, Ic, Bd, U, Rt, dst, kch);
  TDK_LAUNCH_CHECK(ctx);
  if (ks > 1) {
    sum_split_kernel<float><<<(unsigned)std::min<int64_t>((out_n + 255) / 256, 1024), 256, 0, ctx->stream>>>(
        part, ks, out_n, Xo);
    TDK_LAUNCH_CHECK(ctx);
  }
  return TDK_OK;
}

template int launch_ttm_mid<double>(tdk_ctx*, const double*, int64_t, int64_t, int64_t, const double*, int, double*,
                                    double*, int64_t);

int launch_ttm_mid_bf16(tdk_ctx* ctx, const __nv_bfloat16* X, int64_t A, int64_t Ic, int64_t Bd, const float* U,
                        int Rt, float* Xo) {
  const int64_t nb = (Bd + 63) / 64;
  dim3 grid((unsigned)A, (unsigned)std::min<int64_t>(nb, 65535), 1);
  ttm_mid_kernel<float, __nv_bfloat16><<<grid, NT, 0, ctx->stream>>>(X, Ic, Bd, U, Rt, Xo, Ic);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

template <class T>
int launch_ttm_last(tdk_ctx* ctx, const T* X, int64_t M, int64_t L, const T* U, int Rt, T* Xo, double* parts,
                    int grid) {
  switch ((Rt + 15) / 16) {
    case 1: return launch_last<T, T, 1>(ctx, X, M, L, U, Rt, Xo, parts, grid);
    case 2: return launch_last<T, T, 2>(ctx, X, M, L, U, Rt, Xo, parts, grid);
    case 3: return launch_last<T, T, 3>(ctx, X, M, L, U, Rt, Xo, parts, grid);
    case 4: return launch_last<T, T, 4>(ctx, X, M, L, U, Rt, Xo, parts, grid);
  }
  return TDK_EINVAL;
}
template int launch_ttm_last<float>(tdk_ctx*, const float*, int64_t, int64_t, const float*, int, float*, double*, int);
template int launch_ttm_last<double>(tdk_ctx*, const double*, int64_t, int64_t, const double*, int, double*, double*,
                                     int);

// core chain from a partly contracted tensor X with dims I_0..I_{m0},
// Rt_{m0+1}..Rt_{N-1}: modes m0 down to m_stop are contracted (m_stop = 0:
// the core; m_stop = 1: mode 0 stays open); X is neither tmp0 nor tmp1
template <class T>
int core_chain_from(tdk_ctx* ctx, const Geom& g, const T* X, int m0, T* const Ut[], T* G, T* tmp0, T* tmp1,
                    T* part, int64_t part_cap, int m_stop) {
  const int N = g.N;
  const T* cur = X;
  int64_t Bd = 1;
  for (int k = m0 + 1; k < N; ++k) Bd *= g.Rt[k];
  if (m0 < m_stop) {  // nothing left to contract
    int64_t n = Bd;
    for (int k = 0; k <= m0; ++k) n *= g.I[k];
    TDK_CUDA_TRY(cudaMemcpyAsync(G, X, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
    return TDK_OK;
  }
  for (int m = m0; m >= m_stop; --m) {
    int64_t A = 1;
    for (int k = 0; k < m; ++k) A *= g.I[k];
    T* out = (m == m_stop) ? G : ((m % 2) ? tmp0 : tmp1);
    const int rc = launch_ttm_mid<T>(ctx, cur, A, g.I[m], Bd, Ut[m], g.Rt[m], out, part, part_cap);
    if (rc) return rc;
    cur = out;
    Bd *= g.Rt[m];
  }
  return TDK_OK;
}
template int core_chain_from<float>(tdk_ctx*, const Geom&, const float*, int, float* const[], float*, float*,
                                    float*, float*, int64_t, int);

// core chain shared by both forms once X_1 exists (modes N-2 .. m_stop)
template <class T>
int core_chain_rest(tdk_ctx* ctx, const Geom& g, const T* X1, T* const Ut[], T* G, T* tmp0, T* tmp1, T* part,
                    int64_t part_cap, int m_stop) {
  return core_chain_from<T>(ctx, g, X1, g.N - 2, Ut, G, tmp0, tmp1, part, part_cap, m_stop);
}
template int core_chain_rest<float>(tdk_ctx*, const Geom&, const float*, float* const[], float*, float*, float*,
                                    float*, int64_t, int);
template int core_chain_rest<double>(tdk_ctx*, const Geom&, const double*, double* const[], double*, double*,
                                     double*, double*, int64_t, int);

template <class TY, class T>
static int core_simt_t(tdk_ctx* ctx, const Geom& g, const void* Y, const double* const U[], void* Gv,
                       double* normY2, int open0) {
  const int N = g.N;
  const int RtL = g.Rt[N - 1];
  const int TC = (RtL + 15) / 16;
  const int64_t ntiles = (g.M + BM - 1) / BM;
  int grid = (int)((int64_t)ctx->num_sms * 4 < ntiles ? (int64_t)ctx->num_sms * 4 : ntiles);
  // workspace: U in T, X1, two ping-pong buffers, norm partials
  int64_t tmpsz = 0;
  {
    int64_t Bd = RtL;
    for (int m = N - 2; m >= 1; --m) {
      int64_t A = 1;
      for (int k = 0; k < m; ++k) A *= g.I[k];
      int64_t s = A * g.Rt[m] * Bd;
      if (s > tmpsz) tmpsz = s;
      Bd *= g.Rt[m];
    }
  }
  Planner pl;
  for (int n = 0; n < N; ++n) pl.take<T>((size_t)g.I[n] * g.Rt[n]);
  pl.take<T>((size_t)g.M * RtL);
  pl.take<T>((size_t)tmpsz);
  pl.take<T>((size_t)tmpsz);
  pl.take<double>((size_t)grid);
  const int64_t pcap = chain_split_cap(g);
  pl.take<T>((size_t)pcap);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  T* Ut[TDK_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    Ut[n] = cv.take<T>((size_t)g.I[n] * g.Rt[n]);
    if (open0 && n == 0) continue;  // mode 0 stays open: U_1 is not read
    cvt_f64_kernel<T><<<64, 256, 0, ctx->stream>>>(U[n], Ut[n], g.I[n] * g.Rt[n]);
    TDK_LAUNCH_CHECK(ctx);
  }
  T* X1 = cv.take<T>((size_t)g.M * RtL);
  T* tmp0 = cv.take<T>((size_t)tmpsz);
  T* tmp1 = cv.take<T>((size_t)tmpsz);
  double* parts = cv.take<double>((size_t)grid);
  T* spl = cv.take<T>((size_t)pcap);
  switch (TC) {
    case 1: rc = launch_last<TY, T, 1>(ctx, Y, g.M, g.L, Ut[N - 1], RtL, X1, parts, grid); break;
    case 2: rc = launch_last<TY, T, 2>(ctx, Y, g.M, g.L, Ut[N - 1], RtL, X1, parts, grid); break;
    case 3: rc = launch_last<TY, T, 3>(ctx, Y, g.M, g.L, Ut[N - 1], RtL, X1, parts, grid); break;
    case 4: rc = launch_last<TY, T, 4>(ctx, Y, g.M, g.L, Ut[N - 1], RtL, X1, parts, grid); break;
    default: return TDK_EINVAL;
  }
  if (rc) return rc;
  if (normY2) {
    sum_parts_kernel<<<1, 256, 0, ctx->stream>>>(parts, grid, normY2);
    TDK_LAUNCH_CHECK(ctx);
  }
  return core_chain_rest<T>(ctx, g, X1, Ut, reinterpret_cast<T*>(Gv), tmp0, tmp1, spl, pcap, open0 ? 1 : 0);
}

int core_simt(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const U[], void* G,
              double* normY2, int open0) {
  switch (dtype) {
    case TDK_F64: return core_simt_t<double, double>(ctx, g, Y, U, G, normY2, open0);
    case TDK_F32: return core_simt_t<float, float>(ctx, g, Y, U, G, normY2, open0);
    case TDK_BF16: return core_simt_t<__nv_bfloat16, float>(ctx, g, Y, U, G, normY2, open0);
  }
  return TDK_EINVAL;
}

}  // namespace tdk

namespace tdk {
TDK_CHECKED_UNIT(core_simt)
}  // namespace tdk
