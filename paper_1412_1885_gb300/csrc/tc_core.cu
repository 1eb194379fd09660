// Tensor-core (tcgen05) first contraction of the core chain (Alg. 2, the
// first "Y <- Y x_n U^T", taken over the contiguous mode N):
//   X_1[row, r] = sum_k Y[row, k] U_N[k, r],   row = (i_1..i_{N-1}),
// plus ||Y||^2.  Y streams through shared memory by TMA (128-byte swizzle);
// the B operand is [U_hi | U_lo] in BF16 so that products keep ~16
// significant bits (FP32 data are also split hi + lo in place by converter
// warps, two MMAs per step).  A CTA tile is MT sub-tiles of 128 rows that share each staged U
// tile; accumulators live in TMEM (double-buffered per tile so the epilogue
// overlaps the next tile's MMAs).  ||Y||^2 is summed by the threads that
// already touch the data (the epilogue warps for BF16, the converters for
// FP32).  The remaining, shrunken contractions run on CUDA cores.
#include <algorithm>

#include "tc_common.cuh"

namespace tdk {

template <class T>
int core_chain_rest(tdk_ctx* ctx, const Geom& g, const T* X1, T* const Ut[], T* G, T* tmp0, T* tmp1);

namespace {

using namespace tc;

constexpr int KB = 1024;
constexpr uint32_t BOX_BYTES = 16 * KB;  // one 128-row x 128-byte box

struct CoArgs {
  int64_t M;     // rows
  int L;         // contiguous mode
  int KC;        // 64-column chunks
  int NB;        // B rows: Rtp (BF16 data) or 2 * Rtp (hi | lo, FP32 data)
  int Rt, Rtp;
  int hilo;
  int tmem_cols;  // power of two >= 2 * MT * NB
  int64_t ntiles;
  float* X;      // [M][Rt]
  double* nrm_part;
  unsigned* status;
};

template <bool F32, int MT>
struct CoLayout {
  static constexpr int STAGES = 4;
  static constexpr uint32_t SUB_BYTES = F32 ? 32 * KB : 16 * KB;  // one 128-row sub-tile x 64 columns
  static constexpr uint32_t Y_BYTES = MT * SUB_BYTES;
  static constexpr int THREADS = F32 ? 320 : 192;
};

template <bool F32, int MT>
__global__ void __launch_bounds__(CoLayout<F32, MT>::THREADS, 1)
    tc_core_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmU, const CoArgs a) {
  using Lay = CoLayout<F32, MT>;
  constexpr int S = Lay::STAGES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned start, by offset so that the pointer stays in the shared space
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t b_bytes = (uint32_t)a.NB * 128u;
  const uint32_t stage_bytes = Lay::Y_BYTES + ((b_bytes + 1023) & ~1023u);
  const uint32_t dcols = (uint32_t)MT * a.NB;  // TMEM columns per accumulator buffer
  unsigned char* st_base = base;
  uint64_t* bars = reinterpret_cast<uint64_t*>(st_base + S * stage_bytes);
  uint64_t* full = bars;            // [S]
  uint64_t* empty = bars + S;       // [S]
  uint64_t* cfull = bars + 2 * S;   // [S]
  uint64_t* dfull = bars + 3 * S;   // [2]
  uint64_t* dempty = bars + 3 * S + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * S + 4);
  double* nred = reinterpret_cast<double*>(bars + 3 * S + 6);  // [10]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), F32 ? 1 : 5);
      mbar_init(smem_u32(&cfull[i]), 4);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&dfull[i]), 1);
      mbar_init(smem_u32(&dempty[i]), 4);
    }
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  unsigned* status = a.status;
  bool ok = true;
  float nrm = 0.f, nrm_c = 0.f;  // Kahan sum of y^2 over the rows this thread reads

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      prefetch_tmap(&tmY);
      prefetch_tmap(&tmU);
      uint32_t it = 0;
      for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        for (int kc = 0; kc < a.KC; ++kc, ++it) {
          const int s = it % S;
          const uint32_t n = it / S;
          if (!mbar_wait(smem_u32(&empty[s]), (n & 1) ^ 1, status)) { ok = false; break; }
          unsigned char* dst = st_base + s * stage_bytes;
          mbar_expect_tx(smem_u32(&full[s]), Lay::Y_BYTES + b_bytes);
#pragma unroll
          for (int m = 0; m < MT; ++m) {
            const int row = (int)(t * 128 * MT + 128 * m);
            unsigned char* sub = dst + m * Lay::SUB_BYTES;
            tma_load_3d(smem_u32(sub), &tmY, kc * 64, row, 0, smem_u32(&full[s]));
            if (F32) tma_load_3d(smem_u32(sub + BOX_BYTES), &tmY, kc * 64 + 32, row, 0, smem_u32(&full[s]));
          }
          tma_load_3d(smem_u32(dst + Lay::Y_BYTES), &tmU, kc * 64, 0, 0, smem_u32(&full[s]));
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id = idesc_bf16(128, a.NB, 0, 0);
      uint32_t it = 0, tl = 0;
      for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tl) {
        const int db = tl & 1;
        if (!mbar_wait(smem_u32(&dempty[db]), ((tl >> 1) & 1) ^ 1, status)) { ok = false; break; }
        tc_fence_after();
        for (int kc = 0; kc < a.KC; ++kc, ++it) {
          const int s = it % S;
          const uint32_t n = it / S;
          if (!mbar_wait(smem_u32(F32 ? &cfull[s] : &full[s]), n & 1, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sb = smem_u32(st_base + s * stage_bytes);
          const uint32_t bb = sb + Lay::Y_BYTES;
#pragma unroll
          for (int m = 0; m < MT; ++m) {
            const uint32_t d = tmem + db * dcols + m * a.NB;
            const uint32_t ab = sb + m * Lay::SUB_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t bd = smem_desc(bb + kk * 32, 16, 1024, SW128);
              mma_bf16(d, smem_desc(ab + kk * 32, 16, 1024, SW128), bd, id, (kc | kk) != 0);
              if (F32) mma_bf16(d, smem_desc(ab + BOX_BYTES + kk * 32, 16, 1024, SW128), bd, id, 1);
            }
          }
          umma_commit(smem_u32(&empty[s]));
        }
        umma_commit(smem_u32(&dfull[db]));
      }
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int rl = 32 * q + lane;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    uint32_t it = 0, tl = 0;
    for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tl) {
      if (!F32) {
        for (int kc = 0; kc < a.KC; ++kc, ++it) {
          const int s = it % S;
          const uint32_t n = it / S;
          if (!mbar_wait(smem_u32(&full[s]), n & 1, status)) { ok = false; break; }
          float part = 0.f;
#pragma unroll
          for (int m = 0; m < MT; ++m) {
            const unsigned char* row = st_base + s * stage_bytes + m * Lay::SUB_BYTES + rl * 128;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              // walk the chunks in swizzled order: 8 consecutive rows then hit 8 distinct bank groups
              const uint4 w = *reinterpret_cast<const uint4*>(row + ((c ^ (rl & 7)) << 4));
              const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float lo = __uint_as_float(ws[e] << 16), hi = __uint_as_float(ws[e] & 0xFFFF0000u);
                part = fmaf(lo, lo, part);
                part = fmaf(hi, hi, part);
              }
            }
          }
          const float y = part - nrm_c;
          const float tt = nrm + y;
          nrm_c = (tt - nrm) - y;
          nrm = tt;
          // the stage is refilled by TMA (async proxy): order these generic reads first
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
        }
        if (!ok) break;
      }
      const int db = tl & 1;
      if (!mbar_wait(smem_u32(&dfull[db]), (tl >> 1) & 1, status)) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        float v[128];
#pragma unroll
        for (int c16 = 0; c16 < 8; ++c16)
          if (c16 * 16 < a.NB) tmem_ld16(tmem + db * dcols + m * a.NB + c16 * 16 + lane_addr, v + c16 * 16);
        tmem_wait_ld();
        if (m == MT - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&dempty[db]));
        }
        const int64_t row = (t * MT + m) * 128 + rl;
        if (row < a.M) {
          float* xr = a.X + row * a.Rt;
#pragma unroll
          for (int r = 0; r < 64; ++r) {
            if (r < a.Rt) {
              float x = v[r];
              if (a.hilo) {
#pragma unroll
                for (int h = 16; h <= 64; h += 16)
                  if (a.Rtp == h) x += v[h + r];
              }
              xr[r] = x;
            }
          }
        }
      }
    }
  } else if (F32) {
    // ------------------------------------------------------------ converters (FP32 data)
    const int q = warp - 6;
    const int r = 32 * q + lane;
    uint32_t it = 0;
    for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
      for (int kc = 0; kc < a.KC; ++kc, ++it) {
        const int s = it % S;
        const uint32_t n = it / S;
        if (!mbar_wait(smem_u32(&full[s]), n & 1, status)) { ok = false; break; }
        unsigned char* sb = st_base + s * stage_bytes;
        float part = 0.f;
#pragma unroll
        for (int m = 0; m < MT; ++m)
          part += split_row64(sb + m * Lay::SUB_BYTES + r * 128, sb + m * Lay::SUB_BYTES + BOX_BYTES + r * 128, r);
        const float y = part - nrm_c;
        const float tt = nrm + y;
        nrm_c = (tt - nrm) - y;
        nrm = tt;
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&cfull[s]));
      }
    }
  }
  // per-CTA ||Y||^2 from the threads that read the tiles
  double mine = (double)nrm - (double)nrm_c;
  mine = warp_sum(mine);
  if (lane == 0) nred[warp] = mine;
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += nred[w];
    a.nrm_part[blockIdx.x] = s;
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

// U_N^T as BF16 rows (channel-major, columns = L padded to ldu): rows [0, Rtp)
// hold the nearest BF16 of U; with hilo, rows [Rtp, 2 Rtp) hold the remainder
__global__ void build_u_bf16(const double* __restrict__ U, int L, int Rt, int Rtp, int hilo, int ldu,
                             __nv_bfloat16* __restrict__ out) {
  const int64_t total = (int64_t)(hilo ? 2 : 1) * Rtp * ldu;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / ldu);
    const int k = (int)(e % ldu);
    const int r = c < Rtp ? c : c - Rtp;
    float v = 0.f;
    if (r < Rt && k < L) {
      const double x = U[(int64_t)k * Rt + r];
      const float hi = __bfloat162float(__float2bfloat16_rn((float)x));
      v = (c < Rtp) ? hi : (float)(x - (double)hi);
    }
    out[e] = __float2bfloat16_rn(v);
  }
}

__global__ void sum_doubles(const double* __restrict__ parts, int n, double* __restrict__ out) {
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

__global__ void cvt_u(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (float)s[e];
}

template <bool F32, int MT>
int launch_core(tdk_ctx* ctx, const CUtensorMap& tmY, const CUtensorMap& tmU, const CoArgs& a, int grid) {
  using Lay = CoLayout<F32, MT>;
  const uint32_t stage = Lay::Y_BYTES + ((a.NB * 128 + 1023) & ~1023);
  const size_t smem = 1024 + (size_t)Lay::STAGES * stage + 8 * (3 * Lay::STAGES + 6) + 8 * 16;
  if (smem > (size_t)ctx->max_smem_optin) return TDK_ENOTSUP;
  auto k = tc_core_kernel<F32, MT>;
  TDK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(ctx, 1);
  k<<<grid, Lay::THREADS, smem, ctx->stream>>>(tmY, tmU, a);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // namespace

int core_tc(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const U[], void* Gv,
            double* normY2) {
  if (!tc_shape_ok(g, dtype) || dtype == TDK_F64) return TDK_ENOTSUP;
  const bool f32 = dtype == TDK_F32;
  constexpr int MT_BF16 = 2, MT_F32 = 1;
  const int MT = f32 ? MT_F32 : MT_BF16;
  const int N = g.N;
  CoArgs a{};
  a.M = g.M;
  a.L = (int)g.L;
  a.KC = (a.L + 63) / 64;
  a.Rt = g.Rt[N - 1];
  a.Rtp = (a.Rt + 15) / 16 * 16;
  // U split hi + lo for both data types: the first-order error of a single
  // BF16 rounding of U would show in ||Y||^2 - ||G||^2 (the reconstruction
  // error by Pythagoras)
  a.hilo = 1;
  a.NB = a.hilo ? 2 * a.Rtp : a.Rtp;
  a.tmem_cols = 32;
  while (a.tmem_cols < 2 * MT * a.NB) a.tmem_cols *= 2;
  if (a.tmem_cols > 512) return TDK_ENOTSUP;  // two accumulator buffers of MT x NB columns
  a.ntiles = (g.M + 128 * MT - 1) / (128 * MT);
  a.status = ctx->d_status;
  const int grid = (int)std::min<int64_t>(a.ntiles, ctx->num_sms);
  const int ldu = (a.L + 7) / 8 * 8;
  int64_t tmpsz = 0;
  {
    int64_t Bd = a.Rt;
    for (int m = N - 2; m >= 1; --m) {
      int64_t A = 1;
      for (int k = 0; k < m; ++k) A *= g.I[k];
      tmpsz = std::max<int64_t>(tmpsz, A * g.Rt[m] * Bd);
      Bd *= g.Rt[m];
    }
  }
  Planner pl;
  pl.take<__nv_bfloat16>((size_t)a.NB * ldu);
  for (int n = 0; n < N; ++n) pl.take<float>((size_t)g.I[n] * g.Rt[n]);
  pl.take<float>((size_t)g.M * a.Rt);
  pl.take<float>((size_t)tmpsz);
  pl.take<float>((size_t)tmpsz);
  pl.take<double>((size_t)grid);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  __nv_bfloat16* ub = cv.take<__nv_bfloat16>((size_t)a.NB * ldu);
  build_u_bf16<<<128, 256, 0, ctx->stream>>>(U[N - 1], a.L, a.Rt, a.Rtp, a.hilo, ldu, ub);
  TDK_LAUNCH_CHECK(ctx);
  float* Ut[TDK_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    Ut[n] = cv.take<float>((size_t)g.I[n] * g.Rt[n]);
    cvt_u<<<64, 256, 0, ctx->stream>>>(U[n], Ut[n], g.I[n] * g.Rt[n]);
    TDK_LAUNCH_CHECK(ctx);
  }
  a.X = cv.take<float>((size_t)g.M * a.Rt);
  float* tmp0 = cv.take<float>((size_t)tmpsz);
  float* tmp1 = cv.take<float>((size_t)tmpsz);
  a.nrm_part = cv.take<double>((size_t)grid);

  CUtensorMap tmY, tmU;
  {
    const int es = f32 ? 4 : 2;
    uint64_t dims[3] = {(uint64_t)a.L, (uint64_t)g.M, 1};
    uint64_t str[2] = {(uint64_t)a.L * es, (uint64_t)a.L * es * (uint64_t)g.M};
    uint32_t box[3] = {f32 ? 32u : 64u, 128u, 1u};
    rc = encode_tmap(&tmY, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Y, dims,
                     str, box, true);
    if (rc) return rc;
    uint64_t ud[3] = {(uint64_t)a.L, (uint64_t)a.NB, 1};
    uint64_t us[2] = {(uint64_t)ldu * 2, (uint64_t)ldu * 2 * a.NB};
    uint32_t ubx[3] = {64u, (uint32_t)a.NB, 1u};
    rc = encode_tmap(&tmU, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ub, ud, us, ubx, true);
    if (rc) return rc;
  }
  rc = f32 ? launch_core<true, MT_F32>(ctx, tmY, tmU, a, grid) : launch_core<false, MT_BF16>(ctx, tmY, tmU, a, grid);
  if (rc) return rc;
  if (normY2) {
    sum_doubles<<<1, 256, 0, ctx->stream>>>(a.nrm_part, grid, normY2);
    TDK_LAUNCH_CHECK(ctx);
  }
  return core_chain_rest<float>(ctx, g, a.X, Ut, reinterpret_cast<float*>(Gv), tmp0, tmp1);
}

}  // namespace tdk
