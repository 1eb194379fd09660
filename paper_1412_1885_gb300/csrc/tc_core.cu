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
int core_chain_rest(tdk_ctx* ctx, const Geom& g, const T* X1, T* const Ut[], T* G, T* tmp0, T* tmp1, T* part,
                    int64_t part_cap, int m_stop);
template <class T>
int core_chain_from(tdk_ctx* ctx, const Geom& g, const T* X, int m0, T* const Ut[], T* G, T* tmp0, T* tmp1,
                    T* part, int64_t part_cap, int m_stop);

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
            if (r < a.Rt && TDK_IN(row * a.Rt + r, a.M * a.Rt)) {
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

// ---------------------------------------------------------------------------
// Contraction of the leading mode (BF16 data): Alg. 2's first
// "Y <- Y x_1 U_1^T", and the projection shared by the later modes of a
// RandTucker2i pass (Alg. 3).  Y is read as [I_1][B] (B = the product of the
// other dimensions, contiguous) and
//   X[r, b] = sum_i U_1[i, r] Y[i, b].
// A CTA tile is LD_MT sub-tiles of 128 columns b.  The MMA reads the Y tile as
// its A operand MN-major (M = 128 columns b in two 64-column boxes, K = 16
// rows i per step) and [U_hi | U_lo]^T as the K-major B operand (N = 2 Rtp),
// so D[b, c] holds the hi products in columns c < Rtp and the lo ones at
// Rtp + c; the epilogue adds the two and writes X[r, b], coalesced over b.
// Rows i past I_1 and columns b past B arrive as zeros from TMA.
struct LdArgs {
  int64_t B;     // columns
  int KC;        // 64-row chunks of I_1
  int NB, Rt, Rtp;
  int tmem_cols;
  int64_t ntiles;
  float* X;      // [Rt][B]
  unsigned* status;
};

constexpr int LD_S = 4;                  // stage ring
constexpr int LD_MT = 2;                 // 128-column sub-tiles per CTA tile
constexpr uint32_t LD_BOX = 8 * KB;      // 64 rows i x 64 columns b
constexpr uint32_t LD_SUB = 2 * LD_BOX;  // one 128-column sub-tile
constexpr int LD_THREADS = 192;

__host__ __device__ inline uint32_t ld_stage_bytes(int NB) {
  return LD_MT * LD_SUB + (((uint32_t)NB * 128u + 1023u) & ~1023u);
}
inline size_t ld_smem_bytes(int NB) { return 1024 + (size_t)LD_S * ld_stage_bytes(NB) + 8 * (2 * LD_S + 4) + 16; }

__global__ void __launch_bounds__(LD_THREADS, 1)
    tc_ttm_lead_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmU,
                       const LdArgs a) {
  constexpr int S = LD_S;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t b_bytes = (uint32_t)a.NB * 128u;
  const uint32_t stage_bytes = ld_stage_bytes(a.NB);
  const uint32_t dcols = (uint32_t)LD_MT * a.NB;  // TMEM columns per accumulator buffer
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + S * stage_bytes);
  uint64_t* full = bars;            // [S]
  uint64_t* empty = bars + S;       // [S]
  uint64_t* dfull = bars + 2 * S;   // [2]
  uint64_t* dempty = dfull + 2;     // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), 1);
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
          unsigned char* dst = base + s * stage_bytes;
          mbar_expect_tx(smem_u32(&full[s]), LD_MT * LD_SUB + b_bytes);
#pragma unroll
          for (int m = 0; m < LD_MT; ++m)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              // x = a multiple of 64 columns (128 bytes)
              const int col = (int)(t * 128 * LD_MT + 128 * m + 64 * h);
              tma_load_2d(smem_u32(dst + m * LD_SUB + h * LD_BOX), &tmY, col, kc * 64, smem_u32(&full[s]));
            }
          tma_load_2d(smem_u32(dst + LD_MT * LD_SUB), &tmU, kc * 64, 0, smem_u32(&full[s]));
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id = idesc_bf16(128, a.NB, 1, 0);  // A MN-major (Y tile), B K-major (U^T)
      uint32_t it = 0, tl = 0;
      for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tl) {
        const int db = tl & 1;
        if (!mbar_wait(smem_u32(&dempty[db]), ((tl >> 1) & 1) ^ 1, status)) { ok = false; break; }
        tc_fence_after();
        for (int kc = 0; kc < a.KC; ++kc, ++it) {
          const int s = it % S;
          const uint32_t n = it / S;
          if (!mbar_wait(smem_u32(&full[s]), n & 1, status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sb = smem_u32(base + s * stage_bytes);
          const uint32_t bb = sb + LD_MT * LD_SUB;
#pragma unroll
          for (int m = 0; m < LD_MT; ++m) {
            const uint32_t d = tmem + db * dcols + m * a.NB;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // A: 16 rows i (2048 bytes) per step, the two 64-column boxes LD_BOX apart
              const uint64_t ad = smem_desc(sb + m * LD_SUB + kk * 2048, LD_BOX, 1024, SW128);
              const uint64_t bd = smem_desc(bb + kk * 32, 16, 1024, SW128);
              mma_bf16(d, ad, bd, id, (kc | kk) != 0);
            }
          }
          umma_commit(smem_u32(&empty[s]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&dfull[db]));
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int q = warp & 3;
    const int bl = 32 * q + lane;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    uint32_t tl = 0;
    for (int64_t t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tl) {
      const int db = tl & 1;
      if (!mbar_wait(smem_u32(&dfull[db]), (tl >> 1) & 1, status)) { ok = false; break; }
      tc_fence_after();
#pragma unroll 1
      for (int m = 0; m < LD_MT; ++m) {
        float v[128];
#pragma unroll
        for (int c16 = 0; c16 < 8; ++c16)
          if (c16 * 16 < a.NB) tmem_ld16(tmem + db * dcols + m * a.NB + c16 * 16 + lane_addr, v + c16 * 16);
        tmem_wait_ld();
        if (m == LD_MT - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&dempty[db]));
        }
        const int64_t b = (t * LD_MT + m) * 128 + bl;
        if (b < a.B) {
#pragma unroll
          for (int r = 0; r < 64; ++r) {
            if (r < a.Rt) {
              float x = v[r];
#pragma unroll
              for (int h = 16; h <= 64; h += 16)
                if (a.Rtp == h) x += v[h + r];
              if (TDK_IN((int64_t)r * a.B + b, (int64_t)a.Rt * a.B)) a.X[(int64_t)r * a.B + b] = x;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

// ---------------------------------------------------------------------------
// Fused first two contractions (BF16 data).  Y is read as [P][J][L] (L = I_N,
// J = I_{N-1}, P = prod of the other modes); a work item is one p, its tiles
// the 128-row blocks of j.  Per tile, D1 = X_1 rows (as above) and then a
// second product on the tensor cores,
//   D2[s, r] += sum_j U_{N-1}[j, s] X_1[p, j, r],
// accumulated in TMEM over the tiles of p, so X_1 never leaves the SM.  Both
// operands of the second product are split hi + lo (A: rows 0..63 the hi and
// 64..127 the lo part of U_{N-1}^T; B: columns 0..63 hi and 64..127 lo of the
// X_1 tile, written by the epilogue), so D2 holds the four partial products
// and X_2[p, s, r] is their sum.  The second product of a tile is issued after
// the first product of the next tile, so the MMA issuer never waits for the
// epilogue.
struct FuArgs {
  int L, KC, NB, Rt, Rtp;  // contiguous mode, as CoArgs
  int J, JT;               // I_{N-1} and its 128-row tiles
  int P;                   // work items
  int Rt2;                 // sketch width of mode N-1
  float* X2;               // [P][Rt2][Rt]
  double* nrm_part;
  unsigned* status;
  int want_norm;           // 0: no ||Y||^2, the MMA commit alone frees a stage
};

constexpr int FU_S = 4;                 // stage ring
constexpr uint32_t FU_Y = 16 * KB;      // 128 rows x 64 columns BF16
constexpr int FU_THREADS = 192;
constexpr int FU_SCR_LD = 65;           // padded row of the exchange buffer (floats)

inline size_t fused_smem_bytes(int NB) {
  const size_t stage = FU_Y + ((size_t)(NB * 128 + 1023) & ~size_t(1023));
  return 1024 + FU_S * stage + 64 * KB + (size_t)64 * FU_SCR_LD * 4 + 256;
}

__global__ void __launch_bounds__(FU_THREADS, 1)
    tc_core_fused_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmU,
                         const __grid_constant__ CUtensorMap tmV, const FuArgs a) {
  constexpr int S = FU_S;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t b_bytes = (uint32_t)a.NB * 128u;
  const uint32_t stage_bytes = FU_Y + ((b_bytes + 1023) & ~1023u);
  unsigned char* st_base = base;                      // S x (Y tile | U_N tile)
  unsigned char* v_base = base + S * stage_bytes;     // U_{N-1} rows of the tile: two 16 KB boxes (hi, lo)
  unsigned char* x_base = v_base + 32 * KB;           // X_1 tile: two 16 KB boxes (hi, lo)
  float* scr = reinterpret_cast<float*>(x_base + 32 * KB);  // [64][FU_SCR_LD] lo-row partials of D2
  uint64_t* bars = reinterpret_cast<uint64_t*>(scr + 64 * FU_SCR_LD);
  uint64_t* full = bars;           // [S]
  uint64_t* empty = bars + S;      // [S]
  uint64_t* dfull = bars + 2 * S;  // [2]
  uint64_t* dempty = dfull + 2;    // [2]
  uint64_t* vfull = dfull + 4;
  uint64_t* vempty = vfull + 1;
  uint64_t* xfull = vfull + 2;
  uint64_t* xempty = vfull + 3;
  uint64_t* d2full = vfull + 4;
  uint64_t* d2empty = vfull + 5;
  uint64_t* sfull = vfull + 6;
  uint64_t* sempty = vfull + 7;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(vfull + 8);
  double* nred = reinterpret_cast<double*>(vfull + 10);  // [6]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      // the MMA commit, and the four epilogue warps when they sum ||Y||^2
      mbar_init(smem_u32(&empty[i]), a.want_norm ? 5 : 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&dfull[i]), 1);
      mbar_init(smem_u32(&dempty[i]), 4);
    }
    mbar_init(smem_u32(vfull), 1);
    mbar_init(smem_u32(vempty), 1);
    mbar_init(smem_u32(xfull), 4);
    mbar_init(smem_u32(xempty), 1);
    mbar_init(smem_u32(d2full), 1);
    mbar_init(smem_u32(d2empty), 4);
    mbar_init(smem_u32(sfull), 2);
    mbar_init(smem_u32(sempty), 2);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t d2col = 256;  // D1 buffers at columns [0, NB) and [NB, 2 NB), NB <= 128
  unsigned* status = a.status;
  bool ok = true;
  float nrm = 0.f, nrm_c = 0.f;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      prefetch_tmap(&tmY);
      prefetch_tmap(&tmU);
      prefetch_tmap(&tmV);
      // the U_{N-1} rows of tile t are loaded while the next tile streams in,
      // once the second product of tile t-1 has read the single V buffer: after
      // stage vk of the next tile, whose slot was freed by an MMA issued after
      // that product, so the wait is normally already satisfied
      auto load_v = [&](uint32_t t, int jt) -> bool {
        if (!mbar_wait(smem_u32(vempty), (t & 1) ^ 1, status)) return false;
        mbar_expect_tx(smem_u32(vfull), 32 * KB);
        tma_load_3d(smem_u32(v_base), &tmV, 0, jt * 128, 0, smem_u32(vfull));
        tma_load_3d(smem_u32(v_base + 16 * KB), &tmV, 64, jt * 128, 0, smem_u32(vfull));
        return true;
      };
      const int vk = a.KC - 1 < S ? a.KC - 1 : S;
      bool vp = false;
      uint32_t vtl = 0;
      int vjt = 0;
      uint32_t it = 0, tl = 0;
      for (int p = blockIdx.x; p < a.P && ok; p += gridDim.x) {
        for (int jt = 0; jt < a.JT; ++jt, ++tl) {
          for (int kc = 0; kc < a.KC; ++kc, ++it) {
            const int s = it % S;
            const uint32_t n = it / S;
            if (!mbar_wait(smem_u32(&empty[s]), (n & 1) ^ 1, status)) { ok = false; break; }
            unsigned char* dst = st_base + s * stage_bytes;
            mbar_expect_tx(smem_u32(&full[s]), FU_Y + b_bytes);
            tma_load_3d(smem_u32(dst), &tmY, kc * 64, jt * 128, p, smem_u32(&full[s]));
            tma_load_3d(smem_u32(dst + FU_Y), &tmU, kc * 64, 0, 0, smem_u32(&full[s]));
            if (kc == vk && vp) {
              if (!load_v(vtl, vjt)) { ok = false; break; }
              vp = false;
            }
          }
          if (!ok) break;
          vp = true;
          vtl = tl;
          vjt = jt;
        }
      }
      if (ok && vp && !load_v(vtl, vjt)) ok = false;
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id1 = idesc_bf16(128, a.NB, 0, 0);
      const uint32_t id2 = idesc_bf16(128, 128, 1, 1);
      // second product of tile t2 (of item number u2): D2 += V^T X
      auto second = [&](uint32_t t2, uint32_t u2, bool first, bool last) -> bool {
        if (first && !mbar_wait(smem_u32(d2empty), (u2 & 1) ^ 1, status)) return false;
        if (!mbar_wait(smem_u32(vfull), t2 & 1, status)) return false;
        if (!mbar_wait(smem_u32(xfull), t2 & 1, status)) return false;
        tc_fence_after();
        const uint32_t va = smem_u32(v_base), xa = smem_u32(x_base);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          mma_bf16(tmem + d2col, smem_desc(va + kk * 2048, 16 * KB, 1024, SW128),
                   smem_desc(xa + kk * 2048, 16 * KB, 1024, SW128), id2, !(first && kk == 0));
        umma_commit(smem_u32(vempty));
        umma_commit(smem_u32(xempty));
        if (last) umma_commit(smem_u32(d2full));
        return true;
      };
      uint32_t it = 0, tl = 0, ui = 0;
      bool pend = false, pfirst = false, plast = false;
      uint32_t ptl = 0, pui = 0;
      for (int p = blockIdx.x; p < a.P && ok; p += gridDim.x, ++ui) {
        for (int jt = 0; jt < a.JT; ++jt, ++tl) {
          const int db = tl & 1;
          if (!mbar_wait(smem_u32(&dempty[db]), ((tl >> 1) & 1) ^ 1, status)) { ok = false; break; }
          tc_fence_after();
          for (int kc = 0; kc < a.KC; ++kc, ++it) {
            const int s = it % S;
            const uint32_t n = it / S;
            if (!mbar_wait(smem_u32(&full[s]), n & 1, status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sb = smem_u32(st_base + s * stage_bytes);
            const uint32_t bb = sb + FU_Y;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(tmem + db * a.NB, smem_desc(sb + kk * 32, 16, 1024, SW128),
                       smem_desc(bb + kk * 32, 16, 1024, SW128), id1, (kc | kk) != 0);
            umma_commit(smem_u32(&empty[s]));
          }
          if (!ok) break;
          umma_commit(smem_u32(&dfull[db]));
          if (pend && !second(ptl, pui, pfirst, plast)) { ok = false; break; }
          pend = true;
          ptl = tl;
          pui = ui;
          pfirst = jt == 0;
          plast = jt == a.JT - 1;
        }
      }
      if (ok && pend && !second(ptl, pui, pfirst, plast)) ok = false;
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2-5)
    const int q = warp & 3;
    const int rl = 32 * q + lane;  // TMEM lane: tile row j (D1), row of V^T (D2)
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    const bool upper = q >= 2;     // D2 rows 64..127: the lo part of U_{N-1}
    // X_2[p] = the four quadrants of D2 (rows s (hi) and 64 + s (lo), columns r
    // and 64 + r).  Run after the next tile's stages have been read, so that the
    // stage ring keeps moving while the issuer still has the first product of
    // that tile ahead of this item's last second product.
    auto finalise = [&](int fp, uint32_t fu) -> bool {
      if (!mbar_wait(smem_u32(d2full), fu & 1, status)) return false;
      tc_fence_after();
      float y[64];  // this row's hi-column plus lo-column products
#pragma unroll
      for (int c16 = 0; c16 < 4; ++c16) {
        float t0[16], t1[16];
        tmem_ld16(tmem + d2col + c16 * 16 + lane_addr, t0);
        tmem_ld16(tmem + d2col + 64 + c16 * 16 + lane_addr, t1);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 16; ++e) y[c16 * 16 + e] = t0[e] + t1[e];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(d2empty));
      if (upper) {
        if (!mbar_wait(smem_u32(sempty), (fu & 1) ^ 1, status)) return false;
        float* sr = scr + (rl - 64) * FU_SCR_LD;
#pragma unroll
        for (int r = 0; r < 64; ++r) sr[r] = y[r];
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(sfull));
      } else {
        if (!mbar_wait(smem_u32(sfull), fu & 1, status)) return false;
        const float* sr = scr + rl * FU_SCR_LD;
        if (rl < a.Rt2) {
          const int64_t o = ((int64_t)fp * a.Rt2 + rl) * a.Rt;
          float* out = a.X2 + o;
#pragma unroll
          for (int r = 0; r < 64; ++r)
            if (r < a.Rt && TDK_IN(o + r, (int64_t)a.P * a.Rt2 * a.Rt)) out[r] = y[r] + sr[r];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(sempty));
      }
      return true;
    };
    bool fin = false;
    int fin_p = 0;
    uint32_t fin_u = 0;
    uint32_t it = 0, tl = 0, ui = 0;
    for (int p = blockIdx.x; p < a.P && ok; p += gridDim.x, ++ui) {
      for (int jt = 0; jt < a.JT; ++jt, ++tl) {
        // ||Y||^2 from the staged tiles
        if (!a.want_norm) it += a.KC;
        for (int kc = 0; kc < a.KC && a.want_norm; ++kc, ++it) {
          const int s = it % S;
          const uint32_t n = it / S;
          if (!mbar_wait(smem_u32(&full[s]), n & 1, status)) { ok = false; break; }
          float part = 0.f;
          const unsigned char* row = st_base + s * stage_bytes + rl * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint4 w = *reinterpret_cast<const uint4*>(row + ((c ^ (rl & 7)) << 4));
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float lo = __uint_as_float(ws[e] << 16), hi = __uint_as_float(ws[e] & 0xFFFF0000u);
              part = fmaf(lo, lo, part);
              part = fmaf(hi, hi, part);
            }
          }
          const float y = part - nrm_c;
          const float tt = nrm + y;
          nrm_c = (tt - nrm) - y;
          nrm = tt;
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
        }
        if (!ok) break;
        if (fin) {
          if (!finalise(fin_p, fin_u)) { ok = false; break; }
          fin = false;
        }
        // X_1 row j = rl of this tile (sum of the U_hi and U_lo columns of D1)
        const int db = tl & 1;
        if (!mbar_wait(smem_u32(&dfull[db]), (tl >> 1) & 1, status)) { ok = false; break; }
        tc_fence_after();
        float xr[128];  // D1 row; its first 64 entries become the X_1 row
#pragma unroll
        for (int c16 = 0; c16 < 8; ++c16)
          if (c16 * 16 < a.NB) tmem_ld16(tmem + db * a.NB + c16 * 16 + lane_addr, xr + c16 * 16);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&dempty[db]));
        // in increasing r, so that each read column Rtp + r > r is still unwritten
#pragma unroll
        for (int r = 0; r < 64; ++r) {
          float x = 0.f;
          if (r < a.Rt) {
            x = xr[r];
#pragma unroll
            for (int h = 16; h <= 64; h += 16)
              if (a.Rtp == h) x += xr[h + r];
          }
          xr[r] = x;
        }
        // B operand of the second product: row j, hi part in box 0, lo part in box 1
        if (!mbar_wait(smem_u32(xempty), (tl & 1) ^ 1, status)) { ok = false; break; }
        {
          unsigned char* rowh = x_base + rl * 128;
          const int ph = rl & 7;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint32_t wh[4], wl[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float x0 = xr[8 * c + 2 * e], x1 = xr[8 * c + 2 * e + 1];
              const float h0 = __bfloat162float(__float2bfloat16_rn(x0));
              const float h1 = __bfloat162float(__float2bfloat16_rn(x1));
              wh[e] = pack_bf16x2(h0, h1);
              wl[e] = pack_bf16x2(x0 - h0, x1 - h1);
            }
            *reinterpret_cast<uint4*>(rowh + ((c ^ ph) << 4)) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
            *reinterpret_cast<uint4*>(rowh + 16 * KB + ((c ^ ph) << 4)) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(xfull));
        if (jt == a.JT - 1) {
          fin = true;
          fin_p = p;
          fin_u = ui;
        }
      }
    }
    if (ok && fin && !finalise(fin_p, fin_u)) ok = false;
  }
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
    tmem_dealloc(tmem, 512);
  }
}

// U_{N-1} as the A operand rows of the second product: row j holds the
// nearest BF16 of U[j, s] at column s and the remainder at column 64 + s
__global__ void build_v_bf16(const double* __restrict__ U, int J, int Rt, __nv_bfloat16* __restrict__ out) {
  const int64_t total = (int64_t)J * 128;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / 128;
    const int c = (int)(e % 128);
    const int s = c & 63;
    float v = 0.f;
    if (s < Rt) {
      const double x = U[j * Rt + s];
      const float hi = __bfloat162float(__float2bfloat16_rn((float)x));
      v = (c < 64) ? hi : (float)(x - (double)hi);
    }
    out[e] = __float2bfloat16_rn(v);
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

// BF16 data, N >= 3: the fused first two contractions, then the rest of the
// chain from X_2 on CUDA cores
static int core_tc_fused(tdk_ctx* ctx, const Geom& g, const void* Y, const double* const U[], void* Gv,
                         double* normY2, int open0) {
  const int N = g.N;
  FuArgs a{};
  a.L = (int)g.L;
  a.KC = (a.L + 63) / 64;
  a.Rt = g.Rt[N - 1];
  a.Rtp = (a.Rt + 15) / 16 * 16;
  a.NB = 2 * a.Rtp;  // U_N split hi + lo
  a.J = (int)g.I[N - 2];
  a.JT = (a.J + 127) / 128;
  int64_t P = 1;
  for (int k = 0; k < N - 2; ++k) P *= g.I[k];
  if (P > (int64_t)0x7fffffff) return TDK_ENOTSUP;
  a.P = (int)P;
  a.Rt2 = g.Rt[N - 2];
  a.status = ctx->d_status;
  const size_t smem = fused_smem_bytes(a.NB);
  if (smem > (size_t)ctx->max_smem_optin) return TDK_ENOTSUP;
  const int grid = (int)std::min<int64_t>(P, ctx->num_sms);
  const int ldu = (a.L + 7) / 8 * 8;
  int64_t tmpsz = 1;
  {
    int64_t Bd = (int64_t)a.Rt * a.Rt2;
    for (int m = N - 3; m >= 1; --m) {
      int64_t A = 1;
      for (int k = 0; k < m; ++k) A *= g.I[k];
      tmpsz = std::max<int64_t>(tmpsz, A * g.Rt[m] * Bd);
      Bd *= g.Rt[m];
    }
  }
  Planner pl;
  pl.take<__nv_bfloat16>((size_t)a.NB * ldu);
  pl.take<__nv_bfloat16>((size_t)a.J * 128);
  for (int n = 0; n < N; ++n) pl.take<float>((size_t)g.I[n] * g.Rt[n]);
  pl.take<float>((size_t)P * a.Rt2 * a.Rt);
  pl.take<float>((size_t)tmpsz);
  pl.take<float>((size_t)tmpsz);
  pl.take<double>((size_t)grid);
  const int64_t pcap = chain_split_cap(g);
  pl.take<float>((size_t)pcap);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  __nv_bfloat16* ub = cv.take<__nv_bfloat16>((size_t)a.NB * ldu);
  build_u_bf16<<<128, 256, 0, ctx->stream>>>(U[N - 1], a.L, a.Rt, a.Rtp, 1, ldu, ub);
  TDK_LAUNCH_CHECK(ctx);
  __nv_bfloat16* vb = cv.take<__nv_bfloat16>((size_t)a.J * 128);
  build_v_bf16<<<128, 256, 0, ctx->stream>>>(U[N - 2], a.J, a.Rt2, vb);
  TDK_LAUNCH_CHECK(ctx);
  float* Ut[TDK_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    Ut[n] = cv.take<float>((size_t)g.I[n] * g.Rt[n]);
    if (n < N - 2 && !(open0 && n == 0)) {
      cvt_u<<<64, 256, 0, ctx->stream>>>(U[n], Ut[n], g.I[n] * g.Rt[n]);
      TDK_LAUNCH_CHECK(ctx);
    }
  }
  // with mode 0 open and N = 3, X_2 is the result itself
  a.X2 = (open0 && N == 3) ? reinterpret_cast<float*>(Gv) : cv.take<float>((size_t)P * a.Rt2 * a.Rt);
  float* tmp0 = cv.take<float>((size_t)tmpsz);
  float* tmp1 = cv.take<float>((size_t)tmpsz);
  a.want_norm = normY2 != nullptr;
  a.nrm_part = cv.take<double>((size_t)grid);
  float* spl = cv.take<float>((size_t)pcap);

  CUtensorMap tmY, tmU, tmV;
  {
    uint64_t dims[3] = {(uint64_t)a.L, (uint64_t)a.J, (uint64_t)P};
    uint64_t str[2] = {(uint64_t)a.L * 2, (uint64_t)a.L * 2 * (uint64_t)a.J};
    uint32_t box[3] = {64u, 128u, 1u};
    rc = encode_tmap(&tmY, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Y, dims, str, box, true);
    if (rc) return rc;
    uint64_t ud[3] = {(uint64_t)a.L, (uint64_t)a.NB, 1};
    uint64_t us[2] = {(uint64_t)ldu * 2, (uint64_t)ldu * 2 * a.NB};
    uint32_t ubx[3] = {64u, (uint32_t)a.NB, 1u};
    rc = encode_tmap(&tmU, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ub, ud, us, ubx, true);
    if (rc) return rc;
    uint64_t vd[3] = {128, (uint64_t)a.J, 1};
    uint64_t vs[2] = {256, 256 * (uint64_t)a.J};
    uint32_t vbx[3] = {64u, 128u, 1u};
    rc = encode_tmap(&tmV, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, vb, vd, vs, vbx, true);
    if (rc) return rc;
  }
  {
    TDK_CUDA_TRY(cudaFuncSetAttribute(tc_core_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(ctx, 1);
    tc_core_fused_kernel<<<grid, FU_THREADS, smem, ctx->stream>>>(tmY, tmU, tmV, a);
    TDK_LAUNCH_CHECK(ctx);
  }
  if (normY2) {
    sum_doubles<<<1, 256, 0, ctx->stream>>>(a.nrm_part, grid, normY2);
    TDK_LAUNCH_CHECK(ctx);
  }
  if (open0 && N == 3) return TDK_OK;
  return core_chain_from<float>(ctx, g, a.X2, N - 3, Ut, reinterpret_cast<float*>(Gv), tmp0, tmp1, spl, pcap,
                                open0 ? 1 : 0);
}

int core_tc(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const U[], void* Gv,
            double* normY2, int open0) {
  if (!tc_shape_ok(g, dtype) || dtype == TDK_F64) return TDK_ENOTSUP;
  if (dtype == TDK_BF16 && g.N >= 3) {
    const int rc = core_tc_fused(ctx, g, Y, U, Gv, normY2, open0);
    if (rc != TDK_ENOTSUP) return rc;
  }
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
  const int64_t pcap = chain_split_cap(g);
  pl.take<float>((size_t)pcap);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  __nv_bfloat16* ub = cv.take<__nv_bfloat16>((size_t)a.NB * ldu);
  build_u_bf16<<<128, 256, 0, ctx->stream>>>(U[N - 1], a.L, a.Rt, a.Rtp, a.hilo, ldu, ub);
  TDK_LAUNCH_CHECK(ctx);
  float* Ut[TDK_MAX_MODES];
  for (int n = 0; n < N; ++n) {
    Ut[n] = cv.take<float>((size_t)g.I[n] * g.Rt[n]);
    if (open0 && n == 0) continue;
    cvt_u<<<64, 256, 0, ctx->stream>>>(U[n], Ut[n], g.I[n] * g.Rt[n]);
    TDK_LAUNCH_CHECK(ctx);
  }
  a.X = cv.take<float>((size_t)g.M * a.Rt);
  float* tmp0 = cv.take<float>((size_t)tmpsz);
  float* tmp1 = cv.take<float>((size_t)tmpsz);
  a.nrm_part = cv.take<double>((size_t)grid);
  float* spl = cv.take<float>((size_t)pcap);

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
  return core_chain_rest<float>(ctx, g, a.X, Ut, reinterpret_cast<float*>(Gv), tmp0, tmp1, spl, pcap,
                               open0 ? 1 : 0);
}

int ttm_lead_tc(tdk_ctx* ctx, const Geom& g, const void* Y, const double* U1, float* X) {
  const int64_t I0 = g.I[0];
  const int64_t B = g.numel / I0;
  LdArgs a{};
  a.B = B;
  a.Rt = g.Rt[0];
  a.Rtp = (a.Rt + 15) / 16 * 16;
  a.NB = 2 * a.Rtp;  // U_1 split hi + lo
  // TMA: 16-byte row stride of Y; 32-bit coordinates of the last tile
  if (a.Rt > 64 || B % 8 != 0 || B + 128 * LD_MT > (int64_t)0x7fffffff || I0 > (int64_t)0x7fffffff)
    return TDK_ENOTSUP;
  a.KC = (int)((I0 + 63) / 64);
  a.tmem_cols = 32;
  while (a.tmem_cols < 2 * LD_MT * a.NB) a.tmem_cols *= 2;
  if (a.tmem_cols > 512) return TDK_ENOTSUP;
  const size_t smem = ld_smem_bytes(a.NB);
  if (smem > (size_t)ctx->max_smem_optin) return TDK_ENOTSUP;
  a.ntiles = (B + 128 * LD_MT - 1) / (128 * LD_MT);
  a.X = X;
  a.status = ctx->d_status;
  const int grid = (int)std::min<int64_t>(a.ntiles, ctx->num_sms);
  const int64_t ldu = (I0 + 7) / 8 * 8;
  Planner pl;
  pl.take<__nv_bfloat16>((size_t)a.NB * ldu);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  __nv_bfloat16* ub = cv.take<__nv_bfloat16>((size_t)a.NB * ldu);
  build_u_bf16<<<128, 256, 0, ctx->stream>>>(U1, (int)I0, a.Rt, a.Rtp, 1, (int)ldu, ub);
  TDK_LAUNCH_CHECK(ctx);
  CUtensorMap tmY, tmU;
  {
    uint64_t dims[2] = {(uint64_t)B, (uint64_t)I0};
    uint64_t str[1] = {(uint64_t)B * 2};
    uint32_t box[2] = {64u, 64u};
    rc = encode_tmap(&tmY, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Y, dims, str, box, true);
    if (rc) return rc;
    uint64_t ud[2] = {(uint64_t)I0, (uint64_t)a.NB};
    uint64_t us[1] = {(uint64_t)ldu * 2};
    uint32_t ubx[2] = {64u, (uint32_t)a.NB};
    rc = encode_tmap(&tmU, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ub, ud, us, ubx, true);
    if (rc) return rc;
  }
  TDK_CUDA_TRY(cudaFuncSetAttribute(tc_ttm_lead_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tc_ttm_lead_kernel<<<grid, LD_THREADS, smem, ctx->stream>>>(tmY, tmU, a);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // namespace tdk

namespace tdk {
TDK_CHECKED_UNIT(tc_core)
}  // namespace tdk
