// Tensor-core (tcgen05) forms of the two passes over Y.
//
// SKETCH (Sec. IV-A step 2; Alg. 2; Eq. 22), N >= 3.  Y is read as a 3-D
// array [P][J][L] with L = I_N (contiguous), J = I_{N-1}, P = prod_{k<N-1} I_k.
// A tile is 128 consecutive j (one p) x 128 consecutive columns, staged by TMA
// into shared memory with the 128-byte swizzle, and used twice:
//   G1 (K-major A):  D1[j, c] += sum_k Y[p, j, k] WN[c, k]  for the channels
//                    c of every mode n < N-1 (WN = W_N^(n) blocks, each padded
//                    to 16 channels), accumulated in TMEM over the unit's
//                    column range and read once per p;
//   G2 (MN-major A): D2[k, r] += sum_j Y[p, j, k] K_p[j, r] with the Khatri-Rao
//                    rows K_p[j, r] = W_{N-1}^(N)[j, r] prod_{k<N-1} W_k^(N)[i_k(p), r]
//                    generated per p by the epilogue warps, accumulated in TMEM
//                    over the whole unit.
// The epilogue turns D1 into the sketches of modes < N: mode N-1 (the tile's
// row mode) accumulates per TMEM lane across p; modes < N-1 are constant over
// the tile and need a 128-lane reduction.  Each work unit (j-tile, column
// range, p-range) writes its own partial block (the blockwise sums of Eq. 22);
// a fixed-order compensated FP32 reduction produces Z.
//
// CORE (Alg. 2, the first projection step, contiguous mode): X_1 = Y_(rows) U_N
// with U split hi+lo into one B operand [U_hi | U_lo]; ||Y||^2 on the side.
//
// FP32 data: TMA brings FP32 boxes; converter warps split every value into
// BF16 hi + lo in place, and both parts are multiplied (two MMAs per step).
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "tc_common.cuh"

namespace tdk {

int encode_tmap(CUtensorMap* map, CUtensorMapDataType dt, int rank, const void* base, const uint64_t* dims,
                const uint64_t* strides_bytes, const uint32_t* box, bool swizzle128) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return TDK_ENOTSUP;
    }
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  cuuint64_t d[5];
  cuuint64_t s[4];
  cuuint32_t b[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) s[i] = strides_bytes[i];
  }
  CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void*>(base), d, s, b, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    fprintf(stderr, "tdk: cuTensorMapEncodeTiled failed (%d)\n", (int)r);
    return TDK_EINVAL;
  }
  return TDK_OK;
}

namespace {

using namespace tc;


constexpr int KB = 1024;
constexpr uint32_t BOX_BYTES = 16 * KB;  // one 128-row x 128-byte box
constexpr int SK_SMAX = 4;               // deepest stage ring of the sketch
constexpr int SK_KTB = 3;                // K_p tiles in flight (built two p ahead)
constexpr int SK_CB = 4;                 // per-p coefficient buffers (loaded three p ahead)

// =====================================================================
//                               SKETCH
// =====================================================================
struct SkArgs {
  int N;
  int64_t I[TDK_MAX_MODES];
  int Rt[TDK_MAX_MODES];
  int Rtp[TDK_MAX_MODES];          // padded to 16
  int L, J;
  int64_t P;
  int N1;                          // G1 channels (sum of padded widths, modes < N-1)
  int off[TDK_MAX_MODES];          // channel offset of mode n
  int RtL;                         // Rt of the contiguous mode
  int hilo;                        // K rows split hi (cols 0..31) + lo (32..63)
  int KRW, KS;                     // columns per unit (multiple of 128), stages per p
  int JT, KR, PC;
  int64_t PCW;
  int64_t nunits;
  int d1_cols;                     // TMEM column stride of the two D1 buffers
  int S;                           // stages in the ring
  int nd1;                         // D1^T buffers in TMEM (form with W in TMEM)
  double* nrm_part;                // null, or [grid][4]: sums of squares of the staged Y (per warp)
  signed char lane_mode[128];      // form with W in TMEM: mode of channel c (-1: padding)
  unsigned char lane_r[128];       //   and its column r within the mode
  const float* Wf[TDK_MAX_MODES][TDK_MAX_MODES];  // FP32 W_k^(n) [I_k x Rt_n]
  float* part;
  int64_t ustride;                 // floats per unit
  int64_t poff_last, poff_j;
  int64_t poff_p[TDK_MAX_MODES];
  unsigned* status;
  unsigned long long* prof;        // optional cycle counters of CTA 0 (null = off)
  int yhint;                       // L2 policy of Y's boxes: 1 evict-first, 0 normal
};

// Y is read once: its boxes go first out of L2, so that the test-matrix rows
// the epilogue re-reads stay there.  At 3000^3 BF16 this takes the pass from
// 12.36 to 12.14 ms, although DRAM reads grow from 57.1 to 61.0 GB.
__device__ __forceinline__ void load_y_box(const SkArgs& a, uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                           int c2, uint32_t bar) {
  if (a.yhint)
    tma_load_3d_evict_first(dst, map, c0, c1, c2, bar);
  else
    tma_load_3d(dst, map, c0, c1, c2, bar);
}

template <bool F32>
struct SkLayout {
  static constexpr uint32_t STAGE_BYTES = F32 ? 64 * KB : 32 * KB;   // 128 j x 128 columns
  static constexpr uint32_t BOX_STRIDE = F32 ? 32 * KB : 16 * KB;     // between the two 64-column halves
  static constexpr uint32_t KT_BYTES = 16 * KB;                        // K_p tile [128 j][64 r] BF16
};

// epilogue warp groups: two for BF16 data (the epilogue bounds the pass),
// one for FP32 data (whose converter warps take the other four slots)
template <bool F32>
constexpr int sketch_groups() { return F32 ? 1 : 2; }

template <bool F32, int RW>
__global__ void __launch_bounds__(320, 1)
    tc_sketch_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmW,
                     const SkArgs a) {
  using Lay = SkLayout<F32>;
  constexpr int EG = sketch_groups<F32>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned start, by offset so that the pointer stays in the shared space
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* st_base = base;                                   // STAGES x STAGE_BYTES
  unsigned char* wn_base = st_base + a.S * Lay::STAGE_BYTES;  // 2*KS boxes of N1 rows x 128 B
  const uint32_t wn_box = (uint32_t)a.N1 * 128u;
  unsigned char* kt_base = wn_base + ((2 * a.KS * wn_box + 1023) & ~1023u);  // SK_KTB x KT_BYTES
  uint64_t* bars = reinterpret_cast<uint64_t*>(kt_base + SK_KTB * Lay::KT_BYTES);
  const int S = a.S;               // stage ring depth (<= SK_SMAX)
  uint64_t* full = bars;                     // [SK_SMAX]
  uint64_t* empty = bars + SK_SMAX;          // [SK_SMAX]
  uint64_t* cfull = bars + 2 * SK_SMAX;      // [SK_SMAX] (FP32: converted)
  uint64_t* d1full = bars + 3 * SK_SMAX;     // [2]
  uint64_t* d1empty = d1full + 2;            // [2]
  uint64_t* ktfull = d1full + 4;             // [SK_KTB]
  uint64_t* ktempty = ktfull + SK_KTB;       // [SK_KTB]
  uint64_t* wnfull = ktempty + SK_KTB;
  uint64_t* wnempty = wnfull + 1;
  uint64_t* d2full = wnfull + 2;
  uint64_t* d2empty = wnfull + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wnfull + 5);
  float* red = reinterpret_cast<float*>(wnfull + 7);               // [2 groups][4][64]
  float* coef = red + 2 * 4 * 64;                                  // [SK_CB][4][64]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(coef + SK_CB * 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), 1);
      mbar_init(smem_u32(&cfull[i]), 4);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&d1full[i]), 1);
      mbar_init(smem_u32(&d1empty[i]), 4 * EG);
    }
    for (int i = 0; i < SK_KTB; ++i) {
      mbar_init(smem_u32(&ktfull[i]), 4 * EG);
      mbar_init(smem_u32(&ktempty[i]), 1);
    }
    mbar_init(smem_u32(wnfull), 1);
    mbar_init(smem_u32(wnempty), 1);
    mbar_init(smem_u32(d2full), 1);
    mbar_init(smem_u32(d2empty), 4 * EG);
    *abort_flag = 0;
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
  unsigned* status = a.status;
  bool ok = true;
  // cycle accounting of CTA 0 (slot, lane 0 of the role's first warp)
  const bool prof_on = a.prof != nullptr && blockIdx.x == 0 && lane == 0;
  unsigned long long pt = clock64();
  auto pmark = [&](int slot) {
    if (prof_on) {
      const unsigned long long t = clock64();
      atomicAdd(a.prof + slot, t - pt);
      pt = t;
    }
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      prefetch_tmap(&tmY);
      prefetch_tmap(&tmW);
      uint32_t it = 0, un = 0;
      for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x, ++un) {
        const int pc = (int)(u % a.PC);
        const int kr = (int)((u / a.PC) % a.KR);
        const int jt = (int)(u / ((int64_t)a.PC * a.KR));
        const int64_t p0 = (int64_t)pc * a.PCW;
        const int64_t p1 = std::min<int64_t>(a.P, p0 + a.PCW);
        const int k0 = kr * a.KRW, j0 = jt * 128;
        // resident W block of this column range
        if (!mbar_wait(smem_u32(wnempty), (un & 1) ^ 1, status)) { ok = false; break; }
        mbar_expect_tx(smem_u32(wnfull), 2 * a.KS * wn_box);
        for (int b = 0; b < 2 * a.KS; ++b)
          tma_load_3d(smem_u32(wn_base + b * wn_box), &tmW, k0 + 64 * b, 0, 0, smem_u32(wnfull));
        for (int64_t p = p0; p < p1 && ok; ++p) {
          for (int st = 0; st < a.KS; ++st, ++it) {
            const int s = it % S;
            const uint32_t n = it / S;
            pmark(5);
            if (!mbar_wait(smem_u32(&empty[s]), (n & 1) ^ 1, status)) { ok = false; break; }
            pmark(6);  // producer waits for a free stage
            unsigned char* dst = st_base + s * Lay::STAGE_BYTES;
            mbar_expect_tx(smem_u32(&full[s]), Lay::STAGE_BYTES);
            const int kc = k0 + 128 * st;
            if (F32) {
              for (int q = 0; q < 4; ++q)
                load_y_box(a, smem_u32(dst + q * BOX_BYTES), &tmY, kc + 32 * q, j0, (int)p, smem_u32(&full[s]));
            } else {
              for (int q = 0; q < 2; ++q)
                load_y_box(a, smem_u32(dst + q * BOX_BYTES), &tmY, kc + 64 * q, j0, (int)p, smem_u32(&full[s]));
            }
          }
        }
      }
      if (!ok) *abort_flag = 1;
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id1 = idesc_bf16(128, a.N1, 0, 0);
      const uint32_t id2 = idesc_bf16(128, 64, 1, 1);
      const uint32_t d2col = 2 * a.d1_cols;
      uint32_t it = 0, pi = 0, un = 0;
      for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x, ++un) {
        const int pc = (int)(u % a.PC);
        const int64_t p0 = (int64_t)pc * a.PCW;
        const int64_t p1 = std::min<int64_t>(a.P, p0 + a.PCW);
        if (!mbar_wait(smem_u32(wnfull), un & 1, status)) { ok = false; break; }
        if (!mbar_wait(smem_u32(d2empty), (un & 1) ^ 1, status)) { ok = false; break; }
        tc_fence_after();
        bool first_p = true;
        for (int64_t p = p0; p < p1 && ok; ++p, ++pi) {
          const int db = pi & 1, kb = pi % SK_KTB;
          pmark(0);
          if (!mbar_wait(smem_u32(&d1empty[db]), ((pi >> 1) & 1) ^ 1, status)) { ok = false; break; }
          pmark(1);  // MMA waits for the epilogue to free D1
          if (!mbar_wait(smem_u32(&ktfull[kb]), (pi / SK_KTB) & 1, status)) { ok = false; break; }
          pmark(2);  // MMA waits for the K_p tile
          tc_fence_after();
          const uint32_t d1 = tmem + db * a.d1_cols;
          const uint32_t kt = smem_u32(kt_base + kb * Lay::KT_BYTES);
          for (int st = 0; st < a.KS; ++st, ++it) {
            const int s = it % S;
            const uint32_t n = it / S;
            pmark(0);
            if (!mbar_wait(smem_u32(F32 ? &cfull[s] : &full[s]), n & 1, status)) { ok = false; break; }
            pmark(3);  // MMA waits for data
            tc_fence_after();
            const uint32_t sb = smem_u32(st_base + s * Lay::STAGE_BYTES);
            const int nparts = F32 ? 2 : 1;
            for (int part = 0; part < nparts; ++part) {
              const uint32_t ab = sb + part * BOX_BYTES;  // hi at +0, lo at +16 KB (FP32 layout)
              // G1: 8 K-steps of 16 columns (two 64-column boxes)
              for (int kk = 0; kk < 8; ++kk) {
                const uint32_t aaddr = ab + (kk >> 2) * Lay::BOX_STRIDE + (kk & 3) * 32;
                const uint32_t baddr = smem_u32(wn_base) + (2 * st + (kk >> 2)) * wn_box + (kk & 3) * 32;
                mma_bf16(d1, smem_desc(aaddr, 16, 1024, SW128), smem_desc(baddr, 16, 1024, SW128), id1,
                         (st | kk | part) != 0);
              }
              // G2: 8 K-steps of 16 rows; A = the same tile read MN-major
              for (int kk = 0; kk < 8; ++kk) {
                const uint32_t aaddr = ab + kk * 2048;
                const uint32_t baddr = kt + kk * 2048;
                mma_bf16(tmem + d2col + st * 64, smem_desc(aaddr, Lay::BOX_STRIDE, 1024, SW128),
                         smem_desc(baddr, 16, 1024, SW128), id2, !(first_p && kk == 0 && part == 0));
              }
            }
            umma_commit(smem_u32(&empty[s]));
            pmark(4);  // MMA issue
          }
          umma_commit(smem_u32(&d1full[db]));
          umma_commit(smem_u32(&ktempty[kb]));
          first_p = false;
        }
        umma_commit(smem_u32(d2full));
        umma_commit(smem_u32(wnempty));
      }
      if (!ok) *abort_flag = 1;
    }
  } else if (warp < 2 + 4 * EG) {
    // ------------------------------------------------------------ epilogue (EG groups of 4 warps)
    // Group g owns the channels [g*CH, (g+1)*CH) of every mode; the two groups
    // read the same TMEM lanes (warp w reads lanes 32*(w%4)), so each warp's
    // dependent chains are half as long and two warps share each scheduler.
    constexpr int CH = RW / EG;
    constexpr int HW = CH / 2;
    constexpr int NE = 128 * EG;       // epilogue threads
    constexpr int NSLOT = 256 / NE;    // coefficient slots per thread
    const int q = warp & 3;
    const int grp = (warp - 2) >> 2;
    const int cg = grp * CH;           // first channel of this group
    const int jl = 32 * q + lane;      // TMEM lane = tile row j (D1) / column k (D2)
    const int et = grp * 128 + jl;     // epilogue thread index
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    const int Nm = a.N;
    const int nj = Nm - 2;             // tile row mode
    const int nl = Nm - 1;             // contiguous mode
    const int Rj = a.Rt[nj];
    // Per-p coefficient vectors, products of W rows over the outer indices of p
    // (four vectors of 64: [0] Khatri-Rao rows of the contiguous mode, [1] the
    // row mode, [2], [3] modes 0 and 1 when they are outer modes), kept in
    // four shared buffers so that p+3 is loaded while p is in use.
    // raw factors only: the loads are issued three p ahead and multiplied when
    // stored, so their latency overlaps the work on p
    auto coef_load = [&](int64_t pp, float (*cr)[2]) {
      int kidx[2] = {0, 0};
      {
        int rem = (int)pp;
        for (int k = Nm - 3; k >= 0; --k) {
          kidx[k] = rem % (int)a.I[k];
          rem /= (int)a.I[k];
        }
      }
#pragma unroll
      for (int h = 0; h < NSLOT; ++h) {
        const int slot = et + NE * h;
        const int vec = slot >> 6, r = slot & 63;
        const int n = vec == 0 ? nl : (vec == 1 ? nj : vec - 2);
        const bool live = (vec < 2 || vec - 2 < nj) && r < a.Rt[n];
        int f = 0;
        cr[h][0] = live ? 1.f : 0.f;
        cr[h][1] = 1.f;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (k < Nm - 2 && live && !(vec >= 2 && k == n)) {
            cr[h][f] *= __ldg(a.Wf[n][k] + (int64_t)kidx[k] * a.Rt[n] + r);
            f = 1;
          }
        }
      }
    };
    auto coef_store = [&](uint32_t pidx, const float (*cr)[2]) {
      float* cb = coef + (pidx % SK_CB) * 256;
#pragma unroll
      for (int h = 0; h < NSLOT; ++h) cb[et + NE * h] = cr[h][0] * cr[h][1];
    };
    auto unpack = [](uint32_t w, int e) -> float {
      return e ? __uint_as_float(w & 0xFFFF0000u) : __uint_as_float(w << 16);
    };
    uint32_t pi = 0, un = 0;
    for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x, ++un) {
      const int pc = (int)(u % a.PC);
      const int kr = (int)((u / a.PC) % a.KR);
      const int jt = (int)(u / ((int64_t)a.PC * a.KR));
      const int64_t p0 = (int64_t)pc * a.PCW;
      const int64_t p1 = std::min<int64_t>(a.P, p0 + a.PCW);
      const int j0 = jt * 128;
      const int jj = j0 + jl;
      const bool vj = jj < a.J;
      float* up = a.part + u * a.ustride;
      // this lane's row of W_{N-1}^(N) and of W_{N-1}^(m) (m < N-2) over the
      // group's channels, packed BF16 (the test matrices hold BF16 values, so
      // the packing is exact)
      uint32_t wk[HW], wn0[HW], wn1[HW];
#pragma unroll
      for (int i = 0; i < HW; ++i) {
        float k0v = 0.f, k1v = 0.f, a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
        const int r = cg + 2 * i;
        if (vj) {
          const float* wkr = a.Wf[nl][nj] + (int64_t)jj * a.RtL;
          if (r < a.RtL) k0v = __ldg(wkr + r);
          if (r + 1 < a.RtL) k1v = __ldg(wkr + r + 1);
          if (nj > 0) {
            const float* w0 = a.Wf[0][nj] + (int64_t)jj * a.Rt[0];
            if (r < a.Rt[0]) a0 = __ldg(w0 + r);
            if (r + 1 < a.Rt[0]) a1 = __ldg(w0 + r + 1);
          }
          if (nj > 1) {
            const float* w1 = a.Wf[1][nj] + (int64_t)jj * a.Rt[1];
            if (r < a.Rt[1]) b0 = __ldg(w1 + r);
            if (r + 1 < a.Rt[1]) b1 = __ldg(w1 + r + 1);
          }
        }
        wk[i] = pack_bf16x2(k0v, k1v);
        wn0[i] = pack_bf16x2(a0, a1);
        wn1[i] = pack_bf16x2(b0, b1);
      }
      float accj[CH];
#pragma unroll
      for (int r = 0; r < CH; ++r) accj[r] = 0.f;
      // K_p rows for G2 (row j of the tile), MN-major [j][r], 128-byte swizzle;
      // group g writes the 16-byte chunks of its channels
      auto gen_k = [&](uint32_t pidx) -> bool {
        const int kb = pidx % SK_KTB;
        if (!mbar_wait(smem_u32(&ktempty[kb]), ((pidx / SK_KTB) & 1) ^ 1, status)) return false;
        const float* cK = coef + (pidx % SK_CB) * 256;
        unsigned char* row = kt_base + kb * SkLayout<F32>::KT_BYTES + jl * 128;
        const int ph = jl & 7;
        auto put = [&](int c, const uint32_t* w4) {
          *reinterpret_cast<uint4*>(row + ((c ^ ph) << 4)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        };
        if (a.hilo) {
          // single group: chunks 0-3 hold hi, 4-7 lo of channels 0..31
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint32_t w4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float v0 = 0.f, v1 = 0.f;
              const int r = 8 * (c & 3) + 2 * e;
              if (r < CH) {
                const float s0 = unpack(wk[r / 2], 0) * cK[r];
                const float s1 = unpack(wk[r / 2], 1) * cK[r + 1];
                if (c < 4) {
                  v0 = s0;
                  v1 = s1;
                } else {
                  v0 = s0 - __bfloat162float(__float2bfloat16_rn(s0));
                  v1 = s1 - __bfloat162float(__float2bfloat16_rn(s1));
                }
              }
              w4[e] = pack_bf16x2(v0, v1);
            }
            put(c, w4);
          }
        } else {
          // the chunks of this group's channels, then its share of the zero
          // chunks beyond RW (the G2 operand is 64 channels wide)
          constexpr int OWN = CH / 8;
          constexpr int ZERO = (8 - RW / 8) / EG;
#pragma unroll
          for (int cc = 0; cc < OWN; ++cc) {
            uint32_t w4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int rl = 8 * cc + 2 * e;  // channel within the group
              w4[e] = pack_bf16x2(unpack(wk[rl / 2], 0) * cK[cg + rl], unpack(wk[rl / 2], 1) * cK[cg + rl + 1]);
            }
            put(cg / 8 + cc, w4);
          }
#pragma unroll
          for (int cc = 0; cc < ZERO; ++cc) {
            const uint32_t z4[4] = {0u, 0u, 0u, 0u};
            put(RW / 8 + grp * ZERO + cc, z4);
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&ktfull[kb]));
        return true;
      };
      {
        float cr[NSLOT][2];
        for (int d = 0; d < 3; ++d)
          if (p0 + d < p1) {
            coef_load(p0 + d, cr);
            coef_store(pi + d, cr);
          }
      }
      named_bar(1, NE);
      // K tiles run two p ahead of the MMAs, so that the MMA issuer never
      // waits for the epilogue's work on the previous D1
      if (!gen_k(pi)) { ok = false; break; }
      if (p0 + 1 < p1 && !gen_k(pi + 1)) { ok = false; break; }
      for (int64_t p = p0; p < p1 && ok; ++p, ++pi) {
        const int db = pi & 1;
        float cr2[NSLOT][2];
#pragma unroll
        for (int h = 0; h < NSLOT; ++h) cr2[h][0] = cr2[h][1] = 0.f;
        const bool have3 = p + 3 < p1;
        if (have3) coef_load(p + 3, cr2);
        pmark(8);
        if (p + 2 < p1 && !gen_k(pi + 2)) { ok = false; break; }
        pmark(9);  // epilogue: K tile (incl. waiting for the MMA to free it)
        const float* cb = coef + (pi % SK_CB) * 256;
        // ---- D1 -> sketches of modes < N
        if (!mbar_wait(smem_u32(&d1full[db]), (pi >> 1) & 1, status)) { ok = false; break; }
        pmark(10);  // epilogue waits for D1
        tc_fence_after();
        const uint32_t d1 = tmem + db * a.d1_cols + lane_addr;
        // row mode: per-lane accumulation weighted by the outer coefficients
#pragma unroll
        for (int c16 = 0; c16 < CH / 16; ++c16) {
          if (cg + c16 * 16 < a.Rtp[nj]) {
            float v[16];
            tmem_ld16(d1 + a.off[nj] + cg + c16 * 16, v);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; ++e)
              accj[c16 * 16 + e] = fmaf(v[e], cb[64 + cg + c16 * 16 + e], accj[c16 * 16 + e]);
          }
        }
        pmark(11);  // row mode
        // modes constant over the tile: weight by W_{N-1}^(m)[j], reduce over 128 lanes
        for (int m = 0; m < nj; ++m) {
          float v[CH];
#pragma unroll
          for (int c16 = 0; c16 < CH / 16; ++c16) {
            if (cg + c16 * 16 < a.Rtp[m]) {
              tmem_ld16(d1 + a.off[m] + cg + c16 * 16, v + c16 * 16);
            } else {
#pragma unroll
              for (int e = 0; e < 16; ++e) v[c16 * 16 + e] = 0.f;
            }
          }
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < HW; ++i) {
            const uint32_t w = (m == 0) ? wn0[i] : wn1[i];
            v[2 * i] *= unpack(w, 0);
            v[2 * i + 1] *= unpack(w, 1);
          }
          // butterfly transpose-reduce: each lane ends with max(1, CH/32) of
          // the CH sums (CH < 32: the last rounds add the partner's partial)
          int bse = 0;
#pragma unroll
          for (int o = 16, h = CH / 2; o >= 1; o >>= 1, h >>= 1) {
            if (h >= 1) {
              const bool upper = (lane & o) != 0;
#pragma unroll
              for (int i = 0; i < CH / 2; ++i) {
                if (i < h) {
                  const float send = upper ? v[i] : v[i + h];
                  const float keep = upper ? v[i + h] : v[i];
                  v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
              }
              bse += upper ? h : 0;
            } else {
              v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
            }
          }
          float* rg = red + grp * 4 * 64;
          rg[q * 64 + bse] = v[0];
          if (CH == 64) rg[q * 64 + bse + 1] = v[1];
          named_bar(1, NE);
          const int Rm = a.Rt[m];
          if (jl < CH && cg + jl < Rm) {
            const float s = rg[jl] + rg[64 + jl] + rg[128 + jl] + rg[192 + jl];
            const int64_t o = a.poff_p[m] + (p - p0) * Rm + cg + jl;
            if (TDK_IN(o, a.ustride)) up[o] = s * cb[128 + 64 * m + cg + jl];
          }
          named_bar(1, NE);
        }
        pmark(12);  // reductions
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&d1empty[db]));
        if (have3) coef_store(pi + 3, cr2);
        named_bar(1, NE);
        pmark(13);  // tail barrier
      }
      if (!ok) break;
      // ---- unit end: row-mode partial and the contiguous mode from D2
      if (vj) {
#pragma unroll
        for (int r = 0; r < CH; ++r)
          if (cg + r < Rj && TDK_IN(a.poff_j + (int64_t)jl * Rj + cg + r, a.ustride))
            up[a.poff_j + (int64_t)jl * Rj + cg + r] = accj[r];
      }
      if (!mbar_wait(smem_u32(d2full), un & 1, status)) { ok = false; break; }
      tc_fence_after();
      for (int st = grp; st < a.KS; st += EG) {
        float v[64];
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) tmem_ld16(tmem + 2 * a.d1_cols + st * 64 + c16 * 16 + lane_addr, v + c16 * 16);
        tmem_wait_ld();
        const int kloc = 128 * st + jl;
        if (kr * a.KRW + kloc < a.L) {
          float* dst = up + a.poff_last + (int64_t)kloc * a.RtL;
#pragma unroll
          for (int r = 0; r < 64; ++r) {
            if (r < a.RtL && TDK_IN(a.poff_last + (int64_t)kloc * a.RtL + r, a.ustride)) {
              float z = v[r];
              if (a.hilo && r < 32) z += v[32 + (r & 31)];
              dst[r] = z;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(d2empty));
    }
    if (!ok) *abort_flag = 1;
  } else if (F32) {
    // ------------------------------------------------------------ converters (FP32 data)
    const int q = warp - 6;
    const int r = 32 * q + lane;
    uint32_t it = 0;
    double sq = 0.0;  // ||Y||^2 of the rows this thread splits (the split sums the squares)
    for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
      const int pc = (int)(u % a.PC);
      const int64_t p0 = (int64_t)pc * a.PCW;
      const int64_t p1 = std::min<int64_t>(a.P, p0 + a.PCW);
      for (int64_t p = p0; p < p1 && ok; ++p) {
        for (int st = 0; st < a.KS; ++st, ++it) {
          const int s = it % S;
          const uint32_t n = it / S;
          if (!mbar_wait(smem_u32(&full[s]), n & 1, status)) { ok = false; break; }
          unsigned char* sb = st_base + s * SkLayout<true>::STAGE_BYTES;
          for (int h = 0; h < 2; ++h)
            sq += (double)split_row64(sb + h * 2 * BOX_BYTES + r * 128, sb + (h * 2 + 1) * BOX_BYTES + r * 128, r);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&cfull[s]));
        }
      }
    }
    sq = warp_sum(sq);
    if (a.nrm_part && lane == 0) a.nrm_part[4 * blockIdx.x + q] = sq;
    if (!ok) *abort_flag = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// =====================================================================
//        SKETCH, BF16 data: test matrices of the modes < N in TMEM
// =====================================================================
// The first product is taken transposed, D1^T[c, j] = sum_k WN[c, k] Y[p, j, k]:
// the unit's block of the W_N^(n) (channels x columns, BF16) is the A operand
// and lives in Tensor Memory, written once per unit by the epilogue warps; the
// staged Y tile is a K-major B operand.  Shared memory then holds only the
// stage ring and the K_p tiles, so the ring is deeper than with a resident W
// block; and with one channel per TMEM lane, the modes that are constant over
// the tile reduce within the lane (a dot product with W_{N-1}^(m) over the
// tile's rows j) instead of across lanes.
// TMEM, 512 columns: W [0, 64 KS) | D1^T [.., + 128 nd1) | D2 [.., + 64 KS).
constexpr int TW_SMAX = 6;

struct TwLayout {  // byte offsets in the 1024-aligned dynamic shared memory
  uint32_t kt, bars, red, coef, flag, total;
};
__host__ __device__ inline TwLayout tw_layout(int S) {
  TwLayout L{};
  L.kt = (uint32_t)S * 32u * KB;           // stage ring: S x (128 j x 128 columns) BF16
  L.bars = L.kt + SK_KTB * 16u * KB;       // K_p tiles
  L.red = L.bars + 256u;                   // mbarriers and the TMEM address
  L.coef = L.red + 2u * 128u * 4u;         // [2][128] FP32: second j half of the dot products
  L.flag = L.coef + SK_CB * 256u * 4u;     // [SK_CB][256] FP32 per-p coefficients
  L.total = L.flag + 64u;
  return L;
}

__global__ void __launch_bounds__(384, 1)
    tc_sketch_tw_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ SkArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const TwLayout Lay = tw_layout(a.S);
  unsigned char* st_base = base;
  unsigned char* kt_base = base + Lay.kt;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + Lay.bars);
  uint64_t* full = bars;                   // [TW_SMAX]
  uint64_t* empty = bars + TW_SMAX;        // [TW_SMAX]
  uint64_t* d1full = bars + 2 * TW_SMAX;   // [2]
  uint64_t* d1empty = d1full + 2;          // [2]
  uint64_t* ktfull = d1full + 4;           // [SK_KTB]
  uint64_t* ktempty = ktfull + SK_KTB;     // [SK_KTB]
  uint64_t* wfull = ktempty + SK_KTB;
  uint64_t* wempty = wfull + 1;
  uint64_t* d2full = wfull + 2;
  uint64_t* d2empty = wfull + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wfull + 4);
  double* nred = reinterpret_cast<double*>(wfull + 5);  // [2] sums of squares of the norm warps
  float* red = reinterpret_cast<float*>(base + Lay.red);
  float* coef = reinterpret_cast<float*>(base + Lay.coef);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(base + Lay.flag);
  constexpr int EG = 2;          // epilogue warp groups
  constexpr int NE = 128 * EG;   // epilogue threads
  constexpr int CH = 32;         // K_p channels written per group (64 in all)
  constexpr int HW = CH / 2;
  const int S = a.S, KS = a.KS, ND1 = a.nd1;
  const uint32_t w_col = 0, d1_col = 64u * KS, d2_col = 64u * KS + 128u * ND1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool want_norm = a.nrm_part != nullptr;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      // the MMA commit, and the two norm warps when they sum ||Y||^2
      mbar_init(smem_u32(&empty[i]), want_norm ? 3 : 1);
    }
    nred[0] = nred[1] = 0.0;
    for (int i = 0; i < ND1; ++i) {
      mbar_init(smem_u32(&d1full[i]), 1);
      mbar_init(smem_u32(&d1empty[i]), 4 * EG);
    }
    for (int i = 0; i < SK_KTB; ++i) {
      mbar_init(smem_u32(&ktfull[i]), 4 * EG);
      mbar_init(smem_u32(&ktempty[i]), 1);
    }
    mbar_init(smem_u32(wfull), 4 * EG);
    mbar_init(smem_u32(wempty), 1);
    mbar_init(smem_u32(d2full), 1);
    mbar_init(smem_u32(d2empty), 4 * EG);
    *abort_flag = 0;
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
  unsigned* status = a.status;
  bool ok = true;
  // cycle accounting of CTA 0 (test build: lane 0 of each role's first warp)
  const bool prof_on = a.prof != nullptr && blockIdx.x == 0 && lane == 0 && (warp <= 2);
  unsigned long long pt = clock64();
  auto pmark = [&](int slot) {
    if (prof_on) {
      const unsigned long long t = clock64();
      atomicAdd(a.prof + slot, t - pt);
      pt = t;
    }
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      prefetch_tmap(&tmY);
      uint32_t s = 0, sph = 0;  // ring slot and the phase of its barriers
      for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
        const int pc = (int)(u % a.PC);
        const int kr = (int)((u / a.PC) % a.KR);
        const int jt = (int)(u / ((int64_t)a.PC * a.KR));
        const int64_t p0 = (int64_t)pc * a.PCW;
        const int64_t p1 = std::min<int64_t>(a.P, p0 + a.PCW);
        const int k0 = kr * a.KRW, j0 = jt * 128;
        for (int64_t p = p0; p < p1 && ok; ++p) {
          for (int st = 0; st < KS; ++st) {
            pmark(5);
            if (!mbar_wait(smem_u32(&empty[s]), sph ^ 1, status)) { ok = false; break; }
            pmark(6);  // producer waits for a free stage
            const uint32_t dst = smem_u32(st_base) + s * 32 * KB;
            const uint32_t fb = smem_u32(&full[s]);
            mbar_expect_tx(fb, 32 * KB);
            const int kc = k0 + 128 * st;
            load_y_box(a, dst, &tmY, kc, j0, (int)p, fb);
            load_y_box(a, dst + BOX_BYTES, &tmY, kc + 64, j0, (int)p, fb);
            if (++s == (uint32_t)S) {
              s = 0;
              sph ^= 1;
            }
          }
        }
      }
      if (!ok) *abort_flag = 1;
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id1 = idesc_bf16(128, 128, 0, 0);  // D1^T: M = channels (A in TMEM), N = rows j
      const uint32_t id2 = idesc_bf16(128, 64, 1, 1);   // D2: M = columns k, N = K_p channels
      // descriptor bases: the start-address field is addr >> 4 in the low 14
      // bits and every operand lies below 256 KB of shared memory, so the
      // descriptor of base + off is the base's plus off >> 4 (the issue loop
      // then spends one add per operand)
      const uint64_t dB1 = smem_desc(smem_u32(st_base), 16, 1024, SW128);         // Y tile, K-major
      const uint64_t dA2 = smem_desc(smem_u32(st_base), BOX_BYTES, 1024, SW128);  // Y tile, MN-major
      const uint64_t dK = smem_desc(smem_u32(kt_base), 16, 1024, SW128);          // K_p tiles
      uint32_t s = 0, sph = 0;    // ring slot and its phase
      uint32_t kb = 0, kph = 0;   // K tile and its phase
      uint32_t pi = 0, un = 0;
      for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x, ++un) {
        const int pc = (int)(u % a.PC);
        const int64_t p0 = (int64_t)pc * a.PCW;
        const int64_t p1 = std::min<int64_t>(a.P, p0 + a.PCW);
        if (!mbar_wait(smem_u32(wfull), un & 1, status)) { ok = false; break; }
        if (!mbar_wait(smem_u32(d2empty), (un & 1) ^ 1, status)) { ok = false; break; }
        tc_fence_after();
        bool first_p = true;
        for (int64_t p = p0; p < p1 && ok; ++p, ++pi) {
          const int db = ND1 == 2 ? (int)(pi & 1) : 0;
          const uint32_t use = ND1 == 2 ? (pi >> 1) : pi;
          pmark(0);
          if (!mbar_wait(smem_u32(&ktfull[kb]), kph, status)) { ok = false; break; }
          pmark(2);  // MMA waits for the K_p tile
          tc_fence_after();
          const uint64_t kdesc = dK + ((kb * 16 * KB) >> 4);
          const uint32_t d1 = tmem + d1_col + 128u * db;
          for (int st = 0; st < KS; ++st) {
            pmark(0);
            if (!mbar_wait(smem_u32(&full[s]), sph, status)) { ok = false; break; }
            pmark(3);  // MMA waits for data
            tc_fence_after();
            const uint32_t so = (s * 32 * KB) >> 4;
            // G2 first: it does not touch D1^T, so it overlaps the epilogue's
            // read of the previous p's D1^T.  8 K-steps of 16 rows (2048 B)
            const uint32_t d2 = tmem + d2_col + 64u * st;
            mma_bf16(d2, dA2 + so, kdesc, id2, first_p ? 0u : 1u);
#pragma unroll
            for (int kk = 1; kk < 8; ++kk) mma_bf16(d2, dA2 + so + 128 * kk, kdesc + 128 * kk, id2, 1u);
            if (st == 0) {
              pmark(4);
              if (!mbar_wait(smem_u32(&d1empty[db]), (use & 1) ^ 1, status)) { ok = false; break; }
              pmark(1);  // MMA waits for the epilogue to free D1^T
              tc_fence_after();
            }
            // G1^T: 8 K-steps of 16 columns (two 64-column boxes); A = the W
            // columns of this stage in TMEM, 8 TMEM columns per K-step
            const uint32_t wa = tmem + w_col + 64u * st;
            mma_bf16_ts(d1, wa, dB1 + so, id1, st != 0 ? 1u : 0u);
#pragma unroll
            for (int kk = 1; kk < 8; ++kk)
              mma_bf16_ts(d1, wa + 8u * kk, dB1 + so + (uint32_t)((kk >> 2) * (BOX_BYTES >> 4) + (kk & 3) * 2), id1,
                          1u);
            umma_commit(smem_u32(&empty[s]));
            if (++s == (uint32_t)S) {
              s = 0;
              sph ^= 1;
            }
            pmark(4);  // MMA issue
          }
          if (!ok) break;
          umma_commit(smem_u32(&d1full[db]));
          umma_commit(smem_u32(&ktempty[kb]));
          if (++kb == (uint32_t)SK_KTB) {
            kb = 0;
            kph ^= 1;
          }
          first_p = false;
        }
        if (!ok) break;
        umma_commit(smem_u32(d2full));
        umma_commit(smem_u32(wempty));
      }
      if (!ok) *abort_flag = 1;
    }
  } else if (warp < 2 + 4 * EG) {
    // ------------------------------------------------------------ epilogue (2 groups of 4 warps)
    // Two roles per thread.  As TMEM lane c = 32 q + lane it owns channel c
    // of D1^T and the rows j of its group's half of the tile: the row mode
    // accumulates D1^T[c, j] over p (weighted by the outer coefficients), a
    // mode constant over the tile takes the dot product with its W row.  As
    // tile row jl = 32 q + lane it writes its group's 32 channels of K_p.
    const int q = warp & 3;
    const int grp = (warp - 2) >> 2;
    const int cg = grp * CH;
    const int jl = 32 * q + lane;
    const int c = jl;
    const int jh = 64 * grp;
    const int et = grp * 128 + jl;
    const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
    const int Nm = a.N;
    const int nj = Nm - 2;
    const int nl = Nm - 1;
    const int Rj = a.Rt[nj];
    const int lm = a.lane_mode[c];
    const int lr = a.lane_r[c];
    const bool rowrole = lm == nj;
    const bool dotrole = lm >= 0 && lm < nj;
    auto coef_load = [&](int64_t pp, float* cr) {
      // outer indices of p (N = 3: i_1 = p; N = 4: p = i_1 I_2 + i_2)
      const int i1 = Nm == 4 ? (int)(pp / a.I[1]) : (int)pp;
      const int i2 = Nm == 4 ? (int)(pp - (int64_t)i1 * a.I[1]) : 0;
      const int vec = et >> 6, r = et & 63;
      const int n = vec == 0 ? nl : (vec == 1 ? nj : vec - 2);
      const bool live = (vec < 2 || vec - 2 < nj) && r < a.Rt[n];
      cr[0] = live ? 1.f : 0.f;
      cr[1] = 1.f;
      if (live && !(vec >= 2 && n == 0)) cr[0] *= __ldg(a.Wf[n][0] + (int64_t)i1 * a.Rt[n] + r);
      if (live && Nm == 4 && !(vec >= 2 && n == 1)) cr[1] = __ldg(a.Wf[n][1] + (int64_t)i2 * a.Rt[n] + r);
    };
    auto coef_store = [&](uint32_t pidx, const float* cr) { coef[(pidx % SK_CB) * 256 + et] = cr[0] * cr[1]; };
    auto unpack = [](uint32_t w, int e) -> float {
      return e ? __uint_as_float(w & 0xFFFF0000u) : __uint_as_float(w << 16);
    };
    uint32_t pi = 0, un = 0;
    for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x, ++un) {
      const int pc = (int)(u % a.PC);
      const int kr = (int)((u / a.PC) % a.KR);
      const int jt = (int)(u / ((int64_t)a.PC * a.KR));
      const int64_t p0 = (int64_t)pc * a.PCW;
      const int64_t p1 = std::min<int64_t>(a.P, p0 + a.PCW);
      const int j0 = jt * 128;
      const int k0 = kr * a.KRW;
      float* up = a.part + u * a.ustride;
      // ---- this unit's W block into TMEM (lane c = channel c; group g writes
      //      the columns [32 KS g, 32 KS (g + 1)), two W values per column)
      if (!mbar_wait(smem_u32(wempty), (un & 1) ^ 1, status)) { ok = false; break; }
      tc_fence_after();
      for (int cc = 0; cc < 2 * KS; ++cc) {
        const int col0 = 32 * KS * grp + 16 * cc;
        uint32_t r16[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int k = k0 + 2 * (col0 + e);
          float v0 = 0.f, v1 = 0.f;
          if (lm >= 0) {
            const float* wr = a.Wf[lm][nl];
            if (k < a.L) v0 = __ldg(wr + (int64_t)k * a.Rt[lm] + lr);
            if (k + 1 < a.L) v1 = __ldg(wr + (int64_t)(k + 1) * a.Rt[lm] + lr);
          }
          r16[e] = pack_bf16x2(v0, v1);
        }
        tmem_st16(tmem + lane_addr + w_col + col0, r16);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(wfull));
      pmark(13);  // epilogue: W block into TMEM (incl. waiting for the previous unit)
      // ---- per-thread constants of the unit
      // dot role: W_{N-1}^(m)[j0 + jh + jj, r]; row role: the accumulators
      float aw[64];
#pragma unroll
      for (int jj = 0; jj < 64; ++jj) {
        const int j = j0 + jh + jj;
        aw[jj] = (dotrole && j < a.J) ? __ldg(a.Wf[lm][nj] + (int64_t)j * a.Rt[lm] + lr) : 0.f;
      }
      // K_p role: this row's W_{N-1}^(N) over the group's channels, packed BF16
      uint32_t wk[HW];
      {
        const int jj = j0 + jl;
#pragma unroll
        for (int i = 0; i < HW; ++i) {
          float k0v = 0.f, k1v = 0.f;
          const int r = cg + 2 * i;
          if (jj < a.J) {
            const float* wkr = a.Wf[nl][nj] + (int64_t)jj * a.RtL;
            if (r < a.RtL) k0v = __ldg(wkr + r);
            if (r + 1 < a.RtL) k1v = __ldg(wkr + r + 1);
          }
          wk[i] = pack_bf16x2(k0v, k1v);
        }
      }
      // K_p rows for G2 (row jl of the tile), MN-major [j][r], 128-byte swizzle
      auto gen_k = [&](uint32_t pidx) -> bool {
        const int kb = pidx % SK_KTB;
        if (!mbar_wait(smem_u32(&ktempty[kb]), ((pidx / SK_KTB) & 1) ^ 1, status)) return false;
        const float* cK = coef + (pidx % SK_CB) * 256;
        unsigned char* row = kt_base + kb * 16 * KB + jl * 128;
        const int ph = jl & 7;
#pragma unroll
        for (int cc = 0; cc < CH / 8; ++cc) {
          uint32_t w4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int rl = 8 * cc + 2 * e;
            w4[e] = pack_bf16x2(unpack(wk[rl / 2], 0) * cK[cg + rl], unpack(wk[rl / 2], 1) * cK[cg + rl + 1]);
          }
          const int chunk = cg / 8 + cc;
          *reinterpret_cast<uint4*>(row + ((chunk ^ ph) << 4)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&ktfull[kb]));
        return true;
      };
      {
        float cr[2];
        for (int d = 0; d < 3; ++d)
          if (p0 + d < p1) {
            coef_load(p0 + d, cr);
            coef_store(pi + d, cr);
          }
      }
      named_bar(1, NE);
      if (!gen_k(pi)) { ok = false; break; }
      if (p0 + 1 < p1 && !gen_k(pi + 1)) { ok = false; break; }
      for (int64_t p = p0; p < p1 && ok; ++p, ++pi) {
        const int db = ND1 == 2 ? (int)(pi & 1) : 0;
        const uint32_t use = ND1 == 2 ? (pi >> 1) : pi;
        float cr2[2] = {0.f, 0.f};
        const bool have3 = p + 3 < p1;
        if (have3) coef_load(p + 3, cr2);
        const float* cb = coef + (pi % SK_CB) * 256;
        pmark(8);
        // D1^T first: its single buffer holds back the next p's first product
        if (!mbar_wait(smem_u32(&d1full[db]), use & 1, status)) { ok = false; break; }
        pmark(10);  // epilogue waits for D1^T
        tc_fence_after();
        const uint32_t d1 = tmem + lane_addr + d1_col + 128u * db + jh;
        const float rowc = rowrole ? cb[64 + lr] : 0.f;
        float dot = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[32];
          tmem_ld16(d1 + 32 * h, v);
          tmem_ld16(d1 + 32 * h + 16, v + 16);
          tmem_wait_ld();
          if (h == 1) {
            // D1^T is read: the next p's first product may overwrite it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&d1empty[db]));
          }
          if (rowrole) {
#pragma unroll
            for (int e = 0; e < 32; ++e) aw[32 * h + e] = fmaf(v[e], rowc, aw[32 * h + e]);
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) dot = fmaf(v[e], aw[32 * h + e], dot);
          }
        }
        pmark(11);  // D1^T read and the row / dot products
        if (p + 2 < p1 && !gen_k(pi + 2)) { ok = false; break; }
        pmark(9);  // epilogue: K tile (incl. waiting for the MMA to free it)
        // modes constant over the tile: the two j halves meet in shared memory
        float* rb = red + (pi & 1) * 128;
        if (dotrole && grp == 1) rb[c] = dot;
        if (have3) coef_store(pi + 3, cr2);
        named_bar(1, NE);
        if (dotrole && grp == 0)
          if (TDK_IN(a.poff_p[lm] + (p - p0) * a.Rt[lm] + lr, a.ustride))
            up[a.poff_p[lm] + (p - p0) * a.Rt[lm] + lr] = (dot + rb[c]) * cb[128 + 64 * lm + lr];
        pmark(12);  // tail barrier and the partial store
      }
      if (!ok) break;
      // ---- unit end: row-mode partial and the contiguous mode from D2
      if (rowrole) {
#pragma unroll
        for (int jj = 0; jj < 64; ++jj)
          if (j0 + jh + jj < a.J && TDK_IN(a.poff_j + (int64_t)(jh + jj) * Rj + lr, a.ustride))
            up[a.poff_j + (int64_t)(jh + jj) * Rj + lr] = aw[jj];
      }
      if (!mbar_wait(smem_u32(d2full), un & 1, status)) { ok = false; break; }
      tc_fence_after();
      for (int st = grp; st < KS; st += EG) {
        float v[64];
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) tmem_ld16(tmem + d2_col + st * 64 + c16 * 16 + lane_addr, v + c16 * 16);
        tmem_wait_ld();
        const int kloc = 128 * st + jl;
        if (k0 + kloc < a.L) {
          float* dst = up + a.poff_last + (int64_t)kloc * a.RtL;
#pragma unroll
          for (int r = 0; r < 64; ++r)
            if (r < a.RtL && TDK_IN(a.poff_last + (int64_t)kloc * a.RtL + r, a.ustride)) dst[r] = v[r];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(d2empty));
    }
    if (!ok) *abort_flag = 1;
  } else if (want_norm) {
    // ------------------------------------------------------------ ||Y||^2 (warps 10, 11)
    // Each staged tile waits in the ring for its MMAs; meanwhile warp 10 + h
    // sums the squares of box h (64 columns x 128 rows, a 128-byte row per lane
    // and step), so the slot is released no later than the MMAs release it.
    const int h = warp - 2 - 4 * EG;
    uint32_t s = 0, sph = 0;
    double acc = 0.0;
    for (int64_t u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
      const int pc = (int)(u % a.PC);
      const int64_t p0 = (int64_t)pc * a.PCW;
      const int64_t p1 = std::min<int64_t>(a.P, p0 + a.PCW);
      for (int64_t p = p0; p < p1 && ok; ++p) {
        for (int st = 0; st < KS; ++st) {
          if (!mbar_wait(smem_u32(&full[s]), sph, status)) { ok = false; break; }
          const unsigned char* box = st_base + s * 32 * KB + h * BOX_BYTES;
          float part = 0.f, comp = 0.f;
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const int row = lane + 32 * rr;
            const unsigned char* rp = box + row * 128;
            float q = 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const uint4 w = *reinterpret_cast<const uint4*>(rp + ((c ^ (row & 7)) << 4));
              const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float lo = __uint_as_float(ws[e] << 16), hi = __uint_as_float(ws[e] & 0xFFFF0000u);
                q = fmaf(lo, lo, q);
                q = fmaf(hi, hi, q);
              }
            }
            const float y = q - comp;  // Kahan over the rows
            const float t = part + y;
            comp = (t - part) - y;
            part = t;
          }
          acc += (double)part - (double)comp;
          // the slot is refilled by TMA (async proxy): order these reads first
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
          if (++s == (uint32_t)S) {
            s = 0;
            sph ^= 1;
          }
        }
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) nred[h] = acc;
    if (!ok) *abort_flag = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (want_norm && threadIdx.x == 0) {
    a.nrm_part[4 * blockIdx.x] = nred[0];
    a.nrm_part[4 * blockIdx.x + 1] = nred[1];
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// fixed-order reduction of the unit partials into Z (packed by zoff): a
// compensated (Kahan) FP32 sum, since FP64 arithmetic would bound this pass
struct RedArgs {
  SkArgs s;
  int64_t zoff[TDK_MAX_MODES + 1];
  int64_t pstride[TDK_MAX_MODES];  // strides of p over the outer modes
};

__global__ void sketch_tc_reduce(RedArgs ra, double* __restrict__ Z) {
  const SkArgs& a = ra.s;
  const int N = a.N, nj = N - 2, nl = N - 1;
  const int64_t total = ra.zoff[N];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (e >= ra.zoff[n + 1]) ++n;
    const int Rn = a.Rt[n];
    const int64_t i = (e - ra.zoff[n]) / Rn;
    const int r = (int)((e - ra.zoff[n]) % Rn);
    float s = 0.f, cmp = 0.f;  // compensated FP32 sum of FP32 partials, fixed order
    auto add = [&](float v) {
      const float y = v - cmp;
      const float t = s + y;
      cmp = (t - s) - y;
      s = t;
    };
    // one unit's partial entry (the checked build tests the unit and the offset)
    auto part_at = [&](int64_t u, int64_t off) -> float {
      return (TDK_IN(u, a.nunits) && TDK_IN(off, a.ustride)) ? a.part[u * a.ustride + off] : 0.f;
    };
    if (n == nl) {
      const int kr = (int)(i / a.KRW);
      const int64_t kl = i - (int64_t)kr * a.KRW;
      for (int jt = 0; jt < a.JT; ++jt)
        for (int pc = 0; pc < a.PC; ++pc) {
          const int64_t u = ((int64_t)jt * a.KR + kr) * a.PC + pc;
          add(part_at(u, a.poff_last + kl * Rn + r));
        }
    } else if (n == nj) {
      const int jt = (int)(i / 128);
      const int64_t jl = i - (int64_t)jt * 128;
      for (int kr = 0; kr < a.KR; ++kr)
        for (int pc = 0; pc < a.PC; ++pc) {
          const int64_t u = ((int64_t)jt * a.KR + kr) * a.PC + pc;
          add(part_at(u, a.poff_j + jl * Rn + r));
        }
    } else {
      // every p with i_n(p) = i: enumerate the other outer indices
      int64_t cnt = a.P / a.I[n];
      for (int64_t o = 0; o < cnt; ++o) {
        int64_t rem = o, p = i * ra.pstride[n];
        for (int k = N - 3; k >= 0; --k) {
          if (k == n) continue;
          p += (rem % a.I[k]) * ra.pstride[k];
          rem /= a.I[k];
        }
        const int pc = (int)(p / a.PCW);
        const int64_t pl = p - (int64_t)pc * a.PCW;
        for (int jt = 0; jt < a.JT; ++jt)
          for (int kr = 0; kr < a.KR; ++kr) {
            const int64_t u = ((int64_t)jt * a.KR + kr) * a.PC + pc;
            add(part_at(u, a.poff_p[n] + pl * Rn + r));
          }
      }
    }
    Z[e] = (double)s - (double)cmp;
  }
}

// fixed-order sum of per-warp partials (one block)
__global__ void sum_parts_kernel(const double* __restrict__ parts, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += parts[i];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
    *out = t;
  }
}

// FP32 copies of every W_k^(n) in one launch (blockIdx.y: the matrix)
struct WCopies {
  const double* s[TDK_MAX_MODES * TDK_MAX_MODES];
  float* d[TDK_MAX_MODES * TDK_MAX_MODES];
  int64_t n[TDK_MAX_MODES * TDK_MAX_MODES];
};
__global__ void w_to_f32(const __grid_constant__ WCopies c) {
  const int m = blockIdx.y;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < c.n[m]; e += (int64_t)gridDim.x * blockDim.x)
    c.d[m][e] = (float)c.s[m][e];
}

// WN^T block: rows = channels of modes < N-1 (each padded to 16; one block for
// all of them when they share W_{N-1}), columns = L
__global__ void build_wn(const double* const* __restrict__ Wl, SkArgs a, int ldw, __nv_bfloat16* __restrict__ out) {
  const int64_t total = (int64_t)a.N1 * ldw;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / ldw);
    const int k = (int)(e % ldw);
    float v = 0.f;
    int n = 0;
    while (n + 1 < a.N - 1 && c >= a.off[n + 1]) ++n;
    const int r = c - a.off[n];
    if (r < a.Rt[n] && k < a.L) v = (float)Wl[n][(int64_t)k * a.Rt[n] + r];
    out[e] = __float2bfloat16_rn(v);
  }
}

}  // namespace


// ---------------------------------------------------------------- host: sketch
template <bool F32, int RW>
static int launch_sketch(tdk_ctx* ctx, const CUtensorMap& tmY, const CUtensorMap& tmW, const SkArgs& a, int grid,
                         size_t smem) {
  auto k = tc_sketch_kernel<F32, RW>;
  TDK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k<<<grid, 320, smem, ctx->stream>>>(tmY, tmW, a);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

int sketch_tc(tdk_ctx* ctx, const Geom& g, int dtype, const void* Y, const double* const W[], double* Zdst,
              double* normY2) {
  if (g.N < 3 || g.N > 4 || !tc_shape_ok(g, dtype) || dtype == TDK_F64) return TDK_ENOTSUP;
  TDK_HMARK("sketch_tc: start");
  const bool f32 = dtype == TDK_F32;
  const int N = g.N, nj = N - 2, nl = N - 1;
  SkArgs a{};
  a.N = N;
  for (int n = 0; n < N; ++n) {
    a.I[n] = g.I[n];
    a.Rt[n] = g.Rt[n];
    a.Rtp[n] = (g.Rt[n] + 15) / 16 * 16;
  }
  a.L = (int)g.I[nl];
  a.J = (int)g.I[nj];
  a.P = 1;
  for (int k = 0; k < nj; ++k) a.P *= g.I[k];
  // G1 channels: one block per mode n < N-1 holding W_{N-1}^(n).  When every
  // such mode passes the same matrix (a sketch family whose Khatri-Rao factors
  // are shared between the modes, W_k^(n) = W_k), one block serves them all and
  // the G1 contraction is done once for all of them.
  bool shared = true;
  for (int n = 1; n <= nj; ++n)
    if (W[n * N + nl] != W[nl] || g.Rt[n] != g.Rt[0]) shared = false;
  int N1 = 0;
  for (int n = 0; n <= nj; ++n) {
    a.off[n] = shared ? 0 : N1;
    if (!shared || n == 0) N1 += a.Rtp[n];
  }
  a.N1 = N1;
  if (N1 > 256) return TDK_ENOTSUP;
  a.RtL = g.Rt[nl];
  a.hilo = (f32 && a.RtL <= 32) ? 1 : 0;
  if (!f32 && a.RtL > 64) return TDK_ENOTSUP;
  // the form with the test matrices in TMEM takes BF16 data whose channels of
  // the modes < N fit one 128-lane accumulator (each mode's own block; a shared
  // family is not folded there); the form with a resident W block takes the rest
  int N1tw = 0;
  for (int n = 0; n <= nj; ++n) N1tw += a.Rtp[n];
  // (a shared family has half the G1 channels in the resident block, which
  // the resident form exploits)
  bool tw = !f32 && !shared && N1tw <= 128;
#ifdef TDK_TESTING
  if (const char* e = getenv("TDK_SKETCH_FORM")) tw = tw && strcmp(e, "resident") != 0;
#endif
  if (tw) {
    int off = 0;
    for (int c = 0; c < 128; ++c) {
      a.lane_mode[c] = -1;
      a.lane_r[c] = 0;
    }
    for (int n = 0; n <= nj; ++n) {
      a.off[n] = off;
      for (int r = 0; r < a.Rtp[n]; ++r) {
        a.lane_mode[off + r] = (signed char)(r < a.Rt[n] ? n : -1);
        a.lane_r[off + r] = (unsigned char)r;
      }
      off += a.Rtp[n];
    }
    a.N1 = N1 = off;
    a.d1_cols = 128;
    // columns per unit: KS = 3 leaves TMEM room for one D1^T buffer, KS <= 2
    // for two (W 64 KS + D1^T 128 nd1 + D2 64 KS <= 512 columns); least
    // padding of the contiguous mode, ties to the widest; deepest ring
    a.KS = 0;
    int64_t best_cols = 0;
    int fit_st = 0;
    for (int st = TW_SMAX; st >= 2 && !fit_st; --st)
      if (1024 + (size_t)tw_layout(st).total <= (size_t)ctx->max_smem_optin) fit_st = st;
    if (!fit_st) return TDK_ENOTSUP;
    for (int ks = 3; ks >= 1; --ks) {
      if (ks > (a.L + 127) / 128 && ks > 1) continue;
      const int64_t w = 128LL * ks;
      const int64_t cols = (a.L + w - 1) / w * w;
      if (!a.KS || cols < best_cols) {
        a.KS = ks;
        best_cols = cols;
      }
    }
    a.S = fit_st;
#ifdef TDK_TESTING
    if (const char* e = getenv("TDK_SKETCH_KS")) a.KS = std::max(1, std::min(3, atoi(e)));
    if (const char* e = getenv("TDK_SKETCH_S")) a.S = std::max(2, std::min(fit_st, atoi(e)));
#endif
    a.nd1 = a.KS == 3 ? 1 : 2;
  }
  a.d1_cols = tw ? 128 : (N1 + 31) / 32 * 32;
  // columns per unit (KS blocks of 128): among the widths that TMEM (two D1
  // buffers + KS D2 blocks) and shared memory (ring of at least two stages +
  // resident W block) allow, the one that pads the contiguous mode least (a
  // padded column costs a full column of work), ties to the widest (the per-p
  // epilogue is amortised over more bytes); then the deepest ring that fits
  if (!tw) {
    const uint32_t stage_b = f32 ? SkLayout<true>::STAGE_BYTES : SkLayout<false>::STAGE_BYTES;
    a.KS = 0;
    int64_t best_cols = 0;
    for (int ks = 4; ks >= 1; --ks) {
      if (ks > (a.L + 127) / 128 && ks > 1) continue;
      if (2 * a.d1_cols + ks * 64 > 512) continue;
      int fit_st = 0;
      for (int st = SK_SMAX; st >= 2 && !fit_st; --st) {
        const size_t need = 1024 + (size_t)st * stage_b + ((2 * ks * N1 * 128 + 1023) & ~1023) + SK_KTB * 16 * KB +
                            256 + 2 * 4 * 64 * 4 + SK_CB * 256 * 4 + 64;
        if (need <= (size_t)ctx->max_smem_optin) fit_st = st;
      }
      if (!fit_st) continue;
      const int64_t w = 128LL * ks;
      const int64_t cols = (a.L + w - 1) / w * w;
      if (!a.KS || cols < best_cols) {
        a.KS = ks;
        a.S = fit_st;
        best_cols = cols;
      }
    }
    if (!a.KS) return TDK_ENOTSUP;
#ifdef TDK_TESTING
    // test build: the column blocks per unit and the ring depth can be forced
    // (for sweeps of the launch shape); a shape that does not fit is refused
    if (const char* e = getenv("TDK_SKETCH_KS")) {
      const int ks = atoi(e);
      const char* es = getenv("TDK_SKETCH_S");
      const int st = es ? atoi(es) : 2;
      const size_t need = 1024 + (size_t)st * stage_b + ((2 * ks * N1 * 128 + 1023) & ~1023) + SK_KTB * 16 * KB +
                          256 + 2 * 4 * 64 * 4 + SK_CB * 256 * 4 + 64;
      if (ks < 1 || ks > 4 || st < 2 || st > SK_SMAX || 2 * a.d1_cols + ks * 64 > 512 ||
          need > (size_t)ctx->max_smem_optin)
        return TDK_ENOTSUP;
      a.KS = ks;
      a.S = st;
    }
#endif
  }
  a.KRW = 128 * a.KS;
  a.JT = (a.J + 127) / 128;
  a.KR = (a.L + a.KRW - 1) / a.KRW;
  const int64_t base_units = (int64_t)a.JT * a.KR;
  int64_t want = 8LL * ctx->num_sms;
  int64_t PC = (want + base_units - 1) / base_units;
  if (PC > a.P) PC = a.P;
  if (PC < 1) PC = 1;
  a.PCW = (a.P + PC - 1) / PC;
  a.PC = (int)((a.P + a.PCW - 1) / a.PCW);
  a.nunits = base_units * a.PC;
  a.poff_last = 0;
  a.poff_j = (int64_t)a.KRW * a.RtL;
  int64_t o = a.poff_j + 128LL * g.Rt[nj];
  for (int n = 0; n < nj; ++n) {
    a.poff_p[n] = o;
    o += a.PCW * g.Rt[n];
  }
  a.ustride = (o + 63) / 64 * 64;
  a.status = ctx->d_status;
  a.yhint = 1;
#ifdef TDK_TESTING
  if (const char* e = getenv("TDK_SKETCH_YHINT")) a.yhint = atoi(e) != 0;
#endif
#ifdef TDK_TESTING
  const bool want_prof = getenv("TDK_SKETCH_PROFILE") != nullptr;
#else
  const bool want_prof = false;
#endif
  if (want_prof) {
    TDK_CUDA_TRY(cudaMallocAsync((void**)&a.prof, 16 * sizeof(unsigned long long), ctx->stream));
    TDK_CUDA_TRY(cudaMemsetAsync(a.prof, 0, 16 * sizeof(unsigned long long), ctx->stream));
  }

  // workspace: FP32 W copies, WN^T (BF16), partials
  const int ldw = (a.L + 7) / 8 * 8;
  Planner pl;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k)
      if (k != n) pl.take<float>((size_t)g.I[k] * g.Rt[n]);
  if (!tw) {
    pl.take<__nv_bfloat16>((size_t)N1 * ldw);
    pl.take<const double*>(TDK_MAX_MODES);
  }
  pl.take<float>((size_t)a.nunits * a.ustride);
  pl.take<double>((size_t)4 * ctx->num_sms);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  WCopies wc{};
  int nw = 0;
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < N; ++k) {
      a.Wf[n][k] = nullptr;
      if (k == n) continue;
      float* d = cv.take<float>((size_t)g.I[k] * g.Rt[n]);
      wc.s[nw] = W[n * N + k];
      wc.d[nw] = d;
      wc.n[nw] = g.I[k] * g.Rt[n];
      ++nw;
      a.Wf[n][k] = d;
    }
  w_to_f32<<<dim3(16, nw), 256, 0, ctx->stream>>>(wc);
  TDK_LAUNCH_CHECK(ctx);
  TDK_HMARK("sketch_tc: plan, workspace, W to FP32");
  __nv_bfloat16* wn = nullptr;
  if (!tw) {
    wn = cv.take<__nv_bfloat16>((size_t)N1 * ldw);
    const double** wl = cv.take<const double*>(TDK_MAX_MODES);
    const double* hw[TDK_MAX_MODES] = {};
    for (int n = 0; n <= nj; ++n) hw[n] = W[n * N + nl];
    TDK_CUDA_TRY(cudaMemcpyAsync(wl, hw, sizeof(hw), cudaMemcpyHostToDevice, ctx->stream));
    build_wn<<<128, 256, 0, ctx->stream>>>(wl, a, ldw, wn);
    TDK_LAUNCH_CHECK(ctx);
  }
  TDK_HMARK("sketch_tc: W block");
  a.part = cv.take<float>((size_t)a.nunits * a.ustride);
  // ||Y||^2 on the side of the pass: the norm warps of the TMEM-W form, the
  // converter warps of FP32 data; per warp and CTA, summed in a fixed order
  double* nrmp = cv.take<double>((size_t)4 * ctx->num_sms);
  a.nrm_part = (normY2 && (tw || f32)) ? nrmp : nullptr;
  if (a.nrm_part) TDK_CUDA_TRY(cudaMemsetAsync(nrmp, 0, sizeof(double) * 4 * ctx->num_sms, ctx->stream));

  CUtensorMap tmY, tmW;
  {
    const int es = f32 ? 4 : 2;
    uint64_t dims[3] = {(uint64_t)a.L, (uint64_t)a.J, (uint64_t)a.P};
    uint64_t str[2] = {(uint64_t)a.L * es, (uint64_t)a.L * a.J * es};
    uint32_t box[3] = {f32 ? 32u : 64u, 128u, 1u};
    rc = encode_tmap(&tmY, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Y, dims,
                     str, box, true);
    if (rc) return rc;
    if (!tw) {
      uint64_t wd[3] = {(uint64_t)a.L, (uint64_t)N1, 1};
      uint64_t ws_[2] = {(uint64_t)ldw * 2, (uint64_t)ldw * 2 * N1};
      uint32_t wb[3] = {64u, (uint32_t)N1, 1u};
      rc = encode_tmap(&tmW, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, wn, wd, ws_, wb, true);
      if (rc) return rc;
    }
  }
  TDK_HMARK("sketch_tc: tensor maps");
  int grid = (int)std::min<int64_t>(a.nunits, ctx->num_sms);
  if (tw) {
    const size_t smem = 1024 + (size_t)tw_layout(a.S).total;
    if (smem > (size_t)ctx->max_smem_optin) return TDK_ENOTSUP;
    ProfScope ps(ctx, 0);
    auto k = tc_sketch_tw_kernel;
    TDK_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, 384, smem, ctx->stream>>>(tmY, a);
    TDK_LAUNCH_CHECK(ctx);
  } else {
    const uint32_t stage = f32 ? SkLayout<true>::STAGE_BYTES : SkLayout<false>::STAGE_BYTES;
    const size_t smem = 1024 + (size_t)a.S * stage + ((2 * a.KS * N1 * 128 + 1023) & ~1023) + SK_KTB * 16 * KB +
                        256 + 2 * 4 * 64 * 4 + SK_CB * 256 * 4 + 64;
    if (smem > (size_t)ctx->max_smem_optin) return TDK_ENOTSUP;
    ProfScope ps(ctx, 0);
    int rw = 0;
    for (int n = 0; n < N; ++n) rw = std::max(rw, a.Rtp[n]);
    rc = (rw <= 32) ? (f32 ? launch_sketch<true, 32>(ctx, tmY, tmW, a, grid, smem)
                           : launch_sketch<false, 32>(ctx, tmY, tmW, a, grid, smem))
                    : (f32 ? launch_sketch<true, 64>(ctx, tmY, tmW, a, grid, smem)
                           : launch_sketch<false, 64>(ctx, tmY, tmW, a, grid, smem));
    if (rc) return rc;
  }
  TDK_HMARK("sketch_tc: kernel launched");
  RedArgs ra{};
  ra.s = a;
  for (int n = 0; n <= N; ++n) ra.zoff[n] = g.zoff[n];
  {
    int64_t s = 1;
    for (int k = nj - 1; k >= 0; --k) {
      ra.pstride[k] = s;
      s *= g.I[k];
    }
  }
  sketch_tc_reduce<<<(unsigned)std::min<int64_t>((g.zoff[N] + 255) / 256, 65535), 256, 0, ctx->stream>>>(ra, Zdst);
  TDK_LAUNCH_CHECK(ctx);
  if (normY2) {
    if (a.nrm_part) {
      sum_parts_kernel<<<1, 256, 0, ctx->stream>>>(nrmp, 4 * grid, normY2);
      TDK_LAUNCH_CHECK(ctx);
    } else {
      rc = norm2_pass(ctx, g, dtype, Y, normY2);
      if (rc) return rc;
    }
  }
  if (want_prof) {
    unsigned long long hp[16];
    TDK_CUDA_TRY(cudaMemcpyAsync(hp, a.prof, sizeof(hp), cudaMemcpyDeviceToHost, ctx->stream));
    TDK_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    cudaFree(a.prof);
    const char* nm_res[14] = {"mma:other", "mma:wait_d1empty", "mma:wait_ktile", "mma:wait_data", "mma:issue",
                              "tma:other", "tma:wait_empty", "-", "epi:other", "epi:ktile", "epi:wait_d1",
                              "epi:rowmode", "epi:reduce", "epi:tailbar"};
    const char* nm_tw[14] = {"mma:other", "mma:wait_d1empty", "mma:wait_ktile", "mma:wait_data", "mma:issue",
                             "tma:other", "tma:wait_empty", "-", "epi:other", "epi:ktile", "epi:wait_d1",
                             "epi:read+fma", "epi:bar+store", "epi:unit_setup"};
    const char* const* nm = tw ? nm_tw : nm_res;
    fprintf(stderr, "tdk sketch profile (%s form, KS %d, S %d, CTA 0, Mcycles, units %lld):",
            tw ? "TMEM-W" : "resident-W", a.KS, a.S, (long long)a.nunits);
    for (int i = 0; i < 14; ++i)
      if (i != 7) fprintf(stderr, " %s=%.2f", nm[i], hp[i] / 1e6);
    fprintf(stderr, "\n");
  }
  return TDK_OK;
}

}  // namespace tdk

#ifdef TDK_TESTING
// ---- test library only (not in the public header): a bounded wait that cannot be
// satisfied.  One thread waits for the first phase of an mbarrier that nothing
// arrives at; after limit_ns it raises the timeout bit in the context's status
// word and returns, exactly as the waits of the passes above do.
namespace tdk {
namespace {
__global__ void wait_probe_kernel(unsigned* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    tc::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t0 = tc::globaltimer();
    while (!tc::mbar_try_wait(tc::smem_u32(&bar), 0)) {
      if (tc::globaltimer() - t0 > limit_ns) {
        atomicOr(status, TDK_STATUS_TIMEOUT);
        break;
      }
    }
  }
}
}  // namespace
}  // namespace tdk

extern "C" int tdk_test_bounded_wait(tdk_ctx* ctx, unsigned long long limit_ns) {
  using namespace tdk;
  if (!ctx || limit_ns == 0 || limit_ns > 100000000ull) return TDK_EINVAL;  // at most 0.1 s
  cudaSetDevice(ctx->device);
  wait_probe_kernel<<<1, 32, 0, ctx->stream>>>(ctx->d_status, limit_ns);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}
#endif  // TDK_TESTING

namespace tdk {
TDK_CHECKED_UNIT(tc_sketch)
}  // namespace tdk
