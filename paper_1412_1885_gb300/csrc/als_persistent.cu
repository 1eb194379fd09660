// FFCP sweep loop as ONE persistent cooperative kernel (Alg. 1, Eqs. 9, 12-14).
//
// Every CTA holds all normalised factors B_p and their Grams in shared memory.
// Per mode n:
//   1. each CTA forms T_n = HADAMARD_{p != n} Gram_p and its Cholesky factor in
//      FP64 (redundantly, so nothing has to be broadcast);
//   2. CTA c computes rows i = c, c+G, ... of H_n = G_(n) [KRP_{p != n} B_p]
//      from the core slice G[.., i, ..] staged in shared memory, contracting
//      one mode at a time (the last other mode first as a small GEMM, then
//      weighted sums over the others), and solves its rows of B_n = H_n T_n^{-1}
//      in FP64 (Eq. 14);
//   3. grid barrier; every CTA reads the new rows, computes lambda, the
//      normalised factor and its Gram -- identically, in the same order.
// Nonnegative form: rows of H_n, barrier, rows of A_n = max(0, U_n H_n T_n^{-1})
// (T_n from the Grams of the A_p), barrier, then lambda, the Gram of A_n and
// B_n = U_n^T A_n.  After the last mode every CTA evaluates the same fit from
// the Gram identities, so all CTAs stop on the same sweep.  A Cholesky pivot
// at or below R*eps*max(diag) is seen by every CTA alike; they all leave and
// the host reruns the call on the multi-kernel form, which has the
// pseudo-inverse.  Barrier waits are bounded (timeout bit, then exit).
#include <chrono>
#include <cmath>
#include <cstdlib>

#include "tc_common.cuh"

namespace tdk {

// outputs of an ALS run: B_io <- B (normalised), A_io <- U_n B_n (or the
// nonnegative A_n given in Aw), lambda absorbed into the last factor
int als_finish(tdk_ctx* ctx, const Geom& g, int R, bool dbl, const void* const* Bw, const double* const* U,
               const double* lam, double* const* Aw, double* const* B_io, double* const* A_io, double* lambda_out,
               const float* const* Uf);

namespace {

constexpr int RMAXP = TDK_MAX_RANK;
constexpr int NTP = 256;
constexpr int ST_TIMEOUT = 0x100, ST_NEEDPINV = 0x200;
constexpr int NS_MAX_IT = 8;  // Newton-Schulz updates before Gauss-Jordan takes over
constexpr int NORM_BLOCKS = 64;  // blocks of the ||G||^2 pass

struct PState {
  int sweeps;
  int converged;
  int status;
  int pad;
  double fit;
  double fitY;
};

template <class T>
struct PArgs {
  int N, R, nonneg, max_sweeps;
  int nn_rule;                  // nonneg: 0 projected LS, 1 HALS (Eq. 8), 2 multiplicative (Eq. 15)
  int clip;                     // nonneg path: project onto x >= 0 (0: the signed l1 form)
  double l1;                    // soft threshold of the LS rows (Eq. 16), 0 = none
  double tol;
  int Rt[TDK_MAX_MODES];
  int64_t I[TDK_MAX_MODES];
  int64_t stride[TDK_MAX_MODES];
  int64_t gnumel;
  int64_t Qmax, Amax;           // shared buffers (entries)
  const T* G;
  const T* Uf[TDK_MAX_MODES];   // U_n in the working precision [I_n x Rt_n]
  const T* Ulo[TDK_MAX_MODES];  // FP32 cores, nonneg: U_n - Uf_n, so that Uf + Ulo carries U to ~2^-48
  const double* init[TDK_MAX_MODES];  // B0 (Rt_n x R) or, nonneg, A0 (I_n x R)
  T* Bnew;                      // [max(Rt,I) x R] update rows (unnormalised)
  T* H;                         // [Rtmax x R]
  T* Hpart;                     // [grid x R] partial rows of H_n
  T* Bout[TDK_MAX_MODES];       // final normalised B_n (CTA 0)
  double* Aout[TDK_MAX_MODES];  // nonneg: final normalised A_n (CTA 0)
  double* lam_out;
  double* hist;
  int hist_cap;
  PState* st;
  unsigned* bar;                // arrival counter, generation
  unsigned* status;
  const double* nG2;
  const double* nY2;            // may be null
  double* rpart;                // [grid] per-CTA residual partials
  unsigned long long* prof;     // optional: cycles per phase, CTA 0 (null = off)
  float* xprev;                 // grid kernel: [grid][N][R*R] each CTA's last FP32 inverse of T_n
  float ns_gate;                // Newton-Schulz start accepted while ||I - T X||_F < ns_gate
  int64_t ulo_elems;            // FP32 nonneg: max I_n Rt_n (the staged low part of U_n)
  int64_t cache_elems;          // > 0: each CTA keeps its core slice of every mode in shared memory
  int64_t coff[TDK_MAX_MODES];  //   at these offsets of the cache (entries)
};

__device__ bool grid_sync(unsigned* bar, unsigned* status) {
  __syncthreads();
  __shared__ int fail;
  if (threadIdx.x == 0) {
    // the arrival counter only grows (zeroed before the launch): barrier k
    // completes when it reaches (k + 1) * gridDim.x, so the last CTA to
    // arrive releases the others with its own increment and no reset
    fail = 0;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    const unsigned target = (arrived / gridDim.x + 1u) * gridDim.x;
    volatile unsigned* cnt = bar;
    const unsigned long long t0 = tc::globaltimer();
    while ((int)(*cnt - target) < 0) {
      if (tc::globaltimer() - t0 > tc::WAIT_LIMIT_NS) {
        atomicOr(status, TDK_STATUS_TIMEOUT);
        fail = 1;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return fail == 0;
}

// FP32 -> FP64 by integer operations, which run on the integer pipes (FP64
// instructions, conversions included, issue at a small fraction of the FP32
// rate on this GPU): exact for zeros, normal numbers, infinities and NaNs;
// subnormal inputs take the hardware conversion.
__device__ __forceinline__ double f2d_int(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (ex == 0u) return (u & 0x7fffffu) ? (double)x : __longlong_as_double((long long)sign);
  const unsigned long long e64 = ex == 0xffu ? 0x7ffull : (unsigned long long)(ex + 896u);
  return __longlong_as_double((long long)(sign | (e64 << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// block-wide FP64 sum, the same value (same order) in every thread; the warp
// partials are added by one thread (FP64 arithmetic is scarce on this GPU)
// Gram entries of FP32 factors with compensated accumulation: each product is
// split exactly (FMA) and the running sum carries its rounding error (TwoSum),
// so an entry is accurate to a few FP32 units squared.  The fit of the
// nonnegative form subtracts two sums of Gram products of nearly equal size;
// with plain FP32 sums their rounding noise (about 1e-7 of ||G||^2) exceeded
// the stopping tolerance and made the sweep count a matter of summation order.
template <class T>
struct GramAcc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x, T y) {
    if (sizeof(T) == 8) {
      s = fma(x, y, s);
    } else {
      const T p = x * y;
      const T e = fma(x, y, -p);
      const T t = s + p;
      const T z = t - s;
      c += ((s - (t - z)) + (p - z)) + e;
      s = t;
    }
  }
  __device__ __forceinline__ T value() const { return s + c; }
};

// dst[e] = src[e] for e < n by the threads t < nt, eight loads in flight per
// thread before their stores (a plain loop waits out the L2 latency once per
// element: the loads cannot pass the shared-memory stores).  L2-coherent
// loads: src may have been written by other CTAs before a grid barrier.
template <class D, class S>
__device__ __forceinline__ void stage_cg(D* dst, const S* src, int64_t n, int t, int nt) {
  constexpr int U = 8;
  for (int64_t b = t; b < n; b += (int64_t)U * nt) {
    S v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = b + (int64_t)u * nt;
      v[u] = e < n ? __ldcg(src + e) : S(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = b + (int64_t)u * nt;
      if (e < n) dst[e] = (D)v[u];
    }
  }
}

// Gram matrix out = X^T X of X [rows x R] (row stride ldx) with compensated
// sums, by the threads t < nt of the block: the entries r <= s only, two per
// thread in flight, each written to (r, s) and (s, r).  A product and its
// FMA error are the same with the operands swapped, so the result is the one
// the full R x R loop gives, for half the work.
template <class T>
__device__ void gram_sym(const T* X, int64_t rows, int ldx, int R, T* out, int t, int nt) {
  const int np = R * (R + 1) / 2;
  auto decode = [](int q, int& r, int& s) {  // q = s (s + 1) / 2 + r, r <= s
    s = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
    while (s * (s + 1) / 2 > q) --s;
    while ((s + 1) * (s + 2) / 2 <= q) ++s;
    r = q - s * (s + 1) / 2;
  };
  for (int q0 = t; q0 < np; q0 += 2 * nt) {
    const int q1 = q0 + nt < np ? q0 + nt : q0;
    int r0, s0, r1, s1;
    decode(q0, r0, s0);
    decode(q1, r1, s1);
    GramAcc<T> a0, a1;
    for (int64_t i = 0; i < rows; ++i) {
      const T* x = X + i * ldx;
      a0.add(x[r0], x[s0]);
      a1.add(x[r1], x[s1]);
    }
    const T v0 = a0.value(), v1 = a1.value();
    out[r0 * R + s0] = v0;
    out[s0 * R + r0] = v0;
    if (q0 + nt < np) {
      out[r1 * R + s1] = v1;
      out[s1 * R + r1] = v1;
    }
  }
}

// Float-float arithmetic (value = hi + lo) for the explicit residual of the
// FP32 fit.  Products are split exactly by an FMA and every sum keeps its
// rounding error (TwoSum), the compensated scheme of Ogita, Rump and Oishi
// (SIAM J. Sci. Comput. 26, 2005).  The residual norm then comes out accurate
// to about 2^-44 whatever the order of the sums, so the stopping test sees the
// change of the fit between sweeps rather than FP32 rounding noise, which near
// convergence is as large as a relative change of 1e-7 and made the sweep
// count differ between two kernels that sum in different orders.
struct FFAcc {
  float s = 0.f, c = 0.f;
  // s + c += ph + pl
  __device__ __forceinline__ void add(float ph, float pl) {
    const float t = s + ph;
    const float z = t - s;
    c += ((s - (t - z)) + (ph - z)) + pl;
    s = t;
  }
  // s + c += (xh + xl) y
  __device__ __forceinline__ void fma2(float xh, float xl, float y) {
    const float p = xh * y;
    add(p, fmaf(xl, y, fmaf(xh, y, -p)));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
// (xh + xl) y as a float-float pair
__device__ __forceinline__ void ff_mul(float xh, float xl, float y, float& ph, float& pl) {
  ph = xh * y;
  pl = fmaf(xl, y, fmaf(xh, y, -ph));
}
// acc += (g - (xh + xl))^2, the difference and its square in float-float
__device__ __forceinline__ void ff_add_sq_diff(FFAcc& acc, float g, float xh, float xl) {
  const float d0 = g - xh;  // TwoSum: d0 + e0 = g - xh exactly
  const float z = d0 - g;
  const float e0 = (g - (d0 - z)) + (-xh - z);
  const float e1 = e0 - xl;
  const float dh = d0 + e1;  // renormalised: dh + dl = d0 + e1
  const float dl = e1 - (dh - d0);
  const float q = dh * dh;
  acc.add(q, fmaf(2.f * dh, dl, fmaf(dh, dh, -q)));
}

// block-wide sum of float-float accumulators, the same value in every
// thread: a butterfly over each warp in float-float, the warps' pairs added
// in order by one thread, one conversion to FP64 at the end (the FP64 form
// of the same sum spends most of its time in FP64 shuffles and additions)
__device__ __forceinline__ double block_sum_ff(FFAcc a, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, a.s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, a.c, o);
    a.add(s2, c2);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* rf = reinterpret_cast<float2*>(red);
  __syncthreads();
  if (lane == 0) rf[w] = make_float2(a.s, a.c);
  __syncthreads();
  if (threadIdx.x == 0) {
    FFAcc t;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t.add(rf[i].x, rf[i].y);
    red[0] = t.value();
  }
  __syncthreads();
  const double v = red[0];
  __syncthreads();
  return v;
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[0] = s;
  }
  __syncthreads();
  const double s = red[0];
  __syncthreads();
  return s;
}

#define PROF_MARK(ph)                                                            \
  do {                                                                           \
    if (a.prof && blockIdx.x == 0) {                                             \
      __syncthreads();                                                           \
      if (threadIdx.x == 0) {                                                    \
        const unsigned long long t_ = clock64();                                 \
        s_pf[(ph)] += t_ - prof_t; /* shared: no global round trip per mark */   \
        prof_t = t_;                                                             \
      }                                                                          \
    }                                                                            \
  } while (0)

// shared-memory plan of the persistent kernel, every region 16-byte aligned
template <class T>
struct PLayout {
  size_t o_bs, o_gram, o_bgram, o_tm, o_invd, o_part, o_lam, o_xrow, o_hrow, o_red, o_lf, o_tid, o_gjs, o_yf,
      o_lamt, o_ilamt, o_slice, o_work, o_egram, o_ns, o_cache, o_ulo, total;
  __host__ __device__ void plan(int N, int R, int btot, int64_t Qmax, int64_t Amax, bool egram, int64_t cache,
                                int64_t ulo) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
      const size_t o = (off + 15) & ~size_t(15);
      off = o + bytes;
      return o;
    };
    o_bs = take(sizeof(T) * btot);
    o_gram = take(sizeof(T) * N * R * R);
    o_bgram = take(sizeof(T) * N * R * R);
    o_tm = take(sizeof(double) * R * R);
    o_invd = take(sizeof(double) * RMAXP);
    o_part = take(sizeof(double) * 8 * RMAXP);  // partial sums of the solve's products
    o_lam = take(sizeof(double) * RMAXP);
    o_xrow = take(sizeof(double) * RMAXP);
    o_hrow = take(sizeof(double) * RMAXP);
    o_red = take(sizeof(double) * 32);
    o_lf = take(sizeof(float) * R * R);
    o_tid = take(sizeof(double) * R * R);
    o_gjs = take(sizeof(double) * 4 * RMAXP);
    o_yf = take(sizeof(float) * RMAXP);
    o_lamt = take(sizeof(T) * RMAXP);
    o_ilamt = take(sizeof(T) * RMAXP);
    o_slice = take(sizeof(T) * (size_t)Qmax);
    o_work = take(sizeof(T) * (size_t)(Amax * R));
    o_egram = take(egram ? sizeof(T) * N * R * R : 0);  // Grams of A_p - U_p B_p
    o_ns = take(sizeof(float) * R * R);                 // Newton-Schulz iterate
    o_cache = take(sizeof(T) * (size_t)cache);          // core slices kept across sweeps
    o_ulo = take(egram ? sizeof(T) * (size_t)ulo : 0);  // FP32 nonneg: U_n - Uf_n staged
    total = (off + 15) & ~size_t(15);
  }
};

// In-place inverse of a symmetric positive definite R x R matrix (row-major)
// by Gauss-Jordan elimination without pivoting, spread over a group of nt
// threads (named barrier bar_id).  A pivot is the Schur complement a Cholesky
// factorisation would meet, so the breakdown test (pivot not above
// R * eps * max diag) is the same.  Each thread keeps its entries
// e = t + q nt (at most EPT of them) in registers for the whole elimination,
// with their row and column decoded once.  Per pivot k it loads the pivot row
// and column entries it needs from `buf` (4 R entries, two halves) before
// any store, updates its entries, and the threads that hold row k+1 and
// column k+1 copy them into the other half: one barrier per pivot, and the
// loads of a step in flight together.  Returns the same value in every
// thread of the group.
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

template <class F, int EPT>
__device__ int gj_inverse_regs(F* A, F* buf, int R, F eps, int t, int nt, int bar_id) {
  tc::named_bar(bar_id, nt);  // `buf` may still be read by a previous call
  F mx = F(0);
  for (int j = 0; j < R; ++j) mx = A[j * R + j] > mx ? A[j * R + j] : mx;
  const F tiny = (F)R * eps * mx;
  const int RR = R * R;
  F a[EPT];
  int ri[EPT], ci[EPT];  // row and column of each entry; -1: none
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = t + q * nt;
    ri[q] = e < RR ? e / R : -1;
    ci[q] = e < RR ? e - ri[q] * R : 0;
    a[q] = e < RR ? A[e] : F(0);
  }
  if (t < R) {
    buf[t] = A[t];
    buf[R + t] = A[t * R];
  }
  tc::named_bar(bar_id, nt);
  int ok = 1;
  for (int k = 0; k < R; ++k) {
    const F* rowk = buf + (k & 1) * 2 * R;
    const F* colk = rowk + R;
    F* rown = buf + ((k + 1) & 1) * 2 * R;
    F* coln = rown + R;
    const F p = rowk[k];
    if (!(p > tiny)) {
      ok = 0;
      break;
    }
    const F ip = rcp_rn(p);
    F rv[EPT], cv[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      rv[q] = ri[q] >= 0 ? rowk[ci[q]] : F(0);
      cv[q] = ri[q] >= 0 ? colk[ri[q]] : F(0);
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const bool rk = ri[q] == k, ck = ci[q] == k;
      a[q] = rk ? (ck ? ip : rv[q] * ip) : (ck ? -cv[q] * ip : fma(-cv[q], rv[q] * ip, a[q]));
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      if (ri[q] == k + 1) rown[ci[q]] = a[q];
      if (ri[q] >= 0 && ci[q] == k + 1) coln[ri[q]] = a[q];
    }
    tc::named_bar(bar_id, nt);
  }
  if (!ok) return 0;
#pragma unroll
  for (int q = 0; q < EPT; ++q)
    if (ri[q] >= 0) A[t + q * nt] = a[q];
  tc::named_bar(bar_id, nt);
  return 1;
}

// The same elimination, two pivots per barrier: step k takes pivots k and
// k+1 together, each entry composed from the two single-pivot updates (the
// first pivot's update of the entry, of its row's entry in column k+1 and of
// its column's entry in row k+1, then the second pivot's), so the result is
// the one-pivot-per-step elimination's to the rounding of the same
// operations, with half the barriers and dependency chains.  `buf` holds,
// double-buffered, rows k and k+1 and columns k and k+1 (8 R entries); an
// odd last pivot is a single step.  FP32 only (the FP64 fallback keeps the
// one-pivot form and its 4 R buffer).
template <int EPT>
__device__ int gj_inverse_regs2(float* A, float* buf, int R, float eps, int t, int nt, int bar_id) {
  tc::named_bar(bar_id, nt);  // `buf` may still be read by a previous call
  float mx = 0.f;
  for (int j = 0; j < R; ++j) mx = A[j * R + j] > mx ? A[j * R + j] : mx;
  const float tiny = (float)R * eps * mx;
  const int RR = R * R;
  float a[EPT];
  int ri[EPT], ci[EPT];  // row and column of each entry; -1: none
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = t + q * nt;
    ri[q] = e < RR ? e / R : -1;
    ci[q] = e < RR ? e - ri[q] * R : 0;
    a[q] = e < RR ? A[e] : 0.f;
  }
  if (t < R) {
    buf[t] = A[t];
    buf[2 * R + t] = A[t * R];
    if (R > 1) {
      buf[R + t] = A[R + t];
      buf[3 * R + t] = A[t * R + 1];
    }
  }
  tc::named_bar(bar_id, nt);
  int ok = 1;
  for (int k = 0, h = 0; k < R; k += 2, h ^= 1) {
    const float* rk = buf + h * 4 * R;  // row k
    const float* rk1 = rk + R;          // row k+1
    const float* ck = rk + 2 * R;       // column k
    const float* ck1 = rk + 3 * R;      // column k+1
    float* nx = buf + (h ^ 1) * 4 * R;  // rows and columns k+2, k+3
    const float p00 = rk[k];
    if (!(p00 > tiny)) {
      ok = 0;
      break;
    }
    const float ip0 = rcp_rn(p00);
    if (k + 1 == R) {  // the odd last pivot alone
      float rv[EPT], cv[EPT];
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        rv[q] = ri[q] >= 0 ? rk[ci[q]] : 0.f;
        cv[q] = ri[q] >= 0 ? ck[ri[q]] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const bool r0 = ri[q] == k, c0 = ci[q] == k;
        a[q] = r0 ? (c0 ? ip0 : rv[q] * ip0) : (c0 ? -cv[q] * ip0 : fmaf(-cv[q], rv[q] * ip0, a[q]));
      }
      tc::named_bar(bar_id, nt);
      break;
    }
    const int k1 = k + 1;
    const float u = rk[k1] * ip0;   // A[k][k1] / p00
    const float w = rk1[k];         // A[k1][k]
    const float s = fmaf(-w, u, rk1[k1]);
    if (!(s > tiny)) {
      ok = 0;
      break;
    }
    const float is = rcp_rn(s);
    float rv0[EPT], rv1[EPT], cv0[EPT], cv1[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const bool on = ri[q] >= 0;
      rv0[q] = on ? rk[ci[q]] : 0.f;
      rv1[q] = on ? rk1[ci[q]] : 0.f;
      cv0[q] = on ? ck[ri[q]] : 0.f;
      cv1[q] = on ? ck1[ri[q]] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int i = ri[q], j = ci[q];
      // after the first pivot: the entry, its row's entry in column k1, its
      // column's entry in row k1
      const float aij = i == k ? (j == k ? ip0 : rv0[q] * ip0)
                               : (j == k ? -cv0[q] * ip0 : fmaf(-cv0[q], rv0[q] * ip0, a[q]));
      const float aik1 = i == k ? u : fmaf(-cv0[q], u, cv1[q]);
      const float ak1j = j == k ? -w * ip0 : fmaf(-w, rv0[q] * ip0, rv1[q]);
      a[q] = i == k1 ? (j == k1 ? is : ak1j * is) : (j == k1 ? -aik1 * is : fmaf(-aik1, ak1j * is, aij));
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      if (ri[q] < 0) continue;
      if (ri[q] == k + 2) nx[ci[q]] = a[q];
      if (ri[q] == k + 3) nx[R + ci[q]] = a[q];
      if (ci[q] == k + 2) nx[2 * R + ri[q]] = a[q];
      if (ci[q] == k + 3) nx[3 * R + ri[q]] = a[q];
    }
    tc::named_bar(bar_id, nt);
  }
  if (!ok) return 0;
#pragma unroll
  for (int q = 0; q < EPT; ++q)
    if (ri[q] >= 0) A[t + q * nt] = a[q];
  tc::named_bar(bar_id, nt);
  return 1;
}

template <class F>
__device__ int group_gj_inverse_smem(F* A, F* buf, int R, F eps, int t, int nt, int bar_id);

// entries per thread chosen by the size (R <= 64 and nt >= 256); MAXEPT caps
// the register arrays (a kernel short of registers takes the shared-memory
// form above it)
template <class F, int MAXEPT = 16>
__device__ int group_gj_inverse(F* A, F* buf, int R, F eps, int t, int nt, int bar_id) {
  const int per = (R * R + nt - 1) / nt;
  if constexpr (sizeof(F) == 4) {
    float* Af = reinterpret_cast<float*>(A);
    float* bf = reinterpret_cast<float*>(buf);
    if (per <= 4) return gj_inverse_regs2<4>(Af, bf, R, (float)eps, t, nt, bar_id);
    if (MAXEPT >= 8 && per <= 8) return gj_inverse_regs2<(MAXEPT >= 8 ? 8 : 4)>(Af, bf, R, (float)eps, t, nt, bar_id);
  }
  if (per <= 4) return gj_inverse_regs<F, 4>(A, buf, R, eps, t, nt, bar_id);
  if (MAXEPT >= 8 && per <= 8) return gj_inverse_regs<F, (MAXEPT >= 8 ? 8 : 4)>(A, buf, R, eps, t, nt, bar_id);
  if (MAXEPT >= 16) return gj_inverse_regs<F, (MAXEPT >= 16 ? 16 : 4)>(A, buf, R, eps, t, nt, bar_id);
  return group_gj_inverse_smem<F>(A, buf, R, eps, t, nt, bar_id);
}

// the same elimination with the matrix kept in shared memory (every entry
// read and written per pivot): the single-CTA kernel's form, whose small
// matrices leave most of the register form's slots idle (51.9 against
// 53.8 us per sweep on a 20^3 core, R = 10); the register form takes the
// 60^3 core, R = 40, from 59k to 42k cycles per inverse
template <class F>
__device__ int group_gj_inverse_smem(F* A, F* buf, int R, F eps, int t, int nt, int bar_id) {
  tc::named_bar(bar_id, nt);
  F mx = F(0);
  for (int j = 0; j < R; ++j) mx = A[j * R + j] > mx ? A[j * R + j] : mx;
  const F tiny = (F)R * eps * mx;
  const int RR = R * R;
  const float invR = 1.0f / (float)R;
  if (t < R) {
    buf[t] = A[t];
    buf[R + t] = A[t * R];
  }
  tc::named_bar(bar_id, nt);
  for (int k = 0; k < R; ++k) {
    const F* rowk = buf + (k & 1) * 2 * R;
    const F* colk = rowk + R;
    F* rown = buf + ((k + 1) & 1) * 2 * R;
    F* coln = rown + R;
    const F p = rowk[k];
    if (!(p > tiny)) return 0;
    const F ip = F(1) / p;
    for (int e = t; e < RR; e += nt) {
      const int i = __float2int_rz(((float)e + 0.5f) * invR);  // e / R (exact for e < 4096)
      const int j = e - i * R;
      F v;
      if (i == k) v = (j == k) ? ip : rowk[j] * ip;
      else v = (j == k) ? -colk[i] * ip : fma(-colk[i], rowk[j] * ip, A[e]);
      A[e] = v;
      if (i == k + 1) rown[j] = v;
      if (j == k + 1) coln[i] = v;
    }
    tc::named_bar(bar_id, nt);
  }
  return 1;
}

// Newton-Schulz refinement of an approximate inverse X of T (Schulz 1933;
// Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed., 14.5):
//   E = I - T X,   X <- X + X E,
// after which I - T X = E^2, so the Frobenius norm f of the residual at
// least squares at every step once it is below 1.  Started from the inverse
// of the previous sweep's T_n, which moved only as far as the factors did, it
// reaches the FP32 floor in a few steps: two R x R products per step instead
// of the R barrier-separated pivot steps of Gauss-Jordan elimination.
// T, X0, X1, E: R x R row-major FP32 (shared memory), X0 holding the start;
// computed by the nt threads of a group (named barrier bar_id) in 2 x 4
// register tiles; red: nt / 32 floats.  Returns the buffer that holds the
// inverse once f <= tol (at most max_it updates), with f in *dev and the
// updates in *nit, or null when the start's f is not below `gate` or f stops
// falling; the same outcome in every thread.
__device__ const float* ns_inverse(const float* T, float* X0, float* X1, float* E, float* red, int R, float tol,
                                   int max_it, float gate, float* dev, int* nit, int t, int nt, int bar_id) {
  const int tr = (R + 1) / 2, tcn = (R + 3) / 4;
  // C = I - A B (sub = true: returns the sum of squares of C) or C = Xc + A B
  auto prod = [&](const float* A, const float* B, const float* Xc, float* C, bool sub) -> float {
    float sq = 0.f;
    for (int tile = t; tile < tr * tcn; tile += nt) {
      const int i0 = (tile / tcn) * 2, j0 = (tile % tcn) * 4;
      float acc[2][4] = {};
      for (int k = 0; k < R; ++k) {
        float a2[2], b4[4];
#pragma unroll
        for (int u = 0; u < 2; ++u) a2[u] = (i0 + u < R) ? A[(i0 + u) * R + k] : 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) b4[v] = (j0 + v < R) ? B[k * R + j0 + v] : 0.f;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a2[u], b4[v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (i0 + u < R && j0 + v < R) {
            const int e = (i0 + u) * R + j0 + v;
            if (sub) {
              const float cv = ((i0 + u == j0 + v) ? 1.f : 0.f) - acc[u][v];
              C[e] = cv;
              sq = fmaf(cv, cv, sq);
            } else {
              C[e] = Xc[e] + acc[u][v];
            }
          }
    }
    return sq;
  };
  auto group_sum = [&](float v) -> float {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[t >> 5] = v;
    tc::named_bar(bar_id, nt);
    float m = 0.f;
    for (int w = 0; w < (nt >> 5); ++w) m += red[w];
    tc::named_bar(bar_id, nt);  // red is rewritten by the next call
    return m;
  };
  tc::named_bar(bar_id, nt);  // T and X0 written by the group
  float* X = X0;
  float* Xn = X1;
  float f = sqrtf(group_sum(prod(T, X, nullptr, E, true)));
  for (int it = 0;; ++it) {
    *nit = it;
    *dev = f;
    if (f <= tol) return X;
    if (!(f < gate) || it == max_it) return nullptr;
    prod(X, E, X, Xn, false);
    tc::named_bar(bar_id, nt);
    float* tmp = X;
    X = Xn;
    Xn = tmp;
    const float fn = sqrtf(group_sum(prod(T, X, nullptr, E, true)));
    // below 1 the residual at least squares: stop when it falls by less than
    // half (the FP32 floor); above 1, while it falls at all (its spectral
    // radius, which squares, may be below 1 with a larger Frobenius norm)
    if (!(fn <= tol) && !(fn < (f < 1.f ? 0.5f * f : f))) {
      *nit = it + 1;
      *dev = fn;
      return nullptr;
    }
    f = fn;
  }
}

template <class T>
__global__ void __launch_bounds__(NTP, 1) als_persistent_kernel(PArgs<T> a) {
  unsigned long long prof_t = clock64();
  __shared__ unsigned long long s_pf[32];  // cycles per phase and counts (CTA 0, profiled runs)
  if (threadIdx.x < 32) s_pf[threadIdx.x] = 0;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ double s_irows[TDK_MAX_MODES];  // 1 / sqrt(rows of the updated factor of mode n)
  const int N = a.N, R = a.R;
  int boff[TDK_MAX_MODES];
  int btot = 0;
  for (int p = 0; p < N; ++p) {
    boff[p] = btot;
    btot += a.Rt[p] * R;
  }
  PLayout<T> L;
  const bool leak32 = sizeof(T) == 4 && a.nonneg;  // FP32 nonneg: the out-of-subspace term from E_p
  L.plan(N, R, btot, a.Qmax, a.Amax, leak32, a.cache_elems, a.ulo_elems);
  T* Bs = reinterpret_cast<T*>(sm + L.o_bs);         // factors, packed
  T* egram = reinterpret_cast<T*>(sm + L.o_egram);   // [N][R*R] Grams of D_p = A_p - U_p B_p
  T* gram = reinterpret_cast<T*>(sm + L.o_gram);     // [N][R*R]
  T* bgram = reinterpret_cast<T*>(sm + L.o_bgram);   // [N][R*R] (nonneg: Grams of B_p)
  double* Tm = reinterpret_cast<double*>(sm + L.o_tm);  // [R*R] T_n (FP64)
  double* invd = reinterpret_cast<double*>(sm + L.o_invd);
  double* spart = reinterpret_cast<double*>(sm + L.o_part);  // [8][RMAXP]
  double* lam = reinterpret_cast<double*>(sm + L.o_lam);
  double* xrow = reinterpret_cast<double*>(sm + L.o_xrow);
  double* hrow = reinterpret_cast<double*>(sm + L.o_hrow);  // right-hand side
  double* red = reinterpret_cast<double*>(sm + L.o_red);    // [32]
  float* Lf = reinterpret_cast<float*>(sm + L.o_lf);        // [R*R] FP32 inverse of T_n
  double* Tid = reinterpret_cast<double*>(sm + L.o_tid);   // [R*R] FP64 inverse (fallback); Newton-Schulz X, E
  float* nsX1 = reinterpret_cast<float*>(sm + L.o_ns);       // [R*R] Newton-Schulz iterate
  double* gjs = reinterpret_cast<double*>(sm + L.o_gjs);   // Gauss-Jordan pivot rows / columns (two pairs)
  float* yf = reinterpret_cast<float*>(sm + L.o_yf);       // [R] FP32 right-hand side of a solve step
  T* lamT = reinterpret_cast<T*>(sm + L.o_lamt);
  T* ilamT = reinterpret_cast<T*>(sm + L.o_ilamt);
  T* slice = reinterpret_cast<T*>(sm + L.o_slice);   // [Qmax]
  T* work = reinterpret_cast<T*>(sm + L.o_work);     // [Amax * R]
  T* cache = reinterpret_cast<T*>(sm + L.o_cache);   // [cache_elems]
  T* ulo_s = reinterpret_cast<T*>(sm + L.o_ulo);     // [ulo_elems]

  const int tid = threadIdx.x;
  const int G = gridDim.x, c = blockIdx.x;
  bool ok = true;
  if (tid < N) s_irows[tid] = 1.0 / sqrt((double)(a.nonneg ? a.I[tid] : a.Rt[tid]));
  // the HALS and multiplicative rules start every mode from its running A_n:
  // in the first sweep that is the given A0 (read after a grid barrier)
  if (a.nonneg && a.nn_rule != 0 && c == 0)
    for (int n = 0; n < N; ++n)
      for (int64_t e = tid; e < a.I[n] * R; e += NTP) a.Aout[n][e] = a.init[n][e];

  // ---- initial factors (raw) and their Grams.  Unconstrained: B_n as
  //      given.  Nonnegative: A_n staged in FP32 in the update-rows buffer
  //      and U_n (with its low part, FP32 nonneg) beside it, B_n = U_n^T A_n,
  //      and for FP32 cores D_n = A_n - U_n B_n and its Gram E_n (see below),
  //      all from shared memory
  for (int n = 0; n < N; ++n) {
    const int Rn = a.Rt[n];
    if (!a.nonneg) {
      for (int e = tid; e < Rn * R; e += NTP) Bs[boff[n] + e] = (T)a.init[n][e];
      __syncthreads();
      gram_sym<T>(Bs + boff[n], Rn, R, R, gram + n * R * R, tid, NTP);
      gram_sym<T>(Bs + boff[n], Rn, R, R, bgram + n * R * R, tid, NTP);
    } else {
      const int64_t rows = a.I[n];
      T* nb = slice;
      stage_cg(nb, a.init[n], rows * R, tid, NTP);
      stage_cg(work, a.Uf[n], rows * Rn, tid, NTP);
      if (leak32) stage_cg(ulo_s, a.Ulo[n], rows * Rn, tid, NTP);
      __syncthreads();
      for (int e = tid; e < Rn * R; e += NTP) {
        const int q = e / R, r = e % R;
        T s4[4] = {T(0), T(0), T(0), T(0)};
        int64_t i = 0;
        for (; i + 3 < rows; i += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) s4[u] = fma(work[(i + u) * Rn + q], nb[(i + u) * R + r], s4[u]);
        }
        for (; i < rows; ++i) s4[0] = fma(work[i * Rn + q], nb[i * R + r], s4[0]);
        Bs[boff[n] + e] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
      }
      gram_sym<T>(nb, rows, R, R, gram + n * R * R, tid, NTP);
      __syncthreads();
      gram_sym<T>(Bs + boff[n], Rn, R, R, bgram + n * R * R, tid, NTP);
      if (leak32) {
        const int nE = (int)(rows * R);
        for (int e0 = tid; e0 < nE; e0 += 2 * NTP) {
          const int e1 = e0 + NTP < nE ? e0 + NTP : e0;
          const int i0 = e0 / R, r0 = e0 - i0 * R, i1 = e1 / R, r1 = e1 - i1 * R;
          GramAcc<T> d0, d1;
          T l0 = T(0), l1 = T(0);  // (U_n's low part: its product needs no compensation)
          d0.s = nb[e0];
          d1.s = nb[e1];
          for (int q = 0; q < Rn; ++q) {
            const T b0 = Bs[boff[n] + q * R + r0], b1 = Bs[boff[n] + q * R + r1];
            d0.add(-work[i0 * Rn + q], b0);
            d1.add(-work[i1 * Rn + q], b1);
            l0 = fma(ulo_s[i0 * Rn + q], b0, l0);
            l1 = fma(ulo_s[i1 * Rn + q], b1, l1);
          }
          nb[e0] = d0.value() - l0;
          if (e0 + NTP < nE) nb[e1] = d1.value() - l1;
        }
        __syncthreads();
        gram_sym<T>(nb, rows, R, R, egram + n * R * R, tid, NTP);
      }
    }
    __syncthreads();
  }
  for (int r = tid; r < R; r += NTP) {
    lam[r] = 1.0;
    lamT[r] = T(1);
  }
  __syncthreads();
  const double nG2 = *a.nG2;
  const double nY2 = a.nY2 ? *a.nY2 : 0.0;

  double fit = 0.0, fitY = nan("");
  int sweep = 0, converged = 0, needpinv = 0;
  unsigned have_prev = 0;  // modes whose last FP32 inverse is in this CTA's xprev slot
  for (sweep = 1; sweep <= a.max_sweeps && ok; ++sweep) {
    double inner = 0.0;
    for (int n = 0; n < N && ok; ++n) {
      PROF_MARK(8);
      const int Rn = a.Rt[n];
      // ---- 1. T_n (FP64) and a Cholesky factor: FP32 by default, the solves
      //         then refined against T_n in FP64; FP64 factor in place if an
      //         FP32 pivot is not positive enough
      for (int e = tid; e < R * R; e += NTP) {
        T vt = T(1);
        for (int p = 0; p < N; ++p)
          if (p != n) vt *= gram[p * R * R + e];
        Lf[e] = (float)vt;
        double v = 1.0;
        if (sizeof(T) == 4) {
          // the product of the FP32 entries in float-float (exact for two
          // factors, 2^-48 for more), one FP64 addition to join the halves
          float h = 0.f, l = 0.f;
          bool first = true;
          for (int p = 0; p < N; ++p) {
            if (p == n) continue;
            const float y = (float)gram[p * R * R + e];
            if (first) {
              h = y;
              first = false;
            } else {
              const float ph = h * y;
              l = fmaf(l, y, fmaf(h, y, -ph));
              h = ph;
            }
          }
          v = f2d_int(h) + f2d_int(l);
        } else {
          for (int p = 0; p < N; ++p)
            if (p != n) v *= (double)gram[p * R * R + e];
        }
        Tm[e] = v;
      }
      __syncthreads();
      PROF_MARK(7);
      // ---- 1b. inverse of T_n: FP32 by default (the solves are refined against
      //          T_n in FP64), FP64 if an FP32 pivot breaks down.  From the
      //          second sweep on, Newton-Schulz steps from the previous sweep's
      //          inverse, Gauss-Jordan when they do not converge.  The solve
      //          error after k refinement steps is f^(k+1), f = ||I - T X||_F:
      //          FP32 cores accept f <= 2^-9 and take one step when f <= 2^-13
      //          (error below 2^-26), else two; FP64 cores accept f <= 2^-17
      //          and take two.
      // (the HALS and multiplicative rules use T_n itself, not its inverse)
      bool use32 = true;
      int nref = 2;
      if (!(a.nonneg && a.nn_rule != 0)) {
        float* xp = a.xprev + ((int64_t)c * N + n) * R * R;
        const float* Xi = nullptr;
        if (have_prev & (1u << n)) {
          float* X0 = reinterpret_cast<float*>(Tid);
          for (int e = tid; e < R * R; e += NTP) X0[e] = xp[e];
          float dev = 1.f;
          int nit = 0;
          Xi = ns_inverse(Lf, X0, nsX1, X0 + R * R, reinterpret_cast<float*>(gjs), R,
                          sizeof(T) == 4 ? 0x1p-9f : 0x1p-17f, NS_MAX_IT, a.ns_gate, &dev, &nit, tid, NTP, 1);
          if (a.prof && blockIdx.x == 0 && tid == 0) {
            s_pf[18] += nit;
            if (!Xi) s_pf[nit == 0 ? 16 : 17] += 1;  // rejected at the start / stalled
          }
          if (Xi) {
            for (int e = tid; e < R * R; e += NTP) Lf[e] = Xi[e];
            if (sizeof(T) == 4 && dev <= 0x1p-13f) nref = 1;
          }
        }
        if (!Xi) {
          use32 = group_gj_inverse<float>(Lf, reinterpret_cast<float*>(gjs), R, 1.1920929e-7f, tid, NTP, 1) != 0;
          if (a.prof && !use32 && blockIdx.x == 0 && tid == 0) s_pf[9] += 1;  // FP64 inverses
          if (!use32) {
            for (int e = tid; e < R * R; e += NTP) Tid[e] = Tm[e];
            __syncthreads();
            if (!group_gj_inverse<double>(Tid, gjs, R, 2.220446049250313e-16, tid, NTP, 1)) {
              needpinv = 1;
              ok = false;  // identical in every CTA: all leave here
              break;
            }
          }
        } else if (a.prof && blockIdx.x == 0 && tid == 0) {
          s_pf[10] += 1;  // Newton-Schulz inverses
        }
        __syncthreads();
        if (use32) {
          for (int e = tid; e < R * R; e += NTP) xp[e] = Lf[e];
          have_prev |= 1u << n;
        } else {
          have_prev &= ~(1u << n);
        }
      }
      __syncthreads();
      // x <- x T_n^{-1} for the row in xrow, block-parallel: one product with the
      // inverse, then nref refinement steps against T_n in FP64 (invd: residual)
      // (the FP32 products read FP32 copies of the right-hand side and the
      // residual: one conversion per entry instead of one per term, FP64
      // conversions running at the FP64 rate)
      // Each product of the solve (R outputs, R terms) runs on SP * R threads:
      // part p of output o sums its range of terms, and the parts are added
      // in order, which keeps the dependent FMA chains (FP64 ones above all)
      // short.
      const int SP = R >= NTP ? 1 : (NTP / R > 8 ? 8 : NTP / R);
      float* partf = reinterpret_cast<float*>(spart);
      auto prod32 = [&](const float* v, const float* M) {  // partf[o] <- sum_q v[q] M[q, o] (FP32)
        if (tid < SP * R) {
          const int o = tid % R, pp = tid / R;
          float acc = 0.f;
          for (int q = pp * R / SP; q < (pp + 1) * R / SP; ++q) acc = fmaf(v[q], M[q * R + o], acc);
          partf[pp * RMAXP + o] = acc;
        }
        __syncthreads();
      };
      auto prod64 = [&](const double* v, const double* M) {  // spart[o] <- sum_q v[q] M[q, o] (FP64)
        if (tid < SP * R) {
          const int o = tid % R, pp = tid / R;
          double acc = 0.0;
          for (int q = pp * R / SP; q < (pp + 1) * R / SP; ++q) acc = fma(v[q], M[q * R + o], acc);
          spart[pp * RMAXP + o] = acc;
        }
        __syncthreads();
      };
      auto sum32 = [&](int o) {
        float s2 = 0.f;
        for (int pp = 0; pp < SP; ++pp) s2 += partf[pp * RMAXP + o];
        return s2;
      };
      auto sum64 = [&](int o) {
        double s2 = 0.0;
        for (int pp = 0; pp < SP; ++pp) s2 += spart[pp * RMAXP + o];
        return s2;
      };
      auto solve_row = [&]() {
        for (int r = tid; r < R; r += NTP) {
          hrow[r] = xrow[r];
          yf[r] = (float)xrow[r];
        }
        __syncthreads();
        if (use32) prod32(yf, Lf);
        else prod64(hrow, Tid);
        for (int r = tid; r < R; r += NTP) xrow[r] = use32 ? (double)sum32(r) : sum64(r);
        __syncthreads();
        for (int it = 0; it < nref; ++it) {
          prod64(xrow, Tm);  // (x T_n)[q]
          for (int q = tid; q < R; q += NTP) {
            const double rr = hrow[q] - sum64(q);
            invd[q] = rr;
            yf[q] = (float)rr;
          }
          __syncthreads();
          if (use32) prod32(yf, Lf);
          else prod64(invd, Tid);
          for (int r = tid; r < R; r += NTP) xrow[r] += use32 ? (double)sum32(r) : sum64(r);
          __syncthreads();
        }
      };

      PROF_MARK(0);
      // ---- 2. rows of H_n (unconstrained: and of B_n).  Each row is split over
      //         Pn CTAs by ranges of the slowest other mode; the partial rows
      //         are summed in a fixed order after one more grid barrier.
      int oth[TDK_MAX_MODES];
      int no = 0;
      for (int p = 0; p < N; ++p)
        if (p != n) oth[no++] = p;
      const int last = oth[no - 1];
      const int Rl = a.Rt[last];
      const int64_t sl = a.stride[last];
      const int R0o = a.Rt[oth[0]];
      const int64_t A1 = a.gnumel / Rn / Rl;  // slice rows: all other modes but the last
      const int64_t per0 = A1 / R0o;          // slice rows per index of the slowest other mode
      int Pn = G / Rn;
      Pn = Pn < 1 ? 1 : (Pn > R0o ? R0o : Pn);
      for (int wk = c; wk < Rn * Pn; wk += G) {
        const int i = wk % Rn, part = wk / Rn;
        const int lo = (int)((int64_t)part * R0o / Pn), hi = (int)((int64_t)(part + 1) * R0o / Pn);
        const int64_t rows0 = (int64_t)(hi - lo) * per0;
        // slice S[a1, l] of this part, one index decode per slice row
        // slice S[a1, l] of this part, eight loads in flight per thread; with
        // the cache on, this CTA's part is the same in every sweep and the
        // slice is read from the core once
        const T* Gi = a.G + (int64_t)i * a.stride[n];
        T* S = a.cache_elems > 0 ? cache + a.coff[n] : slice;
        if (a.cache_elems == 0 || sweep == 1) {
          // (32-bit index arithmetic: a slice of the core holds far fewer
          // than 2^31 entries, and 64-bit division is a long subroutine)
          constexpr int U = 8;
          const int ns = (int)(rows0 * Rl);
          for (int b = tid; b < ns; b += U * NTP) {
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int e = b + u * NTP;
              v[u] = T(0);
              if (e < ns) {
                const int a1 = e / Rl;
                const int l = e - a1 * Rl;
                int rem = a1 + lo * (int)per0;
                int off = 0;
                for (int k = no - 2; k >= 0; --k) {
                  const int p = oth[k];
                  off += (rem % a.Rt[p]) * (int)a.stride[p];
                  rem /= a.Rt[p];
                }
                off += l * (int)sl;
                if (TDK_IN((int64_t)i * a.stride[n] + off, a.gnumel)) v[u] = Gi[off];
              }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int e = b + u * NTP;
              if (e < ns) S[e] = v[u];
            }
          }
        }
        __syncthreads();
        PROF_MARK(11);
        // work[a1, r] = sum_l S[a1, l] B_last[l, r] in 4 x 4 register tiles
        {
          const T* Bq = Bs + boff[last];
          const int64_t ta = (rows0 + 3) / 4;
          const int tr = (R + 3) / 4;
          for (int64_t tile = tid; tile < ta * tr; tile += NTP) {
            const int64_t a0 = (tile / tr) * 4;
            const int r0 = (int)(tile % tr) * 4;
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
            for (int l = 0; l < Rl; ++l) {
              T s4[4], b4[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) s4[u] = (a0 + u < rows0) ? S[(a0 + u) * Rl + l] : T(0);
#pragma unroll
              for (int v = 0; v < 4; ++v) b4[v] = (r0 + v < R) ? Bq[l * R + r0 + v] : T(0);
#pragma unroll
              for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(s4[u], b4[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v)
                if (a0 + u < rows0 && r0 + v < R) work[(a0 + u) * R + r0 + v] = acc[u][v];
          }
        }
        __syncthreads();
        PROF_MARK(12);
        // remaining other modes, last to first: out[b, r] = sum_m in[b*Rp + m, r] B_p[m, r];
        // the slowest one only over this part's range
        T* in = work;
        T* out = slice;
        int64_t rows = rows0;
        for (int k = no - 2; k >= 0; --k) {
          const int p = oth[k];
          const int Rp = (k == 0) ? (hi - lo) : a.Rt[p];
          const int64_t nrows = rows / Rp;
          const T* Bp = Bs + boff[p] + (k == 0 ? (int64_t)lo * R : 0);
          for (int64_t e = tid; e < nrows * R; e += NTP) {
            const int64_t b = e / R;
            const int r = (int)(e % R);
            T acc = T(0);
            for (int m = 0; m < Rp; ++m) acc = fma(in[(b * Rp + m) * R + r], Bp[m * R + r], acc);
            out[e] = acc;
          }
          __syncthreads();
          T* tt = in;
          in = out;
          out = tt;
          rows = nrows;
        }
        PROF_MARK(13);
        if (Pn == 1) {
          for (int r = tid; r < R; r += NTP) {
            if (TDK_IN((int64_t)i * R + r, (int64_t)Rn * R)) a.H[(int64_t)i * R + r] = in[r];
            xrow[r] = (double)in[r];
          }
          __syncthreads();
          if (!a.nonneg) {
            solve_row();
            __syncthreads();
            for (int r = tid; r < R; r += NTP)
              if (TDK_IN((int64_t)i * R + r, (int64_t)Rn * R)) a.Bnew[(int64_t)i * R + r] = (T)xrow[r];
          }
        } else {
          for (int r = tid; r < R; r += NTP)
            if (TDK_IN(((int64_t)part * Rn + i) * R + r, (int64_t)gridDim.x * R))
              a.Hpart[((int64_t)part * Rn + i) * R + r] = in[r];
        }
        __syncthreads();
      }
      if (Pn > 1) {
        if (!grid_sync(a.bar, a.status)) { ok = false; break; }
        for (int i = c; i < Rn; i += G) {
          for (int r = tid; r < R; r += NTP) {
            T sum = T(0);
            for (int part = 0; part < Pn; ++part) sum += __ldcg(a.Hpart + ((int64_t)part * Rn + i) * R + r);
            a.H[(int64_t)i * R + r] = sum;
            xrow[r] = (double)sum;
          }
          __syncthreads();
          if (!a.nonneg) {
            solve_row();
            __syncthreads();
            for (int r = tid; r < R; r += NTP) a.Bnew[(int64_t)i * R + r] = (T)xrow[r];
          }
          __syncthreads();
        }
      }
      PROF_MARK(1);
      if (!grid_sync(a.bar, a.status)) { ok = false; break; }
      PROF_MARK(2);

      if (a.nonneg) {
        // rows of A_n = max(0, (U_n H_n) T_n^{-1}); H_n staged in shared memory
        stage_cg(work, a.H, (int64_t)Rn * R, tid, NTP);
        __syncthreads();
        for (int64_t i = c; i < a.I[n]; i += G) {
          for (int r = tid; r < R; r += NTP) {
            T m = T(0);
            for (int q = 0; q < Rn; ++q) m = fma(a.Uf[n][i * Rn + q], work[q * R + r], m);
            xrow[r] = (double)m;
          }
          __syncthreads();
          if (a.nn_rule == 0) {
            solve_row();
            __syncthreads();
            for (int r = tid; r < R; r += NTP) {
              double x = xrow[r];
              if (a.l1 > 0.0) x = copysign(fmax(fabs(x) - a.l1, 0.0), x);
              if (TDK_IN(i * R + r, a.I[n] * R)) a.Bnew[i * R + r] = (T)(a.clip ? fmax(x, 0.0) : x);
            }
          } else {
            // from the current iterate of the row, A_n[i, :] diag(lambda) (FP64)
            for (int r = tid; r < R; r += NTP) hrow[r] = __ldcg(a.Aout[n] + i * R + r) * lam[r];
            __syncthreads();
            if (a.nn_rule == 2) {
              // multiplicative: a <- a (*) P_+(m) (/) (a T_n); 0 where a T_n is not positive
              for (int r = tid; r < R; r += NTP) {
                double d = 0.0;
                for (int q = 0; q < R; ++q) d = fma(hrow[q], Tm[q * R + r], d);
                if (TDK_IN(i * R + r, a.I[n] * R)) a.Bnew[i * R + r] = (T)(d > 0.0 ? hrow[r] * fmax(xrow[r], 0.0) / d : 0.0);
              }
            } else {
              // HALS, column by column: a_r <- P_+(a_r + (m_r - a t_r) / t_rr), one warp
              if (tid < 32) {
                for (int r = 0; r < R; ++r) {
                  double part = 0.0;
                  for (int q = tid; q < R; q += 32) part = fma(hrow[q], Tm[q * R + r], part);
                  part = warp_sum(part);
                  if (tid == 0) hrow[r] = fmax(0.0, hrow[r] + (xrow[r] - part) / Tm[r * R + r]);
                  __syncwarp();
                }
              }
              __syncthreads();
              for (int r = tid; r < R; r += NTP)
                if (TDK_IN(i * R + r, a.I[n] * R)) a.Bnew[i * R + r] = (T)hrow[r];
            }
          }
          __syncthreads();
        }
        if (!grid_sync(a.bar, a.status)) { ok = false; break; }
      }

      PROF_MARK(3);
      // ---- 3. lambda, normalised factor and its Gram (every CTA, same order)
      const int64_t rows = a.nonneg ? a.I[n] : Rn;
      T* nb = slice;  // [rows x R] the update rows, then normalised (the slice is free here)
      stage_cg(nb, a.Bnew, rows * R, tid, NTP);
      __syncthreads();
      {
        const int w = tid >> 5, lane = tid & 31;
        for (int r = w; r < R; r += NTP / 32) {
          T s2 = T(0);
          for (int64_t i = lane; i < rows; i += 32) {
            const T v = nb[i * R + r];
            s2 = fma(v, v, s2);
          }
          s2 = warp_sum(s2);
          if (lane == 0) {
            const T l = sqrt(s2);
            lamT[r] = l;
            ilamT[r] = l > T(0) ? T(1) / l : T(0);
            lam[r] = (double)l;
          }
        }
      }
      __syncthreads();
      const T inv_rows = (T)s_irows[n];
      for (int64_t e = tid; e < rows * R; e += NTP) {
        const int r = (int)(e % R);
        nb[e] = lamT[r] > T(0) ? nb[e] * ilamT[r] : inv_rows;
      }
      if (a.nonneg)  // U_n staged in the work buffer for B_n = U_n^T A_n
        stage_cg(work, a.Uf[n], rows * Rn, tid, NTP);
      if (leak32) stage_cg(ulo_s, a.Ulo[n], rows * Rn, tid, NTP);
      __syncthreads();
      PROF_MARK(14);
      gram_sym<T>(nb, rows, R, R, gram + n * R * R, tid, NTP);
      PROF_MARK(15);
      if (!a.nonneg) {
        for (int e = tid; e < Rn * R; e += NTP) Bs[boff[n] + e] = nb[e];
      } else {
        // (four partial sums over the rows in flight, added in a fixed order)
        for (int e = tid; e < Rn * R; e += NTP) {
          const int q = e / R, r = e % R;
          T s4[4] = {T(0), T(0), T(0), T(0)};
          int64_t i = 0;
          for (; i + 3 < rows; i += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) s4[u] = fma(work[(i + u) * Rn + q], nb[(i + u) * R + r], s4[u]);
          }
          for (; i < rows; ++i) s4[0] = fma(work[i * Rn + q], nb[i * R + r], s4[0]);
          Bs[boff[n] + e] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        }
        if (c == 0)
          for (int64_t e = tid; e < rows * R; e += NTP) a.Aout[n][e] = (double)nb[e];
        __syncthreads();
        gram_sym<T>(Bs + boff[n], Rn, R, R, bgram + n * R * R, tid, NTP);
        if (leak32) {
          // the part of the normalised A_n outside the Tucker subspace,
          // D_n = A_n - U_n B_n (U_n = Uf + Ulo), in place of the staged rows,
          // and its Gram E_n.  The out-of-subspace term of the fit is then a
          // sum of products that contain E (no difference of near-equal
          // norms), so its error stays far below the stopping tolerance
          // (U_n's low part staged beside its high part; two entries per
          // thread in flight, their compensated chains independent)
          __syncthreads();
          const int nE = (int)(rows * R);
          for (int e0 = tid; e0 < nE; e0 += 2 * NTP) {
            const int e1 = e0 + NTP < nE ? e0 + NTP : e0;
            const int i0 = e0 / R, r0 = e0 - i0 * R, i1 = e1 / R, r1 = e1 - i1 * R;
            GramAcc<T> d0, d1;
            T l0 = T(0), l1 = T(0);  // (U_n's low part: its product needs no compensation)
            d0.s = nb[e0];
            d1.s = nb[e1];
            for (int q = 0; q < Rn; ++q) {
              const T b0 = Bs[boff[n] + q * R + r0], b1 = Bs[boff[n] + q * R + r1];
              d0.add(-work[i0 * Rn + q], b0);
              d1.add(-work[i1 * Rn + q], b1);
              l0 = fma(ulo_s[i0 * Rn + q], b0, l0);
              l1 = fma(ulo_s[i1 * Rn + q], b1, l1);
            }
            nb[e0] = d0.value() - l0;
            if (e0 + NTP < nE) nb[e1] = d1.value() - l1;
          }
          __syncthreads();
          gram_sym<T>(nb, rows, R, R, egram + n * R * R, tid, NTP);
        }
      }
      __syncthreads();
      if (n == N - 1) {
        if (sizeof(T) == 8) {
          // FP64 form: <G, [[lambda; B]]> from H (Gram identity, as the FP64 oracle)
          double s2 = 0.0;
          for (int e = tid; e < Rn * R; e += NTP)
            s2 += (double)__ldcg(a.H + e) * lam[e % R] * (double)Bs[boff[n] + e];
          inner = block_sum_d(s2, red);
        } else {
          // FP32 forms: ||G - [[lambda; B]]||^2 summed explicitly over this CTA's
          // share of the core (the Gram identity cancels to rounding noise near
          // convergence in FP32)
          FFAcc racc;
          if (N == 3) {
            // slab i of mode 1: P[j, r] = lambda_r B_1[i, r] B_2[j, r], then the
            // model slab P B_3^T in 4 x 4 register tiles against G[i, :, :],
            // P and the sums in float-float
            const int R1 = a.Rt[1], R2 = a.Rt[2];
            const T* B0 = Bs + boff[0];
            const T* B1 = Bs + boff[1];
            const T* B2 = Bs + boff[2];
            const int tj = (R1 + 3) / 4, tk = (R2 + 3) / 4;
            for (int i = c; i < a.Rt[0]; i += G) {
              for (int tile = tid; tile < tj * tk; tile += NTP) {
                const int j0 = (tile / tk) * 4, k0 = (tile % tk) * 4;
                FFAcc acc[4][4];
                for (int r = 0; r < R; ++r) {
                  float lh, ll;  // lambda_r B_1[i, r]
                  ff_mul((float)lamT[r], 0.f, (float)B0[i * R + r], lh, ll);
                  float ph[4], pl[4], b4[4];
#pragma unroll
                  for (int u = 0; u < 4; ++u) ff_mul(lh, ll, (j0 + u < R1) ? (float)B1[(j0 + u) * R + r] : 0.f, ph[u], pl[u]);
#pragma unroll
                  for (int v = 0; v < 4; ++v) b4[v] = (k0 + v < R2) ? (float)B2[(k0 + v) * R + r] : 0.f;
#pragma unroll
                  for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v].fma2(ph[u], pl[u], b4[v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                  for (int v = 0; v < 4; ++v)
                    if (j0 + u < R1 && k0 + v < R2)
                      ff_add_sq_diff(racc,
                                     (float)a.G[(int64_t)i * a.stride[0] + (int64_t)(j0 + u) * a.stride[1] + k0 + v],
                                     acc[u][v].s, acc[u][v].c);
              }
            }
          } else {
          const int64_t chunk = (a.gnumel + G - 1) / G;
          const int64_t e0 = (int64_t)c * chunk, e1 = e0 + chunk < a.gnumel ? e0 + chunk : a.gnumel;
          for (int64_t e = e0 + tid; e < e1; e += NTP) {
            int rem = (int)e;
            int ix[TDK_MAX_MODES];
            for (int p = N - 1; p >= 0; --p) {
              ix[p] = rem % a.Rt[p];
              rem /= a.Rt[p];
            }
            FFAcc x;
            for (int r = 0; r < R; ++r) {
              float vh = (float)lamT[r], vl = 0.f;
              for (int p = 0; p < N; ++p) ff_mul(vh, vl, (float)Bs[boff[p] + ix[p] * R + r], vh, vl);
              x.add(vh, vl);
            }
            ff_add_sq_diff(racc, (float)a.G[e], x.s, x.c);
          }
          }
          double s2 = block_sum_ff(racc, red);
          if (tid == 0) a.rpart[c] = s2;
        }
      }
      PROF_MARK(4);
      // H / Bnew are overwritten by the next mode only after every CTA read them
      if (!grid_sync(a.bar, a.status)) { ok = false; break; }
      PROF_MARK(5);
    }
    if (!ok) break;
    // ---- fit (identical in every CTA)
    // ||[[lambda; A]]||^2 from the Grams, in FP64; FP32 nonneg: the term
    // ||[[lambda; A]]||^2 - ||[[lambda; U B]]||^2 = sum lambda lambda (prod (BtB + E)
    // - prod BtB), the products in FP64 from the FP32 Grams
    // (an FP32 unconstrained core needs neither: its fit is the explicit
    // residual; FP64 arithmetic runs at a small fraction of the FP32 rate)
    double m2 = 0.0, lk = 0.0;
    for (int e = tid; e < ((sizeof(T) == 8 || leak32) ? R * R : 0); e += NTP) {
      double v = (double)lamT[e / R] * (double)lamT[e % R];
      double va = v, vb = v;
      for (int p = 0; p < N; ++p) {
        v *= (double)gram[p * R * R + e];
        if (leak32) {
          va *= (double)bgram[p * R * R + e] + (double)egram[p * R * R + e];
          vb *= (double)bgram[p * R * R + e];
        }
      }
      m2 += v;
      lk += va - vb;
    }
    const double model2 = sizeof(T) == 8 ? block_sum_d(m2, red) : 0.0;
    // [[A]] leaves the Tucker subspace (nonneg): add ||[[A]]||^2 - ||P [[A]]||^2,
    // P [[A]] = [[U B]] with B_p = U_p^T A_p
    const double leak = leak32 ? block_sum_d(lk, red) : 0.0;
    // FP32 cores: the CTAs' residual partials, summed in a fixed order by
    // the first warp
    double rsum = 0.0;
    if (sizeof(T) == 4) {
      if (tid < 32) {
        double v = 0.0;
        for (int q = tid; q < G; q += 32) v += __ldcg(a.rpart + q);
        v = warp_sum(v);
        if (tid == 0) red[0] = v;
      }
      __syncthreads();
      rsum = red[0];
      __syncthreads();
    }
    PROF_MARK(6);
    // the scalar tail by one thread, shared through `red` (same value in every CTA)
    if (tid == 0) {
      double res2;
      if (sizeof(T) == 8) {
        res2 = fmax(0.0, nG2 - 2.0 * inner + model2);
      } else {
        res2 = rsum;
        if (a.nonneg) res2 += fmax(0.0, leak);
      }
      const double f = 1.0 - sqrt(res2) / sqrt(nG2);
      red[0] = f;
      red[1] = a.nY2 ? 1.0 - sqrt(fmax(0.0, nY2 - nG2 + res2)) / sqrt(nY2) : fitY;
      red[2] = (sweep > 1 && fabs(f - fit) < a.tol * fabs(fit)) ? 1.0 : 0.0;
      if (c == 0 && sweep - 1 < a.hist_cap) a.hist[sweep - 1] = f;
    }
    __syncthreads();
    PROF_MARK(19);
    fit = red[0];
    fitY = red[1];
    const bool conv = red[2] != 0.0;
    __syncthreads();
    PROF_MARK(20);
    if (conv) {
      converged = 1;
      break;
    }
  }
  if (a.prof && blockIdx.x == 0) {
    __syncthreads();
    if (threadIdx.x < 32) a.prof[threadIdx.x] = s_pf[threadIdx.x];
  }
  if (sweep > a.max_sweeps) sweep = a.max_sweeps;
  if (c == 0) {
    for (int n = 0; n < N; ++n)
      for (int e = tid; e < a.Rt[n] * R; e += NTP) a.Bout[n][e] = Bs[boff[n] + e];
    for (int r = tid; r < R; r += NTP) a.lam_out[r] = lam[r];
    if (tid == 0) {
      a.st->sweeps = sweep;
      a.st->converged = converged;
      a.st->status = needpinv ? ST_NEEDPINV : (ok ? 0 : ST_TIMEOUT);
      a.st->fit = fit;
      a.st->fitY = fitY;
    }
  }
}

// ---------------------------------------------------------------------------
// Whole FFCP on one CTA for 3-way cores that fit in shared memory (the core,
// the factors and one intermediate of Rt_1 Rt_2 x R stay resident).  Same
// steps and stopping rule as the grid-wide kernel, without grid barriers:
//   mode 1: W[(i1,i2), r] = sum_i3 G[i1,i2,i3] B_3[i3, r], H_1 = sum_i2 W B_2;
//   mode 2: H_2 = sum_i1 W B_1 (W unchanged: B_3 has not moved);
//   mode 3: V[(i1,i3), r] = sum_i2 G[i1,i2,i3] B_2[i2, r], H_3 = sum_i1 V B_1;
// T_n is inverted by warps 0-7 (Gauss-Jordan) while warps 8-15 form H_n; the
// solve B_n = H_n T_n^-1 is one product plus two FP64 refinement steps.
constexpr int NTS = 512;

template <class T>
struct SLayout {
  size_t o_g, o_b0, o_b1, o_b2, o_gram, o_w, o_h, o_x, o_res, o_tm, o_ld, o_lid, o_lf, o_lif, o_lam, o_lamt, o_red,
      o_xp, o_ns, o_resf, total;
  __host__ __device__ void plan(int R0, int R1, int R2, int R) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
      const size_t o = (off + 15) & ~size_t(15);
      off = o + bytes;
      return o;
    };
    const int Rtm = R0 > R1 ? (R0 > R2 ? R0 : R2) : (R1 > R2 ? R1 : R2);
    const size_t RR = (size_t)R * R;
    o_g = take(sizeof(T) * (size_t)R0 * R1 * R2);
    o_b0 = take(sizeof(T) * (size_t)R0 * R);
    o_b1 = take(sizeof(T) * (size_t)R1 * R);
    o_b2 = take(sizeof(T) * (size_t)R2 * R);
    o_gram = take(sizeof(T) * 3 * RR);
    o_w = take(sizeof(T) * (size_t)R0 * (R1 > R2 ? R1 : R2) * R);
    o_h = take(sizeof(T) * (size_t)Rtm * R);
    o_x = take(sizeof(double) * (size_t)Rtm * R);
    o_res = take(sizeof(double) * (size_t)Rtm * R);
    o_tm = take(sizeof(double) * RR);
    o_ld = take(sizeof(double) * RR);
    o_lid = take(sizeof(double) * (RR > 128 ? RR : 128));
    o_lf = take(sizeof(float) * RR);
    o_lif = take(sizeof(float) * (RR > 128 ? RR : 128));
    o_lam = take(sizeof(double) * 64);
    o_lamt = take(sizeof(T) * 64);
    o_red = take(sizeof(double) * 32);
    o_xp = take(sizeof(float) * 3 * RR);  // last FP32 inverse of each T_n
    o_ns = take(sizeof(float) * RR);      // Newton-Schulz iterate
    o_resf = take(sizeof(float) * (size_t)(Rtm + 1) * R);  // FP32 residual / solution, reciprocal norms
    total = (off + 15) & ~size_t(15);
  }
};

template <class T>
__global__ void __launch_bounds__(NTS, 1) als_small_kernel(PArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int R = a.R, RR = R * R;
  const int Rt[3] = {a.Rt[0], a.Rt[1], a.Rt[2]};
  const int M01 = Rt[0] * Rt[1];
  const int nel = M01 * Rt[2];
  const int Rtm = Rt[0] > Rt[1] ? (Rt[0] > Rt[2] ? Rt[0] : Rt[2]) : (Rt[1] > Rt[2] ? Rt[1] : Rt[2]);
  SLayout<T> L;
  L.plan(Rt[0], Rt[1], Rt[2], R);
  T* Gc = reinterpret_cast<T*>(sm + L.o_g);
  T* B[3] = {reinterpret_cast<T*>(sm + L.o_b0), reinterpret_cast<T*>(sm + L.o_b1), reinterpret_cast<T*>(sm + L.o_b2)};
  T* gram = reinterpret_cast<T*>(sm + L.o_gram);
  T* W = reinterpret_cast<T*>(sm + L.o_w);
  T* H = reinterpret_cast<T*>(sm + L.o_h);
  double* X = reinterpret_cast<double*>(sm + L.o_x);
  double* Res = reinterpret_cast<double*>(sm + L.o_res);
  double* Tm = reinterpret_cast<double*>(sm + L.o_tm);
  double* Ld = reinterpret_cast<double*>(sm + L.o_ld);
  double* Lid = reinterpret_cast<double*>(sm + L.o_lid);
  float* Lf = reinterpret_cast<float*>(sm + L.o_lf);
  float* Lif = reinterpret_cast<float*>(sm + L.o_lif);
  float* Xp = reinterpret_cast<float*>(sm + L.o_xp);
  float* Xns = reinterpret_cast<float*>(sm + L.o_ns);
  float* Resf = reinterpret_cast<float*>(sm + L.o_resf);
  double* lam = reinterpret_cast<double*>(sm + L.o_lam);
  T* lamT = reinterpret_cast<T*>(sm + L.o_lamt);
  double* red = reinterpret_cast<double*>(sm + L.o_red);
  __shared__ int s_mode;  // 1: FP32 factor, 2: FP64 factor, 0: singular
  __shared__ int s_nref;  // refinement steps of the solve
  __shared__ T s_irows[3];  // 1 / sqrt(Rt_n): the column a zero column is replaced by
  __shared__ unsigned long long s_prof[10];
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr bool F64 = sizeof(T) == 8;
  // optional cycle accounting per phase (block-wide phases; thread 0 records)
  const bool prof_on = a.prof != nullptr;
  unsigned long long prof_t = clock64();
  if (tid < 10) s_prof[tid] = 0;
  auto pms = [&](int k) {
    if (prof_on) {
      __syncthreads();
      if (tid == 0) {
        const unsigned long long t = clock64();
        s_prof[k] += t - prof_t;
        prof_t = t;
      }
    }
  };

  if (tid < 3) s_irows[tid] = (T)(1.0 / sqrt((double)Rt[tid]));
  for (int e = tid; e < nel; e += NTS) Gc[e] = a.G[e];
  for (int n = 0; n < 3; ++n)
    for (int e = tid; e < Rt[n] * R; e += NTS) B[n][e] = (T)a.init[n][e];
  for (int r = tid; r < R; r += NTS) {
    lam[r] = 1.0;
    lamT[r] = T(1);
  }
  __syncthreads();
  for (int n = 0; n < 3; ++n)
    for (int e = tid; e < RR; e += NTS) {
      const int r = e / R, c = e % R;
      T acc = T(0);
      for (int q = 0; q < Rt[n]; ++q) acc = fma(B[n][q * R + r], B[n][q * R + c], acc);
      gram[n * RR + e] = acc;
    }
  __syncthreads();
  const double nG2 = *a.nG2;
  const double nY2 = a.nY2 ? *a.nY2 : 0.0;
  double fit = 0.0, fitY = nan("");
  int sweep = 0, converged = 0, singular = 0;
  unsigned have_prev = 0;  // warps 0-7: modes whose last FP32 inverse is in Xp
  for (sweep = 1; sweep <= a.max_sweeps; ++sweep) {
    for (int n = 0; n < 3; ++n) {
      const int Rn = Rt[n];
      pms(7);
      // ---- T_n (FP64 and FP32 copies)
      for (int e = tid; e < RR; e += NTS) {
        const int p0 = n == 0 ? 1 : 0, p1 = n == 2 ? 1 : 2;
        if (F64) {
          const double v = (double)gram[p0 * RR + e] * (double)gram[p1 * RR + e];
          Tm[e] = v;
          Ld[e] = v;
          Lf[e] = (float)v;
        } else {
          // the exact product of two FP32 entries as hi + lo, joined in FP64
          const float ga = (float)gram[p0 * RR + e], gb = (float)gram[p1 * RR + e];
          const float ph = ga * gb;
          Tm[e] = f2d_int(ph) + f2d_int(fmaf(ga, gb, -ph));
          Lf[e] = ph;
        }
      }
      __syncthreads();
      pms(0);
      if (warp < 8) {
        // ---- invert T_n, warps 0-7: FP32 cores by Newton-Schulz steps from the
        //      previous sweep's inverse (accepted at f <= 2^-9, one refinement
        //      step of the solve when f <= 2^-13, as in the grid kernel), else
        //      by FP32 Gauss-Jordan; FP64 cores and the fallback by FP64
        //      Gauss-Jordan
        const unsigned long long pt0 = clock64();
        int mode = 0, nref = 2;
        if (!F64) {
          const float* Xi = nullptr;
          if (have_prev & (1u << n)) {
            float* X0 = reinterpret_cast<float*>(Ld);
            for (int e = tid; e < RR; e += 256) X0[e] = Xp[n * RR + e];
            float dev = 1.f;
            int nit = 0;
            Xi = ns_inverse(Lf, X0, Xns, X0 + RR, Lif, R, 0x1p-9f, NS_MAX_IT, a.ns_gate, &dev, &nit, tid, 256, 2);
            if (Xi) {
              for (int e = tid; e < RR; e += 256) Lf[e] = Xi[e];
              mode = 1;
              nref = dev <= 0x1p-13f ? 1 : 2;
            }
          }
          if (!Xi && group_gj_inverse_smem<float>(Lf, Lif, R, 1.1920929e-7f, tid, 256, 2)) mode = 1;
          if (mode == 1) {
            for (int e = tid; e < RR; e += 256) Xp[n * RR + e] = Lf[e];
            have_prev |= 1u << n;
          } else {
            have_prev &= ~(1u << n);
            for (int e = tid; e < RR; e += 256) Ld[e] = Tm[e];
            tc::named_bar(2, 256);
          }
        }
        if (mode == 0 && group_gj_inverse_smem<double>(Ld, Lid, R, 2.220446049250313e-16, tid, 256, 2)) mode = 2;
        if (tid == 0) {
          s_mode = mode;
          s_nref = nref;
          if (prof_on) s_prof[8] += clock64() - pt0;
        }
      } else {
        // ---- H_n, warps 8-15
        const unsigned long long pt1 = clock64();
        const int t = tid - 256, nt = NTS - 256;
        if (n == 0) {
          // W = G_(12) B_3 in 4 x 4 register tiles
          const int tm = (M01 + 3) / 4, tr = (R + 3) / 4;
          for (int tile = t; tile < tm * tr; tile += nt) {
            const int m0 = (tile / tr) * 4, r0 = (tile % tr) * 4;
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
            for (int k = 0; k < Rt[2]; ++k) {
              T g4[4], b4[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) g4[u] = (m0 + u < M01) ? Gc[(m0 + u) * Rt[2] + k] : T(0);
#pragma unroll
              for (int v = 0; v < 4; ++v) b4[v] = (r0 + v < R) ? B[2][k * R + r0 + v] : T(0);
#pragma unroll
              for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(g4[u], b4[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v)
                if (m0 + u < M01 && r0 + v < R) W[(m0 + u) * R + r0 + v] = acc[u][v];
          }
          tc::named_bar(1, nt);
          for (int e = t; e < Rt[0] * R; e += nt) {
            const int i = e / R, r = e % R;
            T acc = T(0);
            for (int j = 0; j < Rt[1]; ++j) acc = fma(W[(i * Rt[1] + j) * R + r], B[1][j * R + r], acc);
            H[e] = acc;
          }
        } else if (n == 1) {
          for (int e = t; e < Rt[1] * R; e += nt) {
            const int j = e / R, r = e % R;
            T acc = T(0);
            for (int i = 0; i < Rt[0]; ++i) acc = fma(W[(i * Rt[1] + j) * R + r], B[0][i * R + r], acc);
            H[e] = acc;
          }
        } else {
          // V[(i1, i3), r] = sum_i2 G[i1, i2, i3] B_2[i2, r] in 4 x 4 tiles (4
          // consecutive i3 of one i1), then H_3 = sum_i1 V B_1
          const int tq = (Rt[2] + 3) / 4, tm = Rt[0] * tq, tr = (R + 3) / 4;
          for (int tile = t; tile < tm * tr; tile += nt) {
            const int mt = tile / tr, r0 = (tile % tr) * 4;
            const int i0 = mt / tq, k0 = (mt % tq) * 4;
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
            for (int j = 0; j < Rt[1]; ++j) {
              T g4[4], b4[4];
              const T* gr = Gc + (i0 * Rt[1] + j) * Rt[2] + k0;
#pragma unroll
              for (int u = 0; u < 4; ++u) g4[u] = (k0 + u < Rt[2]) ? gr[u] : T(0);
#pragma unroll
              for (int v = 0; v < 4; ++v) b4[v] = (r0 + v < R) ? B[1][j * R + r0 + v] : T(0);
#pragma unroll
              for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(g4[u], b4[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v)
                if (k0 + u < Rt[2] && r0 + v < R) W[(i0 * Rt[2] + k0 + u) * R + r0 + v] = acc[u][v];
          }
          tc::named_bar(1, nt);
          for (int e = t; e < Rt[2] * R; e += nt) {
            const int k = e / R, r = e % R;
            T acc = T(0);
            for (int i = 0; i < Rt[0]; ++i) acc = fma(W[(i * Rt[2] + k) * R + r], B[0][i * R + r], acc);
            H[e] = acc;
          }
        }
        if (prof_on && tid == 256) s_prof[9] += clock64() - pt1;
      }
      __syncthreads();
      pms(1);
      if (s_mode == 0) {
        singular = 1;
        break;
      }
      // ---- B_n = H_n T_n^-1, refined against T_n in FP64 (s_nref steps)
      const bool f32 = s_mode == 1;
      const int nref = s_nref;
      for (int e = tid; e < Rn * R; e += NTS) {
        const int i = e / R, c = e % R;
        double acc = 0.0;
        if (f32) {
          float af = 0.f;
          for (int r = 0; r < R; ++r) af = fmaf((float)H[i * R + r], Lf[r * R + c], af);
          acc = af;
        } else {
          for (int r = 0; r < R; ++r) acc = fma((double)H[i * R + r], Ld[r * R + c], acc);
        }
        X[e] = acc;
      }
      __syncthreads();
      pms(2);
      for (int it = 0; it < nref; ++it) {
        for (int e = tid; e < Rn * R; e += NTS) {
          const int i = e / R, c = e % R;
          double rr = (double)H[e];
          for (int r = 0; r < R; ++r) rr = fma(-X[i * R + r], Tm[r * R + c], rr);
          Res[e] = rr;
          Resf[e] = (float)rr;  // one conversion per entry, not per term
        }
        __syncthreads();
        for (int e = tid; e < Rn * R; e += NTS) {
          const int i = e / R, c = e % R;
          double acc = 0.0;
          if (f32) {
            float af = 0.f;
            for (int r = 0; r < R; ++r) af = fmaf(Resf[i * R + r], Lf[r * R + c], af);
            acc = af;
          } else {
            for (int r = 0; r < R; ++r) acc = fma(Res[i * R + r], Ld[r * R + c], acc);
          }
          X[e] += acc;
        }
        __syncthreads();
      }
      pms(3);
      // ---- lambda (column norms), normalised B_n and its Gram (FP32 cores:
      //      in FP32 from the solution rounded once, as B_n is stored)
      if (F64) {
        for (int r = warp; r < R; r += NTS / 32) {
          double s2 = 0.0;
          for (int i = tid & 31; i < Rn; i += 32) s2 = fma(X[i * R + r], X[i * R + r], s2);
          s2 = warp_sum(s2);
          if ((tid & 31) == 0) {
            lam[r] = sqrt(s2);
            lamT[r] = (T)lam[r];
            Res[r] = lam[r] > 0.0 ? 1.0 / lam[r] : 0.0;  // reciprocal (Res is free here)
          }
        }
      } else {
        for (int e = tid; e < Rn * R; e += NTS) Resf[e] = (float)X[e];
        __syncthreads();
        for (int r = warp; r < R; r += NTS / 32) {
          float s2 = 0.f;
          for (int i = tid & 31; i < Rn; i += 32) s2 = fmaf(Resf[i * R + r], Resf[i * R + r], s2);
          s2 = warp_sum(s2);
          if ((tid & 31) == 0) {
            const float l = sqrtf(s2);
            lam[r] = f2d_int(l);
            lamT[r] = (T)l;
            Resf[Rtm * R + r] = l > 0.f ? 1.f / l : 0.f;
          }
        }
      }
      __syncthreads();
      const T inv_rows = s_irows[n];
      for (int e = tid; e < Rn * R; e += NTS) {
        const int r = e % R;
        if (F64)
          B[n][e] = lam[r] > 0.0 ? (T)(X[e] * Res[r]) : inv_rows;
        else
          B[n][e] = lamT[r] > T(0) ? (T)(Resf[e] * Resf[Rtm * R + r]) : inv_rows;
      }
      __syncthreads();
      for (int e = tid; e < RR; e += NTS) {
        const int r = e / R, c = e % R;
        T acc = T(0);
        for (int q = 0; q < Rn; ++q) acc = fma(B[n][q * R + r], B[n][q * R + c], acc);
        gram[n * RR + e] = acc;
      }
      __syncthreads();
      pms(4);
    }
    if (singular) break;
    // ---- fit (||[[lambda; B]]||^2 for FP64 cores only: FP32 cores take the
    //      explicit residual)
    double m2 = 0.0;
    for (int e = tid; e < (F64 ? RR : 0); e += NTS) {
      double v = lam[e / R] * lam[e % R];
      for (int p = 0; p < 3; ++p) v *= (double)gram[p * RR + e];
      m2 += v;
    }
    const double model2 = F64 ? block_sum_d(m2, red) : 0.0;
    double res2;
    if (F64) {
      // <G, [[lambda; B]]> from H_3 (Gram identity, as the FP64 oracle)
      double in = 0.0;
      for (int e = tid; e < Rt[2] * R; e += NTS) in += (double)H[e] * lam[e % R] * (double)B[2][e];
      const double inner = block_sum_d(in, red);
      res2 = fmax(0.0, nG2 - 2.0 * inner + model2);
    } else {
      // explicit ||G - [[lambda; B]]||^2: model (B_1 (.) B_2) diag(lambda) B_3^T,
      // tile by tile, in float-float
      FFAcc racc;
      const int tm = (M01 + 3) / 4, tk = (Rt[2] + 3) / 4;
      for (int tile = tid; tile < tm * tk; tile += NTS) {
        const int m0 = (tile / tk) * 4, k0 = (tile % tk) * 4;
        FFAcc acc[4][4];
        int ia[4], ib[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int m = m0 + u < M01 ? m0 + u : 0;
          ia[u] = (m / Rt[1]) * R;
          ib[u] = (m % Rt[1]) * R;
        }
        for (int r = 0; r < R; ++r) {
          float wh[4], wl[4], b4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float h, l;  // B_1[i, r] B_2[j, r] lambda_r
            ff_mul((float)B[0][ia[u] + r], 0.f, (float)B[1][ib[u] + r], h, l);
            ff_mul(h, l, (m0 + u < M01) ? (float)lamT[r] : 0.f, wh[u], wl[u]);
          }
#pragma unroll
          for (int v = 0; v < 4; ++v) b4[v] = (k0 + v < Rt[2]) ? (float)B[2][(k0 + v) * R + r] : 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v].fma2(wh[u], wl[u], b4[v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (m0 + u < M01 && k0 + v < Rt[2])
              ff_add_sq_diff(racc, (float)Gc[(m0 + u) * Rt[2] + k0 + v], acc[u][v].s, acc[u][v].c);
      }
      res2 = block_sum_ff(racc, red);
    }
    pms(5);
    // the scalar tail by one thread, shared through `red`
    if (tid == 0) {
      const double f = 1.0 - sqrt(res2) / sqrt(nG2);
      red[0] = f;
      red[1] = a.nY2 ? 1.0 - sqrt(fmax(0.0, nY2 - nG2 + res2)) / sqrt(nY2) : fitY;
      red[2] = (sweep > 1 && fabs(f - fit) < a.tol * fabs(fit)) ? 1.0 : 0.0;
      if (sweep - 1 < a.hist_cap) a.hist[sweep - 1] = f;
    }
    __syncthreads();
    fit = red[0];
    fitY = red[1];
    const bool conv = red[2] != 0.0;
    __syncthreads();
    if (conv) {
      converged = 1;
      break;
    }
    pms(6);
  }
  if (prof_on && tid < 10) a.prof[tid] = s_prof[tid];
  if (sweep > a.max_sweeps) sweep = a.max_sweeps;
  for (int n = 0; n < 3; ++n)
    for (int e = tid; e < Rt[n] * R; e += NTS) a.Bout[n][e] = B[n][e];
  for (int r = tid; r < R; r += NTS) a.lam_out[r] = lam[r];
  if (tid == 0) {
    a.st->sweeps = sweep;
    a.st->converged = converged;
    a.st->status = singular ? ST_NEEDPINV : 0;
    a.st->fit = fit;
    a.st->fitY = fitY;
  }
}

// ||G||^2 in two launches: each block sums a grid-stride share (FP64 cores in
// FP64; FP32 cores in float-float, each square split exactly into hi + lo by
// an FMA, FP64 arithmetic being scarce on this GPU) into parts[block], then
// one block adds the parts in order.  (A Kahan sum that feeds its correction
// back into the next addend loses up to half an FP32 unit of every square:
// 7.8e-10 of ||G||^2 on a 20^3 core.)
template <class T>
__global__ void norm2_core(const T* __restrict__ G, int64_t n, double* __restrict__ parts) {
  __shared__ double red[32];
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  double v;
  if (sizeof(T) == 8) {
    double s = 0.0;
    for (int64_t e = t0; e < n; e += st) {
      const double x = (double)G[e];
      s = fma(x, x, s);
    }
    v = block_sum_d(s, red);
  } else {
    FFAcc acc;
    for (int64_t e = t0; e < n; e += st) {
      const float x = (float)G[e];
      const float sq = x * x;
      acc.add(sq, fmaf(x, x, -sq));
    }
    v = block_sum_ff(acc, red);
  }
  if (threadIdx.x == 0) parts[blockIdx.x] = v;
}
__global__ void norm2_finish(const double* __restrict__ parts, int n, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += parts[i];
    *out = s;
  }
}

template <class T>
__global__ void u_to_t(const double* __restrict__ s, T* __restrict__ d, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (T)s[e];
}
// the FP32 remainder U - (float)U
__global__ void u_lo_f32(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (float)(s[e] - (double)(float)s[e]);
}

}  // namespace

// TDK_ENOTSUP: the core does not fit the persistent form (the caller falls back)
template <class T>
int als_persistent_t(tdk_ctx* ctx, const Geom& g, const T* G, const double* const U[], const double* normY2,
                     const tdk_als_opts* o, double* const B_io[], double* const A_io[], double* lambda_out,
                     tdk_als_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  const int N = g.N, R = o->R;
  if (o->init != TDK_INIT_GIVEN || o->timeout_s > 0) return TDK_ENOTSUP;
  // the row slices of H_n are indexed by the other modes but the last one:
  // with two modes there are none, and the multi-kernel form takes over
  if (N < 3) return TDK_ENOTSUP;
  if (g.core_numel >= ((int64_t)1 << 31)) return TDK_ENOTSUP;  // the kernel indexes the core in 32 bits
  PArgs<T> a{};
  a.N = N;
  a.R = R;
  a.ns_gate = 1.f;
#ifdef TDK_TESTING
  if (const char* e = getenv("TDK_ALS_NS_GATE")) a.ns_gate = (float)atof(e);
#endif
  // the l1 form updates the factors as A_n like the nonnegative forms
  a.nonneg = (o->nonneg || o->l1 > 0.0) ? 1 : 0;
  a.nn_rule = o->nonneg == TDK_NONNEG_HALS ? 1 : (o->nonneg == TDK_NONNEG_MU ? 2 : 0);
  a.clip = o->nonneg ? 1 : 0;
  a.l1 = o->l1;
  a.max_sweeps = o->max_sweeps;
  a.tol = o->tol;
  int64_t Rtmax = 0, Imax = 0, btot = 0;
  {
    int64_t s = 1;
    for (int n = N - 1; n >= 0; --n) {
      a.stride[n] = s;
      s *= g.Rt[n];
    }
  }
  a.gnumel = g.core_numel;
  for (int n = 0; n < N; ++n) {
    a.Rt[n] = g.Rt[n];
    a.I[n] = g.I[n];
    Rtmax = std::max<int64_t>(Rtmax, g.Rt[n]);
    Imax = std::max<int64_t>(Imax, g.I[n]);
    btot += (int64_t)g.Rt[n] * R;
    const int64_t Q = g.core_numel / g.Rt[n];
    a.Qmax = std::max<int64_t>(a.Qmax, Q);
    const int last = (n == N - 1) ? N - 2 : N - 1;
    a.Amax = std::max<int64_t>(a.Amax, Q / g.Rt[last]);
  }
  // the slice buffer also holds the normalised rows of the update
  a.Qmax = std::max<int64_t>(a.Qmax, (a.nonneg ? Imax : Rtmax) * R);
  // and the work buffer the staged H and U_n (nonneg)
  a.Amax = std::max<int64_t>(a.Amax, Rtmax);
  if (a.nonneg)
    for (int n = 0; n < N; ++n) a.Amax = std::max<int64_t>(a.Amax, (g.I[n] * g.Rt[n] + R - 1) / R);
  if (sizeof(T) == 4 && a.nonneg)
    for (int n = 0; n < N; ++n) a.ulo_elems = std::max<int64_t>(a.ulo_elems, g.I[n] * g.Rt[n]);
  // Buffer sizes for a grid: Qmax and Amax above hold whole rows of H_n;
  // with the rows split over Pn CTAs a CTA stages and contracts only its
  // part, so the slice and work buffers are sized for the largest part.
  const int64_t Qwhole = a.Qmax, Awhole = a.Amax;
  int64_t q_rows = 0;
  auto size_for = [&](int grid_) {
    q_rows = (a.nonneg ? Imax : Rtmax) * R;
    int64_t q_slice = 0, a_rows = Rtmax;
    if (a.nonneg)
      for (int n = 0; n < N; ++n) a_rows = std::max<int64_t>(a_rows, (g.I[n] * g.Rt[n] + R - 1) / R);
    for (int n = 0; n < N; ++n) {
      int oth[TDK_MAX_MODES], no = 0;
      for (int p = 0; p < N; ++p)
        if (p != n) oth[no++] = p;
      const int Rn = g.Rt[n], Rl = g.Rt[oth[no - 1]], R0o = g.Rt[oth[0]];
      const int64_t per0 = g.core_numel / Rn / Rl / R0o;
      const int Pn = std::max(1, std::min(grid_ / Rn, R0o));
      const int64_t part = (R0o + Pn - 1) / Pn, rows0 = part * per0;
      q_slice = std::max(q_slice, rows0 * Rl);
      a_rows = std::max(a_rows, rows0);  // first product, in the work buffer
      int64_t rows = rows0;
      bool to_slice = true;  // the products alternate between the slice and work buffers
      for (int k = no - 2; k >= 0; --k) {
        rows /= (k == 0) ? part : g.Rt[oth[k]];
        if (to_slice) q_rows = std::max(q_rows, rows * R);
        else a_rows = std::max(a_rows, rows);
        to_slice = !to_slice;
      }
    }
    a.Amax = std::min(Awhole, a_rows);
    a.Qmax = std::min(Qwhole, std::max(q_rows, q_slice));
    PLayout<T> l;
    l.plan(N, R, (int)btot, a.Qmax, a.Amax, sizeof(T) == 4 && a.nonneg, 0, a.ulo_elems);
    return l.total + 64;
  };
  // rows of H_n are split over several CTAs (by ranges of the slowest other
  // mode) when the whole GPU gives at least four per row; otherwise one CTA per
  // row keeps the grid barriers cheap.  The sizes at one CTA per SM bound the
  // shared memory; the occupancy they allow sets the grid, whose parts are no
  // larger.
  const int64_t rows_cap = a.nonneg ? std::max(Rtmax, Imax) : Rtmax;
  auto grid_of = [&](int per_sm_) {
    const int all = per_sm_ * ctx->num_sms;
    return (all >= 4 * Rtmax) ? all : (int)std::min<int64_t>(all, rows_cap);
  };
  size_t smem = size_for(grid_of(1));
  if (smem > (size_t)ctx->max_smem_optin) return TDK_ENOTSUP;
  auto kern = als_persistent_kernel<T>;
  TDK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TDK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTP, smem));
  if (per_sm < 1) return TDK_ENOTSUP;
  int grid = grid_of(per_sm);
#ifdef TDK_TESTING
  // test hook: TDK_ALS_GRID=1 takes the grid kernel on a core the one-CTA
  // kernel would take; a larger value also caps the grid (another split of
  // the rows over the CTAs, so other orders of the sums)
  const int grid_cap = getenv("TDK_ALS_GRID") ? atoi(getenv("TDK_ALS_GRID")) : 0;
  if (grid_cap > 1) grid = std::min(grid, grid_cap);
#endif
  smem = size_for(grid);
  if (smem > (size_t)ctx->max_smem_optin) return TDK_ENOTSUP;  // (a capped test grid)
  TDK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // Core slices kept in shared memory across sweeps, when every CTA has at
  // most one part of H_n per mode (the same part every sweep, as the kernel
  // splits the rows) and the slices fit beside the rest without lowering
  // the CTAs per SM.
  {
    int64_t cache = 0;
    bool one_part = true;
    for (int n = 0; n < N; ++n) {
      int oth[TDK_MAX_MODES], no = 0;
      for (int p = 0; p < N; ++p)
        if (p != n) oth[no++] = p;
      const int Rn = g.Rt[n], Rl = g.Rt[oth[no - 1]], R0o = g.Rt[oth[0]];
      const int64_t per0 = g.core_numel / Rn / Rl / R0o;
      const int Pn = std::max(1, std::min(grid / Rn, R0o));
      if ((int64_t)Rn * Pn > grid) one_part = false;
      a.coff[n] = cache;
      cache += ((int64_t)(R0o + Pn - 1) / Pn * per0 * Rl + 3) / 4 * 4;
    }
    if (one_part && cache > 0) {
      // the slice buffer then holds only the products and the update rows
      const int64_t qc = std::min(a.Qmax, q_rows);
      PLayout<T> lc;
      lc.plan(N, R, (int)btot, qc, a.Amax, sizeof(T) == 4 && a.nonneg, cache, a.ulo_elems);
      int per_sm_c = 0;
      if (lc.total + 64 <= (size_t)ctx->max_smem_optin &&
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(lc.total + 64)) ==
              cudaSuccess &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, kern, NTP, lc.total + 64) == cudaSuccess &&
          per_sm_c >= per_sm) {
        a.cache_elems = cache;
        a.Qmax = qc;
        smem = lc.total + 64;
      } else {
        cudaGetLastError();
        TDK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      }
    }
  }

  Planner pl;
  pl.take<T>((size_t)(a.nonneg ? std::max(Rtmax, Imax) : Rtmax) * R);
  pl.take<T>((size_t)Rtmax * R);
  pl.take<T>((size_t)grid * R);
  for (int n = 0; n < N; ++n) pl.take<T>((size_t)g.Rt[n] * R);
  for (int n = 0; n < N; ++n) pl.take<T>((size_t)g.I[n] * g.Rt[n]);
  const bool leak32 = sizeof(T) == 4 && a.nonneg;
  if (leak32)
    for (int n = 0; n < N; ++n) pl.take<T>((size_t)g.I[n] * g.Rt[n]);
  if (a.nonneg)
    for (int n = 0; n < N; ++n) pl.take<double>((size_t)g.I[n] * R);
  pl.take<double>(R);
  pl.take<double>(std::min(o->max_sweeps, 65536));
  pl.take<PState>(1);
  pl.take<unsigned>(2);
  pl.take<double>(1);
  pl.take<double>(NORM_BLOCKS);
  pl.take<double>(grid);
  pl.take<float>((size_t)grid * N * R * R);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  a.Bnew = cv.take<T>((size_t)(a.nonneg ? std::max(Rtmax, Imax) : Rtmax) * R);
  a.H = cv.take<T>((size_t)Rtmax * R);
  a.Hpart = cv.take<T>((size_t)grid * R);
  for (int n = 0; n < N; ++n) a.Bout[n] = cv.take<T>((size_t)g.Rt[n] * R);
  T* uf[TDK_MAX_MODES];
  for (int n = 0; n < N; ++n) uf[n] = cv.take<T>((size_t)g.I[n] * g.Rt[n]);
  T* ulo[TDK_MAX_MODES] = {};
  if (leak32)
    for (int n = 0; n < N; ++n) ulo[n] = cv.take<T>((size_t)g.I[n] * g.Rt[n]);
  double* aw[TDK_MAX_MODES] = {};
  if (a.nonneg)
    for (int n = 0; n < N; ++n) aw[n] = cv.take<double>((size_t)g.I[n] * R);
  a.lam_out = cv.take<double>(R);
  a.hist_cap = std::min(o->max_sweeps, 65536);
  a.hist = cv.take<double>(a.hist_cap);
  a.st = cv.take<PState>(1);
  a.bar = cv.take<unsigned>(2);
  double* nG2 = cv.take<double>(1);
  double* nparts = cv.take<double>(NORM_BLOCKS);
  a.rpart = cv.take<double>(grid);
  a.xprev = cv.take<float>((size_t)grid * N * R * R);
  unsigned long long* prof = nullptr;
#ifdef TDK_TESTING
  const bool want_prof = getenv("TDK_ALS_PROFILE") != nullptr;
#else
  const bool want_prof = false;
#endif
  if (want_prof) {
    TDK_CUDA_TRY(cudaMallocAsync((void**)&prof, 32 * sizeof(unsigned long long), ctx->stream));
    TDK_CUDA_TRY(cudaMemsetAsync(prof, 0, 32 * sizeof(unsigned long long), ctx->stream));
  }
  a.prof = prof;
  a.status = ctx->d_status;
  a.G = G;
  a.nG2 = nG2;
  a.nY2 = normY2;
  cudaStream_t s = ctx->stream;
  for (int n = 0; n < N; ++n) {
    u_to_t<T><<<64, 256, 0, s>>>(U[n], uf[n], g.I[n] * g.Rt[n]);
    TDK_LAUNCH_CHECK(ctx);
    a.Uf[n] = uf[n];
    if (leak32) {
      u_lo_f32<<<64, 256, 0, s>>>(U[n], reinterpret_cast<float*>(ulo[n]), g.I[n] * g.Rt[n]);
      TDK_LAUNCH_CHECK(ctx);
      a.Ulo[n] = ulo[n];
    }
    a.init[n] = a.nonneg ? A_io[n] : B_io[n];
    a.Aout[n] = aw[n];  // running A_n; the caller's A_io stays the init until the end
  }
  norm2_core<T><<<NORM_BLOCKS, 256, 0, s>>>(G, g.core_numel, nparts);
  TDK_LAUNCH_CHECK(ctx);
  norm2_finish<<<1, 32, 0, s>>>(nparts, NORM_BLOCKS, nG2);
  TDK_LAUNCH_CHECK(ctx);
  TDK_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s));
  // 3-way unconstrained cores that fit in one SM: the single-CTA kernel
  SLayout<T> sl;
  sl.plan(g.Rt[0], g.Rt[N > 1 ? 1 : 0], g.Rt[N > 2 ? 2 : 0], R);
  bool small = N == 3 && !a.nonneg && sl.total + 64 <= (size_t)ctx->max_smem_optin;
#ifdef TDK_TESTING
  if (grid_cap > 0) small = false;
#endif
  if (small) {
    auto ks = als_small_kernel<T>;
    TDK_CUDA_TRY(cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sl.total + 64)));
    ks<<<1, NTS, sl.total + 64, s>>>(a);
    TDK_LAUNCH_CHECK(ctx);
  } else {
    void* args[] = {&a};
    TDK_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(NTP), args, smem, s));
    ctx->launches++;
  }
  // the lift is queued before the one synchronisation: if the kernel asks for
  // the pseudo-inverse (the kernel-per-step form then runs and rewrites the
  // outputs) or ran out of time (the outputs hold the last iterate either
  // way), lifting first does no harm
  rc = als_finish(ctx, g, R, sizeof(T) == 8, reinterpret_cast<const void* const*>(a.Bout), U, a.lam_out,
                  a.nonneg ? aw : nullptr, B_io, A_io, lambda_out,
                  sizeof(T) == 4 ? reinterpret_cast<const float* const*>(a.Uf) : nullptr);
  if (rc) return rc;
  PState hs{};
  TDK_CUDA_TRY(cudaMemcpyAsync(&hs, a.st, sizeof(PState), cudaMemcpyDeviceToHost, s));
  TDK_CUDA_TRY(cudaStreamSynchronize(s));
  if (want_prof) {
    unsigned long long hp[32];
    TDK_CUDA_TRY(cudaMemcpyAsync(hp, prof, sizeof(hp), cudaMemcpyDeviceToHost, s));
    TDK_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(prof);
    if (small) {
      const char* names[10] = {"T_n", "inverse|H", "solve", "refine", "normalise+gram", "fit", "check", "loop",
                               "[warp0 inverse]", "[warp1 H]"};
      fprintf(stderr, "tdk ALS profile (single CTA, Mcycles over %d sweeps):", hs.sweeps);
      for (int i = 0; i < 10; ++i) fprintf(stderr, " %s=%.3f", names[i], hp[i] / 1e6);
    } else {
      fprintf(stderr, "tdk ALS profile: T_n build=%.3f Mcycles, FP64 inverses=%llu, Newton-Schulz inverses=%llu"
              " (starts rejected %llu, stalled %llu, updates %llu)\n", hp[7] / 1e6, hp[9], hp[10], hp[16], hp[17],
              hp[18]);
      const char* names[7] = {"inverse", "H_rows", "barrier1", "nonneg_rows+barrier2", "normalise+gram+resid",
                              "barrier3", "fit"};
      fprintf(stderr, "tdk ALS profile (CTA 0, Mcycles over %d sweeps, grid %d):", hs.sweeps, grid);
      for (int i = 0; i < 7; ++i) fprintf(stderr, " %s=%.3f", names[i], hp[i] / 1e6);
      fprintf(stderr, "\n  inside H_rows: slice=%.3f first_product=%.3f other_products=%.3f (H_rows above: the"
              " solve and stores); inside normalise: norms+scale=%.3f gram=%.3f; sweep loop and fit tail=%.3f",
              hp[11] / 1e6, hp[12] / 1e6, hp[13] / 1e6, hp[14] / 1e6, hp[15] / 1e6, hp[8] / 1e6);
      fprintf(stderr, " (scalar tail %.3f, its barrier %.3f)", hp[19] / 1e6, hp[20] / 1e6);
    }
    fprintf(stderr, "\n");
  }
  if (hs.status & ST_NEEDPINV) return TDK_ENOTSUP;  // the multi-kernel form has the pseudo-inverse
  if (hs.status & ST_TIMEOUT) return TDK_ETIMEOUT;
  int status = TDK_OK;
  if (!hs.converged) status |= TDK_WNOCONV;
  if (rep) {
    rep->sweeps = hs.sweeps;
    rep->status = status;
    rep->fit_core = hs.fit;
    rep->fit_Y = normY2 ? hs.fitY : nan("");
    rep->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rep->form = small ? TDK_ALS_RAN_ONE_CTA : TDK_ALS_RAN_GRID;
    rep->grid = small ? 1 : grid;
  }
  return status;
}

template int als_persistent_t<float>(tdk_ctx*, const Geom&, const float*, const double* const[], const double*,
                                     const tdk_als_opts*, double* const[], double* const[], double*, tdk_als_report*);
template int als_persistent_t<double>(tdk_ctx*, const Geom&, const double*, const double* const[], const double*,
                                      const tdk_als_opts*, double* const[], double* const[], double*,
                                      tdk_als_report*);

}  // namespace tdk

namespace tdk {
TDK_CHECKED_UNIT(als_persistent)
}  // namespace tdk
