// Learned initialiser for FFCP (no counterpart in the paper, whose ALS starts
// from random or HOSVD factors, the first step of Alg. 1).  A small MLP maps a
// Tucker core G (Alg. 2 output) to initial core-space factors B_n.
//
//   canonicalise  V_n = eigenvectors of G_(n) G_(n)^T (HOSVD of the core) by
//                 decreasing eigenvalue, column signs chosen so that the
//                 ambient vectors U_n v_j have a nonnegative entry sum (the
//                 rule sees only colsum_n = 1^T U_n), S = G x_n V_n^T / ||G||.
//   MLP           x = bf16(sqrt(Rt^N) vec S) (unit RMS) -> 1024 -> 1024 -> N Rt^2, GELU, BF16
//                 operands on tcgen05 tensor cores with FP32 accumulation,
//                 FP32 master weights (mlp_gemm.cu).
//   loss          mean over samples of ||S - [[Bhat]]||^2
//                 + alpha ||[[Bhat]] - [[T]]||^2 over the first R columns,
//                 by the Gram identities (no model tensor is formed):
//                 ||[[B]]||^2 = 1^T (HADAMARD_n B_n^T B_n) 1 (Eq. 9 form) and
//                 <S, [[B]]> = sum(B_1 * H_1), H_1 = S_(1) KRP_{p != 1} B_p
//                 (the Y_(n) B term of Eq. 5).  T = V_n^T B*_n: converged FFCP factors.
//   training      back-propagation through the same GEMM kernel, Adam.
//   inference     B_n = V_n Bhat_n, FP64, ready as ffcp_als's B_io.
#include <cmath>
#include <cstring>
#include <vector>

#include "mlp_internal.cuh"

struct tdk_mlp {
  int device;
  int N, Rt, H, din, dout, max_batch;
  int ld_din, ld_H, ld_dout;
  int64_t P;
  int64_t off[7];  // W1, b1, W2, b2, W3, b3, end
  int64_t step;
  void* block;
  float *theta, *grad, *m, *v;
  __nv_bfloat16 *W1b, *W2b, *W3b;
  __nv_bfloat16 *Xb, *H1, *H2, *dO, *dZ2, *dZ1;
  float *Xs, *Z1, *Z2, *O, *V, *T;
  double *nrm, *lpart, *cs;
  double* gsq;    // per-block partial sums of the squared gradient
  float* gscale;  // the clipping factor of the last step
  int* Rdev;
  int last_batch;
};

namespace tdk {
namespace {

constexpr int CT = 256;  // threads of the per-sample kernels

inline int ru8(int x) { return (x + 7) / 8 * 8; }

struct Dims {
  int N, Rt, din, dout, ld_din, ld_dout;
};

__device__ __forceinline__ float blk_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}
__device__ __forceinline__ double blk_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// cyclic Jacobi on a symmetric Rt x Rt matrix in shared memory, one warp
// (lane i owns row / column i); A becomes diagonal, V accumulates the rotations
__device__ void warp_jacobi(float* A, float* V, int Rt) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < Rt; ++i)
    if (lane < Rt) V[i * Rt + lane] = (i == lane) ? 1.f : 0.f;
  __syncwarp();
  for (int sweep = 0; sweep < 20; ++sweep) {
    float off = 0.f, tot = 0.f;
    if (lane < Rt)
      for (int j = 0; j < Rt; ++j) {
        const float x = A[lane * Rt + j];
        tot += x * x;
        if (j != lane) off += x * x;
      }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if (!(off > 1e-13f * tot)) break;
    for (int p = 0; p < Rt - 1; ++p)
      for (int q = p + 1; q < Rt; ++q) {
        const float apq = A[p * Rt + q];
        const float app = A[p * Rt + p], aqq = A[q * Rt + q];
        __syncwarp();
        if (apq == 0.f) continue;
        const float tau = (aqq - app) / (2.f * apq);
        const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
        const float c = rsqrtf(1.f + t * t), s = t * c;
        if (lane < Rt) {  // columns p, q: A <- A J
          const float aip = A[lane * Rt + p], aiq = A[lane * Rt + q];
          A[lane * Rt + p] = c * aip - s * aiq;
          A[lane * Rt + q] = s * aip + c * aiq;
        }
        __syncwarp();
        if (lane < Rt) {  // rows p, q: A <- J^T A
          const float apj = A[p * Rt + lane], aqj = A[q * Rt + lane];
          A[p * Rt + lane] = c * apj - s * aqj;
          A[q * Rt + lane] = s * apj + c * aqj;
          const float vip = V[lane * Rt + p], viq = V[lane * Rt + q];
          V[lane * Rt + p] = c * vip - s * viq;
          V[lane * Rt + q] = s * vip + c * viq;
        }
        __syncwarp();
      }
  }
}

// one CTA per sample: canonical core S (FP32 and BF16 rows), rotations V_n,
// ||G||, and the canonical targets T_n = V_n^T B*_n (last mode / ||G||)
template <class TG>
__global__ void __launch_bounds__(CT) canon_kernel(const TG* __restrict__ G, const double* __restrict__ colsums,
                                                   const double* __restrict__ Bstar, const double* __restrict__ lam,
                                                   const int* __restrict__ Rs,
                                                   Dims d, float* __restrict__ Xs, __nv_bfloat16* __restrict__ Xb,
                                                   float* __restrict__ Vout, float* __restrict__ Tout,
                                                   double* __restrict__ nrm_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = d.N, Rt = d.Rt, din = d.din, RR = Rt * Rt;
  float* bufA = reinterpret_cast<float*>(smem_raw);
  float* bufB = bufA + din;
  float* Am = bufB + din;         // [N][Rt][Rt] Grams, then diagonalised
  float* Vm = Am + N * RR;        // [N][Rt][Rt] eigenvectors (sorted, signed)
  float* Vt = Vm + N * RR;        // [N][Rt][Rt] unsorted
  __shared__ double redd[32];
  const int b = blockIdx.x;
  const int t = threadIdx.x;
  const TG* g = G + (int64_t)b * din;
  double ss = 0.0;
  for (int e = t; e < din; e += CT) {
    const float x = (float)g[e];
    bufA[e] = x;
    ss += (double)x * (double)x;
  }
  const double n2 = blk_sum_d(ss, redd);  // ends with a barrier: bufA complete
  // Grams of every unfolding, upper triangle
  int stride[8];
  {
    int s = 1;
    for (int k = N - 1; k >= 0; --k) {
      stride[k] = s;
      s *= Rt;
    }
  }
  const int others = din / Rt;
  const int npairs = Rt * (Rt + 1) / 2;
  for (int task = t; task < N * npairs; task += CT) {
    const int n = task / npairs;
    int pr = task % npairs, a = 0;
    while (pr >= Rt - a) {
      pr -= Rt - a;
      ++a;
    }
    const int bb = a + pr;
    const int sn = stride[n];
    float acc = 0.f;
    for (int j = 0; j < others; ++j) {
      const int e0 = (j / sn) * (sn * Rt) + (j % sn);
      acc = fmaf(bufA[e0 + a * sn], bufA[e0 + bb * sn], acc);
    }
    Am[n * RR + a * Rt + bb] = acc;
    Am[n * RR + bb * Rt + a] = acc;
  }
  __syncthreads();
  const int warp = t >> 5, lane = t & 31;
  if (warp < N) {
    float* A = Am + warp * RR;
    float* Vu = Vt + warp * RR;
    warp_jacobi(A, Vu, Rt);
    // order by decreasing eigenvalue (ties by index), then fix the signs
    float lam = lane < Rt ? A[lane * Rt + lane] : 0.f;
    int rank = 0;
    for (int j = 0; j < Rt; ++j) {
      const float lj = __shfl_sync(0xffffffffu, lam, j);
      if (lane < Rt && (lj > lam || (lj == lam && j < lane))) ++rank;
    }
    float* Vs = Vm + warp * RR;
    if (lane < Rt) {
      const double* cs = colsums + ((int64_t)b * N + warp) * Rt;
      double s = 0.0;
      for (int i = 0; i < Rt; ++i) s += cs[i] * (double)Vu[i * Rt + lane];
      const float sg = (s < 0.0) ? -1.f : 1.f;
      for (int i = 0; i < Rt; ++i) Vs[i * Rt + rank] = sg * Vu[i * Rt + lane];
    }
  }
  __syncthreads();
  // S = G x_1 V_1^T ... x_N V_N^T
  float* in = bufA;
  float* out = bufB;
  for (int n = 0; n < N; ++n) {
    const int sn = stride[n];
    const float* Vn = Vm + n * RR;
    for (int e = t; e < din; e += CT) {
      const int r = (e / sn) % Rt;
      const int e0 = e - r * sn;
      float acc = 0.f;
      for (int i = 0; i < Rt; ++i) acc = fmaf(Vn[i * Rt + r], in[e0 + i * sn], acc);
      out[e] = acc;
    }
    __syncthreads();
    float* tmp = in;
    in = out;
    out = tmp;
  }
  const double nrm = sqrt(n2);
  const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
  const float xs = sqrtf((float)din);  // network input at unit RMS
  for (int e = t; e < din; e += CT) {
    const float x = in[e] * inv;
    Xs[(int64_t)b * din + e] = x;
    Xb[(int64_t)b * d.ld_din + e] = __float2bfloat16_rn(x * xs);
  }
  for (int e = t; e < N * RR; e += CT) Vout[(int64_t)b * N * RR + e] = Vm[e];
  if (t == 0) nrm_out[b] = nrm;
  if (Bstar) {
    const int R = Rs[b];
    for (int e = t; e < N * RR; e += CT) {
      const int n = e / RR, i = (e % RR) / Rt, r = e % Rt;
      float v = 0.f;
      if (r < R) {
        const double* Bn = Bstar + ((int64_t)b * N + n) * RR;
        double acc = 0.0;
        for (int k = 0; k < Rt; ++k) acc += (double)Vm[n * RR + k * Rt + i] * Bn[k * Rt + r];
        if (n == N - 1) {
          if (lam) acc *= lam[(int64_t)b * Rt + r];
          acc = nrm > 0.0 ? acc / nrm : 0.0;
        }
        v = (float)acc;
      }
      Tout[(int64_t)b * N * RR + e] = v;
    }
  }
}

// one CTA per sample: loss and dL/dO (BF16, scaled by 1/batch) by the Gram
// identities over the first R columns
__global__ void __launch_bounds__(CT) loss_kernel(const float* __restrict__ Xs, const float* __restrict__ O,
                                                  const float* __restrict__ T, const int* __restrict__ Rs, Dims d,
                                                  float alpha, float inv_batch, int has_target,
                                                  __nv_bfloat16* __restrict__ dO, double* __restrict__ lpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = d.N, Rt = d.Rt, din = d.din, RR = Rt * Rt;
  const int b = blockIdx.x, t = threadIdx.x;
  const int R = Rs[b];
  float* S = reinterpret_cast<float*>(smem_raw);  // [din]
  float* Bh = S + din;                             // [N][Rt][Rt] (columns < R used)
  float* Tm = Bh + N * RR;                         // [N][Rt][Rt]
  float* Hm = Tm + N * RR;                         // [N][Rt][Rt] MTTKRP
  float* Gm = Hm + N * RR;                         // [N][Rt][Rt] B_p^T B_p
  float* Cm = Gm + N * RR;                         // [N][Rt][Rt] T_p^T B_p
  float* Dm = Cm + N * RR;                         // [N][Rt][Rt] T_p^T T_p
  __shared__ float red[32];
  for (int e = t; e < din; e += CT) S[e] = Xs[(int64_t)b * din + e];
  for (int e = t; e < N * RR; e += CT) {
    const int r = e % Rt;
    Bh[e] = r < R ? O[(int64_t)b * d.dout + e] : 0.f;
    Tm[e] = (has_target && r < R) ? T[(int64_t)b * N * RR + e] : 0.f;
  }
  __syncthreads();
  int stride[8];
  {
    int s = 1;
    for (int k = N - 1; k >= 0; --k) {
      stride[k] = s;
      s *= Rt;
    }
  }
  // small Grams
  for (int e = t; e < 3 * N * RR; e += CT) {
    const int which = e / (N * RR), rem = e % (N * RR);
    const int p = rem / RR, r1 = (rem % RR) / Rt, r2 = rem % Rt;
    const float* X1 = (which == 0 ? Bh : Tm) + p * RR;
    const float* X2 = (which == 2 ? Tm : Bh) + p * RR;
    float acc = 0.f;
    if (r1 < R && r2 < R)
      for (int i = 0; i < Rt; ++i) acc = fmaf(X1[i * Rt + r1], X2[i * Rt + r2], acc);
    (which == 0 ? Gm : which == 1 ? Cm : Dm)[p * RR + r1 * Rt + r2] = acc;
  }
  // MTTKRP of S with Bhat for every mode
  const int others = din / Rt;
  for (int task = t; task < N * RR; task += CT) {
    const int n = task / RR, i = (task % RR) / Rt, r = task % Rt;
    float acc = 0.f;
    if (r < R) {
      const int sn = stride[n];
      for (int j = 0; j < others; ++j) {
        const int e0 = (j / sn) * (sn * Rt) + (j % sn);
        const int e = e0 + i * sn;
        float prod = S[e];
        for (int p = 0; p < N; ++p) {
          if (p == n) continue;
          const int ip = (e / stride[p]) % Rt;
          prod *= Bh[p * RR + ip * Rt + r];
        }
        acc += prod;
      }
    }
    Hm[task] = acc;
  }
  __syncthreads();
  // scalar pieces
  float pS = 0.f, pin = 0.f, pnb = 0.f, pcr = 0.f, pnt = 0.f;
  for (int e = t; e < din; e += CT) pS = fmaf(S[e], S[e], pS);
  for (int e = t; e < RR; e += CT) pin = fmaf(Bh[e], Hm[e], pin);  // mode 0
  for (int e = t; e < RR; e += CT) {
    const int r1 = e / Rt, r2 = e % Rt;
    if (r1 < R && r2 < R) {
      float g = 1.f, c = 1.f, dd = 1.f;
      for (int p = 0; p < N; ++p) {
        g *= Gm[p * RR + e];
        c *= Cm[p * RR + e];
        dd *= Dm[p * RR + e];
      }
      pnb += g;
      pcr += c;
      pnt += dd;
    }
  }
  const double sS = blk_sum(pS, red), sin_ = blk_sum(pin, red), snb = blk_sum(pnb, red);
  const double scr = blk_sum(pcr, red), snt = blk_sum(pnt, red);
  double L = sS - 2.0 * sin_ + snb;
  if (has_target) L += (double)alpha * (snb - 2.0 * scr + snt);
  if (t == 0) lpart[b] = L;
  // gradient: -2 H_n + 2 (1 + alpha) B_n G^{!n} - 2 alpha T_n C^{!n}
  const float wB = 2.f * (1.f + (has_target ? alpha : 0.f));
  for (int e = t; e < N * RR; e += CT) {
    const int n = e / RR, i = (e % RR) / Rt, r = e % Rt;
    float gval = 0.f;
    if (r < R) {
      float s1 = 0.f, s2 = 0.f;
      for (int r2 = 0; r2 < R; ++r2) {
        float gp = 1.f, cp = 1.f;
        for (int p = 0; p < N; ++p) {
          if (p == n) continue;
          gp *= Gm[p * RR + r2 * Rt + r];
          cp *= Cm[p * RR + r2 * Rt + r];
        }
        s1 = fmaf(Bh[n * RR + i * Rt + r2], gp, s1);
        s2 = fmaf(Tm[n * RR + i * Rt + r2], cp, s2);
      }
      gval = -2.f * Hm[e] + wB * s1;
      if (has_target) gval -= 2.f * alpha * s2;
      gval *= inv_batch;
    }
    dO[(int64_t)b * d.ld_dout + e] = __float2bfloat16_rn(gval);
  }
}

// bias gradient: column sums of a BF16 [rows][ld] matrix, fixed order
__global__ void colsum_kernel(const __nv_bfloat16* __restrict__ D, int rows, int cols, int ld,
                              float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += __bfloat162float(D[(int64_t)r * ld + c]);
  out[c] = s;
}

struct Segs {
  int64_t off[7];
  int rows[3], cols[3], ld[3];
  __nv_bfloat16* dst[3];
};

// BF16 copy of the weight matrices from the FP32 master parameters
__device__ __forceinline__ void store_bf16_copy(const Segs& sg, int64_t e, float x) {
#pragma unroll
  for (int w = 0; w < 3; ++w) {
    const int64_t o = sg.off[2 * w];
    if (e >= o && e < sg.off[2 * w + 1]) {
      const int64_t k = e - o;
      const int r = (int)(k / sg.cols[w]), c = (int)(k % sg.cols[w]);
      sg.dst[w][(int64_t)r * sg.ld[w] + c] = __float2bfloat16_rn(x);
    }
  }
}

__global__ void refresh_kernel(const float* __restrict__ theta, Segs sg) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sg.off[6];
       e += (int64_t)gridDim.x * blockDim.x)
    store_bf16_copy(sg, e, theta[e]);
}

// Adam (Kingma and Ba, Algorithm 1) on the FP32 master parameters
constexpr int GN_BLOCKS = 256;  // blocks of the gradient-norm reduction

// squared gradient norm: one FP64 partial per block, summed in a fixed order
__global__ void gradsq_kernel(const float* __restrict__ g, int64_t n, double* __restrict__ parts) {
  __shared__ double red[CT / 32];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = g[e];
    s = fma(x, x, s);
  }
  s = blk_sum_d(s, red);
  if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// clipping factor min(1, clip / ||g||)
__global__ void clip_scale_kernel(const double* __restrict__ parts, int nparts, double clip, float* __restrict__ scale) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < nparts; ++i) s += parts[i];
  const double nrm = sqrt(s);
  *scale = (float)(nrm > clip ? clip / nrm : 1.0);
}

// gscale: null, or the clipping factor applied to the gradient first
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, Segs sg, float lr, float b1, float b2, float eps,
                            float bc1, float bc2, const float* __restrict__ gscale) {
  const float sc = gscale ? *gscale : 1.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sg.off[6];
       e += (int64_t)gridDim.x * blockDim.x) {
    const float ge = g[e] * sc;
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    const float x = theta[e] - lr * (me / bc1) / (sqrtf(ve / bc2) + eps);
    theta[e] = x;
    store_bf16_copy(sg, e, x);
  }
}

// column sums 1^T U_n (FP64), one block per mode
struct UPtrs {
  const double* p[TDK_MAX_MODES];
  int64_t I[TDK_MAX_MODES];
};
__global__ void ucolsum_kernel(UPtrs u, int Rt, double* __restrict__ out) {
  const int n = blockIdx.x;
  const int r = threadIdx.x;
  if (r >= Rt) return;
  double s = 0.0;
  for (int64_t i = 0; i < u.I[n]; ++i) s += u.p[n][i * Rt + r];
  out[n * Rt + r] = s;
}

// B_n = V_n Bhat_n (first R columns), FP64, for sample 0
struct BPtrs {
  double* p[TDK_MAX_MODES];
};
__global__ void decanon_kernel(const float* __restrict__ V, const float* __restrict__ O, Dims d, int R, BPtrs out) {
  const int Rt = d.Rt, RR = Rt * Rt;
  for (int e = threadIdx.x; e < d.N * Rt * R; e += blockDim.x) {
    const int n = e / (Rt * R), i = (e % (Rt * R)) / R, r = e % R;
    double acc = 0.0;
    for (int j = 0; j < Rt; ++j) acc += (double)V[n * RR + i * Rt + j] * (double)O[n * RR + j * Rt + r];
    out.p[n][i * R + r] = acc;
  }
}

Dims dims_of(const tdk_mlp* m) {
  Dims d;
  d.N = m->N;
  d.Rt = m->Rt;
  d.din = m->din;
  d.dout = m->dout;
  d.ld_din = m->ld_din;
  d.ld_dout = m->ld_dout;
  return d;
}

Segs segs_of(const tdk_mlp* m) {
  Segs s{};
  for (int i = 0; i < 7; ++i) s.off[i] = m->off[i];
  s.rows[0] = m->H;
  s.cols[0] = m->din;
  s.ld[0] = m->ld_din;
  s.dst[0] = m->W1b;
  s.rows[1] = m->H;
  s.cols[1] = m->H;
  s.ld[1] = m->ld_H;
  s.dst[1] = m->W2b;
  s.rows[2] = m->dout;
  s.cols[2] = m->H;
  s.ld[2] = m->ld_H;
  s.dst[2] = m->W3b;
  return s;
}

size_t canon_smem(const tdk_mlp* m) {
  return sizeof(float) * (2 * (size_t)m->din + 3 * (size_t)m->N * m->Rt * m->Rt);
}
size_t loss_smem(const tdk_mlp* m) {
  return sizeof(float) * ((size_t)m->din + 6 * (size_t)m->N * m->Rt * m->Rt);
}

int run_canon(tdk_ctx* ctx, tdk_mlp* m, int batch, const void* G, int g_f64, const double* colsums,
              const double* Bstar, const double* lam, const int* R) {
  const Dims d = dims_of(m);
  const size_t sm = canon_smem(m);
  if (sm > (size_t)ctx->max_smem_optin) return TDK_EINVAL;
  if (g_f64) {
    TDK_CUDA_TRY(cudaFuncSetAttribute(canon_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    canon_kernel<double><<<batch, CT, sm, ctx->stream>>>(static_cast<const double*>(G), colsums, Bstar, lam, R, d, m->Xs,
                                                         m->Xb, m->V, m->T, m->nrm);
  } else {
    TDK_CUDA_TRY(cudaFuncSetAttribute(canon_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    canon_kernel<float><<<batch, CT, sm, ctx->stream>>>(static_cast<const float*>(G), colsums, Bstar, lam, R, d, m->Xs,
                                                        m->Xb, m->V, m->T, m->nrm);
  }
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

int run_forward(tdk_ctx* ctx, tdk_mlp* m, int batch) {
  GemmOp op{};
  op.M = batch;
  op.N = m->H;
  op.K = m->din;
  op.A = m->Xb;
  op.lda = m->ld_din;
  op.B = m->W1b;
  op.ldb = m->ld_din;
  op.mode = GEMM_BIAS_GELU;
  op.bias = m->theta + m->off[1];
  op.outf = m->Z1;
  op.ldf = m->H;
  op.outb = m->H1;
  op.ldob = m->ld_H;
  int rc = gemm_bf16(ctx, op);
  if (rc) return rc;
  op.K = m->H;
  op.A = m->H1;
  op.lda = m->ld_H;
  op.B = m->W2b;
  op.ldb = m->ld_H;
  op.bias = m->theta + m->off[3];
  op.outf = m->Z2;
  op.outb = m->H2;
  rc = gemm_bf16(ctx, op);
  if (rc) return rc;
  op.N = m->dout;
  op.A = m->H2;
  op.B = m->W3b;
  op.mode = GEMM_BIAS_F32;
  op.bias = m->theta + m->off[5];
  op.outf = m->O;
  op.ldf = m->dout;
  op.outb = nullptr;
  return gemm_bf16(ctx, op);
}

int run_backward(tdk_ctx* ctx, tdk_mlp* m, int batch) {
  float* g = m->grad;
  auto colsum = [&](const __nv_bfloat16* D, int cols, int ld, float* out) {
    colsum_kernel<<<(cols + 255) / 256, 256, 0, ctx->stream>>>(D, batch, cols, ld, out);
  };
  // layer 3
  GemmOp op{};
  op.M = m->dout;
  op.N = m->H;
  op.K = batch;
  op.A = m->dO;
  op.lda = m->ld_dout;
  op.a_mn = 1;
  op.B = m->H2;
  op.ldb = m->ld_H;
  op.b_mn = 1;
  op.mode = GEMM_STORE_F32;
  op.outf = g + m->off[4];
  op.ldf = m->H;
  int rc = gemm_bf16(ctx, op);
  if (rc) return rc;
  colsum(m->dO, m->dout, m->ld_dout, g + m->off[5]);
  TDK_LAUNCH_CHECK(ctx);
  GemmOp dz{};
  dz.M = batch;
  dz.N = m->H;
  dz.K = m->dout;
  dz.A = m->dO;
  dz.lda = m->ld_dout;
  dz.B = m->W3b;
  dz.ldb = m->ld_H;
  dz.b_mn = 1;
  dz.mode = GEMM_GELU_GRAD;
  dz.zin = m->Z2;
  dz.ldz = m->H;
  dz.outb = m->dZ2;
  dz.ldob = m->ld_H;
  rc = gemm_bf16(ctx, dz);
  if (rc) return rc;
  // layer 2
  op.M = m->H;
  op.A = m->dZ2;
  op.lda = m->ld_H;
  op.B = m->H1;
  op.outf = g + m->off[2];
  rc = gemm_bf16(ctx, op);
  if (rc) return rc;
  colsum(m->dZ2, m->H, m->ld_H, g + m->off[3]);
  TDK_LAUNCH_CHECK(ctx);
  dz.K = m->H;
  dz.A = m->dZ2;
  dz.lda = m->ld_H;
  dz.B = m->W2b;
  dz.zin = m->Z1;
  dz.outb = m->dZ1;
  rc = gemm_bf16(ctx, dz);
  if (rc) return rc;
  // layer 1
  op.N = m->din;
  op.A = m->dZ1;
  op.B = m->Xb;
  op.ldb = m->ld_din;
  op.outf = g + m->off[0];
  op.ldf = m->din;
  rc = gemm_bf16(ctx, op);
  if (rc) return rc;
  colsum(m->dZ1, m->H, m->ld_H, g + m->off[1]);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // namespace
}  // namespace tdk

using namespace tdk;

extern "C" {

int tdk_mlp_create(tdk_ctx* ctx, const tdk_mlp_desc* d, tdk_mlp** out) {
  if (!ctx || !d || !out) return TDK_EINVAL;
  *out = nullptr;
  if (d->N < 2 || d->N > 4 || d->Rt < 2 || d->Rt > 32 || d->hidden < 8 || d->hidden > 8192 || d->max_batch < 1 ||
      d->max_batch > 65536)
    return TDK_EINVAL;
  int64_t din = 1;
  for (int n = 0; n < d->N; ++n) din *= d->Rt;
  if (din > 12288) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  tdk_mlp* m = new tdk_mlp();
  m->device = ctx->device;
  m->N = d->N;
  m->Rt = d->Rt;
  m->H = d->hidden;
  m->din = (int)din;
  m->dout = d->N * d->Rt * d->Rt;
  m->max_batch = d->max_batch;
  m->ld_din = ru8(m->din);
  m->ld_H = ru8(m->H);
  m->ld_dout = ru8(m->dout);
  const int64_t sizes[6] = {(int64_t)m->H * m->din, m->H, (int64_t)m->H * m->H, m->H, (int64_t)m->dout * m->H,
                            m->dout};
  m->off[0] = 0;
  for (int i = 0; i < 6; ++i) m->off[i + 1] = m->off[i] + sizes[i];
  m->P = m->off[6];
  const int64_t Bt = m->max_batch, RR = (int64_t)m->Rt * m->Rt;
  Planner pl;
  for (int i = 0; i < 4; ++i) pl.take<float>((size_t)m->P);
  pl.take<__nv_bfloat16>((size_t)m->H * m->ld_din);
  pl.take<__nv_bfloat16>((size_t)m->H * m->ld_H);
  pl.take<__nv_bfloat16>((size_t)m->dout * m->ld_H);
  pl.take<__nv_bfloat16>((size_t)Bt * m->ld_din);
  for (int i = 0; i < 2; ++i) pl.take<__nv_bfloat16>((size_t)Bt * m->ld_H);
  pl.take<__nv_bfloat16>((size_t)Bt * m->ld_dout);
  for (int i = 0; i < 2; ++i) pl.take<__nv_bfloat16>((size_t)Bt * m->ld_H);
  pl.take<float>((size_t)Bt * m->din);
  for (int i = 0; i < 2; ++i) pl.take<float>((size_t)Bt * m->H);
  pl.take<float>((size_t)Bt * m->dout);
  for (int i = 0; i < 2; ++i) pl.take<float>((size_t)Bt * m->N * RR);
  for (int i = 0; i < 2; ++i) pl.take<double>((size_t)Bt);
  pl.take<double>((size_t)m->N * m->Rt);
  pl.take<int>((size_t)Bt);
  pl.take<double>((size_t)GN_BLOCKS);
  pl.take<float>(1);
  if (cudaMalloc(&m->block, pl.off) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return TDK_ENOMEM;
  }
  Carver cv(m->block);
  m->theta = cv.take<float>((size_t)m->P);
  m->grad = cv.take<float>((size_t)m->P);
  m->m = cv.take<float>((size_t)m->P);
  m->v = cv.take<float>((size_t)m->P);
  m->W1b = cv.take<__nv_bfloat16>((size_t)m->H * m->ld_din);
  m->W2b = cv.take<__nv_bfloat16>((size_t)m->H * m->ld_H);
  m->W3b = cv.take<__nv_bfloat16>((size_t)m->dout * m->ld_H);
  m->Xb = cv.take<__nv_bfloat16>((size_t)Bt * m->ld_din);
  m->H1 = cv.take<__nv_bfloat16>((size_t)Bt * m->ld_H);
  m->H2 = cv.take<__nv_bfloat16>((size_t)Bt * m->ld_H);
  m->dO = cv.take<__nv_bfloat16>((size_t)Bt * m->ld_dout);
  m->dZ2 = cv.take<__nv_bfloat16>((size_t)Bt * m->ld_H);
  m->dZ1 = cv.take<__nv_bfloat16>((size_t)Bt * m->ld_H);
  m->Xs = cv.take<float>((size_t)Bt * m->din);
  m->Z1 = cv.take<float>((size_t)Bt * m->H);
  m->Z2 = cv.take<float>((size_t)Bt * m->H);
  m->O = cv.take<float>((size_t)Bt * m->dout);
  m->V = cv.take<float>((size_t)Bt * m->N * RR);
  m->T = cv.take<float>((size_t)Bt * m->N * RR);
  m->nrm = cv.take<double>((size_t)Bt);
  m->lpart = cv.take<double>((size_t)Bt);
  m->cs = cv.take<double>((size_t)m->N * m->Rt);
  m->Rdev = cv.take<int>((size_t)Bt);
  m->gsq = cv.take<double>((size_t)GN_BLOCKS);
  m->gscale = cv.take<float>(1);
  if (cudaMemsetAsync(m->block, 0, pl.off, ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(m->block);
    delete m;
    return TDK_ECUDA;
  }
  *out = m;
  return TDK_OK;
}

int tdk_mlp_destroy(tdk_mlp* m) {
  if (!m) return TDK_EINVAL;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  cudaFree(m->block);
  delete m;
  return TDK_OK;
}

int64_t tdk_mlp_param_count(const tdk_mlp* m) { return m ? m->P : -1; }

int tdk_mlp_set_params(tdk_ctx* ctx, tdk_mlp* m, const float* host_params) {
  if (!ctx || !m || !host_params) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  TDK_CUDA_TRY(cudaMemcpyAsync(m->theta, host_params, sizeof(float) * m->P, cudaMemcpyHostToDevice, ctx->stream));
  TDK_CUDA_TRY(cudaMemsetAsync(m->m, 0, sizeof(float) * m->P, ctx->stream));
  TDK_CUDA_TRY(cudaMemsetAsync(m->v, 0, sizeof(float) * m->P, ctx->stream));
  refresh_kernel<<<2 * ctx->num_sms, 256, 0, ctx->stream>>>(m->theta, segs_of(m));
  TDK_LAUNCH_CHECK(ctx);
  m->step = 0;
  TDK_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return TDK_OK;
}

int tdk_mlp_get(tdk_ctx* ctx, tdk_mlp* m, int what, float* host_out) {
  if (!ctx || !m || !host_out) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  const float* src = nullptr;
  size_t n = 0;
  const int64_t B = m->last_batch, RR = (int64_t)m->Rt * m->Rt;
  // stored BF16 intermediates: [batch x cols] rows of pitch ld, widened on the host
  const __nv_bfloat16* sb = nullptr;
  int cols = 0, ld = 0;
  switch (what) {
    case TDK_MLP_PARAMS: src = m->theta; n = m->P; break;
    case TDK_MLP_GRADS: src = m->grad; n = m->P; break;
    case TDK_MLP_CANON_CORE: src = m->Xs; n = B * m->din; break;
    case TDK_MLP_ROTATIONS: src = m->V; n = B * m->N * RR; break;
    case TDK_MLP_OUTPUT: src = m->O; n = B * m->dout; break;
    case TDK_MLP_Z1: src = m->Z1; n = B * m->H; break;
    case TDK_MLP_Z2: src = m->Z2; n = B * m->H; break;
    case TDK_MLP_INPUT: sb = m->Xb; cols = m->din; ld = m->ld_din; break;
    case TDK_MLP_H1: sb = m->H1; cols = m->H; ld = m->ld_H; break;
    case TDK_MLP_H2: sb = m->H2; cols = m->H; ld = m->ld_H; break;
    case TDK_MLP_DO: sb = m->dO; cols = m->dout; ld = m->ld_dout; break;
    case TDK_MLP_DZ2: sb = m->dZ2; cols = m->H; ld = m->ld_H; break;
    case TDK_MLP_DZ1: sb = m->dZ1; cols = m->H; ld = m->ld_H; break;
    default: return TDK_EINVAL;
  }
  if (sb) {
    std::vector<uint16_t> raw((size_t)B * ld);
    if (!raw.empty())
      TDK_CUDA_TRY(cudaMemcpyAsync(raw.data(), sb, sizeof(uint16_t) * raw.size(), cudaMemcpyDeviceToHost,
                                   ctx->stream));
    TDK_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int64_t b = 0; b < B; ++b)
      for (int c = 0; c < cols; ++c) {
        // a BF16 value is the upper half of the FP32 value with the same bits
        const uint32_t bits = (uint32_t)raw[(size_t)b * ld + c] << 16;
        float f;
        std::memcpy(&f, &bits, sizeof f);
        host_out[b * cols + c] = f;
      }
    return TDK_OK;
  }
  if (n) TDK_CUDA_TRY(cudaMemcpyAsync(host_out, src, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
  TDK_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return TDK_OK;
}

// checkpoint file: tag, shape, parameter count, Adam step, then the
// parameters and Adam's two moment vectors (FP32, host byte order, which is
// little-endian on every platform this library builds for)
static const char kMlpTag[8] = {'T', 'D', 'K', 'M', 'L', 'P', '0', '1'};

int tdk_mlp_save(tdk_ctx* ctx, const tdk_mlp* m, const char* path) {
  if (!ctx || !m || !path) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  std::vector<float> buf((size_t)3 * m->P);
  const float* src[3] = {m->theta, m->m, m->v};
  for (int i = 0; i < 3; ++i)
    TDK_CUDA_TRY(cudaMemcpyAsync(buf.data() + (size_t)i * m->P, src[i], sizeof(float) * m->P,
                                 cudaMemcpyDeviceToHost, ctx->stream));
  TDK_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  FILE* f = fopen(path, "wb");
  if (!f) return TDK_EIO;
  const int32_t shape[4] = {m->N, m->Rt, m->H, 0};
  const int64_t counts[2] = {m->P, m->step};
  bool ok = fwrite(kMlpTag, 1, 8, f) == 8 && fwrite(shape, sizeof(int32_t), 4, f) == 4 &&
            fwrite(counts, sizeof(int64_t), 2, f) == 2 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? TDK_OK : TDK_EIO;
}

int tdk_mlp_load(tdk_ctx* ctx, tdk_mlp* m, const char* path) {
  if (!ctx || !m || !path) return TDK_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return TDK_EIO;
  char tag[8];
  int32_t shape[4];
  int64_t counts[2];
  std::vector<float> buf((size_t)3 * m->P);
  bool ok = fread(tag, 1, 8, f) == 8 && std::memcmp(tag, kMlpTag, 8) == 0 && fread(shape, sizeof(int32_t), 4, f) == 4 &&
            shape[0] == m->N && shape[1] == m->Rt && shape[2] == m->H && fread(counts, sizeof(int64_t), 2, f) == 2 &&
            counts[0] == m->P && counts[1] >= 0 && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  if (ok) {
    char extra;
    ok = fread(&extra, 1, 1, f) == 0;  // nothing after the three vectors
  }
  fclose(f);
  if (!ok) return TDK_EIO;
  cudaSetDevice(ctx->device);
  float* dst[3] = {m->theta, m->m, m->v};
  for (int i = 0; i < 3; ++i)
    TDK_CUDA_TRY(cudaMemcpyAsync(dst[i], buf.data() + (size_t)i * m->P, sizeof(float) * m->P, cudaMemcpyHostToDevice,
                                 ctx->stream));
  refresh_kernel<<<2 * ctx->num_sms, 256, 0, ctx->stream>>>(m->theta, segs_of(m));
  TDK_LAUNCH_CHECK(ctx);
  m->step = counts[1];
  TDK_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return TDK_OK;
}

int tdk_mlp_colsums(tdk_ctx* ctx, const tdk_tucker_desc* desc, const double* const U[], double* out) {
  if (!ctx || !desc || !U || !out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  UPtrs u{};
  for (int n = 0; n < g.N; ++n) {
    if (!U[n] || g.Rt[n] != g.Rt[0]) return TDK_EINVAL;
    u.p[n] = U[n];
    u.I[n] = g.I[n];
  }
  cudaSetDevice(ctx->device);
  ucolsum_kernel<<<g.N, 64, 0, ctx->stream>>>(u, g.Rt[0], out);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

int tdk_mlp_train_step(tdk_ctx* ctx, tdk_mlp* m, int batch, const float* G, const double* colsums, const int* R,
                       const double* Bstar, const double* lambda, const tdk_mlp_train_opts* o, double* loss_out) {
  if (!ctx || !m || !G || !colsums || !R || !o) return TDK_EINVAL;
  if (batch < 1 || batch > m->max_batch) return TDK_EINVAL;
  if (!(o->lr >= 0.0) || !(o->beta1 >= 0.0 && o->beta1 < 1.0) || !(o->beta2 >= 0.0 && o->beta2 < 1.0) ||
      !(o->eps > 0.0) || !(o->clip >= 0.0))
    return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  int rc = run_canon(ctx, m, batch, G, 0, colsums, Bstar, lambda, R);
  if (rc) return rc;
  m->last_batch = batch;
  rc = run_forward(ctx, m, batch);
  if (rc) return rc;
  const Dims d = dims_of(m);
  const size_t sm = loss_smem(m);
  if (sm > (size_t)ctx->max_smem_optin) return TDK_EINVAL;
  TDK_CUDA_TRY(cudaFuncSetAttribute(loss_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const int has_t = (Bstar && o->alpha != 0.0) ? 1 : 0;
  loss_kernel<<<batch, CT, sm, ctx->stream>>>(m->Xs, m->O, m->T, R, d, (float)o->alpha, 1.f / (float)batch, has_t,
                                              m->dO, m->lpart);
  TDK_LAUNCH_CHECK(ctx);
  rc = run_backward(ctx, m, batch);
  if (rc) return rc;
  if (o->update) {
    m->step++;
    const double bc1 = 1.0 - std::pow(o->beta1, (double)m->step), bc2 = 1.0 - std::pow(o->beta2, (double)m->step);
    const float* gsc = nullptr;
    if (o->clip > 0.0) {
      gradsq_kernel<<<GN_BLOCKS, CT, 0, ctx->stream>>>(m->grad, m->P, m->gsq);
      TDK_LAUNCH_CHECK(ctx);
      clip_scale_kernel<<<1, 32, 0, ctx->stream>>>(m->gsq, GN_BLOCKS, o->clip, m->gscale);
      TDK_LAUNCH_CHECK(ctx);
      gsc = m->gscale;
    }
    adam_kernel<<<4 * ctx->num_sms, 256, 0, ctx->stream>>>(m->theta, m->m, m->v, m->grad, segs_of(m), (float)o->lr,
                                                           (float)o->beta1, (float)o->beta2, (float)o->eps,
                                                           (float)bc1, (float)bc2, gsc);
    TDK_LAUNCH_CHECK(ctx);
  }
  if (loss_out) {
    std::vector<double> lp(batch);
    TDK_CUDA_TRY(cudaMemcpyAsync(lp.data(), m->lpart, sizeof(double) * batch, cudaMemcpyDeviceToHost, ctx->stream));
    TDK_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    double s = 0.0;
    for (int i = 0; i < batch; ++i) s += lp[i];
    *loss_out = s / batch;
  }
  return TDK_OK;
}

int ffcp_predict_init(tdk_ctx* ctx, tdk_mlp* m, const tdk_tucker_desc* desc, const void* G, const double* const U[],
                      int R, double* const B_out[]) {
  if (!ctx || !m || !desc || !G || !U || !B_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  if (g.N != m->N || R < 1 || R > m->Rt) return TDK_EINVAL;
  for (int n = 0; n < g.N; ++n)
    if (g.Rt[n] != m->Rt || !B_out[n] || !U[n]) return TDK_EINVAL;
  rc = tdk_mlp_colsums(ctx, desc, U, m->cs);
  if (rc) return rc;
  rc = run_canon(ctx, m, 1, G, desc->dtype == TDK_F64, m->cs, nullptr, nullptr, nullptr);
  if (rc) return rc;
  m->last_batch = 1;
  rc = run_forward(ctx, m, 1);
  if (rc) return rc;
  BPtrs bp{};
  for (int n = 0; n < g.N; ++n) bp.p[n] = B_out[n];
  decanon_kernel<<<1, 256, 0, ctx->stream>>>(m->V, m->O, dims_of(m), R, bp);
  TDK_LAUNCH_CHECK(ctx);
  return TDK_OK;
}

}  // extern "C"

namespace tdk {
TDK_CHECKED_UNIT(mlp)
}  // namespace tdk
