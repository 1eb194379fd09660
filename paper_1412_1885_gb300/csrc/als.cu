// FFCP: CP-ALS on the Tucker core (Sec. III-B, Alg. 1; Eqs. 9, 11-14, 17).
//
// Per sweep, for every mode n (Gauss-Seidel order 1..N):
//   H_n = G_(n) [KRP_{p != n} B_p]      (als_mttkrp: the Khatri-Rao product is
//                                         never formed; each core entry is
//                                         multiplied by the product of the
//                                         factor rows it touches, Sec. III-B)
//   T_n = HADAMARD_{p != n} B_p^T B_p   (Eq. 9; A_p^T A_p for the nonneg form)
//   B_n = H_n T_n^{-1}                  (Eq. 14 in core space; FP64 Cholesky,
//                                         pseudo-inverse on breakdown)
//   lambda = column norms, B_n scaled to unit columns, Gram_n refreshed
// then the fit from the Gram identities; the sweep loop runs on the device
// (captured once as a CUDA graph) and the host checks the done flag every
// `check_every` sweeps.  Nonnegative form: A_n = max(0, U_n H_n T_n^{-1}),
// B_n = U_n^T A_n (Eq. 13; P_+ of Eq. 8).
#include <chrono>
#include <cmath>

#include "tdk_internal.cuh"

namespace tdk {
namespace {

constexpr int RMAX = TDK_MAX_RANK;

struct AlsState {
  int sweep;
  int done;
  int status;  // TDK_WNOCONV / TDK_WPINV bits
  int converged;
  double fit;
  double fit_old;
  double fitY;
  double nG2;
  double nY2;
};

template <class T>
struct AlsArgs {
  int N, R, nonneg, max_sweeps;  // nonneg: the factors are updated as A_n (ambient rows)
  int nn_rule;                   // 0 LS solve, 1 HALS (Eq. 8), 2 multiplicative (Eq. 15)
  int clip;                      // project onto the nonnegative orthant (P_+)
  double l1;                     // > 0: soft threshold of the LS solution (Eq. 16)
  double tol;
  int64_t Rt[TDK_MAX_MODES];
  int64_t I[TDK_MAX_MODES];
  int64_t stride[TDK_MAX_MODES];  // strides of G (row-major)
  int64_t gnumel;
  const T* G;
  T* B[TDK_MAX_MODES];           // working core-space factors, [Rt_n x R]
  double* A[TDK_MAX_MODES];      // nonneg: current A_n [I_n x R] (normalised)
  const double* U[TDK_MAX_MODES];
  double* gram;                  // [N][R*R]
  double* lam;                   // [R]
  double* Bnew;                  // [max(Rt, I) x R] FP64 update before scaling
  double* Hfull;                 // [Rtmax x R] reduced H of the current mode
  T* Hpart;                      // [S][Rtmax x R]
  int S[TDK_MAX_MODES];          // partial count per mode
  int64_t chunk[TDK_MAX_MODES];  // entries per partial
  double* inner;                 // [R]
  double* hist;                  // [max_sweeps] fit history (capped)
  int hist_cap;
  AlsState* st;
  const double* normY2;
};

// ---------------------------------------------------------------- MTTKRP
template <class T>
__global__ void __launch_bounds__(256) als_mttkrp(AlsArgs<T> a, int n) {
  if (a.st->done) return;
  const int R = a.R;
  const int i = blockIdx.x;        // row of H_n
  const int s = blockIdx.y;        // partial index
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  extern __shared__ unsigned char sm_raw[];
  T* Bs = reinterpret_cast<T*>(sm_raw);  // all factors except n, packed
  __shared__ int64_t boff[TDK_MAX_MODES];
  __shared__ T red[8][RMAX];
  if (threadIdx.x == 0) {
    int64_t o = 0;
    for (int p = 0; p < a.N; ++p) {
      boff[p] = o;
      if (p != n) o += a.Rt[p] * R;
    }
  }
  __syncthreads();
  for (int p = 0; p < a.N; ++p) {
    if (p == n) continue;
    for (int e = threadIdx.x; e < a.Rt[p] * R; e += blockDim.x) Bs[boff[p] + e] = a.B[p][e];
  }
  __syncthreads();
  // the other-index space, row-major over p != n
  const int64_t Q = a.gnumel / a.Rt[n];
  const int64_t j0 = (int64_t)s * a.chunk[n];
  const int64_t j1 = (j0 + a.chunk[n] < Q) ? j0 + a.chunk[n] : Q;
  T acc0 = T(0), acc1 = T(0);
  for (int64_t jb = j0 + (int64_t)w * 32; jb < j1; jb += 8 * 32) {
    // lane decodes entry jb + lane
    int64_t j = jb + lane;
    int64_t goff = (int64_t)i * a.stride[n];
    int rowoff[TDK_MAX_MODES];
    bool valid = j < j1;
    {
      int64_t rem = valid ? j : 0;
      for (int p = a.N - 1; p >= 0; --p) {
        if (p == n) continue;
        int64_t ip = rem % a.Rt[p];
        rem /= a.Rt[p];
        goff += ip * a.stride[p];
        rowoff[p] = (int)(boff[p] + ip * R);
      }
    }
    T gv = valid ? a.G[goff] : T(0);
    const int cnt = (int)((j1 - jb) < 32 ? (j1 - jb) : 32);
    for (int e = 0; e < cnt; ++e) {
      T g = __shfl_sync(0xffffffffu, gv, e);
      T prod0 = g, prod1 = g;
      for (int p = 0; p < a.N; ++p) {
        if (p == n) continue;
        int ro = __shfl_sync(0xffffffffu, rowoff[p], e);
        if (lane < R) prod0 *= Bs[ro + lane];
        if (lane + 32 < R) prod1 *= Bs[ro + lane + 32];
      }
      acc0 += prod0;
      acc1 += prod1;
    }
  }
  if (lane < R) red[w][lane] = acc0;
  if (lane + 32 < R) red[w][lane + 32] = acc1;
  __syncthreads();
  if (threadIdx.x < R) {
    T v = T(0);
    for (int q = 0; q < 8; ++q) v += red[q][threadIdx.x];
    a.Hpart[((int64_t)s * RMAX + i) * R + threadIdx.x] = v;
  }
}

// ------------------------------------------------ FP64 R x R helpers (1 CTA)
// T = HADAMARD_{p != n} gram[p]; Cholesky in place (lower).  Returns 1 if a
// pivot is not above R * eps * max diag.
__device__ int build_and_cholesky(const double* gram, int N, int n, int R, double* Tm) {
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double v = 1.0;
    for (int p = 0; p < N; ++p)
      if (p != n) v *= gram[(int64_t)p * R * R + e];
    Tm[e] = v;
  }
  __syncthreads();
  double mx = 0.0;
  for (int j = 0; j < R; ++j) mx = fmax(mx, Tm[j * R + j]);
  const double tiny = R * 2.220446049250313e-16 * mx;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int j = 0; j < R; ++j) {
    __syncthreads();
    double d = Tm[j * R + j];
    if (!(d > tiny)) {
      if (threadIdx.x == 0) bad = 1;
      break;
    }
    double ljj = sqrt(d);
    __syncthreads();
    if (threadIdx.x == 0) Tm[j * R + j] = ljj;
    for (int r = j + 1 + threadIdx.x; r < R; r += blockDim.x) Tm[r * R + j] /= ljj;
    __syncthreads();
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      int r = e / R, c = e % R;
      if (c > j && r >= c) Tm[e] = fma(-Tm[r * R + j], Tm[c * R + j], Tm[e]);
    }
  }
  __syncthreads();
  int b = bad;
  __syncthreads();
  return b;
}

// x <- x T^{-1} using the Cholesky factor (lower L, T = L L^T); x in smem
__device__ void chol_solve_row(const double* L, int R, double* x) {
  for (int j = 0; j < R; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) x[j] /= L[j * R + j];
    __syncthreads();
    for (int r = j + 1 + threadIdx.x; r < R; r += blockDim.x) x[r] = fma(-L[r * R + j], x[j], x[r]);
  }
  for (int j = R - 1; j >= 0; --j) {
    __syncthreads();
    if (threadIdx.x == 0) x[j] /= L[j * R + j];
    __syncthreads();
    for (int r = threadIdx.x; r < j; r += blockDim.x) x[r] = fma(-L[j * R + r], x[j], x[r]);
  }
  __syncthreads();
}

// symmetric eigendecomposition by parallel cyclic Jacobi (round-robin pairs).
// A (R x R, smem) is destroyed (its diagonal holds the eigenvalues on exit);
// V (R x R, smem) receives the eigenvectors as columns.
__device__ void jacobi_eig(double* A, double* V, int R) {
  __shared__ double cs[RMAX / 2 + 1][2];
  __shared__ int pr[RMAX / 2 + 1][2];
  __shared__ int perm[RMAX + 1];
  __shared__ double off;
  const int Rp = R + (R & 1);  // even count, dummy index R when odd
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) V[e] = (e / R == e % R) ? 1.0 : 0.0;
  for (int e = threadIdx.x; e < Rp; e += blockDim.x) perm[e] = e;
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) {
      double o = 0.0, d = 0.0;
      for (int r = 0; r < R; ++r)
        for (int c = 0; c < R; ++c) {
          if (r != c) o += A[r * R + c] * A[r * R + c];
          else d += A[r * R + c] * A[r * R + c];
        }
      off = (o <= 1e-30 * d || o == 0.0) ? -1.0 : o;
    }
    __syncthreads();
    if (off < 0) break;
    for (int step = 0; step < Rp - 1; ++step) {
      // pairs (perm[k], perm[Rp-1-k])
      for (int k = threadIdx.x; k < Rp / 2; k += blockDim.x) {
        int p = perm[k], q = perm[Rp - 1 - k];
        if (p > q) { int tt = p; p = q; q = tt; }
        double c = 1.0, s = 0.0;
        if (q < R) {
          double apq = A[p * R + q];
          if (apq != 0.0) {
            double th = (A[q * R + q] - A[p * R + p]) / (2.0 * apq);
            double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pr[k][0] = p; pr[k][1] = q; cs[k][0] = c; cs[k][1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = threadIdx.x; e < (Rp / 2) * R; e += blockDim.x) {
        int k = e / R, col = e % R;
        int p = pr[k][0], q = pr[k][1];
        if (q >= R) continue;
        double c = cs[k][0], s = cs[k][1];
        double ap = A[p * R + col], aq = A[q * R + col];
        A[p * R + col] = c * ap - s * aq;
        A[q * R + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = threadIdx.x; e < (Rp / 2) * R; e += blockDim.x) {
        int k = e / R, row = e % R;
        int p = pr[k][0], q = pr[k][1];
        if (q >= R) continue;
        double c = cs[k][0], s = cs[k][1];
        double ap = A[row * R + p], aq = A[row * R + q];
        A[row * R + p] = c * ap - s * aq;
        A[row * R + q] = s * ap + c * aq;
        double vp = V[row * R + p], vq = V[row * R + q];
        V[row * R + p] = c * vp - s * vq;
        V[row * R + q] = s * vp + c * vq;
      }
      __syncthreads();
      if (threadIdx.x == 0) {  // rotate the round-robin schedule (keep perm[0])
        int lastv = perm[Rp - 1];
        for (int k = Rp - 1; k > 1; --k) perm[k] = perm[k - 1];
        perm[1] = lastv;
      }
      __syncthreads();
    }
  }
  __syncthreads();
}

// x <- x T^+ with T^+ from the eigendecomposition (cutoff R*eps*lambda_max);
// T is rebuilt from the Grams since the Cholesky attempt destroyed it.
__device__ void pinv_solve_row(const double* gram, int N, int n, int R, double* Tm, double* V,
                               double* x, double* tmp) {
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double v = 1.0;
    for (int p = 0; p < N; ++p)
      if (p != n) v *= gram[(int64_t)p * R * R + e];
    Tm[e] = v;
  }
  __syncthreads();
  jacobi_eig(Tm, V, R);
  double wmax = 0.0;
  for (int j = 0; j < R; ++j) wmax = fmax(wmax, Tm[j * R + j]);
  const double cut = R * 2.220446049250313e-16 * wmax;
  // tmp = x V, scaled by 1/w, then x = tmp V^T
  for (int j = threadIdx.x; j < R; j += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(x[k], V[k * R + j], s);
    double wj = Tm[j * R + j];
    tmp[j] = (wj > cut) ? s / wj : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < R; j += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < R; ++k) s = fma(tmp[k], V[j * R + k], s);
    x[j] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- solve
// unconstrained: one CTA per row i of B_n.  nonneg: one CTA per row i of A_n.
template <class T>
__global__ void __launch_bounds__(64) als_solve(AlsArgs<T> a, int n) {
  if (a.st->done) return;
  const int R = a.R;
  const int64_t Rtn = a.Rt[n];
  const int i = blockIdx.x;
  __shared__ double Tm[RMAX * RMAX];
  __shared__ double V[RMAX * RMAX];
  __shared__ double x[RMAX], tmp[RMAX];
  const double* gram = a.gram;
  if (a.nonneg && a.nn_rule != 0) {
    // HALS and multiplicative rules: T_n itself, the row of M = U_n H_n and
    // the current iterate of the row, A_n[i, :] diag(lambda)
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      double v = 1.0;
      for (int p = 0; p < a.N; ++p)
        if (p != n) v *= gram[(int64_t)p * R * R + e];
      Tm[e] = v;
    }
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      double m = 0.0;
      for (int64_t q = 0; q < Rtn; ++q) {
        double h = 0.0;
        for (int s = 0; s < a.S[n]; ++s) h += (double)a.Hpart[((int64_t)s * RMAX + q) * R + r];
        if (i == 0) a.Hfull[q * R + r] = h;
        m = fma(a.U[n][(int64_t)i * Rtn + q], h, m);
      }
      x[r] = m;
      tmp[r] = a.A[n][(int64_t)i * R + r] * a.lam[r];
    }
    __syncthreads();
    if (a.nn_rule == 2) {
      // multiplicative: a <- a (*) P_+(m) (/) (a T_n); 0 where a T_n is not positive
      for (int r = threadIdx.x; r < R; r += blockDim.x) {
        double d = 0.0;
        for (int q = 0; q < R; ++q) d = fma(tmp[q], Tm[q * R + r], d);
        a.Bnew[(int64_t)i * R + r] = d > 0.0 ? tmp[r] * fmax(x[r], 0.0) / d : 0.0;
      }
    } else if (threadIdx.x < 32) {
      // HALS, column by column: a_r <- P_+(a_r + (m_r - a t_r) / t_rr), each
      // column seeing the ones already updated (one warp; the row is short)
      for (int r = 0; r < R; ++r) {
        double part = 0.0;
        for (int q = threadIdx.x; q < R; q += 32) part = fma(tmp[q], Tm[q * R + r], part);
        part = warp_sum(part);
        if (threadIdx.x == 0) tmp[r] = fmax(0.0, tmp[r] + (x[r] - part) / Tm[r * R + r]);
        __syncwarp();
      }
      for (int r = threadIdx.x; r < R; r += 32) a.Bnew[(int64_t)i * R + r] = tmp[r];
    }
    return;
  }
  int bad = build_and_cholesky(gram, a.N, n, R, Tm);
  if (!a.nonneg) {
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      double h = 0.0;
      for (int s = 0; s < a.S[n]; ++s) h += (double)a.Hpart[((int64_t)s * RMAX + i) * R + r];
      x[r] = h;
      a.Hfull[(int64_t)i * R + r] = h;
    }
  } else {
    // m = U_n[i, :] H_n, H_n reduced from the partials on the fly
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      double m = 0.0;
      for (int64_t q = 0; q < Rtn; ++q) {
        double h = 0.0;
        for (int s = 0; s < a.S[n]; ++s) h += (double)a.Hpart[((int64_t)s * RMAX + q) * R + r];
        if (i == 0) a.Hfull[q * R + r] = h;
        m = fma(a.U[n][(int64_t)i * Rtn + q], h, m);
      }
      x[r] = m;
    }
  }
  __syncthreads();
  if (!bad) {
    chol_solve_row(Tm, R, x);
  } else {
    pinv_solve_row(gram, a.N, n, R, Tm, V, x, tmp);
    if (threadIdx.x == 0 && i == 0) atomicOr(&a.st->status, TDK_WPINV);
  }
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double v = x[r];
    if (a.l1 > 0.0) v = copysign(fmax(fabs(v) - a.l1, 0.0), v);
    if (a.clip) v = v > 0.0 ? v : 0.0;
    a.Bnew[(int64_t)i * R + r] = v;
  }
}

// ------------------------------------------------------------- normalise
// one CTA per column r.  rows = Rt_n (unconstrained) or I_n (nonneg).
// raw = 1: take Bnew as the new factor without scaling (initialisation).
template <class T>
__global__ void __launch_bounds__(128) als_normalize(AlsArgs<T> a, int n, int raw) {
  if (a.st->done) return;
  const int R = a.R;
  const int r = blockIdx.x;
  const int64_t rows = a.nonneg ? a.I[n] : a.Rt[n];
  const int64_t Rtn = a.Rt[n];
  __shared__ double lam[RMAX];
  __shared__ double red[4][RMAX];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // all column norms (redundantly per CTA)
  for (int c = 0; c < R; ++c) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
      double v = a.Bnew[i * R + c];
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) red[w][c] = s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    double s = red[0][c] + red[1][c] + red[2][c] + red[3][c];
    lam[c] = raw ? 1.0 : sqrt(s);
  }
  __syncthreads();
  const double inv_rows = 1.0 / sqrt((double)rows);
  // scaled value of (i, c): Bnew/lam, or the constant unit column when lam = 0
#define SCALED(i, c) (lam[c] > 0.0 ? a.Bnew[(i) * R + (c)] / lam[c] : inv_rows)
  // Gram row r
  for (int c = 0; c < R; ++c) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) s = fma(SCALED(i, r), SCALED(i, c), s);
    s = warp_sum(s);
    if (lane == 0) red[w][c] = s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += blockDim.x)
    a.gram[(int64_t)n * R * R + (int64_t)r * R + c] = red[0][c] + red[1][c] + red[2][c] + red[3][c];
  if (!a.nonneg) {
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) a.B[n][i * R + r] = (T)SCALED(i, r);
  } else {
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) a.A[n][i * R + r] = SCALED(i, r);
    // B_n[:, r] = U_n^T A_n[:, r]
    for (int64_t q = threadIdx.x; q < Rtn; q += blockDim.x) {
      double s = 0.0;
      for (int64_t i = 0; i < rows; ++i) s = fma(a.U[n][i * Rtn + q], SCALED(i, r), s);
      a.B[n][q * R + r] = (T)s;
    }
  }
#undef SCALED
  __syncthreads();
  // lambda of the model [[lambda; A]]: 1 for a raw start (the HALS and
  // multiplicative rules read it as the weights of the current iterate)
  if (r == 0)
    for (int c = threadIdx.x; c < R; c += blockDim.x) a.lam[c] = lam[c];
  if (n == a.N - 1 && !raw) {
    // inner = <G, [[lambda; B]]> = sum_{q, c} H[q, c] lambda_c B_n[q, c]  (column r)
    __syncthreads();
    double s = 0.0;
    for (int64_t q = threadIdx.x; q < Rtn; q += blockDim.x)
      s = fma(a.Hfull[q * R + r], (double)a.B[n][q * R + r] * lam[r], s);
    s = warp_sum(s);
    if (lane == 0) red[w][0] = s;
    __syncthreads();
    if (threadIdx.x == 0) a.inner[r] = red[0][0] + red[1][0] + red[2][0] + red[3][0];
  }
}

// ------------------------------------------------------------- fit / stop
template <class T>
__global__ void als_fit(AlsArgs<T> a) {
  if (a.st->done) return;
  const int R = a.R;
  __shared__ double red[2];
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int e = threadIdx.x; e < R * R; e += 32) {
      double v = a.lam[e / R] * a.lam[e % R];
      for (int p = 0; p < a.N; ++p) v *= a.gram[(int64_t)p * R * R + e];
      m += v;
    }
    m = warp_sum(m);
    double in = 0.0;
    for (int c = threadIdx.x; c < R; c += 32) in += a.inner[c];
    in = warp_sum(in);
    if (threadIdx.x == 0) { red[0] = m; red[1] = in; }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  AlsState* st = a.st;
  const double model2 = red[0], inner = red[1];
  const double res2 = fmax(0.0, st->nG2 - 2.0 * inner + model2);
  const double fit = 1.0 - sqrt(res2) / sqrt(st->nG2);
  if (st->nY2 > 0.0) st->fitY = 1.0 - sqrt(fmax(0.0, st->nY2 - 2.0 * inner + model2)) / sqrt(st->nY2);
  const int sw = st->sweep + 1;
  st->sweep = sw;
  if (sw - 1 < a.hist_cap) a.hist[sw - 1] = fit;
  st->fit_old = st->fit;
  st->fit = fit;
  if (sw > 1 && fabs(fit - st->fit_old) < a.tol * fabs(st->fit_old)) {
    st->done = 1;
    st->converged = 1;
  } else if (sw >= a.max_sweeps) {
    st->done = 1;
  }
}

template <class T>
__global__ void norm2_kernel(const T* __restrict__ G, int64_t n, AlsState* st, const double* nY2) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    double v = (double)G[e];
    s = fma(v, v, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    st->nG2 = v;
    st->nY2 = nY2 ? *nY2 : 0.0;
    st->sweep = 0;
    st->done = 0;
    st->status = 0;
    st->converged = 0;
    st->fit = 0.0;
    st->fit_old = 0.0;
    st->fitY = nan("");
  }
}

__global__ void copy_f64_kernel(const double* __restrict__ s, double* __restrict__ d, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = s[e];
}

// A_n = U_n B_n (FP64), lambda absorbed into the last factor
template <class T>
__global__ void lift_kernel(const double* __restrict__ U, const T* __restrict__ B, int64_t I, int64_t Rt, int R,
                            const double* __restrict__ lam, double* __restrict__ A, double* __restrict__ Bout,
                            const float* __restrict__ Uf = nullptr) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < I * R; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / R;
    int r = (int)(e % R);
    double s;
    if (sizeof(T) == 8) {
      s = 0.0;
      for (int64_t q = 0; q < Rt; ++q) s = fma(U[i * Rt + q], (double)B[q * R + r], s);
    } else {
      // FP32 factors B: the product in FP32 (U rounded to FP32 adds one
      // rounding of the same size as B's own), FP64 arithmetic being scarce;
      // from the FP32 copy of U when the caller has one (the conversions run
      // at the FP64 rate)
      float sf = 0.f;
      if (Uf)
        for (int64_t q = 0; q < Rt; ++q) sf = fmaf(Uf[i * Rt + q], (float)B[q * R + r], sf);
      else
        for (int64_t q = 0; q < Rt; ++q) sf = fmaf((float)U[i * Rt + q], (float)B[q * R + r], sf);
      s = (double)sf;
    }
    A[e] = lam ? s * lam[r] : s;
  }
  if (Bout)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Rt * R; e += (int64_t)gridDim.x * blockDim.x)
      Bout[e] = (double)B[e];
}

// one thread per entry of A_n, capped
static inline unsigned lift_grid(int64_t I, int R) {
  const int64_t b = (I * R + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

__global__ void scale_cols_kernel(const double* __restrict__ A, int64_t I, int R, const double* __restrict__ lam,
                                  double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < I * R; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = lam ? A[e] * lam[e % R] : A[e];
}

// HOSVD initialisation: eigenvectors of G_(n) G_(n)^T (Jacobi, FP64), the
// R leading ones, sign fixed so that the largest-magnitude entry is positive.
template <class T>
__global__ void __launch_bounds__(128) hosvd_init_kernel(AlsArgs<T> a, int n, double* Bout) {
  const int64_t Rt = a.Rt[n];
  const int R = a.R;
  __shared__ double M[RMAX * RMAX];
  __shared__ double V[RMAX * RMAX];
  __shared__ int order[RMAX];
  const int64_t Q = a.gnumel / Rt;
  for (int e = threadIdx.x; e < Rt * Rt; e += blockDim.x) {
    int64_t p = e / Rt, q = e % Rt;
    double s = 0.0;
    for (int64_t j = 0; j < Q; ++j) {
      // G_(n)[p, j] via the strides: decode j over modes != n
      int64_t rem = j, op = p * a.stride[n], oq = q * a.stride[n];
      for (int m = a.N - 1; m >= 0; --m) {
        if (m == n) continue;
        int64_t im = rem % a.Rt[m];
        rem /= a.Rt[m];
        op += im * a.stride[m];
        oq += im * a.stride[m];
      }
      s = fma((double)a.G[op], (double)a.G[oq], s);
    }
    M[e] = s;
  }
  __syncthreads();
  jacobi_eig(M, V, (int)Rt);
  if (threadIdx.x == 0) {
    // order by eigenvalue, descending (selection; Rt <= 64)
    bool used[RMAX];
    for (int k = 0; k < Rt; ++k) used[k] = false;
    for (int k = 0; k < R; ++k) {
      int best = -1;
      for (int c = 0; c < Rt; ++c)
        if (!used[c] && (best < 0 || M[c * Rt + c] > M[best * Rt + best])) best = c;
      used[best] = true;
      order[k] = best;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < R; k += blockDim.x) {
    int c = order[k];
    int arg = 0;
    double mx = -1.0;
    for (int p = 0; p < Rt; ++p)
      if (fabs(V[p * Rt + c]) > mx) { mx = fabs(V[p * Rt + c]); arg = p; }
    double sg = V[arg * Rt + c] < 0 ? -1.0 : 1.0;
    for (int p = 0; p < Rt; ++p) Bout[(int64_t)p * R + k] = sg * V[p * Rt + c];
  }
}

// |U_n B_n| as a nonnegative starting point
__global__ void abs_lift_kernel(const double* __restrict__ U, const double* __restrict__ B, int64_t I, int64_t Rt,
                                int R, double* __restrict__ A, bool take_abs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < I * R; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / R;
    int r = (int)(e % R);
    double s = 0.0;
    for (int64_t q = 0; q < Rt; ++q) s = fma(U[i * Rt + q], B[q * R + r], s);
    A[e] = take_abs ? fabs(s) : s;
  }
}

template <class T>
int als_run_t(tdk_ctx* ctx, const Geom& g, const T* G, const double* const U[], const double* normY2,
              const tdk_als_opts* o, double* const B_io[], double* const A_io[], double* lambda_out,
              tdk_als_report* rep) {
  auto t0 = std::chrono::steady_clock::now();
  const int N = g.N, R = o->R;
  AlsArgs<T> a{};
  a.N = N;
  a.R = R;
  // the l1 form updates the factors as A_n like the nonnegative forms
  a.nonneg = (o->nonneg || o->l1 > 0.0) ? 1 : 0;
  a.nn_rule = o->nonneg == TDK_NONNEG_HALS ? 1 : (o->nonneg == TDK_NONNEG_MU ? 2 : 0);
  a.clip = o->nonneg ? 1 : 0;
  a.l1 = o->l1;
  a.max_sweeps = o->max_sweeps;
  a.tol = o->tol;
  int64_t Rtmax = 0, Imax = 0, bsum = 0;
  for (int n = 0; n < N; ++n) {
    a.Rt[n] = g.Rt[n];
    a.I[n] = g.I[n];
    Rtmax = g.Rt[n] > Rtmax ? g.Rt[n] : Rtmax;
    Imax = g.I[n] > Imax ? g.I[n] : Imax;
    bsum += (int64_t)g.Rt[n] * R;
  }
  a.gnumel = g.core_numel;
  {
    int64_t s = 1;
    for (int n = N - 1; n >= 0; --n) {
      a.stride[n] = s;
      s *= g.Rt[n];
    }
  }
  int Smax = 1;
  for (int n = 0; n < N; ++n) {
    int64_t Q = g.core_numel / g.Rt[n];
    int S = (int)((2 * ctx->num_sms + g.Rt[n] - 1) / g.Rt[n]);
    int64_t minchunk = 2048;
    if ((Q + S - 1) / S < minchunk) S = (int)((Q + minchunk - 1) / minchunk);
    if (S < 1) S = 1;
    a.S[n] = S;
    a.chunk[n] = (Q + S - 1) / S;
    Smax = S > Smax ? S : Smax;
  }
  a.hist_cap = o->max_sweeps < 65536 ? o->max_sweeps : 65536;
  Planner pl;
  for (int n = 0; n < N; ++n) pl.take<T>((size_t)g.Rt[n] * R);
  if (a.nonneg)
    for (int n = 0; n < N; ++n) pl.take<double>((size_t)g.I[n] * R);
  pl.take<double>((size_t)N * R * R);
  pl.take<double>(R);
  pl.take<double>((size_t)(a.nonneg ? (Imax > Rtmax ? Imax : Rtmax) : Rtmax) * R);
  pl.take<double>((size_t)Rtmax * R);
  pl.take<T>((size_t)Smax * RMAX * R);
  pl.take<double>(R);
  pl.take<double>(a.hist_cap);
  pl.take<AlsState>(1);
  int rc = ws_reserve(ctx, pl.off);
  if (rc) return rc;
  Carver cv(ctx->ws);
  for (int n = 0; n < N; ++n) a.B[n] = cv.take<T>((size_t)g.Rt[n] * R);
  if (a.nonneg)
    for (int n = 0; n < N; ++n) a.A[n] = cv.take<double>((size_t)g.I[n] * R);
  a.gram = cv.take<double>((size_t)N * R * R);
  a.lam = cv.take<double>(R);
  a.Bnew = cv.take<double>((size_t)(a.nonneg ? (Imax > Rtmax ? Imax : Rtmax) : Rtmax) * R);
  a.Hfull = cv.take<double>((size_t)Rtmax * R);
  a.Hpart = cv.take<T>((size_t)Smax * RMAX * R);
  a.inner = cv.take<double>(R);
  a.hist = cv.take<double>(a.hist_cap);
  a.st = cv.take<AlsState>(1);
  a.G = G;
  for (int n = 0; n < N; ++n) a.U[n] = U[n];
  a.normY2 = normY2;
  // the sweep graph is captured on the context's private stream, fenced by
  // events against the caller's stream (which may be the legacy stream)
  cudaStream_t s = ctx->aux;
  TDK_CUDA_TRY(cudaEventRecord(ctx->ev_in, ctx->stream));
  TDK_CUDA_TRY(cudaStreamWaitEvent(s, ctx->ev_in, 0));

  norm2_kernel<T><<<1, 1024, 0, s>>>(G, g.core_numel, a.st, normY2);
  TDK_LAUNCH_CHECK(ctx);
  // ---- initial factors
  for (int n = 0; n < N; ++n) {
    const int64_t rows = a.nonneg ? g.I[n] : g.Rt[n];
    if (o->init == TDK_INIT_GIVEN) {
      const double* src = a.nonneg ? A_io[n] : B_io[n];
      copy_f64_kernel<<<64, 256, 0, s>>>(src, a.Bnew, rows * R);
      TDK_LAUNCH_CHECK(ctx);
    } else {
      hosvd_init_kernel<T><<<1, 128, 0, s>>>(a, n, a.nonneg ? a.Hfull : a.Bnew);
      TDK_LAUNCH_CHECK(ctx);
      if (a.nonneg) {
        abs_lift_kernel<<<64, 256, 0, s>>>(U[n], a.Hfull, g.I[n], g.Rt[n], R, a.Bnew, a.clip != 0);
        TDK_LAUNCH_CHECK(ctx);
      }
    }
    als_normalize<T><<<R, 128, 0, s>>>(a, n, 1);
    TDK_LAUNCH_CHECK(ctx);
  }
  // ---- one sweep, captured as a graph
  size_t bsm = sizeof(T) * (size_t)bsum;
  auto mk = als_mttkrp<T>;
  TDK_CUDA_TRY(cudaFuncSetAttribute(mk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  TDK_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int64_t launches_per_sweep = 0;
  for (int n = 0; n < N; ++n) {
    mk<<<dim3((unsigned)g.Rt[n], (unsigned)a.S[n]), 256, bsm, s>>>(a, n);
    als_solve<T><<<(unsigned)(a.nonneg ? g.I[n] : g.Rt[n]), 64, 0, s>>>(a, n);
    als_normalize<T><<<R, 128, 0, s>>>(a, n, 0);
    launches_per_sweep += 3;
  }
  als_fit<T><<<1, 64, 0, s>>>(a);
  launches_per_sweep += 1;
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (ce != cudaSuccess) {
    fprintf(stderr, "tdk: graph capture failed: %s\n", cudaGetErrorString(ce));
    return TDK_ECUDA;
  }
  TDK_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
  const int every = o->check_every > 0 ? o->check_every : 8;
  AlsState hs{};
  int launched = 0;
  int result = TDK_OK;
  while (true) {
    int batch = every;
    if (launched + batch > o->max_sweeps) batch = o->max_sweeps - launched;
    for (int b = 0; b < batch; ++b) {
      cudaError_t e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) {
        fprintf(stderr, "tdk: graph launch failed: %s\n", cudaGetErrorString(e));
        result = TDK_ECUDA;
        break;
      }
      ctx->launches += launches_per_sweep;
    }
    launched += batch;
    if (result) break;
    if (cudaMemcpyAsync(&hs, a.st, sizeof(AlsState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      result = TDK_ECUDA;
      break;
    }
    if (hs.done || launched >= o->max_sweeps) break;
    if (o->timeout_s > 0) {
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > o->timeout_s) {
        result = TDK_ETIMEOUT;
        break;
      }
    }
  }
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (result == TDK_ECUDA) return result;
  // ---- outputs
  for (int n = 0; n < N; ++n) {
    const double* lamp = (n == N - 1) ? a.lam : nullptr;
    if (!a.nonneg) {
      lift_kernel<T><<<lift_grid(g.I[n], R), 256, 0, s>>>(U[n], a.B[n], g.I[n], g.Rt[n], R, lamp, A_io[n], B_io[n]);
      TDK_LAUNCH_CHECK(ctx);
    } else {
      scale_cols_kernel<<<128, 256, 0, s>>>(a.A[n], g.I[n], R, lamp, A_io[n]);
      TDK_LAUNCH_CHECK(ctx);
      lift_kernel<T><<<1, 256, 0, s>>>(U[n], a.B[n], 0, g.Rt[n], R, nullptr, nullptr, B_io[n]);
      TDK_LAUNCH_CHECK(ctx);
    }
  }
  if (lambda_out) {
    copy_f64_kernel<<<1, 64, 0, s>>>(a.lam, lambda_out, R);
    TDK_LAUNCH_CHECK(ctx);
  }
  TDK_CUDA_TRY(cudaMemcpyAsync(&hs, a.st, sizeof(AlsState), cudaMemcpyDeviceToHost, s));
  TDK_CUDA_TRY(cudaStreamSynchronize(s));
  TDK_CUDA_TRY(cudaEventRecord(ctx->ev_out, s));
  TDK_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0));
  int status = result;
  if (status == TDK_OK) {
    if (!hs.converged) status |= TDK_WNOCONV;
    status |= (hs.status & TDK_WPINV);
  }
  if (rep) {
    rep->sweeps = hs.sweep;
    rep->status = status;
    rep->fit_core = hs.fit;
    rep->fit_Y = normY2 ? hs.fitY : nan("");
    rep->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rep->form = TDK_ALS_RAN_STEPS;
    rep->grid = 0;
  }
  return status;
}

}  // namespace

int als_finish(tdk_ctx* ctx, const Geom& g, int R, bool dbl, const void* const* Bw, const double* const* U,
               const double* lam, double* const* Aw, double* const* B_io, double* const* A_io, double* lambda_out,
               const float* const* Uf) {
  cudaStream_t s = ctx->stream;
  for (int n = 0; n < g.N; ++n) {
    const double* lamp = (n == g.N - 1) ? lam : nullptr;
    if (!Aw) {
      if (dbl)
        lift_kernel<double><<<lift_grid(g.I[n], R), 256, 0, s>>>(U[n], reinterpret_cast<const double*>(Bw[n]), g.I[n], g.Rt[n], R, lamp,
                                                A_io[n], B_io[n]);
      else
        lift_kernel<float><<<lift_grid(g.I[n], R), 256, 0, s>>>(U[n], reinterpret_cast<const float*>(Bw[n]), g.I[n], g.Rt[n], R, lamp,
                                               A_io[n], B_io[n], Uf ? Uf[n] : nullptr);
      TDK_LAUNCH_CHECK(ctx);
    } else {
      scale_cols_kernel<<<128, 256, 0, s>>>(Aw[n], g.I[n], R, lamp, A_io[n]);
      TDK_LAUNCH_CHECK(ctx);
      if (dbl)
        lift_kernel<double><<<1, 256, 0, s>>>(U[n], reinterpret_cast<const double*>(Bw[n]), 0, g.Rt[n], R, nullptr,
                                              nullptr, B_io[n]);
      else
        lift_kernel<float><<<1, 256, 0, s>>>(U[n], reinterpret_cast<const float*>(Bw[n]), 0, g.Rt[n], R, nullptr,
                                             nullptr, B_io[n]);
      TDK_LAUNCH_CHECK(ctx);
    }
  }
  if (lambda_out) {
    copy_f64_kernel<<<1, 64, 0, s>>>(lam, lambda_out, R);
    TDK_LAUNCH_CHECK(ctx);
  }
  return TDK_OK;
}

template <class T>
int als_persistent_t(tdk_ctx* ctx, const Geom& g, const T* G, const double* const U[], const double* normY2,
                     const tdk_als_opts* o, double* const B_io[], double* const A_io[], double* lambda_out,
                     tdk_als_report* rep);

// HOSVD start written into the caller's B_io (nonnegative form: |U_n B_n|
// into A_io), on the context's stream, so that either ALS form can then
// start from it as a given initialisation
template <class T>
int hosvd_into(tdk_ctx* ctx, const Geom& g, const T* G, const double* const U[], const tdk_als_opts* o,
               double* const B_io[], double* const A_io[]) {
  AlsArgs<T> a{};
  a.N = g.N;
  a.R = o->R;
  int64_t Rtmax = 0, s = 1;
  for (int n = g.N - 1; n >= 0; --n) {
    a.Rt[n] = g.Rt[n];
    a.I[n] = g.I[n];
    a.stride[n] = s;
    s *= g.Rt[n];
    Rtmax = g.Rt[n] > Rtmax ? g.Rt[n] : Rtmax;
  }
  a.gnumel = g.core_numel;
  a.G = G;
  // factors updated as A_n (nonneg, l1): the start lifted, A_n = U_n B_n
  // (its magnitudes for the nonnegative forms)
  const bool ambient = o->nonneg || o->l1 > 0.0;
  double* tmp = nullptr;
  if (ambient) {
    int rc = ws_reserve(ctx, sizeof(double) * (size_t)Rtmax * o->R + 256);
    if (rc) return rc;
    tmp = reinterpret_cast<double*>(ctx->ws);
  }
  for (int n = 0; n < g.N; ++n) {
    hosvd_init_kernel<T><<<1, 128, 0, ctx->stream>>>(a, n, ambient ? tmp : B_io[n]);
    TDK_LAUNCH_CHECK(ctx);
    if (ambient) {
      abs_lift_kernel<<<64, 256, 0, ctx->stream>>>(U[n], tmp, g.I[n], g.Rt[n], o->R, A_io[n], o->nonneg != 0);
      TDK_LAUNCH_CHECK(ctx);
    }
  }
  return TDK_OK;
}

int als_run(tdk_ctx* ctx, const Geom& g, int dtype, const void* G, const double* const U[], const double* normY2,
            const tdk_als_opts* o_in, double* const B_io[], double* const A_io[], double* lambda_out,
            tdk_als_report* rep) {
  // one persistent cooperative kernel when the core fits; otherwise (or when a
  // normal equation needs the pseudo-inverse) the kernel-per-step form.  A
  // HOSVD start is computed first and handed to either form as a given start.
  tdk_als_opts oo = *o_in;
  const tdk_als_opts* o = &oo;
  const bool steps = oo.form == TDK_ALS_FORM_STEPS;
  if (oo.init == TDK_INIT_HOSVD && !steps && !(oo.timeout_s > 0)) {
    const int rc0 = (dtype == TDK_F64) ? hosvd_into<double>(ctx, g, reinterpret_cast<const double*>(G), U, o, B_io, A_io)
                                       : hosvd_into<float>(ctx, g, reinterpret_cast<const float*>(G), U, o, B_io, A_io);
    if (rc0) return rc0;
    oo.init = TDK_INIT_GIVEN;
  }
  int rc = TDK_ENOTSUP;
  if (!steps) {
    rc = (dtype == TDK_F64)
             ? als_persistent_t<double>(ctx, g, reinterpret_cast<const double*>(G), U, normY2, o, B_io, A_io,
                                        lambda_out, rep)
             : als_persistent_t<float>(ctx, g, reinterpret_cast<const float*>(G), U, normY2, o, B_io, A_io,
                                       lambda_out, rep);
  }
  if (rc != TDK_ENOTSUP) return rc;
  if (dtype == TDK_F64)
    return als_run_t<double>(ctx, g, reinterpret_cast<const double*>(G), U, normY2, o, B_io, A_io, lambda_out, rep);
  return als_run_t<float>(ctx, g, reinterpret_cast<const float*>(G), U, normY2, o, B_io, A_io, lambda_out, rep);
}

}  // namespace tdk

namespace tdk {
TDK_CHECKED_UNIT(als)
}  // namespace tdk
