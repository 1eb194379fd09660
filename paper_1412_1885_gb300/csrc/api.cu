// C-ABI entry points of libtdk.so: argument validation, workspace, dispatch.
#include <cmath>
#include <cstring>

#include "tdk_internal.cuh"

namespace tdk {

int ws_reserve(tdk_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_size) return TDK_OK;
#ifdef TDK_TESTING
  if (ctx->fail_alloc_after == 0) return TDK_ENOMEM;
  if (ctx->fail_alloc_after > 0) ctx->fail_alloc_after--;
#endif
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
  }
  size_t want = bytes + bytes / 8 + (1 << 20);
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return TDK_ENOMEM;
  }
  ctx->ws_size = want;
  return TDK_OK;
}

// A stream-ordered allocation from the context's own pool, whose release
// threshold keeps freed memory for the next call: with the device's default
// pool (threshold 0) every call paid about 100 us of host time to map its
// buffers again after a synchronisation.
int pool_alloc(tdk_ctx* ctx, void** p, size_t bytes) {
  const cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream)
                                  : cudaMallocAsync(p, bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return TDK_ENOMEM;
  }
  return TDK_OK;
}

// geometry of a descriptor; the rule R_n + p <= I_n is checked against
// i1_check for the first mode (a slab of a tensor whose first dimension is
// i1_check may hold fewer rows than the sketch width)
static int make_geom_checked(const tdk_tucker_desc* d, int64_t i1_check, Geom* g) {
  if (!d || !g) return TDK_EINVAL;
  if (d->N < 2 || d->N > TDK_MAX_MODES) return TDK_EINVAL;
  if (d->dtype != TDK_F64 && d->dtype != TDK_F32 && d->dtype != TDK_BF16) return TDK_EINVAL;
  if (d->prec != TDK_PREC_SIMT && d->prec != TDK_PREC_TC) return TDK_EINVAL;
  if (d->p < 0) return TDK_EINVAL;
  g->N = d->N;
  g->numel = 1;
  g->core_numel = 1;
  g->zoff[0] = 0;
  for (int n = 0; n < d->N; ++n) {
    if (d->I[n] < 1 || d->R[n] < 1) return TDK_EINVAL;
    int64_t rt = (int64_t)d->R[n] + d->p;
    if (rt > TDK_MAX_RANK || rt > (n == 0 ? i1_check : d->I[n])) return TDK_EINVAL;
    g->I[n] = d->I[n];
    g->Rt[n] = (int)rt;
    if (g->numel > (((int64_t)1 << 62) / d->I[n])) return TDK_EINVAL;
    g->numel *= d->I[n];
    g->core_numel *= rt;
    g->zoff[n + 1] = g->zoff[n] + d->I[n] * rt;
  }
  g->L = d->I[d->N - 1];
  g->M = g->numel / g->L;
  return TDK_OK;
}

int make_geom(const tdk_tucker_desc* d, Geom* g) { return make_geom_checked(d, d ? d->I[0] : 0, g); }

// geometry of a slab of rows of mode 1 (the sharded form)
static int make_geom_slab(const tdk_tucker_desc* d, int64_t row_off, int64_t I1_total, Geom* g) {
  if (!d || row_off < 0 || I1_total < 1 || d->I[0] < 1 || d->I[0] > I1_total - row_off) return TDK_EINVAL;
  return make_geom_checked(d, I1_total, g);
}

// W_k^(n) drawn from the seed into one stream-ordered allocation: rows
// [row0[k], row0[k] + rows[k]) of every W_k^(n); ptrs[n*N + k] point into it
static int seeded_w(tdk_ctx* ctx, const Geom& g, uint64_t seed, const int64_t* rows, const int64_t* row0,
                    double** buf, const double** ptrs) {
  size_t total = 0;
  for (int n = 0; n < g.N; ++n)
    for (int k = 0; k < g.N; ++k)
      if (k != n) total += (size_t)rows[k] * g.Rt[n];
  *buf = nullptr;
  if (pool_alloc(ctx, (void**)buf, sizeof(double) * total)) return TDK_ENOMEM;
  double* mats[TDK_MAX_MODES * TDK_MAX_MODES] = {};
  size_t off = 0;
  for (int n = 0; n < g.N; ++n)
    for (int k = 0; k < g.N; ++k) {
      ptrs[n * g.N + k] = nullptr;
      if (k == n) continue;
      mats[n * g.N + k] = *buf + off;
      ptrs[n * g.N + k] = *buf + off;
      off += (size_t)rows[k] * g.Rt[n];
    }
  const int rc = draw_sketch_matrices(ctx, g.N, rows, row0, g.Rt, seed, mats);
  if (rc) {
    cudaFreeAsync(*buf, ctx->stream);
    *buf = nullptr;
  }
  return rc;
}

// the sketch pass alone: Z_n of every mode, packed by zoff, into a
// stream-ordered allocation that the caller frees (Z stays out of the
// workspace, which the sub-steps carve)
static int sketch_pass(tdk_ctx* ctx, const Geom& g, const tdk_tucker_desc* desc, const void* Y,
                       const double* const W[], double** Zout, double* normY2) {
  double* Z = nullptr;
  if (pool_alloc(ctx, (void**)&Z, sizeof(double) * (size_t)g.zoff[g.N])) return TDK_ENOMEM;
  int rc = desc->prec == TDK_PREC_TC ? sketch_tc(ctx, g, desc->dtype, Y, W, Z, normY2)
                                     : sketch_simt(ctx, g, desc->dtype, Y, W, Z);
  if (rc == TDK_OK && normY2 && desc->prec != TDK_PREC_TC) rc = norm2_pass(ctx, g, desc->dtype, Y, normY2);
  if (rc) {
    cudaFreeAsync(Z, ctx->stream);
    return rc;
  }
  *Zout = Z;
  return TDK_OK;
}

}  // namespace tdk

#ifdef TDK_CHECKED
namespace tdk {
// the check words of every translation unit (checked build)
int tdk_chk_take_als(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_als_persistent(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_api(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_cholqr(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_core_simt(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_mlp(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_mlp_gemm(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_refine(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_rng(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_sketch_simt(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_tc_core(cudaStream_t, unsigned*, unsigned*);
int tdk_chk_take_tc_sketch(cudaStream_t, unsigned*, unsigned*);

// OR of every unit's bounds-check word; the first failure of each unit is
// reported on stderr with its source line
static unsigned checked_take_all(cudaStream_t s) {
  struct Unit {
    const char* name;
    int (*take)(cudaStream_t, unsigned*, unsigned*);
  };
  static const Unit units[] = {{"als.cu", tdk_chk_take_als},
                               {"als_persistent.cu", tdk_chk_take_als_persistent},
                               {"api.cu", tdk_chk_take_api},
                               {"cholqr.cu", tdk_chk_take_cholqr},
                               {"core_simt.cu", tdk_chk_take_core_simt},
                               {"mlp.cu", tdk_chk_take_mlp},
                               {"mlp_gemm.cu", tdk_chk_take_mlp_gemm},
                               {"refine.cu", tdk_chk_take_refine},
                               {"rng.cu", tdk_chk_take_rng},
                               {"sketch_simt.cu", tdk_chk_take_sketch_simt},
                               {"tc_core.cu", tdk_chk_take_tc_core},
                               {"tc_sketch.cu", tdk_chk_take_tc_sketch}};
  unsigned any = 0;
  for (const Unit& u : units) {
    unsigned w = 0, l = 0;
    if (u.take(s, &w, &l) != 0) continue;
    if (w) {
      fprintf(stderr, "tdk: bounds check failed in %s, line %u\n", u.name, l);
      any = TDK_STATUS_OOB;
    }
  }
  return any;
}
}  // namespace tdk
#endif

namespace tdk {
namespace {
constexpr size_t PULL_MIN_BYTES = (size_t)1 << 26;  // 64 MiB
// dst[i] = src[i] for 16-byte words, src in page-locked host memory seen
// through its device mapping; four loads in flight per thread
__global__ void __launch_bounds__(512) pull_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                   int64_t n16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += 4 * stride) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i + u * stride < n16) v[u] = __ldg(src + i + u * stride);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i + u * stride < n16 && TDK_IN(i + u * stride, n16)) dst[i + u * stride] = v[u];
  }
}
}  // namespace
}  // namespace tdk

#ifdef TDK_TESTING
namespace tdk {
namespace {
// one store guarded by the checked build's bounds check: index outside
// [0, n) is reported and skipped, never performed
__global__ void checked_store_kernel(int* buf, long long index, long long n) {
  if (TDK_IN(index, n)) buf[index] = 1;
}
}  // namespace
}  // namespace tdk
#endif

using namespace tdk;

extern "C" {

int tdk_tucker_check(const tdk_tucker_desc* desc) {
  Geom g;
  return make_geom(desc, &g);
}

const char* tdk_strerror(int code) {
  switch (code) {
    case TDK_OK: return "ok";
    case TDK_EINVAL: return "invalid argument or configuration";
    case TDK_ENOMEM: return "workspace allocation failed";
    case TDK_ECUDA: return "CUDA call failed";
    case TDK_ETIMEOUT: return "bounded wait or time limit exceeded";
    case TDK_ENOTSUP: return "not supported for this configuration";
    case TDK_ESCRATCH: return "problem exceeds the static scratch array (TDK_SKETCH_STATIC_MAX_BYTES)";
    case TDK_EIO: return "file could not be read or written, or does not hold what the call expects";
    case TDK_WRANKDEF: return "warning: rank-deficient sketch completed";
    case TDK_WNOCONV: return "warning: ALS stopped at max_sweeps";
    case TDK_WPINV: return "warning: pseudo-inverse used in an ALS solve";
  }
  if (code > 0) return "warning (several bits)";
  return "unknown error";
}

int tdk_ctx_create(tdk_ctx** out, int device, void* stream) {
  if (!out) return TDK_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return TDK_ECUDA;
  }
  TDK_CUDA_TRY(cudaSetDevice(device));
  tdk_ctx* c = new tdk_ctx();
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (cudaMalloc(&c->d_status, sizeof(unsigned) * 4) != cudaSuccess) {
    delete c;
    return TDK_ENOMEM;
  }
  cudaMemset(c->d_status, 0, sizeof(unsigned) * 4);
  {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      c->pool = nullptr;  // the device's default pool then
    }
  }
  if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->d_status);
    delete c;
    return TDK_ECUDA;
  }
  *out = c;
  return TDK_OK;
}

int tdk_ctx_destroy(tdk_ctx* c) {
  if (!c) return TDK_EINVAL;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->ws) cudaFree(c->ws);
  if (c->aux) cudaStreamSynchronize(c->aux);
  if (c->d_status) cudaFree(c->d_status);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->pool) cudaMemPoolDestroy(c->pool);
  delete c;
  return TDK_OK;
}

int tdk_ctx_set_stream(tdk_ctx* c, void* stream) {
  if (!c) return TDK_EINVAL;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  return TDK_OK;
}

int tdk_ctx_sync_status(tdk_ctx* c, int* flags_out) {
  if (!c) return TDK_EINVAL;
  cudaSetDevice(c->device);
  unsigned h = 0;
  TDK_CUDA_TRY(cudaMemcpyAsync(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  TDK_CUDA_TRY(cudaStreamSynchronize(c->stream));
  TDK_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream));
  TDK_CUDA_TRY(cudaStreamSynchronize(c->stream));
#ifdef TDK_CHECKED
  h |= checked_take_all(c->stream);
#endif
  if (flags_out) *flags_out = (int)h;
  return TDK_OK;
}

int64_t tdk_ctx_launch_count(const tdk_ctx* c) { return c ? c->launches : -1; }

int tdk_copy_in(tdk_ctx* c, void* dst, const void* src_host, size_t bytes) {
  if (!c || (bytes && (!dst || !src_host))) return TDK_EINVAL;
  if (!bytes) return TDK_OK;
  cudaSetDevice(c->device);
  // page-locked source: the SMs pull it through its mapped device address
  // (GB300: about 210 GB/s against 140-180 for the copy engine); the rest
  // and pageable sources go through the copy engine
  cudaPointerAttributes at{};
  const bool pinned = cudaPointerGetAttributes(&at, src_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                      at.devicePointer != nullptr;
  cudaGetLastError();
  size_t done = 0;
  if (pinned && bytes >= PULL_MIN_BYTES && ((reinterpret_cast<uintptr_t>(at.devicePointer) |
                                             reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const int64_t n16 = (int64_t)(bytes / 16);
    pull_kernel<<<2 * c->num_sms, 512, 0, c->stream>>>(static_cast<const uint4*>(at.devicePointer),
                                                       static_cast<uint4*>(dst), n16);
    TDK_LAUNCH_CHECK(c);
    done = (size_t)n16 * 16;
  }
  if (done < bytes)
    TDK_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(dst) + done, static_cast<const char*>(src_host) + done,
                                 bytes - done, cudaMemcpyHostToDevice, c->stream));
  return TDK_OK;
}

int tdk_copy_out(tdk_ctx* c, void* dst_host, const void* src, size_t bytes) {
  if (!c || (bytes && (!dst_host || !src))) return TDK_EINVAL;
  if (!bytes) return TDK_OK;
  cudaSetDevice(c->device);
  TDK_CUDA_TRY(cudaMemcpyAsync(dst_host, src, bytes, cudaMemcpyDeviceToHost, c->stream));
  TDK_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return TDK_OK;
}

static void prof_drain(tdk_ctx* c, int r) {
  auto& v = c->prof_ev[r];
  for (size_t i = 0; i + 1 < v.size(); i += 2) {
    float ms = 0.f;
    if (cudaEventSynchronize(v[i + 1]) == cudaSuccess && cudaEventElapsedTime(&ms, v[i], v[i + 1]) == cudaSuccess) {
      c->prof_ms[r] += ms;
      c->prof_n[r] += 1;
    }
    cudaEventDestroy(v[i]);
    cudaEventDestroy(v[i + 1]);
  }
  v.clear();
}

int tdk_ctx_profile(tdk_ctx* c, int enable) {
  if (!c) return TDK_EINVAL;
  for (int r = 0; r < 2; ++r) {
    prof_drain(c, r);
    c->prof_ms[r] = 0.0;
    c->prof_n[r] = 0;
  }
  c->prof = enable != 0;
  return TDK_OK;
}

int tdk_ctx_profile_read(tdk_ctx* c, int region, double* total_ms, int64_t* launches) {
  if (!c || region < 0 || region > 1) return TDK_EINVAL;
  prof_drain(c, region);
  if (total_ms) *total_ms = c->prof_ms[region];
  if (launches) *launches = c->prof_n[region];
  return TDK_OK;
}

size_t tdk_ctx_workspace_bytes(const tdk_ctx* c) { return c ? c->ws_size : 0; }

#ifdef TDK_TESTING
// test library only: exercise the bounds-check reporting with one guarded
// store into a fresh n-element buffer (index outside it sets the OOB bit)
int tdk_test_checked_store(tdk_ctx* c, long long index, long long n) {
  if (!c || n < 1 || n > (1 << 20)) return TDK_EINVAL;
  cudaSetDevice(c->device);
  int* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, sizeof(int) * (size_t)n, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return TDK_ENOMEM;
  }
  tdk::checked_store_kernel<<<1, 1, 0, c->stream>>>(buf, index, n);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(buf, c->stream);
  c->launches++;
  return e == cudaSuccess ? TDK_OK : TDK_ECUDA;
}

// test library only (not in the public header): make the n-th workspace
// growth fail (after = 0: the next one; -1: none)
int tdk_ctx_test_fail_alloc(tdk_ctx* c, int after) {
  if (!c) return TDK_EINVAL;
  c->fail_alloc_after = after;
  return TDK_OK;
}
#endif

int tucker_sketch(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
                  double* const U_out[], double* const Z_out[], double* normY2) {
  if (!ctx || !desc || !Y || !U_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n) {
    if (!U_out[n]) return TDK_EINVAL;
    for (int k = 0; k < g.N; ++k)
      if (W && k != n && !W[n * g.N + k]) return TDK_EINVAL;
  }
  if (desc->prec == TDK_PREC_TC && desc->dtype == TDK_F64) return TDK_ENOTSUP;
  TDK_HMARK("tucker_sketch: entry");
  cudaSetDevice(ctx->device);
  double* wbuf = nullptr;
  const double* wp[TDK_MAX_MODES * TDK_MAX_MODES];
  if (!W) {
    int64_t row0[TDK_MAX_MODES] = {};
    rc = seeded_w(ctx, g, desc->seed, g.I, row0, &wbuf, wp);
    if (rc) return rc;
    W = wp;
  }
  double* Z = nullptr;
  rc = sketch_pass(ctx, g, desc, Y, W, &Z, normY2);
  TDK_HMARK("tucker_sketch: sketch pass queued");
  if (rc == TDK_OK) rc = cholqr2(ctx, g, Z, U_out);
  TDK_HMARK("tucker_sketch: CholQR2 queued");
  if (rc == TDK_OK && Z_out) {
    for (int n = 0; n < g.N; ++n)
      if (Z_out[n]) {
        if (cudaMemcpyAsync(Z_out[n], Z + g.zoff[n], sizeof(double) * g.I[n] * g.Rt[n],
                            cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
          rc = TDK_ECUDA;
      }
  }
  if (Z) cudaFreeAsync(Z, ctx->stream);
  if (wbuf) cudaFreeAsync(wbuf, ctx->stream);
  return rc;
}

int tucker_sketch_partial(tdk_ctx* ctx, const tdk_tucker_desc* slab, int64_t row_off, int64_t I1_total,
                          const void* Y, const double* const W[], double* const Z_out[]) {
  if (!ctx || !slab || !Y || !Z_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom_slab(slab, row_off, I1_total, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n) {
    if (!Z_out[n]) return TDK_EINVAL;
    for (int k = 0; k < g.N; ++k)
      if (W && k != n && !W[n * g.N + k]) return TDK_EINVAL;
  }
  if (slab->prec == TDK_PREC_TC && slab->dtype == TDK_F64) return TDK_ENOTSUP;
  cudaSetDevice(ctx->device);
  double* wbuf = nullptr;
  const double* wp[TDK_MAX_MODES * TDK_MAX_MODES];
  if (!W) {
    int64_t row0[TDK_MAX_MODES] = {};
    row0[0] = row_off;  // the slab's rows of every W_1^(n), at their global index
    rc = seeded_w(ctx, g, slab->seed, g.I, row0, &wbuf, wp);
    if (rc) return rc;
  } else {
    // the slab's rows of W_1^(n): Z_n (n >= 2) sums Eq. 22's products over
    // the slab's i_1 only, and Z_1's rows are the slab's own
    for (int n = 0; n < g.N; ++n)
      for (int k = 0; k < g.N; ++k)
        wp[n * g.N + k] = (k == n) ? nullptr : (k == 0 ? W[n * g.N] + row_off * g.Rt[n] : W[n * g.N + k]);
  }
  double* Z = nullptr;
  rc = sketch_pass(ctx, g, slab, Y, wp, &Z, nullptr);
  if (rc == TDK_OK)
    for (int n = 0; n < g.N; ++n)
      if (cudaMemcpyAsync(Z_out[n], Z + g.zoff[n], sizeof(double) * g.I[n] * g.Rt[n], cudaMemcpyDeviceToDevice,
                          ctx->stream) != cudaSuccess)
        rc = TDK_ECUDA;
  if (Z) cudaFreeAsync(Z, ctx->stream);
  if (wbuf) cudaFreeAsync(wbuf, ctx->stream);
  return rc;
}

int tucker_core_partial(tdk_ctx* ctx, const tdk_tucker_desc* slab, int64_t I1_total, const void* Y,
                        const double* const U[], void* G_out, double* normY2) {
  if (!ctx || !slab || !Y || !U || !G_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom_slab(slab, 0, I1_total, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n)
    if (!U[n]) return TDK_EINVAL;
  if (slab->prec == TDK_PREC_TC && slab->dtype == TDK_F64) return TDK_ENOTSUP;
  cudaSetDevice(ctx->device);
  if (slab->prec == TDK_PREC_TC) return core_tc(ctx, g, slab->dtype, Y, U, G_out, normY2);
  return core_simt(ctx, g, slab->dtype, Y, U, G_out, normY2);
}

int tdk_gram(tdk_ctx* ctx, const double* Z, int64_t rows, int cols, double* gram_out) {
  if (!ctx || !Z || !gram_out || rows < 1 || cols < 1 || cols > TDK_MAX_RANK) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  return gram_one(ctx, Z, rows, cols, gram_out);
}

int tdk_orth_apply(tdk_ctx* ctx, const double* gram, const double* Z, int64_t rows, int cols, double* Q_out) {
  if (!ctx || !gram || !Z || !Q_out || rows < 1 || cols < 1 || cols > TDK_MAX_RANK) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  return orth_apply_one(ctx, gram, Z, rows, cols, Q_out);
}

int tdk_orth(tdk_ctx* ctx, const double* Z, int64_t rows, int cols, double* U_out) {
  if (!ctx || !Z || !U_out || cols < 1 || cols > TDK_MAX_RANK || rows < cols) return TDK_EINVAL;
  cudaSetDevice(ctx->device);
  Geom g{};
  g.N = 1;
  g.I[0] = rows;
  g.Rt[0] = cols;
  g.zoff[0] = 0;
  g.zoff[1] = rows * cols;
  double* const dst[1] = {U_out};
  return cholqr2(ctx, g, Z, dst);
}

int tucker_refine(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
                  double* const U_io[]) {
  if (!ctx || !desc || !Y || !U_io) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n) {
    if (!U_io[n]) return TDK_EINVAL;
    for (int k = 0; k < g.N; ++k)
      if (W && k != n && !W[n * g.N + k]) return TDK_EINVAL;
  }
  if (desc->prec == TDK_PREC_TC && desc->dtype == TDK_F64) return TDK_ENOTSUP;
  cudaSetDevice(ctx->device);
  double* wbuf = nullptr;
  const double* wp[TDK_MAX_MODES * TDK_MAX_MODES];
  if (!W) {
    // the pass matrices are Rt_k x Rt_n: the first Rt_k rows of the seed's draw
    int64_t rows[TDK_MAX_MODES], row0[TDK_MAX_MODES] = {};
    for (int n = 0; n < g.N; ++n) rows[n] = g.Rt[n];
    rc = seeded_w(ctx, g, desc->seed, rows, row0, &wbuf, wp);
    if (rc) return rc;
    W = wp;
  }
  rc = refine_pass(ctx, g, desc->dtype, desc->prec, Y, W, U_io);
  if (wbuf) cudaFreeAsync(wbuf, ctx->stream);
  return rc;
}

int tucker_seq(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
               double* const U_out[], void* G_out, double* normY2) {
  if (!ctx || !desc || !Y || !U_out || !G_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n) {
    if (!U_out[n]) return TDK_EINVAL;
    for (int k = 0; k < g.N; ++k)
      if (W && k != n && !W[n * g.N + k]) return TDK_EINVAL;
  }
  if (desc->prec == TDK_PREC_TC && desc->dtype == TDK_F64) return TDK_ENOTSUP;
  cudaSetDevice(ctx->device);
  double* wbuf = nullptr;
  const double* wp[TDK_MAX_MODES * TDK_MAX_MODES];
  if (!W) {
    // the one-pass sketch's draw; a shrunk mode k reads the first Rt_k rows
    int64_t row0[TDK_MAX_MODES] = {};
    rc = seeded_w(ctx, g, desc->seed, g.I, row0, &wbuf, wp);
    if (rc) return rc;
    W = wp;
  }
  rc = seq_tucker(ctx, g, desc, Y, W, U_out, G_out, normY2);
  if (wbuf) cudaFreeAsync(wbuf, ctx->stream);
  return rc;
}

int tucker_core(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const U[], void* G_out,
                double* normY2) {
  if (!ctx || !desc || !Y || !U || !G_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n)
    if (!U[n]) return TDK_EINVAL;
  if (desc->prec == TDK_PREC_TC && desc->dtype == TDK_F64) return TDK_ENOTSUP;
  cudaSetDevice(ctx->device);
  if (desc->prec == TDK_PREC_TC) return core_tc(ctx, g, desc->dtype, Y, U, G_out, normY2);
  return core_simt(ctx, g, desc->dtype, Y, U, G_out, normY2);
}

int ffcp_als(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* G, const double* const U[],
             const double* normY2, const tdk_als_opts* opts, double* const B_io[], double* const A_io[],
             double* lambda_out, tdk_als_report* rep) {
  if (!ctx || !desc || !G || !U || !opts || !B_io || !A_io) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  if (opts->R < 1 || opts->R > TDK_MAX_RANK || opts->max_sweeps < 1 || !(opts->tol >= 0.0)) return TDK_EINVAL;
  if (opts->init != TDK_INIT_GIVEN && opts->init != TDK_INIT_HOSVD) return TDK_EINVAL;
  if (opts->nonneg < TDK_NONNEG_NONE || opts->nonneg > TDK_NONNEG_MU) return TDK_EINVAL;
  if (!(opts->l1 >= 0.0) || opts->l1 > 1e300) return TDK_EINVAL;
  if (opts->l1 > 0.0 && opts->nonneg > TDK_NONNEG_LS) return TDK_EINVAL;
  if (opts->form != TDK_ALS_FORM_AUTO && opts->form != TDK_ALS_FORM_STEPS) return TDK_EINVAL;
  for (int n = 0; n < g.N; ++n) {
    if (opts->R > g.Rt[n]) return TDK_EINVAL;
    if (!U[n] || !B_io[n] || !A_io[n]) return TDK_EINVAL;
  }
  cudaSetDevice(ctx->device);
  return als_run(ctx, g, desc->dtype, G, U, normY2, opts, B_io, A_io, lambda_out, rep);
}

}  // extern "C"

namespace tdk {
TDK_CHECKED_UNIT(api)
}  // namespace tdk
