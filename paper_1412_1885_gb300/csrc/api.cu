// C-ABI entry points of libtdk.so: argument validation, workspace, dispatch.
#include <cmath>
#include <cstring>

#include "tdk_internal.cuh"

namespace tdk {

int ws_reserve(tdk_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_size) return TDK_OK;
  if (ctx->fail_alloc_after == 0) return TDK_ENOMEM;
  if (ctx->fail_alloc_after > 0) ctx->fail_alloc_after--;
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

int make_geom(const tdk_tucker_desc* d, Geom* g) {
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
    if (rt > TDK_MAX_RANK || rt > d->I[n]) return TDK_EINVAL;
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

}  // namespace tdk

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
  if (flags_out) *flags_out = (int)h;
  return TDK_OK;
}

int64_t tdk_ctx_launch_count(const tdk_ctx* c) { return c ? c->launches : -1; }

int tdk_copy_in(tdk_ctx* c, void* dst, const void* src_host, size_t bytes) {
  if (!c || (bytes && (!dst || !src_host))) return TDK_EINVAL;
  if (!bytes) return TDK_OK;
  cudaSetDevice(c->device);
  TDK_CUDA_TRY(cudaMemcpyAsync(dst, src_host, bytes, cudaMemcpyHostToDevice, c->stream));
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

// selects the ALS form: 0 = persistent kernel when the core fits (default),
// 1 = one kernel per step (test hook, not in the public header)
int tdk_ctx_test_als_form(tdk_ctx* c, int multi) {
  if (!c) return TDK_EINVAL;
  c->als_multi_kernel = multi != 0;
  return TDK_OK;
}

// test hook (not in the public header): make the n-th workspace growth fail
int tdk_ctx_test_fail_alloc(tdk_ctx* c, int after) {
  if (!c) return TDK_EINVAL;
  c->fail_alloc_after = after;
  return TDK_OK;
}

int tucker_sketch(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
                  double* const U_out[], double* const Z_out[]) {
  if (!ctx || !desc || !Y || !W || !U_out) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n) {
    if (!U_out[n]) return TDK_EINVAL;
    for (int k = 0; k < g.N; ++k)
      if (k != n && !W[n * g.N + k]) return TDK_EINVAL;
  }
  if (desc->prec == TDK_PREC_TC && desc->dtype == TDK_F64) return TDK_ENOTSUP;
  cudaSetDevice(ctx->device);
  // the packed sketch lives at the end of a separate workspace slice: allocate
  // it first so the kernels' own carving does not overlap it
  double* Z = nullptr;
  {
    size_t zbytes = sizeof(double) * (size_t)g.zoff[g.N];
    // Z is kept in its own allocation to survive the sub-steps' workspace use
    static_assert(sizeof(double) == 8, "");
    if (cudaMallocAsync((void**)&Z, zbytes, ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      return TDK_ENOMEM;
    }
  }
  if (desc->prec == TDK_PREC_TC)
    rc = sketch_tc(ctx, g, desc->dtype, Y, W, Z);
  else
    rc = sketch_simt(ctx, g, desc->dtype, Y, W, Z);
  if (rc == TDK_OK) rc = cholqr2(ctx, g, Z, U_out);
  if (rc == TDK_OK && Z_out) {
    for (int n = 0; n < g.N; ++n)
      if (Z_out[n]) {
        if (cudaMemcpyAsync(Z_out[n], Z + g.zoff[n], sizeof(double) * g.I[n] * g.Rt[n],
                            cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
          rc = TDK_ECUDA;
      }
  }
  cudaFreeAsync(Z, ctx->stream);
  return rc;
}

int tucker_refine(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
                  double* const U_io[]) {
  if (!ctx || !desc || !Y || !W || !U_io) return TDK_EINVAL;
  Geom g;
  int rc = make_geom(desc, &g);
  if (rc) return rc;
  for (int n = 0; n < g.N; ++n) {
    if (!U_io[n]) return TDK_EINVAL;
    for (int k = 0; k < g.N; ++k)
      if (k != n && !W[n * g.N + k]) return TDK_EINVAL;
  }
  if (desc->dtype != TDK_F64 && desc->dtype != TDK_F32) return TDK_ENOTSUP;
  cudaSetDevice(ctx->device);
  return refine_pass(ctx, g, desc->dtype, Y, W, U_io);
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
  for (int n = 0; n < g.N; ++n) {
    if (opts->R > g.Rt[n]) return TDK_EINVAL;
    if (!U[n] || !B_io[n] || !A_io[n]) return TDK_EINVAL;
  }
  cudaSetDevice(ctx->device);
  return als_run(ctx, g, desc->dtype, G, U, normY2, opts, B_io, A_io, lambda_out, rep);
}

}  // extern "C"
