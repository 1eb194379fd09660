/*
 * tdk.h -- C ABI of the GB300 randomized-Tucker + FFCP library (libtdk.so).
 *
 * The library computes the data-parallel path of "Decomposition of Big
 * Tensors With Low Multilinear Rank" (Zhou, Cichocki, Xie):
 *
 *   tucker_sketch   Z_n = Y_(n) Omega_n for every mode n in one pass over Y,
 *                   Omega_n = KRP_{k != n} W_k^(n) never formed (Sec. IV-A,
 *                   range-finder steps 1-2; Alg. 2; Eq. 22), then an
 *                   orthonormal basis U_n of range(Z_n) (range-finder step 3;
 *                   Eq. 23 gives the Gram-based variant used in spirit here:
 *                   FP64 CholQR2).
 *   tucker_core     G = Y x_1 U_1^T ... x_N U_N^T (Alg. 2, TTM chain; Eq. 1).
 *   ffcp_als        CP-ALS on the core with the lift A_n = U_n B_n
 *                   (Sec. III-B, Alg. 1; Eqs. 9, 11-14, 17), unconstrained or
 *                   with projected nonnegative updates (P_+ of Eq. 8).
 *   ffcp_predict_init  learned initial core-space factors from a small MLP
 *                   (no counterpart in the paper; see the tdk_mlp section).
 *
 * Conventions for every entry point:
 *   - Tensors and matrices are ROW-MAJOR, last index fastest.  The mode-n
 *     unfolding Y_(n) has row i_n and columns the other indices in row-major
 *     order; KRP_{k != n} orders its factors with the smallest k slowest.
 *   - Every data pointer is CALLER-OWNED DEVICE memory on the context's
 *     device, unless the comment says "host".  The library never frees them.
 *   - Calls are asynchronous on the context's stream, except ffcp_als, which
 *     synchronises once at the end to fill its host report.
 *   - Return value: 0 = TDK_OK; negative = error (no output is guaranteed);
 *     positive = warning (outputs valid).  Device-side conditions found by
 *     asynchronous calls (rank-deficient sketch, wait timeout) are ORed into
 *     the context's status word; tdk_ctx_sync_status() waits for the stream
 *     and returns and clears it.
 *   - A context is not thread-safe; separate contexts are independent.
 *   - The context owns its workspace (grown on demand with cudaMalloc) and
 *     frees it in tdk_ctx_destroy.
 */
#ifndef TDK_H
#define TDK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TDK_OK 0
#define TDK_EINVAL (-1)    /* invalid argument or configuration            */
#define TDK_ENOMEM (-2)    /* workspace allocation failed                  */
#define TDK_ECUDA (-3)     /* a CUDA runtime/driver call failed            */
#define TDK_ETIMEOUT (-4)  /* a bounded device-side wait gave up           */
#define TDK_ENOTSUP (-5)   /* a form or option that does not cover the case */
#define TDK_ESCRATCH (-6)  /* problem needs more scratch than the fixed
                              static array of tucker_sketch_static holds   */
#define TDK_EIO (-7)       /* a file could not be read or written, or holds
                              something else than what the call expects     */
#define TDK_WRANKDEF 1     /* a sketch was numerically rank deficient; the
                              orthonormal basis was completed (see below)  */
#define TDK_WNOCONV 2      /* ALS stopped at max_sweeps                    */
#define TDK_WPINV 4        /* an ALS normal equation used the pseudo-inverse */

#define TDK_MAX_MODES 8
#define TDK_MAX_RANK 64    /* max sketch width R_n + p and max CP rank R   */

/* storage type of the data tensor Y (and of the core G: F64 data -> F64
   core, otherwise F32 core) */
enum { TDK_F64 = 0, TDK_F32 = 1, TDK_BF16 = 2 };

/* arithmetic form of the two passes over Y */
enum {
  TDK_PREC_SIMT = 0, /* CUDA-core FMAs in the storage precision (FP32 for
                        BF16 data): the plain form                        */
  TDK_PREC_TC = 1    /* tcgen05 tensor cores, BF16 operands, FP32
                        accumulation; FP32 data is split hi+lo so products
                        keep ~16 significant bits, except that the
                        Khatri-Rao rows of the last mode's sketch are rounded
                        once to BF16 when its width exceeds 32 (the sketch is
                        then exact for a test matrix within 2^-9 of Omega_N);
                        F64 data: not supported                            */
};

typedef struct tdk_ctx tdk_ctx;

/* Create a context on `device` (CUDA ordinal) that launches on `cuda_stream`
   (a cudaStream_t; NULL = the legacy default stream).  *out receives the
   handle.  Errors: TDK_EINVAL (null out), TDK_ECUDA. */
int tdk_ctx_create(tdk_ctx** out, int device, void* cuda_stream);
/* Free the workspace and the handle.  Waits for the stream first. */
int tdk_ctx_destroy(tdk_ctx* ctx);
/* Switch the stream later calls launch on. */
int tdk_ctx_set_stream(tdk_ctx* ctx, void* cuda_stream);
/* Wait for the stream, then return (and clear) the OR of the device-side
   status flags raised since the last call (TDK_WRANKDEF, TDK_ETIMEOUT as
   bit 8; in the test library, built with bounds checks, bit 9 when an index
   fell outside its range and the access was skipped).  Returns TDK_ECUDA if
   the stream reported a CUDA error. */
int tdk_ctx_sync_status(tdk_ctx* ctx, int* flags_out /* host */);
/* Number of kernel launches this context has issued since creation. */
int64_t tdk_ctx_launch_count(const tdk_ctx* ctx);
/* Bytes of device workspace the context holds now (0 until an entry point
   first needs one; it only grows, and tdk_ctx_destroy frees it). */
size_t tdk_ctx_workspace_bytes(const tdk_ctx* ctx);
/* Kernel timing by CUDA events recorded on the launching stream around the
   main kernel of each region (0 = the pass of tucker_sketch over Y, 1 = the
   pass of tucker_core over Y).  tdk_ctx_profile(ctx, 1) starts recording and
   clears the totals; tdk_ctx_profile_read waits for the recorded events and
   returns the summed milliseconds and the number of timed launches of a
   region.  Errors: TDK_EINVAL (bad region), TDK_ECUDA. */
int tdk_ctx_profile(tdk_ctx* ctx, int enable);
int tdk_ctx_profile_read(tdk_ctx* ctx, int region, double* total_ms /* host */,
                         int64_t* launches /* host */);
/* Host <-> device copies on the context's stream, for callers whose data
   live in host memory (pinned memory for full link speed).  tdk_copy_in is
   asynchronous: later calls on the stream see the data.  A page-locked
   source of 64 MiB or more, with both addresses 16-byte aligned, is read by
   a copy kernel on the SMs through its mapped device address (on GB300
   about 210 GB/s against 140-180 GB/s for the copy engine); any other
   source, and the last bytes past a multiple of 16, go through
   cudaMemcpyAsync.  tdk_copy_out waits for the stream, so *dst_host is valid
   on return.  Both buffers are caller-owned; bytes = 0 is a no-op.  Errors:
   TDK_EINVAL (null context or buffer), TDK_ECUDA. */
int tdk_copy_in(tdk_ctx* ctx, void* dst /* device */, const void* src_host, size_t bytes);
int tdk_copy_out(tdk_ctx* ctx, void* dst_host, const void* src /* device */, size_t bytes);
/* Human-readable text for a return code. */
const char* tdk_strerror(int code);

/* Problem description, following the paper's problem statement: tensor
   dimensions I_n, multilinear ranks R_n and the oversampling p, so that the
   sketch width is Rt_n = R_n + p (Sec. IV-A), and the seed of the random test
   matrices (Sec. IV-B shares a seed between workers, not the matrices). */
typedef struct {
  int N;                    /* order, 2 <= N <= TDK_MAX_MODES               */
  int dtype;                /* TDK_F64 / TDK_F32 / TDK_BF16 storage of Y    */
  int prec;                 /* TDK_PREC_SIMT / TDK_PREC_TC                  */
  int p;                    /* oversampling                                 */
  int64_t I[TDK_MAX_MODES]; /* dimensions                                   */
  int R[TDK_MAX_MODES];     /* Tucker ranks; need 1 <= R_n + p <= min(I_n,
                               TDK_MAX_RANK)                                */
  uint64_t seed;            /* seed of the test matrices W_k^(n) that the
                               library draws when a call gets W = NULL     */
} tdk_tucker_desc;

/*
 * The seeded test matrices.  Entry (i, r) of W_k^(n) (mode n's sketch, factor
 * of mode k, 0-based n, k, i, r) is one standard normal value rounded to the
 * nearest BF16 value (ties to even), drawn from the counter-based generator
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *   key     = (seed mod 2^32, seed div 2^32),
 *   counter = (r, i mod 2^32, i div 2^32, 256 n + k),
 * whose four output words x0..x3 give a = (x0 2^32 + x1) div 2^11 and
 * b = (x2 2^32 + x3) div 2^11 (53-bit integers), u1 = (a + 1/2) 2^-53,
 * u2 = b 2^-53 and the value sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller, FP64).
 * Every entry is independent of the matrix sizes, so a slab of rows of
 * W_k^(n) is drawn alone with the same values (the sharded form uses this).
 * tdk_sketch_matrices writes the matrices that desc->seed defines: W_out is
 * N*N device pointers, W_out[n*N + k] (k != n) FP64 [I_k x Rt_n], the
 * diagonal entries ignored (may be NULL).  Errors: TDK_EINVAL, TDK_ECUDA.
 */
int tdk_sketch_matrices(tdk_ctx* ctx, const tdk_tucker_desc* desc, double* const W_out[]);

/* Host-only check of a descriptor, the one every entry point applies before
   any CUDA call: 2 <= N <= TDK_MAX_MODES, a known dtype and prec, p >= 0,
   every I_n >= 1 and R_n >= 1, R_n + p <= min(I_n, TDK_MAX_RANK), and the
   element count below 2^62.  Returns TDK_OK or TDK_EINVAL.  Forms that do
   not cover a valid problem return TDK_ENOTSUP at the entry point: the
   tensor-core sketch wants 3 <= N <= 4, no tensor-core form takes FP64 data,
   and both want the contiguous mode's row pitch a multiple of 16 bytes. */
int tdk_tucker_check(const tdk_tucker_desc* desc);

/*
 * tucker_sketch -- all-mode randomized range finder (Sec. IV-A; Alg. 2, the
 * sketch of every mode and its orthonormal basis; Eq. 22 for the blockwise
 * sums).
 *
 *   Y      [I_1 x ... x I_N] in desc->dtype.
 *   W      NULL: the matrices are drawn from desc->seed (see
 *          tdk_sketch_matrices).  Otherwise an array of N*N device pointers;
 *          W[n*N + k] (k != n) is the FP64 matrix W_k^(n) [I_k x Rt_n];
 *          W[n*N + n] is ignored.  The random test matrix of mode n is
 *          Omega_n = KRP_{k != n} W_k^(n).  Values are rounded to the operand
 *          precision of the chosen form (exact if they are BF16 values, as
 *          both the seeded draw and the bundled generator make them).
 *   U_out  N device pointers, U_out[n] FP64 [I_n x Rt_n]: orthonormal columns
 *          spanning range(Z_n), diag of the triangular factor positive
 *          (CholQR2: two rounds of Gram -> Cholesky -> Z R^-1, all FP64).
 *          If a Cholesky pivot is not positive (numerically rank-deficient
 *          Z_n) that mode is redone by two-pass Gram-Schmidt in FP64 whose
 *          dependent columns are replaced by fixed pseudo-random vectors made
 *          orthogonal, and TDK_WRANKDEF is raised in the status word.
 *   Z_out  NULL or N device pointers (entries may be NULL); Z_out[n] FP64
 *          [I_n x Rt_n] receives the raw sketch Z_n.
 *   normY2 NULL or one FP64 device scalar receiving ||Y||_F^2 (the fit needs
 *          it).  The tensor-core forms sum it while the pass stages the
 *          tiles of Y; the CUDA-core form and the shared-family tensor-core
 *          form of BF16 data take one more streaming pass over Y.  Asking for
 *          it here lets tucker_core skip its own sum (pass it NULL there).
 * Errors: TDK_EINVAL (bad desc, null pointers), TDK_ENOMEM, TDK_ENOTSUP
 * (TDK_PREC_TC with F64 data), TDK_ECUDA.
 */
int tucker_sketch(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y,
                  const double* const W[], double* const U_out[], double* const Z_out[],
                  double* normY2);

/*
 * tucker_sketch_static -- the sketch pass of tucker_sketch alone (Z_n for
 * every mode, no orthonormalisation), computed without allocating any memory.
 * The paper has no counterpart: it is a deployment variant of the CUDA-core
 * sketch kernel for callers that cannot allocate device memory.
 *
 *   desc   as tucker_sketch; prec must be TDK_PREC_SIMT (else TDK_ENOTSUP).
 *   Y, W   as tucker_sketch, except that W must not be NULL (the seeded draw
 *          would need scratch of its own): use tdk_sketch_matrices once.
 *   Z_out  N device pointers, all non-NULL; Z_out[n] FP64 [I_n x Rt_n]
 *          receives Z_n = Y_(n) Omega_n.
 * Scratch: a file-scope device array of TDK_SKETCH_STATIC_MAX_BYTES bytes
 * (converted W, per-CTA partial sketches, the packed FP64 sum).  No
 * cudaMalloc/cudaFree or allocating library routine is called.  A problem
 * whose converted W plus the packed sketch plus one CTA's partial sketch do
 * not fit returns TDK_ESCRATCH before anything is launched; otherwise the grid
 * is reduced until the partials fit, which only changes the order of the
 * fixed-order FP64 sum.
 * Sharing: every call on a device uses the same array.  Calls whose work
 * overlaps on the GPU (other streams, other contexts, other threads) race
 * and give wrong results; serialise them (one stream, or events).
 * Set-up: the first call on each device resolves the array's address with
 * cudaGetSymbolAddress (this may load the module); make that first call
 * before any stream capture begins.  The address is kept per device together
 * with the identity of the CUDA context it was resolved in; a call that finds
 * another context current on the device (after cudaDeviceReset, say)
 * resolves it again, so that call is a set-up call too.
 * Errors: TDK_EINVAL (bad desc, null pointers), TDK_ENOTSUP, TDK_ESCRATCH,
 * TDK_ECUDA.
 */
#define TDK_SKETCH_STATIC_MAX_BYTES ((size_t)16 << 20)
int tucker_sketch_static(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y,
                         const double* const W[], double* const Z_out[]);

/*
 * tucker_refine -- one refinement pass of RandTucker2i (Alg. 3, the loop
 * body; RandTucker2i is two passes from random factors, then tucker_core).
 * For n = 1..N in order, each mode using the factors already refined:
 *   X = Y x_{p != n} U_p^T (Alg. 3 prints U_p; read U_p^T),
 *   Z_n = X_(n) Omega_n with Omega_n = KRP_{k != n} W[n*N + k],
 *   U_n <- orthonormal basis of Z_n (CholQR2, FP64; rank-deficient Z_n
 *   completed as in tucker_sketch).
 *   Y      [I_1 x ... x I_N] in desc->dtype.  The pass reads Y twice: the
 *          core pass with mode 1 left open (X of n = 1), and Y x_1 U_1^T with
 *          the U_1 just refined, from which every n >= 2 shrinks its X.  For
 *          BF16 data with desc->prec TDK_PREC_TC both run on the tensor cores
 *          (U split hi + lo in BF16, FP32 accumulation); the shrunk tensors
 *          are FP32 (FP64 for FP64 data).  TDK_PREC_SIMT: CUDA cores only.
 *   W      N*N device pointers; W[n*N + k] (k != n) FP64 [Rt_k x Rt_n],
 *          a fresh draw per pass; W[n*N + n] is ignored.  NULL: drawn from
 *          desc->seed as in tdk_sketch_matrices with I_k replaced by Rt_k
 *          (the first Rt_k rows of that seed's matrices), so give every pass
 *          its own seed.  The tensor-core sketch of a shrunk tensor rounds W
 *          to BF16 as tucker_sketch does.
 *   U_io   N device pointers, FP64 [I_n x Rt_n]: the factors in (any full
 *          rank start, e.g. Gaussian), refined in place.
 * Workspace: the context's, plus stream-ordered allocations for the shrunk
 * tensors (the largest is Y x_1 U_1^T: numel / I_1 * Rt_1 elements).
 * Errors: TDK_EINVAL (bad desc, null pointers), TDK_ENOMEM, TDK_ENOTSUP
 * (TDK_PREC_TC with FP64 data).
 */
int tucker_refine(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
                  double* const U_io[]);

/*
 * tucker_seq -- the sequential randomized Tucker compression of Alg. 2 as
 * printed, with Khatri-Rao test matrices: for n = 1..N in order, starting
 * from X = Y,
 *   Z_n = X_(n) Omega_n,  Omega_n = KRP_{k != n} (first d_k rows of W[n*N + k]),
 *   U_n = orthonormal basis of Z_n (CholQR2, FP64),
 *   X  <- X x_n U_n^T  (mode n shrinks to Rt_n),
 * with d_k the size of mode k when mode n is sketched (Rt_k for k < n, I_k
 * for k > n).  The last X is the core.  It reads Y twice (the sketch of mode
 * 1 and Y x_1 U_1^T); later modes work on the shrunk tensor.
 *   desc   as tucker_sketch (dtype, prec, seed).
 *   Y      [I_1 x ... x I_N] in desc->dtype.  BF16 data with TDK_PREC_TC:
 *          the sketch of Y and Y x_1 U_1^T on the tensor cores (as in
 *          tucker_sketch and tucker_core), the shrunk tensors in FP32.
 *   W      NULL or N*N device pointers as for tucker_sketch (FP64
 *          [I_k x Rt_n]); only the first d_k rows are read.  NULL: the
 *          matrices tdk_sketch_matrices draws for desc->seed.
 *   U_out  N device pointers, FP64 [I_n x Rt_n].
 *   G_out  the core [Rt_1 x ... x Rt_N], FP64 for FP64 data, FP32 otherwise.
 *   normY2 NULL or an FP64 device scalar receiving ||Y||_F^2.
 * Workspace: as tucker_refine.
 * Errors: TDK_EINVAL, TDK_ENOMEM, TDK_ENOTSUP (TDK_PREC_TC with FP64 data),
 * TDK_ECUDA, TDK_ETIMEOUT (status word).
 */
int tucker_seq(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
               double* const U_out[], void* G_out, double* normY2);

/*
 * tucker_core -- G = Y x_1 U_1^T x_2 ... x_N U_N^T (Alg. 2, the projection
 * step of every mode; Eq. 1), plus ||Y||_F^2.
 *
 *   U       N device pointers, U[n] FP64 [I_n x Rt_n] (e.g. from tucker_sketch).
 *   G_out   [Rt_1 x ... x Rt_N], FP64 for F64 data, FP32 otherwise.
 *   normY2  NULL or one FP64 device scalar receiving ||Y||_F^2.  NULL makes
 *           the BF16 tensor-core pass faster: its stage ring is then released
 *           by the MMAs alone (take the norm from tucker_sketch instead).
 * The first, tensor-sized contraction is over the contiguous mode N; in the
 * TC form it runs on tcgen05 tensor cores (BF16 operands, U split hi+lo, Y
 * split hi+lo when stored as FP32).  Errors as tucker_sketch.
 */
int tucker_core(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y,
                const double* const U[], void* G_out, double* normY2);

enum { TDK_INIT_GIVEN = 0, TDK_INIT_HOSVD = 1 };
/* ALS form: AUTO picks the fastest form that covers the problem; STEPS forces
   the kernel-per-step form (any core size, pseudo-inverse, time limit). */
enum { TDK_ALS_FORM_AUTO = 0, TDK_ALS_FORM_STEPS = 1 };
/* form that ran (tdk_als_report.form) */
enum { TDK_ALS_RAN_ONE_CTA = 1, TDK_ALS_RAN_GRID = 2, TDK_ALS_RAN_STEPS = 3 };
enum { TDK_NONNEG_NONE = 0, TDK_NONNEG_LS = 1, TDK_NONNEG_HALS = 2, TDK_NONNEG_MU = 3 };

typedef struct {
  int R;            /* CP rank, 1 <= R <= min_n Rt_n                       */
  int max_sweeps;   /* >= 1                                                */
  double tol;       /* stop when |f_t - f_{t-1}| < tol * |f_{t-1}|, f the
                       fit of the core (Sec. V-A uses an absolute 1e-6)     */
  int nonneg;       /* 0: LS update (Eq. 14); TDK_NONNEG_LS (1): projected
                       nonnegative LS; TDK_NONNEG_HALS (2): column-wise
                       HALS (Eq. 8); TDK_NONNEG_MU (3): multiplicative
                       update in the low-rank form (Eq. 15).  HALS and MU
                       start each mode from A_n diag(lambda) and need the
                       persistent kernel or, for rows that do not fit on
                       chip, the kernel-per-step form                       */
  int init;         /* TDK_INIT_GIVEN: start from B_io (nonneg or l1: A_io);
                       TDK_INIT_HOSVD: leading R left singular vectors of
                       every G_(n) (nonneg: their magnitudes lifted)        */
  int check_every;  /* sweeps per convergence check on the host (<= 0: 8) */
  int form;         /* TDK_ALS_FORM_AUTO or TDK_ALS_FORM_STEPS             */
  double timeout_s; /* bound on the whole call in seconds; <= 0 or NaN =
                       none; exceeded -> TDK_ETIMEOUT with the last
                       iterate in the outputs.  A limit selects the
                       one-kernel-per-step form                            */
  double l1;        /* >= 0.  > 0: l1-regularised update of Eq. 16, the
                       LS solution for A_n soft-thresholded, S_c(x) =
                       sign(x) max(|x| - c, 0) with c = l1, then projected
                       if nonneg = TDK_NONNEG_LS.  The factors are updated
                       as A_n (start from A_io, or the HOSVD start lifted);
                       needs nonneg NONE or LS, else TDK_EINVAL            */
} tdk_als_opts;

typedef struct {
  int sweeps;       /* sweeps performed                                    */
  int status;       /* same value as the return code                       */
  double fit_core;  /* 1 - ||G - [[B]]|| / ||G|| (nonneg: vs [[G;U]])       */
  double fit_Y;     /* 1 - ||Y - [[A]]|| / ||Y|| via the Gram identities
                       (NaN if normY2 was NULL)                             */
  double ms;        /* wall time of the call in milliseconds               */
  int form;         /* TDK_ALS_RAN_*: the form that produced the result    */
  int grid;         /* CTAs of the persistent launch (1 for ONE_CTA, 0 for
                       the kernel-per-step form)                           */
} tdk_als_report;

/*
 * ffcp_als -- FFCP (Alg. 1): CP-ALS on the core G with core-space factors
 * B_n = U_n^T A_n (Eq. 13); per mode H_n = G_(n) [KRP_{p != n} B_p]
 * (Eq. 12), T_n = HADAMARD_{p != n} B_p^T B_p (Eq. 9; A_p^T A_p for the
 * nonnegative form), B_n <- H_n T_n^-1 (Eq. 14; FP64 Cholesky, pseudo-inverse
 * with cutoff R*eps*lambda_max when a pivot is not above R*eps*max T_jj);
 * columns normalised to unit 2-norm with the norms in lambda.  Nonnegative
 * form: A_n <- max(0, U_n H_n T_n^-1), B_n <- U_n^T A_n.
 *
 *   G       core from tucker_core (FP64 for F64 data, FP32 otherwise).
 *   U       N device pointers, FP64 [I_n x Rt_n].
 *   normY2  NULL or FP64 device scalar ||Y||^2 (for report->fit_Y).
 *   B_io    N device pointers, FP64 [Rt_n x R]: initial values when
 *           init = GIVEN and not nonneg; on return the normalised B_n.
 *   A_io    N device pointers, FP64 [I_n x R]: initial A_n when nonneg and
 *           init = GIVEN; on return A_n = U_n B_n with lambda absorbed into
 *           A_N (Sec. II) -- for the nonnegative form the projected A_n.
 *   lambda_out  NULL or FP64 device [R].
 *   rep     NULL or host report.
 * Returns TDK_OK, TDK_WNOCONV, TDK_WPINV (ORed warnings) or an error.
 */
int ffcp_als(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* G,
             const double* const U[], const double* normY2, const tdk_als_opts* opts,
             double* const B_io[], double* const A_io[], double* lambda_out,
             tdk_als_report* rep);

/* ======================================================================
 * Sharded form (Sec. IV-B): Y split along its first mode into slabs of
 * consecutive rows i_1, one slab per worker.  The calls below compute one
 * worker's share; the caller sums the shares over the workers (an allreduce)
 * between the calls, which is the whole exchange of the method:
 *   1. tucker_sketch_partial on each slab; sum the Z_n shares (n >= 2).
 *   2. U_n (n >= 2) = tdk_orth(Z_n), on every worker (same input, same bits).
 *   3. U_1 by CholQR2 over the row blocks of Z_1 (Eq. 23: the Gram of the
 *      stacked blocks is the sum of the blocks' Grams): gram = sum of
 *      tdk_gram(Z_1 slab rows); Q = tdk_orth_apply(gram, Z_1 rows); then the
 *      same again on Q gives the slab's rows of U_1.
 *   4. tucker_core_partial on each slab with its rows of U_1; sum the core
 *      shares and the ||Y||^2 shares.
 *   5. ffcp_als on the summed core, on every worker.
 * A slab descriptor is the whole tensor's descriptor with I[0] replaced by
 * the slab's row count (any count >= 1; the rule R_1 + p <= I_1 applies to
 * I1_total instead).
 * ====================================================================== */

/*
 * tucker_sketch_partial -- one slab's share of the all-mode sketch (Eq. 22).
 *   slab   slab descriptor (rows [row_off, row_off + slab->I[0]) of mode 1 of
 *          a tensor whose first dimension is I1_total).
 *   Y      the slab, [slab->I[0] x I_2 x ... x I_N] in slab->dtype.
 *   W      NULL (draw from slab->seed, rows of W_1^(n) at their global index)
 *          or the whole tensor's N*N pointers as in tucker_sketch (W_1^(n)
 *          with I1_total rows; the library reads the slab's rows).
 *   Z_out  N device pointers: Z_out[0] FP64 [slab->I[0] x Rt_1] receives the
 *          slab's rows of Z_1; Z_out[n] (n >= 1) FP64 [I_n x Rt_n] the slab's
 *          share of Z_n (sum over its i_1).
 * Errors: TDK_EINVAL (bad desc, offsets or pointers), TDK_ENOMEM, TDK_ENOTSUP
 * (as tucker_sketch), TDK_ECUDA.
 */
int tucker_sketch_partial(tdk_ctx* ctx, const tdk_tucker_desc* slab, int64_t row_off, int64_t I1_total,
                          const void* Y, const double* const W[], double* const Z_out[]);
/*
 * tucker_core_partial -- one slab's share of the core and of ||Y||^2:
 * G_share = Y_slab x_1 U_1[slab rows]^T x_2 U_2^T ... x_N U_N^T (Eq. 1 summed
 * over the slabs).  U[0] points at the slab's rows of U_1, FP64
 * [slab->I[0] x Rt_1]; U[n] (n >= 1) FP64 [I_n x Rt_n].  G_out and normY2 as
 * tucker_core, for the share.  Errors as tucker_core.
 */
int tucker_core_partial(tdk_ctx* ctx, const tdk_tucker_desc* slab, int64_t I1_total, const void* Y,
                        const double* const U[], void* G_out, double* normY2);
/*
 * tdk_gram -- gram_out = upper triangle of Z^T Z (FP64 [cols x cols], rows
 * <= cols entries set, the others 0) for Z FP64 [rows x cols] (row-major,
 * 1 <= cols <= TDK_MAX_RANK).  The sum of the Grams of row blocks is the
 * Gram of the stacked matrix (Eq. 23).  Errors: TDK_EINVAL, TDK_ENOMEM,
 * TDK_ECUDA.
 */
int tdk_gram(tdk_ctx* ctx, const double* Z, int64_t rows, int cols, double* gram_out);
/*
 * tdk_orth_apply -- Q = Z R^-1 with R the upper Cholesky factor of the
 * symmetric matrix whose upper triangle `gram` holds (one round of CholQR;
 * Eq. 23 with a Cholesky factor in place of the eigendecomposition).  If a
 * pivot is not above cols * eps * max diag, Q is not written and the
 * context's status word gets TDK_WRANKDEF (tdk_ctx_sync_status).
 * Errors: TDK_EINVAL, TDK_ENOMEM, TDK_ECUDA.
 */
int tdk_orth_apply(tdk_ctx* ctx, const double* gram, const double* Z, int64_t rows, int cols, double* Q_out);
/*
 * tdk_orth -- orthonormal basis U of range(Z) for one matrix, the step 3 of
 * the range finder that tucker_sketch applies to each mode: CholQR2 in FP64,
 * completed by two-pass Gram-Schmidt when Z is numerically rank deficient
 * (status TDK_WRANKDEF).  Z, U_out FP64 [rows x cols], cols <= min(rows,
 * TDK_MAX_RANK).  Errors: TDK_EINVAL, TDK_ENOMEM, TDK_ECUDA.
 */
int tdk_orth(tdk_ctx* ctx, const double* Z, int64_t rows, int cols, double* U_out);

/* ======================================================================
 * Learned initialiser (no counterpart in the paper: its ALS starts from random
 * or HOSVD factors, Alg. 1's first step).  A small MLP maps a Tucker core G
 * (output of tucker_core, all sketch widths equal to Rt) to initial
 * core-space factors B_n for ffcp_als.
 *
 * Canonical form of a core: V_n = eigenvectors of G_(n) G_(n)^T, by
 * decreasing eigenvalue, column j negated when colsum_n . v_j < 0, where
 * colsum_n = 1^T U_n (so that the ambient vector U_n v_j has a nonnegative
 * entry sum: the rule does not depend on the basis U_n the sketch produced);
 * S = G x_1 V_1^T ... x_N V_N^T / ||G||.
 * Network: x = BF16(sqrt(Rt^N) vec S) (unit RMS) -> hidden -> hidden -> N*Rt*Rt, GELU
 * activations, BF16 weights and activations on tcgen05 tensor cores with FP32
 * accumulation, FP32 master weights.  Output O[(n*Rt + i)*Rt + r] =
 * Bhat_n[i, r] in canonical coordinates; only the first R columns are used.
 * Loss per sample: ||S - [[Bhat]]||^2 + alpha ||[[Bhat]] - [[T]]||^2 with
 * T_n = V_n^T B*_n (B*_N / ||G||), the converged FFCP factors of the same
 * core; both terms are invariant under a permutation of the R columns; the
 * batch loss is the mean.  Training: back-propagation and Adam.
 * ====================================================================== */
typedef struct tdk_mlp tdk_mlp;

typedef struct {
  int N;          /* order of the cores, 2..4                               */
  int Rt;         /* sketch width of every mode, 2..32; Rt^N <= 12288       */
  int hidden;     /* width of the two hidden layers, 8..8192               */
  int max_batch;  /* largest batch of tdk_mlp_train_step, 1..65536          */
} tdk_mlp_desc;

/* Parameter vector layout (FP32, row-major blocks in this order): W1
   [hidden x Rt^N], b1 [hidden], W2 [hidden x hidden], b2 [hidden], W3
   [N*Rt*Rt x hidden], b3 [N*Rt*Rt]. */
enum {
  TDK_MLP_PARAMS = 0,      /* the parameter vector                          */
  TDK_MLP_GRADS = 1,       /* gradient of the last train step's batch loss   */
  TDK_MLP_CANON_CORE = 2,  /* last batch: S, FP32 [batch x Rt^N]            */
  TDK_MLP_ROTATIONS = 3,   /* last batch: V_n, FP32 [batch][N][Rt][Rt]      */
  TDK_MLP_OUTPUT = 4,      /* last batch: network output, FP32 [batch x N*Rt*Rt] */
  /* last batch, the stored intermediates of the forward and backward passes
     (BF16 values returned as FP32; rows of the batch, no padding): */
  TDK_MLP_INPUT = 5,       /* x = BF16(sqrt(Rt^N) vec S)   [batch x Rt^N]   */
  TDK_MLP_Z1 = 6,          /* x W1^T + b1, FP32            [batch x hidden] */
  TDK_MLP_H1 = 7,          /* BF16(gelu(Z1))               [batch x hidden] */
  TDK_MLP_Z2 = 8,          /* H1 W2^T + b2, FP32           [batch x hidden] */
  TDK_MLP_H2 = 9,          /* BF16(gelu(Z2))               [batch x hidden] */
  TDK_MLP_DO = 10,         /* BF16(dLoss/dO)               [batch x N*Rt*Rt] */
  TDK_MLP_DZ2 = 11,        /* BF16((dO W3) * gelu'(Z2))    [batch x hidden] */
  TDK_MLP_DZ1 = 12         /* BF16((dZ2 W2) * gelu'(Z1))   [batch x hidden] */
};

typedef struct {
  double alpha;   /* weight of the target term (used when Bstar != NULL)   */
  double lr;      /* Adam step size                                        */
  double beta1, beta2, eps;  /* Adam moments and denominator guard        */
  int update;     /* 0: loss and gradients only; 1: also one Adam step      */
  int reserved;
  double clip;    /* > 0: before the Adam step the gradient is scaled by
                     min(1, clip / ||g||_2), the norm over all parameters
                     (gradient-norm clipping); 0: no clipping.  The stored
                     gradient (TDK_MLP_GRADS) stays unscaled.              */
} tdk_mlp_train_opts;

/* Create a model (weights zero until tdk_mlp_set_params) with device
   buffers for max_batch samples.  Errors: TDK_EINVAL, TDK_ENOMEM, TDK_ECUDA. */
int tdk_mlp_create(tdk_ctx* ctx, const tdk_mlp_desc* desc, tdk_mlp** out);
/* Free the model (waits for the device first). */
int tdk_mlp_destroy(tdk_mlp* m);
/* Number of FP32 parameters. */
int64_t tdk_mlp_param_count(const tdk_mlp* m);
/* Copy a host parameter vector in (layout above); resets Adam's moments and
   step counter.  Synchronous. */
int tdk_mlp_set_params(tdk_ctx* ctx, tdk_mlp* m, const float* host_params);
/* Copy one of the TDK_MLP_* arrays out to host memory.  Synchronous. */
int tdk_mlp_get(tdk_ctx* ctx, tdk_mlp* m, int what, float* host_out);
/* Checkpoint: tdk_mlp_save writes the model's shape (N, Rt, hidden), the
   parameter vector, Adam's two moment vectors and its step counter to the
   file `path` (little-endian; an 8-byte tag "TDKMLP01", four int32 N, Rt,
   hidden, 0, int64 parameter count, int64 step, then three FP32 vectors of
   that count: parameters, first and second moments).  tdk_mlp_load reads
   such a file into a model of the same shape, so that training resumes where
   it stopped.  Both synchronous.  Errors: TDK_EINVAL (null argument),
   TDK_EIO (file error, wrong tag, shape or size), TDK_ECUDA. */
int tdk_mlp_save(tdk_ctx* ctx, const tdk_mlp* m, const char* path);
int tdk_mlp_load(tdk_ctx* ctx, tdk_mlp* m, const char* path);
/* colsum_n = 1^T U_n for every mode, FP64 [N][Rt] device output (the sign
   rule's input; all Rt_n must be equal). */
int tdk_mlp_colsums(tdk_ctx* ctx, const tdk_tucker_desc* desc, const double* const U[], double* out);
/*
 * One training step on a batch of cores (device inputs):
 *   G        FP32 [batch][Rt^N] raw cores from tucker_core;
 *   colsums  FP64 [batch][N][Rt] (tdk_mlp_colsums of each core's U);
 *   R        int32 [batch], CP rank of each sample, 1..Rt;
 *   Bstar    NULL or FP64 [batch][N][Rt][Rt]: converged FFCP factors of each
 *            core (columns >= R ignored);
 *   lambda   NULL or FP64 [batch][Rt]: weights of Bstar's columns, so that
 *            G ~ [[lambda; B*]] (NULL: the weights are already absorbed).
 * Computes the loss and its gradient (TDK_MLP_GRADS) and, with
 * opts->update, one Adam step.  *loss_out (host, may be NULL) receives the
 * batch loss, which makes the call synchronous.
 */
int tdk_mlp_train_step(tdk_ctx* ctx, tdk_mlp* m, int batch, const float* G, const double* colsums, const int* R,
                       const double* Bstar, const double* lambda, const tdk_mlp_train_opts* opts,
                       double* loss_out);
/*
 * ffcp_predict_init -- initial core-space factors for ffcp_als from the
 * model: canonicalise G (desc->dtype F64 -> FP64 core, else FP32), run the
 * network, B_out[n] = V_n Bhat_n[:, :R] as FP64 [Rt x R] (pass as B_io with
 * init = TDK_INIT_GIVEN).  U: the Tucker factors of the core (for the sign
 * rule).  Errors: TDK_EINVAL (shape mismatch with the model), TDK_ECUDA.
 */
int ffcp_predict_init(tdk_ctx* ctx, tdk_mlp* m, const tdk_tucker_desc* desc, const void* G,
                      const double* const U[], int R, double* const B_out[]);

#ifdef __cplusplus
}
#endif
#endif /* TDK_H */
