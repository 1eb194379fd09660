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
   bit 8).  Returns TDK_ECUDA if the stream reported a CUDA error. */
int tdk_ctx_sync_status(tdk_ctx* ctx, int* flags_out /* host */);
/* Number of kernel launches this context has issued since creation. */
int64_t tdk_ctx_launch_count(const tdk_ctx* ctx);
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
   asynchronous: later calls on the stream see the data.  tdk_copy_out waits
   for the stream, so *dst_host is valid on return.  Both buffers are
   caller-owned; bytes = 0 is a no-op.  Errors: TDK_EINVAL (null context or
   buffer), TDK_ECUDA. */
int tdk_copy_in(tdk_ctx* ctx, void* dst /* device */, const void* src_host, size_t bytes);
int tdk_copy_out(tdk_ctx* ctx, void* dst_host, const void* src /* device */, size_t bytes);
/* Human-readable text for a return code. */
const char* tdk_strerror(int code);

/* Problem description, following the paper's problem statement: tensor
   dimensions I_n, multilinear ranks R_n and the oversampling p, so that the
   sketch width is Rt_n = R_n + p (Sec. IV-A). */
typedef struct {
  int N;                    /* order, 2 <= N <= TDK_MAX_MODES               */
  int dtype;                /* TDK_F64 / TDK_F32 / TDK_BF16 storage of Y    */
  int prec;                 /* TDK_PREC_SIMT / TDK_PREC_TC                  */
  int p;                    /* oversampling                                 */
  int64_t I[TDK_MAX_MODES]; /* dimensions                                   */
  int R[TDK_MAX_MODES];     /* Tucker ranks; need 1 <= R_n + p <= min(I_n,
                               TDK_MAX_RANK)                                */
} tdk_tucker_desc;

/* Host-only check of a descriptor, the one every entry point applies before
   any CUDA call: 2 <= N <= TDK_MAX_MODES, a known dtype and prec, p >= 0,
   every I_n >= 1 and R_n >= 1, R_n + p <= min(I_n, TDK_MAX_RANK), and the
   element count below 2^62.  Returns TDK_OK or TDK_EINVAL.  Forms that do
   not cover a valid problem return TDK_ENOTSUP at the entry point: the
   tensor-core sketch wants 3 <= N <= 4, no tensor-core form takes FP64 data,
   and both want the contiguous mode's row pitch a multiple of 16 bytes. */
int tdk_tucker_check(const tdk_tucker_desc* desc);

/*
 * tucker_sketch -- all-mode randomized range finder (Sec. IV-A; Alg. 2 lines
 * "Z = Y_(n) Omega" and "U = orth(Z)"; Eq. 22 for the blockwise sums).
 *
 *   Y      [I_1 x ... x I_N] in desc->dtype.
 *   W      array of N*N device pointers; W[n*N + k] (k != n) is the FP64
 *          matrix W_k^(n) [I_k x Rt_n]; W[n*N + n] is ignored.  The random
 *          test matrix of mode n is Omega_n = KRP_{k != n} W_k^(n).  Values
 *          are rounded to the operand precision of the chosen form (exact if
 *          they are BF16 values, as the bundled generator draws them).
 *   U_out  N device pointers, U_out[n] FP64 [I_n x Rt_n]: orthonormal columns
 *          spanning range(Z_n), diag of the triangular factor positive
 *          (CholQR2: two rounds of Gram -> Cholesky -> Z R^-1, all FP64).
 *          If a Cholesky pivot is not positive (numerically rank-deficient
 *          Z_n) that mode is redone by two-pass Gram-Schmidt in FP64 whose
 *          dependent columns are replaced by fixed pseudo-random vectors made
 *          orthogonal, and TDK_WRANKDEF is raised in the status word.
 *   Z_out  NULL or N device pointers (entries may be NULL); Z_out[n] FP64
 *          [I_n x Rt_n] receives the raw sketch Z_n.
 * Errors: TDK_EINVAL (bad desc, null pointers), TDK_ENOMEM, TDK_ENOTSUP
 * (TDK_PREC_TC with F64 data), TDK_ECUDA.
 */
int tucker_sketch(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y,
                  const double* const W[], double* const U_out[], double* const Z_out[]);

/*
 * tucker_sketch_static -- the sketch pass of tucker_sketch alone (Z_n for
 * every mode, no orthonormalisation), computed without allocating any memory.
 * The paper has no counterpart: it is a deployment variant of the CUDA-core
 * sketch kernel for callers that cannot allocate device memory.
 *
 *   desc   as tucker_sketch; prec must be TDK_PREC_SIMT (else TDK_ENOTSUP).
 *   Y, W   as tucker_sketch.
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
 * before any stream capture begins.
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
 *   Y      [I_1 x ... x I_N], desc->dtype FP64 or FP32 (CUDA-core form).
 *   W      N*N device pointers; W[n*N + k] (k != n) FP64 [Rt_k x Rt_n],
 *          a fresh draw per pass; W[n*N + n] is ignored.
 *   U_io   N device pointers, FP64 [I_n x Rt_n]: the factors in (any full
 *          rank start, e.g. Gaussian), refined in place.
 * Errors: TDK_EINVAL (bad desc, null pointers), TDK_ENOMEM, TDK_ENOTSUP
 * (BF16 data).
 */
int tucker_refine(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y, const double* const W[],
                  double* const U_io[]);

/*
 * tucker_core -- G = Y x_1 U_1^T x_2 ... x_N U_N^T (Alg. 2 line
 * "Y <- Y x_n U^T" for every n; Eq. 1), plus ||Y||_F^2.
 *
 *   U       N device pointers, U[n] FP64 [I_n x Rt_n] (e.g. from tucker_sketch).
 *   G_out   [Rt_1 x ... x Rt_N], FP64 for F64 data, FP32 otherwise.
 *   normY2  NULL or one FP64 device scalar receiving ||Y||_F^2.
 * The first, tensor-sized contraction is over the contiguous mode N; in the
 * TC form it runs on tcgen05 tensor cores (BF16 operands, U split hi+lo, Y
 * split hi+lo when stored as FP32).  Errors as tucker_sketch.
 */
int tucker_core(tdk_ctx* ctx, const tdk_tucker_desc* desc, const void* Y,
                const double* const U[], void* G_out, double* normY2);

enum { TDK_INIT_GIVEN = 0, TDK_INIT_HOSVD = 1 };
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
                       persistent kernel (N >= 3, core fits on chip, no
                       time limit): otherwise TDK_ENOTSUP                  */
  int init;         /* TDK_INIT_GIVEN: start from B_io (nonneg or l1: A_io);
                       TDK_INIT_HOSVD: leading R left singular vectors of
                       every G_(n) (nonneg: their magnitudes lifted)        */
  int check_every;  /* sweeps per convergence check on the host (<= 0: 8) */
  int reserved;
  double timeout_s; /* bound on the whole call in seconds; <= 0 or NaN =
                       none; exceeded -> TDK_ETIMEOUT with the last
                       iterate in the outputs.  A limit selects the
                       one-kernel-per-step form                            */
  double l1;        /* >= 0.  > 0: l1-regularised update of Eq. 16, the
                       LS solution for A_n soft-thresholded, S_c(x) =
                       sign(x) max(|x| - c, 0) with c = l1, then projected
                       if nonneg = TDK_NONNEG_LS.  The factors are updated
                       as A_n (start from A_io, or the HOSVD start lifted);
                       needs the persistent kernel and nonneg NONE or LS,
                       else TDK_ENOTSUP / TDK_EINVAL                        */
} tdk_als_opts;

typedef struct {
  int sweeps;       /* sweeps performed                                    */
  int status;       /* same value as the return code                       */
  double fit_core;  /* 1 - ||G - [[B]]|| / ||G|| (nonneg: vs [[G;U]])       */
  double fit_Y;     /* 1 - ||Y - [[A]]|| / ||Y|| via the Gram identities
                       (NaN if normY2 was NULL)                             */
  double ms;        /* wall time of the call in milliseconds               */
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
 * Learned initialiser (no counterpart in the paper: its ALS starts from random
 * or HOSVD factors, Alg. 1 "Initialize A").  A small MLP maps a Tucker core G
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
  TDK_MLP_OUTPUT = 4       /* last batch: network output, FP32 [batch x N*Rt*Rt] */
};

typedef struct {
  double alpha;   /* weight of the target term (used when Bstar != NULL)   */
  double lr;      /* Adam step size                                        */
  double beta1, beta2, eps;  /* Adam moments and denominator guard        */
  int update;     /* 0: loss and gradients only; 1: also one Adam step      */
  int reserved;
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
