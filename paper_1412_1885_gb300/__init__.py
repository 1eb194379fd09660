"""Python binding of libtdk.so (randomized Tucker + FFCP on one GB300).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libtdk.so, reached through its C ABI (include/tdk.h).  PyTorch
supplies device memory and the current stream.  There is no CPU fallback: if
the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdk.so")
TEST_LIB_PATH = os.path.join(HERE, "libtdk_test.so")  # the same library with test hooks

TDK_OK, TDK_EINVAL, TDK_ENOMEM, TDK_ECUDA, TDK_ETIMEOUT, TDK_ENOTSUP = 0, -1, -2, -3, -4, -5
TDK_ESCRATCH, TDK_EIO = -6, -7
SKETCH_STATIC_MAX_BYTES = 16 << 20
TDK_WRANKDEF, TDK_WNOCONV, TDK_WPINV = 1, 2, 4
F64, F32, BF16 = 0, 1, 2
PREC = {"simt": 0, "tc": 1}
INIT = {"given": 0, "hosvd": 1}
ALS_FORM = {"auto": 0, "steps": 1}
ALS_RAN = {1: "one_cta", 2: "grid", 3: "steps"}
# nonnegative update rule: projected LS, HALS (Eq. 8), multiplicative (Eq. 15)
NONNEG = {False: 0, True: 1, "ls": 1, "hals": 2, "mu": 3}
MAX_MODES = 8
MAX_RANK = 64

# symbols the header declares (checked by the CPU tests)
EXPORTS = ["tdk_ctx_create", "tdk_ctx_destroy", "tdk_ctx_set_stream", "tdk_ctx_sync_status",
           "tdk_ctx_launch_count", "tdk_strerror", "tdk_ctx_profile", "tdk_ctx_profile_read", "tucker_sketch",
           "tucker_core", "ffcp_als", "tucker_sketch_static", "tdk_mlp_create", "tdk_mlp_destroy",
           "tdk_mlp_param_count", "tdk_mlp_set_params", "tdk_mlp_get", "tdk_mlp_colsums", "tdk_mlp_train_step",
           "ffcp_predict_init", "tdk_tucker_check", "tdk_copy_in", "tdk_copy_out", "tucker_refine",
           "tdk_ctx_workspace_bytes", "tdk_sketch_matrices", "tucker_sketch_partial", "tucker_core_partial",
           "tdk_gram", "tdk_orth_apply", "tdk_orth", "tdk_mlp_save", "tdk_mlp_load", "tucker_seq"]
# symbols only the test library exports
TEST_EXPORTS = ["tdk_ctx_test_fail_alloc", "tdk_test_bounded_wait", "tdk_test_gemm_bf16", "tdk_test_ttm_lead",
                "tdk_test_checked_store"]
MLP_PARAMS, MLP_GRADS, MLP_CANON_CORE, MLP_ROTATIONS, MLP_OUTPUT = 0, 1, 2, 3, 4
MLP_INPUT, MLP_Z1, MLP_H1, MLP_Z2, MLP_H2, MLP_DO, MLP_DZ2, MLP_DZ1 = 5, 6, 7, 8, 9, 10, 11, 12


class TuckerDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("dtype", ctypes.c_int), ("prec", ctypes.c_int), ("p", ctypes.c_int),
                ("I", ctypes.c_int64 * MAX_MODES), ("R", ctypes.c_int * MAX_MODES), ("seed", ctypes.c_uint64)]


class AlsOpts(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int), ("max_sweeps", ctypes.c_int), ("tol", ctypes.c_double),
                ("nonneg", ctypes.c_int), ("init", ctypes.c_int), ("check_every", ctypes.c_int),
                ("form", ctypes.c_int), ("timeout_s", ctypes.c_double), ("l1", ctypes.c_double)]


class AlsReport(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("status", ctypes.c_int), ("fit_core", ctypes.c_double),
                ("fit_Y", ctypes.c_double), ("ms", ctypes.c_double), ("form", ctypes.c_int), ("grid", ctypes.c_int)]


class MlpDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("Rt", ctypes.c_int), ("hidden", ctypes.c_int), ("max_batch", ctypes.c_int)]


class MlpTrainOpts(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("lr", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double), ("update", ctypes.c_int),
                ("reserved", ctypes.c_int), ("clip", ctypes.c_double)]


class TdkError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None
_lib_test = None


def lib():
    """Load libtdk.so (built in-tree by build.build()); raises if absent."""
    global _lib
    if _lib is None:
        _lib = _load(LIB_PATH)
    return _lib


def lib_test():
    """Load libtdk_test.so, the library with its test hooks compiled in
    (for the failure-detection and raw-GEMM tests); raises if absent."""
    global _lib_test
    if _lib_test is None:
        _lib_test = _load(TEST_LIB_PATH)
    return _lib_test


def _load(path):
    """Open one build of the library and declare the argument types."""
    if True:  # one indentation level kept for the declarations below
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1412_1885_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        pp = ctypes.POINTER(ctypes.c_void_p)
        L.tdk_ctx_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
        L.tdk_ctx_destroy.argtypes = [vp]
        L.tdk_ctx_set_stream.argtypes = [vp, vp]
        L.tdk_ctx_sync_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.tdk_ctx_launch_count.argtypes = [vp]
        L.tdk_ctx_launch_count.restype = i64
        L.tdk_ctx_workspace_bytes.argtypes = [vp]
        L.tdk_ctx_workspace_bytes.restype = ctypes.c_size_t
        L.tdk_sketch_matrices.argtypes = [vp, ctypes.POINTER(TuckerDesc), pp]
        L.tucker_sketch_partial.argtypes = [vp, ctypes.POINTER(TuckerDesc), i64, i64, vp, pp, pp]
        L.tucker_core_partial.argtypes = [vp, ctypes.POINTER(TuckerDesc), i64, vp, pp, vp, vp]
        L.tdk_gram.argtypes = [vp, vp, i64, ctypes.c_int, vp]
        L.tdk_orth_apply.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp]
        L.tdk_orth.argtypes = [vp, vp, i64, ctypes.c_int, vp]
        L.tdk_mlp_save.argtypes = [vp, vp, ctypes.c_char_p]
        L.tdk_mlp_load.argtypes = [vp, vp, ctypes.c_char_p]
        L.tdk_strerror.argtypes = [ctypes.c_int]
        L.tdk_strerror.restype = ctypes.c_char_p
        L.tdk_tucker_check.argtypes = [ctypes.POINTER(TuckerDesc)]
        L.tdk_copy_in.argtypes = [vp, vp, vp, ctypes.c_size_t]
        L.tdk_copy_out.argtypes = [vp, vp, vp, ctypes.c_size_t]
        L.tucker_sketch.argtypes = [vp, ctypes.POINTER(TuckerDesc), vp, pp, pp, pp, vp]
        L.tucker_core.argtypes = [vp, ctypes.POINTER(TuckerDesc), vp, pp, vp, vp]
        L.tucker_refine.argtypes = [vp, ctypes.POINTER(TuckerDesc), vp, pp, pp]
        L.tucker_seq.argtypes = [vp, ctypes.POINTER(TuckerDesc), vp, pp, pp, vp, vp]
        L.tucker_sketch_static.argtypes = [vp, ctypes.POINTER(TuckerDesc), vp, pp, pp]
        L.ffcp_als.argtypes = [vp, ctypes.POINTER(TuckerDesc), vp, pp, vp, ctypes.POINTER(AlsOpts), pp, pp, vp,
                               ctypes.POINTER(AlsReport)]
        L.tdk_mlp_create.argtypes = [vp, ctypes.POINTER(MlpDesc), ctypes.POINTER(vp)]
        L.tdk_mlp_destroy.argtypes = [vp]
        L.tdk_mlp_param_count.argtypes = [vp]
        L.tdk_mlp_param_count.restype = i64
        L.tdk_mlp_set_params.argtypes = [vp, vp, vp]
        L.tdk_mlp_get.argtypes = [vp, vp, ctypes.c_int, vp]
        L.tdk_mlp_colsums.argtypes = [vp, ctypes.POINTER(TuckerDesc), pp, vp]
        L.tdk_mlp_train_step.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp, vp, vp, ctypes.POINTER(MlpTrainOpts),
                                         ctypes.POINTER(ctypes.c_double)]
        L.ffcp_predict_init.argtypes = [vp, vp, ctypes.POINTER(TuckerDesc), vp, pp, ctypes.c_int, pp]
        if hasattr(L, "tdk_test_gemm_bf16"):
            L.tdk_test_gemm_bf16.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                             ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                             ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int]
        L.tdk_ctx_profile.argtypes = [vp, ctypes.c_int]
        L.tdk_ctx_profile_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64)]
        if hasattr(L, "tdk_ctx_test_fail_alloc"):
            L.tdk_ctx_test_fail_alloc.argtypes = [vp, ctypes.c_int]
        if hasattr(L, "tdk_test_bounded_wait"):
            L.tdk_test_bounded_wait.argtypes = [vp, ctypes.c_ulonglong]
        if hasattr(L, "tdk_test_checked_store"):
            L.tdk_test_checked_store.argtypes = [vp, ctypes.c_longlong, ctypes.c_longlong]
        if hasattr(L, "tdk_test_ttm_lead"):
            L.tdk_test_ttm_lead.argtypes = [vp, ctypes.POINTER(TuckerDesc), vp, vp, vp]
        return L


def strerror(code: int) -> str:
    try:
        return lib().tdk_strerror(int(code)).decode()
    except Exception:
        return str(code)


def _check(rc, what):
    if rc < 0:
        raise TdkError(rc, what)
    return rc


def _ptrs(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def _dtype_code(t):
    import torch

    return {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[t.dtype]


def make_desc(shape, dtype_code, ranks, p, prec="simt", seed=0) -> TuckerDesc:
    d = TuckerDesc()
    d.N = len(shape)
    d.dtype = dtype_code
    d.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    d.p = int(p)
    d.seed = int(seed) & ((1 << 64) - 1)
    if len(ranks) != len(shape) or len(shape) > MAX_MODES:
        raise ValueError("ranks must match the tensor order (<= 8 modes)")
    for n, (I, R) in enumerate(zip(shape, ranks)):
        d.I[n] = int(I)
        d.R[n] = int(R)
    return d


def tucker_check(shape, dtype_code, ranks, p, prec="simt") -> int:
    """The library's own descriptor check (host only, no CUDA call): TDK_OK or
    TDK_EINVAL."""
    return int(lib().tdk_tucker_check(ctypes.byref(make_desc(shape, dtype_code, ranks, p, prec))))


class Context:
    """A library context on one CUDA device; calls run on torch's current stream.
    testing=True opens it in libtdk_test.so, the build with the test hooks."""

    def __init__(self, device: int = 0, testing: bool = False):
        import torch

        self.device = int(device)
        self.L = lib_test() if testing else lib()
        self.als_form = "auto"  # default ALS form of ffcp_als calls on this context
        self._h = ctypes.c_void_p()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        _check(self.L.tdk_ctx_create(ctypes.byref(self._h), self.device, ctypes.c_void_p(stream)), "tdk_ctx_create")

    @property
    def handle(self):
        return self._h

    def _bind_stream(self):
        import torch

        self.L.tdk_ctx_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def sync_status(self) -> int:
        f = ctypes.c_int(0)
        self._bind_stream()
        _check(self.L.tdk_ctx_sync_status(self._h, ctypes.byref(f)), "tdk_ctx_sync_status")
        return f.value

    def launch_count(self) -> int:
        return int(self.L.tdk_ctx_launch_count(self._h))

    def workspace_bytes(self) -> int:
        return int(self.L.tdk_ctx_workspace_bytes(self._h))

    def profile(self, enable: bool):
        self._bind_stream()
        _check(self.L.tdk_ctx_profile(self._h, int(bool(enable))), "tdk_ctx_profile")

    def profile_read(self, region: int):
        """(total milliseconds, launches) of the main kernel of a region
        (0: sketch pass over Y, 1: core pass over Y) since profile(True)."""
        ms = ctypes.c_double(0)
        n = ctypes.c_int64(0)
        _check(self.L.tdk_ctx_profile_read(self._h, int(region), ctypes.byref(ms), ctypes.byref(n)),
               "tdk_ctx_profile_read")
        return ms.value, n.value

    def set_als_form(self, multi_kernel: bool):
        """Default ALS form of later ffcp_als calls: "steps" (one kernel per
        step, also the fallback for cores that do not fit) or "auto"."""
        self.als_form = "steps" if multi_kernel else "auto"

    def close(self):
        if self._h:
            self.L.tdk_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _w_array(W, N):
    """N*N pointer array of the W_k^(n) (diagonal NULL), or NULL for W=None
    (the library draws them from the descriptor's seed)."""
    if W is None:
        return None
    Wf = []
    for n in range(N):
        for k in range(N):
            Wf.append(None if k == n else W[n][k].contiguous())
    return _ptrs(Wf)


def sketch_matrices(ctx: Context, shape, ranks, p, seed):
    """The test matrices W[n][k] (FP64 device [I_k x (R_n + p)], W[n][n] None)
    that the library draws from `seed` (tdk_sketch_matrices)."""
    import torch

    N = len(shape)
    Rt = [int(r) + int(p) for r in ranks]
    W = [[None if k == n else torch.empty((shape[k], Rt[n]), dtype=torch.float64, device=f"cuda:{ctx.device}")
          for k in range(N)] for n in range(N)]
    desc = make_desc(shape, F32, ranks, p, "simt", seed)
    ctx._bind_stream()
    _check(ctx.L.tdk_sketch_matrices(ctx.handle, ctypes.byref(desc), _w_array(W, N)), "tdk_sketch_matrices")
    return W


def tucker_sketch(ctx: Context, Y, W, ranks, p, prec="simt", want_Z=False, seed=0, normY2=None):
    """All-mode sketch + CholQR2 (see include/tdk.h).  W[n][k] are FP64 device
    tensors [I_k x (R_n + p)] (W[n][n] unused), or None to let the library
    draw them from `seed`.  normY2: optional FP64 device scalar tensor that
    receives ||Y||^2.  Returns (U list, Z list|None)."""
    import torch

    N = Y.dim()
    desc = make_desc(Y.shape, _dtype_code(Y), ranks, p, prec, seed)
    Rt = [int(r) + int(p) for r in ranks]
    dev = Y.device
    U = [torch.empty((Y.shape[n], Rt[n]), dtype=torch.float64, device=dev) for n in range(N)]
    Z = [torch.empty((Y.shape[n], Rt[n]), dtype=torch.float64, device=dev) for n in range(N)] if want_Z else None
    ctx._bind_stream()
    _check(ctx.L.tucker_sketch(ctx.handle, ctypes.byref(desc), ctypes.c_void_p(Y.data_ptr()), _w_array(W, N),
                               _ptrs(U), _ptrs(Z) if Z is not None else None,
                               ctypes.c_void_p(normY2.data_ptr() if normY2 is not None else None)), "tucker_sketch")
    return U, Z


def tucker_sketch_static(ctx: Context, Y, W, ranks, p, Z_out=None):
    """Sketch pass only (Z_n for every mode), through the allocation-free
    entry point (CUDA-core form; scratch in a fixed static device array, see
    include/tdk.h).  Z_out: optional preallocated FP64 device tensors
    [I_n x (R_n + p)].  Returns the Z list."""
    import torch

    N = Y.dim()
    desc = make_desc(Y.shape, _dtype_code(Y), ranks, p, "simt")
    Rt = [int(r) + int(p) for r in ranks]
    if Z_out is None:
        Z_out = [torch.empty((Y.shape[n], Rt[n]), dtype=torch.float64, device=Y.device) for n in range(N)]
    ctx._bind_stream()
    _check(ctx.L.tucker_sketch_static(ctx.handle, ctypes.byref(desc), ctypes.c_void_p(Y.data_ptr()),
                                      _w_array(W, N), _ptrs(Z_out)), "tucker_sketch_static")
    return Z_out


def tucker_refine(ctx: Context, Y, W, U, ranks, p, seed=0, prec="simt"):
    """One RandTucker2i refinement pass (see include/tdk.h): U (FP64 device
    tensors [I_n x Rt_n]) refined in place with the pass matrices W[n][k]
    (FP64 device [Rt_k x Rt_n]), or with matrices drawn from `seed` when W is
    None.  prec "tc" runs the two passes over BF16 data on the tensor cores.
    Returns U."""
    N = Y.dim()
    desc = make_desc(Y.shape, _dtype_code(Y), ranks, p, prec, seed)
    ctx._bind_stream()
    _check(ctx.L.tucker_refine(ctx.handle, ctypes.byref(desc), ctypes.c_void_p(Y.data_ptr()), _w_array(W, N),
                               _ptrs(U)), "tucker_refine")
    return U


def rand_tucker_2i(ctx: Context, Y, U0, W_passes, ranks, p, prec="simt"):
    """RandTucker2i (Alg. 3): the starting factors U0 refined by one pass
    per entry of W_passes (two in the paper; an entry may be an int seed),
    then the core.  Returns (U, G, ||Y||^2)."""
    U = [u.clone() for u in U0]
    for W in W_passes:
        if isinstance(W, int):
            tucker_refine(ctx, Y, None, U, ranks, p, seed=W, prec=prec)
        else:
            tucker_refine(ctx, Y, W, U, ranks, p, prec=prec)
    G, nrm = tucker_core(ctx, Y, U, ranks, p, prec)
    return U, G, nrm


def tucker_seq(ctx: Context, Y, W, ranks, p, prec="simt", seed=0):
    """Alg. 2 as printed, with Khatri-Rao test matrices (tucker_seq): W as
    for tucker_sketch (None: drawn from `seed`).  Returns (U, G, ||Y||^2)
    with U FP64 device [I_n x Rt_n], G the core (FP64 for FP64 data, else
    FP32) and the norm an FP64 device scalar."""
    import torch

    N = Y.dim()
    desc = make_desc(Y.shape, _dtype_code(Y), ranks, p, prec, seed)
    Rt = [int(r) + int(p) for r in ranks]
    U = [torch.empty((Y.shape[n], Rt[n]), dtype=torch.float64, device=Y.device) for n in range(N)]
    gdt = torch.float64 if Y.dtype == torch.float64 else torch.float32
    G = torch.empty(Rt, dtype=gdt, device=Y.device)
    nrm = torch.empty((), dtype=torch.float64, device=Y.device)
    ctx._bind_stream()
    _check(ctx.L.tucker_seq(ctx.handle, ctypes.byref(desc), ctypes.c_void_p(Y.data_ptr()), _w_array(W, N), _ptrs(U),
                            ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(nrm.data_ptr())), "tucker_seq")
    return U, G, nrm


def tucker_core(ctx: Context, Y, U, ranks, p, prec="simt", want_norm=True):
    """G = Y x_1 U_1^T ... x_N U_N^T and ||Y||^2 (device FP64 scalar, None
    when want_norm is False)."""
    import torch

    desc = make_desc(Y.shape, _dtype_code(Y), ranks, p, prec)
    Rt = [int(r) + int(p) for r in ranks]
    gdt = torch.float64 if Y.dtype == torch.float64 else torch.float32
    G = torch.empty(Rt, dtype=gdt, device=Y.device)
    nrm = torch.empty((), dtype=torch.float64, device=Y.device) if want_norm else None
    ctx._bind_stream()
    _check(ctx.L.tucker_core(ctx.handle, ctypes.byref(desc), ctypes.c_void_p(Y.data_ptr()),
                             _ptrs([u.contiguous() for u in U]), ctypes.c_void_p(G.data_ptr()),
                             ctypes.c_void_p(nrm.data_ptr() if want_norm else None)), "tucker_core")
    return G, nrm


# ---- sharded form (Sec. IV-B): one slab of rows of mode 1 per worker

def tucker_sketch_partial(ctx: Context, Y_slab, row_off, I1_total, W, ranks, p, prec="simt", seed=0):
    """The slab's share of the all-mode sketch: (slab rows of Z_1, shares of
    Z_n for n >= 2), FP64 device tensors (tucker_sketch_partial)."""
    import torch

    N = Y_slab.dim()
    desc = make_desc(Y_slab.shape, _dtype_code(Y_slab), ranks, p, prec, seed)
    Rt = [int(r) + int(p) for r in ranks]
    Z = [torch.empty((Y_slab.shape[n], Rt[n]), dtype=torch.float64, device=Y_slab.device) for n in range(N)]
    ctx._bind_stream()
    _check(ctx.L.tucker_sketch_partial(ctx.handle, ctypes.byref(desc), int(row_off), int(I1_total),
                                       ctypes.c_void_p(Y_slab.data_ptr()), _w_array(W, N), _ptrs(Z)),
           "tucker_sketch_partial")
    return Z


def tucker_core_partial(ctx: Context, Y_slab, I1_total, U, ranks, p, prec="simt"):
    """The slab's share of the core and of ||Y||^2; U[0] holds the slab's rows
    of U_1 (tucker_core_partial)."""
    import torch

    desc = make_desc(Y_slab.shape, _dtype_code(Y_slab), ranks, p, prec)
    Rt = [int(r) + int(p) for r in ranks]
    gdt = torch.float64 if Y_slab.dtype == torch.float64 else torch.float32
    G = torch.empty(Rt, dtype=gdt, device=Y_slab.device)
    nrm = torch.empty((), dtype=torch.float64, device=Y_slab.device)
    ctx._bind_stream()
    _check(ctx.L.tucker_core_partial(ctx.handle, ctypes.byref(desc), int(I1_total), ctypes.c_void_p(Y_slab.data_ptr()),
                                     _ptrs([u.contiguous() for u in U]), ctypes.c_void_p(G.data_ptr()),
                                     ctypes.c_void_p(nrm.data_ptr())), "tucker_core_partial")
    return G, nrm


def gram(ctx: Context, Z):
    """Upper triangle of Z^T Z (tdk_gram), FP64 device [cols x cols]."""
    import torch

    Z = Z.contiguous()
    out = torch.empty((Z.shape[1], Z.shape[1]), dtype=torch.float64, device=Z.device)
    ctx._bind_stream()
    _check(ctx.L.tdk_gram(ctx.handle, ctypes.c_void_p(Z.data_ptr()), int(Z.shape[0]), int(Z.shape[1]),
                          ctypes.c_void_p(out.data_ptr())), "tdk_gram")
    return out


def orth_apply(ctx: Context, G, Z):
    """Z R^-1 with R the Cholesky factor of the Gram G (tdk_orth_apply); a
    breakdown shows as TDK_WRANKDEF in ctx.sync_status()."""
    import torch

    Z = Z.contiguous()
    Q = torch.empty_like(Z)
    ctx._bind_stream()
    _check(ctx.L.tdk_orth_apply(ctx.handle, ctypes.c_void_p(G.contiguous().data_ptr()), ctypes.c_void_p(Z.data_ptr()),
                                int(Z.shape[0]), int(Z.shape[1]), ctypes.c_void_p(Q.data_ptr())), "tdk_orth_apply")
    return Q


def orth(ctx: Context, Z):
    """Orthonormal basis of range(Z) by CholQR2 with completion (tdk_orth)."""
    import torch

    Z = Z.contiguous()
    U = torch.empty_like(Z)
    ctx._bind_stream()
    _check(ctx.L.tdk_orth(ctx.handle, ctypes.c_void_p(Z.data_ptr()), int(Z.shape[0]), int(Z.shape[1]),
                          ctypes.c_void_p(U.data_ptr())), "tdk_orth")
    return U


def ffcp_als(ctx: Context, G, U, shape, ranks, p, dtype_code, R, max_sweeps=1000, tol=1e-7, nonneg=False,
             init="given", B0=None, A0=None, normY2=None, check_every=8, timeout_s=0.0, l1=0.0, form=None):
    """FFCP on the core (see include/tdk.h).  Returns dict(A, B, lam, report).
    form: "auto" or "steps" (default: the context's als_form)."""
    import torch

    N = len(shape)
    desc = make_desc(shape, dtype_code, ranks, p, "simt")
    Rt = [int(r) + int(p) for r in ranks]
    dev = G.device
    B = [torch.zeros((Rt[n], R), dtype=torch.float64, device=dev) for n in range(N)]
    A = [torch.zeros((shape[n], R), dtype=torch.float64, device=dev) for n in range(N)]
    if B0 is not None:
        for n in range(N):
            B[n].copy_(B0[n])
    if A0 is not None:
        for n in range(N):
            A[n].copy_(A0[n])
    lam = torch.empty(R, dtype=torch.float64, device=dev)
    o = AlsOpts(R=int(R), max_sweeps=int(max_sweeps), tol=float(tol), nonneg=NONNEG[nonneg],
                init=INIT[init], check_every=int(check_every), form=ALS_FORM[form or ctx.als_form],
                timeout_s=float(timeout_s), l1=float(l1))
    rep = AlsReport()
    ctx._bind_stream()
    rc = _check(ctx.L.ffcp_als(ctx.handle, ctypes.byref(desc), ctypes.c_void_p(G.data_ptr()),
                               _ptrs([u.contiguous() for u in U]),
                               ctypes.c_void_p(normY2.data_ptr() if normY2 is not None else None),
                               ctypes.byref(o), _ptrs(B), _ptrs(A), ctypes.c_void_p(lam.data_ptr()),
                               ctypes.byref(rep)), "ffcp_als")
    return {"A": A, "B": B, "lam": lam, "status": rc, "sweeps": rep.sweeps, "fit_core": rep.fit_core,
            "fit_Y": rep.fit_Y, "ms": rep.ms, "form": ALS_RAN.get(rep.form, "?"), "grid": rep.grid}


class Mlp:
    """Learned FFCP initialiser (see include/tdk.h, tdk_mlp section): an MLP
    from a canonicalised Tucker core to initial core-space factors."""

    def __init__(self, ctx: Context, N: int, Rt: int, hidden: int = 1024, max_batch: int = 256):
        self.ctx = ctx
        self.N, self.Rt, self.hidden, self.max_batch = int(N), int(Rt), int(hidden), int(max_batch)
        self._h = ctypes.c_void_p()
        d = MlpDesc(N=self.N, Rt=self.Rt, hidden=self.hidden, max_batch=self.max_batch)
        ctx._bind_stream()
        _check(ctx.L.tdk_mlp_create(ctx.handle, ctypes.byref(d), ctypes.byref(self._h)), "tdk_mlp_create")
        self.din = self.Rt ** self.N
        self.dout = self.N * self.Rt * self.Rt
        self._last = 0

    @property
    def handle(self):
        return self._h

    def param_count(self) -> int:
        return int(self.ctx.L.tdk_mlp_param_count(self._h))

    def set_params(self, theta):
        import numpy as np

        a = np.ascontiguousarray(theta, dtype=np.float32)
        if a.size != self.param_count():
            raise ValueError("parameter vector has the wrong size")
        self.ctx._bind_stream()
        _check(self.ctx.L.tdk_mlp_set_params(self.ctx.handle, self._h, a.ctypes.data_as(ctypes.c_void_p)),
               "tdk_mlp_set_params")

    def get(self, what: int):
        """A TDK_MLP_* array as float32 numpy (batch arrays of the last call)."""
        import numpy as np

        B, RR = self._last, self.Rt * self.Rt
        n = {MLP_PARAMS: self.param_count(), MLP_GRADS: self.param_count(), MLP_CANON_CORE: B * self.din,
             MLP_ROTATIONS: B * self.N * RR, MLP_OUTPUT: B * self.dout, MLP_INPUT: B * self.din,
             MLP_Z1: B * self.hidden, MLP_H1: B * self.hidden, MLP_Z2: B * self.hidden, MLP_H2: B * self.hidden,
             MLP_DO: B * self.dout, MLP_DZ2: B * self.hidden, MLP_DZ1: B * self.hidden}[what]
        out = np.empty(n, dtype=np.float32)
        self.ctx._bind_stream()
        _check(self.ctx.L.tdk_mlp_get(self.ctx.handle, self._h, int(what), out.ctypes.data_as(ctypes.c_void_p)),
               "tdk_mlp_get")
        return out

    def save(self, path: str):
        """Write parameters, Adam moments and step to a checkpoint file."""
        _check(self.ctx.L.tdk_mlp_save(self.ctx.handle, self._h, os.fsencode(path)), "tdk_mlp_save")

    def load(self, path: str):
        """Read a checkpoint of a model of the same shape."""
        _check(self.ctx.L.tdk_mlp_load(self.ctx.handle, self._h, os.fsencode(path)), "tdk_mlp_load")

    def train_step(self, G, colsums, R, Bstar=None, alpha=0.0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   update=True, lam=None, clip=0.0):
        """One step on a device batch: G FP32 [B, Rt^N], colsums FP64 [B, N, Rt],
        R int32 [B], Bstar FP64 [B, N, Rt, Rt] or None, lam FP64 [B, Rt] or None
        (weights of Bstar's columns); clip > 0 caps the gradient's global norm
        before the Adam step.  Returns the batch loss."""
        o = MlpTrainOpts(alpha=float(alpha), lr=float(lr), beta1=float(beta1), beta2=float(beta2), eps=float(eps),
                         update=int(bool(update)), reserved=0, clip=float(clip))
        loss = ctypes.c_double(0.0)
        B = int(G.shape[0])
        self.ctx._bind_stream()
        _check(self.ctx.L.tdk_mlp_train_step(self.ctx.handle, self._h, B, ctypes.c_void_p(G.data_ptr()),
                                             ctypes.c_void_p(colsums.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                             ctypes.c_void_p(Bstar.data_ptr() if Bstar is not None else None),
                                             ctypes.c_void_p(lam.data_ptr() if lam is not None else None),
                                             ctypes.byref(o), ctypes.byref(loss)), "tdk_mlp_train_step")
        self._last = B
        return loss.value

    def colsums(self, U, shape, ranks, p):
        """1^T U_n for every mode, FP64 device [N, Rt]."""
        import torch

        desc = make_desc(shape, F32, ranks, p)
        out = torch.empty((len(shape), self.Rt), dtype=torch.float64, device=U[0].device)
        self.ctx._bind_stream()
        _check(self.ctx.L.tdk_mlp_colsums(self.ctx.handle, ctypes.byref(desc), _ptrs([u.contiguous() for u in U]),
                                          ctypes.c_void_p(out.data_ptr())), "tdk_mlp_colsums")
        return out

    def predict_init(self, G, U, shape, ranks, p, dtype_code, R):
        """Initial core-space factors B_n (FP64 [Rt, R]) for ffcp_als."""
        import torch

        desc = make_desc(shape, dtype_code, ranks, p)
        B = [torch.empty((self.Rt, int(R)), dtype=torch.float64, device=G.device) for _ in range(self.N)]
        self.ctx._bind_stream()
        _check(self.ctx.L.ffcp_predict_init(self.ctx.handle, self._h, ctypes.byref(desc),
                                            ctypes.c_void_p(G.data_ptr()), _ptrs([u.contiguous() for u in U]),
                                            int(R), _ptrs(B)), "ffcp_predict_init")
        self._last = 1
        return B

    def close(self):
        if self._h:
            self.ctx.L.tdk_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def copy_in(ctx: Context, dst, src_host):
    """Host tensor -> device tensor of the same size, on the context's stream
    (tdk_copy_in)."""
    nbytes = src_host.numel() * src_host.element_size()
    if dst.numel() * dst.element_size() != nbytes or not dst.is_cuda or src_host.is_cuda:
        raise ValueError("copy_in: a host source and a device destination of equal size")
    ctx._bind_stream()
    _check(ctx.L.tdk_copy_in(ctx.handle, ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(src_host.data_ptr()),
                             nbytes), "tdk_copy_in")
    return dst


def copy_out(ctx: Context, src, dst_host=None):
    """Device tensor -> host tensor (allocated when dst_host is None); waits
    for the context's stream (tdk_copy_out)."""
    import torch

    if dst_host is None:
        dst_host = torch.empty(src.shape, dtype=src.dtype)
    nbytes = src.numel() * src.element_size()
    ctx._bind_stream()
    _check(ctx.L.tdk_copy_out(ctx.handle, ctypes.c_void_p(dst_host.data_ptr()), ctypes.c_void_p(src.data_ptr()),
                              nbytes), "tdk_copy_out")
    return dst_host


def decompose(ctx: Context, Y, W, ranks, p, R, prec="simt", nonneg=False, max_sweeps=1000, tol=1e-7,
              init="given", B0=None, A0=None, check_every=8, model=None, Y_dev=None, l1=0.0, seed=0):
    """The whole path: sketch -> CholQR2 -> core -> FFCP -> lift.  Y may be a
    host tensor (copied in by tdk_copy_in, into Y_dev when given) or a device
    tensor; results stay on the device.  W=None draws the test matrices from
    `seed` inside the library.
    Without a start (B0, or A0 for the nonnegative form) FFCP starts from the
    HOSVD of the core.
    With `model` (an Mlp) and the unconstrained form, the ALS starts from the
    learned initial factors instead of B0."""
    if not Y.is_cuda:
        import torch

        if Y_dev is None:
            Y_dev = torch.empty(Y.shape, dtype=Y.dtype, device=f"cuda:{ctx.device}")
        Y = copy_in(ctx, Y_dev, Y.contiguous())
    ambient = bool(NONNEG[nonneg]) or l1 > 0.0
    if init == "given" and model is None and (A0 is None if ambient else B0 is None):
        init = "hosvd"  # no start given: the HOSVD start of the core
    import torch

    nrm = torch.empty((), dtype=torch.float64, device=Y.device)
    U, _ = tucker_sketch(ctx, Y, W, ranks, p, prec, seed=seed, normY2=nrm)  # ||Y||^2 from the sketch pass
    G, _ = tucker_core(ctx, Y, U, ranks, p, prec, want_norm=False)
    if model is not None and not ambient:
        B0 = model.predict_init(G, U, tuple(Y.shape), ranks, p, _dtype_code(Y), R)
        init = "given"
    out = ffcp_als(ctx, G, U, tuple(Y.shape), ranks, p, _dtype_code(Y), R, max_sweeps, tol, nonneg, init, B0, A0,
                   nrm, check_every, l1=l1)
    out.update({"U": U, "G": G, "normY2": nrm})
    return out


__all__ = ["Context", "Mlp", "tucker_check", "copy_in", "copy_out", "tucker_sketch", "tucker_refine",
           "rand_tucker_2i", "tucker_sketch_static", "tucker_core", "ffcp_als", "decompose", "lib", "lib_test",
           "make_desc", "TdkError", "EXPORTS", "TEST_EXPORTS", "strerror", "sketch_matrices",
           "tucker_sketch_partial", "tucker_core_partial", "gram", "orth_apply", "orth"]
