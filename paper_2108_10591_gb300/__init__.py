"""Thin Python binding of libbcs.so (include/bcs.h, include/bcs_tune.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Device vectors are passed as torch CUDA tensors (their data_ptr())
or raw integer device pointers; host arrays as numpy arrays.  Import fails
loudly when the compiled library is missing: there is no CPU fallback.

Names follow the C ABI: csr_upload, matrix_info, matrix_export, spmv, dot,
dot_noalloc, solver_create, solve, solve_host, get_history, get_scalars,
solve_batched, Batch (bcs_batch_*), autotune, batch_autotune,
autotune_sell_sigma, status_string; include/bcs_dist.h: partition_rows,
halo_plan, Dist (bcs_dist_*).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbcs.so")

SSBICGSAFE2, P_BICGSAFE, P_BICGSAFE_RR = 0, 1, 2
KINDS = {"ssBiCGSafe2": SSBICGSAFE2, "p-BiCGSafe": P_BICGSAFE, "p-BiCGSafe-rr": P_BICGSAFE_RR}
FP64, FP32_REFINE, BF16MAT_REFINE = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32_REFINE, "bf16": BF16MAT_REFINE}
LAYOUT_AUTO, LAYOUT_CSR, LAYOUT_SELL = 0, 1, 2
STORE_F64, STORE_F32, STORE_BF16 = 1, 2, 4
OK, NOT_CONVERGED, ERR_ARG, ERR_CUDA, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_NONFINITE, ERR_OOM = 0, 1, -1, -2, -3, -4, -5, -6

EXPORTED = ["bcs_options_default", "bcs_csr_upload", "bcs_matrix_info", "bcs_matrix_export", "bcs_spmv", "bcs_dot", "bcs_dot_noalloc",
            "bcs_matrix_free", "bcs_solver_create", "bcs_solve", "bcs_solve_host", "bcs_get_history",
            "bcs_get_scalars", "bcs_solver_destroy", "bcs_solve_batched", "bcs_batch_create", "bcs_batch_solve",
            "bcs_batch_destroy", "bcs_autotune", "bcs_batch_autotune", "bcs_status_string",
            "bcs_autotune_sell_sigma", "bcs_partition_rows", "bcs_halo_plan", "bcs_dist_create", "bcs_dist_solve",
            "bcs_dist_get_history", "bcs_dist_get_scalars", "bcs_dist_info", "bcs_dist_destroy",
            "bcs_dist_rank_create", "bcs_dist_rank_export", "bcs_dist_rank_connect", "bcs_solver_precond_blocks"]


class Options(ctypes.Structure):
    _fields_ = [("rr_m", ctypes.c_int), ("rr_M", ctypes.c_int), ("precision", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("history_len", ctypes.c_int),
                ("layout", ctypes.c_int), ("threads_per_row", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("max_ctas", ctypes.c_int), ("spin_budget_ms", ctypes.c_double), ("inner_maxit", ctypes.c_int),
                ("inner_stall", ctypes.c_int), ("tile_order", ctypes.c_int), ("precond", ctypes.c_int),
                ("big_ctas", ctypes.c_int), ("big_systems", ctypes.c_int), ("block_size", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("outer_steps", ctypes.c_int),
                ("rr_steps", ctypes.c_int), ("fallbacks", ctypes.c_int), ("rel_res_recursive", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("r0_norm", ctypes.c_double), ("seconds", ctypes.c_double),
                ("grid_syncs", ctypes.c_int), ("reductions", ctypes.c_int), ("spmv_passes", ctypes.c_int),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = status_string(self.status)
        return d


class TuneEntry(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_int), ("threads_per_row", ctypes.c_int), ("cluster_ctas", ctypes.c_int),
                ("us_per_iter", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libbcs.so is not built (%s); run __graft_entry__.build() or "
                          "python paper_2108_10591_gb300/build.py" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.bcs_options_default.argtypes = [ctypes.POINTER(Options)]
    L.bcs_options_default.restype = None
    L.bcs_csr_upload.argtypes = [I64, I64, P, P, P, I, I, I, I, P, ctypes.POINTER(P)]
    L.bcs_matrix_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                  ctypes.POINTER(I), ctypes.POINTER(I)]
    L.bcs_matrix_export.argtypes = [P] * 10
    L.bcs_spmv.argtypes = [P, I, I, P, P, I, I, P]
    L.bcs_dot.argtypes = [I64, P, P, I, ctypes.POINTER(D), P]
    L.bcs_dot_noalloc.argtypes = [I64, P, P, I, P, P]
    L.bcs_matrix_free.argtypes = [P]
    L.bcs_matrix_free.restype = None
    L.bcs_solver_create.argtypes = [P, I, D, I, ctypes.POINTER(Options), ctypes.POINTER(P)]
    L.bcs_solve.argtypes = [P, P, P, ctypes.POINTER(Result), P]
    L.bcs_solve_host.argtypes = [P, P, P, ctypes.POINTER(Result), P]
    L.bcs_get_history.argtypes = [P, P, I, ctypes.POINTER(I)]
    L.bcs_get_scalars.argtypes = [P, P, I, ctypes.POINTER(I)]
    L.bcs_solver_precond_blocks.argtypes = [P, P, P, ctypes.POINTER(I)]
    L.bcs_solver_destroy.argtypes = [P]
    L.bcs_solver_destroy.restype = None
    L.bcs_solve_batched.argtypes = [I, P, I, D, I, ctypes.POINTER(Options), P, P, P, P]
    L.bcs_batch_create.argtypes = [I, P, I, D, I, ctypes.POINTER(Options), ctypes.POINTER(P)]
    L.bcs_batch_solve.argtypes = [P, P, P, P, P]
    L.bcs_batch_destroy.argtypes = [P]
    L.bcs_batch_destroy.restype = None
    L.bcs_autotune.argtypes = [P, I, I, I, P, I, ctypes.POINTER(I), ctypes.POINTER(TuneEntry), P]
    L.bcs_batch_autotune.argtypes = [I, P, I, ctypes.POINTER(Options), I, P, I, ctypes.POINTER(I),
                                     ctypes.POINTER(Options), P]
    L.bcs_autotune_sell_sigma.argtypes = [P, I, I, I, P, I, P, ctypes.POINTER(I), ctypes.POINTER(P), P]
    L.bcs_partition_rows.argtypes = [I64, P, I, P]
    L.bcs_halo_plan.argtypes = [I64, P, P, I, P, I, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                P, P, P, P, P, P]
    L.bcs_dist_create.argtypes = [I64, I64, P, P, P, I, P, I, D, I, ctypes.POINTER(Options), ctypes.POINTER(P)]
    L.bcs_dist_solve.argtypes = [P, P, P, ctypes.POINTER(Result), P]
    L.bcs_dist_get_history.argtypes = [P, P, I, ctypes.POINTER(I)]
    L.bcs_dist_get_scalars.argtypes = [P, P, I, ctypes.POINTER(I)]
    L.bcs_dist_info.argtypes = [P, I, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64),
                                ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I)]
    L.bcs_dist_rank_create.argtypes = [I64, I64, P, P, P, I, P, I, I, D, I, ctypes.POINTER(Options), ctypes.POINTER(P)]
    L.bcs_dist_rank_export.argtypes = [P, P]
    L.bcs_dist_rank_connect.argtypes = [P, P]
    L.bcs_dist_destroy.argtypes = [P]
    L.bcs_dist_destroy.restype = None
    L.bcs_status_string.argtypes = [I]
    L.bcs_status_string.restype = ctypes.c_char_p
    for name in EXPORTED:
        getattr(L, name)
    return L


lib = _load()


class BcsError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, status_string(code), code))
        self.code = code


def status_string(code):
    return lib.bcs_status_string(int(code)).decode()


def _check(code, what):
    if code < 0:
        raise BcsError(code, what)
    return code


def _ptr(t):
    """Device pointer of a torch tensor (or an int)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _dvec(t, n, name, dtypes=("float64",)):
    """Check a device vector argument before its pointer reaches the library: a torch tensor must
    live on the GPU, be contiguous, have one of `dtypes` and n elements (n=None: any).  A raw integer
    device pointer is passed through unchecked.  A host tensor here would otherwise be read by a
    kernel as device memory."""
    if t is None or isinstance(t, int):
        return
    if not getattr(t, "is_cuda", False):
        raise ValueError("%s must be a CUDA tensor (got %s)" % (name, type(t).__name__))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    dt = str(t.dtype).replace("torch.", "")
    if dt not in dtypes:
        raise ValueError("%s must have dtype %s (got %s)" % (name, " or ".join(dtypes), dt))
    if n is not None and t.numel() != n:
        raise ValueError("%s must have %d elements (got %d)" % (name, n, t.numel()))


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _stream(stream):
    """The CUDA stream handle to pass: an explicit stream (torch stream or raw handle), else torch's
    current stream, so that a call made inside `with torch.cuda.stream(s)` is ordered after the work
    already queued on s (torch creates its side streams non-blocking: the legacy default stream does
    not wait for them).  NULL when torch has not initialised CUDA (its current stream is then the
    default stream)."""
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import sys
    torch = sys.modules.get("torch")
    if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
        return torch.cuda.current_stream().cuda_stream or None
    return None


def _precision(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def options(**kw):
    o = Options()
    lib.bcs_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "precond" and isinstance(v, str):
            v = {"none": 0, "jacobi": 1, "block-jacobi": 2}[v]
        if k == "layout" and isinstance(v, str):
            v = {"auto": LAYOUT_AUTO, "csr": LAYOUT_CSR, "sell": LAYOUT_SELL}[v]
        setattr(o, k, v)
    return o


class Matrix:
    """Device matrix handle (bcs_matrix)."""

    def __init__(self, handle, n, nnz):
        self.handle, self.n, self.nnz = handle, n, nnz

    def __del__(self):
        if getattr(self, "handle", None):
            lib.bcs_matrix_free(self.handle)
            self.handle = None

    def info(self):
        return matrix_info(self)


def csr_upload(A, layouts=LAYOUT_CSR, sell_C=32, sell_sigma=256, stores=STORE_F64, stream=None):
    """bcs_csr_upload. A: object with n, rowptr (int64), col (int32), val (float64) host arrays."""
    rp, ci, va = _np(A.rowptr, np.int64), _np(A.col, np.int32), _np(A.val, np.float64)
    h = ctypes.c_void_p()
    _check(lib.bcs_csr_upload(int(A.n), int(rp[-1]), rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                              va.ctypes.data if len(va) else None, layouts, sell_C, sell_sigma, stores,
                              _stream(stream), ctypes.byref(h)), "bcs_csr_upload")
    return Matrix(h.value, int(A.n), int(rp[-1]))


def matrix_info(M):
    n, nnz, pad = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lay, sto = ctypes.c_int(), ctypes.c_int()
    _check(lib.bcs_matrix_info(M.handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(pad), ctypes.byref(lay),
                               ctypes.byref(sto)), "bcs_matrix_info")
    return dict(n=n.value, nnz=nnz.value, sell_padded=pad.value, layouts=lay.value, stores=sto.value)


def matrix_export(M, csr=True, f32=False, bf16=False, sell=False):
    """bcs_matrix_export into fresh numpy arrays."""
    info = matrix_info(M)
    n, nnz, pad = info["n"], info["nnz"], info["sell_padded"]
    out = {}
    args = [None] * 9
    if csr:
        out["rowptr"] = np.zeros(n + 1, np.int32)
        out["col"] = np.zeros(max(nnz, 1), np.int32)
        out["val64"] = np.zeros(max(nnz, 1), np.float64)
        args[0], args[1], args[2] = out["rowptr"].ctypes.data, out["col"].ctypes.data, out["val64"].ctypes.data
    if f32:
        out["val32"] = np.zeros(max(nnz, 1), np.float32)
        args[3] = out["val32"].ctypes.data
    if bf16:
        out["valbf16"] = np.zeros(max(nnz, 1), np.uint16)
        args[4] = out["valbf16"].ctypes.data
    if sell:
        ns = (n + 31) // 32
        out["perm"] = np.zeros(max(n, 1), np.int32)
        out["slice_ptr"] = np.zeros(ns + 1, np.int64)
        out["scol"] = np.zeros(max(pad, 1), np.int32)
        out["sval64"] = np.zeros(max(pad, 1), np.float64)
        args[5], args[6] = out["perm"].ctypes.data, out["slice_ptr"].ctypes.data
        args[7], args[8] = out["scol"].ctypes.data, out["sval64"].ctypes.data
    _check(lib.bcs_matrix_export(M.handle, *args), "bcs_matrix_export")
    for k in ["col", "val64", "val32", "valbf16"]:
        if k in out:
            out[k] = out[k][:nnz]
    if sell:
        out["perm"] = out["perm"][:n]
        out["scol"], out["sval64"] = out["scol"][:pad], out["sval64"][:pad]
    return out


def spmv(M, x, y, layout=LAYOUT_CSR, store=STORE_F64, threads_per_row=0, stream=None):
    """bcs_spmv: y = A x on the device (x, y torch CUDA tensors, float64 or float32)."""
    import torch
    _dvec(x, M.n, "x", ("float64", "float32"))
    _dvec(y, M.n, "y", (str(x.dtype).replace("torch.", ""),))
    f32 = x.dtype == torch.float32
    _check(lib.bcs_spmv(M.handle, layout, store, _ptr(x), _ptr(y), int(f32), threads_per_row, _stream(stream)),
           "bcs_spmv")
    return y


def dot(x, y, stream=None):
    """bcs_dot: correctly rounded (x, y) of two torch CUDA tensors (float64 or float32)."""
    import torch
    _dvec(x, None, "x", ("float64", "float32"))
    _dvec(y, x.numel(), "y", (str(x.dtype).replace("torch.", ""),))
    out = ctypes.c_double()
    _check(lib.bcs_dot(x.numel(), _ptr(x), _ptr(y), int(x.dtype == torch.float32), ctypes.byref(out),
                       _stream(stream)), "bcs_dot")
    return out.value


def dot_noalloc(x, y, out, stream=None):
    """bcs_dot_noalloc: (x, y) of two torch CUDA tensors into the one-element float64 CUDA
    tensor `out`, asynchronously, with no device allocation."""
    import torch
    _dvec(x, None, "x", ("float64", "float32"))
    _dvec(y, x.numel(), "y", (str(x.dtype).replace("torch.", ""),))
    _dvec(out, 1, "out")
    _check(lib.bcs_dot_noalloc(x.numel(), _ptr(x), _ptr(y), int(x.dtype == torch.float32), _ptr(out),
                               _stream(stream)), "bcs_dot_noalloc")
    return out


class Solver:
    """Solver handle (bcs_solver)."""

    def __init__(self, M, kind, tol, maxit, opts):
        self.M = M  # keeps the matrix alive
        self.opts = opts
        self.handle = None
        h = ctypes.c_void_p()
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        _check(lib.bcs_solver_create(M.handle, k, float(tol), int(maxit), ctypes.byref(opts), ctypes.byref(h)),
               "bcs_solver_create")
        self.handle = h.value

    def __del__(self):
        if getattr(self, "handle", None):
            lib.bcs_solver_destroy(self.handle)
            self.handle = None


def solver_create(M, kind="p-BiCGSafe", tol=1e-10, maxit=10000, **kw):
    return Solver(M, kind, tol, maxit, options(**kw))


def solve(S, b, x, stream=None):
    """bcs_solve with device vectors b, x (x holds x_0 on entry). Returns the result as a dict."""
    _dvec(b, S.M.n, "b")
    _dvec(x, S.M.n, "x")
    r = Result()
    code = lib.bcs_solve(S.handle, _ptr(b), _ptr(x), ctypes.byref(r), _stream(stream))
    if code == ERR_ARG or code == ERR_CUDA or code == ERR_OOM:
        raise BcsError(code, "bcs_solve")
    return r.as_dict()


def solve_host(S, b, x, stream=None):
    """bcs_solve_host with numpy float64 b and x (x updated in place)."""
    assert x.dtype == np.float64 and x.flags.c_contiguous
    bb = _np(b, np.float64)
    r = Result()
    code = lib.bcs_solve_host(S.handle, bb.ctypes.data, x.ctypes.data, ctypes.byref(r), _stream(stream))
    if code == ERR_ARG or code == ERR_CUDA or code == ERR_OOM:
        raise BcsError(code, "bcs_solve_host")
    return r.as_dict()


def get_history(S):
    ln = ctypes.c_int()
    _check(lib.bcs_get_history(S.handle, None, 0, ctypes.byref(ln)), "bcs_get_history")
    out = np.zeros(max(ln.value, 1))
    _check(lib.bcs_get_history(S.handle, out.ctypes.data, ln.value, ctypes.byref(ln)), "bcs_get_history")
    return out[:ln.value]


def get_scalars(S):
    ln = ctypes.c_int()
    _check(lib.bcs_get_scalars(S.handle, None, 0, ctypes.byref(ln)), "bcs_get_scalars")
    out = np.zeros(4 * max(ln.value, 1))
    _check(lib.bcs_get_scalars(S.handle, out.ctypes.data, ln.value, ctypes.byref(ln)), "bcs_get_scalars")
    return out[:4 * ln.value].reshape(-1, 4)


def precond_blocks(S):
    """bcs_solver_precond_blocks: the diagonal blocks D and their inverses E of a block-Jacobi
    solver as [n, block_size] numpy arrays (row i: its entries in its block's columns)."""
    bs = ctypes.c_int()
    _check(lib.bcs_solver_precond_blocks(S.handle, None, None, ctypes.byref(bs)), "bcs_solver_precond_blocks")
    n = S.M.n
    D = np.zeros((max(n, 1), bs.value))
    E = np.zeros((max(n, 1), bs.value))
    _check(lib.bcs_solver_precond_blocks(S.handle, D.ctypes.data, E.ctypes.data, None), "bcs_solver_precond_blocks")
    return D[:n], E[:n]


def solve_batched(Ms, bs, xs, kind="p-BiCGSafe", tol=1e-10, maxit=10000, stream=None, **kw):
    """bcs_solve_batched: lists of matrices and device vectors. Returns (worst status, list of result dicts)."""
    n = len(Ms)
    if len(bs) != n or len(xs) != n:
        raise ValueError("one b and one x per system")
    for k, (m, b, x) in enumerate(zip(Ms, bs, xs)):
        _dvec(b, m.n, "b[%d]" % k)
        _dvec(x, m.n, "x[%d]" % k)
    opts = options(**kw)
    H = (ctypes.c_void_p * n)(*[m.handle for m in Ms])
    B = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    R = (Result * n)()
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    code = lib.bcs_solve_batched(n, ctypes.cast(H, ctypes.c_void_p), k, float(tol), int(maxit), ctypes.byref(opts),
                                 ctypes.cast(B, ctypes.c_void_p), ctypes.cast(X, ctypes.c_void_p),
                                 ctypes.cast(R, ctypes.c_void_p), _stream(stream))
    if code == ERR_ARG or code == ERR_CUDA or code == ERR_OOM:
        raise BcsError(code, "bcs_solve_batched")
    return code, [R[i].as_dict() for i in range(n)]


class Batch:
    """Reusable batched solve (bcs_batch): the systems are fixed at creation,
    every solve takes new device vectors b[k], x[k]."""

    def __init__(self, Ms, kind="p-BiCGSafe", tol=1e-10, maxit=10000, **kw):
        self.Ms = list(Ms)  # keeps the matrices alive
        self.handle = None
        n = len(self.Ms)
        opts = options(**kw)
        H = (ctypes.c_void_p * n)(*[m.handle for m in self.Ms])
        h = ctypes.c_void_p()
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        _check(lib.bcs_batch_create(n, ctypes.cast(H, ctypes.c_void_p), k, float(tol), int(maxit), ctypes.byref(opts),
                                    ctypes.byref(h)), "bcs_batch_create")
        self.handle = h.value

    def solve(self, bs, xs, stream=None):
        """Returns (worst status, list of result dicts)."""
        n = len(self.Ms)
        if len(bs) != n or len(xs) != n:
            raise ValueError("one b and one x per system")
        for k, (m, b, x) in enumerate(zip(self.Ms, bs, xs)):
            _dvec(b, m.n, "b[%d]" % k)
            _dvec(x, m.n, "x[%d]" % k)
        B = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
        X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
        R = (Result * n)()
        code = lib.bcs_batch_solve(self.handle, ctypes.cast(B, ctypes.c_void_p), ctypes.cast(X, ctypes.c_void_p),
                                   ctypes.cast(R, ctypes.c_void_p), _stream(stream))
        if code == ERR_ARG or code == ERR_CUDA or code == ERR_OOM:
            raise BcsError(code, "bcs_batch_solve")
        return code, [R[i].as_dict() for i in range(n)]

    def __del__(self):
        if getattr(self, "handle", None):
            lib.bcs_batch_destroy(self.handle)
            self.handle = None


def autotune(M, kind="p-BiCGSafe", precision="fp64", iters=20, stream=None):
    """bcs_autotune: times every layout / lanes-per-row candidate of the persistent solver on M and
    records the fastest in M for that precision.  Returns (best, list of measured candidates)."""
    E = (TuneEntry * 8)()
    cnt = ctypes.c_int()
    best = TuneEntry()
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib.bcs_autotune(M.handle, k, _precision(precision), int(iters), ctypes.cast(E, ctypes.c_void_p), 8,
                            ctypes.byref(cnt), ctypes.byref(best), _stream(stream)), "bcs_autotune")
    return best.as_dict(), [E[i].as_dict() for i in range(min(cnt.value, 8))]


def autotune_sell_sigma(M, kind="p-BiCGSafe", precision="fp64", sigmas=(32, 128, 256, 1024, 4096), iters=20,
                        tuned=True, stream=None):
    """bcs_autotune_sell_sigma: times the SELL layout built with each sorting window sigma, on copies of M
    (M itself is not modified).  Returns (best sigma, {sigma: us per iteration}, a new Matrix with M's
    layouts and the SELL layout at the best sigma, or None when tuned is False)."""
    sig = np.ascontiguousarray(sigmas, dtype=np.int32)
    us = np.zeros(len(sig), dtype=np.float64)
    best = ctypes.c_int()
    h = ctypes.c_void_p()
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib.bcs_autotune_sell_sigma(M.handle, k, _precision(precision), int(iters), sig.ctypes.data, len(sig),
                                       us.ctypes.data, ctypes.byref(best), ctypes.byref(h) if tuned else None,
                                       _stream(stream)), "bcs_autotune_sell_sigma")
    T = Matrix(h.value, M.n, M.nnz) if tuned else None
    return best.value, {int(s_): float(t) for s_, t in zip(sig, us)}, T


def batch_autotune(Ms, kind="p-BiCGSafe", iters=20, stream=None, **kw):
    """bcs_batch_autotune: returns (keyword options for Batch / solve_batched, measured candidates)."""
    n = len(Ms)
    H = (ctypes.c_void_p * n)(*[m.handle for m in Ms])
    opts = options(**kw)
    out = Options()
    E = (TuneEntry * 16)()
    cnt = ctypes.c_int()
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(lib.bcs_batch_autotune(n, ctypes.cast(H, ctypes.c_void_p), k, ctypes.byref(opts), int(iters),
                                  ctypes.cast(E, ctypes.c_void_p), 16, ctypes.byref(cnt), ctypes.byref(out),
                                  _stream(stream)), "bcs_batch_autotune")
    best = dict(kw)
    best.update(threads_per_row=out.threads_per_row, ctas_per_sm=out.ctas_per_sm)
    return best, [E[i].as_dict() for i in range(min(cnt.value, 16))]


# ---- row-partitioned solve (include/bcs_dist.h) ------------------------------------------------

def partition_rows(A, nparts):
    """bcs_partition_rows: contiguous row blocks balanced by nnz + n; returns int64 bounds[nparts+1]."""
    rp = _np(A.rowptr, np.int64)
    out = np.zeros(nparts + 1, dtype=np.int64)
    _check(lib.bcs_partition_rows(int(A.n), rp.ctypes.data, int(nparts), out.ctypes.data), "bcs_partition_rows")
    return out


def halo_plan(A, bounds, rank):
    """bcs_halo_plan: rank's local columns (offsets from its first row: left halo negative, right halo
    from npad = its rows rounded up to 32), halo columns and send list."""
    rp, ci = _np(A.rowptr, np.int64), _np(A.col, np.int32)
    bd = _np(bounds, np.int64)
    nparts = len(bd) - 1
    nl, nr, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    args = [int(A.n), rp.ctypes.data, ci.ctypes.data if len(ci) else None, nparts, bd.ctypes.data, int(rank),
            ctypes.byref(nl), ctypes.byref(nr), ctypes.byref(ns)]
    _check(lib.bcs_halo_plan(*args, None, None, None, None, None, None), "bcs_halo_plan")
    nz = int(rp[bd[rank + 1]] - rp[bd[rank]])
    out = dict(local_col=np.zeros(max(nz, 1), np.int32), left=np.zeros(max(nl.value, 1), np.int64),
               right=np.zeros(max(nr.value, 1), np.int64), send_row=np.zeros(max(ns.value, 1), np.int32),
               send_rank=np.zeros(max(ns.value, 1), np.int32), send_off=np.zeros(max(ns.value, 1), np.int64))
    _check(lib.bcs_halo_plan(*args, *[out[k].ctypes.data for k in ["local_col", "left", "right", "send_row",
                                                                   "send_rank", "send_off"]]), "bcs_halo_plan")
    out["local_col"] = out["local_col"][:nz]
    out["left"], out["right"] = out["left"][:nl.value], out["right"][:nr.value]
    for k in ["send_row", "send_rank", "send_off"]:
        out[k] = out[k][:ns.value]
    out["row0"], out["nloc"] = int(bd[rank]), int(bd[rank + 1] - bd[rank])
    out["npad"] = ((out["nloc"] + 31) // 32) * 32
    return out


class Dist:
    """Row-partitioned solver (bcs_dist): nparts ranks, each a group of CTAs of one cooperative
    launch with its own row block, halo and Krylov vectors.  A: host CSR (n, rowptr, col, val)."""

    def __init__(self, A, nparts, kind="p-BiCGSafe", tol=1e-10, maxit=10000, bounds=None, **kw):
        self.handle = None
        self.n = int(A.n)
        rp, ci, va = _np(A.rowptr, np.int64), _np(A.col, np.int32), _np(A.val, np.float64)
        bd = None if bounds is None else _np(bounds, np.int64)
        opts = options(**kw)
        h = ctypes.c_void_p()
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        _check(lib.bcs_dist_create(self.n, int(rp[-1]), rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                                   va.ctypes.data if len(va) else None, int(nparts),
                                   None if bd is None else bd.ctypes.data, k, float(tol), int(maxit),
                                   ctypes.byref(opts), ctypes.byref(h)), "bcs_dist_create")
        self.handle = h.value
        self.nparts = int(nparts)

    def solve(self, b, x, stream=None):
        _dvec(b, self.n, "b")
        _dvec(x, self.n, "x")
        r = Result()
        code = lib.bcs_dist_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(r), _stream(stream))
        if code == ERR_ARG or code == ERR_CUDA or code == ERR_OOM:
            raise BcsError(code, "bcs_dist_solve")
        return r.as_dict()

    def history(self):
        ln = ctypes.c_int()
        _check(lib.bcs_dist_get_history(self.handle, None, 0, ctypes.byref(ln)), "bcs_dist_get_history")
        out = np.zeros(max(ln.value, 1))
        _check(lib.bcs_dist_get_history(self.handle, out.ctypes.data, ln.value, ctypes.byref(ln)),
               "bcs_dist_get_history")
        return out[:ln.value]

    def scalars(self):
        ln = ctypes.c_int()
        _check(lib.bcs_dist_get_scalars(self.handle, None, 0, ctypes.byref(ln)), "bcs_dist_get_scalars")
        out = np.zeros(4 * max(ln.value, 1))
        _check(lib.bcs_dist_get_scalars(self.handle, out.ctypes.data, ln.value, ctypes.byref(ln)),
               "bcs_dist_get_scalars")
        return out[:4 * ln.value].reshape(-1, 4)

    def info(self, rank):
        v = [ctypes.c_int64() for _ in range(5)]
        c = ctypes.c_int()
        _check(lib.bcs_dist_info(self.handle, int(rank), *[ctypes.byref(t) for t in v], ctypes.byref(c)),
               "bcs_dist_info")
        return dict(row0=v[0].value, nloc=v[1].value, nleft=v[2].value, nright=v[3].value, nsend=v[4].value,
                    ctas=c.value)

    def __del__(self):
        if getattr(self, "handle", None):
            lib.bcs_dist_destroy(self.handle)
            self.handle = None


DIST_HANDLE_BYTES = 64


class DistRank(Dist):
    """One rank of a partitioned solve with one process per GPU (bcs_dist_rank_*): create on every
    process, exchange export_handle() bytes (for example with torch.distributed.all_gather_object),
    connect(handles in rank order), then solve() on every process with full-length b and x."""

    def __init__(self, A, nparts, rank, kind="p-BiCGSafe", tol=1e-10, maxit=10000, bounds=None, **kw):
        self.handle = None
        self.n = int(A.n)
        rp, ci, va = _np(A.rowptr, np.int64), _np(A.col, np.int32), _np(A.val, np.float64)
        bd = None if bounds is None else _np(bounds, np.int64)
        opts = options(**kw)
        h = ctypes.c_void_p()
        k = KINDS[kind] if isinstance(kind, str) else int(kind)
        _check(lib.bcs_dist_rank_create(self.n, int(rp[-1]), rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                                        va.ctypes.data if len(va) else None, int(nparts),
                                        None if bd is None else bd.ctypes.data, int(rank), k, float(tol), int(maxit),
                                        ctypes.byref(opts), ctypes.byref(h)), "bcs_dist_rank_create")
        self.handle = h.value
        self.nparts, self.rank = int(nparts), int(rank)

    def export_handle(self):
        buf = ctypes.create_string_buffer(DIST_HANDLE_BYTES)
        _check(lib.bcs_dist_rank_export(self.handle, buf), "bcs_dist_rank_export")
        return buf.raw

    def connect(self, handles):
        if len(handles) != self.nparts or any(len(h) != DIST_HANDLE_BYTES for h in handles):
            raise ValueError("one %d-byte handle per rank" % DIST_HANDLE_BYTES)
        blob = ctypes.create_string_buffer(b"".join(handles), DIST_HANDLE_BYTES * self.nparts)
        _check(lib.bcs_dist_rank_connect(self.handle, blob), "bcs_dist_rank_connect")
