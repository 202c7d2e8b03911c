"""TEST INFRASTRUCTURE — the CPU oracle.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library in
``paper_2108_10591_gb300``) never calls it; the two share no code.

``bicgsafe_oracle.c`` is a plain, single-threaded FP64 implementation of the
paper's Algorithms 3 (ssBiCGSafe2), 4 (p-BiCGSafe) and 5 (p-BiCGSafe-rr),
statement by statement; ``exact.py`` runs the same algorithms in exact
rational arithmetic for tiny systems.  This module is a ctypes wrapper.

Pins (tests/test_oracle_*.py): dense LU solutions, exact-arithmetic finite
termination and plain == pipelined == rr equivalence (Section 3, the claim
that Alg. 4 is an equivalent rewrite of Alg. 3), the definitions the
recurrences maintain (s=Ar, q=Ao, w=Au, l=At, g=Ay, r=b-Ax; Eqs. (s)-(g)),
zeta/eta as the least-squares minimiser of the associate residual
(Eq. eta&zeta_ssBiCGSafe2), alpha as BiCG's alpha, hand-computed i=0 values
on a 2x2 system (tests/golden/), and SELL/BF16 format invariants.
"""
import ctypes
import os

import numpy as np

from . import build as _build

KINDS = {"ssBiCGSafe2": 0, "p-BiCGSafe": 1, "p-BiCGSafe-rr": 2}
SV = ["x", "r", "rs", "s", "y", "t", "p", "u", "z", "w", "o", "q", "l", "g", "As", "Aw"]
SC = ["alpha", "beta", "zeta", "eta", "a", "b", "c", "d", "e", "f", "g", "h", "r", "rr", "i"]
STATUS = {0: "ok", 1: "not_converged", -1: "err_arg", -3: "breakdown", -5: "nonfinite"}


class _Opts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("rr_m", ctypes.c_int), ("rr_M", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("dump_iter", ctypes.c_int), ("dump_phase", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("status", ctypes.c_int),
                ("fallbacks", ctypes.c_int), ("rr_steps", ctypes.c_int),
                ("rel_res_recursive", ctypes.c_double), ("rel_res_true", ctypes.c_double),
                ("r0_norm", ctypes.c_double)]


_LIBS = {}
_DP = ctypes.POINTER(ctypes.c_double)
_MV_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, _DP, _DP)
_DOT_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, _DP, _DP)


def lib(parallel=False):
    """The oracle library: the single-threaded parity build, or (parallel=True) the same source
    built with OpenMP, used only to time the CPU baseline on every host core."""
    if parallel not in _LIBS:
        path = _build.build(parallel=parallel)
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.orc_spmv.argtypes = [ctypes.c_int64, P, P, P, P, P]
        L.orc_spmv.restype = None
        L.orc_dot.argtypes = [ctypes.c_int64, P, P]
        L.orc_dot.restype = ctypes.c_double
        L.orc_true_residual.argtypes = [ctypes.c_int64, P, P, P, P, P]
        L.orc_true_residual.restype = ctypes.c_double
        L.orc_solve.argtypes = [ctypes.c_int64, P, P, P, P, P, ctypes.POINTER(_Opts),
                                P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), P, P, P,
                                ctypes.POINTER(_Result)]
        L.orc_solve.restype = ctypes.c_int
        L.orc_sell_build.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int, ctypes.c_int, P, P, P, P]
        L.orc_sell_build.restype = ctypes.c_int64
        L.orc_to_bf16.argtypes = [ctypes.c_int64, P, P]
        L.orc_to_bf16.restype = None
        L.orc_dot_limbs.argtypes = []
        L.orc_dot_limbs.restype = ctypes.c_int
        L.orc_dot_partial.argtypes = [ctypes.c_int64, P, P, P]
        L.orc_dot_partial.restype = ctypes.c_int
        L.orc_dot_merge.argtypes = [P, P]
        L.orc_dot_merge.restype = None
        L.orc_dot_round.argtypes = [P]
        L.orc_dot_round.restype = ctypes.c_double
        L.orc_solve_hooked.argtypes = [ctypes.c_int64, P, P, ctypes.POINTER(_Opts), _MV_FN, _DOT_FN, P, P,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_int), P, ctypes.POINTER(_Result)]
        L.orc_solve_hooked.restype = ctypes.c_int
        L.orc_bjacobi_blocks.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int, P, P]
        L.orc_bjacobi_blocks.restype = ctypes.c_int
        L.orc_bjacobi_apply.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P]
        L.orc_bjacobi_apply.restype = None
        L.orc_solve_bjacobi.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int, P, P, ctypes.POINTER(_Opts),
                                        P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), P, ctypes.POINTER(_Result)]
        L.orc_solve_bjacobi.restype = ctypes.c_int
        _LIBS[parallel] = L
    return _LIBS[parallel]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(A):
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, ci, va


def spmv(A, x, parallel=False):
    """y = A x (rows summed sequentially with fma)."""
    rp, ci, va = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(A.n, dtype=np.float64)
    lib(parallel).orc_spmv(A.n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def dot(x, y, parallel=False):
    """Correctly rounded inner product (exact sum of exact products, rounded once)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib(parallel).orc_dot(len(x), _p(x), _p(y))


def true_residual(A, b, x):
    rp, ci, va = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_true_residual(A.n, _p(rp), _p(ci), _p(va), _p(b), _p(x))


def solve(A, b, x0=None, kind="p-BiCGSafe", tol=1e-10, maxit=10000, rr_m=100, rr_M=None,
          max_restarts=0, hist_cap=None, dump_iter=-1, dump_phase=0, parallel=False):
    """Run Algorithm 3/4/5 (see bicgsafe_oracle.c).  Returns a dict with x,
    hist (sqrt(r_i)/||r_0|| per stop test), scalars (alpha, beta, zeta, eta per
    iteration of the first run), result fields and, when dump_iter >= 0, the
    state dump (dict of vectors) and dumped scalars."""
    rp, ci, va = _csr(A)
    n = A.n
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    o = _Opts(KINDS[kind] if isinstance(kind, str) else int(kind), tol, maxit, rr_m,
              maxit + 1 if rr_M is None else rr_M, max_restarts, dump_iter, dump_phase)
    cap = (maxit + 1) * (max_restarts + 1) + 4 if hist_cap is None else hist_cap
    hist = np.zeros(cap)
    scal = np.zeros(4 * cap)
    hl = ctypes.c_int(0)
    res = _Result()
    state = np.zeros(len(SV) * max(n, 1)) if dump_iter >= 0 else None
    sdump = np.zeros(len(SC)) if dump_iter >= 0 else None
    st = lib(parallel).orc_solve(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), ctypes.byref(o), _p(hist), cap,
                         ctypes.byref(hl), _p(scal), None if state is None else _p(state),
                         None if sdump is None else _p(sdump), ctypes.byref(res))
    out = dict(x=x, hist=hist[:hl.value].copy(), status=st, status_name=STATUS.get(st, str(st)),
               iterations=res.iterations, restarts=res.restarts, fallbacks=res.fallbacks,
               rr_steps=res.rr_steps, rel_res_recursive=res.rel_res_recursive,
               rel_res_true=res.rel_res_true, r0_norm=res.r0_norm)
    k = min(res.iterations + 1, cap)
    out["scalars"] = scal[:4 * k].reshape(-1, 4).copy()
    if dump_iter >= 0:
        out["state"] = {name: state[i * n:(i + 1) * n].copy() for i, name in enumerate(SV)}
        out["dump_scalars"] = {name: sdump[i] for i, name in enumerate(SC)}
    return out


def sell_build(A, C=32, sigma=256):
    """SELL-C-sigma arrays (perm, slice_ptr, col, val) built by the oracle."""
    rp, ci, va = _csr(A)
    n = A.n
    ns = (n + C - 1) // C
    perm = np.zeros(max(n, 1), dtype=np.int32)
    sp = np.zeros(ns + 1, dtype=np.int64)
    L = lib()
    total = L.orc_sell_build(n, _p(rp), _p(ci), _p(va), C, sigma, _p(perm), _p(sp), None, None)
    scol = np.zeros(max(total, 1), dtype=np.int32)
    sval = np.zeros(max(total, 1), dtype=np.float64)
    L.orc_sell_build(n, _p(rp), _p(ci), _p(va), C, sigma, _p(perm), _p(sp), _p(scol), _p(sval))
    return dict(perm=perm[:n], slice_ptr=sp, col=scol[:total], val=sval[:total])


def to_bf16_bits(v):
    """Round-to-nearest-even FP64 -> BF16, as uint16 bit patterns."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(len(v), dtype=np.uint16)
    lib().orc_to_bf16(len(v), _p(v), _p(out))
    return out


# ---- a row-partitioned run (orc_solve_hooked) --------------------------------------------------

def dot_partial(x, y):
    """Exact partial sum of x_i y_i as integer limbs (uint64 array) and whether every operand was
    finite; partials of disjoint row blocks merge exactly (dot_merge) and round once (dot_round)."""
    L = lib()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    limbs = np.zeros(L.orc_dot_limbs(), dtype=np.uint64)
    ok = L.orc_dot_partial(len(x), _p(x), _p(y), _p(limbs))
    return limbs, bool(ok)


def dot_merge(partials):
    """Exact sum of partials (in the given order; the sum is exact, so any order gives it)."""
    L = lib()
    acc = np.zeros(L.orc_dot_limbs(), dtype=np.uint64)
    for p in partials:
        p = np.ascontiguousarray(p, dtype=np.uint64)
        L.orc_dot_merge(_p(acc), _p(p))
    return acc


def dot_round(limbs):
    limbs = np.ascontiguousarray(limbs, dtype=np.uint64)
    return lib().orc_dot_round(_p(limbs))


def solve_hooked(n_local, b, mv, dot, x0=None, kind="p-BiCGSafe", tol=1e-10, maxit=10000, rr_m=100, rr_M=None,
                 max_restarts=0, hist_cap=None):
    """Algorithms 3/4/5 over one block of rows of a partitioned system: mv(x, y) sets y = A x on
    the block's rows and dot(x, y) returns the inner product over all rows (numpy views of the
    block's parts).  Returns the same dict as solve() without the state dump."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n_local) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    errors = []

    def _mv(ctx, xp, yp):
        try:
            mv(np.ctypeslib.as_array(xp, (n_local,)), np.ctypeslib.as_array(yp, (n_local,)))
        except Exception as e:  # noqa: BLE001  (reported after the run)
            errors.append(e)

    def _dot(ctx, xp, yp):
        try:
            return float(dot(np.ctypeslib.as_array(xp, (n_local,)), np.ctypeslib.as_array(yp, (n_local,))))
        except Exception as e:  # noqa: BLE001
            errors.append(e)
            return float("nan")

    mvf, dotf = _MV_FN(_mv), _DOT_FN(_dot)
    o = _Opts(KINDS[kind] if isinstance(kind, str) else int(kind), tol, maxit, rr_m,
              maxit + 1 if rr_M is None else rr_M, max_restarts, -1, 0)
    cap = (maxit + 1) * (max_restarts + 1) + 4 if hist_cap is None else hist_cap
    hist = np.zeros(cap)
    scal = np.zeros(4 * cap)
    hl = ctypes.c_int(0)
    res = _Result()
    st = lib().orc_solve_hooked(n_local, _p(b), _p(x), ctypes.byref(o), mvf, dotf, None, _p(hist), cap,
                                ctypes.byref(hl), _p(scal), ctypes.byref(res))
    if errors:
        raise errors[0]
    k = min(res.iterations + 1, cap)
    return dict(x=x, hist=hist[:hl.value].copy(), status=st, status_name=STATUS.get(st, str(st)),
                iterations=res.iterations, restarts=res.restarts, rr_steps=res.rr_steps,
                rel_res_true=res.rel_res_true, scalars=scal[:4 * k].reshape(-1, 4).copy())


def bjacobi_blocks(A, bs):
    """Diagonal blocks D of A (bs consecutive rows each, the last block ragged) and their inverses
    E by Gauss-Jordan with partial pivoting, as [n, bs] arrays: row i holds its block row's
    entries in the block's columns (zero beyond the block).  Raises ValueError for a singular
    block."""
    rp, ci, va = _csr(A)
    n = A.n
    D = np.zeros((max(n, 1), bs))
    E = np.zeros((max(n, 1), bs))
    st = lib().orc_bjacobi_blocks(n, _p(rp), _p(ci), _p(va), int(bs), _p(D), _p(E))
    if st != 0:
        raise ValueError("singular diagonal block (or bad block size)")
    return D[:n], E[:n]


def bjacobi_apply(M, v, bs):
    """z = M v block by block (M = D or E from bjacobi_blocks)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    z = np.zeros(len(v))
    lib().orc_bjacobi_apply(len(v), int(bs), _p(M), _p(v), _p(z))
    return z


def solve_bjacobi(A, b, bs, x0=None, kind="p-BiCGSafe", tol=1e-10, maxit=10000, rr_m=100, rr_M=None,
                  max_restarts=0, hist_cap=None, parallel=False):
    """Algorithm 3/4/5 with block-Jacobi right preconditioning (see orc_solve_bjacobi): the runs
    on A M^-1 from y_0 = M x_0, x = M^-1 y.  Returns the same dict as solve() without the state
    dump."""
    rp, ci, va = _csr(A)
    n = A.n
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    o = _Opts(KINDS[kind] if isinstance(kind, str) else int(kind), tol, maxit, rr_m,
              maxit + 1 if rr_M is None else rr_M, max_restarts, -1, 0)
    cap = (maxit + 1) * (max_restarts + 1) + 4 if hist_cap is None else hist_cap
    hist = np.zeros(cap)
    scal = np.zeros(4 * cap)
    hl = ctypes.c_int(0)
    res = _Result()
    st = lib(parallel).orc_solve_bjacobi(n, _p(rp), _p(ci), _p(va), int(bs), _p(b), _p(x), ctypes.byref(o), _p(hist), cap,
                                 ctypes.byref(hl), _p(scal), ctypes.byref(res))
    k = min(res.iterations + 1, cap)
    return dict(x=x, hist=hist[:hl.value].copy(), status=st, status_name=STATUS.get(st, str(st)),
                iterations=res.iterations, restarts=res.restarts, fallbacks=res.fallbacks,
                rr_steps=res.rr_steps, rel_res_recursive=res.rel_res_recursive,
                rel_res_true=res.rel_res_true, r0_norm=res.r0_norm,
                scalars=scal[:4 * k].reshape(-1, 4).copy())
