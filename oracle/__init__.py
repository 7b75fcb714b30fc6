"""Python access to the plain FP64 C oracle (ctypes).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline / reference legs may import this package; the CUDA
library never calls it and has no fallback to it.

`build()` compiles oracle/mrcg_oracle.c with gcc into oracle/_build/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrcg_oracle.c")
_HDR = os.path.join(_HERE, "mrcg_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")

OK, ERR_INVALID, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_MAXITER, ERR_NONFINITE = range(6)
MCG_IDENTITY, MCG_JACOBI, MCG_SMW, MCG_ILU0, MCG_SMW_ILU0 = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "NOT_SPD", 3: "BREAKDOWN", 4: "MAXITER", 5: "NONFINITE"}


def _build_one(out, extra):
    os.makedirs(os.path.dirname(out), exist_ok=True)
    stale = (not os.path.exists(out)) or any(os.path.getmtime(p) > os.path.getmtime(out) for p in (_SRC, _HDR))
    if stale:
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the serial oracle (the pinned one) and its all-core build for
    the CPU baseline (the same source with -fopenmp); returns the serial
    library's path."""
    if force:
        for p in (_OUT, _OUT_OMP):
            if os.path.exists(p):
                os.remove(p)
    _build_one(_OUT_OMP, ["-fopenmp"])
    return _build_one(_OUT, [])


class _Ilu(C.Structure):
    _fields_ = [("n", C.c_int64), ("block", C.c_int64), ("lrow", C.c_void_p), ("urow", C.c_void_p),
                ("lcol", C.c_void_p), ("ucol", C.c_void_p), ("lval", C.c_void_p), ("uval", C.c_void_p)]


class _System(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("val", C.c_void_p),
                ("k", C.c_int32), ("V", C.c_void_p), ("lam", C.c_void_p), ("ilu", C.POINTER(_Ilu))]


class _Info(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("restarts", C.c_int32), ("inner_iters_total", C.c_int64),
                ("prec_calls", C.c_int64), ("true_relres", C.c_double), ("history_len", C.c_int32),
                ("status", C.c_int32)]


PREC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                      C.c_int64, C.POINTER(C.c_int64))

_lib = None
_lib_omp = None


def lib(threads: bool = False):
    """The serial oracle library, or (threads=True) its all-core OpenMP build,
    which the benchmark's CPU baseline times (same arithmetic, the length-n
    loops split over the cores)."""
    global _lib, _lib_omp
    if threads:
        if _lib_omp is None:
            build()
            _lib_omp = _declare(C.CDLL(_OUT_OMP))
        return _lib_omp
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def threads_available() -> int:
    """Cores the all-core build may use: OMP_NUM_THREADS if set, else the
    process's CPU affinity."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env and env.isdigit():
        return int(env)
    return len(os.sched_getaffinity(0))


def _declare(L):
    """Argument and result types of the C entry points."""
    P = C.c_void_p
    L.orc_csr_spmv.argtypes = [C.POINTER(_System), P, P]
    L.orc_mmr_apply.argtypes = [C.POINTER(_System), P, P, P, C.POINTER(C.c_int64)]
    L.orc_mmr_diag.argtypes = [C.POINTER(_System), P]
    L.orc_mcg_apply.argtypes = [C.POINTER(_System), C.c_int, P, P, P]
    L.orc_mcg_apply.restype = C.c_int
    L.orc_cg.argtypes = [C.POINTER(_System), C.c_int, P, P, C.c_double, C.c_int64,
                            C.POINTER(C.c_int64), P]
    L.orc_cg.restype = C.c_int
    L.orc_minres.argtypes = [C.POINTER(_System), P, P, PREC_FN, P, C.c_double, C.c_int32,
                                C.c_int64, C.c_double, P, P, C.c_int32, C.POINTER(_Info)]
    L.orc_minres.restype = C.c_int
    L.orc_minres_cg.argtypes = [C.POINTER(_System), C.c_int, P, P, C.c_double, C.c_double,
                                   C.c_int64, C.c_int32, C.c_double, P, P, C.c_int32, C.POINTER(_Info)]
    L.orc_minres_cg.restype = C.c_int
    L.orc_abs_2x2.argtypes = [C.c_double, C.c_double, C.c_double, P, P, P]
    L.orc_true_relres.argtypes = [C.POINTER(_System), P, P, P]
    L.orc_true_relres.restype = C.c_double
    L.orc_ilu0_factor.argtypes = [C.POINTER(_System), C.c_int64, C.POINTER(_Ilu)]
    L.orc_ilu0_factor.restype = C.c_int
    L.orc_ilu0_free.argtypes = [C.POINTER(_Ilu)]
    L.orc_ilu0_free.restype = None
    L.orc_ilu0_apply.argtypes = [C.POINTER(_Ilu), P, P]
    L.orc_ilu0_apply.restype = None
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class System:
    """Holds contiguous copies of (A, V_hat, Lambda_hat) for the C oracle.

    V is given n x k (rows = unknowns); it is stored column-major.
    """

    def __init__(self, rowptr, colind, val, V=None, lam=None):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.colind = np.ascontiguousarray(colind, dtype=np.int32)
        self.val = _f64(val)
        self.n = len(self.rowptr) - 1
        if V is None or lam is None or np.size(lam) == 0:
            self.k = 0
            self.Vc = np.zeros(1)
            self.lam = np.zeros(1)
        else:
            V = np.asarray(V, dtype=np.float64).reshape(self.n, -1)
            self.k = V.shape[1]
            self.Vc = np.ascontiguousarray(V.T)
            self.lam = _f64(lam)
        self._s = _System(self.n, self.rowptr.ctypes.data, self.colind.ctypes.data, self.val.ctypes.data,
                          self.k, self.Vc.ctypes.data, self.lam.ctypes.data, None)
        self._ilu = None

    def set_ilu0(self, block=None):
        """Factor A by block-Jacobi ILU(0) (diagonal blocks of `block` rows; None:
        one block) for the MCG_ILU0 / MCG_SMW_ILU0 inner preconditioners.
        Returns the status (OK or ERR_BREAKDOWN on a zero pivot)."""
        self.clear_ilu0()
        f = _Ilu()
        st = lib().orc_ilu0_factor(C.byref(self._s), int(block or self.n), C.byref(f))
        if st == OK:
            self._ilu = f
            self._s.ilu = C.pointer(self._ilu)
        return st

    def clear_ilu0(self):
        if self._ilu is not None:
            self._s.ilu = None
            lib().orc_ilu0_free(C.byref(self._ilu))
            self._ilu = None

    def __del__(self):
        try:
            self.clear_ilu0()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def ilu0_factors(self):
        """(L, U) of the current factorisation as dense arrays (small n only):
        L unit lower triangular, U upper triangular with its diagonal."""
        f = self._ilu
        n = self.n
        L = np.eye(n)
        U = np.zeros((n, n))
        lrow = np.ctypeslib.as_array(C.cast(f.lrow, C.POINTER(C.c_int64)), shape=(n + 1,))
        urow = np.ctypeslib.as_array(C.cast(f.urow, C.POINTER(C.c_int64)), shape=(n + 1,))
        nl, nu = int(lrow[n]), int(urow[n])
        lcol = np.ctypeslib.as_array(C.cast(f.lcol, C.POINTER(C.c_int32)), shape=(max(nl, 1),))
        ucol = np.ctypeslib.as_array(C.cast(f.ucol, C.POINTER(C.c_int32)), shape=(max(nu, 1),))
        lval = np.ctypeslib.as_array(C.cast(f.lval, C.POINTER(C.c_double)), shape=(max(nl, 1),))
        uval = np.ctypeslib.as_array(C.cast(f.uval, C.POINTER(C.c_double)), shape=(max(nu, 1),))
        for i in range(n):
            for p in range(int(lrow[i]), int(lrow[i + 1])):
                L[i, lcol[p]] = lval[p]
            for p in range(int(urow[i]), int(urow[i + 1])):
                U[i, ucol[p]] = uval[p]
        return L, U

    def ilu0_apply(self, r):
        r = _f64(r); out = np.empty(self.n)
        lib().orc_ilu0_apply(C.byref(self._ilu), r.ctypes.data, out.ctypes.data)
        return out

    @classmethod
    def from_problem(cls, p):
        return cls(p.rowptr, p.colind, p.val, p.V, p.lam)

    @property
    def ptr(self):
        return C.byref(self._s)

    def spmv(self, x):
        x = _f64(x); y = np.empty(self.n)
        lib().orc_csr_spmv(self.ptr, x.ctypes.data, y.ctypes.data)
        return y

    def mmr_apply(self, u, count_flops=False):
        u = _f64(u); out = np.empty(self.n); t = np.empty(max(self.k, 1)); fl = C.c_int64(0)
        lib().orc_mmr_apply(self.ptr, u.ctypes.data, out.ctypes.data, t.ctypes.data, C.byref(fl))
        return (out, fl.value) if count_flops else out

    def mmr_diag(self):
        d = np.empty(self.n)
        lib().orc_mmr_diag(self.ptr, d.ctypes.data)
        return d

    def mcg_apply(self, r, mcg):
        """M_cg^{-1} r (identity, Jacobi on M_mr, or the MINRES-CG* form).  Returns (out, status)."""
        r = _f64(r); out = np.empty(self.n); work = np.empty(self.n + self.k + 1)
        st = lib().orc_mcg_apply(self.ptr, mcg, r.ctypes.data, out.ctypes.data, work.ctypes.data)
        return out, st

    def cg(self, y, tol, maxit, mcg=MCG_IDENTITY):
        """Inner CG on M_mr z = y.  Returns (z, iters, status)."""
        y = _f64(y); z = np.empty(self.n); it = C.c_int64(0)
        work = np.empty(5 * self.n + self.k + 1)
        st = lib().orc_cg(self.ptr, mcg, y.ctypes.data, z.ctypes.data, tol, int(maxit), C.byref(it),
                          work.ctypes.data)
        return z, it.value, st

    def true_relres(self, b, x):
        b = _f64(b); x = _f64(x); w = np.empty(self.n)
        return lib().orc_true_relres(self.ptr, b.ctypes.data, x.ctypes.data, w.ctypes.data)


@dataclass
class SolveResult:
    x: np.ndarray
    status: int
    outer_iters: int
    restarts: int
    inner_iters_total: int
    prec_calls: int
    true_relres: float
    relres_history: np.ndarray
    eta_history: np.ndarray


def _result(x, info, hr, he):
    L = info.history_len
    return SolveResult(x, info.status, info.outer_iters, info.restarts, info.inner_iters_total,
                       info.prec_calls, info.true_relres, hr[:L].copy(), he[:L].copy())


def minres_cg(sys: System, b, x0=None, outer_tol=1e-10, inner_tol=1e-3, max_iters=10**9,
              max_outer=200, restart_factor=0.5, mcg=MCG_IDENTITY, hist_cap=4096, threads=False) -> SolveResult:
    """Alg. 1: outer preconditioned MINRES, inner CG on M_mr (all FP64).
    threads=True runs the all-core build (CPU baseline timing only)."""
    b = _f64(b)
    x = np.zeros(sys.n) if x0 is None else _f64(x0).copy()
    hr = np.zeros(hist_cap); he = np.zeros(hist_cap); info = _Info()
    lib(threads).orc_minres_cg(sys.ptr, mcg, b.ctypes.data, x.ctypes.data, outer_tol, inner_tol, int(max_iters),
                        int(max_outer), restart_factor, hr.ctypes.data, he.ctypes.data, hist_cap,
                        C.byref(info))
    return _result(x, info, hr, he)


def minres(sys: System, b, prec, x0=None, outer_tol=1e-10, max_outer=200, max_inner_total=10**9,
           restart_factor=0.5, hist_cap=4096) -> SolveResult:
    """Generic preconditioned MINRES with a Python preconditioner z = prec(v).

    prec returns z, or (z, iterations_used).
    """
    b = _f64(b)
    x = np.zeros(sys.n) if x0 is None else _f64(x0).copy()
    n = sys.n

    def _cb(ctx, nn, vp, zp, budget, itp):
        v = np.ctypeslib.as_array(vp, shape=(n,))
        out = prec(v.copy())
        its = 1
        if isinstance(out, tuple):
            out, its = out
        np.ctypeslib.as_array(zp, shape=(n,))[:] = out
        itp[0] = its
        return OK

    cb = PREC_FN(_cb)
    hr = np.zeros(hist_cap); he = np.zeros(hist_cap); info = _Info()
    lib().orc_minres(sys.ptr, b.ctypes.data, x.ctypes.data, cb, None, outer_tol, int(max_outer),
                     int(max_inner_total), restart_factor, hr.ctypes.data, he.ctypes.data, hist_cap,
                     C.byref(info))
    return _result(x, info, hr, he)


def negative_eigenpairs_dense(rowptr, colind, val):
    """Setup stage 2 by its definition (Sec. 2): every eigenpair of the
    symmetric A with a negative eigenvalue, from a dense symmetric
    eigendecomposition (numpy.linalg.eigh; small n only).  Returns (V n x k,
    lam[k] ascending, all eigenvalues)."""
    n = len(rowptr) - 1
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(int(rowptr[i]), int(rowptr[i + 1])):
            A[i, int(colind[p])] += float(val[p])
    w, Q = np.linalg.eigh(0.5 * (A + A.T))
    k = int(np.sum(w < 0.0))
    return Q[:, :k].copy(), w[:k].copy(), w


def abs_2x2(a, b, c):
    """Sec. 1 2x2 replacement.  Returns (block[2,2], (l1, l2), (cs, sn))."""
    out = np.zeros(3); eig = np.zeros(2); rot = np.zeros(2)
    lib().orc_abs_2x2(float(a), float(b), float(c), out.ctypes.data, eig.ctypes.data, rot.ctypes.data)
    return np.array([[out[0], out[1]], [out[1], out[2]]]), tuple(eig), tuple(rot)
