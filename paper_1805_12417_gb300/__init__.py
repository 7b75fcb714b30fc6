"""GB300 (sm_103a) MINRES-CG for sparse symmetric indefinite systems.

Thin ctypes binding of the C ABI in include/mrcg.h (same entry-point names
without the ``mrcg_`` prefix).  It only marshals arguments: every step of the
solve runs in the CUDA library ``libmrcg.so`` built from ``csrc/``.  There is
no CPU fallback; loading fails loudly when the library is missing.

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory); the library detects which.  Device inputs must be complete before a
call (the binding synchronises torch's current stream first).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmrcg.so")

OK, ERR_INVALID, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_MAXITER, ERR_NONFINITE, ERR_CUDA, ERR_OOM = range(8)
FP64, MIXED_FP32, MIXED_BF16M = 0, 1, 2
MCG_IDENTITY, MCG_JACOBI, MCG_SMW, MCG_ILU0, MCG_SMW_ILU0 = 0, 1, 2, 3, 4


class CreateArgs(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("val", C.c_void_p), ("k", C.c_int32), ("V", C.c_void_p), ("lambda_", C.c_void_p),
                ("precision", C.c_int32), ("inner_prec", C.c_int32), ("validate", C.c_int32),
                ("max_outer", C.c_int32), ("restart_factor", C.c_double), ("stream", C.c_void_p),
                ("ilu_block", C.c_int32), ("reserved", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("restarts", C.c_int32), ("inner_iters_total", C.c_int64),
                ("prec_calls", C.c_int64), ("kernel_launches", C.c_int64), ("true_relres", C.c_double), ("solve_ms", C.c_double),
                ("relres_history", C.c_void_p), ("history_cap", C.c_int32), ("history_len", C.c_int32),
                ("status", C.c_int32)]


class EigInfo(C.Structure):
    _fields_ = [("negative_found", C.c_int32), ("rayleigh_ritz_steps", C.c_int32), ("block_spmvs", C.c_int64),
                ("max_residual", C.c_double), ("spectrum_lo", C.c_double), ("spectrum_hi", C.c_double),
                ("seconds", C.c_double), ("status", C.c_int32)]


class ComplexArgs(C.Structure):
    _fields_ = [("n", C.c_int64), ("ke_rowptr", C.c_void_p), ("ke_colind", C.c_void_p), ("ke_val", C.c_void_p),
                ("k_rowptr", C.c_void_p), ("k_colind", C.c_void_p), ("k_val", C.c_void_p),
                ("d_rowptr", C.c_void_p), ("d_colind", C.c_void_p), ("d_val", C.c_void_p),
                ("mass", C.c_void_p), ("gamma_abs", C.c_double), ("k", C.c_int32), ("V", C.c_void_p),
                ("lambda_", C.c_void_p), ("eig_block", C.c_int32), ("precision", C.c_int32),
                ("inner_prec", C.c_int32), ("reserved", C.c_int32), ("stream", C.c_void_p)]


class ComplexInfo(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("s2_iters_total", C.c_int32), ("inner_solves", C.c_int64),
                ("inner_cg_iters", C.c_int64), ("true_relres", C.c_double), ("solve_ms", C.c_double),
                ("status", C.c_int32)]


_lib = None


def lib() -> C.CDLL:
    """Load libmrcg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.mrcg_solver_create.argtypes = [C.POINTER(CreateArgs), C.POINTER(C.c_void_p)]
        L.mrcg_solver_create.restype = C.c_int
        L.mrcg_solve.argtypes = [P, P, P, C.c_double, C.c_double, C.c_int64, C.POINTER(Info)]
        L.mrcg_solve.restype = C.c_int
        L.mrcg_apply_A.argtypes = [P, P, P]
        L.mrcg_apply_A.restype = C.c_int
        L.mrcg_apply_mmr.argtypes = [P, P, P]
        L.mrcg_apply_mmr.restype = C.c_int
        L.mrcg_inner_solve.argtypes = [P, P, P, C.c_double, C.c_int64, C.POINTER(C.c_int64)]
        L.mrcg_inner_solve.restype = C.c_int
        L.mrcg_time_inner_kernels.argtypes = [P, C.c_int32, P]
        L.mrcg_time_inner_kernels.restype = C.c_int
        L.mrcg_launch_config.argtypes = [P, P]
        L.mrcg_launch_config.restype = C.c_int
        L.mrcg_time_inner_graph.argtypes = [P, C.c_int32, C.POINTER(C.c_double)]
        L.mrcg_time_inner_graph.restype = C.c_int
        L.mrcg_fp64_fma_peak.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.mrcg_fp64_fma_peak.restype = C.c_int
        L.mrcg_negative_eigenpairs.argtypes = [C.c_int64, P, P, P, C.c_int32, C.c_double, C.c_int64, C.c_uint64,
                                               C.POINTER(C.c_int32), P, P, C.POINTER(EigInfo)]
        L.mrcg_negative_eigenpairs.restype = C.c_int
        L.mrcg_complex_create.argtypes = [C.POINTER(ComplexArgs), C.POINTER(C.c_void_p)]
        L.mrcg_complex_create.restype = C.c_int
        L.mrcg_complex_negative_count.argtypes = [P]
        L.mrcg_complex_negative_count.restype = C.c_int32
        L.mrcg_complex_solve.argtypes = [P, C.c_double, C.c_double, P, P, P, P, C.c_double, C.c_int32, C.c_int32,
                                         C.c_double, C.c_int32, C.c_double, C.c_double, C.POINTER(ComplexInfo)]
        L.mrcg_complex_solve.restype = C.c_int
        L.mrcg_complex_destroy.argtypes = [P]
        L.mrcg_complex_destroy.restype = None
        L.mrcg_batch_create.argtypes = [C.c_int32, C.POINTER(CreateArgs), C.POINTER(C.c_void_p)]
        L.mrcg_batch_create.restype = C.c_int
        L.mrcg_batched_solve.argtypes = [P, P, P, C.c_double, C.c_double, C.c_int64, C.POINTER(Info)]
        L.mrcg_batched_solve.restype = C.c_int
        L.mrcg_batch_size.argtypes = [P]
        L.mrcg_batch_size.restype = C.c_int32
        L.mrcg_batch_launch_config.argtypes = [P, P]
        L.mrcg_batch_launch_config.restype = C.c_int
        L.mrcg_batch_destroy.argtypes = [P]
        L.mrcg_batch_destroy.restype = None
        L.mrcg_shifted_create.argtypes = [C.POINTER(CreateArgs), C.c_int32, P, P, C.c_int32,
                                          C.POINTER(C.c_void_p)]
        L.mrcg_shifted_create.restype = C.c_int
        L.mrcg_shifted_solve.argtypes = [P, P, P, C.c_double, C.c_double, C.c_int64, C.POINTER(Info)]
        L.mrcg_shifted_solve.restype = C.c_int
        L.mrcg_shifted_columns.argtypes = [P]
        L.mrcg_shifted_columns.restype = C.c_int32
        L.mrcg_shifted_launch_config.argtypes = [P, P]
        L.mrcg_shifted_launch_config.restype = C.c_int
        L.mrcg_shifted_destroy.argtypes = [P]
        L.mrcg_shifted_destroy.restype = None
        L.mrcg_solver_destroy.argtypes = [P]
        L.mrcg_solver_destroy.restype = None
        L.mrcg_status_string.argtypes = [C.c_int]
        L.mrcg_status_string.restype = C.c_char_p
        _lib = L
    return _lib


def _ptr(a):
    """(pointer, keep-alive) for a numpy array or a torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data, a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if a.is_cuda:
            import torch
            torch.cuda.current_stream(a.device).synchronize()
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)}")


def _check_dtype(a, dtype, name):
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError(f"{name} must be {np.dtype(dtype).name}, got {a.dtype}")
    elif hasattr(a, "dtype"):
        import torch
        tmap = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}
        if a.dtype != tmap[dtype]:
            raise TypeError(f"{name} must be {np.dtype(dtype).name}, got {a.dtype}")


def status_string(s: int) -> str:
    return lib().mrcg_status_string(int(s)).decode()


class MrcgError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: {status_string(status)}")
        self.status = status


def solver_create(n, rowptr, colind, val, V=None, lam=None, precision=FP64, inner_prec=MCG_IDENTITY,
                  validate=True, max_outer=0, restart_factor=0.0, stream=None, ilu_block=0) -> int:
    """mrcg_solver_create.  V is n x k (row index = unknown); it is passed
    column-major.  Returns the opaque handle (int)."""
    _check_dtype(rowptr, np.int64, "rowptr"); _check_dtype(colind, np.int32, "colind")
    _check_dtype(val, np.float64, "val")
    keep = []
    k = 0
    Vp = lamp = None
    if V is not None and lam is not None and len(lam) > 0:
        if isinstance(V, np.ndarray):
            V = np.asarray(V, dtype=np.float64).reshape(n, -1)
            k = V.shape[1]
            V = np.ascontiguousarray(V.T)
        else:
            k = V.shape[1]
            V = V.t().contiguous()
        lam = np.ascontiguousarray(lam, dtype=np.float64) if isinstance(lam, (np.ndarray, list)) else lam
        Vp, kv = _ptr(V); lamp, kl = _ptr(lam); keep += [kv, kl]
    rp, k1 = _ptr(rowptr); ci, k2 = _ptr(colind); va, k3 = _ptr(val)
    keep += [k1, k2, k3]
    a = CreateArgs(int(n), int(rowptr[-1]), rp, ci, va, k, Vp, lamp, int(precision), int(inner_prec),
                   1 if validate else 0, int(max_outer), float(restart_factor), stream, int(ilu_block), 0)
    h = C.c_void_p()
    st = lib().mrcg_solver_create(C.byref(a), C.byref(h))
    if st != OK:
        raise MrcgError(st, "mrcg_solver_create")
    return h.value


def solver_destroy(h) -> None:
    lib().mrcg_solver_destroy(h)


@dataclass
class SolveInfo:
    status: int
    outer_iters: int
    restarts: int
    inner_iters_total: int
    prec_calls: int
    kernel_launches: int
    true_relres: float
    solve_ms: float
    relres_history: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def status_name(self):
        return status_string(self.status)


def solve(h, b, x, outer_tol=1e-10, inner_tol=1e-3, max_iters=0, history_cap=512) -> SolveInfo:
    """mrcg_solve: x (in: x0, out: solution) is updated in place."""
    _check_dtype(b, np.float64, "b"); _check_dtype(x, np.float64, "x")
    hist = np.zeros(max(history_cap, 1))
    info = Info()
    info.relres_history = hist.ctypes.data
    info.history_cap = history_cap
    bp, kb = _ptr(b); xp, kx = _ptr(x)
    st = lib().mrcg_solve(h, bp, xp, float(outer_tol), float(inner_tol), int(max_iters), C.byref(info))
    if st in (ERR_INVALID, ERR_CUDA, ERR_OOM):
        raise MrcgError(st, "mrcg_solve")
    return SolveInfo(st, info.outer_iters, info.restarts, info.inner_iters_total, info.prec_calls,
                     info.kernel_launches, info.true_relres, info.solve_ms, hist[: info.history_len].copy())


def apply_A(h, x, y) -> None:
    """mrcg_apply_A: y = A x."""
    xp, kx = _ptr(x); yp, ky = _ptr(y)
    st = lib().mrcg_apply_A(h, xp, yp)
    if st != OK:
        raise MrcgError(st, "mrcg_apply_A")


def apply_mmr(h, u, out) -> None:
    """mrcg_apply_mmr: out = M_mr u in the handle's inner precision."""
    up, ku = _ptr(u); op, ko = _ptr(out)
    st = lib().mrcg_apply_mmr(h, up, op)
    if st != OK:
        raise MrcgError(st, "mrcg_apply_mmr")


def inner_solve(h, y, z, inner_tol=1e-3, max_iters=0):
    """mrcg_inner_solve: z ~ M_mr^{-1} y by the inner CG.  Returns (status, iters)."""
    yp, ky = _ptr(y); zp, kz = _ptr(z)
    it = C.c_int64(0)
    st = lib().mrcg_inner_solve(h, yp, zp, float(inner_tol), int(max_iters), C.byref(it))
    if st in (ERR_INVALID, ERR_CUDA, ERR_OOM):
        raise MrcgError(st, "mrcg_inner_solve")
    return st, it.value


def launch_config(h):
    """mrcg_launch_config: the autotuned launch shape of the inner-CG kernels."""
    cfg = np.zeros(7, dtype=np.int32)
    st = lib().mrcg_launch_config(h, cfg.ctypes.data)
    if st != OK:
        raise MrcgError(st, "mrcg_launch_config")
    return {"step_a_variant": int(cfg[0]), "step_a_grid": int(cfg[1]), "step_b_grid": int(cfg[2]),
            "unroll": int(cfg[3]), "k_bucket": int(cfg[4]), "index_bytes": int(cfg[5]),
            "stages": int(cfg[6])}


def time_inner_kernels(h, iters=20):
    """mrcg_time_inner_kernels: average ms of (step a, step b) of one inner CG iteration."""
    ms = np.zeros(2)
    st = lib().mrcg_time_inner_kernels(h, int(iters), ms.ctypes.data)
    if st != OK:
        raise MrcgError(st, "mrcg_time_inner_kernels")
    return float(ms[0]), float(ms[1])


def time_inner_graph(h, iters=256):
    """mrcg_time_inner_graph: ms of one inner CG iteration inside the solver's own loop."""
    ms = C.c_double(0.0)
    st = lib().mrcg_time_inner_graph(h, int(iters), C.byref(ms))
    if st != OK:
        raise MrcgError(st, "mrcg_time_inner_graph")
    return float(ms.value)


def fp64_fma_peak():
    """mrcg_fp64_fma_peak: (TFLOP/s, ms of the best launch) of FP64 FMAs on the current device."""
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    st = lib().mrcg_fp64_fma_peak(C.byref(tf), C.byref(ms))
    if st != OK:
        raise MrcgError(st, "mrcg_fp64_fma_peak")
    return float(tf.value), float(ms.value)


def negative_eigenpairs(n, rowptr, colind, val, block, tol=1e-11, max_spmv=400000, seed=1):
    """mrcg_negative_eigenpairs: the negative eigenpairs of the CSR matrix A
    (setup stage 2).  Returns (V n x k, lam[k] ascending, info dict); raises
    MrcgError on failure (info is attached to the error as .info)."""
    _check_dtype(rowptr, np.int64, "rowptr"); _check_dtype(colind, np.int32, "colind")
    _check_dtype(val, np.float64, "val")
    V = np.zeros(int(n) * int(block))
    lam = np.zeros(int(block))
    k = C.c_int32(0)
    info = EigInfo()
    rp, k1 = _ptr(rowptr); ci, k2 = _ptr(colind); va, k3 = _ptr(val)
    st = lib().mrcg_negative_eigenpairs(int(n), rp, ci, va, int(block), float(tol), int(max_spmv), int(seed),
                                        C.byref(k), V.ctypes.data, lam.ctypes.data, C.byref(info))
    d = {f: getattr(info, f) for f, _ in EigInfo._fields_}
    if st != OK:
        err = MrcgError(st, "mrcg_negative_eigenpairs")
        err.info = d
        raise err
    kk = int(k.value)
    return V[: int(n) * kk].reshape(kk, int(n)).T.copy(), lam[:kk].copy(), d


class Solver:
    """Owning wrapper of one handle."""

    def __init__(self, n, rowptr, colind, val, V=None, lam=None, **kw):
        self.n = int(n)
        self.h = solver_create(n, rowptr, colind, val, V, lam, **kw)

    @classmethod
    def from_problem(cls, p, **kw):
        return cls(p.n, p.rowptr, p.colind, p.val, p.V, p.lam, **kw)

    def solve(self, b, x=None, **kw):
        if x is None:
            x = np.zeros(self.n) if isinstance(b, np.ndarray) else b.new_zeros(b.shape)
        info = solve(self.h, b, x, **kw)
        return x, info

    def apply_A(self, x, y=None):
        y = np.empty(self.n) if y is None else y
        apply_A(self.h, x, y)
        return y

    def apply_mmr(self, u, out=None):
        out = np.empty(self.n) if out is None else out
        apply_mmr(self.h, u, out)
        return out

    def inner_solve(self, y, z=None, **kw):
        z = np.empty(self.n) if z is None else z
        st, it = inner_solve(self.h, y, z, **kw)
        return z, st, it

    def close(self):
        if getattr(self, "h", None):
            solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _create_args(n, rowptr, colind, val, V, lam, precision, inner_prec, validate, max_outer, restart_factor,
                 stream, keep):
    _check_dtype(rowptr, np.int64, "rowptr"); _check_dtype(colind, np.int32, "colind")
    _check_dtype(val, np.float64, "val")
    k = 0
    Vp = lamp = None
    if V is not None and lam is not None and len(lam) > 0:
        V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(n, -1).T)
        k = V.shape[0]
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        Vp, kv = _ptr(V); lamp, kl = _ptr(lam); keep += [kv, kl]
    rp, k1 = _ptr(rowptr); ci, k2 = _ptr(colind); va, k3 = _ptr(val)
    keep += [k1, k2, k3]
    return CreateArgs(int(n), int(rowptr[-1]), rp, ci, va, k, Vp, lamp, int(precision), int(inner_prec),
                      1 if validate else 0, int(max_outer), float(restart_factor), stream, 0, 0)


def batch_create(problems, precision=FP64, inner_prec=MCG_IDENTITY, validate=True, max_outer=0,
                 restart_factor=0.0, stream=None) -> int:
    """mrcg_batch_create from a list of objects with n, rowptr, colind, val, V, lam."""
    keep = []
    arr = (CreateArgs * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = _create_args(p.n, p.rowptr, p.colind, p.val, p.V if p.k else None, p.lam if p.k else None,
                              precision, inner_prec, validate, max_outer, restart_factor, stream, keep)
    h = C.c_void_p()
    st = lib().mrcg_batch_create(len(problems), arr, C.byref(h))
    if st != OK:
        raise MrcgError(st, "mrcg_batch_create")
    return h.value


def batched_solve(h, B, X, outer_tol=1e-10, inner_tol=1e-3, max_iters=0, history_cap=256):
    """mrcg_batched_solve: returns (status, [SolveInfo per system])."""
    _check_dtype(B, np.float64, "B"); _check_dtype(X, np.float64, "X")
    S = lib().mrcg_batch_size(h)
    infos = (Info * S)()
    hists = [np.zeros(max(history_cap, 1)) for _ in range(S)]
    for i in range(S):
        infos[i].relres_history = hists[i].ctypes.data
        infos[i].history_cap = history_cap
    bp, kb = _ptr(B); xp, kx = _ptr(X)
    st = lib().mrcg_batched_solve(h, bp, xp, float(outer_tol), float(inner_tol), int(max_iters), infos)
    if st in (ERR_INVALID, ERR_CUDA, ERR_OOM):
        raise MrcgError(st, "mrcg_batched_solve")
    out = [SolveInfo(f.status, f.outer_iters, f.restarts, f.inner_iters_total, f.prec_calls, f.kernel_launches,
                     f.true_relres, f.solve_ms, hists[i][: f.history_len].copy()) for i, f in enumerate(infos)]
    return st, out


def batch_launch_config(h):
    """mrcg_batch_launch_config: the autotuned launch shape of a batch handle."""
    cfg = np.zeros(4, dtype=np.int32)
    st = lib().mrcg_batch_launch_config(h, cfg.ctypes.data)
    if st != OK:
        raise MrcgError(st, "mrcg_batch_launch_config")
    return {"chunk_rows": int(cfg[0]), "step_a_grid": int(cfg[1]), "step_b_grid": int(cfg[2]), "chunks": int(cfg[3])}


class Batch:
    """Owning wrapper of one batch handle; vectors are concatenated in system order."""

    def __init__(self, problems, **kw):
        self.sizes = [int(p.n) for p in problems]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.h = batch_create(problems, **kw)

    def solve(self, B, X=None, **kw):
        if X is None:
            X = np.zeros(int(self.offsets[-1])) if isinstance(B, np.ndarray) else B.new_zeros(B.shape)
        st, infos = batched_solve(self.h, B, X, **kw)
        return X, st, infos

    def split(self, X):
        return [X[self.offsets[i]:self.offsets[i + 1]] for i in range(len(self.sizes))]

    def close(self):
        if getattr(self, "h", None):
            lib().mrcg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def shifted_create(fam, precision=FP64, max_outer=0, restart_factor=0.0, stream=None) -> int:
    """mrcg_shifted_create from an object with n, rowptr, colind, val (of L),
    V (n x kmax eigenvectors of L), lamL, sigma, k (per shift), nrhs."""
    keep = []
    a = _create_args(fam.n, fam.rowptr, fam.colind, fam.val, None, None, precision, MCG_IDENTITY, False,
                     max_outer, restart_factor, stream, keep)
    V = np.ascontiguousarray(np.asarray(fam.V, dtype=np.float64).reshape(fam.n, -1).T)
    lamL = np.ascontiguousarray(fam.lamL, dtype=np.float64)
    a.k = V.shape[0]
    a.V = V.ctypes.data
    a.lambda_ = lamL.ctypes.data
    sig = np.ascontiguousarray(fam.sigma, dtype=np.float64)
    ks = np.ascontiguousarray(fam.k, dtype=np.int32)
    h = C.c_void_p()
    st = lib().mrcg_shifted_create(C.byref(a), len(sig), sig.ctypes.data, ks.ctypes.data, int(fam.nrhs), C.byref(h))
    if st != OK:
        raise MrcgError(st, "mrcg_shifted_create")
    return h.value


def shifted_solve(h, B, X, outer_tol=1e-10, inner_tol=1e-3, max_iters=0, history_cap=256):
    """mrcg_shifted_solve on n x ncols row-major blocks: returns (status, [SolveInfo per column])."""
    _check_dtype(B, np.float64, "B"); _check_dtype(X, np.float64, "X")
    S = lib().mrcg_shifted_columns(h)
    infos = (Info * S)()
    hists = [np.zeros(max(history_cap, 1)) for _ in range(S)]
    for i in range(S):
        infos[i].relres_history = hists[i].ctypes.data
        infos[i].history_cap = history_cap
    bp, kb = _ptr(B); xp, kx = _ptr(X)
    st = lib().mrcg_shifted_solve(h, bp, xp, float(outer_tol), float(inner_tol), int(max_iters), infos)
    if st in (ERR_INVALID, ERR_CUDA, ERR_OOM):
        raise MrcgError(st, "mrcg_shifted_solve")
    out = [SolveInfo(f.status, f.outer_iters, f.restarts, f.inner_iters_total, f.prec_calls, f.kernel_launches,
                     f.true_relres, f.solve_ms, hists[i][: f.history_len].copy()) for i, f in enumerate(infos)]
    return st, out


def shifted_launch_config(h):
    """mrcg_shifted_launch_config: the autotuned launch shape of a shifted-family handle."""
    cfg = np.zeros(5, dtype=np.int32)
    st = lib().mrcg_shifted_launch_config(h, cfg.ctypes.data)
    if st != OK:
        raise MrcgError(st, "mrcg_shifted_launch_config")
    return {"grid": int(cfg[0]), "blocks_per_sm": int(cfg[1]), "ell8": int(cfg[2]), "v_width": int(cfg[3]),
            "padded_columns": int(cfg[4])}


class Shifted:
    """Owning wrapper of one shifted-family handle."""

    def __init__(self, fam, **kw):
        self.n = int(fam.n)
        self.ncols = len(fam.sigma) * int(fam.nrhs)
        self.h = shifted_create(fam, **kw)

    def solve(self, B, X=None, **kw):
        if X is None:
            X = np.zeros((self.n, self.ncols)) if isinstance(B, np.ndarray) else B.new_zeros(B.shape)
        st, infos = shifted_solve(self.h, B, X, **kw)
        return X, st, infos

    def close(self):
        if getattr(self, "h", None):
            lib().mrcg_shifted_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class ComplexShifted:
    """Owning wrapper of a complex-shift handle (Sec. 3): built from a system
    object with n, KE, K, D (scipy CSR), mass and gamma (its modulus fixes the
    inner level); V, lam (n x k, k) are used when given, else the eigenpairs
    are computed at create."""

    def __init__(self, sysobj, precision=FP64, inner_prec=MCG_IDENTITY, V=None, lam=None, eig_block=0,
                 stream=None):
        self.n = int(sysobj.n)
        keep = []

        def csr(M):
            M = M.tocsr()
            M.sort_indices()
            arrs = (np.ascontiguousarray(M.indptr, dtype=np.int64), np.ascontiguousarray(M.indices, dtype=np.int32),
                    np.ascontiguousarray(M.data, dtype=np.float64))
            keep.extend(arrs)
            return [a.ctypes.data for a in arrs]
        ke, kk, dd = csr(sysobj.KE), csr(sysobj.K), csr(sysobj.D)
        mass = np.ascontiguousarray(sysobj.mass, dtype=np.float64)
        keep.append(mass)
        k, Vp, lamp = -1, None, None
        if V is not None:
            Vc = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(self.n, -1).T)
            lam = np.ascontiguousarray(lam, dtype=np.float64)
            keep += [Vc, lam]
            k, Vp, lamp = Vc.shape[0], Vc.ctypes.data, lam.ctypes.data
        a = ComplexArgs(self.n, *ke, *kk, *dd, mass.ctypes.data, float(abs(sysobj.gamma)), k, Vp, lamp,
                        int(eig_block), int(precision), int(inner_prec), 0, stream)
        h = C.c_void_p()
        st = lib().mrcg_complex_create(C.byref(a), C.byref(h))
        if st != OK:
            raise MrcgError(st, "mrcg_complex_create")
        self.h = h.value

    @property
    def negative_count(self):
        return int(lib().mrcg_complex_negative_count(self.h))

    def solve(self, gamma, f, g, tol=1e-10, restart=40, max_iters=200, s2_tol=1e-6, s2_max=60, inner_tol=1e-8,
              cg_tol=1e-3):
        """x + i y with (gamma B - A)(x + i y) = f + i g.  Returns (x, y, status, info dict)."""
        _check_dtype(f, np.float64, "f"); _check_dtype(g, np.float64, "g")
        if isinstance(f, np.ndarray):
            x = np.zeros(2 * self.n); y = np.zeros(2 * self.n)
        else:
            x = f.new_zeros(2 * self.n); y = f.new_zeros(2 * self.n)
        info = ComplexInfo()
        fp, kf = _ptr(f); gp, kg = _ptr(g); xp, kx = _ptr(x); yp, ky = _ptr(y)
        st = lib().mrcg_complex_solve(self.h, float(gamma.real), float(gamma.imag), fp, gp, xp, yp, float(tol),
                                      int(restart), int(max_iters), float(s2_tol), int(s2_max), float(inner_tol),
                                      float(cg_tol), C.byref(info))
        if st in (ERR_INVALID, ERR_CUDA, ERR_OOM):
            raise MrcgError(st, "mrcg_complex_solve")
        return x, y, st, {f_: getattr(info, f_) for f_, _ in ComplexInfo._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().mrcg_complex_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
