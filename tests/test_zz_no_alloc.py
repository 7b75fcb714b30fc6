"""The allocation-free M_mr product, checked against the handle-based one and
against the FP64 CPU oracle.

mrcg_mmr_apply_noalloc serves callers that cannot allocate device memory
(fixed memory pools of a host framework, plugins barred from allocating
after start-up): it takes only caller-owned device arrays and uses a fixed
static scratch array inside the library.  Here it is called through the C ABI
twice in a row -- on two different systems, so that stale scratch from the
first call would show -- and each output is compared with mrcg_apply_mmr on a
solver handle for the same system and with the oracle's orc_mmr_apply, at the
FP64 M_mr tolerance of the parity tests.  k covers 0 (no low-rank pass), 1
and the documented limit 32, on the default stream and on a stream of the
caller's.  This file is collected last; it also passes on its own.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from gen import shifted_laplacian_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

DEV = torch.device("cuda:0")


def _fn():
    L = m.lib()
    f = L.mrcg_mmr_apply_noalloc
    P = C.c_void_p
    f.argtypes = [C.c_int64, P, P, P, C.c_int32, P, P, P, P, P]
    f.restype = C.c_int
    return f


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _noalloc(p, u, stream=None):
    """One call on `stream` (a torch.cuda.Stream, or None for the default stream)."""
    f = _fn()
    rp, ci, va = _dev(p.rowptr), _dev(p.colind), _dev(p.val)
    V = _dev(p.V_colmajor()) if p.k else torch.zeros(1, dtype=torch.float64, device=DEV)
    lam = _dev(p.lam) if p.k else torch.zeros(1, dtype=torch.float64, device=DEV)
    ud = _dev(u)
    out = torch.full((p.n,), float("nan"), dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    handle = None if stream is None else stream.cuda_stream
    st = f(p.n, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), p.k, V.data_ptr(), lam.data_ptr(), ud.data_ptr(),
           out.data_ptr(), handle)
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    assert st == m.OK, m.status_string(st)
    return out.cpu().numpy()


def _check(p, u, out):
    with m.Solver.from_problem(p) as g:
        ref = g.apply_mmr(u)
    orc = O.System.from_problem(p).mmr_apply(u)
    assert np.all(np.isfinite(out))
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max() * 10
    assert np.abs(out - orc).max() <= 1e-13 * np.abs(orc).max() * 10


def test_noalloc_matches_handle_path_two_calls():
    probs = [shifted_laplacian_problem("na1", (23, 17, 9), 10, seed=21),
             shifted_laplacian_problem("na2", (41, 33), 3, seed=22)]
    for i, p in enumerate(probs):
        u = np.random.default_rng(100 + i).standard_normal(p.n)
        _check(p, u, _noalloc(p, u))


@pytest.mark.parametrize("k", [0, 1, 32])
def test_noalloc_k_range_on_caller_stream(k):
    """k = 0 skips the V^T u pass; k = 32 fills every partial row; both calls of
    a pair go to a stream the caller created, the second on another system."""
    side = 40 if k < 32 else 48
    p1 = shifted_laplacian_problem(f"na_k{k}", (side, side - 3), k, seed=30 + k)
    p2 = shifted_laplacian_problem(f"na_k{k}b", (17, 15, 13), min(k, 20), seed=60 + k)
    s = torch.cuda.Stream(device=DEV)
    for i, p in enumerate((p1, p2)):
        u = np.random.default_rng(200 + i).standard_normal(p.n)
        _check(p, u, _noalloc(p, u, stream=s))


def test_noalloc_rejects_sizes_beyond_limit():
    f = _fn()
    one = torch.zeros(4, dtype=torch.float64, device=DEV)
    st = f(2, one.data_ptr(), one.data_ptr(), one.data_ptr(), 33, one.data_ptr(), one.data_ptr(), one.data_ptr(),
           one.data_ptr(), None)
    assert st == m.ERR_INVALID
    st = f(0, one.data_ptr(), one.data_ptr(), one.data_ptr(), 1, one.data_ptr(), one.data_ptr(), one.data_ptr(),
           one.data_ptr(), None)
    assert st == m.ERR_INVALID
