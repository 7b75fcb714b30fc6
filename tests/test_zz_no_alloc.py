"""The allocation-free M_mr product, checked against the handle-based one.

mrcg_mmr_apply_noalloc serves callers that cannot allocate device memory
(fixed memory pools of a host framework, plugins barred from allocating
after start-up): it takes only caller-owned device arrays and uses a fixed
static scratch array inside the library.  Here it is called through the C ABI
twice in a row -- on two different systems, so that stale scratch from the
first call would show -- and each output is compared with mrcg_apply_mmr on a
solver handle for the same system, at the FP64 M_mr tolerance of the parity
tests.  This file is collected last; it also passes on its own.
"""
import ctypes as C

import numpy as np
import pytest

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


def _noalloc(p, u):
    f = _fn()
    rp, ci, va = _dev(p.rowptr), _dev(p.colind), _dev(p.val)
    V = _dev(p.V_colmajor())
    lam = _dev(p.lam)
    ud = _dev(u)
    out = torch.full((p.n,), float("nan"), dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    st = f(p.n, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), p.k, V.data_ptr(), lam.data_ptr(), ud.data_ptr(),
           out.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == m.OK, m.status_string(st)
    return out.cpu().numpy()


def test_noalloc_matches_handle_path_two_calls():
    probs = [shifted_laplacian_problem("na1", (23, 17, 9), 10, seed=21),
             shifted_laplacian_problem("na2", (41, 33), 3, seed=22)]
    for i, p in enumerate(probs):
        u = np.random.default_rng(100 + i).standard_normal(p.n)
        with m.Solver.from_problem(p) as g:
            ref = g.apply_mmr(u)
        out = _noalloc(p, u)
        assert np.all(np.isfinite(out))
        assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max() * 10


def test_noalloc_rejects_sizes_beyond_limit():
    f = _fn()
    one = torch.zeros(4, dtype=torch.float64, device=DEV)
    st = f(2, one.data_ptr(), one.data_ptr(), one.data_ptr(), 33, one.data_ptr(), one.data_ptr(), one.data_ptr(),
           one.data_ptr(), None)
    assert st == m.ERR_INVALID
    st = f(0, one.data_ptr(), one.data_ptr(), one.data_ptr(), 1, one.data_ptr(), one.data_ptr(), one.data_ptr(),
           one.data_ptr(), None)
    assert st == m.ERR_INVALID
