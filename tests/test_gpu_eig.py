"""GPU parity of setup stage 2 (Sec. 2): the negative eigenpairs of A from
mrcg_negative_eigenpairs (Chebyshev-filtered subspace iteration on the
library's block SpMV) against their definition.

  * small systems: the dense symmetric eigendecomposition of the oracle
    (same count, eigenvalues to 1e-9 ||A||, the same invariant subspace:
    projector distance below 1e-7);
  * shifted Laplacians: the analytic sine-mode spectrum, at small and at full
    size (128^3, k = 10);
  * saddle systems: Sylvester's count (k = nb) and the eigenvalues of the
    setup eigensolver of the generators (block Krylov, independent code);
  * end to end: a solver created from the computed pairs passes create's
    validation and solves to the parity tolerance.
"""
import numpy as np
import pytest

import oracle as O
from gen import lap3d_128_k10, random_indefinite_dense, dense_to_csr, shifted_laplacian_problem, small_saddle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

DEV = torch.device("cuda:0")


def _projector_gap(V, U):
    """|| V V^T - U U^T ||_2 for orthonormal V, U of equal width."""
    M = V.T @ U
    s = np.linalg.svd(M, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - s.min() ** 2))) if len(s) else 0.0


def _check_pairs(rp, ci, va, V, lam, tol):
    A = O.System(rp, ci, va)
    for j in range(V.shape[1]):
        r = A.spmv(V[:, j]) - lam[j] * V[:, j]
        assert np.linalg.norm(r) <= tol, (j, np.linalg.norm(r))
    assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-10)


@pytest.mark.parametrize("n,k,block", [(300, 5, 16), (700, 12, 24), (1200, 3, 40)])
def test_eigenpairs_match_dense_eigh(n, k, block):
    """Dense symmetric Q diag(d) Q^T with k negative eigenvalues (rows of n
    entries: the block SpMV's long-row path)."""
    A, _, _, _, _ = random_indefinite_dense(n, k, seed=n + k, spread=(0.5, 4.0))
    rp, ci, va = dense_to_csr(A)
    Vd, lamd, w = O.negative_eigenpairs_dense(rp, ci, va)
    V, lam, info = m.negative_eigenpairs(n, rp, ci, va, block, tol=1e-12)
    assert len(lam) == len(lamd) == k
    anorm = np.abs(w).max()
    assert np.allclose(lam, lamd, rtol=0, atol=1e-9 * anorm)
    assert _projector_gap(V, Vd) <= 1e-7
    _check_pairs(rp, ci, va, V, lam, 1e-10 * anorm)
    assert info["negative_found"] == k and info["block_spmvs"] > 0


def test_eigenpairs_of_a_shifted_laplacian_are_analytic():
    p = shifted_laplacian_problem("eig2d", (40, 37), 6, seed=9)
    V, lam, info = m.negative_eigenpairs(p.n, p.rowptr, p.colind, p.val, 16, tol=1e-12)
    assert len(lam) == p.k
    assert np.allclose(lam, p.lam, rtol=0, atol=1e-10 * 8.0)
    assert _projector_gap(V, p.V) <= 1e-7  # clusters included whole: the subspace is unique
    _check_pairs(p.rowptr, p.colind, p.val, V, lam, 1e-10 * 8.0)


def test_eigenpairs_of_a_small_saddle_system():
    q = small_saddle()
    Vd, lamd, w = O.negative_eigenpairs_dense(q.rowptr, q.colind, q.val)
    V, lam, _ = m.negative_eigenpairs(q.n, q.rowptr, q.colind, q.val, 16, tol=1e-12)
    assert len(lam) == q.k == len(lamd)  # Sylvester: nb negative eigenvalues
    anorm = np.abs(w).max()
    assert np.allclose(lam, lamd, rtol=0, atol=1e-9 * anorm)
    assert _projector_gap(V, Vd) <= 1e-7


def test_block_too_small_reports_maxiter():
    """Six negative eigenvalues, a block of four: no nonnegative Ritz value
    can appear, so the call runs out of its (small) budget and says so."""
    p = shifted_laplacian_problem("eig_small_block", (30, 29), 6, seed=3)
    with pytest.raises(m.MrcgError) as e:
        m.negative_eigenpairs(p.n, p.rowptr, p.colind, p.val, 4, tol=1e-12, max_spmv=400)
    assert e.value.status == m.ERR_MAXITER
    assert e.value.info["negative_found"] == 4


def test_invalid_arguments():
    p = shifted_laplacian_problem("eig_inv", (9, 8), 2, seed=3)
    for block in (1, 65):
        with pytest.raises(m.MrcgError) as e:
            m.negative_eigenpairs(p.n, p.rowptr, p.colind, p.val, block)
        assert e.value.status == m.ERR_INVALID
    ci = p.colind.copy()
    ci[4] = p.n
    with pytest.raises(m.MrcgError) as e:
        m.negative_eigenpairs(p.n, p.rowptr, ci, p.val, 8)
    assert e.value.status == m.ERR_INVALID


def test_full_size_128_eigenpairs_drive_a_solve():
    """128^3 shifted Laplacian: the ten computed eigenvalues equal the analytic
    ones, create's validation accepts the pairs, and MINRES-CG with them
    solves to the parity tolerance (x* within 1e-8 at outer_tol 1e-12)."""
    p = lap3d_128_k10()
    V, lam, info = m.negative_eigenpairs(p.n, p.rowptr, p.colind, p.val, 24, tol=1e-11)
    assert len(lam) == p.k == 10
    assert np.allclose(lam, p.lam, rtol=0, atol=1e-9 * 12.0)
    with m.Solver(p.n, p.rowptr, p.colind, p.val, V, lam, precision=m.MIXED_FP32, validate=True) as g:
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        _, sinfo = g.solve(torch.from_numpy(p.b).to(DEV), x, outer_tol=1e-12, inner_tol=1e-3)
    assert sinfo.status == m.OK
    x = x.cpu().numpy()
    assert np.linalg.norm(x - p.xstar) / np.linalg.norm(p.xstar) <= 1e-8
    print(f"eig 128^3: {info['block_spmvs']} block SpMVs, {info['rayleigh_ritz_steps']} RR steps, "
          f"{info['seconds']:.2f} s, max residual {info['max_residual']:.2e}")


def test_full_size_saddle_eigenpairs():
    """96^3 saddle system: exactly 20 negative eigenvalues (Sylvester), equal to
    those of the generators' block-Krylov eigensolver to 1e-8 relative, and a
    mixed solve with them reaches the benchmark tolerance."""
    from gen import saddle_96_b20x64
    q = saddle_96_b20x64()
    V, lam, info = m.negative_eigenpairs(q.n, q.rowptr, q.colind, q.val, 32, tol=1e-11)
    assert len(lam) == 20
    assert np.allclose(lam, np.sort(q.lam), rtol=1e-8, atol=0)
    with m.Solver(q.n, q.rowptr, q.colind, q.val, V, lam, precision=m.MIXED_FP32, validate=True) as g:
        x = torch.zeros(q.n, dtype=torch.float64, device=DEV)
        _, sinfo = g.solve(torch.from_numpy(q.b).to(DEV), x, outer_tol=1e-10, inner_tol=1e-3)
    assert sinfo.status == m.OK
    rr = O.System.from_problem(q).true_relres(q.b, x.cpu().numpy())
    assert rr <= 1e-10
    print(f"eig saddle: {info['block_spmvs']} block SpMVs, {info['seconds']:.2f} s")


@pytest.mark.parametrize("name", ["laplacian", "dense", "saddle"])
def test_fp32_filter_steps_reach_the_fp64_result(name, monkeypatch):
    """The filter's early FP32 steps (the default) and FP64 throughout
    (MRCG_EIG_FP32=0) give the same pairs to the tolerance: the FP32 steps only
    bring the block near the subspace, FP64 steps and FP64 Rayleigh-Ritz finish.
    Covers the stencil path (4 rows per warp), dense rows and a saddle matrix."""
    if name == "laplacian":
        p = shifted_laplacian_problem("eig32", (23, 21, 19), 7, seed=4)
        rp, ci, va, n, block = p.rowptr, p.colind, p.val, p.n, 16
    elif name == "dense":
        D = random_indefinite_dense(500, 6, seed=9)[0]
        rp, ci, va = dense_to_csr(D)
        n, block = 500, 16
    else:
        q = small_saddle()
        rp, ci, va, n, block = q.rowptr, q.colind, q.val, q.n, 24
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("MRCG_EIG_FP32", mode)
        out[mode] = m.negative_eigenpairs(n, rp, ci, va, block, tol=1e-12)
    (V1, l1, i1), (V0, l0, i0) = out["1"], out["0"]
    assert len(l1) == len(l0) > 0
    anorm = max(abs(i0["spectrum_lo"]), abs(i0["spectrum_hi"]))
    assert np.allclose(l1, l0, rtol=0, atol=1e-10 * anorm)
    _check_pairs(rp, ci, va, V1, l1, 1e-11 * anorm)
    assert _projector_gap(V1, V0) <= 1e-7
    print(f"{name}: FP32 filter {i1['block_spmvs']} block SpMVs, FP64 only {i0['block_spmvs']}")
