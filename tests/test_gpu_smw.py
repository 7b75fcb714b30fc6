"""GPU parity of MINRES-CG* (Sec. 2.1): the inner CG preconditioned by
M_cg^{-1} = diag(A)^{-1} - 2 V Lambda^{-1} V^T, against the FP64 oracle.

Bars as for the other inner preconditioners: FP64 inner solves within one
iteration of the oracle and 1e-8 relative in the solution; FP32 inner solves
meet the tolerance in the M_mr residual recomputed in FP64; full solves agree
with the oracle's to 1e-8 (FP64) or reach the FP64 true residual (mixed).
"""
import numpy as np
import pytest

import oracle as O
from gen import lap3d_128_k10, dense_to_csr, random_sparse_symmetric, shifted_laplacian_problem, small_3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

DEV = torch.device("cuda:0")


def near_sigma(dims=(24, 20), k=4, seed=0):
    """sigma close to lambda_k: the negative eigenvalues are the small ones."""
    return shifted_laplacian_problem("near", dims, k, seed=seed, sigma_frac=0.05)


def _inner(p, prec, tol, seed, var=None, monkeypatch=None):
    if var is not None:
        monkeypatch.setenv("MRCG_VAR_A", str(var[0]))
        if var[1] is not None:
            monkeypatch.setenv("MRCG_STAGES", str(var[1]))
    s = O.System.from_problem(p)
    y = np.random.default_rng(seed).standard_normal(p.n)
    zr, itr, st_r = s.cg(y, tol, 100000, O.MCG_SMW)
    assert st_r == O.OK
    with m.Solver.from_problem(p, precision=prec, inner_prec=m.MCG_SMW) as g:
        if var is not None:
            assert m.launch_config(g.h)["step_a_variant"] == var[0]
        z, st, it = g.inner_solve(y, inner_tol=tol)
    assert st == m.OK
    if prec == m.FP64:
        assert abs(it - itr) <= 1
        assert np.linalg.norm(z - zr) <= 1e-8 * np.linalg.norm(zr)
    res = np.linalg.norm(y - s.mmr_apply(z))
    assert res <= tol * np.linalg.norm(y) * (1.001 if prec == m.FP64 else 1.5)
    return it, itr


@pytest.mark.parametrize("prob", [small_3d, near_sigma], ids=["lap3d_12x11x10_k5", "lap2d_24x20_near_sigma"])
@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_smw_inner_matches_oracle(prob, prec):
    # FP32 at 1e-3 (the inner tolerance of the solves): the near-sigma M_mr has
    # kappa ~ 1e4, so FP32 arithmetic bounds the true residual near 1e-4
    _inner(prob(), prec, 1e-6 if prec == m.FP64 else 1e-3, 3)


@pytest.mark.parametrize("var", [(0, None), (3, None), (5, 3), (6, 2), (7, 3)],
                         ids=["v0", "v3", "staged3", "staged4bpsm", "pipelined3"])
def test_smw_every_step_a_variant(var, monkeypatch):
    """Step a is the same kernel as with M_cg = I (it forms V^T A p'); every variant."""
    _inner(small_3d(), m.FP64, 1e-8, 5, var, monkeypatch)


@pytest.mark.parametrize("k", [1, 10, 17, 32])
def test_smw_k_buckets(k):
    p = shifted_laplacian_problem("t", (13, 11, 9), k, seed=k, sigma_frac=0.2)
    _inner(p, m.FP64, 1e-8, k)
    _inner(p, m.MIXED_FP32, 1e-4, k)


def test_smw_cuts_inner_iterations_near_sigma():
    """Sec. 2.1 / 4.3: with the negative eigenvalues closest to zero, the
    MINRES-CG* inner CG needs far fewer iterations than the plain one, on the
    GPU as in the oracle."""
    p = near_sigma()
    y = np.random.default_rng(0).standard_normal(p.n)
    its = {}
    for mcg in (m.MCG_IDENTITY, m.MCG_SMW):
        with m.Solver.from_problem(p, inner_prec=mcg) as g:
            z, st, it = g.inner_solve(y, inner_tol=1e-6)
        assert st == m.OK
        its[mcg] = it
    assert its[m.MCG_SMW] < 0.7 * its[m.MCG_IDENTITY]


@pytest.mark.parametrize("prob", [small_3d, lambda: near_sigma((30, 29), 5, 8)], ids=["lap3d_small", "lap2d_near"])
def test_minres_cg_star_matches_oracle(prob):
    p = prob()
    ref = O.minres_cg(O.System.from_problem(p), p.b, outer_tol=1e-12, inner_tol=1e-3, mcg=O.MCG_SMW)
    assert ref.status == O.OK
    with m.Solver.from_problem(p, inner_prec=m.MCG_SMW) as g:
        x, info = g.solve(p.b.copy(), outer_tol=1e-12, inner_tol=1e-3)
    assert info.status == m.OK
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-8
    assert abs(info.outer_iters - ref.outer_iters) <= 2
    assert abs(info.inner_iters_total - ref.inner_iters_total) <= max(4, 0.02 * ref.inner_iters_total)


def test_minres_cg_star_mixed_reaches_fp64_residual():
    p = near_sigma((30, 29), 5, 8)
    with m.Solver.from_problem(p, precision=m.MIXED_FP32, inner_prec=m.MCG_SMW) as g:
        x, info = g.solve(p.b.copy(), outer_tol=1e-10, inner_tol=1e-3)
    assert info.status == m.OK
    assert np.linalg.norm(p.b - p.scipy() @ x) / np.linalg.norm(p.b) <= 1e-10


def test_smw_rejects_zero_diagonal_and_batches():
    A = np.array([[2.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 3.0]])  # a saddle-type row
    rp, ci, va = dense_to_csr(A)
    with pytest.raises(m.MrcgError) as e:
        m.Solver(3, rp, ci, va, inner_prec=m.MCG_SMW)
    assert e.value.status == m.ERR_INVALID
    p = small_3d()
    with pytest.raises(m.MrcgError) as e:
        m.batch_create([p, p], inner_prec=m.MCG_SMW)
    assert e.value.status == m.ERR_INVALID


def test_smw_indefinite_diagonal_runs_or_reports():
    """diag(A) with negative entries: Sec. 2.1 allows an indefinite M_cg; the
    solve either converges or stops with a reported status (never a wrong OK)."""
    n = 600
    rp, ci, va = random_sparse_symmetric(n, 4, density_rows=(2, 8), diag_shift=6.0, empty_rows=0)
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    A[[0, 7, 11], [0, 7, 11]] = -6.0  # three negative diagonal entries
    rp, ci, va = dense_to_csr(A)
    w, Q = np.linalg.eigh(A)
    k = int((w < 0).sum())
    if k == 0 or k > 32:
        pytest.skip("draw without 1..32 negative eigenvalues")
    y = np.random.default_rng(1).standard_normal(n)
    with m.Solver(n, rp, ci, va, Q[:, :k], w[:k], inner_prec=m.MCG_SMW, validate=False) as g:
        z, st, it = g.inner_solve(y, inner_tol=1e-8)
    s = O.System(rp, ci, va, Q[:, :k], w[:k])
    if st == m.OK:
        assert np.linalg.norm(y - s.mmr_apply(z)) <= 1.001e-8 * np.linalg.norm(y)
    else:
        assert st in (m.ERR_BREAKDOWN, m.ERR_MAXITER, m.ERR_NOT_SPD)


def test_smw_full_size_mixed():
    """128^3 shifted Laplacian, mixed precision, MINRES-CG*: the FP64 true
    residual reaches the benchmark tolerance."""
    p = lap3d_128_k10()
    with m.Solver.from_problem(p, precision=m.MIXED_FP32, inner_prec=m.MCG_SMW) as g:
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        _, info = g.solve(torch.from_numpy(p.b).to(DEV), x, outer_tol=1e-10, inner_tol=1e-3)
    x = x.cpu().numpy()
    assert info.status == m.OK
    assert O.System.from_problem(p).true_relres(p.b, x) <= 1e-10
