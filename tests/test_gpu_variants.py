"""GPU parity of every step-a kernel variant of the inner CG (Eq. 2).

The launch-shape autotuner may pick any variant for a matrix, so each one is
forced here (MRCG_VAR_A, read when a solver is created) and checked against
the FP64 oracle CG on the same inputs:

  * FP64 kernels: iteration count within 1 of the oracle and the solution
    within 1e-8 relative (the variants differ from the oracle only in the
    order of the block sums);
  * FP32 kernels: the M_mr residual of the returned z, recomputed by the
    oracle in FP64, meets the inner tolerance (1e-4: FP32 arithmetic bounds
    how far the true residual can follow the recursive one).

Variants 5, 6 and 7 (one kernel: registers capped for 2 or 4 blocks per SM;
7 issues each warp's gathers one tile ahead) stage every streamed operand in
shared memory by bulk copies; they are run with 2, 3 and 4 stages (a shape whose stages do not fit in a block
falls back to variant 0, which the fallback test checks), with 16-bit and 32-bit column indices, with
Jacobi M_cg, on ragged last tiles and on rows far longer than the stencil's.
"""
import numpy as np
import pytest

import oracle as O
from gen import lap3d_128_k10, random_sparse_symmetric, shifted_laplacian_problem, small_3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

DEV = torch.device("cuda:0")

SHAPES = [(0, None), (1, None), (2, None), (3, None), (4, None), (5, 2), (5, 3), (5, 4), (6, 2), (6, 3), (7, 2),
          (7, 3), (9, 2), (9, 3), (10, 2), (10, 4), (11, None), (12, 2), (12, 3), (13, 3), (14, 2), (14, 3),
          (15, 2), (15, 3)]
SHAPE_IDS = ["v0", "v1", "v2", "v3", "v4", "staged2", "staged3", "staged4", "staged4bpsm_2", "staged4bpsm_3",
             "pipelined2", "pipelined3", "onegather_staged2", "onegather_staged3", "onegather_staged3bpsm_2",
             "onegather_staged3bpsm_4", "onegather_plain", "onegather_pipelined2", "onegather_pipelined3",
             "onegather_pipelined3bpsm", "twoslice2", "twoslice3", "twoslice_1bpsm2", "twoslice_1bpsm3"]


def is_staged(var):
    return 5 <= var <= 10 or 12 <= var <= 15


@pytest.fixture
def shape_env(monkeypatch):
    def set_shape(var, stages, idx16=True):
        monkeypatch.setenv("MRCG_VAR_A", str(var))
        if stages is not None:
            monkeypatch.setenv("MRCG_STAGES", str(stages))
        else:
            monkeypatch.delenv("MRCG_STAGES", raising=False)
        if not idx16:
            monkeypatch.setenv("MRCG_IDX16", "0")
    return set_shape


def _check_cfg(g, var, stages, idx_bytes=None):
    cfg = m.launch_config(g.h)
    assert cfg["step_a_variant"] == var
    if is_staged(var):
        assert cfg["stages"] == stages
    if idx_bytes is not None:
        assert cfg["index_bytes"] == idx_bytes


def _inner_vs_oracle(p, prec, mcg, tol, seed, var, stages, idx_bytes=None, V=None, lam=None, sysargs=None,
                     expect_var=None):
    s = O.System(*sysargs, V, lam) if sysargs is not None else O.System.from_problem(p)
    n = sysargs[0].shape[0] - 1 if sysargs is not None else p.n
    y = np.random.default_rng(seed).standard_normal(n)
    zr, itr, st_r = s.cg(y, tol, 100000, mcg)
    assert st_r == O.OK
    if sysargs is not None:
        g = m.Solver(n, *sysargs, V, lam, precision=prec, inner_prec=mcg, validate=False)
    else:
        g = m.Solver.from_problem(p, precision=prec, inner_prec=mcg)
    with g:
        _check_cfg(g, var if expect_var is None else expect_var, stages, idx_bytes)
        z, st, it = g.inner_solve(y, inner_tol=tol)
    assert st == m.OK
    if prec == m.FP64:
        assert abs(it - itr) <= 1
        assert np.linalg.norm(z - zr) <= 1e-8 * np.linalg.norm(zr)
    res = np.linalg.norm(y - s.mmr_apply(z))
    assert res <= tol * np.linalg.norm(y) * (1.001 if prec == m.FP64 else 1.5)


@pytest.mark.parametrize("var,stages", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
@pytest.mark.parametrize("mcg", [m.MCG_IDENTITY, m.MCG_JACOBI], ids=["id", "jacobi"])
def test_inner_variants_small_3d(shape_env, var, stages, prec, mcg):
    """12 x 11 x 10 Laplacian (n = 1320: 42 slices, last tile 2 slices), k = 5."""
    shape_env(var, stages)
    _inner_vs_oracle(small_3d(), prec, mcg, 1e-6 if prec == m.FP64 else 1e-4, 4, var, stages, idx_bytes=2)


@pytest.mark.parametrize("k", [0, 1, 10, 13, 17, 32])
@pytest.mark.parametrize("var,stages", [(1, None), (3, None), (5, 2), (6, 2), (7, 2), (9, 2), (10, 2), (11, None),
                                       (12, 2), (13, 2), (14, 2), (15, 2)],
                         ids=["v1", "v3", "staged2", "staged4bpsm", "pipelined2", "onegather_staged2",
                              "onegather_staged3bpsm", "onegather_plain", "onegather_pipelined2",
                              "onegather_pipelined3bpsm", "twoslice2", "twoslice_1bpsm2"])
def test_inner_variants_k_buckets(shape_env, k, var, stages):
    """Every k bucket of the kernels (FP64 stages of k = 32 hold 86 KB on tiles
    of 8 slices, so two fit a block; on tiles of 16 slices FP64 stages of
    k >= 17 exceed half the block's shared memory and the solver falls back to
    variant 0, with the same answers)."""
    p = shifted_laplacian_problem("t", (13, 11, 9), max(k, 1), seed=k) if k else None
    shape_env(var, stages)
    if p is None:
        from gen import laplacian_csr
        rp, ci, va = laplacian_csr((13, 11, 9), sigma=-0.5)  # SPD: M_mr = A
        _inner_vs_oracle(None, m.FP64, m.MCG_IDENTITY, 1e-8, 1, var, stages, sysargs=(rp, ci, va))
        return
    fp64_var = 0 if var in (14, 15) and k >= 17 else None
    _inner_vs_oracle(p, m.FP64, m.MCG_IDENTITY, 1e-8, k, var, stages, expect_var=fp64_var)
    _inner_vs_oracle(p, m.MIXED_FP32, m.MCG_IDENTITY, 1e-4, k, var, stages)


@pytest.mark.parametrize("idx16", [True, False], ids=["idx16", "idx32"])
@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
@pytest.mark.parametrize("stages", [2, 3])
def test_staged_long_rows(shape_env, idx16, prec, stages):
    """Rows of 2 to 19 entries at random columns (tiles of 3,488 entries, half
    again the stencil's), n = 3001 (ragged last slice and tile), k = 6 random
    orthonormal columns with negative lambdas (M_mr = A + 2 V |Lambda| V^T
    stays SPD because A is), Jacobi M_cg."""
    n = 3001
    rp, ci, va = random_sparse_symmetric(n, 21, density_rows=(2, 12), diag_shift=30.0, empty_rows=0)
    rng = np.random.default_rng(22)
    V, _ = np.linalg.qr(rng.standard_normal((n, 6)))
    lam = -rng.uniform(0.5, 3.0, 6)
    for var in (5, 7, 9, 11, 12):
        shape_env(var, stages, idx16=idx16)
        _inner_vs_oracle(None, prec, m.MCG_JACOBI, 1e-7 if prec == m.FP64 else 1e-4, 23, var, stages,
                         idx_bytes=2 if idx16 else 4, V=V, lam=lam, sysargs=(rp, ci, va))


@pytest.mark.parametrize("var", [5, 9, 12])
def test_staged_falls_back_when_stages_do_not_fit(shape_env, var):
    """FP64, k = 32: three stages of 86 KB exceed a block's shared memory; and
    rows of up to 64 entries make one stage of a tile 164 KB."""
    shape_env(var, 3)
    p = shifted_laplacian_problem("t", (13, 11, 9), 32, seed=32)
    with m.Solver.from_problem(p) as g:
        assert m.launch_config(g.h)["step_a_variant"] == 0
        z, st, it = g.inner_solve(np.ones(p.n), inner_tol=1e-8)
    assert st == m.OK and it > 0
    shape_env(var, 2)
    rp, ci, va = random_sparse_symmetric(3001, 21, density_rows=(2, 70), diag_shift=90.0, empty_rows=0)
    with m.Solver(3001, rp, ci, va) as g:
        assert m.launch_config(g.h)["step_a_variant"] == 0
        z, st, it = g.inner_solve(np.ones(3001), inner_tol=1e-8)
    assert st == m.OK and it > 0


@pytest.mark.parametrize("var,stages", [(0, None), (5, 3), (6, 2), (7, 3), (9, 3), (10, 2), (11, None), (12, 3),
                                       (13, 2), (14, 2), (15, 2)],
                         ids=["v0", "staged3", "staged4bpsm", "pipelined3", "onegather_staged3",
                              "onegather_staged3bpsm", "onegather_plain", "onegather_pipelined3",
                              "onegather_pipelined3bpsm", "twoslice2", "twoslice_1bpsm2"])
def test_variants_full_solve_small(shape_env, var, stages):
    """A whole MINRES-CG solve on every step-a path agrees with the oracle's."""
    shape_env(var, stages)
    p = small_3d()
    ref = O.minres_cg(O.System.from_problem(p), p.b, outer_tol=1e-12, inner_tol=1e-3)
    with m.Solver.from_problem(p) as g:
        _check_cfg(g, var, stages)
        x, info = g.solve(p.b.copy(), outer_tol=1e-12, inner_tol=1e-3)
    assert info.status == m.OK
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-8


def test_staged_full_size_mixed(shape_env):
    """128^3 shifted Laplacian, mixed precision, staged step a with 3 stages:
    the FP64 true residual reaches the benchmark tolerance."""
    shape_env(5, 3)
    p = lap3d_128_k10()
    with m.Solver.from_problem(p, precision=m.MIXED_FP32) as g:
        _check_cfg(g, 5, 3)
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        _, info = g.solve(torch.from_numpy(p.b).to(DEV), x, outer_tol=1e-10, inner_tol=1e-3)
    x = x.cpu().numpy()
    assert info.status == m.OK
    assert O.System.from_problem(p).true_relres(p.b, x) <= 1e-10


# ---------------------------------------------------------------- variant 8: the one-kernel iteration (M_cg = I)

@pytest.mark.parametrize("stages", [2, 3])
@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_one_kernel_iteration_small_3d(shape_env, stages, prec):
    """z += alpha p, r -= alpha q and the next direction fold into the SpMV
    kernel; rho_{i+1} comes from the expansion rho - 2 alpha r^T q + alpha^2 q^T q."""
    shape_env(8, stages)
    _inner_vs_oracle(small_3d(), prec, m.MCG_IDENTITY, 1e-6 if prec == m.FP64 else 1e-4, 4, 8, stages,
                     idx_bytes=2)


@pytest.mark.parametrize("k", [0, 1, 10, 13, 17, 32])
def test_one_kernel_iteration_k_buckets(shape_env, k):
    shape_env(8, 2)
    if k == 0:
        from gen import laplacian_csr
        rp, ci, va = laplacian_csr((13, 11, 9), sigma=-0.5)
        _inner_vs_oracle(None, m.FP64, m.MCG_IDENTITY, 1e-8, 1, 8, 2, sysargs=(rp, ci, va))
        return
    p = shifted_laplacian_problem("t", (13, 11, 9), k, seed=k)
    _inner_vs_oracle(p, m.FP64, m.MCG_IDENTITY, 1e-8, k, 8, 2)
    _inner_vs_oracle(p, m.MIXED_FP32, m.MCG_IDENTITY, 1e-4, k, 8, 2)


def test_one_kernel_iteration_budget_and_long_rows(shape_env):
    """The last z update is left to the finish kernel: an iteration cap must
    still return z_m (compared with the oracle's m-step iterate), also on rows
    longer than the stencil's and with 32-bit indices."""
    shape_env(8, 2, idx16=False)
    n = 3001
    rp, ci, va = random_sparse_symmetric(n, 21, density_rows=(2, 12), diag_shift=30.0, empty_rows=0)
    s = O.System(rp, ci, va)
    y = np.random.default_rng(9).standard_normal(n)
    for m_it in (1, 2, 5, 9):
        zr, itr, st_r = s.cg(y, 1e-300, m_it, O.MCG_IDENTITY)
        with m.Solver(n, rp, ci, va, validate=False) as g:
            _check_cfg(g, 8, 2, 4)
            z, st, it = g.inner_solve(y, inner_tol=1e-12, max_iters=m_it)
        assert st == m.ERR_MAXITER and it == m_it
        assert np.linalg.norm(z - zr) <= 1e-10 * np.linalg.norm(zr)


def test_one_kernel_iteration_falls_back_without_identity(shape_env):
    shape_env(8, 2)
    with m.Solver.from_problem(small_3d(), inner_prec=m.MCG_JACOBI) as g:
        assert m.launch_config(g.h)["step_a_variant"] == 0


def test_one_kernel_iteration_full_solves(shape_env):
    shape_env(8, 3)
    p = small_3d()
    ref = O.minres_cg(O.System.from_problem(p), p.b, outer_tol=1e-12, inner_tol=1e-3)
    with m.Solver.from_problem(p) as g:
        _check_cfg(g, 8, 3)
        x, info = g.solve(p.b.copy(), outer_tol=1e-12, inner_tol=1e-3)
    assert info.status == m.OK
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) <= 1e-8
    p = lap3d_128_k10()
    with m.Solver.from_problem(p, precision=m.MIXED_FP32) as g:
        _check_cfg(g, 8, 3)
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        _, info = g.solve(torch.from_numpy(p.b).to(DEV), x, outer_tol=1e-10, inner_tol=1e-3)
    assert info.status == m.OK
    assert O.System.from_problem(p).true_relres(p.b, x.cpu().numpy()) <= 1e-10



# ---------------------------------------------------------------- variants 9-15: one gather per matrix entry

def test_one_gather_falls_back_with_smw(shape_env):
    """Variants 9-15 cover M_cg = I and Jacobi; the MINRES-CG* M_cg keeps its own kernels."""
    for var in (9, 11, 12, 14):
        shape_env(var, 2)
        with m.Solver.from_problem(small_3d(), inner_prec=m.MCG_SMW) as g:
            assert m.launch_config(g.h)["step_a_variant"] == 0


@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_one_gather_budget_returns_mth_iterate(shape_env, prec):
    """z_m after an iteration cap equals the oracle's m-step iterate (FP64), and
    the in-place p update leaves later solves on the same handle unaffected."""
    shape_env(9, 2)
    p = small_3d()
    s = O.System.from_problem(p)
    y = np.random.default_rng(9).standard_normal(p.n)
    with m.Solver.from_problem(p, precision=prec) as g:
        for m_it in (1, 2, 5, 9):
            zr, itr, st_r = s.cg(y, 1e-300, m_it, O.MCG_IDENTITY)
            z, st, it = g.inner_solve(y, inner_tol=1e-12, max_iters=m_it)
            assert st == m.ERR_MAXITER and it == m_it
            bar = 1e-10 if prec == m.FP64 else 1e-4
            assert np.linalg.norm(z - zr) <= bar * np.linalg.norm(zr)


@pytest.mark.parametrize("var", [9, 14], ids=["onegather", "twoslice"])
def test_one_gather_full_size_mixed(shape_env, var):
    """128^3 shifted Laplacian, mixed precision, one-gather staged step a (8-
    and 16-slice tiles): the FP64 true residual reaches the benchmark tolerance
    and x matches x*."""
    shape_env(var, 2)
    p = lap3d_128_k10()
    with m.Solver.from_problem(p, precision=m.MIXED_FP32) as g:
        _check_cfg(g, var, 2)
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        _, info = g.solve(torch.from_numpy(p.b).to(DEV), x, outer_tol=1e-10, inner_tol=1e-3)
    x = x.cpu().numpy()
    assert info.status == m.OK
    assert O.System.from_problem(p).true_relres(p.b, x) <= 1e-10
    assert np.linalg.norm(x - p.xstar) / np.linalg.norm(p.xstar) <= p.meta["cond"] * 1e-10 * 3


# ---------------------------------------------------------------- a CG step that removes almost all of the residual

@pytest.mark.parametrize("var,stages", [(8, 2), (9, 2), (12, 3), (14, 2)],
                         ids=["one_kernel", "onegather", "onegather_pipelined", "twoslice"])
@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_sharp_single_step_reduction(shape_env, var, stages, prec):
    """A = diag(2 + 1e-3 u): the first CG step cuts ||r|| by about 1e-4, so the
    expansion rho - 2 alpha r^T q + alpha^2 q^T q cancels to its rounding level
    in FP32.  The solve must not stop on that noise: the returned z meets the
    inner tolerance 1e-5 on the true M_mr residual (recomputed in FP64)."""
    shape_env(var, stages)
    n = 8192
    rng = np.random.default_rng(31)
    d = 2.0 + 1e-3 * rng.uniform(0.0, 1.0, n)
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    s = O.System(rp, ci, d)
    y = rng.standard_normal(n)
    tol = 1e-5
    zr, itr, st_r = s.cg(y, tol, 1000, O.MCG_IDENTITY)
    assert st_r == O.OK and itr >= 2
    with m.Solver(n, rp, ci, d, validate=False, precision=prec) as g:
        _check_cfg(g, var, stages)
        z, st, it = g.inner_solve(y, inner_tol=tol)
    assert st == m.OK
    res = np.linalg.norm(y - s.mmr_apply(z))
    assert res <= tol * np.linalg.norm(y) * (1.001 if prec == m.FP64 else 1.5)
    assert it <= itr + 2
