"""GPU parity of the block-Jacobi ILU(0) inner preconditioner (the paper's
experiments precondition the inner CG with an incomplete LU factorisation of
A, Sec. 4; MINRES-CG* uses it as Atilde, Sec. 2.1) against the oracle's
ILU(0) with the same blocks:

  * FP64 inner solves: iteration count within 1 and z within 1e-8 of the
    oracle's CG with the same M_cg, for blocks of 32 rows up to one block;
  * FP32 inner solves: the true M_mr residual of z (oracle, FP64) meets the
    inner tolerance;
  * whole MINRES-CG solves: x within 1e-8 of the oracle's (FP64) and the FP64
    true residual at the tolerance (mixed);
  * a zero pivot is MRCG_ERR_BREAKDOWN at create, a bad block size
    MRCG_ERR_INVALID.
"""
import numpy as np
import pytest

import oracle as O
from gen import lap3d_128_k10, random_sparse_symmetric, shifted_laplacian_problem, small_3d, small_saddle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

DEV = torch.device("cuda:0")
MCG = {m.MCG_ILU0: O.MCG_ILU0, m.MCG_SMW_ILU0: O.MCG_SMW_ILU0}


def _oracle(p, block, sysargs=None, V=None, lam=None):
    s = O.System(*sysargs, V, lam) if sysargs is not None else O.System.from_problem(p)
    assert s.set_ilu0(block) == O.OK
    return s


@pytest.mark.parametrize("block", [32, 256, 2048])
@pytest.mark.parametrize("mcg", [m.MCG_ILU0, m.MCG_SMW_ILU0], ids=["ilu0", "smw_ilu0"])
@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_inner_solve_matches_oracle(block, mcg, prec):
    """12 x 11 x 10 shifted Laplacian (n = 1320, k = 5): blocks of 32 (one
    SELL slice), 256 and 2048 (one block over all 1344 padded rows)."""
    p = small_3d()
    s = _oracle(p, block)
    y = np.random.default_rng(block).standard_normal(p.n)
    tol = 1e-8 if prec == m.FP64 else 1e-4
    zr, itr, st_r = s.cg(y, tol, 100000, MCG[mcg])
    assert st_r == O.OK
    with m.Solver.from_problem(p, precision=prec, inner_prec=mcg, ilu_block=block) as g:
        z, st, it = g.inner_solve(y, inner_tol=tol)
    assert st == m.OK
    if prec == m.FP64:
        assert abs(it - itr) <= 1
        assert np.linalg.norm(z - zr) <= 1e-8 * np.linalg.norm(zr)
    res = np.linalg.norm(y - s.mmr_apply(z))
    assert res <= tol * np.linalg.norm(y) * (1.001 if prec == m.FP64 else 1.5)


def test_inner_solve_long_rows():
    """Random symmetric rows of 2..12 entries (diagonally dominant, so every
    pivot is nonzero), n = 3001 (ragged last block), k = 4 random orthonormal
    columns: levels with many entries and long dependency chains."""
    n = 3001
    rp, ci, va = random_sparse_symmetric(n, 41, density_rows=(2, 12), diag_shift=30.0, empty_rows=0)
    rng = np.random.default_rng(42)
    V, _ = np.linalg.qr(rng.standard_normal((n, 4)))
    lam = -rng.uniform(0.5, 3.0, 4)
    for block in (96, 1024):
        s = _oracle(None, block, (rp, ci, va), V, lam)
        y = rng.standard_normal(n)
        zr, itr, st_r = s.cg(y, 1e-9, 10000, O.MCG_ILU0)
        with m.Solver(n, rp, ci, va, V, lam, inner_prec=m.MCG_ILU0, ilu_block=block, validate=False) as g:
            z, st, it = g.inner_solve(y, inner_tol=1e-9)
        assert st == m.OK and abs(it - itr) <= 1
        assert np.linalg.norm(z - zr) <= 1e-8 * np.linalg.norm(zr)


@pytest.mark.parametrize("mcg", [m.MCG_ILU0, m.MCG_SMW_ILU0], ids=["ilu0", "smw_ilu0"])
def test_full_solve_matches_oracle(mcg):
    p = shifted_laplacian_problem("ilu_full", (45, 37), 6, seed=11)
    s = _oracle(p, 512)
    ref = O.minres_cg(s, p.b, outer_tol=1e-12, inner_tol=1e-3, mcg=MCG[mcg])
    assert ref.status == O.OK
    with m.Solver.from_problem(p, inner_prec=mcg, ilu_block=512) as g:
        x, info = g.solve(p.b.copy(), outer_tol=1e-12, inner_tol=1e-3)
    assert info.status == m.OK
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    assert abs(info.outer_iters - ref.outer_iters) <= 2
    with m.Solver.from_problem(p, precision=m.MIXED_FP32, inner_prec=mcg, ilu_block=512) as g:
        x, info = g.solve(p.b.copy(), outer_tol=1e-10, inner_tol=1e-3)
    assert info.status == m.OK
    assert s.true_relres(p.b, x) <= 1e-10


def test_zero_pivot_and_bad_block():
    q = small_saddle()  # the constraint rows have no diagonal entry: zero pivot
    with pytest.raises(m.MrcgError) as e:
        m.Solver.from_problem(q, inner_prec=m.MCG_ILU0, ilu_block=64)
    assert e.value.status == m.ERR_BREAKDOWN
    p = small_3d()
    for bad in (48, 16384):  # not a multiple of 32; beyond the FP64 cap
        with pytest.raises(m.MrcgError) as e:
            m.Solver.from_problem(p, inner_prec=m.MCG_ILU0, ilu_block=bad)
        assert e.value.status == m.ERR_INVALID
    with pytest.raises(m.MrcgError):
        m.Batch([p], inner_prec=m.MCG_ILU0)


def test_full_size_mixed_solve_with_ilu():
    """128^3 shifted Laplacian, mixed precision, blocks of 8192 rows (half a
    grid plane): the FP64 true residual reaches the benchmark tolerance and
    the inner iterations drop below the M_cg = I count."""
    p = lap3d_128_k10()
    with m.Solver.from_problem(p, precision=m.MIXED_FP32, inner_prec=m.MCG_ILU0, ilu_block=8192,
                               validate=False) as g:
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        _, info = g.solve(torch.from_numpy(p.b).to(DEV), x, outer_tol=1e-10, inner_tol=1e-3)
    assert info.status == m.OK
    assert O.System.from_problem(p).true_relres(p.b, x.cpu().numpy()) <= 1e-10
    assert info.inner_iters_total < 2184  # M_cg = I needs 2184 at this tolerance
    print(f"ILU(0) 8192-row blocks at 128^3: outer {info.outer_iters}, inner {info.inner_iters_total}, "
          f"{info.solve_ms:.1f} ms")


@pytest.mark.parametrize("block", [64, 2048])
@pytest.mark.parametrize("mcg", [m.MCG_ILU0, m.MCG_SMW_ILU0], ids=["ilu0", "smw_ilu0"])
@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_staged_sweeps_equal_global_sweeps(block, mcg, prec, monkeypatch):
    """The sweeps from the per-block images copied into shared memory do the
    same operations in the same order as the sweeps from global memory:
    bitwise the same inner solve (and the oracle's within its bar)."""
    p = small_3d()
    y = np.random.default_rng(block + 1).standard_normal(p.n)
    out = []
    for stage in ("1", "0"):
        monkeypatch.setenv("MRCG_ILU_STAGE", stage)
        with m.Solver.from_problem(p, precision=prec, inner_prec=mcg, ilu_block=block) as g:
            out.append(g.inner_solve(y, inner_tol=1e-8 if prec == m.FP64 else 1e-4))
    (z1, st1, it1), (z0, st0, it0) = out
    assert st1 == st0 == m.OK and it1 == it0
    assert np.array_equal(z1, z0)
