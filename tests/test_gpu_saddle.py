"""GPU parity on saddle-point systems [K B^T; B 0] (27-point log-normal K,
random sparse B): irregular rows (27-28 entries, 64-entry constraint rows)
and eigenpairs from the setup eigensolver instead of closed forms."""
import numpy as np
import pytest

import oracle as O
from gen import saddle_96_b20x64, small_saddle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("mcg", [m.MCG_IDENTITY, m.MCG_JACOBI], ids=["identity", "jacobi"])
def test_small_saddle_fp64_matches_oracle(mcg):
    p = small_saddle()
    ref = O.minres_cg(O.System.from_problem(p), p.b, outer_tol=1e-12, inner_tol=1e-3,
                      mcg=O.MCG_JACOBI if mcg == m.MCG_JACOBI else O.MCG_IDENTITY)
    assert ref.status == O.OK
    with m.Solver.from_problem(p, inner_prec=mcg) as g:
        x, info = g.solve(p.b.copy(), outer_tol=1e-12)
    assert info.status == m.OK
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
    assert np.linalg.norm(x - p.xstar) <= 1e-8 * np.linalg.norm(p.xstar)


def test_small_saddle_mmr_product():
    p = small_saddle()
    u = np.random.default_rng(1).standard_normal(p.n)
    with m.Solver.from_problem(p) as g:
        out = g.apply_mmr(u)
    ref = O.System.from_problem(p).mmr_apply(u)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.fixture(scope="module")
def big():
    return saddle_96_b20x64()


def test_saddle_96_eigenpairs(big):
    p = big
    assert p.k == 20 and p.n == 96 ** 3 + 20
    assert np.all(p.lam < 0)
    assert p.meta["eig_residual_max"] < 1e-9


@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_saddle_96_solve(big, prec):
    """Full-size saddle system at the benchmark tolerance: FP64 true residual
    recomputed on the host and the error against x*."""
    p = big
    with m.Solver.from_problem(p, precision=prec, validate=False) as g:
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        _, info = g.solve(torch.from_numpy(p.b).to(DEV), x, outer_tol=1e-10, inner_tol=1e-3)
    x = x.cpu().numpy()
    assert info.status == m.OK, info
    rr = O.System.from_problem(p).true_relres(p.b, x)
    assert rr <= 1e-10
    assert np.linalg.norm(x - p.xstar) / np.linalg.norm(p.xstar) <= 1e-6


@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_saddle_96_solve_at_parity_tolerance(big, prec):
    """Full-size saddle system at outer_tol 1e-12: relative error against x* at
    most 1e-8 (x* solves the generated system up to kappa * eps) and FP64 true
    residual at most 1e-12."""
    p = big
    with m.Solver.from_problem(p, precision=prec, validate=False) as g:
        x = torch.zeros(p.n, dtype=torch.float64, device=DEV)
        _, info = g.solve(torch.from_numpy(p.b).to(DEV), x, outer_tol=1e-12, inner_tol=1e-3)
    x = x.cpu().numpy()
    assert info.status == m.OK, info
    rr = O.System.from_problem(p).true_relres(p.b, x)
    assert rr <= 1e-12
    assert np.linalg.norm(x - p.xstar) / np.linalg.norm(p.xstar) <= 1e-8
