"""GPU parity of the batched solver (many independent systems in one launch
sequence) against the FP64 CPU oracle, system by system."""
import numpy as np
import pytest

import oracle as O
from gen import batch64_lap2d, laplacian_csr, shifted_laplacian_problem, small_3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

DEV = torch.device("cuda:0")


class _P:
    """A bare SPD system (k = 0)."""

    def __init__(self, dims, seed):
        self.rowptr, self.colind, self.val = laplacian_csr(dims)
        self.n = len(self.rowptr) - 1
        self.k = 0
        self.V = None
        self.lam = None
        self.b = np.random.default_rng(seed).standard_normal(self.n)


def _small_batch():
    return [shifted_laplacian_problem("b0", (21, 21), 3, seed=1),
            small_3d(),
            _P((17, 13), 5),
            shifted_laplacian_problem("b3", (47, 31), 9, seed=2),
            shifted_laplacian_problem("b4", (5, 7), 1, seed=3),
            shifted_laplacian_problem("b5", (60, 60), 17, seed=4)]


def _oracle(p, tol, mcg=O.MCG_IDENTITY):
    s = O.System(p.rowptr, p.colind, p.val, p.V, p.lam) if p.k else O.System(p.rowptr, p.colind, p.val)
    return O.minres_cg(s, p.b, outer_tol=tol, inner_tol=1e-3, mcg=mcg)


@pytest.mark.parametrize("mcg", [m.MCG_IDENTITY, m.MCG_JACOBI], ids=["identity", "jacobi"])
@pytest.mark.parametrize("device", [True, False], ids=["device_ptrs", "host_ptrs"])
def test_batch_fp64_matches_oracle(mcg, device):
    ps = _small_batch()
    B = np.concatenate([p.b for p in ps])
    with m.Batch(ps, inner_prec=mcg) as bt:
        if device:
            X = torch.zeros(len(B), dtype=torch.float64, device=DEV)
            _, st, infos = bt.solve(torch.from_numpy(B).to(DEV), X, outer_tol=1e-12)
            X = X.cpu().numpy()
        else:
            X, st, infos = bt.solve(B.copy(), outer_tol=1e-12)
        xs = bt.split(X)
    assert st == m.OK
    for p, x, inf in zip(ps, xs, infos):
        ref = _oracle(p, 1e-12, O.MCG_JACOBI if mcg == m.MCG_JACOBI else O.MCG_IDENTITY)
        assert ref.status == O.OK and inf.status == m.OK
        assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        A = O.System(p.rowptr, p.colind, p.val)
        assert A.true_relres(p.b, x) <= 1e-11
        assert abs(inf.outer_iters - ref.outer_iters) <= 2
        assert len(inf.relres_history) == inf.outer_iters


@pytest.mark.parametrize("kmax", [5, 12, 20, 28], ids=["kb8", "kb16", "kb24", "kb32"])
@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_batch_each_v_width_bucket_matches_oracle(kmax, prec):
    """The batch kernels are compiled for V_hat widths of 8, 16, 24 and 32
    columns and the batch's largest k picks one: a batch per bucket (its
    largest system on a rectangle, whose low Laplacian eigenvalues are simple)
    against the oracle, system by system."""
    ps = [shifted_laplacian_problem("w0", (33, 29), 2, seed=11),
          shifted_laplacian_problem("w1", (61, 47), kmax, seed=12),
          _P((19, 23), 13)]
    assert ps[1].k == kmax
    B = np.concatenate([p.b for p in ps])
    tol = 1e-12 if prec == m.FP64 else 1e-10
    with m.Batch(ps, precision=prec) as bt:
        X, st, infos = bt.solve(B.copy(), outer_tol=tol)
        xs = bt.split(X)
    assert st == m.OK
    for p, x, inf in zip(ps, xs, infos):
        ref = _oracle(p, 1e-12)
        A = O.System(p.rowptr, p.colind, p.val)
        assert inf.status == m.OK and A.true_relres(p.b, x) <= tol
        assert np.linalg.norm(x - ref.x) <= (1e-8 if prec == m.FP64 else 1e-6) * np.linalg.norm(ref.x)


def test_batch_matches_single_system_solver():
    ps = _small_batch()[:4]
    B = np.concatenate([p.b for p in ps])
    with m.Batch(ps) as bt:
        X, st, infos = bt.solve(B.copy(), outer_tol=1e-11)
        xs = bt.split(X)
    for p, x, inf in zip(ps, xs, infos):
        with m.Solver(p.n, p.rowptr, p.colind, p.val, p.V if p.k else None, p.lam if p.k else None) as g:
            x1, i1 = g.solve(p.b.copy(), outer_tol=1e-11)
        assert np.linalg.norm(x - x1) <= 1e-8 * np.linalg.norm(x1)
        assert abs(inf.inner_iters_total - i1.inner_iters_total) <= 2 * max(1, i1.outer_iters)


@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_batch_host_driven_loop_is_identical(prec, monkeypatch):
    """MRCG_INNER_LOOP=host (the profiling mode) runs the graph's kernels in the
    same order from a host loop: bitwise the same solutions and counts."""
    ps = _small_batch()
    B = np.concatenate([p.b for p in ps])
    out = []
    for mode in (None, "host"):
        if mode:
            monkeypatch.setenv("MRCG_INNER_LOOP", mode)
        with m.Batch(ps, precision=prec) as bt:
            X, st, infos = bt.solve(B.copy(), outer_tol=1e-10)
        out.append((X, st, [(i.outer_iters, i.inner_iters_total) for i in infos]))
    assert out[0][1] == out[1][1] == m.OK
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][2] == out[1][2]


def test_batch_mixed_reaches_fp64_residual():
    ps = _small_batch()
    B = np.concatenate([p.b for p in ps])
    with m.Batch(ps, precision=m.MIXED_FP32) as bt:
        X, st, infos = bt.solve(B.copy(), outer_tol=1e-10)
        xs = bt.split(X)
    assert st == m.OK
    for p, x in zip(ps, xs):
        A = O.System(p.rowptr, p.colind, p.val)
        assert A.true_relres(p.b, x) <= 1e-10


def test_batch_per_system_edge_cases():
    ps = _small_batch()[:3]
    ps[1] = shifted_laplacian_problem("zero_rhs", (9, 9), 2, seed=0)
    ps[1].b = np.zeros(ps[1].n)
    B = np.concatenate([p.b for p in ps])
    with m.Batch(ps) as bt:
        X, st, infos = bt.solve(B.copy(), outer_tol=1e-10)
        xs = bt.split(X)
        assert infos[1].status == m.OK and infos[1].outer_iters == 0 and not xs[1].any()
        assert infos[0].status == m.OK and infos[2].status == m.OK
        # x0 = solution for one system: it needs no step while the others iterate
        X0 = X.copy()
        X0[bt.offsets[0]:bt.offsets[1]] = 0.0
        X2, st2, inf2 = bt.solve(B.copy(), X0, outer_tol=1e-10)
        assert inf2[2].outer_iters == 0 and inf2[0].outer_iters > 0
        # a tiny budget stops each system with MAXITER, independently
        X3, st3, inf3 = bt.solve(B.copy(), outer_tol=1e-12, max_iters=6)
        assert st3 == m.ERR_MAXITER
        assert inf3[0].status == m.ERR_MAXITER and inf3[0].inner_iters_total <= 6
        B4 = B.copy(); B4[3] = np.nan
        X4, st4, inf4 = bt.solve(B4, outer_tol=1e-10)
        assert inf4[0].status == m.ERR_NONFINITE and inf4[2].status == m.OK


def test_batch64_lap2d_mixed():
    """64 uneven 2D systems (sides 100..400, k_i up to 17): every system reaches
    FP64 true relative residual 1e-10 in one batched solve."""
    ps = batch64_lap2d()
    B = np.concatenate([p.b for p in ps])
    with m.Batch(ps, precision=m.MIXED_FP32, validate=False) as bt:
        Bd = torch.from_numpy(B).to(DEV)
        X = torch.zeros_like(Bd)
        _, st, infos = bt.solve(Bd, X, outer_tol=1e-10)
        xs = bt.split(X.cpu().numpy())
    assert st == m.OK, [i.status for i in infos]
    for p, x in zip(ps, xs):
        A = O.System(p.rowptr, p.colind, p.val)
        assert A.true_relres(p.b, x) <= 1e-10


def test_batch_autotuned_shape_solves_like_the_default(monkeypatch):
    """The batch autotuner (forced with MRCG_AUTOTUNE=2) picks the chunk height
    and the grids by timing calibration solves; the solutions match the
    default shape's to the FP64 tolerance."""
    from gen import shifted_laplacian_problem
    ps = [shifted_laplacian_problem(f"bt{i}", (37 + 9 * i, 31 + 4 * i), 2 + i, seed=60 + i) for i in range(5)]
    B = np.concatenate([p.b for p in ps])
    out = {}
    for mode in ("0", "2"):
        monkeypatch.setenv("MRCG_AUTOTUNE", mode)
        with m.Batch(ps) as bt:
            cfg = m.batch_launch_config(bt.h)
            X, st, infos = bt.solve(B.copy(), outer_tol=1e-12)
        assert st == m.OK
        out[mode] = (X, cfg)
    assert out["0"][1]["chunk_rows"] == 4096 and out["2"][1]["chunk_rows"] in (1024, 2048, 4096, 8192)
    assert np.linalg.norm(out["0"][0] - out["2"][0]) <= 1e-8 * np.linalg.norm(out["0"][0])
