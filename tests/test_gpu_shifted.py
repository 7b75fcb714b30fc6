"""GPU parity of the shifted-family / right-hand-side-block solver: every
column (shift j, right-hand side r) is checked against the FP64 CPU oracle
run on that column as a stand-alone system A_j = L - sigma_j I with
V_hat_j = V[:, :k_j], Lambda_hat_j = lambda_L[:k_j] - sigma_j."""
import numpy as np
import pytest

import oracle as O
from gen import shifted_lap3d_160, small_shifted

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_12417_gb300 as m  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def fam():
    return small_shifted()


@pytest.fixture(scope="module")
def oracle_x(fam):
    xs = []
    for c in range(fam.ncols):
        p = fam.column_problem(c)
        r = O.minres_cg(O.System.from_problem(p), p.b, outer_tol=1e-12, inner_tol=1e-3)
        assert r.status == O.OK
        xs.append(r.x)
    return np.stack(xs, axis=1)


@pytest.mark.parametrize("device", [True, False], ids=["device_ptrs", "host_ptrs"])
def test_shifted_fp64_matches_oracle(fam, oracle_x, device):
    with m.Shifted(fam) as sh:
        if device:
            X = torch.zeros(fam.n, fam.ncols, dtype=torch.float64, device=DEV)
            _, st, infos = sh.solve(torch.from_numpy(fam.B).to(DEV), X, outer_tol=1e-12)
            X = X.cpu().numpy()
        else:
            X, st, infos = sh.solve(fam.B.copy(), outer_tol=1e-12)
    assert st == m.OK
    for c in range(fam.ncols):
        p = fam.column_problem(c)
        x = X[:, c]
        assert infos[c].status == m.OK
        assert np.linalg.norm(x - oracle_x[:, c]) <= 1e-8 * np.linalg.norm(oracle_x[:, c])
        assert np.linalg.norm(x - p.xstar) <= 1e-8 * np.linalg.norm(p.xstar)
        assert O.System.from_problem(p).true_relres(p.b, x) <= 1e-11


def test_shifted_mixed_reaches_fp64_residual(fam):
    with m.Shifted(fam, precision=m.MIXED_FP32) as sh:
        X, st, infos = sh.solve(fam.B.copy(), outer_tol=1e-10)
    assert st == m.OK
    for c in range(fam.ncols):
        p = fam.column_problem(c)
        assert O.System.from_problem(p).true_relres(p.b, X[:, c]) <= 1e-10


def test_shifted_column_edge_cases(fam):
    B = fam.B.copy()
    B[:, 1] = 0.0
    X0 = np.zeros_like(B)
    X0[:, 2] = fam.xstar[:, 2]
    with m.Shifted(fam) as sh:
        X, st, infos = sh.solve(B, X0.copy(), outer_tol=1e-10)
        assert infos[1].status == m.OK and infos[1].outer_iters == 0 and not X[:, 1].any()
        assert infos[2].outer_iters == 0
        assert all(i.status == m.OK for i in infos)
        X, st, infos = sh.solve(fam.B.copy(), outer_tol=1e-12, max_iters=5)
        assert st == m.ERR_MAXITER and all(i.inner_iters_total <= 5 for i in infos)


def test_shifted_matches_batch_of_separate_systems(fam):
    """The shared-operator engine and the batched engine solve the same
    systems: the solutions agree to the FP64 tolerance."""
    ps = [fam.column_problem(c) for c in range(fam.ncols)]
    with m.Batch(ps) as bt:
        Xb, st, _ = bt.solve(np.concatenate([p.b for p in ps]), outer_tol=1e-12)
        xb = bt.split(Xb)
    with m.Shifted(fam) as sh:
        X, st2, _ = sh.solve(fam.B.copy(), outer_tol=1e-12)
    for c in range(fam.ncols):
        assert np.linalg.norm(X[:, c] - xb[c]) <= 1e-8 * np.linalg.norm(xb[c])


@pytest.mark.parametrize("prec", [m.FP64, m.MIXED_FP32], ids=["fp64", "mixed"])
def test_shifted_host_driven_loop_is_identical(fam, prec, monkeypatch):
    """MRCG_INNER_LOOP=host (the profiling mode) runs the graph's kernels in the
    same order from a host loop: bitwise the same solutions, counts and
    statuses, including a run stopped by the iteration budget."""
    out = []
    for mode in (None, "host"):
        if mode:
            monkeypatch.setenv("MRCG_INNER_LOOP", mode)
        with m.Shifted(fam, precision=prec) as sh:
            X, st, infos = sh.solve(fam.B.copy(), outer_tol=1e-10)
            X5, st5, inf5 = sh.solve(fam.B.copy(), outer_tol=1e-12, max_iters=5)
        out.append((X, st, [(i.outer_iters, i.inner_iters_total, i.status) for i in infos],
                    X5, st5, [(i.inner_iters_total, i.status) for i in inf5]))
    (a, b) = out
    assert a[1] == b[1] == m.OK and a[4] == b[4] == m.ERR_MAXITER
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
    assert a[2] == b[2] and a[5] == b[5]


@pytest.fixture(scope="module")
def fam160():
    return shifted_lap3d_160()


def test_shifted64_full_size_mixed(fam160):
    """The 160^3 family (16 shifts x 4 right-hand sides, k_j up to 32) at full
    size in mixed precision: every one of the 64 columns reaches an FP64 true
    residual (recomputed here on the host) of at most 1e-10, and its error
    against x* stays within kappa_j * 1e-10 * 3."""
    fam = fam160
    L = fam_scipy(fam)
    with m.Shifted(fam, precision=m.MIXED_FP32) as sh:
        X = torch.zeros((fam.n, fam.ncols), dtype=torch.float64, device=DEV)
        _, st, infos = sh.solve(torch.from_numpy(fam.B).to(DEV), X, outer_tol=1e-10, inner_tol=1e-3)
    X = X.cpu().numpy()
    assert st == m.OK
    for c in range(fam.ncols):
        j = c // fam.nrhs
        r = fam.B[:, c] - (L @ X[:, c] - fam.sigma[j] * X[:, c])
        rr = np.linalg.norm(r) / np.linalg.norm(fam.B[:, c])
        assert infos[c].status == m.OK and rr <= 1e-10, (c, rr)
        kappa = shift_condition(fam, j)
        err = np.linalg.norm(X[:, c] - fam.xstar[:, c]) / np.linalg.norm(fam.xstar[:, c])
        assert err <= kappa * 1e-10 * 3, (c, err)


def test_shifted64_full_size_fp64_one_shift(fam160):
    """FP64 engine on the four right-hand sides of shift 0 of the 160^3 family
    at outer_tol 1e-12: every column matches x* to a relative error of 1e-8."""
    sub = fam160.subfamily([0])
    with m.Shifted(sub, precision=m.FP64) as sh:
        X = torch.zeros((sub.n, sub.ncols), dtype=torch.float64, device=DEV)
        _, st, infos = sh.solve(torch.from_numpy(sub.B).to(DEV), X, outer_tol=1e-12, inner_tol=1e-3)
    X = X.cpu().numpy()
    assert st == m.OK
    for c in range(sub.ncols):
        err = np.linalg.norm(X[:, c] - sub.xstar[:, c]) / np.linalg.norm(sub.xstar[:, c])
        assert infos[c].status == m.OK and err <= 1e-8, (c, err)


def fam_scipy(fam):
    import scipy.sparse as sp
    return sp.csr_matrix((fam.val, fam.colind, fam.rowptr), shape=(fam.n, fam.n))


def shift_condition(fam, j):
    """kappa of L - sigma_j I from its analytic spectrum: largest |eigenvalue|
    over the smallest (the eigenvalues of L closest to sigma_j sit next to the
    k_j-th and (k_j+1)-th)."""
    from gen import laplacian_smallest_eigs
    kj = int(fam.k[j])
    ev = [v for v, _ in laplacian_smallest_eigs(fam.dims, kj + 1)]
    gap = min(abs(ev[kj - 1] - fam.sigma[j]), abs(ev[kj] - fam.sigma[j]))
    lam_max = 4.0 * len(fam.dims)
    return (lam_max - fam.sigma[j]) / gap


def test_shifted_autotuned_shape_solves_like_the_default(fam, monkeypatch):
    """The autotuner (forced with MRCG_AUTOTUNE=2 at this small size) picks a
    grid and the ELL-8 or CSR row path by timing calibration solves; the
    solution is the same to the FP64 tolerance as with the default shape."""
    out = {}
    for mode in ("0", "2"):
        monkeypatch.setenv("MRCG_AUTOTUNE", mode)
        with m.Shifted(fam) as sh:
            cfg = m.shifted_launch_config(sh.h)
            X, st, infos = sh.solve(fam.B.copy(), outer_tol=1e-12)
        assert st == m.OK
        out[mode] = (X, cfg)
    assert out["0"][1]["blocks_per_sm"] == 0 and out["2"][1]["blocks_per_sm"] >= 1
    assert out["2"][1]["ell8"] in (0, 1) and out["2"][1]["v_width"] in (8, 16, 24, 32)
    for c in range(fam.ncols):
        a, b = out["0"][0][:, c], out["2"][0][:, c]
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(a)
